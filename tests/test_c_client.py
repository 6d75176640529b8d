"""The library from plain C (tests/c_abi_client.c): the header compiles as
C11 and every call the client makes links against libcpra.so (CPU); on a
GPU the client runs one small reconstruction through the C ABI alone."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_2402_05283_gb300 import build as b
    lib = b.build()
    pkg = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_client")
    cmd = [cc, "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-L", pkg, "-lcpra", f"-Wl,-rpath,{pkg}",
           "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_client_runs_a_reconstruction(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    words = r.stdout.split()
    assert words[0] == "ok"
    e_first, e_last = float(words[1]), float(words[2])
    assert 0.0 <= e_last < e_first  # 20 iterations lower the mean Fourier error
    print(r.stdout.strip())
