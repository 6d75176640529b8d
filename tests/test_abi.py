"""Host-side checks of the C-ABI library (no GPU compute).

The library must load, export every function include/cpra.h declares, and
validate configurations on the host.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cp():
    import paper_2402_05283_gb300 as pkg
    from paper_2402_05283_gb300 import build as b
    b.build()
    pkg.lib()
    return pkg


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cpra_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(cp):
    names = _declared()
    assert {"cpra_plan", "cpra_load_intensities", "cpra_iterate", "cpra_assemble_3d",
            "cpra_result"} <= names
    L = C.CDLL(cp.binding.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared but not exported"


def test_default_config_values(cp):
    cfg = cp.cpra_default_config(64, 32)
    assert (cfg.N, cfg.Np, cfg.n_ei, cfg.n_taps) == (64, 32, 10, 3)
    assert list(cfg.alpha[:3]) == [0.2, 0.6, 0.2]
    assert abs(cfg.beta - 0.9) < 1e-7 and abs(cfg.sw_tau - 0.1) < 1e-7
    assert cfg.hio_iters == 200 and cfg.er_iters == 20 and cfg.com_align == 1
    assert cfg.update == cp.UPDATE_HIO and cfg.seed == 0


def test_config_layout_matches_c(cp):
    """The ctypes mirror of cpra_config has the C layout: a field past the
    padding before seed round-trips through the library's validation."""
    cfg = cp.make_config(64, 8, update=cp.UPDATE_RAAR, seed=(1 << 63) + 5)
    cp.cpra_plan_bytes(cfg)  # RAAR is valid
    cfg.update = 5
    with pytest.raises(cp.CpraError, match="update"):
        cp.cpra_plan_bytes(cfg)


def test_plan_bytes_scales(cp):
    a64, b64 = cp.cpra_plan_bytes(cp.make_config(64, 32))
    a512, b512 = cp.cpra_plan_bytes(cp.make_config(512, 360))
    assert a512 > 100 * a64 and b512 > b64
    # iteration state of the metric workload: a few GB at most
    assert a512 < 4 << 30


@pytest.mark.parametrize("kw,status", [
    (dict(N=100), 6), (dict(N=8), 6), (dict(N=2048), 6), (dict(N=80), 6),
    (dict(Np=0), 1), (dict(n_ei=0), 1),
    (dict(alpha=(0.2, 0.6, 0.3)), 1), (dict(alpha=(0.5, 0.5)), 1),
    (dict(alpha=(1.0 / 17,) * 17), 1),
    (dict(wrap_mode=7), 1), (dict(blend_target=3), 1), (dict(hio_iters=-1), 1),
    (dict(shrinkwrap_every=5, sw_sigma=0.0), 1), (dict(precision=9), 1),
    (dict(update=2), 1), (dict(update=-1), 1), (dict(sweep=2), 1),
    (dict(sweep=1, shrinkwrap_every=15), 6),
])
def test_config_validation(cp, kw, status):
    N = kw.pop("N", 64)
    Np = kw.pop("Np", 8)
    alpha = kw.pop("alpha", None)
    cfg = cp.cpra_default_config(max(N, 16) if N > 0 else 64, max(Np, 1))
    cfg.N, cfg.Np = N, Np
    if alpha is not None:
        if len(alpha) > cp.MAX_TAPS:
            cfg.n_taps = len(alpha)
        else:
            cfg.n_taps = len(alpha)
            for i, a in enumerate(alpha):
                cfg.alpha[i] = a
    for k, v in kw.items():
        setattr(cfg, k, v)
    with pytest.raises(cp.CpraError) as ei:
        cp.cpra_plan_bytes(cfg)
    assert ei.value.status == status
    assert cp.cpra_last_error(None)


def test_supported_sizes_validate(cp):
    for N in (16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024):
        cp.cpra_plan_bytes(cp.make_config(N, 4))
