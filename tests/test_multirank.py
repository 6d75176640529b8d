"""The N > 1 host path of bench.py on CPU with gloo (world size 2): each rank
runs an independent replica; the job's rate is the units of all ranks over
the slowest rank's time; only rank 0 reports, and the reference arm does no
work on other ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms_local = 100.0 * (rank + 1)  # rank 1 is the slower one
    value, ms = bench.job_rate(1000, ms_local, dist)
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == 200.0  # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1000 / 0.2)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0

    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(1))
    bench.run_reference(A())
    assert not called and capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 prints one JSON line with every key of the bench line, its e2e
    moving no bytes and its cpu_baseline describing the same run."""
    import json
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        gpus, steps, warmup = 1, 3, 1

    rates = iter([1.0, 40.0, 60.0, 50.0])
    monkeypatch.setattr(bench, "sample_inputs", lambda *a: (np.zeros((8, 4, 4)), None))

    class _Pool:
        def close(self):
            pass

        def join(self):
            pass

    monkeypatch.setattr(bench, "oracle_pool", lambda n: _Pool())
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: {
        "value": next(rates), "unit": "angle-iterations/s", "cores": 4, "kind": "oracle",
        "sample": "stub"})
    bench.run_reference(A())
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] == 50.0  # median of the timed steps
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
