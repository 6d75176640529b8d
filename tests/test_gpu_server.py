"""The serving loop: admission by device memory, streamed patterns, continuous
batching, and results identical to standalone reconstructions."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REQS = [(64, 16, 1), (128, 8, 2), (96, 6, 3), (64, 12, 4)]


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


def _cfg(cp, N, Np, seed):
    return cp.make_config(N, Np, seed=seed, hio_iters=25, er_iters=5, n_ei=10)


def test_served_requests_equal_standalone(cp):
    data = [synth.make_case("tiny", N=N, Np=Np, request=seed) for N, Np, seed in REQS]
    srv = cp.Server(hbm_reserve_bytes=1 << 30, iters_per_round=10)
    ids = [srv.submit(_cfg(cp, N, Np, seed)) for N, Np, seed in REQS]
    # stream the patterns of all requests interleaved, a few angles at a time
    pos = [0] * len(REQS)
    while any(pos[i] < REQS[i][1] for i in range(len(REQS))):
        for i, (N, Np, _) in enumerate(REQS):
            if pos[i] < Np:
                k = min(3, Np - pos[i])
                srv.push(ids[i], data[i]["I"][pos[i]:pos[i] + k], pos[i], data[i]["thetas"][pos[i]:pos[i] + k])
                pos[i] += k
        time.sleep(0.002)
    for rid in ids:
        srv.wait(rid, 120.0)
    events = srv.poll(64)
    kinds = {(e["id"], e["kind"]) for e in events}
    for rid in ids:
        assert (rid, cp.EVENT_FIRST_ESTIMATE) in kinds and (rid, cp.EVENT_FINAL) in kinds
        info = srv.info(rid)
        assert info["iterations_done"] == 30 and info["t_final"] >= info["t_first_estimate"] >= 0
    st = srv.stats()
    assert st["completed"] == len(REQS) and st["angle_iterations"] == 30 * sum(r[1] for r in REQS)
    for (N, Np, seed), d, rid in zip(REQS, data, ids):
        p = cp.Plan(_cfg(cp, N, Np, seed))
        p.load_intensities(d["I"], 0, d["thetas"])
        p.iterate(30)
        vol = np.empty((N, N, N), np.complex64)
        p.assemble_3d(vol)
        assert np.array_equal(srv.result(rid, cp.RESULT_STATE), p.result(cp.RESULT_STATE))
        assert np.array_equal(srv.result(rid, cp.RESULT_VOLUME), vol)
        p.close()
        srv.release(rid)
    srv.stop()


def test_requests_overlap_on_device(cp):
    """A request that completes its patterns while another runs joins its rounds."""
    srv = cp.Server(hbm_reserve_bytes=1 << 30, iters_per_round=5)
    a = srv.submit(cp.make_config(64, 8, seed=5, hio_iters=2000, er_iters=0))
    b = srv.submit(cp.make_config(128, 8, seed=6, hio_iters=60, er_iters=0))
    da = synth.make_case("tiny", N=64, Np=8, request=5)
    db = synth.make_case("tiny", N=128, Np=8, request=6)
    srv.push(a, da["I"], 0, da["thetas"])
    time.sleep(0.02)
    assert srv.info(a)["state"] in (1, 2)  # a is resident or running when b arrives
    srv.push(b, db["I"], 0, db["thetas"])
    srv.wait(a, 120.0)
    srv.wait(b, 120.0)
    assert srv.stats()["max_batch"] >= 2
    srv.stop()


def test_admission_waits_for_memory(cp):
    srv = cp.Server(hbm_reserve_bytes=1 << 62)  # never enough free memory
    rid = srv.submit(cp.make_config(64, 4))
    d = synth.make_case("tiny", N=64, Np=4)
    srv.push(rid, d["I"], 0, d["thetas"])
    time.sleep(0.3)
    assert srv.info(rid)["state"] == 0  # still queued
    with pytest.raises(cp.CpraError) as e:
        srv.result(rid, cp.RESULT_STATE)
    assert e.value.status == cp.ERR_NOT_READY
    with pytest.raises(cp.CpraError) as e:
        srv.wait(rid, 0.1)
    assert e.value.status == cp.ERR_TIMEOUT
    srv.stop()


def test_early_start_iterates_while_streaming(cp):
    """early_start: a request iterates its arrived angles while the rest
    stream in, holds the tail of its schedule (by default half of it, in
    whole episodes: 40 of 70 iterations here) until every angle is there, and
    reaches the quality of a standalone reconstruction within a factor 2."""
    N, Np, seed = 64, 16, 9
    d = synth.make_case("tiny", N=N, Np=Np, request=seed)
    cfg = cp.make_config(N, Np, seed=seed, hio_iters=50, er_iters=20, n_ei=10)
    srv = cp.Server(hbm_reserve_bytes=1 << 30, iters_per_round=5, early_start=True)
    rid = srv.submit(cfg)
    done_while_streaming = 0
    for f in range(0, Np, 4):
        if f + 4 >= Np:  # before the last patterns arrive
            done_while_streaming = srv.info(rid)["iterations_done"]
        srv.push(rid, d["I"][f:f + 4], f, d["thetas"][f:f + 4])
        time.sleep(0.05)
    srv.wait(rid, 120.0)
    info = srv.info(rid)
    assert info["iterations_done"] == 70 and info["t_final"] >= info["t_first_estimate"] >= 0
    assert 0 < done_while_streaming <= 30  # started early, held the tail
    po = srv.result(rid, cp.RESULT_PO)
    e_srv = srv.result(rid, cp.RESULT_ERRORS)[-1]
    srv.release(rid)
    srv.stop()
    p = cp.Plan(cfg)
    p.load_intensities(d["I"], 0, d["thetas"])
    p.iterate(70)
    e_alone = p.result(cp.RESULT_ERRORS)[-1]
    p.close()
    assert np.all(np.isfinite(po))
    print(f"early start: {done_while_streaming} iterations before the last patterns, "
          f"final error {e_srv.mean():.4f} vs {e_alone.mean():.4f} alone")
    assert e_srv.mean() <= 2.0 * e_alone.mean(), (e_srv.mean(), e_alone.mean())
