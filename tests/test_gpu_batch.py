"""Batching (many reconstructions per launch, CUDA graph) and the autotuner.

A batch must compute, for every plan, exactly what the plan computes alone:
the kernels are the same and each (plan, angle) tile does the same
arithmetic, so states and error histories are compared bit for bit.
"""
import json

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


MIX = [(64, 12, 3, {}), (128, 6, 4, {"n_ei": 5}), (96, 5, 5, {}), (64, 9, 6, {"hio_iters": 7}),
       (256, 3, 7, {"alpha": (0.1, 0.2, 0.4, 0.2, 0.1)}), (48, 4, 8, {"engine": 1})]


def _plans(cp, mix):
    plans = []
    for N, Np, seed, kw in mix:
        d = synth.make_case("tiny", N=N, Np=Np, request=seed)
        p = cp.Plan(cp.make_config(N, Np, seed=seed, **kw))
        p.load_intensities(d["I"], 0, d["thetas"])
        p.load_support(d["support"])
        plans.append(p)
    return plans


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(cp, use_graph):
    alone = _plans(cp, MIX)
    for p in alone:
        p.iterate(13)
    mixed = _plans(cp, MIX)
    b = cp.Batch(mixed, use_graph=use_graph)
    b.iterate(6)
    b.iterate(7)
    for pa, pm in zip(alone, mixed):
        assert pm.iteration == 13
        assert np.array_equal(pa.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
        # error sums are FP64 atomics in launch order: equal to rounding
        np.testing.assert_allclose(pa.result(cp.RESULT_ERRORS), pm.result(cp.RESULT_ERRORS),
                                   rtol=1e-12)
    b.close()


def test_batch_graph_replay(cp):
    """The same call pattern replays the captured graph; results stay exact."""
    alone = _plans(cp, MIX[:3])
    for p in alone:
        p.iterate(40)
    mixed = _plans(cp, MIX[:3])
    b = cp.Batch(mixed, use_graph=True)
    for _ in range(4):
        b.iterate(10)
    for pa, pm in zip(alone, mixed):
        assert np.array_equal(pa.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
    b.close()


def test_batch_rejects_shrinkwrap_and_unloaded(cp):
    p = cp.Plan(cp.make_config(32, 2, shrinkwrap_every=5))
    with pytest.raises(cp.CpraError) as e:
        cp.Batch([p])
    assert e.value.status == cp.ERR_UNSUPPORTED
    q = cp.Plan(cp.make_config(32, 2))
    b = cp.Batch([q])
    with pytest.raises(cp.CpraError) as e:
        b.iterate(1)
    assert e.value.status == cp.ERR_NOT_READY


def test_autotune_cache(cp, tmp_path):
    path = str(tmp_path / "tune.json")
    eng, ms = cp.cpra_autotune(128, cp.FP32, path)
    assert eng in (cp.ENGINE_TWO_PASS, cp.ENGINE_WARP, cp.ENGINE_FUSED) and ms > 0
    doc = json.load(open(path))
    assert len(doc["entries"]) == 1 and doc["entries"][0]["engine"] == eng
    assert cp.cpra_autotune(128, cp.FP32, path) == (eng, pytest.approx(ms))
    eng2, _ = cp.cpra_autotune(192, cp.FP32, path)  # TWO_PASS and WARP exist for 192
    assert eng2 in (cp.ENGINE_TWO_PASS, cp.ENGINE_WARP)
    assert len(json.load(open(path))["entries"]) == 2


# ---------------------------------------------------------------- persistent work queue
# uneven sizes on the warp engine (the sizes of the batching workload, and
# small angle counts so the oracle-free comparison stays quick)
UNEVEN = [(128, 6, 11, {}), (192, 5, 12, {"hio_iters": 9}), (256, 4, 13, {"n_ei": 4}),
          (384, 3, 14, {"alpha": (0.1, 0.2, 0.4, 0.2, 0.1)}), (128, 3, 15, {"update": 1})]


def _warp_plans(cp, mix):
    return _plans(cp, [(N, Np, seed, {**kw, "engine": cp.ENGINE_WARP}) for N, Np, seed, kw in mix])


@pytest.mark.parametrize("use_graph,chunk", [(False, 0), (True, 0), (True, 2), (False, 5)])
def test_persistent_batch_uneven_n_equals_alone(cp, use_graph, chunk):
    """One persistent work-queue launch per size group and segment (split at
    the coupling steps), the groups forked onto their own streams: every
    member's iterates equal the plan run alone bit for bit, over calls that
    cross episode boundaries and the HIO -> ER switch.  chunk_tiles 2 and 5
    run the queue in chunks (with a shorter last chunk where the tile count
    is not a multiple); 0 takes the chunk from the L2 size (here every tile)."""
    alone = _warp_plans(cp, UNEVEN)
    for p in alone:
        p.iterate(23)
    mixed = _warp_plans(cp, UNEVEN)
    b = cp.Batch(mixed, use_graph=use_graph)
    b.set_persistent(1, chunk_tiles=chunk)
    b.iterate(11)  # the first call also runs each member's seeded start
    expect = b.launches(12)
    n0 = cp.cpra_launch_count()
    b.iterate(12)
    assert cp.cpra_launch_count() - n0 == expect
    for pa, pm in zip(alone, mixed):
        assert pm.iteration == 23
        assert np.array_equal(pa.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
        np.testing.assert_allclose(pa.result(cp.RESULT_ERRORS), pm.result(cp.RESULT_ERRORS),
                                   rtol=1e-12)
    b.close()


def test_persistent_512_chunks_equal_alone(cp):
    """The bench size's angle loop in the persistent queue in L2 chunks: two
    plans of N = 512 with 12 angles each, 24 tiles in chunks of 5 (the last
    of 4; one chunk crosses from the first member to the second), 14
    iterations across a coupling step, states equal to the plans alone bit
    for bit."""
    mix = [(512, 12, 31, {}), (512, 12, 32, {"hio_iters": 6})]
    alone = _warp_plans(cp, mix)
    for p in alone:
        p.iterate(14)
    mixed = _warp_plans(cp, mix)
    b = cp.Batch(mixed, use_graph=True)
    b.set_persistent(1, chunk_tiles=5)
    b.iterate(14)
    for pa, pm in zip(alone, mixed):
        assert np.array_equal(pa.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
        np.testing.assert_allclose(pa.result(cp.RESULT_ERRORS), pm.result(cp.RESULT_ERRORS),
                                   rtol=1e-12)
    b.close()


def test_persistent_wait_runs_out_and_recovers(cp):
    """The bounded device wait: in mode 2 the first task of every launch
    waits on a count that no task increments, so its wait runs out after the
    budget (1 ms), the launch ends and every member reports TIMEOUT; a reset
    clears it and the normal mode then equals the plans alone."""
    plans = _warp_plans(cp, UNEVEN[:2])
    b = cp.Batch(plans, use_graph=False)
    b.set_persistent(2, wait_budget_s=1e-3)
    b.iterate(3)
    for p in plans:
        with pytest.raises(cp.CpraError) as e:
            p.sync()
        assert e.value.status == cp.ERR_TIMEOUT
        assert "wait" in cp.cpra_last_error(p.h)
        with pytest.raises(cp.CpraError):  # sticky until reset
            p.iterate(1)
    for p in plans:
        p.reset()
    b.set_persistent(1)
    b.iterate(4)
    ref = _warp_plans(cp, UNEVEN[:2])
    for pr, pm in zip(ref, plans):
        pr.iterate(4)
        assert np.array_equal(pr.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
    b.close()


def test_persistent_needs_the_warp_engine(cp):
    plans = _plans(cp, [(128, 3, 1, {"engine": cp.ENGINE_FUSED}), (192, 2, 2, {})])
    b = cp.Batch(plans, use_graph=False)
    with pytest.raises(cp.CpraError) as e:
        b.set_persistent(1)
    assert e.value.status == cp.ERR_UNSUPPORTED
    with pytest.raises(cp.CpraError) as e:
        b.set_persistent(3)
    assert e.value.status == cp.ERR_INVALID_ARG
    with pytest.raises(cp.CpraError) as e:
        b.set_persistent(0, chunk_tiles=-1)
    assert e.value.status == cp.ERR_INVALID_ARG
    b.close()
