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
    eng2, _ = cp.cpra_autotune(192, cp.FP32, path)  # only TWO_PASS exists for 192
    assert eng2 == cp.ENGINE_TWO_PASS
    assert len(json.load(open(path))["entries"]) == 2
