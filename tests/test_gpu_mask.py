"""Missing data (cpra_load_mask, reading R23) on the GPU against the oracle.

A centred beamstop removes the lowest frequencies of the cfg 1 patterns; ER
iterations (continuous, so trajectories compare) on the true-projection
supports must track the oracle within 1e-4 per iterate on every engine, with
one mask for all angles and with a different mask per angle; an all-measured
mask must give exactly the unmasked iterates.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
ENGINES = {"two_pass": 1, "warp": 3, "fused": 2}


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def case():
    d = synth.make_case("cfg1", N=64, Np=8)
    d["S_true"] = (d["proj"].numpy() > 1e-9).astype(np.uint8)
    return d


def _beamstop(N, r, cy=0, cx=0):
    y, x = np.meshgrid(np.arange(N) - N // 2 - cy, np.arange(N) - N // 2 - cx, indexing="ij")
    return ((x * x + y * y) > r * r).astype(np.uint8)


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def _gpu(cp, d, mask, iters, **kw):
    plan = cp.Plan(cp.make_config(64, 8, **kw))
    if mask is not None:
        plan.load_mask(mask)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(d["S_true"])
    e = plan.iterate(iters, errors=True)
    g = plan.result(cp.RESULT_STATE)
    plan.close()
    return g, e


@pytest.mark.parametrize("engine", ["two_pass", "warp", "fused"])
def test_beamstop_er_matches_oracle(cp, case, engine):
    mask = _beamstop(64, 3)
    kw = dict(seed=2, hio_iters=0, er_iters=20, n_ei=10, engine=ENGINES[engine])
    g, e = _gpu(cp, case, mask, 20, **kw)
    oc = O.OracleConfig(N=64, Np=8, n_ei=10, hio_iters=0, er_iters=20, seed=2)
    run = O.OracleRun.start(oc, case["I"], case["S_true"], mask=mask).run(20)
    r = _rel(g, run.g).max()
    er = (np.abs(e - np.array(run.errors)) / np.array(run.errors)).max()
    print(f"{engine}: beamstop ER 20: iterate {r:.2e}, errors {er:.2e}")
    assert r < TOL and er < TOL


def test_per_angle_masks_and_raar(cp, case):
    masks = np.stack([_beamstop(64, 2 + n % 3, n % 2, -(n % 2)) for n in range(8)])
    g, e = _gpu(cp, case, masks, 6, seed=3, hio_iters=6, er_iters=0, n_ei=10,
                update=cp.UPDATE_RAAR)
    oc = O.OracleConfig(N=64, Np=8, n_ei=10, hio_iters=6, er_iters=0, seed=3, update=O.RAAR)
    run = O.OracleRun.start(oc, case["I"], case["S_true"], mask=masks).run(6)
    r = _rel(g, run.g).max()
    print(f"per-angle masks, RAAR 6: iterate {r:.2e}")
    assert r < TOL and (np.abs(e - np.array(run.errors)) / np.array(run.errors)).max() < TOL


def test_all_measured_mask_is_no_mask(cp, case):
    kw = dict(seed=4, hio_iters=5, er_iters=5, n_ei=4)
    g0, e0 = _gpu(cp, case, None, 10, **kw)
    g1, e1 = _gpu(cp, case, np.ones((64, 64), np.uint8), 10, **kw)
    assert np.array_equal(g0, g1)
    # the FP64 error constants are block sums added in launch order
    np.testing.assert_allclose(e1, e0, rtol=1e-12, atol=0)
