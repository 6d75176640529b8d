"""Gauss-Seidel sweep of Step B (cpra_config.sweep = 1) on the GPU against the
oracle's sweep_episode (reading R22).

ER iterations (continuous in the sign test) on the true-projection supports
over two episodes, every engine: each angle's iterate within 1e-4 relative
L2 and every error within 1e-4; Step A (3 HIO iterations on angle 0) before
the sweeps; one RAAR episode of 3 iterations.  The sweep must differ from
the Jacobi episodes it replaces, and calls must cover whole episodes.  A
batch runs the sweeps of many guesses together (one launch per angle over
all of them) and must give every member's standalone result bit for bit.
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


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def _both(cp, d, iters, **kw):
    cfg = cp.make_config(64, 8, **kw)
    plan = cp.Plan(cfg)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(d["S_true"])
    e_gpu = plan.iterate(iters, errors=True)
    g_gpu = plan.result(cp.RESULT_STATE)
    plan.close()
    oc = O.OracleConfig(N=64, Np=8, n_ei=cfg.n_ei, hio_iters=cfg.hio_iters, er_iters=cfg.er_iters,
                        seed=cfg.seed, n_pre=cfg.n_pre, sweep=bool(cfg.sweep),
                        update=O.RAAR if cfg.update == 1 else O.HIO,
                        beta=float(np.float32(cfg.beta)))
    run = O.OracleRun.start(oc, d["I"], d["S_true"]).run(iters)
    return g_gpu, e_gpu, run.g, np.array(run.errors)


@pytest.mark.parametrize("engine", ["two_pass", "warp", "fused"])
def test_sweep_er_two_episodes(cp, case, engine):
    g, e, g_ref, e_ref = _both(cp, case, 10, seed=3, hio_iters=0, er_iters=10, n_ei=5,
                               engine=ENGINES[engine], sweep=1)
    r = _rel(g, g_ref).max()
    er = (np.abs(e - e_ref) / e_ref).max()
    print(f"{engine}: sweep ER 2 x 5: iterate {r:.2e}, errors {er:.2e}")
    assert r < TOL and er < TOL


def test_sweep_after_step_a_and_raar(cp, case):
    g, e, g_ref, e_ref = _both(cp, case, 10, seed=4, hio_iters=0, er_iters=10, n_ei=5, n_pre=3,
                               sweep=1)
    assert _rel(g, g_ref).max() < TOL and (np.abs(e - e_ref) / e_ref).max() < TOL
    g, e, g_ref, e_ref = _both(cp, case, 3, seed=5, hio_iters=3, er_iters=0, n_ei=3,
                               update=cp.UPDATE_RAAR, sweep=1)
    r = _rel(g, g_ref).max()
    print(f"sweep RAAR 1 x 3: iterate {r:.2e}")
    assert r < TOL and (np.abs(e - e_ref) / e_ref).max() < TOL


def test_sweep_with_shrinkwrap_at_episode_ends(cp, case):
    """Shrink-wrap every episode (sigma 2, tau 0.1) after ER sweeps: iterates
    and supports equal to the oracle's."""
    kw = dict(seed=6, hio_iters=0, er_iters=10, n_ei=5, shrinkwrap_every=5, sweep=1)
    cfg = cp.make_config(64, 8, **kw)
    plan = cp.Plan(cfg)
    plan.load_intensities(case["I"], 0, case["thetas"])
    plan.load_support(case["S_true"])
    plan.iterate(10)
    g = plan.result(cp.RESULT_STATE)
    S = plan.result(cp.RESULT_SUPPORT).astype(bool)
    plan.close()
    oc = O.OracleConfig(N=64, Np=8, n_ei=5, hio_iters=0, er_iters=10, seed=6, sweep=True,
                        shrinkwrap_every=5, sw_sigma=float(np.float32(cfg.sw_sigma)),
                        sw_tau=float(np.float32(cfg.sw_tau)))
    run = O.OracleRun.start(oc, case["I"], case["S_true"]).run(10)
    assert np.array_equal(S, run.S)
    r = _rel(g, run.g).max()
    print(f"sweep + shrink-wrap: iterate {r:.2e}")
    assert r < TOL


def test_sweep_differs_from_jacobi_and_runs_whole_episodes(cp, case):
    kw = dict(seed=3, hio_iters=0, er_iters=10, n_ei=5)
    g_s, _, _, _ = _both(cp, case, 5, sweep=1, **kw)
    g_j, _, _, _ = _both(cp, case, 5, sweep=0, **kw)
    assert _rel(g_s, g_j).max() > 1e-3
    plan = cp.Plan(cp.make_config(64, 8, sweep=1, **kw))
    plan.load_intensities(case["I"], 0, case["thetas"])
    with pytest.raises(cp.CpraError) as ei:
        plan.iterate(3)
    assert ei.value.status == cp.ERR_INVALID_ARG
    with pytest.raises(cp.CpraError) as ei:
        plan.set_present(np.arange(8) < 4)
    assert ei.value.status == cp.ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("engine", ["two_pass", "fused"])
def test_batched_sweeps_equal_standalone(cp, case, engine):
    """Four guesses (different seeds, Step A on two of them, one with 6
    angles instead of 8, shrink-wrap every episode on one) as one batch:
    each ends bit for bit where it ends alone."""
    import torch
    d = case

    def plans():
        out = []
        for i in range(4):
            Np = 6 if i == 3 else 8
            kw = dict(seed=20 + i, hio_iters=6, er_iters=4, n_ei=5, sweep=1,
                      engine=ENGINES[engine], update=cp.UPDATE_RAAR if i % 2 else cp.UPDATE_HIO,
                      n_pre=3 if i < 2 else 0, shrinkwrap_every=5 if i == 2 else 0)
            p = cp.Plan(cp.make_config(64, Np, **kw), stream=torch.cuda.current_stream().cuda_stream)
            p.load_intensities(d["I"][:Np], 0, d["thetas"][:Np])
            p.load_support(d["S_true"][:Np])
            out.append(p)
        return out

    alone = plans()
    for p in alone:
        p.iterate(10)
    together = plans()
    b = cp.Batch(together, use_graph=True)
    b.iterate(5)
    b.iterate(5)
    for a, t in zip(alone, together):
        assert np.array_equal(a.result(cp.RESULT_STATE), t.result(cp.RESULT_STATE))
        assert np.array_equal(a.result(cp.RESULT_SUPPORT), t.result(cp.RESULT_SUPPORT))
        np.testing.assert_allclose(t.result(cp.RESULT_ERRORS), a.result(cp.RESULT_ERRORS), rtol=1e-12)
    with pytest.raises(cp.CpraError) as ei:
        b.iterate(3)
    assert ei.value.status == cp.ERR_INVALID_ARG
    b.close()
    for p in alone + together:
        p.close()
