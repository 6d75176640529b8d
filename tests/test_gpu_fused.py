"""The cluster-resident fused engine (one launch per window of iterations,
spectra held in distributed shared memory).

Up to N = 256 it runs the same FP32 line transforms, with the same
task-to-lane maps, as the two-pass warp engine, so on the same schedule the
two must produce the same iterates bit for bit; the per-iteration Fourier
errors differ only in the FP64 summation order (1e-12 relative).  At
N = 512 it uses the one-line-per-warp FFT (16-point DFTs and a lane-pair
radix-2 step), so the two engines agree to FP32 rounding instead.  Oracle parity of the fused
engine itself: the 1e-4 bar over windows of many iterations (ER, continuous
in the sign test) at every supported N.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
FUSED_N = [64, 128, 256, 512]


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


def _run(cp, cfg, d, S, chunks):
    plan = cp.Plan(cfg)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(S)
    errs = np.concatenate([plan.iterate(k, errors=True) for k in chunks])
    g = plan.result(cp.RESULT_STATE)
    sup = plan.result(cp.RESULT_SUPPORT)
    plan.close()
    return g, errs, sup


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


@pytest.mark.parametrize("N,update", [(64, 0), (128, 0), (256, 0), (64, 1), (256, 1)])
def test_fused_equals_warp_engine(cp, N, update):
    """HIO (update 0) or RAAR (update 1) with coupling every 4, the switch to
    ER inside a window, and a mid-episode split of the iterate calls (the
    fused engine re-primes)."""
    Np = 3
    d = synth.make_case("tiny", N=N, Np=Np)
    kw = dict(n_ei=4, seed=11, hio_iters=6, er_iters=5, update=update)
    gw, ew, _ = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_WARP, **kw), d, d["support"], [11])
    for chunks in ([11], [3, 5, 3]):
        gf, ef, _ = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_FUSED, **kw), d, d["support"], chunks)
        assert np.array_equal(gf, gw), f"chunks {chunks}: max diff {np.abs(gf - gw).max():.3e}"
        np.testing.assert_allclose(ef, ew, rtol=1e-12, atol=0)


def test_fused_512_tracks_warp_engine(cp):
    """N = 512: two HIO iterations then ER with coupling every 4, windows of
    11 and of 3 + 5 + 3; both engines are FP32, so they agree to rounding."""
    N, Np = 512, 3
    d = synth.make_case("tiny", N=N, Np=Np)
    kw = dict(n_ei=4, seed=11, hio_iters=2, er_iters=9)
    gw, ew, _ = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_WARP, **kw), d, d["support"], [11])
    for chunks in ([11], [3, 5, 3]):
        gf, ef, _ = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_FUSED, **kw), d, d["support"], chunks)
        r = _rel(gf, gw).max()
        er = np.max(np.abs(ef - ew) / ew)
        print(f"chunks {chunks}: iterate rel-L2 {r:.2e}, errors {er:.2e}")
        assert r < TOL and er < TOL


def test_fused_equals_warp_engine_variants(cp):
    """Five taps, MIRROR wrap, OBJECT blend, Step A, shrink-wrap every 3."""
    N, Np = 128, 5
    d = synth.make_case("tiny", N=N, Np=Np)
    kw = dict(n_ei=4, seed=12, hio_iters=7, er_iters=4, alpha=(0.1, 0.2, 0.4, 0.2, 0.1),
              wrap_mode=cp.WRAP_MIRROR, blend_target=cp.BLEND_OBJECT, n_pre=2,
              shrinkwrap_every=3)
    gw, ew, sw = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_WARP, **kw), d, d["support"], [11])
    gf, ef, sf = _run(cp, cp.make_config(N, Np, engine=cp.ENGINE_FUSED, **kw), d, d["support"], [11])
    assert np.array_equal(sf, sw)
    assert np.array_equal(gf, gw), f"max diff {np.abs(gf - gw).max():.3e}"
    np.testing.assert_allclose(ef, ew, rtol=1e-12, atol=0)


def test_fused_cfg1_er_windows_vs_oracle(cp):
    """cfg 1 (N = 64, Np = 32), ER on the true support with coupling every 10:
    50 iterations in five windowed launches, every iterate within 1e-4."""
    d = synth.make_case("cfg1")
    S = (d["proj"].numpy() > 1e-9).astype(np.uint8)
    cfg = cp.make_config(64, 32, seed=1, hio_iters=0, er_iters=50, n_ei=10, engine=cp.ENGINE_FUSED)
    plan = cp.Plan(cfg)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(S)
    oc = O.OracleConfig(N=64, Np=32, n_ei=10, beta=float(np.float32(cfg.beta)), hio_iters=0,
                        er_iters=50, seed=1)
    run = O.OracleRun.start(oc, d["I"], S)
    errs = []
    worst = 0.0
    for w in range(5):
        errs.append(plan.iterate(10, errors=True))
        run.run(10)
        r = _rel(plan.result(cp.RESULT_STATE), run.g).max()
        worst = max(worst, r)
        assert r < TOL, f"after window {w}: rel-L2 {r:.3e}"
    e = np.concatenate(errs)
    e_ref = np.array(run.errors)
    assert np.max(np.abs(e - e_ref) / e_ref) < TOL
    plan.close()
    print(f"fused cfg1 ER 50 iterations: worst rel-L2 {worst:.2e}")


@pytest.mark.parametrize("N", FUSED_N)
def test_fused_sizes_vs_oracle(cp, N):
    """Coupling, then 6 ER iterations split into windows of 1 and 5."""
    Np = 2
    d = synth.make_case("tiny", N=N, Np=Np)
    S = d["support"]
    cfg = cp.make_config(N, Np, n_ei=3, seed=2, hio_iters=0, er_iters=6, engine=cp.ENGINE_FUSED)
    plan = cp.Plan(cfg)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(S)
    e1 = plan.iterate(1, errors=True)
    g1 = plan.result(cp.RESULT_STATE)
    e2 = plan.iterate(5, errors=True)
    g6 = plan.result(cp.RESULT_STATE)
    plan.close()
    oc = O.OracleConfig(N=N, Np=Np, n_ei=3, beta=float(np.float32(cfg.beta)), hio_iters=0,
                        er_iters=6, seed=2)
    run = O.OracleRun.start(oc, d["I"], S)
    run.run(1)
    r1 = _rel(g1, run.g)
    run.run(5)
    r6 = _rel(g6, run.g)
    e_ref = np.array(run.errors)
    erel = np.abs(np.concatenate([e1, e2]) - e_ref) / e_ref
    print(f"N={N}: after 1 {r1.max():.2e}, after 6 {r6.max():.2e}, errors {erel.max():.2e}")
    assert r1.max() < TOL and r6.max() < TOL and erel.max() < TOL


def test_fused_rejects_unsupported(cp):
    for N, prec in ((1024, 0), (96, 0), (64, 1)):
        with pytest.raises(cp.CpraError) as e:
            cp.Plan(cp.make_config(N, 2, engine=cp.ENGINE_FUSED, precision=prec))
        assert e.value.status == cp.ERR_UNSUPPORTED


@pytest.mark.parametrize("use_graph", [False, True])
def test_fused_batch_rounds(cp, use_graph):
    """Fused plans at different iterations in one batch: each round launches
    every member's next window; results equal the plans run alone, and the
    launch count is the predicted number of rounds."""
    N, Np = 128, 4
    starts = [0, 3, 7]
    d = [synth.make_case("tiny", N=N, Np=Np, request=r) for r in range(3)]

    def mk(r):
        p = cp.Plan(cp.make_config(N, Np, seed=r, n_ei=5, hio_iters=9, er_iters=20,
                                   engine=cp.ENGINE_FUSED))
        p.load_intensities(d[r]["I"], 0, d[r]["thetas"])
        p.load_support(d[r]["support"])
        return p

    alone = [mk(r) for r in range(3)]
    for p, s0 in zip(alone, starts):
        p.iterate(s0 + 12)
    mixed = [mk(r) for r in range(3)]
    for p, s0 in zip(mixed, starts):
        p.iterate(s0)  # also seeds the start of the plan at 0 (one launch)
    b = cp.Batch(mixed, use_graph=use_graph)
    predicted = b.launches(12)
    n0 = cp.cpra_launch_count()
    b.iterate(12)
    for p in mixed:
        p.sync()
    assert cp.cpra_launch_count() - n0 == predicted
    for pa, pm in zip(alone, mixed):
        assert pm.iteration == pa.iteration
        assert np.array_equal(pa.result(cp.RESULT_STATE), pm.result(cp.RESULT_STATE))
        # the per-angle constants sum A^2 and C_n are FP64 atomics at load
        np.testing.assert_allclose(pa.result(cp.RESULT_ERRORS), pm.result(cp.RESULT_ERRORS),
                                   rtol=1e-12)
    b.close()
    for p in alone + mixed:
        p.close()
