"""Partial presence (cpra_set_present): only the angles marked present
iterate, and Eq. 4 couples each with its present neighbours, alpha
renormalised over them (the reading R13 of the oracle).  Checked on every
engine against the FP64 oracle, including a mask that grows mid-run."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


@pytest.mark.parametrize("engine", ["two_pass", "warp", "fused"])
def test_present_mask_tracks_oracle(cp, engine):
    N, Np = 64, 6
    d = synth.make_case("tiny", N=N, Np=Np, request=3)
    S = (d["proj"].numpy() > 1e-9).astype(np.uint8)
    eng = {"two_pass": cp.ENGINE_TWO_PASS, "warp": cp.ENGINE_WARP, "fused": cp.ENGINE_FUSED}[engine]
    cfg = cp.make_config(N, Np, n_ei=3, seed=8, hio_iters=0, er_iters=12, engine=eng)
    plan = cp.Plan(cfg)
    # only the present angles need intensities before they iterate
    mask1 = np.array([1, 1, 0, 1, 0, 1], np.uint8)
    I = d["I"].numpy() if hasattr(d["I"], "numpy") else np.asarray(d["I"])
    for n in np.flatnonzero(mask1):
        plan.load_intensities(I[n:n + 1], int(n), d["thetas"][n:n + 1])
    plan.load_support(S)
    plan.set_present(mask1)
    oc = O.OracleConfig(N=N, Np=Np, n_ei=3, beta=float(np.float32(cfg.beta)), hio_iters=0,
                        er_iters=12, seed=8)
    run = O.OracleRun.start(oc, d["I"], S)
    g0 = run.g.copy()
    run.present = mask1
    errs = [plan.iterate(5, errors=True)]
    run.run(5)
    g = plan.result(cp.RESULT_STATE)
    on = mask1 == 1
    r = _rel(g[on], run.g[on]).max()
    assert r < TOL, f"partial: rel-L2 {r:.3e}"
    assert np.array_equal(g[~on], g0[~on].astype(np.float32))  # the seeded start, untouched
    with pytest.raises(cp.CpraError) as e:
        plan.assemble_3d()
    assert e.value.status == cp.ERR_NOT_READY
    # the rest of the angles arrive: every angle iterates from here on
    for n in np.flatnonzero(~on):
        plan.load_intensities(I[n:n + 1], int(n), d["thetas"][n:n + 1])
    plan.set_present(None)
    run.present = None
    errs.append(plan.iterate(7, errors=True))
    run.run(7)
    r = _rel(plan.result(cp.RESULT_STATE), run.g).max()
    e = np.concatenate(errs)
    e_ref = np.array(run.errors)
    erel = np.abs(e - e_ref) / np.maximum(e_ref, 1e-300)
    plan.close()
    print(f"{engine}: rel-L2 {r:.2e}, errors {erel.max():.2e}")
    assert r < TOL and erel.max() < TOL
    assert np.all(e[:5, ~on] == 0.0)


def test_present_mask_rejections(cp):
    plan = cp.Plan(cp.make_config(32, 3))
    with pytest.raises(cp.CpraError) as e:
        plan.set_present(np.zeros(3))
    assert e.value.status == cp.ERR_INVALID_ARG
    plan.set_present([1, 0, 1])
    with pytest.raises(cp.CpraError) as e:
        plan.iterate(1)  # angles 0 and 2 have no intensities
    assert e.value.status == cp.ERR_NOT_READY
    plan.close()
    sw = cp.Plan(cp.make_config(32, 3, shrinkwrap_every=4))
    with pytest.raises(cp.CpraError) as e:
        sw.set_present([1, 0, 1])
    assert e.value.status == cp.ERR_UNSUPPORTED
    sw.close()


def test_batch_follows_present_masks(cp):
    """A batch member whose mask changes between calls equals the plan alone."""
    N, Np = 128, 5
    d = synth.make_case("tiny", N=N, Np=Np, request=4)

    def mk():
        p = cp.Plan(cp.make_config(N, Np, seed=2, n_ei=4, hio_iters=6, er_iters=10))
        p.load_intensities(d["I"], 0, d["thetas"])
        p.load_support(d["support"])
        return p

    m = np.array([1, 0, 1, 1, 0], np.uint8)
    alone = mk()
    alone.set_present(m)
    alone.iterate(6)
    alone.set_present(None)
    alone.iterate(6)
    mixed = mk()
    other = mk()
    b = cp.Batch([mixed, other], use_graph=True)
    mixed.set_present(m)
    b.iterate(6)
    mixed.set_present(None)
    b.iterate(6)
    assert np.array_equal(alone.result(cp.RESULT_STATE), mixed.result(cp.RESULT_STATE))
    b.close()
    for p in (alone, mixed, other):
        p.close()
