"""Step C (cpra_merge) on the GPU against the oracle's merge_episodes.

Four guesses of the same 8 patterns start from states built from the true
projections (synthetic phantom, not from the GPU): plain with a little noise,
centrally inverted and shifted, shifted, and a random start; both sides run
5 ER iterations from them, then merge the 3 best.  The ranking and the twin
flags must agree exactly (the test checks that the oracle's decisions have
margins far above the 1e-4 parity of the iterates); the merged spectra and
the merged volume within 1e-4 relative L2; the PRTF within 1e-3 absolute:
each ring value is a mean of |sum E'| / sum |E'| ratios whose FP32 inputs
carry ~1e-6 relative error at the ring's typical magnitude but up to ~1e-4
at the weakest pixels of the outer rings.
"""
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
    a = a.reshape(a.shape[0], -1).astype(np.complex128)
    b = b.reshape(b.shape[0], -1).astype(np.complex128)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def _starts(P, S, seed=3):
    r = np.random.default_rng(seed)
    box = S.astype(bool)

    def noisy(x, amp):
        return np.where(box, x + amp * r.standard_normal(x.shape) * x.max(), 0.0).astype(np.float32)

    inv = np.roll(O.centrally_inverted(P), (-1, 1), axis=(-2, -1))
    return [noisy(P, 0.02), noisy(inv, 0.04), noisy(np.roll(P, (1, -1), axis=(-2, -1)), 0.06),
            np.where(box, r.random(P.shape), 0.0).astype(np.float32)]


@pytest.fixture(scope="module")
def case():
    d = synth.make_case("cfg1", N=64, Np=8)
    d["P"] = d["proj"].numpy().astype(np.float64)
    return d


def _gpu_guesses(cp, d, starts, iters, **kw):
    plans = []
    for g0 in starts:
        cfg = cp.make_config(64, 8, hio_iters=0, er_iters=iters, n_ei=1000, **kw)
        p = cp.Plan(cfg)
        p.load_intensities(d["I"], 0, d["thetas"])
        p.load_support(d["support"])
        p.load_state(g0, 1)
        p.iterate(iters)
        plans.append(p)
    return plans


def test_merge_matches_oracle(cp, case):
    d = case
    starts = _starts(d["P"], d["support"])
    iters = 5
    plans = _gpu_guesses(cp, d, starts, iters)
    dst = cp.Plan(cp.make_config(64, 8))
    dst.load_intensities(d["I"], 0, d["thetas"])
    prtf = np.zeros((8, 32), np.float32)
    sel, inv = cp.cpra_merge(plans, 3, 0, dst, prtf)
    E_gpu = dst.result(cp.RESULT_MERGED_SPECTRA)
    vol_gpu = dst.result(cp.RESULT_VOLUME)
    # oracle: the same starts, the same iterations, the same merge
    runs = []
    for g0 in starts:
        oc = O.OracleConfig(N=64, Np=8, n_ei=1000, hio_iters=0, er_iters=iters)
        r = O.OracleRun.start(oc, d["I"], d["support"], g0=g0.astype(np.float64))
        r.t = 1  # the GPU plans were loaded at t = 1
        runs.append(r.run(iters))
    errs = [np.asarray(r.errors[-1]) for r in runs]
    sel_o, inv_o, E_o, prtf_o = O.merge_episodes([r.g for r in runs], [r.S for r in runs], errs, 3, 0)
    ep = sorted(O.episode_error(e) for e in errs)
    assert min(np.diff(ep)) > 1e-3 * ep[0], ep  # ranking margin far above the parity
    assert sel == sel_o and inv == inv_o, (sel, sel_o, inv, inv_o)
    assert inv_o.count(True) == 1  # the inverted start is recognised
    r_spec = _rel(E_gpu, E_o)
    vol_o = O.assemble_spectra(E_o, d["thetas"])
    r_vol = np.linalg.norm(vol_gpu - vol_o) / np.linalg.norm(vol_o)
    d_prtf = np.abs(prtf - prtf_o).max()
    print(f"merge: selected {sel}, inverted {inv}; spectra rel-L2 {r_spec.max():.2e}, "
          f"volume {r_vol:.2e}, PRTF abs {d_prtf:.2e}")
    assert r_spec.max() < TOL and r_vol < TOL
    assert d_prtf < 1e-3
    for p in plans + [dst]:
        p.close()


def test_merge_of_one_guess_is_its_assembly(cp, case):
    """n_r = n_l = 1: the merged spectra are the guess's own moved spectra, so
    the merged volume equals cpra_assemble_3d of that plan bit for bit, and
    every PRTF ring is 1 (written to device memory)."""
    import torch
    d = case
    (p,) = _gpu_guesses(cp, d, _starts(d["P"], d["support"])[:1], 3)
    prtf = torch.zeros(8 * 32, device="cuda")
    sel, inv = cp.cpra_merge([p], 1, 0, p, prtf)
    assert sel == [0] and inv == [False]
    v_merge = p.result(cp.RESULT_VOLUME)
    p.assemble_3d()
    v_plain = p.result(cp.RESULT_VOLUME)
    assert np.array_equal(v_merge, v_plain)
    assert np.allclose(prtf.cpu().numpy(), 1.0, atol=1e-6)
    p.close()


def test_merge_invalid_arguments(cp, case):
    d = case
    plans = _gpu_guesses(cp, d, _starts(d["P"], d["support"])[:2], 1)
    fresh = cp.Plan(cp.make_config(64, 8))
    fresh.load_intensities(d["I"], 0, d["thetas"])
    other = cp.Plan(cp.make_config(32, 8))
    for args, status in [((plans, 3, 0, plans[0]), cp.ERR_INVALID_ARG),
                         ((plans, 0, 0, plans[0]), cp.ERR_INVALID_ARG),
                         ((plans, 1, 8, plans[0]), cp.ERR_INVALID_ARG),
                         ((plans + [other], 1, 0, plans[0]), cp.ERR_INVALID_ARG),
                         ((plans + [fresh], 1, 0, plans[0]), cp.ERR_NOT_READY)]:
        with pytest.raises(cp.CpraError) as ei:
            cp.cpra_merge(*args)
        assert ei.value.status == status
    with pytest.raises(cp.CpraError) as ei:
        fresh.result(cp.RESULT_MERGED_SPECTRA)
    assert ei.value.status == cp.ERR_NOT_READY
    for p in plans + [fresh, other]:
        p.close()
