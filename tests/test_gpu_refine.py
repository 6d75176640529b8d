"""Step D refinement (cpra_refine_3d) on the GPU against the oracle's refine_3d.

The refinement is a sequence of projections onto convex sets (the
support-positivity cone and the spectra equal to the gridded E(q) on the
measured cells), so it does not amplify rounding: the FP32 iterates track
the FP64 oracle over every iteration.  The bar is the suite's 1e-4 relative
L2 on the refined volume and 1e-4 relative on every per-iteration error.
Inputs: the projections of a synthetic phantom (not from the GPU) loaded as
the plan's state, with each angle's support = where its projection is
positive, so the back-projected 3D support is tight.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
N, NP = 32, 16


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


def _case(N_, Np_):
    d = synth.make_case("cfg1", N=N_, Np=Np_)
    P = d["proj"].numpy().astype(np.float64)
    r = np.random.default_rng(5)
    S = P > 1e-9
    g = np.where(S, P * (1 + 0.05 * r.standard_normal(P.shape)), 0.0).astype(np.float32)
    d["g"], d["S2"] = g, S
    return d


@pytest.fixture(scope="module")
def case():
    return _case(N, NP)


def _plan(cp, d):
    N, NP = d["N"], d["Np"]
    p = cp.Plan(cp.make_config(N, NP))
    p.load_intensities(d["I"], 0, d["thetas"])
    p.load_support(d["S2"].astype(np.uint8))
    p.load_state(d["g"], 0)
    p.assemble_3d()
    return p


def _oracle(d, iters, shrink_every=0, sigma=1.5, tau=0.1):
    """Step D volume of the loaded state, then the refinement in its centred
    frame (R19-R21)."""
    th = d["thetas"]
    N = d["N"]
    g = d["g"].astype(np.float64)
    vol_c = O.volume(O.grid_3d(O.spectra(g, d["S2"]), th))
    M = O.measured_cells(N, th)
    S3 = O.backprojected_support(d["S2"], th, O.support_shifts(g, d["S2"]))
    out, S3f, errs = O.refine_3d(O.dft3(vol_c), M, S3, vol_c.real, iters, shrink_every, sigma, tau)
    return out, errs, S3, S3f


def test_refine_matches_oracle(cp, case):
    p = _plan(cp, case)
    e_gpu = p.refine_3d(20)
    vol = p.result(cp.RESULT_VOLUME)
    ref, e_ref, S3, _ = _oracle(case, 20)
    assert (case["vol"] > 0).sum() < S3.sum() < 0.1 * N ** 3  # tight, but holds the object
    r = np.linalg.norm(vol - ref) / np.linalg.norm(ref)
    er = np.abs(e_gpu - e_ref) / np.array(e_ref)
    print(f"refine 20: volume rel-L2 {r:.2e}, errors {er.max():.2e}, "
          f"error {e_ref[0]:.4f} -> {e_ref[-1]:.4f}")
    assert np.abs(vol.imag).max() == 0.0
    assert r < TOL and er.max() < TOL
    assert all(b <= a * (1 + 1e-4) for a, b in zip(e_gpu, e_gpu[1:]))  # the gap never grows
    p.close()


def test_refine_warp_fft_path_matches_oracle(cp):
    """N = 64 runs the line passes on the warp-resident FFTs (N = 32 above
    runs the block-wide ones): 12 iterations with shrink-wrap every 4."""
    d = _case(64, 12)
    p = _plan(cp, d)
    e_gpu = p.refine_3d(12, shrink_every=4, sigma=1.5, tau=0.1)
    vol = p.result(cp.RESULT_VOLUME)
    p.close()
    ref, e_ref, _, _ = _oracle(d, 12, shrink_every=4, sigma=1.5, tau=0.1)
    r = np.linalg.norm(vol - ref) / np.linalg.norm(ref)
    er = np.abs(e_gpu - e_ref) / np.array(e_ref)
    print(f"refine N=64 (warp FFTs) 12: volume rel-L2 {r:.2e}, errors {er.max():.2e}")
    assert r < TOL and er.max() < TOL


def test_refine_with_shrinkwrap_and_split_calls(cp, case):
    """Shrink-wrap every 5 (sigma 1.5, tau 0.1) over 15 iterations against the
    oracle; then 15 iterations as 7 + 8 in two calls equal one call of 15 bit
    for bit in the volume (the shrink-wrap count carries over; a new assembly
    restarts)."""
    p = _plan(cp, case)
    e_gpu = p.refine_3d(15, shrink_every=5, sigma=1.5, tau=0.1)
    vol = p.result(cp.RESULT_VOLUME)
    ref, e_ref, S3, S3f = _oracle(case, 15, shrink_every=5, sigma=1.5, tau=0.1)
    assert S3f.sum() != S3.sum()  # the shrink-wrap changed the support
    r = np.linalg.norm(vol - ref) / np.linalg.norm(ref)
    er = np.abs(e_gpu - e_ref) / np.array(e_ref)
    print(f"refine 15 with shrink-wrap: volume rel-L2 {r:.2e}, errors {er.max():.2e}")
    assert r < TOL and er.max() < TOL
    p.assemble_3d()
    a = p.refine_3d(7, shrink_every=5, sigma=1.5, tau=0.1)
    b = p.refine_3d(8, shrink_every=5, sigma=1.5, tau=0.1)
    assert np.array_equal(p.result(cp.RESULT_VOLUME), vol)
    # the error sums are FP64 atomics in launch order: equal up to summation order
    np.testing.assert_allclose(np.concatenate([a, b]), e_gpu, rtol=1e-12, atol=0)
    p.close()


def test_refine_needs_a_volume_and_valid_arguments(cp, case):
    p = cp.Plan(cp.make_config(case["N"], case["Np"]))
    p.load_intensities(case["I"], 0, case["thetas"])
    with pytest.raises(cp.CpraError) as ei:
        p.refine_3d(3)
    assert ei.value.status == cp.ERR_NOT_READY
    p.load_state(case["g"], 0)
    p.assemble_3d()
    for kw in (dict(shrink_every=-1), dict(shrink_every=2, sigma=0.0), dict(shrink_every=2, tau=1.5)):
        with pytest.raises(cp.CpraError) as ei:
            p.refine_3d(2, **kw)
        assert ei.value.status == cp.ERR_INVALID_ARG
    p.close()
