"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: closed
forms, a library routine (numpy.fft), brute force on tiny inputs, values the
paper prints, or invariants that a dropped term / wrong sign / transposed
operand would break.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def _rand(*shape):
    return rng.standard_normal(shape)


# ---------------------------------------------------------------- transforms
def test_dft_closed_forms():
    N = 8
    d = np.zeros((N, N)); d[0, 0] = 1.0
    assert np.allclose(O.dft2(d), np.ones((N, N)), atol=1e-14)
    # one plane wave -> one delta at its frequency
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    w = np.exp(2j * np.pi * (3 * y + 5 * x) / N)
    W = O.dft2(w)
    expect = np.zeros((N, N), complex); expect[3, 5] = N * N
    assert np.allclose(W, expect, atol=1e-11)
    # hand values: N = 2 -> [[a+b],[a-b]]; N = 4 row DFT of (1, 2, 3, 4)
    assert np.allclose(O.dft_matrix(2, -1), [[1, 1], [1, -1]], atol=1e-15)
    F4 = O.dft_matrix(4, -1)
    assert np.allclose(F4 @ np.array([1, 2, 3, 4.0]), [10, -2 + 2j, -2, -2 - 2j], atol=1e-14)
    # N = 3: exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
    assert np.allclose(O.dft_matrix(3, -1)[1, 1], -0.5 - 0.5j * math.sqrt(3), atol=1e-15)


@pytest.mark.parametrize("N", [16, 24, 48, 64])
def test_dft_matches_numpy_fft(N):
    x = _rand(3, N, N) + 1j * _rand(3, N, N)
    assert np.allclose(O.dft2(x), np.fft.fft2(x), rtol=0, atol=1e-10 * N * N)
    assert np.allclose(O.idft2(x), np.fft.ifft2(x), rtol=0, atol=1e-12)


def test_dft3_matches_numpy_and_roundtrip():
    N = 12
    x = _rand(N, N, N) + 1j * _rand(N, N, N)
    assert np.allclose(O.dft3(x), np.fft.fftn(x), atol=1e-9)
    assert np.allclose(O.idft3(O.dft3(x)), x, atol=1e-12)


def test_parseval_and_roundtrip():
    N = 32
    x = _rand(N, N)
    X = O.dft2(x)
    assert abs((x * x).sum() - (np.abs(X) ** 2).sum() / N ** 2) < 1e-9
    assert np.allclose(O.idft2(X).real, x, atol=1e-13)
    assert np.max(np.abs(O.idft2(X).imag)) < 1e-13


def test_shifts():
    N = 6
    x = np.arange(N * N).reshape(N, N)
    assert np.array_equal(O.fftshift2(x), np.fft.fftshift(x))
    assert np.array_equal(O.ifftshift2(x), np.fft.ifftshift(x))
    v = np.arange(N ** 3).reshape(N, N, N)
    assert np.array_equal(O.fftshift3(v), np.fft.fftshift(v))


# ---------------------------------------------------------------- inputs
def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0: the first two outputs of the published generator
    assert int(O.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    gamma = np.uint64(0x9E3779B97F4A7C15)
    assert int(O.splitmix64(gamma)) == 0x6E789E6AA1B965F4


def test_initial_guess_properties():
    N, Np = 16, 3
    S = np.zeros((N, N), bool); S[4:12, 4:12] = True
    g = O.initial_guess(5, Np, N, np.broadcast_to(S, (Np, N, N)))
    assert g.shape == (Np, N, N)
    assert np.all(g[:, ~S] == 0)
    assert np.all((g[:, S] >= 0) & (g[:, S] < 1))
    assert not np.allclose(g[0], g[1])
    assert np.array_equal(g, O.initial_guess(5, Np, N, np.broadcast_to(S, (Np, N, N))))
    assert abs(g[:, S].mean() - 0.5) < 0.05
    # values are multiples of 2^-24 (24-bit uniform)
    assert np.all(np.mod(g * 2 ** 24, 1) == 0)


def test_amplitudes_reject_negative_and_shift():
    N = 8
    I = np.zeros((N, N)); I[N // 2, N // 2] = 4.0  # centred q = 0
    A = O.amplitudes(I)
    assert A[0, 0] == 2.0 and A.sum() == 2.0
    with pytest.raises(ValueError):
        O.amplitudes(-I)
    with pytest.raises(ValueError):
        O.amplitudes(I * np.nan)


# ---------------------------------------------------------------- projections
def test_modulus_projection_idempotent_and_modulus():
    N = 16
    G = _rand(N, N) + 1j * _rand(N, N)
    G[2, 3] = 0
    A = np.abs(_rand(N, N))
    P = O.modulus_projection(G, A)
    assert np.allclose(np.abs(P), A, atol=1e-14)
    assert np.allclose(O.modulus_projection(P, A), P, atol=1e-14)
    assert P[2, 3] == A[2, 3]  # phase 1 where G = 0
    # phase preserved
    m = np.abs(G) > 0
    assert np.allclose(np.angle(P[m & (A > 0)]), np.angle(G[m & (A > 0)]), atol=1e-12)


def test_object_projection_idempotent():
    g = _rand(2, 8, 8)
    S = rng.random((2, 8, 8)) > 0.3
    p = O.object_estimate(g, S)
    assert np.array_equal(O.object_estimate(p, S), p)
    assert np.all(p >= 0) and np.all(p[~S] == 0)


def test_support_update_cases():
    g = _rand(8, 8); gp = _rand(8, 8)
    S = rng.random((8, 8)) > 0.5
    # with everything allowed and g' >= 0, HIO and ER both return g'
    full = np.ones((8, 8), bool)
    assert np.array_equal(O.support_update(g, np.abs(gp), full, 0.9, O.HIO), np.abs(gp))
    assert np.array_equal(O.support_update(g, np.abs(gp), full, 0.9, O.ER), np.abs(gp))
    # outside the support ER gives 0, HIO gives g - beta g'
    h = O.support_update(g, gp, S, 0.9, O.HIO)
    e = O.support_update(g, gp, S, 0.9, O.ER)
    assert np.all(e[~S] == 0) and np.allclose(h[~S], g[~S] - 0.9 * gp[~S])
    neg = S & (gp < 0)
    assert np.all(e[neg] == 0) and np.allclose(h[neg], g[neg] - 0.9 * gp[neg])


# ---------------------------------------------------------------- RAAR (R14)
def _raar_inputs(shape=(2, 16, 16)):
    g = _rand(*shape)
    gp = _rand(*shape)
    S = rng.random(shape) > 0.4
    return g, gp, S


def test_raar_pixel_cases():
    """The reflection form reduces, pixel by pixel, to: g' where x is in S and
    2g' - g >= 0 (R_M g lies in the constraint set, so R_S leaves it alone),
    beta g + (1 - 2 beta) g' elsewhere (R_S negates it).  Derived by hand
    from R = 2P - I, not from the oracle's expression."""
    g, gp, S = _raar_inputs()
    for beta in (0.9, 0.5, 0.3, 1.0):
        out = O.support_update(g, gp, S, beta, O.RAAR)
        keep = S & (2 * gp - g >= 0)
        assert np.allclose(out[keep], gp[keep], atol=1e-15)
        assert np.allclose(out[~keep], beta * g[~keep] + (1 - 2 * beta) * gp[~keep], atol=1e-14)


def test_raar_beta_one_is_douglas_rachford_and_relaxation():
    """beta = 1 is the averaged alternating reflections (Douglas-Rachford)
    map (R_S R_M + I) / 2, which outside the support equals HIO with beta = 1
    (Bauschke, Combettes and Luke); RAAR is the convex combination
    T_beta = beta T_1 + (1 - beta) P_M (Luke's relaxation)."""
    g, gp, S = _raar_inputs()
    t1 = O.support_update(g, gp, S, 1.0, O.RAAR)
    h1 = O.support_update(g, gp, S, 1.0, O.HIO)
    assert np.allclose(t1[~S], h1[~S], atol=1e-15)
    assert np.allclose(t1[~S], g[~S] - gp[~S], atol=1e-15)
    for beta in (0.9, 0.5, 0.25):
        tb = O.support_update(g, gp, S, beta, O.RAAR)
        assert np.allclose(tb, beta * t1 + (1 - beta) * gp, atol=1e-14)


def test_raar_is_continuous_where_hio_jumps():
    """Across the boundary of its valid set RAAR changes by O(eps) (both sides
    give g' when 2g' = g), while HIO jumps by |g| at g' = 0: the property that
    makes a wrong valid-set test (g' >= 0 instead of 2g' - g >= 0) visible."""
    gp = np.abs(_rand(64)) + 0.1
    S = np.ones(64, bool)
    eps = 1e-9
    lo = O.support_update(2 * gp - eps, gp, S, 0.9, O.RAAR)   # 2g' - g = +eps
    hi = O.support_update(2 * gp + eps, gp, S, 0.9, O.RAAR)   # 2g' - g = -eps
    assert np.max(np.abs(hi - lo)) < 1e-8
    g = np.abs(_rand(64)) + 0.5
    h_pos = O.support_update(g, np.full(64, eps), S, 0.9, O.HIO)
    h_neg = O.support_update(g, np.full(64, -eps), S, 0.9, O.HIO)
    assert np.min(np.abs(h_pos - h_neg)) > 0.4


def test_schedule_uses_raar_before_switch():
    P, A_true = _true_case(16, 8)
    I = np.fft.fftshift(A_true ** 2, axes=(-2, -1))
    cfg = O.OracleConfig(N=16, Np=2, n_ei=2, hio_iters=3, er_iters=2, seed=4, update=O.RAAR, n_pre=2)
    run = O.OracleRun.start(cfg, I)
    g = O.initial_guess(4, 2, 16, run.S)
    for _ in range(2):  # Step A with the same rule
        g1, _, _ = O.iterate_2d(g[0:1], run.A[0:1], run.S[0:1], 0.9, O.RAAR)
        g[0] = g1[0]
    assert np.array_equal(run.g, g)
    for t in range(5):
        if t % 2 == 0:
            g = O.couple(g, cfg.alpha)
        g, _, _ = O.iterate_2d(g, run.A, run.S, 0.9, O.RAAR if t < 3 else O.ER)
        run.step()
        assert np.array_equal(run.g, g)


def _true_case(N=32, seed=3):
    r = np.random.default_rng(seed)
    P = np.zeros((2, N, N))
    P[:, N // 4:3 * N // 4, N // 4:3 * N // 4] = r.random((2, N // 2, N // 2))
    A = np.abs(np.fft.fft2(P))  # library transform, independent of the oracle
    return P, A


def test_true_object_is_fixed_point():
    P, A = _true_case()
    S = P > 0
    for algo in (O.HIO, O.ER, O.RAAR):
        g, num, den = O.iterate_2d(P, A, S, 0.9, algo)
        assert np.max(np.abs(g - P)) < 1e-12
        assert np.all(num / den < 1e-26)


def test_real_state_identity_half_plane():
    """Re IDFT(A G/|G|) = IDFT(A_sym G/|G|) and the error splits exactly (R6)."""
    N = 16
    g = _rand(N, N)
    A = np.abs(_rand(N, N)) + 0.1  # not Hermitian-symmetric
    G = np.fft.fft2(g)
    full = np.fft.ifft2(O.modulus_projection(G, A)).real
    As = O.a_sym(A)
    half = np.fft.ifft2(O.modulus_projection(G, As))
    assert np.max(np.abs(half.imag)) < 1e-13
    assert np.allclose(full, half.real, atol=1e-13)
    m = (-np.arange(N)) % N
    D = 0.5 * (A - A[m[:, None], m[None, :]])
    lhs = ((np.abs(G) - A) ** 2).sum()
    rhs = ((np.abs(G) - As) ** 2).sum() + (D * D).sum()
    assert abs(lhs - rhs) < 1e-9 * lhs


# ---------------------------------------------------------------- missing data (R23)
def _beamstop(N, r):
    y, x = np.meshgrid(np.arange(N) - N // 2, np.arange(N) - N // 2, indexing="ij")
    return (x * x + y * y) > r * r  # measured outside a centred disc


def test_constrained_pairs():
    N = 16
    C = O.constrained_pairs(_beamstop(N, 2))
    k = O.signed_freq(N)
    assert np.array_equal(C, (k[:, None] ** 2 + k[None, :] ** 2) > 4)  # the disc moves to k = 0
    m = np.ones((N, N), bool)
    m[N // 2 + 3, N // 2 + 1] = False  # one unmeasured pixel, at k = (3, 1)
    C = O.constrained_pairs(m)
    assert not C[3, 1] and not C[-3, -1] and C.sum() == N * N - 2  # its partner is freed too


def test_masked_projection_and_error():
    N = 16
    G = np.fft.fft2(_rand(N, N))
    A = np.abs(_rand(N, N)) + 0.1
    C = O.constrained_pairs(_beamstop(N, 3))
    P = O.modulus_projection(G, A, C)
    assert np.allclose(np.abs(P[C]), A[C]) and np.array_equal(P[~C], G[~C])
    assert np.allclose(O.modulus_projection(P, A, C), P)  # idempotent
    num, den = O.fourier_error_terms(G, A, C)
    assert num == pytest.approx(((np.abs(G[C]) - A[C]) ** 2).sum())
    assert den == pytest.approx((A[C] ** 2).sum())
    # an all-measured mask is no mask
    full = O.constrained_pairs(np.ones((N, N), bool))
    assert np.array_equal(O.modulus_projection(G, A, full), O.modulus_projection(G, A))


def test_masked_true_object_fixed_point_and_identity():
    """The true object stays a fixed point whatever is missing; and the
    half-plane identity of R6 holds on the constrained pairs (both members
    of a pair are constrained together, so the projected spectrum stays
    Hermitian)."""
    P, A = _true_case()
    S = P > 0
    C = np.broadcast_to(O.constrained_pairs(_beamstop(32, 4)), A.shape)
    for algo in (O.HIO, O.ER, O.RAAR):
        g, num, den = O.iterate_2d(P, A, S, 0.9, algo, C=C)
        assert np.max(np.abs(g - P)) < 1e-12 and np.all(num / den < 1e-26)
    N = 16
    g = _rand(N, N)
    A2 = np.abs(_rand(N, N)) + 0.1
    C2 = O.constrained_pairs(_beamstop(N, 2))
    G = np.fft.fft2(g)
    full = np.fft.ifft2(O.modulus_projection(G, A2, C2)).real
    half = np.fft.ifft2(O.modulus_projection(G, O.a_sym(A2), C2))
    assert np.max(np.abs(half.imag)) < 1e-13 and np.allclose(full, half.real, atol=1e-13)


def test_beamstop_recovery_noiseless():
    """A central beamstop of radius 2 px removes the lowest frequencies; the
    support constraint restores them: HIO then ER on the tight support
    recovers every PO (real-space error < 0.05)."""
    import synth
    N, Np = 32, 3
    vol = synth.pad_volume(synth.ellipsoid_phantom(16, 3, 11), N)
    P = synth.project(vol, synth.angles(Np), r_max=8).numpy()
    I = np.fft.fftshift(np.abs(np.fft.fft2(P)) ** 2, axes=(-2, -1))
    cfg = O.OracleConfig(N=N, Np=Np, n_ei=1000, alpha=(1.0,), hio_iters=400, er_iters=100, seed=3)
    run = O.OracleRun.start(cfg, I, S0=P > 1e-12, mask=_beamstop(N, 2))
    run.run(500)
    rs = [O.real_space_error(run.po()[n], P[n]) for n in range(Np)]
    assert max(rs) < 0.05, rs


# ---------------------------------------------------------------- coupling
def test_coupling_paper_example_np3():
    gold = json.load(open(os.path.join(GOLD, "coupling_np3.json")))
    x = np.array(gold["inputs"])[:, None, None] * np.ones((3, 4, 4))
    out = O.couple(x, gold["alpha"])
    assert np.allclose(out[:, 0, 0], gold["expected"], atol=1e-15)


def test_coupling_identity_constant_and_linearity():
    g = _rand(5, 6, 6)
    assert np.array_equal(O.couple(g, [1.0]), g)
    assert np.allclose(O.couple(g, [0.0, 1.0, 0.0]), g)
    c = np.broadcast_to(_rand(1, 6, 6), (5, 6, 6))
    assert np.allclose(O.couple(c, [0.2, 0.6, 0.2]), c, atol=1e-15)
    h = _rand(5, 6, 6)
    a = [0.1, 0.2, 0.4, 0.2, 0.1]
    assert np.allclose(O.couple(2 * g + h, a), 2 * O.couple(g, a) + O.couple(h, a))
    # shift equivariance in n (periodic carousel)
    assert np.allclose(O.couple(np.roll(g, 2, axis=0), a), np.roll(O.couple(g, a), 2, axis=0))


def test_iterate_fft_mode_equals_dft_mode():
    """The numpy.fft transforms used at large N agree with the DFT matrices."""
    rng = np.random.default_rng(2)
    N = 24
    g = rng.random((2, N, N))
    A = rng.uniform(0.0, 5.0, size=(2, N, N))
    S = np.zeros((2, N, N), bool)
    S[:, 6:18, 6:18] = True
    for algo in (O.HIO, O.ER):
        a = O.iterate_2d(g, A, S, 0.9, algo, return_gp=True)
        b = O.iterate_2d(g, A, S, 0.9, algo, return_gp=True, fft=True)
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-11, atol=1e-12)
    # a whole run in FFT mode (the CPU baseline's timing mode) follows the
    # DFT-matrix run: ER with coupling, 6 iterations
    I = np.fft.fftshift(A ** 2, axes=(-2, -1))
    runs = [O.OracleRun.start(O.OracleConfig(N=N, Np=2, n_ei=3, alpha=(0.25, 0.5, 0.25), hio_iters=0,
                                             er_iters=6, seed=4, fft=f), I, S[0]).run(6)
            for f in (False, True)]
    assert np.allclose(runs[0].g, runs[1].g, rtol=1e-10, atol=1e-12)
    assert np.allclose(np.array(runs[0].errors), np.array(runs[1].errors), rtol=1e-10, atol=1e-14)


def test_sweep_coupling_hand_case_np3():
    """Gauss-Seidel starts on Np = 3 with the paper's alpha (0.2, 0.6, 0.2),
    old images 1, 2, 3 and this sweep's images 10, 20, 30 (hand arithmetic):
    angle 0 sees old 3, 1, 2 -> 1.6; angle 1 sees new 10, old 2, 3 -> 3.8;
    angle 2 sees new 20, old 3 and (wrapping to angle 0, already done) new
    10 -> 7.8."""
    old = np.array([1.0, 2.0, 3.0])[:, None, None] * np.ones((3, 2, 2))
    new = np.array([10.0, 20.0, 30.0])[:, None, None] * np.ones((3, 2, 2))
    got = [O.couple_sweep_one(old, new, n, (0.2, 0.6, 0.2))[0, 0] for n in range(3)]
    assert np.allclose(got, [1.6, 3.8, 7.8], atol=1e-14)


def test_sweep_spreads_one_episode_around_the_carousel():
    """The point of the sweep: a signal at angle 0 reaches every angle within
    one episode (each start uses the previous angle's new image), while the
    Jacobi coupling moves it one neighbour per episode."""
    Np = 6
    old = np.zeros((Np, 1, 1)); old[0] = 1.0
    new = np.zeros_like(old)
    for n in range(Np):
        new[n] = O.couple_sweep_one(old, new, n, (0.2, 0.6, 0.2))
    assert np.all(new[:, 0, 0] > 0)
    jac = O.couple(old, (0.2, 0.6, 0.2))
    assert np.count_nonzero(jac[:, 0, 0]) == 3
    # one tap: the sweep is the identity, like Jacobi
    assert np.array_equal(O.couple_sweep_one(old, new, 2, (1.0,)), old[2])


def test_sweep_schedule():
    """OracleRun in sweep mode = per angle: the sweep start, then n_ei
    iterations of that angle alone; HIO -> ER by the global index."""
    P, A_true = _true_case(16, 9)
    I = np.fft.fftshift(A_true ** 2, axes=(-2, -1))
    cfg = O.OracleConfig(N=16, Np=2, n_ei=2, hio_iters=3, er_iters=1, seed=2, sweep=True)
    run = O.OracleRun.start(cfg, I)
    g = run.g.copy()
    for ep in range(2):
        new = g.copy()
        for n in range(2):
            x = O.couple_sweep_one(g, new, n, cfg.alpha)[None]
            for it in range(2):
                t = 2 * ep + it
                x, _, _ = O.iterate_2d(x, run.A[n:n + 1], run.S[n:n + 1], 0.9, O.HIO if t < 3 else O.ER)
            new[n] = x[0]
        g = new
    run.run(4)
    assert np.array_equal(run.g, g) and run.t == 4 and len(run.errors) == 4
    # shrink-wrap every episode: after each sweep, for every angle
    cfg2 = O.OracleConfig(N=16, Np=2, n_ei=2, hio_iters=3, er_iters=1, seed=2, sweep=True,
                          shrinkwrap_every=2, sw_sigma=1.0)
    r2 = O.OracleRun.start(cfg2, I).run(2)
    r1 = O.OracleRun.start(cfg, I).run(2)
    assert np.array_equal(r2.g, r1.g)
    assert np.array_equal(r2.S, O.shrinkwrap(r1.g, r1.S, 1.0, 0.1))


def test_coupling_present_mask_hand_case():
    """R13 on Np = 3 with angle 2 absent and alpha = (0.2, 0.6, 0.2), constant
    images 1, 10, 100: angle 0 keeps taps 0 (0.6) and 1 (0.2), renormalised by
    0.8: (0.6 * 1 + 0.2 * 10) / 0.8 = 3.25; angle 1 keeps taps 0 (0.2) and 1
    (0.6): (0.2 * 1 + 0.6 * 10) / 0.8 = 7.75; angle 2 is left as it is."""
    x = np.array([1.0, 10.0, 100.0])[:, None, None] * np.ones((3, 4, 4))
    out = O.couple(x, [0.2, 0.6, 0.2], present=[1, 1, 0])
    assert np.allclose(out[:, 0, 0], [3.25, 7.75, 100.0], rtol=0, atol=1e-13)


def test_coupling_present_mask_invariants():
    g = _rand(7, 6, 6)
    a = [0.1, 0.2, 0.4, 0.2, 0.1]
    # every angle present: exactly the plain coupling
    assert np.array_equal(O.couple(g, a, present=np.ones(7)), O.couple(g, a))
    # one constant image everywhere stays that constant at every present angle
    # (the present weights sum to 1); absent angles keep their own image
    rng = np.random.default_rng(5)
    c = np.broadcast_to(_rand(1, 6, 6), (7, 6, 6)).copy()
    for _ in range(5):
        m = rng.integers(0, 2, size=7)
        m[rng.integers(0, 7)] = 1
        h = np.where(m[:, None, None] == 1, c, g)
        out = O.couple(h, a, wrap=O.WRAP_LITERAL, present=m)
        on = m == 1
        assert np.allclose(out[on], c[on], atol=1e-14)
        assert np.array_equal(out[~on], h[~on])


def test_oracle_run_present_mask():
    """Absent angles keep their state and error 0 through coupling steps."""
    N, Np = 16, 4
    rng = np.random.default_rng(9)
    I = rng.uniform(0.0, 50.0, size=(Np, N, N))
    cfg = O.OracleConfig(N=N, Np=Np, n_ei=2, hio_iters=2, er_iters=3, seed=4)
    run = O.OracleRun.start(cfg, I)
    g0 = run.g.copy()
    run.present = np.array([1, 0, 1, 1])
    run.run(5)
    assert np.array_equal(run.g[1], g0[1])
    assert all(e[1] == 0.0 for e in run.errors)
    assert all(e[0] > 0.0 for e in run.errors)


def test_coupling_mirror_seam():
    Np, N = 4, 6
    g = _rand(Np, N, N)
    out = O.couple(g, [0.25, 0.5, 0.25], wrap=O.WRAP_MIRROR)
    mirror = lambda im: im[:, (-np.arange(N)) % N]  # noqa: E731
    assert np.allclose(out[0], 0.25 * mirror(g[3]) + 0.5 * g[0] + 0.25 * g[1])
    assert np.allclose(out[3], 0.25 * g[2] + 0.5 * g[3] + 0.25 * mirror(g[0]))
    assert np.allclose(out[1], 0.25 * g[0] + 0.5 * g[1] + 0.25 * g[2])


def test_coupling_object_blend():
    g = _rand(3, 4, 4)
    S = rng.random((3, 4, 4)) > 0.4
    out = O.couple(g, [0.2, 0.6, 0.2], blend=O.BLEND_OBJECT, S=S)
    p = np.where(S & (g >= 0), g, 0)
    assert np.allclose(out[1], 0.2 * p[0] + 0.6 * p[1] + 0.2 * p[2])


# ---------------------------------------------------------------- shrink-wrap
def test_wrapped_gaussian():
    w = O.wrapped_gaussian(32, 2.0)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w[1:], w[1:][::-1])  # symmetric on the torus
    # far from the wrap it is the plain normalised Gaussian
    d = np.arange(-16, 16)
    plain = np.exp(-d * d / 8.0); plain /= plain.sum()
    assert np.allclose(np.roll(w, 16), plain, atol=1e-12)


def test_blur_brute_force_and_fft():
    N = 8
    rho = rng.random((N, N))
    b = O.blur(rho, 1.5)
    w = O.wrapped_gaussian(N, 1.5)
    brute = np.zeros((N, N))
    for y in range(N):
        for x in range(N):
            for yy in range(N):
                for xx in range(N):
                    brute[y, x] += w[(y - yy) % N] * w[(x - xx) % N] * rho[yy, xx]
    assert np.allclose(b, brute, atol=1e-14)
    h = np.outer(w, w)
    fft_form = np.fft.ifft2(np.fft.fft2(h) * np.fft.fft2(rho)).real
    assert np.allclose(b, fft_form, atol=1e-13)
    assert np.allclose(O.blur(np.full((N, N), 3.0), 1.5), 3.0)


def test_shrinkwrap_point_source_radius():
    """One bright pixel: support = disc where exp(-r^2 / 2 s^2) >= tau."""
    N, s, tau = 64, 2.0, 0.1
    g = np.zeros((1, N, N)); g[0, 32, 32] = 1.0
    S = np.ones((1, N, N), bool)
    new = O.shrinkwrap(g, S, s, tau)[0]
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    r2 = (y - 32) ** 2 + (x - 32) ** 2
    expect = r2 <= 2 * s * s * math.log(1 / tau)
    assert np.array_equal(new, expect)
    # an all-zero estimate keeps the old support
    assert np.array_equal(O.shrinkwrap(np.zeros((1, N, N)), S, s, tau), S)


# ---------------------------------------------------------------- assembly
def test_centre_of_mass_and_ramp_delta():
    N = 16
    g = np.zeros((1, N, N)); g[0, 5, 11] = 2.0
    S = np.ones((1, N, N), bool)
    assert np.allclose(O.centre_of_mass(g), [[5, 11]])
    E = O.spectra(g, S, com_align=True)
    assert np.allclose(E, 2.0, atol=1e-12)  # mass centre moved to the origin
    E0 = O.spectra(g, S, com_align=False)  # centred at N/2 instead
    k = O.signed_freq(N)
    expect = 2 * np.exp(-2j * np.pi * (k[:, None] * (5 - 8) + k[None, :] * (11 - 8)) / N)
    assert np.allclose(E0[0], expect, atol=1e-12)


def _axis_projection(vol, axis):
    return vol.sum(axis=axis)


def test_fourier_slice_axis_aligned():
    """DFT2 of the projection at 0 / 90 degrees is the central slice of the 3D DFT."""
    N = 12
    vol = rng.random((N, N, N))
    F3 = np.fft.fftn(vol)  # [kz][ky][kx]
    p0 = _axis_projection(vol, 1)  # theta = 0: sum over y -> [z][x]
    p90 = _axis_projection(vol, 2)  # theta = 90: sum over x -> [z][y]
    assert np.allclose(O.dft2(p0), F3[:, 0, :], atol=1e-10)
    assert np.allclose(O.dft2(p90), F3[:, :, 0], atol=1e-10)


def test_grid_single_slice_reproduces_plane():
    N = 8
    E = _rand(2, N, N) + 1j * _rand(2, N, N)
    V = O.grid_3d(E[:1], [0.0])
    assert np.allclose(V[:, 0, :], E[0], atol=1e-14)
    V[:, 0, :] = 0
    assert np.all(V == 0)
    V = O.grid_3d(E[1:], [math.pi / 2])
    assert np.allclose(V[:, :, 0], E[1], atol=1e-12)
    V[:, :, 0] = 0
    assert np.all(V == 0)


def test_grid_bilinear_weights_hand_case():
    """theta = 45 deg on N = 4 (ku in -2..1), only E(kz=0, ku=1) = 1, worked by hand.

    ku = 1 lands at (c, c), c = 1/sqrt(2): weights c*c on cell (1,1),
    c(1-c) on (0,1) and (1,0), (1-c)^2 on (0,0).  ku = 0 sits on (0,0) with
    weight 1; ku = -1 at (-c, -c) also reaches (0,0) with weight (1-c)^2;
    ku = -2 at (-2c, -2c) touches only cells -2 and -1 (indices 2, 3).
    """
    N = 4
    E = np.zeros((1, N, N), complex)
    E[0, 0, 1] = 1.0
    V = O.grid_3d(E, [math.pi / 4])
    c = 1 / math.sqrt(2)
    w00 = (1 - c) ** 2
    assert abs(V[0, 1, 1] - 1.0) < 1e-12  # only ku = 1 reaches (1,1)
    assert abs(V[0, 0, 1] - 1.0) < 1e-12  # ku = 0 reaches (0,1) with weight 0
    assert abs(V[0, 0, 0] - w00 / (1.0 + 2 * w00)) < 1e-12
    assert np.all(V[1:] == 0)  # other kz planes carry no data


def test_grid_plane_is_a_plane_of_grid_3d():
    """grid_plane (one kz plane, Eq. 2-3) against grid_3d on 16 angles at
    N = 16, every plane, bit for bit; and on the 45-degree hand case above."""
    N, Np = 16, 16
    E = _rand(Np, N, N) + 1j * _rand(Np, N, N)
    th = np.arange(Np) * math.pi / Np + 0.013
    V = O.grid_3d(E, th)
    for kz in range(N):
        assert np.array_equal(O.grid_plane(E[:, kz, :], th), V[kz])
    E1 = np.zeros((1, 4), complex)
    E1[0, 1] = 1.0
    c = 1 / math.sqrt(2)
    w00 = (1 - c) ** 2
    P = O.grid_plane(E1, [math.pi / 4])
    assert abs(P[1, 1] - 1.0) < 1e-12 and abs(P[0, 0] - w00 / (1.0 + 2 * w00)) < 1e-12


def test_volume_of_exact_spectrum_is_object():
    N = 10
    vol = rng.random((N, N, N))
    V = np.fft.fftn(np.fft.ifftshift(vol))
    assert np.allclose(O.volume(V), vol, atol=1e-12)


def test_assembly_axis_aligned_roundtrip():
    """A volume symmetric enough that 0/90 degree slices + gridding recover its central planes."""
    N = 16
    vol = np.zeros((N, N, N))
    vol[6:10, 6:10, 6:10] = rng.random((4, 4, 4))
    F3 = np.fft.fftn(np.fft.ifftshift(vol))
    E = np.stack([F3[:, 0, :], F3[:, :, 0]])
    V = O.grid_3d(E, [0.0, math.pi / 2])
    assert np.allclose(V[:, 0, 1:], F3[:, 0, 1:], atol=1e-10)
    assert np.allclose(V[:, 1:, 0], F3[:, 1:, 0], atol=1e-10)
    assert np.allclose(V[:, 0, 0], F3[:, 0, 0], atol=1e-10)


# ---------------------------------------------------------------- Step C merge (R15-R18)
def _po_stack(Np=3, N=16, seed=21):
    """Positive POs inside the central N/2 box (index 0 never touched)."""
    r = np.random.default_rng(seed)
    P = np.zeros((Np, N, N))
    P[:, N // 4:3 * N // 4, N // 4:3 * N // 4] = r.random((Np, N // 2, N // 2)) + 0.1
    return P


def test_merge_undoes_translation_and_inversion():
    """Step C names the two ambiguities it removes: a translation of a PO and
    its central inversion.  A second episode that is the first one inverted
    and shifted by an integer vector merges back onto the first exactly
    (flagged as inverted), the mean equals the first episode's moved spectra,
    and its PRTF is 1 on every ring."""
    N = 16
    A = _po_stack(N=N)
    S = np.ones_like(A, bool)
    B = np.roll(O.centrally_inverted(A), (2, -3), axis=(-2, -1))
    C = np.roll(A, (-1, 2), axis=(-2, -1))
    errs = [np.full(3, 0.1), np.full(3, 0.2), np.full(3, 0.3)]
    sel, inv, E, pr = O.merge_episodes([A, B, C], [S, S, S], errs, n_l=3)
    assert sel == [0, 1, 2] and inv == [False, True, False]
    E_A = O.spectra(A, S)
    assert np.allclose(E, E_A, rtol=0, atol=1e-10 * np.abs(E_A).max())
    assert np.allclose(pr, 1.0, atol=1e-12)


def test_merge_selects_lowest_errors_and_averages():
    N = 16
    A = _po_stack(N=N, seed=5)
    S = np.ones_like(A, bool)
    Z = np.zeros_like(A)
    errs = [np.full(3, 0.3), np.full(3, 0.1), np.array([0.2, 0.2, 0.2])]
    sel, inv, E, pr = O.merge_episodes([Z, A, 2 * A], [S, S, S], errs, n_l=2)
    assert sel == [1, 2] and inv == [False, False]
    # the mean of A and 2A (same mass centres) is 1.5 A
    assert np.allclose(E, 1.5 * O.spectra(A, S), atol=1e-10 * np.abs(E).max())
    assert O.select_best([0.5, 0.2, 0.2, 0.1], 3) == [3, 1, 2]  # ties by index
    assert O.episode_error([[0.1, 0.3], [0.2, 0.4]]) == pytest.approx(0.25)


def test_prtf_hand_cases():
    """|sum E| / sum |E|: 1 for equal phases, 0 for opposite phases, 1/sqrt 2
    for a quarter turn.  On a 4 x 4 grid (signed k in {-2, -1, 0, 1}) ring
    s = round(|k|) = 1 holds the 4 pixels at |k| = 1 and the 4 at |k| = sqrt 2,
    so one pixel with ratio 1 there averages to 1/8."""
    N = 4
    E = np.exp(1j * _rand(2, N, N)) * (1 + np.abs(_rand(2, N, N)))
    assert np.allclose(O.prtf(np.array([E, E])), 1.0)
    assert np.allclose(O.prtf(np.array([E, -E])), 0.0)
    assert np.allclose(O.prtf(np.array([E, 1j * E])), 1 / math.sqrt(2))
    one = np.zeros((1, N, N), complex)
    one[0, 0, 1] = 1.0  # k = (0, 1): ring 1; the other pixels have 0 / 0 -> 0
    pr = O.prtf(np.array([one, one]))
    assert np.allclose(pr[0], [0.0, 0.125])


# ---------------------------------------------------------------- Step D refinement (R19-R21)
def _box3(N, lo, hi):
    S = np.zeros((N, N, N), bool)
    S[lo:hi, lo:hi, lo:hi] = True
    return S


def test_refine_full_data_reaches_the_object_in_one_step():
    """With every cell measured the Fourier replacement is the whole
    spectrum: one iteration returns Re IDFT3(V), here the object itself, and
    the next error is 0 (V from numpy's FFT, a library routine)."""
    N = 12
    S3 = _box3(N, 3, 9)
    obj = np.where(S3, rng.random((N, N, N)), 0.0)
    V = np.fft.fftn(obj)
    M = np.ones((N, N), bool)
    out, _, errs = O.refine_3d(V, M, S3, rng.standard_normal((N, N, N)), 2)
    assert np.allclose(out, obj, atol=1e-12)
    assert errs[0] > 0.1 and errs[1] < 1e-12


def test_refine_without_data_is_the_support_projection():
    N = 10
    S3 = _box3(N, 2, 7)
    rho0 = rng.standard_normal((N, N, N))
    out, _, _ = O.refine_3d(np.zeros((N, N, N), complex), np.zeros((N, N), bool), S3, rho0, 3)
    assert np.allclose(out, np.where(S3 & (rho0 >= 0), rho0, 0.0), atol=1e-12)


def test_refine_error_never_increases():
    """Alternating projections between the support-positivity cone and the
    affine set of spectra equal to V on the measured cells: the gap between
    P_S rho_t and its Fourier replacement cannot grow (each projection is the
    nearest point of its set), whatever the data."""
    N = 12
    th = np.arange(5) * math.pi / 5
    M = O.measured_cells(N, th)
    assert 0 < M.sum() < N * N
    S3 = _box3(N, 2, 10)
    V = np.fft.fftn(np.abs(rng.standard_normal((N, N, N)))) * (1 + 0.3 * rng.standard_normal((N, N, N)))
    _, _, errs = O.refine_3d(V, M, S3, rng.random((N, N, N)), 15)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0]


def test_refine_dc_column_closed_form():
    """Only the (ky, kx) = (0, 0) cells measured: replacing them fixes the sum
    of every z plane, i.e. adds (target plane sum - current plane sum) / N^2
    to each voxel of the plane.  One iteration from rho0 must give
    P_{S3+}(P_{S3+} rho0 + that shift), and its error is the relative L2 gap
    of the plane sums (Parseval along z).  Checks the positivity inside the
    iteration, the real part and the error definition by plain sums."""
    N = 8
    S3 = _box3(N, 2, 6)
    obj = np.where(S3, rng.random((N, N, N)), 0.0)
    V = np.fft.fftn(obj)
    M = np.zeros((N, N), bool)
    M[0, 0] = True
    rho0 = rng.standard_normal((N, N, N))
    p0 = np.where(S3 & (rho0 >= 0), rho0, 0.0)
    t = obj.sum(axis=(1, 2))
    c = p0.sum(axis=(1, 2))
    rho1 = p0 + ((t - c) / N ** 2)[:, None, None]
    out, _, errs = O.refine_3d(V, M, S3, rho0, 1)
    assert np.allclose(out, np.where(S3 & (rho1 >= 0), rho1, 0.0), atol=1e-12)
    assert errs[0] == pytest.approx(np.linalg.norm(c - t) / np.linalg.norm(t), rel=1e-10)


def test_refine_shrinkwrap_point_source_ball():
    """No data, one bright voxel: the 3D shrink-wrap keeps the ball where
    exp(-r^2 / 2 sigma^2) >= tau (the 3D form of the 2D closed form)."""
    N, sg, tau = 24, 1.5, 0.1
    rho0 = np.zeros((N, N, N)); rho0[12, 12, 12] = 1.0
    _, S3, _ = O.refine_3d(np.zeros((N, N, N), complex), np.zeros((N, N), bool),
                           np.ones((N, N, N), bool), rho0, 1, shrink_every=1, sigma=sg, tau=tau)
    z, y, x = np.meshgrid(*(np.arange(N) - 12,) * 3, indexing="ij")
    assert np.array_equal(S3, x * x + y * y + z * z <= 2 * sg * sg * math.log(1 / tau))


def test_measured_cells_axis_aligned():
    N = 8
    M0 = O.measured_cells(N, [0.0])
    assert M0[0].all() and not M0[1:].any()          # theta = 0: the ky = 0 row
    M1 = O.measured_cells(N, [math.pi / 2])
    assert M1[:, 0].all() and not M1[:, 1:].any()    # theta = 90 deg: the kx = 0 column


def test_backprojected_support_axis_aligned():
    N = 8
    S2 = rng.random((2, N, N)) > 0.4
    only0 = O.backprojected_support(S2[:1], [0.0])
    assert np.array_equal(only0, np.broadcast_to(S2[0][:, None, :], (N, N, N)))
    both = O.backprojected_support(S2, [0.0, math.pi / 2])
    assert np.array_equal(both, S2[0][:, None, :] & S2[1][:, :, None])
    # a 2D support moved by (dz, du) = (1, -2) moves the 3D support by (-1, 2) in (z, x)
    moved = O.backprojected_support(S2[:1], [0.0], shifts=[(1, -2)])
    assert np.array_equal(moved, np.roll(only0, (-1, 2), axis=(0, 2)))
    # the shift of a PO whose mass centre sits at (N/2 + 1.2, N/2 - 2.8) is (1, -3)
    g = np.zeros((1, N, N)); g[0, N // 2 + 1, N // 2 - 3] = 0.8; g[0, N // 2 + 2, N // 2 - 2] = 0.2
    assert O.support_shifts(g, np.ones_like(g, bool)).tolist() == [[1, -3]]


def test_backprojected_support_contains_the_object():
    """The supports of the object's projections, projected back, contain the
    object's own support (every voxel of it projects inside at every angle)."""
    import synth
    N, Np = 32, 12
    vol = synth.pad_volume(synth.ellipsoid_phantom(16, 3, 33), N)
    th = synth.angles(Np)
    P = synth.project(vol, th, r_max=8).numpy()
    S3 = O.backprojected_support(P > 1e-9, th)
    inside = vol > 0
    assert np.all(S3[inside])
    assert S3.sum() < 0.2 * N ** 3  # and it is tight


def test_blur3_constant_and_separable():
    N = 8
    c = np.full((N, N, N), 2.5)
    assert np.allclose(O.blur3(c, 1.5), 2.5)
    d = np.zeros((N, N, N)); d[0, 0, 0] = 1.0
    w = O.wrapped_gaussian(N, 1.5)
    assert np.allclose(O.blur3(d, 1.5), w[:, None, None] * w[None, :, None] * w[None, None, :])


# ---------------------------------------------------------------- schedule
def test_schedule_coupling_and_switch():
    """The run applies Eq. 4 at episode starts and switches HIO -> ER at hio_iters."""
    P, A_true = _true_case(16, 7)
    I = np.fft.fftshift(A_true ** 2, axes=(-2, -1))
    cfg = O.OracleConfig(N=16, Np=2, n_ei=3, alpha=(0.25, 0.5, 0.25), hio_iters=4, er_iters=2, seed=1)
    run = O.OracleRun.start(cfg, I)
    g = run.g.copy()
    S = run.S
    A = run.A
    for t in range(6):
        if t % 3 == 0:
            g = O.couple(g, cfg.alpha)
        g, _, _ = O.iterate_2d(g, A, S, 0.9, O.HIO if t < 4 else O.ER)
        run.step()
        assert np.array_equal(run.g, g)
    assert run.t == 6 and len(run.errors) == 6


def test_phantom_recovery_noiseless_true_support():
    """Noiseless patterns, tight support: 400 HIO + 100 ER bring every PO's
    Fourier error below 1e-3 (the proposed end-to-end bound; measured
    2.9e-4 at worst) and its real-space error below 0.05 (measured 0.025)."""
    import synth
    N, Np = 32, 4
    obj = synth.ellipsoid_phantom(16, 3, 11)
    vol = synth.pad_volume(obj, N)
    th = synth.angles(Np)
    P = synth.project(vol, th, r_max=8).numpy()
    I = np.fft.fftshift(np.abs(np.fft.fft2(P)) ** 2, axes=(-2, -1))
    S = P > 1e-12
    cfg = O.OracleConfig(N=N, Np=Np, n_ei=1000, alpha=(1.0,), hio_iters=400, er_iters=100, seed=3)
    run = O.OracleRun.start(cfg, I, S0=S)
    run.run(500)
    err = np.array(run.errors)[-1]
    rs = [O.real_space_error(run.po()[n], P[n]) for n in range(Np)]
    assert np.max(err) < 1e-3, err
    assert np.max(rs) < 0.05, rs


# ---------------------------------------------------------------- evaluation metrics
def test_r_factor_hand_values():
    """R = sum ||G| - A| / sum A per pattern.  Pattern 0: g = delta at the
    origin, |G| = 1 on all 16 pixels of a 4 x 4 grid, A = 2: R = 16 / 32 = 0.5.
    Pattern 1: g = 2 delta, |G| = 2, A = 0, 1, ..., 15: sum |2 - A| =
    2 + 1 + 0 + 1 + 2 + ... + 13 = 94, sum A = 120, R = 94 / 120.  A sum
    over the wrong axes would mix the two patterns."""
    N = 4
    g = np.zeros((2, N, N))
    g[0, 0, 0] = 1.0
    g[1, 0, 0] = 2.0
    A = np.stack([np.full((N, N), 2.0), np.arange(16.0).reshape(N, N)])
    R = O.r_factor(g, A)
    assert R.shape == (2,)
    assert R[0] == pytest.approx(0.5, abs=1e-14)
    assert R[1] == pytest.approx(94.0 / 120.0, abs=1e-14)
    # a perfect modulus fit gives 0
    x = _rand(3, 8, 8)
    assert np.allclose(O.r_factor(x, np.abs(np.fft.fft2(x))), 0.0, atol=1e-13)


def test_real_space_error_removes_shift_inversion_and_scale():
    """A copy of a random volume that is centrally inverted, translated by a
    vector with every component non-zero and scaled by 3 has error 0; the
    same holds for each ambiguity alone.  A
    metric that lost the scale factor, skipped the inversion or searched the
    shift on the wrong axes would fail one of these."""
    v = rng.random((6, 7, 8))
    inv = v[np.ix_(*[(-np.arange(n)) % n for n in v.shape])]  # v(-x)
    for cand in (3.0 * v, np.roll(v, (2, -3, 5), axis=(0, 1, 2)),
                 inv, 3.0 * np.roll(inv, (1, 4, -2), axis=(0, 1, 2)), 0.25 * inv):
        img, err = O.align_to(cand, v)
        assert err < 1e-12
        assert np.allclose(img, v, atol=1e-12)
        assert O.real_space_error(cand, v) < 1e-12
    # a different object stays far
    assert O.real_space_error(rng.random((6, 7, 8)), v) > 0.2


def test_real_space_error_hand_case():
    """true = [[1, 0], [0, 0]], rec = [[2, 1], [0, 0]].  Every shift or
    inversion of rec puts 2 and 1 side by side in one row; the best puts 2
    on the 1 of true: c = <rec, true> / <rec, rec> = 2 / 5, residual
    (0.8 - 1, 0.4), error^2 = 0.04 + 0.16 = 0.2 = 1 - <rec, true>^2 / (|rec|^2 |true|^2)."""
    true = np.array([[1.0, 0.0], [0.0, 0.0]])
    rec = np.array([[2.0, 1.0], [0.0, 0.0]])
    img, err = O.align_to(rec, true)
    assert err == pytest.approx(math.sqrt(0.2), abs=1e-14)
    assert np.allclose(img, [[0.8, 0.4], [0.0, 0.0]], atol=1e-14)
    # in 1D with the better match off the first shift: true = [0, 0, 1, 3],
    # rec = [3, 1, 0, 0]: the inversion [0, 0, 1, 3] itself gives error 0
    assert O.real_space_error(np.array([3.0, 1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0, 3.0])) < 1e-14


def test_positivity_margin_hand_case():
    """min over the support of |g'| divided by max |g'| over the whole frame:
    g' = [[-1, 0.5], [2, -4]] with support [[1, 1], [0, 0]] gives 0.5 / 4;
    a second pattern with the support on the large values gives 2 / 4."""
    gp = np.array([[[-1.0, 0.5], [2.0, -4.0]], [[-1.0, 0.5], [2.0, -4.0]]])
    S = np.array([[[1, 1], [0, 0]], [[0, 0], [1, 1]]], bool)
    m = O.positivity_margin(gp, S)
    assert m.shape == (2,)
    assert m[0] == pytest.approx(0.125, abs=1e-15)
    assert m[1] == pytest.approx(0.5, abs=1e-15)


def test_fsc_identity_scale_and_sign():
    """FSC(V, V) = 1 and FSC(V, c V) = 1 on every shell for c > 0, and -1 for
    c < 0: the numerator must be Re sum F_a conj(F_b) (without the conj,
    FSC(V, V) = Re sum F^2 / sum |F|^2 is not 1 for a random V)."""
    v = rng.random((8, 8, 8))
    assert np.allclose(O.fsc(v, v), 1.0, atol=1e-12)
    assert np.allclose(O.fsc(v, 2.5 * v), 1.0, atol=1e-12)
    assert np.allclose(O.fsc(v, -0.3 * v), -1.0, atol=1e-12)
    # uncorrelated volumes give small values on the outer shells
    w = rng.random((8, 8, 8))
    assert np.all(np.abs(O.fsc(v - v.mean(), w - w.mean())[2:]) < 0.5)


def test_fsc_hand_shells_4cubed():
    """On a 4^3 grid (signed k in {-2, -1, 0, 1}): vol_a = delta at the
    origin (F_a = 1), vol_b = delta one voxel along the last axis
    (F_b = exp(-2 pi i k_x / 4)).  Shell 0 = {0}: FSC 1.  Shell 1 =
    round(|k|) = 1 holds |k|^2 = 1 (6 vectors) and |k|^2 = 2 (12 vectors),
    18 unit-modulus pixels; Re F_a conj F_b = cos(pi k_x / 2) is 1 where
    k_x = 0 (4 + 4 of them) and 0 where k_x = +-1, so FSC(1) = 8 / 18.  A
    floor in place of the rounding would add the 8 vectors of |k|^2 = 3
    (FSC 8 / 26)."""
    a = np.zeros((4, 4, 4))
    b = np.zeros((4, 4, 4))
    a[0, 0, 0] = 1.0
    b[0, 0, 1] = 1.0
    f = O.fsc(a, b)
    assert f.shape == (2,)
    assert f[0] == pytest.approx(1.0, abs=1e-14)
    assert f[1] == pytest.approx(8.0 / 18.0, abs=1e-14)
    assert O.fsc_resolution(f) == 1
    assert O.fsc_resolution(np.array([1.0, 0.9, 0.6])) == 3
    assert O.fsc_resolution(np.array([1.0, 0.5, 0.2])) == 2  # 0.5 is not below 0.5


def test_phantom_recovery_3d_fsc():
    """The whole method on a known phantom, read with the paper's FSC at 0.5
    (results section): N = 32, Np = 48 noiseless patterns, the true 2D
    supports, Eq. 4 with alpha = (0.2, 0.6, 0.2) every 10 iterations,
    200 HIO + 100 ER, Step D assembly.  After alignment with the phantom
    (align_to), the FSC stays above 0.5 out to shell 14 of 16 (measured:
    first shell below 0.5 is none, FSC 0.60 at the last shell); the same
    assembly from the exact projections keeps the FSC above 0.85 on every
    shell, which bounds what the gridding alone loses."""
    import synth
    N, Np = 32, 48
    vol = synth.pad_volume(synth.ellipsoid_phantom(16, 3, 21), N)
    th = synth.angles(Np)
    P = synth.project(vol, th, r_max=8).numpy()
    exact = O.assemble(P, np.ones((Np, N, N), bool), th, com_align=False).real
    f0 = O.fsc(O.align_to(exact, vol)[0], vol)
    assert np.all(f0 > 0.85), f0
    I = np.fft.fftshift(np.abs(np.fft.fft2(P)) ** 2, axes=(-2, -1))
    cfg = O.OracleConfig(N=N, Np=Np, n_ei=10, alpha=(0.2, 0.6, 0.2), hio_iters=200, er_iters=100, seed=3)
    run = O.OracleRun.start(cfg, I, S0=P > 1e-12)
    run.run(300)
    rec = run.assemble(th).real
    f = O.fsc(O.align_to(rec, vol)[0], vol)
    assert O.fsc_resolution(f) >= 14, f
    assert np.max(run.errors[-1]) < 5e-2


def test_assembly_recovers_phantom_from_exact_projections():
    """Step D from exact projections (Fourier slice theorem + gridding + IDFT3)
    reproduces the phantom: correlation above 0.95 at N = 32, Np = 48."""
    import synth
    N, Np = 32, 48
    vol = synth.pad_volume(synth.ellipsoid_phantom(16, 3, 21), N)
    th = synth.angles(Np)
    P = synth.project(vol, th, r_max=8).numpy()
    rec = O.assemble(P, np.ones((Np, N, N), bool), th, com_align=False)
    assert np.corrcoef(rec.real.ravel(), vol.ravel())[0, 1] > 0.95
    assert np.abs(rec.imag).max() < 0.05 * np.abs(rec.real).max()
