"""FP64 CPU oracle of the carousel phase retrieval algorithm (CPRA) hot path.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU baseline of ``bench.py``; never by the GPU library, with which it
shares no code.  Everything is float64 / complex128 numpy, written for
readability: transforms are dense DFT matrices (a matmul as the one library
step), pixel rules are ``np.where`` over whole arrays, loops follow the
paper's order.

Paper passages followed (arXiv 2402.05283, "Real time 3D coherent X-ray
diffraction imaging"):
  * Eq. 1-3   I_n = |FT2(O'_n)|^2: each measured pattern is the modulus of the
              2D FT of one projected object (PO); Fourier slice theorem.
  * Step A    one PO pre-reconstructed, the rest random (``n_pre``).
  * Step B    episodes W_m; each PO runs N_ei conventional 2D iterations
              starting from the Eq. 4 combination of the previous episode.
  * Eq. 4     carousel coupling O_n = sum_k alpha_k O_{n+k}, periodic in n.
  * Step C    N_r guesses, the N_l of lowest error kept, centre-of-mass move
              Delta r_n = -int O'_n r dv, twin (central inversion) choice by
              Euclidean distance to the best episode, average -> E_n; the
              PRTF of the merged guesses (results section, its ref. 23).
  * Step D    interpolation of the spectra E_n into the 3D E(q); inverse 3D FT;
              the tomographic 3D iteration on E(q) with a 3D support from the
              back-projected 2D supports, shrunk every few iterations (results
              section: 50 iterations, shrink every 5, GENFIRE its ref. 33).
  * HIO (Fienup, the paper's ref. 22) and ER updates; shrink-wrap (ref. 36)
    with the paper's 0.1 relative threshold.
  * RAAR (Luke, the paper's ref. 39), the update the paper runs with
    beta = 0.9 on its S. aureus data (results section).
  * Result verification (results section): PRTF and the Fourier shell
    correlation (FSC, its ref. 37) against the known object, each read at
    the 0.5 cut-off.

Readings where the paper is silent or garbled (the same list is kept with the
design notes):
  R1  Eq. 4 index: O_n^(m) = sum_{k=-r..r} alpha_k O^(m-1)_{(n+k) mod Np}
      (alpha_0 pairs with n itself).  Jacobi: every n reads episode m-1.
  R2  Wrap across the 180 degree seam: LITERAL (default) uses the unmirrored
      image; MIRROR flips u (x -> -x about the frame centre) once per wrap.
  R3  What is blended: the stored iterate g (STATE, default) or P_{S+} g
      (OBJECT).
  R4  Schedule: global iteration t = 0..T-1; coupling before t when
      t % n_ei == 0 (including t = 0); HIO while t < hio_iters, then ER;
      shrink-wrap after t when (t + 1) % shrinkwrap_every == 0.
  R5  Initial guess g0(x) = u * [x in S], u = (splitmix64(key) >> 40) * 2^-24,
      key = ((seed * Np + n) * N + y) * N + x  (mod 2^64).
  R6  The PO is real: g' = Re IDFT2(A * G / |G|); phase 1 where G = 0.
  R7  Valid set V = {x in S and g'(x) >= 0}.  HIO: g' on V, g - beta g'
      elsewhere; ER: g' on V, 0 elsewhere.
  R8  Fourier error E_F = sqrt(sum(|G| - A)^2 / sum A^2) of the iterate
      entering each iteration, full plane.
  R9  Shrink-wrap: rho = P_{S+} g, b = wrapped Gaussian (sigma px, periodic,
      normalised on the N x N torus) circularly convolved with rho,
      S <- {b >= tau * max b}; S unchanged when max b <= 0.
  R10 Assembly spectrum E_n = DFT2(P_{S+} g_n) * exp(+2 pi i k.c_n / N),
      signed k in [-N/2, N/2), c_n the centre of mass in pixels (or N/2 when
      com_align is off); this moves the mass centre to the origin.
  R11 Gridding: sample (ku, kz) of angle theta lands at
      (kx, ky, kz) = (ku cos theta, ku sin theta, kz); bilinear scatter in
      (kx, ky), exact kz; divide by the summed weight; cells with summed
      weight < 1e-12 are 0.  Volume = fftshift(IDFT3(V)).
  R12 FFT conventions: forward unnormalised with exp(-2 pi i jk/N), inverse
      carries 1/N per axis; intensities arrive centred and are ifftshifted.
  R13 Partial presence (serving while patterns still arrive, the concluding
      section's concurrent partial reconstruction): only angles marked
      present iterate; Eq. 4 couples each present angle with its present
      neighbours, the alpha_k of the present taps divided by their sum (all
      taps present: the alpha_k as given); absent angles keep their state.
  R14 RAAR with a positivity-constrained support: T = beta/2 (R_S R_M + I)
      + (1 - beta) P_M, reflections R = 2P - I, P_M g = g' (R6) and
      P_S = P_{S+}; it replaces HIO for the iterations before hio_iters
      (and in Step A) when the configuration selects it.
  R15 Episode reconstruction error (Step C ranks episodes by it, the paper
      does not define it): the mean over the POs of E_F (R8) in the last
      recorded iteration.  Ties keep the lower guess index first.
  R16 Twin choice: the distance is taken on one PO (index twin_ref, default
      0) after the mass-centre move, and the version chosen there is used for
      every PO of that episode (inverting the 3D object inverts every
      projection).  The inverted version of a moved PO rho_m is
      conj(rho_m(-x)), whose spectrum is conj(E_n); a tie keeps the plain one.
  R17 The final E_n is the spectrum of the mean of the corrected POs of the
      kept episodes (equivalently the mean of their spectra).
  R18 PRTF per PO: |sum_g E'_g| / sum_g |E'_g| over the kept, corrected
      episodes, averaged on rings s = round(|k|), s < N/2.
  R19 Step D's data: the gridded spectrum V of R11 on the cells the scatter
      reaches (summed weight >= 1e-12, every kz); elsewhere the iteration
      leaves the spectrum free.
  R20 3D support from the 2D supports ("projected back to 3D"): a voxel is
      inside iff its projection lands inside the 2D support at every angle
      (nearest pixel in u, exact z).  Each 2D support first moves with its
      PO: the mass-centre move of R10, rounded to whole pixels, so that it
      frames the moved PO in the centred volume.
  R21 The refinement (GENFIRE-like, the paper gives only "like conventional
      3D CXDI but using E(q)", 50 iterations, shrink every 5): alternating
      projections, P_{S3+} in real space and the replacement of the measured
      cells by the data in Fourier space.  It runs in the centred frame of
      the Step D volume (the frame of the 2D supports): the data are the
      spectrum of the centred volume, DFT3(fftshift3(IDFT3(V))), and the
      start is the real part of that volume (the phases of E(q) make one
      start enough); shrink-wrap as R9 in 3D; the result is P_{S3+} of the
      last iterate, centred.
  R22 Gauss-Seidel sweep (Step B's "consecutively, from n = 1 to n = N_p"):
      within an episode the angles are reconstructed in turn; angle n starts
      from Eq. 4 with the current episode's images of the angles before it
      and the previous episode's images of the others, then runs its N_ei
      iterations; an episode is the unit of a call.  Jacobi (R1) stays the
      default, the equation's literal form.  Shrink-wrap (R9) then runs at
      episode ends, for every angle, when its period is a whole number of
      episodes (the paper's cell run: one CSWA step at the end of each
      episode).
  R23 Missing data (the beamstop of the paper's cell patterns): a mask marks
      the measured pixels; the pair {k, -k} is constrained iff both are
      measured (a real PO has |G(-k)| = |G(k)|, and a centred beamstop is
      symmetric, so this loses nothing there); the modulus projection keeps
      G on the unconstrained pixels and the Fourier error sums over the
      constrained ones only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HIO, ER, RAAR = 0, 1, 2
WRAP_LITERAL, WRAP_MIRROR = 0, 1
BLEND_STATE, BLEND_OBJECT = 0, 1

__all__ = [
    "HIO", "ER", "RAAR", "WRAP_LITERAL", "WRAP_MIRROR", "BLEND_STATE", "BLEND_OBJECT",
    "dft_matrix", "dft2", "idft2", "dft3", "idft3", "fftshift2", "ifftshift2",
    "fftshift3", "amplitudes", "a_sym", "splitmix64", "initial_guess",
    "modulus_projection", "fourier_error_terms", "support_update", "constrained_pairs",
    "iterate_2d", "positivity_margin", "couple", "couple_sweep_one", "wrapped_gaussian", "blur", "shrinkwrap",
    "object_estimate", "centre_of_mass", "signed_freq", "spectra", "grid_3d", "grid_plane",
    "volume", "assemble", "OracleConfig", "OracleRun", "real_space_error",
    "r_factor", "raar_update", "episode_error", "select_best", "centrally_inverted", "prtf",
    "merge_episodes", "assemble_spectra", "measured_cells", "backprojected_support", "blur3",
    "refine_3d", "support_shifts", "align_to", "fsc", "fsc_resolution",
]


# --------------------------------------------------------------------------
# Discrete Fourier transforms by definition (R12)
# --------------------------------------------------------------------------
_DFT = {}


def dft_matrix(N: int, sign: int) -> np.ndarray:
    """F[k, j] = exp(sign * 2 pi i * (j k mod N) / N)."""
    key = (N, sign)
    if key not in _DFT:
        j = np.arange(N)
        jk = np.outer(j, j) % N
        _DFT[key] = np.exp(sign * 2j * np.pi * jk / N)
    return _DFT[key]


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2D DFT over the last two axes."""
    N = x.shape[-1]
    F = dft_matrix(N, -1)
    return F @ x @ F  # F is symmetric


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT over the last two axes (1/N^2)."""
    N = X.shape[-1]
    F = dft_matrix(N, +1)
    return (F @ X @ F) / (N * N)


def _along(F: np.ndarray, x: np.ndarray, axis: int) -> np.ndarray:
    return np.moveaxis(np.tensordot(F, x, axes=([1], [axis])), 0, axis)


def dft3(x: np.ndarray) -> np.ndarray:
    N = x.shape[-1]
    F = dft_matrix(N, -1)
    for ax in range(3):
        x = _along(F, x, ax)
    return x


def idft3(X: np.ndarray) -> np.ndarray:
    N = X.shape[-1]
    F = dft_matrix(N, +1)
    for ax in range(3):
        X = _along(F, X, ax)
    return X / float(N) ** 3


def fftshift2(x):
    N = x.shape[-1]
    return np.roll(x, (N // 2, N // 2), axis=(-2, -1))


def ifftshift2(x):
    N = x.shape[-1]
    return np.roll(x, (-(N // 2), -(N // 2)), axis=(-2, -1))


def fftshift3(x):
    N = x.shape[-1]
    return np.roll(x, (N // 2,) * 3, axis=(-3, -2, -1))


# --------------------------------------------------------------------------
# Inputs (Eq. 1-3): amplitudes and the initial guess
# --------------------------------------------------------------------------
def amplitudes(I_centred: np.ndarray) -> np.ndarray:
    """A = sqrt(I) in FFT order.  Negative or non-finite intensities are rejected."""
    I = np.asarray(I_centred, dtype=np.float64)
    if not np.all(np.isfinite(I)) or np.any(I < 0):
        raise ValueError("intensities must be finite and non-negative")
    return np.sqrt(ifftshift2(I))


def _neg_index(N):
    return (-np.arange(N)) % N


def a_sym(A: np.ndarray) -> np.ndarray:
    """Hermitian-symmetrised amplitude (A(k) + A(-k)) / 2 (used by the R6 identity pins)."""
    m = _neg_index(A.shape[-1])
    return 0.5 * (A + A[..., m[:, None], m[None, :]])


_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key: np.ndarray) -> np.ndarray:
    """First output of SplitMix64 (Steele, Lea, Flood 2014) seeded with ``key``."""
    with np.errstate(over="ignore"):
        z = np.asarray(key, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def initial_guess(seed: int, Np: int, N: int, S: np.ndarray) -> np.ndarray:
    """Seeded random start (R5), zero outside the support."""
    n = np.arange(Np, dtype=np.uint64)[:, None, None]
    y = np.arange(N, dtype=np.uint64)[None, :, None]
    x = np.arange(N, dtype=np.uint64)[None, None, :]
    with np.errstate(over="ignore"):
        key = ((np.uint64(seed) * np.uint64(Np) + n) * np.uint64(N) + y) * np.uint64(N) + x
    u = (splitmix64(key) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    return np.where(S.astype(bool), u, 0.0)


# --------------------------------------------------------------------------
# One conventional 2D iteration (Step B inner loop; R6-R8)
# --------------------------------------------------------------------------
def constrained_pairs(mask_centred: np.ndarray) -> np.ndarray:
    """R23: the FFT-order pixels the modulus constraint applies to: k is
    constrained iff k and -k are both measured (mask nonzero, centred like
    the intensities)."""
    m = ifftshift2(np.asarray(mask_centred).astype(bool))
    neg = _neg_index(m.shape[-1])
    return m & m[..., neg[:, None], neg[None, :]]


def modulus_projection(G: np.ndarray, A: np.ndarray, C=None) -> np.ndarray:
    """Replace |G| by A and keep the phase; phase 1 where G = 0.  With a
    constrained set C (R23), pixels outside it keep G."""
    mag = np.abs(G)
    phase = np.where(mag > 0, G / np.where(mag > 0, mag, 1.0), 1.0)
    return A * phase if C is None else np.where(C, A * phase, G)


def fourier_error_terms(G: np.ndarray, A: np.ndarray, C=None):
    """(sum (|G| - A)^2, sum A^2) per pattern over the full plane, or over the
    constrained pixels C (R23)."""
    d = np.abs(G) - A
    a = A
    if C is not None:
        d = np.where(C, d, 0.0)
        a = np.where(C, A, 0.0)
    return (d * d).sum(axis=(-2, -1)), (a * a).sum(axis=(-2, -1))


def raar_update(g, gp, S, beta):
    """RAAR (R14): beta/2 (R_S R_M g + g) + (1 - beta) P_M g, the operator
    written out with the reflections R = 2P - I of P_M g = g' and P_{S+}."""
    rm = 2.0 * gp - g                      # R_M g
    rs = 2.0 * object_estimate(rm, S) - rm  # R_S R_M g
    return 0.5 * beta * (rs + g) + (1.0 - beta) * gp


def support_update(g, gp, S, beta, algo):
    """HIO or ER real-space step on the valid set V = S and g' >= 0; RAAR (R14)."""
    if algo == RAAR:
        return raar_update(g, gp, S, beta)
    valid = S.astype(bool) & (gp >= 0)
    if algo == HIO:
        return np.where(valid, gp, g - beta * gp)
    return np.where(valid, gp, 0.0)


def iterate_2d(g, A, S, beta, algo, return_gp=False, fft=False, C=None):
    """One iteration for a stack of POs; returns (g_new, err_num, err_den[, g']).
    fft=True takes the transforms from numpy.fft (FP64, the same unnormalised
    forward / 1/N^2 inverse) instead of the dense DFT matrices: for sizes
    where the matrices are too slow.  C: constrained pixels (R23), None =
    every pixel."""
    if fft:
        G = np.fft.fft2(g)
    else:
        G = dft2(g)
    num, den = fourier_error_terms(G, A, C)
    P = modulus_projection(G, A, C)
    gp = (np.fft.ifft2(P) if fft else idft2(P)).real
    out = support_update(g, gp, S, beta, algo)
    return (out, num, den, gp) if return_gp else (out, num, den)


def positivity_margin(gp, S):
    """min over the support of |g'| / max |g'| per pattern: how close the
    sign test of the support update came to flipping (a diagnostic)."""
    sup = S.astype(bool)
    inside = np.where(sup, np.abs(gp), np.inf).reshape(gp.shape[0], -1).min(axis=1)
    return inside / np.maximum(np.abs(gp).reshape(gp.shape[0], -1).max(axis=1), 1e-300)


# --------------------------------------------------------------------------
# Carousel coupling, Eq. 4 (R1-R3)
# --------------------------------------------------------------------------
def _mirror_u(img):
    N = img.shape[-1]
    return img[..., _neg_index(N)]


def object_estimate(g, S):
    """P_{S+} g: the iterate on the valid set, zero elsewhere."""
    return np.where(S.astype(bool) & (g >= 0), g, 0.0)


def couple(g, alpha, wrap=WRAP_LITERAL, blend=BLEND_STATE, S=None, present=None):
    """O_n <- sum_{k=-r..r} alpha_k O_{(n+k) mod Np}, all n from the old stack
    (Eq. 4, R1).  With a present mask (R13) an absent n keeps its g, and a
    present n sums its present taps only, with weights alpha_k / sum of the
    present taps' alpha."""
    Np = g.shape[0]
    alpha = np.asarray(alpha, dtype=np.float64)
    r = len(alpha) // 2
    on = np.ones(Np, dtype=bool) if present is None else np.asarray(present).astype(bool)
    src = g if blend == BLEND_STATE else object_estimate(g, S)
    out = np.zeros_like(g, dtype=np.float64)
    for n in range(Np):
        if not on[n]:
            out[n] = g[n]
            continue
        taps = [k for k in range(-r, r + 1) if on[(n + k) % Np]]
        norm = 1.0 if len(taps) == 2 * r + 1 else sum(alpha[k + r] for k in taps)
        for k in taps:
            j = n + k
            img = src[j % Np]
            if wrap == WRAP_MIRROR and (j // Np) % 2 != 0:
                img = _mirror_u(img)
            out[n] += (alpha[k + r] / norm) * img
    return out


def couple_sweep_one(g_old, g_new, n, alpha, wrap=WRAP_LITERAL, blend=BLEND_STATE, S=None):
    """R22 (Gauss-Seidel sweep): the start of angle n in an episode whose
    angles are reconstructed one after another from n = 0: Eq. 4 with the
    episode-m image for the angles already done in this sweep (index < n,
    g_new) and the episode m-1 image for the others (g_old)."""
    Np = g_old.shape[0]
    alpha = np.asarray(alpha, dtype=np.float64)
    r = len(alpha) // 2
    out = np.zeros(g_old.shape[1:], dtype=np.float64)
    for k in range(-r, r + 1):
        j = n + k
        jm = j % Np
        src = g_new if jm < n else g_old
        img = src[jm] if blend == BLEND_STATE else object_estimate(src[jm], S[jm])
        if wrap == WRAP_MIRROR and (j // Np) % 2 != 0:
            img = _mirror_u(img)
        out += alpha[k + r] * img
    return out


# --------------------------------------------------------------------------
# Shrink-wrap (R9)
# --------------------------------------------------------------------------
def wrapped_gaussian(N: int, sigma: float) -> np.ndarray:
    """w[d] proportional to sum_m exp(-(d + mN)^2 / (2 sigma^2)), sum_d w = 1."""
    d = np.arange(N, dtype=np.float64)
    M = int(math.ceil(12 * sigma / N)) + 1
    w = np.zeros(N)
    for m in range(-M, M + 1):
        w += np.exp(-((d + m * N) ** 2) / (2 * sigma * sigma))
    return w / w.sum()


def blur(rho: np.ndarray, sigma: float) -> np.ndarray:
    """Circular convolution with the separable wrapped Gaussian: W rho W^T."""
    N = rho.shape[-1]
    w = wrapped_gaussian(N, sigma)
    idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
    W = w[idx]
    return W @ rho @ W.T


def shrinkwrap(g, S, sigma, tau):
    """New support {blur(P_{S+} g) >= tau * max}, per pattern."""
    b = blur(object_estimate(g, S), sigma)
    mx = b.max(axis=(-2, -1), keepdims=True)
    new = b >= tau * mx
    return np.where(mx > 0, new, S.astype(bool))


# --------------------------------------------------------------------------
# Assembly, Steps C (mass centre) and D (R10, R11)
# --------------------------------------------------------------------------
def centre_of_mass(rho: np.ndarray) -> np.ndarray:
    """(c_z, c_u) per pattern in pixels; (N/2, N/2) for an empty pattern."""
    N = rho.shape[-1]
    i = np.arange(N, dtype=np.float64)
    m0 = rho.sum(axis=(-2, -1))
    mz = (rho * i[:, None]).sum(axis=(-2, -1))
    mu = (rho * i[None, :]).sum(axis=(-2, -1))
    safe = np.where(m0 > 0, m0, 1.0)
    cz = np.where(m0 > 0, mz / safe, N / 2)
    cu = np.where(m0 > 0, mu / safe, N / 2)
    return np.stack([cz, cu], axis=-1)


def signed_freq(N: int) -> np.ndarray:
    k = np.arange(N)
    return np.where(k >= N // 2, k - N, k).astype(np.float64)


def spectra(g, S, com_align=True):
    """E_n[kz][ku] = DFT2(P_{S+} g_n) * exp(+2 pi i (kz c_z + ku c_u) / N)."""
    N = g.shape[-1]
    rho = object_estimate(g, S)
    if com_align:
        c = centre_of_mass(rho)
    else:
        c = np.full(g.shape[:-2] + (2,), N / 2.0)
    k = signed_freq(N)
    cz = c[..., 0][..., None, None]
    cu = c[..., 1][..., None, None]
    ramp = np.exp(2j * np.pi * (k[:, None] * cz + k[None, :] * cu) / N)
    return dft2(rho) * ramp


def grid_3d(E: np.ndarray, thetas, wmin: float = 1e-12) -> np.ndarray:
    """Literal 3D bilinear scatter of all slices, divided by the summed weight.

    Returns V[kz][ky][kx] in FFT index order.
    """
    Np, N, _ = E.shape
    k = signed_freq(N)
    num = np.zeros((N, N, N), dtype=np.complex128)
    wsum = np.zeros((N, N, N), dtype=np.float64)
    for n in range(Np):
        px = k * math.cos(thetas[n])
        py = k * math.sin(thetas[n])
        i0 = np.floor(px)
        j0 = np.floor(py)
        fx = px - i0
        fy = py - j0
        for di in (0, 1):
            for dj in (0, 1):
                w = (fx if di else 1 - fx) * (fy if dj else 1 - fy)
                ii = (i0.astype(np.int64) + di) % N
                jj = (j0.astype(np.int64) + dj) % N
                np.add.at(num, (slice(None), jj, ii), w[None, :] * E[n])
                np.add.at(wsum, (slice(None), jj, ii), np.broadcast_to(w[None, :], (N, N)))
    return np.where(wsum >= wmin, num / np.where(wsum >= wmin, wsum, 1.0), 0.0)


def grid_plane(E_kz: np.ndarray, thetas, wmin: float = 1e-12) -> np.ndarray:
    """One kz plane of grid_3d: the literal bilinear scatter of the samples
    E_kz[n][ku] = E_n(kz, ku) of every slice into the (ky, kx) plane, divided
    by the summed weight (Eq. 2-3: the slice of angle n passes through
    (ku cos, ku sin, kz) for every kz, so each plane gathers its own samples
    only).  The same loops in the same order as grid_3d, restricted to one
    plane, so it equals grid_3d(E)[kz] bit for bit.  Returns V[ky][kx]."""
    Np, N = E_kz.shape
    k = signed_freq(N)
    num = np.zeros((N, N), dtype=np.complex128)
    wsum = np.zeros((N, N), dtype=np.float64)
    for n in range(Np):
        px = k * math.cos(thetas[n])
        py = k * math.sin(thetas[n])
        i0 = np.floor(px)
        j0 = np.floor(py)
        fx = px - i0
        fy = py - j0
        for di in (0, 1):
            for dj in (0, 1):
                w = (fx if di else 1 - fx) * (fy if dj else 1 - fy)
                ii = (i0.astype(np.int64) + di) % N
                jj = (j0.astype(np.int64) + dj) % N
                np.add.at(num, (jj, ii), w * E_kz[n])
                np.add.at(wsum, (jj, ii), w)
    return np.where(wsum >= wmin, num / np.where(wsum >= wmin, wsum, 1.0), 0.0)


def volume(V: np.ndarray) -> np.ndarray:
    """Centred complex volume fftshift(IDFT3(V))."""
    return fftshift3(idft3(V))


def assemble(g, S, thetas, com_align=True):
    return volume(grid_3d(spectra(g, S, com_align), thetas))


# --------------------------------------------------------------------------
# Step C: repeating and merging (R15-R18)
# --------------------------------------------------------------------------
def episode_error(final_errors) -> float:
    """R15: reconstruction error of an episode = mean over its POs of the
    Fourier error E_F (R8) of its last recorded iteration."""
    return float(np.mean(np.asarray(final_errors, dtype=np.float64)))


def select_best(episode_errors, n_l):
    """The n_l episodes with the lowest error, best first (ties by index)."""
    e = [float(x) for x in episode_errors]
    return sorted(range(len(e)), key=lambda i: (e[i], i))[:n_l]


def centrally_inverted(img):
    """img(-x): central inversion about index 0 of the periodic grid."""
    m = _neg_index(img.shape[-1])
    return img[..., m[:, None], m[None, :]]


def prtf(E_corrected) -> np.ndarray:
    """R18: phase retrieval transfer function of each PO over the merged
    episodes: |sum_g E'_g(k)| / sum_g |E'_g(k)| (0 where the denominator is
    0), averaged over the pixels of each ring s = round(|k|) of signed
    frequencies, s = 0..N/2-1.  Returns [Np][N/2]."""
    num = np.abs(np.sum(E_corrected, axis=0))
    den = np.sum(np.abs(E_corrected), axis=0)
    ratio = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    N = ratio.shape[-1]
    k = signed_freq(N)
    ring = np.rint(np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)).astype(np.int64)
    out = np.zeros(ratio.shape[:-2] + (N // 2,))
    for r in range(N // 2):
        out[..., r] = ratio[..., ring == r].mean(axis=-1)
    return out


def merge_episodes(gs, Ss, final_errors, n_l, twin_ref=0, com_align=True):
    """Step C on N_r finished episodes (gs[i], Ss[i]: iterate and support
    stacks [Np][N][N] of guess i; final_errors[i]: its last E_F per PO).

    1. keep the n_l episodes of lowest error (R15);
    2. move the mass centre of every PO to the origin (R10's phase ramp) and
       return to real space: rho_m = IDFT2(E_n);
    3. twin (R16): compare PO twin_ref of every kept episode with PO twin_ref
       of the best one, as is and centrally inverted, conj(rho_m(-x)) (the
       inversion of the real PO; conj keeps it exact where the ramp leaves an
       imaginary part on the Nyquist lines); the version at the smaller
       Euclidean distance is used for every PO of that episode;
    4. average the corrected episodes (R17) and take the spectra of the mean
       as the final E_n.
    Returns (selected, inverted flags, E [Np][N][N] complex, PRTF [Np][N/2])."""
    sel = select_best([episode_error(e) for e in final_errors], n_l)
    moved = [idft2(spectra(gs[i], Ss[i], com_align)) for i in sel]
    ref = moved[0][twin_ref]
    corrected, inverted = [], []
    for rho in moved:
        twin = np.conj(centrally_inverted(rho))
        d_plain = np.linalg.norm(rho[twin_ref] - ref)
        d_twin = np.linalg.norm(twin[twin_ref] - ref)
        flip = bool(d_twin < d_plain)
        inverted.append(flip)
        corrected.append(twin if flip else rho)
    mean = np.mean(corrected, axis=0)
    E_corr = np.array([dft2(c) for c in corrected])
    return sel, inverted, dft2(mean), prtf(E_corr)


def assemble_spectra(E, thetas):
    """Step D from given spectra E[Np][N][N] (e.g. the merged episode)."""
    return volume(grid_3d(E, thetas))


# --------------------------------------------------------------------------
# Step D refinement: the tomographic 3D iteration (R19-R21)
# --------------------------------------------------------------------------
def measured_cells(N: int, thetas, wmin: float = 1e-12) -> np.ndarray:
    """R19: the (ky, kx) cells the bilinear scatter of R11 reaches with summed
    weight >= wmin; the same for every kz (the slices span all of kz)."""
    k = signed_freq(N)
    wsum = np.zeros((N, N))
    for th in thetas:
        px = k * math.cos(th)
        py = k * math.sin(th)
        i0 = np.floor(px)
        j0 = np.floor(py)
        fx = px - i0
        fy = py - j0
        for di in (0, 1):
            for dj in (0, 1):
                w = (fx if di else 1 - fx) * (fy if dj else 1 - fy)
                np.add.at(wsum, ((j0.astype(np.int64) + dj) % N, (i0.astype(np.int64) + di) % N), w)
    return wsum >= wmin


def backprojected_support(S2: np.ndarray, thetas, shifts=None) -> np.ndarray:
    """R20: voxel (z, y, x) is in the 3D support iff at every angle its
    projection coordinate u = rint((x - c) cos theta + (y - c) sin theta + c),
    c = N/2 (the geometry of R16), lies in [0, N) and the 2D support, moved
    by that angle's whole-pixel shift (dz, du) (periodic), holds (z, u):
    S2[n][(z + dz) mod N][(u + du) mod N]."""
    Np, N, _ = S2.shape
    c = N // 2
    y, x = np.meshgrid(np.arange(N) - c, np.arange(N) - c, indexing="ij")
    out = np.ones((N, N, N), dtype=bool)
    for n in range(Np):
        dz, du = (0, 0) if shifts is None else (int(shifts[n][0]), int(shifts[n][1]))
        moved = np.roll(S2[n].astype(bool), (-dz, -du), axis=(0, 1))
        u = np.rint(x * math.cos(thetas[n]) + y * math.sin(thetas[n]) + c).astype(np.int64)
        inside = (u >= 0) & (u < N)
        uc = np.clip(u, 0, N - 1)
        hit = moved[:, uc] & inside[None, :, :]  # [z][y][x]
        out &= hit
    return out


def support_shifts(g, S, com_align=True):
    """R20: the whole-pixel part of each PO's mass-centre move (R10) in the
    centred frame, (rint(c_z - N/2), rint(c_u - N/2)); zeros without it."""
    N = g.shape[-1]
    if not com_align:
        return np.zeros((g.shape[0], 2), dtype=np.int64)
    c = centre_of_mass(object_estimate(g, S))
    return np.rint(c - N / 2).astype(np.int64)


def blur3(rho: np.ndarray, sigma: float) -> np.ndarray:
    """Circular convolution with the wrapped Gaussian of R9 along every axis."""
    N = rho.shape[-1]
    w = wrapped_gaussian(N, sigma)
    W = w[(np.arange(N)[:, None] - np.arange(N)[None, :]) % N]
    for ax in range(3):
        rho = _along(W, rho, ax)
    return rho


def refine_3d(V, M, S3, rho0, n_iters, shrink_every=0, sigma=2.0, tau=0.1):
    """Step D's tomographic iteration on the assembled spectrum (R21).

    V: the spectrum [kz][ky][kx] (FFT order) of the frame the iteration runs
    in; M: measured cells [ky][kx] (R19); S3: 3D support (R20); rho0: the
    start (real).  Each iteration: rho_S = P_{S3+} rho; X = DFT3(rho_S); error
    sqrt(sum_M |X - V|^2 / sum_M |V|^2); X <- V on the measured cells;
    rho = Re IDFT3(X); every shrink_every iterations the 3D support shrinks
    to {blur(P_{S3+} rho) >= tau max} (R9 in 3D).
    Returns (P_{S3+} rho, S3, errors)."""
    M3 = np.broadcast_to(np.asarray(M, bool)[None], V.shape)
    S3 = np.asarray(S3, bool)
    den = (np.abs(V[M3]) ** 2).sum()
    rho = np.asarray(rho0, dtype=np.float64)
    errs = []
    for t in range(n_iters):
        X = dft3(np.where(S3 & (rho >= 0), rho, 0.0))
        errs.append(math.sqrt((np.abs(X - V)[M3] ** 2).sum() / den) if den > 0 else 0.0)
        rho = idft3(np.where(M3, V, X)).real
        if shrink_every > 0 and (t + 1) % shrink_every == 0:
            b = blur3(np.where(S3 & (rho >= 0), rho, 0.0), sigma)
            mx = b.max()
            if mx > 0:
                S3 = b >= tau * mx
    return np.where(S3 & (rho >= 0), rho, 0.0), S3, errs


# --------------------------------------------------------------------------
# The whole schedule (Steps A, B; R4)
# --------------------------------------------------------------------------
@dataclass
class OracleConfig:
    N: int
    Np: int
    n_ei: int = 10
    alpha: tuple = (0.2, 0.6, 0.2)
    beta: float = 0.9
    wrap: int = WRAP_LITERAL
    blend: int = BLEND_STATE
    hio_iters: int = 200
    er_iters: int = 20
    shrinkwrap_every: int = 0
    sw_sigma: float = 2.0
    sw_tau: float = 0.1
    n_pre: int = 0
    com_align: bool = True
    seed: int = 0
    update: int = HIO  # the rule before hio_iters: HIO or RAAR (R14)
    sweep: bool = False  # Gauss-Seidel episodes (R22) instead of Jacobi (R1)
    fft: bool = False  # Jacobi steps take numpy.fft transforms (iterate_2d fft mode)


@dataclass
class OracleRun:
    """State of one reconstruction: amplitudes, support, iterate, history."""
    cfg: OracleConfig
    A: np.ndarray
    S: np.ndarray
    g: np.ndarray = None
    t: int = 0
    errors: list = field(default_factory=list)
    margins: list = field(default_factory=list)
    present: np.ndarray = None  # R13: angles that iterate (None = all)
    C: np.ndarray = None  # R23: constrained pixels [Np][N][N] (None = all)

    @classmethod
    def start(cls, cfg: OracleConfig, I_centred, S0=None, g0=None, mask=None):
        A = amplitudes(I_centred)
        if S0 is None:
            S0 = np.zeros((cfg.N, cfg.N), dtype=bool)
            o = cfg.N // 4
            S0[o:o + cfg.N // 2, o:o + cfg.N // 2] = True
        S = np.broadcast_to(np.asarray(S0).astype(bool), A.shape).copy()
        g = initial_guess(cfg.seed, cfg.Np, cfg.N, S) if g0 is None else np.array(g0, dtype=np.float64)
        C = None if mask is None else np.broadcast_to(constrained_pairs(mask), A.shape).copy()
        run = cls(cfg=cfg, A=A, S=S, g=g, C=C)
        for _ in range(cfg.n_pre):  # Step A: angle 0 alone, the update rule
            g1, _, _ = iterate_2d(run.g[0:1], A[0:1], S[0:1], cfg.beta, cfg.update, C=run._c(0, 1))
            run.g[0] = g1[0]
        return run

    def _c(self, a, b):
        return None if self.C is None else self.C[a:b]

    def step(self):
        """One global iteration t (coupling first at episode starts)."""
        c = self.cfg
        if self.t % c.n_ei == 0:
            self.g = couple(self.g, c.alpha, c.wrap, c.blend, self.S, self.present)
        algo = c.update if self.t < c.hio_iters else ER
        g, num, den, gp = iterate_2d(self.g, self.A, self.S, c.beta, algo, return_gp=True,
                                     fft=c.fft, C=self.C)
        err = np.sqrt(num / den)
        if self.present is not None:  # absent angles keep their state (R13)
            on = np.asarray(self.present).astype(bool)
            g = np.where(on[:, None, None], g, self.g)
            err = np.where(on, err, 0.0)
        self.g = g
        self.errors.append(err)
        self.margins.append(positivity_margin(gp, self.S))
        if c.shrinkwrap_every > 0 and (self.t + 1) % c.shrinkwrap_every == 0:
            self.S = shrinkwrap(self.g, self.S, c.sw_sigma, c.sw_tau)
        self.t += 1
        return self

    def sweep_episode(self):
        """One Gauss-Seidel episode (R22): angles n = 0 .. Np-1 in turn, each
        started from couple_sweep_one and run n_ei iterations alone."""
        c = self.cfg
        if self.t % c.n_ei != 0:
            raise ValueError("a sweep starts at an episode boundary")
        new = self.g.copy()
        errs = np.zeros((c.n_ei, c.Np))
        for n in range(c.Np):
            x = couple_sweep_one(self.g, new, n, c.alpha, c.wrap, c.blend, self.S)[None]
            for it in range(c.n_ei):
                algo = c.update if self.t + it < c.hio_iters else ER
                x, num, den = iterate_2d(x, self.A[n:n + 1], self.S[n:n + 1], c.beta, algo,
                                         C=self._c(n, n + 1))
                errs[it, n] = math.sqrt(num[0] / den[0]) if den[0] > 0 else 0.0
            new[n] = x[0]
        self.g = new
        self.errors.extend(list(errs))
        self.t += c.n_ei
        if c.shrinkwrap_every > 0 and self.t % c.shrinkwrap_every == 0:  # at episode ends
            self.S = shrinkwrap(self.g, self.S, c.sw_sigma, c.sw_tau)
        return self

    def run(self, n):
        if self.cfg.sweep:
            if n % self.cfg.n_ei != 0:
                raise ValueError("sweeps run whole episodes")
            for _ in range(n // self.cfg.n_ei):
                self.sweep_episode()
            return self
        for _ in range(n):
            self.step()
        return self

    def po(self):
        return object_estimate(self.g, self.S)

    def assemble(self, thetas):
        return assemble(self.g, self.S, thetas, self.cfg.com_align)


# --------------------------------------------------------------------------
# Evaluation metrics
# --------------------------------------------------------------------------
def r_factor(g, A):
    """R = sum ||G| - A| / sum A per pattern, G = DFT2(g): the crystallographic
    R-factor of the modulus fit (reading 11 of the error metrics; the paper
    names only a "reconstruction error").  Sums run over the two pixel axes
    of each pattern; returns one value per pattern."""
    G = dft2(g)
    return np.abs(np.abs(G) - A).sum(axis=(-2, -1)) / A.sum(axis=(-2, -1))


def align_to(rec: np.ndarray, true: np.ndarray):
    """The copy of rec that best matches true under the ambiguities phase
    retrieval leaves for a positive density: central inversion, integer
    (periodic) translation and a scale.  Returns (aligned, error) with
    aligned = c * roll(cand, shift), error = ||aligned - true|| / ||true||,
    minimised over cand in {rec, flip(rec)} with, for each, the shift that
    maximises the circular cross-correlation (an FFT, library step) and the
    least-squares scale c = <moved, true> / <moved, moved>.

    np.flip maps x -> -1 - x, the central inversion x -> -x followed by a
    shift of -1 on every axis, which the shift search absorbs."""
    rec = np.asarray(rec, dtype=np.float64)
    true = np.asarray(true, dtype=np.float64)
    axes = tuple(range(rec.ndim))
    best, best_img = np.inf, None
    Ft = np.fft.fftn(true)
    for cand in (rec, np.flip(rec, axis=axes)):
        xc = np.fft.ifftn(Ft * np.conj(np.fft.fftn(cand))).real
        shift = np.unravel_index(np.argmax(xc), xc.shape)
        moved = np.roll(cand, shift, axis=axes)
        den = (moved * moved).sum()
        c = (moved * true).sum() / den if den > 0 else 0.0
        err = np.linalg.norm(c * moved - true) / np.linalg.norm(true)
        if err < best:
            best, best_img = err, c * moved
    return best_img, float(best)


def real_space_error(rec: np.ndarray, true: np.ndarray) -> float:
    """min over {x, -x} and integer shifts of ||c rec - true|| / ||true||, best
    scale c (reading 11 of the error metrics): the error of align_to."""
    return align_to(rec, true)[1]


def fsc(vol_a: np.ndarray, vol_b: np.ndarray) -> np.ndarray:
    """Fourier shell correlation of two N^3 volumes, the paper's measure of
    agreement between the original and the reconstructed object (results
    section, its ref. 37; the resolution is read where it falls below 0.5):

        FSC(s) = Re sum_{k in s} F_a(k) conj(F_b(k))
                 / sqrt( sum_{k in s} |F_a(k)|^2  sum_{k in s} |F_b(k)|^2 ),

    F = DFT3 of the volume, shell s = {k : round(|k|) = s} over signed
    frequencies k in [-N/2, N/2)^3, s = 0..N/2-1 (the rings of the PRTF, in
    three dimensions); 0 where a shell has no power.  Translation and
    inversion are not removed here: align the volumes first (align_to)."""
    Fa = dft3(np.asarray(vol_a))
    Fb = dft3(np.asarray(vol_b))
    N = Fa.shape[-1]
    k = signed_freq(N)
    shell = np.rint(np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2
                            + k[None, None, :] ** 2)).astype(np.int64)
    out = np.zeros(N // 2)
    for s in range(N // 2):
        m = shell == s
        num = np.real(np.sum(Fa[m] * np.conj(Fb[m])))
        den = math.sqrt(np.sum(np.abs(Fa[m]) ** 2) * np.sum(np.abs(Fb[m]) ** 2))
        out[s] = num / den if den > 0 else 0.0
    return out


def fsc_resolution(curve: np.ndarray, threshold: float = 0.5) -> int:
    """The first shell whose correlation falls below the threshold (0.5, the
    paper's cut-off for FSC and PRTF); len(curve) when none does.  The
    resolution R^-1 is that shell's spatial frequency, shell / (N px)."""
    below = np.nonzero(np.asarray(curve) < threshold)[0]
    return int(below[0]) if below.size else int(len(curve))
