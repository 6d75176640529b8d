"""Ellipsoid phantoms, projections about z, and noisy far-field intensities.

Everything here is input synthesis (the forward model of Eq. 1-3 used to make
test data); the reconstruction method is not here.

Recipe (seeded; seed = case index * 1000 + request id):
  * object: n_obj^3 voxels, a union of ``n_ell`` ellipsoids written in seeded
    order (later ones overwrite earlier ones).  Semi-axes U[n_obj/16, n_obj/4],
    uniformly random orientation, density U[0.5, 1].  Every ellipsoid lies in
    the cylinder of radius n_obj/2 - 2 about z, so each projection stays inside
    the central n_obj x n_obj box (the padded bounding box support).
  * optional texture: density *= (1 + 0.2 * w), w = unit-variance white noise
    blurred with a Gaussian of ``texture_sigma`` voxels; clipped at 0.
  * the object is centred in an N^3 volume; index N/2 is the rotation axis.
  * projection at theta: P(u, z) = integral over t of
    O(u cos(theta) - t sin(theta), u sin(theta) + t cos(theta), z), bilinear
    interpolation of each z-plane at 2x supersampling in u and t.
  * intensity: I = |FFT2(P)|^2, centred, scaled so sum(I) = photons, then
    Poisson noise (numpy PCG64 on the CPU, a seeded torch generator on a GPU).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


def angles(Np: int) -> np.ndarray:
    """theta_n = n * pi / Np for n = 0..Np-1 (uniform over 180 degrees)."""
    return np.arange(Np, dtype=np.float64) * (math.pi / Np)


def _rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid_phantom(n_obj: int, n_ell: int, seed: int,
                      texture_sigma: float | None = None, device=None):
    """n_obj^3 float64 density [z][y][x]; coordinates relative to index n_obj/2.

    With a CUDA ``device`` the inside tests run there with torch (the same
    seeded draws; for large objects the host loop takes minutes) and the
    result is a float32 torch tensor on that device."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = n_obj / 2 - 2
    h = n_obj // 2
    if device is not None and str(device) != "cpu":
        return _ellipsoids_torch(n_obj, n_ell, rng, R, h, device)
    vol = np.zeros((n_obj, n_obj, n_obj))
    for _ in range(n_ell):
        a = rng.uniform(n_obj / 16, n_obj / 4, size=3)
        rot = _rotation(rng)
        amax = min(a.max(), R * 0.95)
        rc = (R - amax) * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        cz = rng.uniform(-(R - amax), R - amax)
        centre = np.array([rc * math.cos(phi), rc * math.sin(phi), cz])
        dens = rng.uniform(0.5, 1.0)
        # evaluate only inside the ellipsoid's bounding cube
        lo = np.maximum(np.floor(centre - a.max()).astype(int) + h, 0)
        hi = np.minimum(np.ceil(centre + a.max()).astype(int) + h + 1, n_obj)
        xs = np.arange(lo[0], hi[0]) - h
        ys = np.arange(lo[1], hi[1]) - h
        zs = np.arange(lo[2], hi[2]) - h
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        P = np.stack([X, Y, Z], axis=-1).astype(np.float64)
        local = (P - centre) @ rot  # coordinates in the ellipsoid frame
        inside = ((local / a) ** 2).sum(-1) <= 1.0
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = dens
    if texture_sigma:
        noise = rng.normal(size=vol.shape)
        k = _gauss_kernel(texture_sigma)
        for ax in range(3):
            noise = _conv1d_circ(noise, k, ax)
        noise /= noise.std()
        vol = np.where(vol > 0, np.clip(vol * (1 + 0.2 * noise), 0, None), 0.0)
    return vol


def _ellipsoids_torch(n_obj, n_ell, rng, R, h, device):
    vol = torch.zeros((n_obj, n_obj, n_obj), dtype=torch.float32, device=device)
    for _ in range(n_ell):
        a = rng.uniform(n_obj / 16, n_obj / 4, size=3)
        rot = _rotation(rng)
        amax = min(a.max(), R * 0.95)
        rc = (R - amax) * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        cz = rng.uniform(-(R - amax), R - amax)
        centre = np.array([rc * math.cos(phi), rc * math.sin(phi), cz])
        dens = rng.uniform(0.5, 1.0)
        lo = np.maximum(np.floor(centre - a.max()).astype(int) + h, 0)
        hi = np.minimum(np.ceil(centre + a.max()).astype(int) + h + 1, n_obj)
        xs = torch.arange(int(lo[0]), int(hi[0]), device=device, dtype=torch.float64) - h
        ys = torch.arange(int(lo[1]), int(hi[1]), device=device, dtype=torch.float64) - h
        zs = torch.arange(int(lo[2]), int(hi[2]), device=device, dtype=torch.float64) - h
        Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
        P = torch.stack([X, Y, Z], dim=-1) - torch.as_tensor(centre, device=device)
        local = P @ torch.as_tensor(rot, device=device)
        inside = ((local / torch.as_tensor(a, device=device)) ** 2).sum(-1) <= 1.0
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = dens
    return vol


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(4 * sigma))
    d = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-d * d / (2 * sigma * sigma))
    return k / k.sum()


def _conv1d_circ(x: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    r = len(k) // 2
    out = np.zeros_like(x)
    for i, w in enumerate(k):
        out += w * np.roll(x, i - r, axis=axis)
    return out


def pad_volume(obj: np.ndarray, N: int) -> np.ndarray:
    """Centre an n_obj^3 object in an N^3 volume (object index n_obj/2 -> N/2)."""
    n = obj.shape[0]
    vol = np.zeros((N, N, N), dtype=obj.dtype)
    o = N // 2 - n // 2
    vol[o:o + n, o:o + n, o:o + n] = obj
    return vol


def project(vol, thetas, r_max: float | None = None, ss: int = 2,
            z_chunk: int = 64, device: str | torch.device = "cpu",
            dtype=torch.float64) -> torch.Tensor:
    """Projections P_n[z][u] of an N^3 volume about z (rotation centre N/2).

    ``r_max`` limits the t integral (and the computed u range) to the radius
    that holds the object; None integrates the full frame.
    """
    vol_t = torch.as_tensor(vol, dtype=dtype, device=device)
    N = vol_t.shape[-1]
    Np = len(thetas)
    out = torch.zeros((Np, N, N), dtype=dtype, device=device)
    if r_max is None:
        r_max = N / 2
    t_half = int(math.ceil(r_max)) + 1
    nt = 2 * t_half * ss
    t = (torch.arange(nt, dtype=dtype, device=device) + 0.5) / ss - t_half
    u_lo = max(0, int(N // 2 - t_half))
    u_hi = min(N, int(N // 2 + t_half + 1))
    iu = torch.arange(u_lo, u_hi, dtype=dtype, device=device)
    sub = (torch.arange(ss, dtype=dtype, device=device) + 0.5) / ss - 0.5
    u = (iu[:, None] + sub[None, :]).reshape(-1) - N / 2  # (nu*ss,)
    z_nz = torch.nonzero(vol_t.abs().sum(dim=(1, 2)) > 0).flatten()
    if len(z_nz) == 0:
        return out
    z0, z1 = int(z_nz[0]), int(z_nz[-1]) + 1
    for n, th in enumerate(thetas):
        c, s = math.cos(th), math.sin(th)
        x = N / 2 + u[None, :] * c - t[:, None] * s  # (nt, nu*ss)
        y = N / 2 + u[None, :] * s + t[:, None] * c
        grid = torch.stack([2 * x / (N - 1) - 1, 2 * y / (N - 1) - 1], dim=-1)[None]
        for za in range(z0, z1, z_chunk):
            zb = min(z1, za + z_chunk)
            planes = vol_t[za:zb][None]  # (1, C=z, H=y, W=x)
            samp = torch.nn.functional.grid_sample(
                planes, grid, mode="bilinear", padding_mode="zeros", align_corners=True)
            # sum over t (step 1/ss), average over the ss sub-samples in u
            line = samp[0].sum(dim=1) / ss  # (z, nu*ss)
            line = line.reshape(zb - za, -1, ss).mean(dim=-1)
            out[n, za:zb, u_lo:u_hi] = line
    return out


def intensities(proj: torch.Tensor, photons: float | None, seed: int) -> np.ndarray | torch.Tensor:
    """Centred far-field intensities |FFT2(P)|^2 with optional Poisson noise.

    Returns float32 (numpy on the CPU, torch on a GPU device).
    """
    F = torch.fft.fft2(proj)
    I = torch.fft.fftshift(F.real ** 2 + F.imag ** 2, dim=(-2, -1))
    if photons is not None:
        I = I * (photons / I.sum(dim=(-2, -1), keepdim=True))
    if proj.device.type == "cpu":
        I = I.numpy()
        if photons is not None:
            rng = np.random.Generator(np.random.PCG64(seed))
            I = rng.poisson(I).astype(np.float64)
        return I.astype(np.float32)
    if photons is not None:
        gen = torch.Generator(device=proj.device)
        gen.manual_seed(seed)
        I = torch.poisson(I.float(), generator=gen)
    return I.float()


def padded_box_support(N: int, n_obj: int | None = None) -> np.ndarray:
    """uint8 [N][N], 1 on the central n_obj x n_obj box (default n_obj = N/2)."""
    if n_obj is None:
        n_obj = N // 2
    S = np.zeros((N, N), dtype=np.uint8)
    o = N // 2 - n_obj // 2
    S[o:o + n_obj, o:o + n_obj] = 1
    return S


@dataclass(frozen=True)
class Case:
    name: str
    N: int
    Np: int
    n_obj: int
    n_ell: int
    photons: float | None
    texture_sigma: float | None
    hio_iters: int
    er_iters: int
    shrinkwrap_every: int
    index: int


CASES = {
    # small cases the oracle finishes in seconds
    "tiny": Case("tiny", 32, 8, 16, 3, 1e6, None, 40, 10, 0, 90),
    "cfg1": Case("cfg1", 64, 32, 32, 6, 1e6, None, 200, 20, 0, 1),
    "cfg2": Case("cfg2", 256, 180, 128, 40, 1e7, 2.0, 500, 0, 20, 2),
    "metric": Case("metric", 512, 360, 256, 6, 1e6, None, 200, 20, 0, 6),
    "cfg5": Case("cfg5", 1024, 720, 512, 200, None, None, 50, 0, 0, 5),
}


def make_case(name: str, request: int = 0, device: str = "cpu", *,
              N: int | None = None, Np: int | None = None, raster_on_device: bool = False) -> dict:
    """Build intensities, angles and the padded-box support for a named case.

    ``N``/``Np`` override the case's sizes (objects scale to N/2 per side).
    ``raster_on_device`` rasterises an untextured object on the CUDA
    ``device`` too (the large configuration's 200-ellipsoid 512^3 object).
    On a CUDA ``device`` the projections and noise are made on the GPU with
    torch (fast for the large cases); the result is a torch float32 tensor
    on that device, otherwise numpy float32.
    """
    c = CASES[name]
    N = N or c.N
    Np = Np or c.Np
    n_obj = N // 2
    seed = c.index * 1000 + request
    if raster_on_device and c.texture_sigma is None:
        obj = ellipsoid_phantom(n_obj, c.n_ell, seed, None, device=device)
        vol = torch.zeros((N, N, N), dtype=obj.dtype, device=obj.device)
        o = N // 2 - n_obj // 2
        vol[o:o + n_obj, o:o + n_obj, o:o + n_obj] = obj
    else:
        obj = ellipsoid_phantom(n_obj, c.n_ell, seed, c.texture_sigma)
        vol = pad_volume(obj, N)
    th = angles(Np)
    dt = torch.float64 if str(device) == "cpu" else torch.float32
    P = project(vol, th, r_max=n_obj / 2, device=device, dtype=dt)
    I = intensities(P, c.photons, seed + 1)
    return dict(I=I, thetas=th, support=padded_box_support(N, n_obj), vol=vol,
                proj=P, N=N, Np=Np, case=c, seed=seed)
