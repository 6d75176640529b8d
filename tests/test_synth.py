"""The seeded input generators (synth/), which both the oracle and the GPU
path read: properties the inputs must have, independent of either side."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import synth  # noqa: E402
import synth.phantom as P  # noqa: E402


@pytest.mark.parametrize("n_obj,n_ell,seed", [(32, 8, 3), (64, 40, 7), (96, 200, 11)])
def test_device_rasteriser_equals_host(n_obj, n_ell, seed):
    """The torch rasteriser (used on the GPU for large objects) draws the same
    seeded ellipsoids as the host loop and marks the same voxels (run here on
    the CPU device)."""
    torch = pytest.importorskip("torch")
    host = P.ellipsoid_phantom(n_obj, n_ell, seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    dev = P._ellipsoids_torch(n_obj, n_ell, rng, n_obj / 2 - 2, n_obj // 2, "cpu")
    assert isinstance(dev, torch.Tensor)
    assert np.array_equal(host.astype(np.float32), dev.numpy())


def test_phantom_stays_inside_its_cylinder():
    """Every ellipsoid lies inside the cylinder of radius n_obj/2 - 2 about z,
    so every projection fits the central box the padded-box support allows."""
    n = 48
    vol = P.ellipsoid_phantom(n, 30, 5)
    z, y, x = np.nonzero(vol)
    r = np.hypot(x - n // 2, y - n // 2)
    assert vol.max() <= 1.0 and vol.min() >= 0.0 and len(x) > 0
    assert r.max() <= n / 2 - 2 + 1.0


def test_projection_at_zero_degrees_is_the_smoothed_voxel_sum():
    """theta = 0: the t axis is y, so the projection is the sum over y; the
    two sub-samples in u (at +-1/4 pixel, bilinear) average each column with
    a quarter of its neighbours, a (1/8, 3/4, 1/8) smoothing along x."""
    torch = pytest.importorskip("torch")
    n = 16
    rng = np.random.default_rng(2)
    vol = np.zeros((n, n, n))
    vol[4:12, 5:11, 6:10] = rng.random((8, 6, 4))
    proj = P.project(torch.from_numpy(vol), np.array([0.0])).cpu().numpy()[0]
    s = vol.sum(axis=1)  # [z][x]
    pad = np.pad(s, ((0, 0), (1, 1)))
    expect = 0.125 * pad[:, :-2] + 0.75 * pad[:, 1:-1] + 0.125 * pad[:, 2:]
    assert np.allclose(proj, expect, rtol=1e-10, atol=1e-12)


def test_angles_and_support():
    th = synth.angles(8)
    assert np.allclose(th, np.arange(8) * math.pi / 8)
    S = synth.padded_box_support(64)
    assert S.shape == (64, 64) and 0 < S.sum() < 64 * 64
    ys, xs = np.nonzero(S)
    assert ys.min() > 0 and xs.min() > 0 and ys.max() < 63 and xs.max() < 63
