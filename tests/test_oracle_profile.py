"""Pins of the oracle's transmural HA profile (histogram of HA against wall depth)."""
import math

import numpy as np

from oracle import profile


def _field(seed=0, shape=(6, 9, 11)):
    rng = np.random.default_rng(seed)
    ha = rng.uniform(-90.0, 90.0, size=shape)
    ha[rng.random(shape) < 0.1] = np.nan
    mask = (rng.random(shape) < 0.8).astype(np.uint8)
    return ha, mask


def test_vectorised_equals_voxel_loops():
    ha, mask = _field()
    args = ((2, 3, 1), (7.3, 6.1, 2.0), (0.2, -0.1, 1.0), 1.5, 6.5, 5, 12)
    a = profile.transmural_profile(ha, mask, *args)
    b = profile.transmural_profile_loops(ha, mask, *args)
    np.testing.assert_array_equal(a, b)
    assert a.sum() > 50


def test_constant_ha_fills_one_column():
    shape = (4, 40, 40)
    ha = np.full(shape, 37.3)
    out = profile.transmural_profile(ha, None, (0, 0, 0), (19.5, 19.5, 0.0), (0, 0, 1), 5.0, 15.0, 4, 36)
    kh = math.floor((37.3 + 90.0) * 36 / 180.0)
    assert out[:, kh].sum() == out.sum() > 0
    assert (out.sum(axis=0) > 0).sum() == 1


def test_ha_range_ends():
    ha = np.array([[[-90.0, 90.0, 0.0, -89.999]]])
    out = profile.transmural_profile(ha, None, (0, 0, 0), (0.0, -10.0, 0.0), (0, 0, 1), 5.0, 15.0, 1, 18)
    assert out[0, 0] == 2 and out[0, 17] == 1 and out[0, 9] == 1


def test_depth_bins_follow_ring_areas():
    """Voxel centres per depth bin of a cylinder wall ~ ring areas pi (r2^2 - r1^2)."""
    n = 101
    ha = np.zeros((2, n, n))
    r_in, r_out, nd = 20.0, 40.0, 4
    out = profile.transmural_profile(ha, None, (0, 0, 0), (50.0, 50.0, 0.0), (0, 0, 1), r_in, r_out, nd, 1)
    edges = np.linspace(r_in, r_out, nd + 1)
    expect = 2 * math.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    np.testing.assert_allclose(out[:, 0].astype(float), expect, rtol=0.03)


def test_rotation_about_the_axis_leaves_the_profile():
    ha, mask = _field(3, shape=(3, 21, 21))
    c, a = (10.0, 10.0, 0.0), (0, 0, 1)
    a1 = profile.transmural_profile(ha, mask, (0, 0, 0), c, a, 2.0, 9.0, 3, 10)
    rot = np.rot90(ha, axes=(1, 2)).copy()  # quarter turn about z through the centre
    mrot = np.rot90(mask, axes=(1, 2)).copy()
    a2 = profile.transmural_profile(rot, mrot, (0, 0, 0), c, a, 2.0, 9.0, 3, 10)
    np.testing.assert_array_equal(a1, a2)


def test_mask_and_nan_excluded():
    ha = np.full((1, 1, 3), 10.0)
    ha[0, 0, 1] = np.nan
    mask = np.array([[[1, 1, 0]]], dtype=np.uint8)
    out = profile.transmural_profile(ha, mask, (0, 0, 0), (0.0, -10.0, 0.0), (0, 0, 1), 5.0, 15.0, 1, 1)
    assert out.sum() == 1
