"""Pins of the oracle's filtering stages against things other than itself.

Gaussian kernels and the gradient / structure tensor (Figure 1b; Architecture,
"orientation"; chunking with padding, Implementation) are checked against
scipy.ndimage (an independent implementation of the same textbook filters),
against direct non-separable triple sums on tiny volumes, against closed forms
(linear ramp, constant volume) and against exact symmetries.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import oracle as O

RNG = np.random.default_rng(12345)


@pytest.mark.parametrize("s,R", [(1.0, 4), (1.5, 6), (2.0, 8), (3.0, 12), (4.0, 16), (6.0, 24), (8.0, 32), (9.0, 36)])
def test_radius_table(s, R):
    # R = floor(4 s + 0.5): the truncation radii of the workloads' scales.
    assert O.radius(s) == R


@pytest.mark.parametrize("s", [0.7, 1.0, 1.5, 2.0, 3.0, 6.0])
def test_kernels_normalised_and_match_scipy(s):
    w, c = O.kernels(s)
    R = O.radius(s)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(w, w[::-1])
    np.testing.assert_array_equal(c, -c[::-1])
    assert c[R] == 0.0
    # scipy's Gaussian: response of a unit impulse (weights of the same sampled kernel)
    delta = np.zeros(4 * R + 1)
    delta[2 * R] = 1.0
    ref = ndi.gaussian_filter1d(delta, s, order=0, mode="constant", truncate=4.0)[R:3 * R + 1]
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-16)
    # scipy order=1 is convolution with the derivative of the sampled Gaussian;
    # the oracle's taps are the equivalent correlation taps.
    ref1 = ndi.gaussian_filter1d(delta, s, order=1, mode="constant", truncate=4.0)[R:3 * R + 1]
    np.testing.assert_allclose(c, ref1[::-1], rtol=0, atol=1e-16)


def _scipy_gradient(vol, s):
    v = vol.astype(np.float64)
    gx = ndi.gaussian_filter(v, s, order=(0, 0, 1), mode="nearest", truncate=4.0)
    gy = ndi.gaussian_filter(v, s, order=(0, 1, 0), mode="nearest", truncate=4.0)
    gz = ndi.gaussian_filter(v, s, order=(1, 0, 0), mode="nearest", truncate=4.0)
    return np.stack([gx, gy, gz])


def _scipy_tensor(vol, s, r):
    g = _scipy_gradient(vol, s)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    return np.stack([ndi.gaussian_filter(g[a] * g[b], r, mode="nearest", truncate=4.0) for a, b in pairs])


@pytest.mark.parametrize("shape,s", [((16, 18, 20), 1.0), ((13, 21, 17), 1.5), ((9, 10, 30), 2.0)])
def test_gradient_matches_scipy(shape, s):
    vol = RNG.integers(0, 4000, size=shape, dtype=np.uint16)
    g = O.gradient(vol, s)
    ref = _scipy_gradient(vol, s)
    scale = np.abs(ref).max()
    assert np.abs(g - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("shape,s,r", [((16, 18, 20), 1.0, 3.0), ((20, 14, 22), 1.5, 2.0), ((12, 12, 40), 1.0, 6.0)])
def test_structure_tensor_matches_scipy(shape, s, r):
    vol = RNG.integers(0, 4000, size=shape, dtype=np.uint16)
    S = O.structure_tensor(vol, s, r)
    ref = _scipy_tensor(vol, s, r)
    scale = np.abs(ref).max()
    assert np.abs(S - ref).max() <= 1e-11 * scale


def _brute_gradient(vol, s):
    """Direct triple sum with per-axis clamping, from the exp definition (numpy only)."""
    nz, ny, nx = vol.shape
    R = int(np.floor(4 * s + 0.5))
    k = np.arange(-R, R + 1)
    w = np.exp(-k * k / (2 * s * s))
    w /= w.sum()
    c = k / (s * s) * w
    v = vol.astype(np.float64)
    out = np.zeros((3,) + vol.shape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                zi = np.clip(z + k, 0, nz - 1)
                yi = np.clip(y + k, 0, ny - 1)
                xi = np.clip(x + k, 0, nx - 1)
                blk = v[np.ix_(zi, yi, xi)]
                out[0, z, y, x] = np.einsum("i,j,k,ijk->", w, w, c, blk)
                out[1, z, y, x] = np.einsum("i,j,k,ijk->", w, c, w, blk)
                out[2, z, y, x] = np.einsum("i,j,k,ijk->", c, w, w, blk)
    return out


def _brute_smooth(f, s):
    nz, ny, nx = f.shape
    R = int(np.floor(4 * s + 0.5))
    k = np.arange(-R, R + 1)
    w = np.exp(-k * k / (2 * s * s))
    w /= w.sum()
    out = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                blk = f[np.ix_(np.clip(z + k, 0, nz - 1), np.clip(y + k, 0, ny - 1), np.clip(x + k, 0, nx - 1))]
                out[z, y, x] = np.einsum("i,j,k,ijk->", w, w, w, blk)
    return out


def test_brute_force_triple_sum_tiny():
    # radii (4 and 6) exceed half the box: heavy clamping on every axis
    vol = RNG.integers(0, 3000, size=(7, 8, 9), dtype=np.uint16)
    s, r = 1.0, 1.5
    g = O.gradient(vol, s)
    gb = _brute_gradient(vol, s)
    assert np.abs(g - gb).max() <= 1e-12 * np.abs(gb).max()
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    Sb = np.stack([_brute_smooth(gb[a] * gb[b], r) for a, b in pairs])
    S = O.structure_tensor(vol, s, r)
    assert np.abs(S - Sb).max() <= 1e-11 * np.abs(Sb).max()


def test_box_equals_whole_bit_exact():
    # padded chunks reproduce the whole-volume result exactly (Implementation)
    vol = RNG.integers(0, 4000, size=(30, 26, 28), dtype=np.uint16)
    s, r = 1.0, 2.0
    S = O.structure_tensor(vol, s, r)
    g = O.gradient(vol, s)
    for lo, n in [((0, 0, 0), (5, 6, 7)), ((10, 3, 20), (9, 11, 10)), ((23, 20, 25), (5, 6, 5)), ((4, 4, 4), (1, 1, 1))]:
        Sb = O.structure_tensor(vol, s, r, lo=lo, n=n)
        gb = O.gradient(vol, s, lo=lo, n=n)
        sl = (slice(None), slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
        np.testing.assert_array_equal(Sb, S[sl])
        np.testing.assert_array_equal(gb, g[sl])


@pytest.mark.parametrize("s", [1.0, 2.0])
def test_linear_ramp_closed_form(s):
    # I = 1000 + 7x: g = (7 * sum_k k^2 w_k / s^2, 0, 0) away from the x edges,
    # the discrete second moment computed here from the exp definition.
    nx = 60
    x = np.arange(nx)
    vol = np.broadcast_to((1000 + 7 * x).astype(np.uint16), (12, 11, nx)).copy()
    R = int(np.floor(4 * s + 0.5))
    k = np.arange(-R, R + 1)
    w = np.exp(-k * k / (2 * s * s))
    w /= w.sum()
    slope = 7.0 * np.sum(k * k * w) / (s * s)
    g = O.gradient(vol, s)
    inner = slice(R, nx - R)
    np.testing.assert_allclose(g[0][:, :, inner], slope, rtol=1e-13)
    assert np.all(g[1] == 0.0) and np.all(g[2] == 0.0)
    r = 1.5
    Rr = int(np.floor(4 * r + 0.5))
    S = O.structure_tensor(vol, s, r)
    inner2 = slice(R + Rr, nx - R - Rr)
    np.testing.assert_allclose(S[0][:, :, inner2], slope * slope, rtol=1e-12)
    assert np.all(S[1:] == 0.0)


def test_constant_volume_is_exactly_zero():
    vol = np.full((10, 12, 14), 1234, dtype=np.uint16)
    assert np.all(O.gradient(vol, 1.5) == 0.0)
    out = O.pipeline(vol, 1.0, 2.0, center=(6.5, 5.5, 4.5), axis=(0, 0, 1))
    assert np.all(out["S"] == 0.0)
    assert np.all(out["evals"] == 0.0)
    assert np.all(out["fa"] == 0.0)


def test_axis_flip_and_transpose_symmetry():
    vol = RNG.integers(0, 4000, size=(14, 16, 18), dtype=np.uint16)
    s, r = 1.0, 2.0
    S = O.structure_tensor(vol, s, r)
    tol = 1e-12 * np.abs(S).max()
    # mirror x: g_x changes sign -> S_xy, S_xz change sign, all fields mirrored
    Sf = O.structure_tensor(np.ascontiguousarray(vol[:, :, ::-1]), s, r)[:, :, :, ::-1]
    sign = np.array([1, 1, 1, -1, -1, 1])[:, None, None, None]
    assert np.abs(Sf - sign * S).max() <= tol
    # swap x and y: components permute (xx<->yy, xz<->yz)
    St = O.structure_tensor(np.ascontiguousarray(vol.transpose(0, 2, 1)), s, r).transpose(0, 1, 3, 2)
    perm = [1, 0, 2, 3, 5, 4]
    assert np.abs(St - S[perm]).max() <= tol
    # swap x and z
    St = O.structure_tensor(np.ascontiguousarray(vol.transpose(2, 1, 0)), s, r).transpose(0, 3, 2, 1)
    perm = [2, 1, 0, 5, 4, 3]
    assert np.abs(St - S[perm]).max() <= tol
