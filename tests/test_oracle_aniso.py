"""Pins of the oracle's anisotropic form: voxel spacing (sx, sy, sz), with
sigma, rho, centre and axis in its units, and a per-slice LV centreline."""
import numpy as np
import pytest

from oracle import oracle
from paper_2508_07476_gb300 import synth


@pytest.fixture(scope="module")
def vol():
    W = synth.single_chunk_64()
    v, _ = synth.generate(W.spec)
    return W, v[8:40, 10:50, 12:56].copy()  # uneven axes


def _angle(u, v):
    """Angle between orientations (degrees), from the cross and dot products."""
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, v, axis=0), axis=0), np.abs((u * v).sum(0))))


def test_unit_spacing_is_the_isotropic_pipeline(vol):
    W, v = vol
    c, a = (20.0, 18.0, 15.0), (0.1, 0.0, 1.0)
    iso = oracle.pipeline(v, 1.0, 2.5, c, a)
    uni = oracle.pipeline(v, 1.0, 2.5, c, a, spacing=(1.0, 1.0, 1.0))
    for k in iso:
        np.testing.assert_array_equal(iso[k], uni[k])


def test_uniform_spacing_is_a_change_of_units(vol):
    """Spacing s with sigma, rho and centre scaled by s: the same voxel-unit
    kernels, S divided by s^2, identical directions and angles."""
    W, v = vol
    c, a = (20.0, 18.0, 15.0), (0.1, 0.0, 1.0)
    base = oracle.pipeline(v, 1.0, 2.5, c, a)
    s = 2.0
    sc = oracle.pipeline(v, s * 1.0, s * 2.5, tuple(s * e for e in c), a, spacing=(s, s, s))
    np.testing.assert_allclose(sc["S"] * s * s, base["S"], rtol=1e-12, atol=1e-12 * np.abs(base["S"]).max())
    for k in ("ha", "ia", "fa"):
        np.testing.assert_allclose(sc[k], base[k], atol=1e-9, equal_nan=True)
    assert _angle(sc["v"], base["v"]).max() < 1e-6


def test_axis_permutation_permutes_the_result(vol):
    """Swapping the x and z axes of the volume together with the spacing, the
    centre and the axis permutes the tensor and the fibre direction."""
    W, v = vol
    sp, c, a = (1.0, 1.5, 0.75), (20.0, 27.0, 12.0), (0.2, 0.1, 1.0)
    r1 = oracle.pipeline(v, 1.5, 3.0, c, a, spacing=sp)
    vt = np.ascontiguousarray(v.transpose(2, 1, 0))
    r2 = oracle.pipeline(vt, 1.5, 3.0, c[::-1], a[::-1], spacing=sp[::-1])
    S2 = r2["S"].transpose(0, 3, 2, 1)  # back to the first volume's [z, y, x]
    perm = [2, 1, 0, 5, 4, 3]  # (xx, yy, zz, xy, xz, yz) with x <-> z
    np.testing.assert_allclose(S2[perm], r1["S"], rtol=1e-9, atol=1e-9 * np.abs(r1["S"]).max())
    v2 = r2["v"].transpose(0, 3, 2, 1)[::-1]
    np.testing.assert_allclose(r2["fa"].transpose(2, 1, 0), r1["fa"], atol=1e-9)
    ok = r1["fa"] > 0.1
    assert _angle(v2[:, ok], r1["v"][:, ok]).max() < 1e-6


def test_ramp_gradient_is_in_physical_units():
    """I = 2 x + 6 z (voxel indices) on spacing (0.5, 1, 2) is the physical
    ramp 4 X + 3 Z.  Away from the edges S is rank one: S_ab = G_a G_b with
    G_a = (ramp slope) times the kernel's unit-slope response sum_k k c_k at
    scale sigma / s_a (derivative taps applied to a unit ramp)."""
    nz, ny, nx = 24, 12, 64
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = (1000 + 2 * x + 6 * z).astype(np.uint16)
    sp, sigma, rho = (0.5, 1.0, 2.0), 1.0, 2.0
    r = oracle.pipeline(v, sigma, rho, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), spacing=sp)

    def unit_slope(s):
        _, c = oracle.kernels(s)
        k = np.arange(len(c)) - (len(c) - 1) // 2
        return float((k * c).sum())

    G = np.array([4.0 * unit_slope(sigma / sp[0]), 0.0, 3.0 * unit_slope(sigma / sp[2])])
    want = [G[0] * G[0], 0.0, G[2] * G[2], 0.0, G[0] * G[2], 0.0]
    core = r["S"][:, 7:17, :, 25:39]  # beyond R(sigma)+R(rho) (z: 2+4, x: 8+16) of the clamped edges
    for k in range(6):
        np.testing.assert_allclose(core[k], want[k], rtol=1e-9, atol=1e-9 * G[0] * G[0])


def test_centreline_gives_each_slice_its_own_centre():
    """v = e_theta about a centre that moves from slice to slice: with that
    centreline HA and IA are 0 everywhere off the axis; a constant centreline
    equals the fixed centre."""
    nz, ny, nx = 6, 20, 22
    sp = (1.0, 1.0, 1.5)
    cen = np.array([[9.3 + 0.4 * k, 10.1 - 0.3 * k] for k in range(nz)])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx, dy = x * sp[0] - cen[z, 0], y * sp[1] - cen[z, 1]
    r = np.hypot(dx, dy)
    v1 = np.stack([-dy / r, dx / r, np.zeros_like(r)])
    ev = np.stack([np.ones_like(r), 2 * np.ones_like(r), 3 * np.ones_like(r)])
    _, ha, ia, _ = oracle.angles_field(v1, ev, (nx, ny, nz), (0, 0, 0), (nx, ny, nz), (0.0, 0.0, 0.0),
                                       (0.0, 0.0, 1.0), spacing=sp, centres=cen)
    assert np.nanmax(np.abs(ha)) < 1e-9 and np.nanmax(np.abs(ia)) < 1e-9
    const = np.tile([[9.3, 10.1]], (nz, 1))
    a1 = oracle.angles_field(v1, ev, (nx, ny, nz), (0, 0, 0), (nx, ny, nz), (9.3, 10.1, 0.0), (0.0, 0.0, 1.0),
                             spacing=sp)
    a2 = oracle.angles_field(v1, ev, (nx, ny, nz), (0, 0, 0), (nx, ny, nz), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0),
                             spacing=sp, centres=const)
    for p, q in zip(a1, a2):
        np.testing.assert_allclose(p, q, atol=1e-12, equal_nan=True)
