"""Pins of the oracle's eigen-solve and angle stages.

The fibre direction is the eigenvector of the smallest eigenvalue of the
structure tensor (Figure 1b); HA, IA and FA are read in a cylindrical
left-ventricle frame (Figure 1c).  Checked against LAPACK (numpy.linalg.eigh),
hand-derived golden fixtures, exact invariants (trace, orthonormality, rotation
covariance) and the analytic fibre field of the synthetic helix volume.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle as O
from paper_2508_07476_gb300 import synth

RNG = np.random.default_rng(777)


def _sym(s6):
    xx, yy, zz, xy, xz, yz = s6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def _s6(A):
    return np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])


def _rand_rotation():
    q, r = np.linalg.qr(RNG.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("row", read_golden("eig3.txt"))
def test_eig_golden(row):
    s6, lam, v1 = row[:6], np.array(row[6:9]), np.array(row[9:12])
    ev, V = O.eig3(s6)
    np.testing.assert_allclose(ev, lam, rtol=0, atol=1e-14 * max(1.0, np.abs(lam).max()))
    assert abs(abs(np.dot(V[0], v1)) - 1.0) < 1e-14


def test_eig_matches_lapack_and_invariants():
    for i in range(300):
        A = RNG.normal(size=(3, 3))
        A = A + A.T
        if i % 2 == 0:
            A = A @ A.T  # positive semi-definite, like a structure tensor
        ev, V = O.eig3(_s6(A))
        w, U = np.linalg.eigh(A)
        nrm = np.linalg.norm(A)
        np.testing.assert_allclose(ev, w, rtol=0, atol=1e-13 * nrm)
        assert abs(ev.sum() - np.trace(A)) <= 1e-13 * nrm
        np.testing.assert_allclose(V @ V.T, np.eye(3), atol=1e-14)
        for k in range(3):
            assert np.linalg.norm(A @ V[k] - ev[k] * V[k]) <= 1e-13 * nrm
        gap = min(w[1] - w[0], w[2] - w[1])
        if gap > 1e-6 * nrm:
            for k in range(3):
                assert abs(abs(np.dot(V[k], U[:, k])) - 1.0) < 1e-12 * (nrm / gap) ** 2 + 1e-14


def test_eig_rotation_covariance():
    for _ in range(100):
        lam = np.sort(RNG.uniform(0.1, 10.0, size=3))
        Q = _rand_rotation()
        A = Q @ np.diag(lam) @ Q.T
        ev, V = O.eig3(_s6(A))
        np.testing.assert_allclose(ev, lam, rtol=1e-13)
        assert abs(abs(np.dot(V[0], Q[:, 0])) - 1.0) < 1e-12
        R = _rand_rotation()
        ev2, V2 = O.eig3(_s6(R @ A @ R.T))
        np.testing.assert_allclose(ev2, ev, rtol=1e-13)
        assert abs(abs(np.dot(V2[0], R @ V[0])) - 1.0) < 1e-12


def test_eig_special_cases():
    ev, V = O.eig3([0, 0, 0, 0, 0, 0])
    assert np.all(ev == 0)
    np.testing.assert_allclose(V @ V.T, np.eye(3))
    # repeated largest pair: smallest eigenvector still unique (rod-like tensor)
    Q = _rand_rotation()
    A = Q @ np.diag([0.5, 4.0, 4.0]) @ Q.T
    ev, V = O.eig3(_s6(A))
    np.testing.assert_allclose(ev, [0.5, 4.0, 4.0], rtol=1e-13)
    assert abs(abs(np.dot(V[0], Q[:, 0])) - 1.0) < 1e-13


@pytest.mark.parametrize("row", read_golden("fa.txt"))
def test_fa_golden(row):
    assert abs(O.fa(row[:3]) - row[3]) < 1e-15


@pytest.mark.parametrize("row", read_golden("ha_ia.txt"))
def test_ha_ia_golden(row):
    p, c, a, v, ha, ia = row[0:3], row[3:6], row[6:9], row[9:12], row[12], row[13]
    h, i, vo = O.ha_ia(p, c, a, v)
    assert abs(h - ha) < 1e-12 and abs(i - ia) < 1e-12


def test_ha_ia_axis_sign_and_orientation():
    for _ in range(200):
        p = RNG.uniform(-50, 50, size=3)
        c = RNG.uniform(-5, 5, size=3)
        a = RNG.normal(size=3)
        v = RNG.normal(size=3)
        v /= np.linalg.norm(v)
        h1, i1, vo1 = O.ha_ia(p, c, a, v)
        h2, i2, vo2 = O.ha_ia(p, c, -a, v)
        h3, i3, vo3 = O.ha_ia(p, c, a, -v)
        # fibre sign is irrelevant; flipping the axis keeps HA and negates IA
        assert abs(h1 - h3) < 1e-12 and abs(i1 - i3) < 1e-12
        assert abs(h1 - h2) < 1e-9 and abs(i1 + i2) < 1e-9
        assert -90.0 < h1 <= 90.0 and -90.0 <= i1 <= 90.0
        # the reported angles rebuild the oriented vector in the frame
        ez = a / np.linalg.norm(a)
        d = p - c
        er = d - np.dot(d, ez) * ez
        er /= np.linalg.norm(er)
        et = np.cross(ez, er)
        H, I = math.radians(h1), math.radians(i1)
        rebuilt = math.sin(I) * er + math.cos(I) * (math.cos(H) * et + math.sin(H) * ez)
        np.testing.assert_allclose(rebuilt, vo1, atol=1e-12)


def test_on_axis_and_mask_fill():
    vol = RNG.integers(900, 1100, size=(9, 10, 11), dtype=np.uint16)
    mask = np.ones(vol.shape, dtype=np.uint8)
    mask[4, 5, :] = 0
    # axis along x through (any, 5, 4): voxels (x, 5, 4) lie on it
    out = O.pipeline(vol, 1.0, 1.5, center=(0.0, 5.0, 4.0), axis=(1.0, 0.0, 0.0), mask=mask, fill=-7.0)
    assert np.all(out["ha"][4, 5, :] == -7.0) and np.all(out["fa"][4, 5, :] == -7.0)
    assert np.all(out["v"][:, 4, 5, :] == -7.0)
    out = O.pipeline(vol, 1.0, 1.5, center=(0.0, 5.0, 4.0), axis=(1.0, 0.0, 0.0), fill=-7.0)
    assert np.all(out["ha"][4, 5, :] == -7.0) and np.all(out["ia"][4, 5, :] == -7.0)
    assert np.all(out["fa"][4, 5, :] != -7.0)
    assert np.all(out["ha"][3] != -7.0)


def test_helix_volume_recovers_fibre_direction():
    """Diagnostic: on the 64^3 helix volume the oracle's fibre field follows the
    analytic rods (few degrees, limited by the grating's blending seams)."""
    W = synth.single_chunk_64()
    vol, _ = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    out = O.pipeline(vol, W.sigma, W.rho, cen, ax)
    z, y, x = np.meshgrid(*[np.arange(k, dtype=float) for k in vol.shape], indexing="ij")
    f0 = synth.truth_fibre(W.spec, x, y, z)
    ang = np.degrees(np.arccos(np.clip(np.abs((np.moveaxis(out["v"], 0, -1) * f0).sum(-1)), 0, 1)))
    r = np.hypot(x - cen[0], y - cen[1])
    R = O.radius(W.sigma) + O.radius(W.rho)
    core = (r > W.spec.r_in + 3) & (r < W.spec.r_out - 3)
    core[:R] = core[-R:] = False
    assert np.median(ang[core]) < 5.0
    assert np.percentile(ang[core], 90) < 10.0
    # HA follows the transmural ramp +60 -> -60 (inner -> outer)
    ha = out["ha"][core]
    t = (r[core] - W.spec.r_in) / (W.spec.r_out - W.spec.r_in)
    ha_true = W.spec.ha_in_deg + t * (W.spec.ha_out_deg - W.spec.ha_in_deg)
    dha = np.abs((ha - ha_true + 90.0) % 180.0 - 90.0)
    assert np.median(dha) < 5.0
