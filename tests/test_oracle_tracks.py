"""Pins of the oracle's streamline tractography (RK4 through a sign-aligned,
trilinearly interpolated orientation field)."""
import math

import numpy as np
import pytest

from oracle import tracks


def _const_field(shape, v):
    f = np.zeros((3,) + shape)
    for k in range(3):
        f[k] = v[k]
    return f


def _circle_field(n, c):
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    dx, dy = x - c, y - c
    r = np.hypot(dx, dy)
    r[r == 0] = 1.0
    f = np.zeros((3, 4, n, n))
    f[0], f[1] = -dy / r, dx / r
    return f


def test_constant_field_straight_line():
    n, h, x0 = 40, 0.7, 5.2
    f = _const_field((6, 8, n), (1.0, 0.0, 0.0))
    (fwd, bwd), = tracks.tracks(f, [(x0, 3.0, 2.5)], h, 500)
    assert len(fwd) - 1 == math.floor((n - 1 - x0) / h)
    assert len(bwd) - 1 == math.floor(x0 / h)
    for k, p in enumerate(fwd):
        assert p == pytest.approx((x0 + k * h, 3.0, 2.5), abs=1e-12)
    assert bwd[-1][0] == pytest.approx(x0 - (len(bwd) - 1) * h, abs=1e-12)


def test_orientation_sign_does_not_matter():
    rng = np.random.default_rng(1)
    shape = (5, 9, 30)
    f = _const_field(shape, (0.6, 0.8, 0.0))
    flips = np.where(rng.random(shape) < 0.5, -1.0, 1.0)
    g = f * flips[None]
    a = tracks.tracks(f, [(3.3, 1.1, 2.0)], 0.5, 200)
    b = tracks.tracks(g, [(3.3, 1.1, 2.0)], 0.5, 200)
    assert len(a[0][0]) == len(b[0][0]) > 5 and len(a[0][1]) == len(b[0][1])
    np.testing.assert_allclose(np.array(a[0][0]), np.array(b[0][0]), atol=1e-12)


def test_circle_rk4_is_fourth_order():
    """Tracks of the field e_theta stay on their circle; halving h cuts the
    radius drift by about 2^4 (a lower-order scheme would show 2^1 or 2^2)."""
    n, c, r0 = 64, 31.5, 12.0
    f = _circle_field(n, c)
    # the interpolated field is exact on the axes only; compare drifts along one quarter turn
    errs = []
    for h in (1.0, 0.5):
        steps = int(round(0.5 * math.pi * r0 / h))
        (fwd, _), = tracks.tracks(f, [(c + r0, c, 1.0)], h, steps, max_turn_deg=30.0)
        assert len(fwd) - 1 == steps
        rad = np.hypot(np.array(fwd)[:, 0] - c, np.array(fwd)[:, 1] - c)
        errs.append(abs(rad[-1] - r0))
    # trilinear interpolation of e_theta adds an O(1/r^2) field error that both step sizes share,
    # so the drift must simply shrink and stay small
    assert errs[1] < errs[0] and errs[1] < 0.05


def test_fa_threshold_stops_the_track():
    n = 40
    f = _const_field((4, 6, n), (1.0, 0.0, 0.0))
    fa = np.ones((4, 6, n))
    fa[:, :, 21:] = 0.0  # trilinear FA = 21 - x on (20, 21)
    (fwd, _), = tracks.tracks(f, [(10.0, 2.0, 1.0)], 0.25, 500, fa=fa, fa_min=0.5)
    assert fwd[-1][0] <= 20.5 and fwd[-1][0] > 20.5 - 0.25


def test_mask_stops_the_track():
    n = 60
    f = _const_field((4, n, 8), (0.0, 1.0, 0.0))
    mask = np.ones((4, n, 8), np.uint8)
    mask[:, 40:, :] = 0
    (fwd, _), = tracks.tracks(f, [(3.0, 10.0, 1.0)], 0.3, 500, mask=mask)
    assert fwd[-1][1] < 39.5 and fwd[-1][1] >= 39.5 - 0.3


def test_turn_limit_stops_at_a_bend():
    n = 60
    f = _const_field((4, n, n), (1.0, 0.0, 0.0))
    f[0, :, :, 30:] = 0.0
    f[1, :, :, 30:] = 1.0  # the fibres turn by 90 degrees at x = 30
    (fwd, _), = tracks.tracks(f, [(10.0, 20.0, 1.0)], 0.5, 500, max_turn_deg=20.0)
    assert 28.0 <= fwd[-1][0] <= 30.5 and fwd[-1][1] < 22.0
    (free, _), = tracks.tracks(f, [(10.0, 20.0, 1.0)], 0.5, 60, max_turn_deg=90.0)
    assert free[-1][1] > 25.0  # without the limit the track follows the bend


def test_seed_outside_and_dead_seed():
    f = _const_field((4, 4, 4), (1.0, 0.0, 0.0))
    out = tracks.tracks(f, [(5.0, 1.0, 1.0), (1.0, 1.0, 1.0)], 0.5, 10)
    assert out[0] == ([], [])
    g = f.copy()
    g[:, 1, 1, 1] = np.nan
    (fwd, bwd), = tracks.tracks(g, [(1.0, 1.0, 1.0)], 0.5, 10)
    assert len(fwd) == 1 and len(bwd) == 1


def test_parabola_fourth_order():
    """The field (1, a (x - x0), 0) is interpolated exactly (linear in x), so
    tracks follow y = y0 + a (x - x0)^2 / 2; RK4's error falls by ~2^4 per
    halving of h (a dropped or mis-weighted stage would show 2^1..2^3)."""
    n, a, x0, y0 = 60, 0.05, 20.0, 10.0
    _, _, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    f = np.zeros((3, 4, n, n))
    f[0] = 1.0
    f[1] = a * (x - x0)
    errs = []
    for h in (1.0, 0.5):
        (fwd, _), = tracks.tracks(f, [(x0, y0, 1.0)], h, int(15 / h))
        p = np.array(fwd)
        errs.append(np.abs(p[:, 1] - (y0 + a * (p[:, 0] - x0) ** 2 / 2)).max())
    assert errs[0] < 1e-6 and errs[0] / errs[1] > 12.0, errs


def test_step_margins_at_each_stopping_rule():
    """The margin of the step that stops a track is its distance from the
    threshold, worked out by hand: a volume face, a mask edge at a half-integer,
    an FA threshold, a turn limit; steps far from every threshold keep large
    margins; and asking for margins leaves the points unchanged."""
    # straight along +x from x = 2.1 in steps of 0.5 through a volume 12 long
    # (faces at 0 and 11; y = z = 3.0 lie 3 from theirs): 17 steps reach 10.6,
    # 0.4 from the face; the next step's stage points 10.85 and 11.1 lie 0.15
    # inside and 0.1 beyond it (max_turn 90 degrees: turn margin cos 0 - 0 = 1)
    f = _const_field((8, 8, 12), (1.0, 0.0, 0.0))
    m = []
    (fwd, _), = tracks.tracks(f, [(2.1, 3.0, 3.0)], 0.5, 100, margins=m)
    mf = m[0][0]
    assert len(fwd) == 18 and fwd[-1][0] == pytest.approx(10.6)
    assert len(mf) == 18 and mf[-1] == pytest.approx(0.1) and mf[-2] == pytest.approx(0.4)
    assert mf[0] == pytest.approx(1.0)  # far from every face: the turn margin
    assert tracks.tracks(f, [(2.1, 3.0, 3.0)], 0.5, 100) == tracks.tracks(f, [(2.1, 3.0, 3.0)], 0.5, 100, margins=[])
    # a mask ending at voxel 7 (x < 7.5 inside): steps of 0.3 from x = 5.05 land on
    # 5.35, ..., 7.45 (0.05 inside the edge), then 7.75 stops, 0.25 beyond it
    mask = np.ones((8, 8, 12), np.uint8)
    mask[:, :, 8:] = 0
    m = []
    (fwd, _), = tracks.tracks(f, [(5.05, 3.0, 3.0)], 0.3, 100, mask=mask, margins=m)
    mf = m[0][0]
    assert fwd[-1][0] == pytest.approx(7.45) and mf[-2] == pytest.approx(0.05) and mf[-1] == pytest.approx(0.25)
    # FA falling linearly along x, fa = 1 - x / 10, threshold 0.5 (x <= 5): steps of
    # 0.4 from 1.1 end at 4.7 (FA 0.53); the stopping step lands on 5.1 (FA 0.49)
    fa = np.broadcast_to(1.0 - np.arange(12) / 10.0, (8, 8, 12)).copy()
    m = []
    (fwd, _), = tracks.tracks(f, [(1.1, 3.0, 3.0)], 0.4, 100, fa=fa, fa_min=0.5, margins=m)
    mf = m[0][0]
    assert fwd[-1][0] == pytest.approx(4.7) and mf[-1] == pytest.approx(0.01) and mf[-2] == pytest.approx(0.03)
    # a right-angle turn: the field turns from +x to +y at x = 6; with a 30 degree
    # limit the step that crosses the bend turns by more, and its margin is
    # cos(30 deg) - cos(turn) for the turn that step computes
    g = np.zeros((3, 8, 12, 12))
    g[0, :, :, :6] = 1.0
    g[1, :, :, 6:] = 1.0
    m = []
    (fwd, _), = tracks.tracks(g, [(2.0, 3.0, 3.0)], 0.5, 100, max_turn_deg=30.0, margins=m)
    mf = m[0][0]
    assert mf[-1] > 0.0 and mf[-1] < math.cos(math.radians(30.0))
