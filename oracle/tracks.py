"""FP64 streamline tractography through a fibre field, voxel by voxel.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by tests
and the benchmark, never by the library.

The paper's tractography module traces cardiomyocyte trajectories through
the orientation field (Figure 1(d)) without stating a scheme; this is the
textbook one, in plain Python, one track at a time:

- dir(q; r): the 8 vectors of q's interpolation cell (corner
  i0 = min(floor(q), n - 2) per axis), each negated when it points against
  the reference direction r, weighted trilinearly, summed and normalised.
  Invalid when q is outside [0, n-1] on an axis, a corner vector is not
  finite, or the sum vanishes.
- one step from p along d (classical Runge-Kutta, 4th order):
  k1 = dir(p; d), k2 = dir(p + h/2 k1; k1), k3 = dir(p + h/2 k2; k2),
  k4 = dir(p + h k3; k3), p' = p + h (k1 + 2 k2 + 2 k3 + k4) / 6, and the new
  direction d' = normalise(k1 + 2 k2 + 2 k3 + k4).
- the track stops before p' when a direction is invalid, d' turns from d by
  more than max_turn_deg, p' is outside the volume, the mask is 0 at the
  nearest voxel floor(p' + 1/2), or trilinear FA at p' is not >= fa_min.
- two tracks per seed: forward along dir(seed; v at the nearest voxel),
  backward along its negation.  Point 0 of each is the seed.

Fields are numpy arrays ``vec[3, z, y, x]``, ``fa[z, y, x]``,
``mask[z, y, x]``; points are (x, y, z) in voxel units.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


def _cell(q, dims):
    """(corner, fractions) of q's interpolation cell, or None outside the volume."""
    i0, t = [], []
    for a in range(3):
        if not (0.0 <= q[a] <= dims[a] - 1):
            return None
        c = min(int(math.floor(q[a])), dims[a] - 2)
        i0.append(c)
        t.append(q[a] - c)
    return i0, t


def _corners(i0, t):
    for c in range(2):
        for b in range(2):
            for a in range(2):
                w = (t[0] if a else 1.0 - t[0]) * (t[1] if b else 1.0 - t[1]) * (t[2] if c else 1.0 - t[2])
                yield (i0[0] + a, i0[1] + b, i0[2] + c), w


def direction(vec: np.ndarray, q, ref) -> Optional[Tuple[float, float, float]]:
    """dir(q; ref) as defined in the module docstring (None when invalid)."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    cell = _cell(q, dims)
    if cell is None:
        return None
    s = [0.0, 0.0, 0.0]
    for (x, y, z), w in _corners(*cell):
        u = [float(vec[0, z, y, x]), float(vec[1, z, y, x]), float(vec[2, z, y, x])]
        if not all(math.isfinite(e) for e in u):
            return None
        if u[0] * ref[0] + u[1] * ref[1] + u[2] * ref[2] < 0.0:
            u = [-e for e in u]
        for a in range(3):
            s[a] += w * u[a]
    n = math.sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2])
    if not (n > 0.0):
        return None
    return (s[0] / n, s[1] / n, s[2] / n)


def trilinear(field: np.ndarray, q) -> float:
    dims = (field.shape[2], field.shape[1], field.shape[0])
    cell = _cell(q, dims)
    if cell is None:
        return float("nan")
    return sum(w * float(field[z, y, x]) for (x, y, z), w in _corners(*cell))


def _nearest(q):
    return tuple(int(math.floor(e + 0.5)) for e in q)


# ---------------------------------------------------------------- margins
# How far one step is from flipping a stopping decision: every test of a step
# compares a rounded quantity with a threshold (a coordinate with the volume's
# faces, with the integer grid that picks an interpolation cell or with the
# half-integers that pick the nearest voxel, a cosine with cos(max_turn), an FA
# with fa_min).  A track computed in another precision may take a decision the
# other way only where that distance is within its rounding; these functions
# report the distance (voxels, cosine or FA units) so that a test can check it.

def _cell_ok(vec, i0) -> bool:
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    if any(not (0 <= i0[a] <= dims[a] - 2) for a in range(3)):
        return False
    for (x, y, z), _ in _corners(i0, (0.0, 0.0, 0.0)):
        if not all(math.isfinite(float(vec[k, z, y, x])) for k in range(3)):
            return False
    return True


def _point_margin(vec, q) -> float:
    """Distance of q from a change of its direction's validity: a volume face,
    or a grid line beyond which the interpolation cell's validity differs."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    m = min(abs(min(q[a], dims[a] - 1 - q[a])) for a in range(3))
    if any(not (0.0 <= q[a] <= dims[a] - 1) for a in range(3)):
        return m
    i0 = [min(int(math.floor(q[a])), dims[a] - 2) for a in range(3)]
    ok = _cell_ok(vec, i0)
    for a in range(3):
        for side in (-1, 1):
            j = list(i0)
            j[a] += side
            if 0 <= j[a] <= dims[a] - 2 and _cell_ok(vec, j) != ok:
                m = min(m, abs(q[a] - (i0[a] if side < 0 else i0[a] + 1)))
    return m


def _mask_margin(mask, q) -> float:
    """Distance of q from a half-integer across which the nearest voxel's mask changes."""
    if mask is None:
        return math.inf
    n = _nearest(q)
    dims = (mask.shape[2], mask.shape[1], mask.shape[0])
    m = math.inf
    for a in range(3):
        f = q[a] - math.floor(q[a])
        alt = list(n)  # the voxel across the half-integer floor(q) + 1/2, the nearer one
        alt[a] += -1 if f >= 0.5 else 1
        if 0 <= alt[a] < dims[a] and 0 <= n[a] < dims[a] and mask[alt[2], alt[1], alt[0]] != mask[n[2], n[1], n[0]]:
            m = min(m, abs(f - 0.5))
    return m


def track_one(vec, fa, mask, p, d, h, fa_min, max_turn_deg, max_steps,
              margins: Optional[list] = None) -> List[Tuple[float, float, float]]:
    """Points after the seed p, integrating from direction d.  With `margins`
    (a list), the smallest margin of every step attempted (taken or the one
    that stopped the track) is appended to it."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    cos_turn = math.cos(math.radians(max_turn_deg))
    out = []
    for _ in range(max_steps):
        m = math.inf
        ks, ok = [], True
        q_stage, ref = p, d
        for frac in (0.0, 0.5, 0.5, 1.0):
            if ks:
                q_stage = [p[a] + frac * h * ks[-1][a] for a in range(3)]
            if margins is not None:
                m = min(m, _point_margin(vec, q_stage))
            k = direction(vec, q_stage, ks[-1] if ks else ref)
            if k is None:
                ok = False
                break
            ks.append(k)
        if not ok:
            if margins is not None:
                margins.append(m)
            break
        k1, k2, k3, k4 = ks
        s = [k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a] for a in range(3)]
        n = math.sqrt(sum(e * e for e in s))
        if not (n > 0.0):
            if margins is not None:
                margins.append(0.0)
            break
        dn = [e / n for e in s]
        q = [p[a] + (h / 6.0) * s[a] for a in range(3)]
        if margins is not None:
            m = min(m, abs(dn[0] * d[0] + dn[1] * d[1] + dn[2] * d[2] - cos_turn),
                    min(abs(min(q[a], dims[a] - 1 - q[a])) for a in range(3)), _mask_margin(mask, q))
            if fa is not None and all(0.0 <= q[a] <= dims[a] - 1 for a in range(3)):
                m = min(m, abs(trilinear(fa, q) - fa_min))
            margins.append(m)
        if dn[0] * d[0] + dn[1] * d[1] + dn[2] * d[2] < cos_turn:
            break
        if any(not (0.0 <= q[a] <= dims[a] - 1) for a in range(3)):
            break
        if mask is not None:
            x, y, z = _nearest(q)
            if mask[z, y, x] == 0:
                break
        if fa is not None and not (trilinear(fa, q) >= fa_min):
            break
        out.append(tuple(q))
        p, d = q, dn
    return out


def tracks(vec: np.ndarray, seeds: Sequence[Sequence[float]], h: float, max_steps: int, fa: Optional[np.ndarray] = None,
           mask: Optional[np.ndarray] = None, fa_min: float = 0.0, max_turn_deg: float = 90.0,
           margins: Optional[list] = None):
    """[(forward points, backward points)] per seed, each list starting with the seed (empty when the
    seed is outside the volume).  With `margins` (a list), ([forward step margins], [backward step
    margins]) is appended per seed (see track_one)."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    result = []
    for sd in seeds:
        p = [float(e) for e in sd]
        mf, mb = [], []
        if margins is not None:
            margins.append((mf, mb))
        if any(not (0.0 <= p[a] <= dims[a] - 1) for a in range(3)):
            result.append(([], []))
            continue
        x, y, z = _nearest(p)
        ref = [float(vec[k, z, y, x]) for k in range(3)]
        d0 = direction(vec, p, ref) if all(math.isfinite(e) for e in ref) and any(ref) else None
        if d0 is None:
            result.append(([tuple(p)], [tuple(p)]))
            continue
        keep = margins is not None
        fwd = [tuple(p)] + track_one(vec, fa, mask, p, list(d0), h, fa_min, max_turn_deg, max_steps,
                                     mf if keep else None)
        bwd = [tuple(p)] + track_one(vec, fa, mask, p, [-e for e in d0], h, fa_min, max_turn_deg, max_steps,
                                     mb if keep else None)
        result.append((fwd, bwd))
    return result
