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


def track_one(vec, fa, mask, p, d, h, fa_min, max_turn_deg, max_steps) -> List[Tuple[float, float, float]]:
    """Points after the seed p, integrating from direction d."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    cos_turn = math.cos(math.radians(max_turn_deg))
    out = []
    for _ in range(max_steps):
        k1 = direction(vec, p, d)
        if k1 is None:
            break
        k2 = direction(vec, [p[a] + 0.5 * h * k1[a] for a in range(3)], k1)
        if k2 is None:
            break
        k3 = direction(vec, [p[a] + 0.5 * h * k2[a] for a in range(3)], k2)
        if k3 is None:
            break
        k4 = direction(vec, [p[a] + h * k3[a] for a in range(3)], k3)
        if k4 is None:
            break
        s = [k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a] for a in range(3)]
        n = math.sqrt(sum(e * e for e in s))
        if not (n > 0.0):
            break
        dn = [e / n for e in s]
        if dn[0] * d[0] + dn[1] * d[1] + dn[2] * d[2] < cos_turn:
            break
        q = [p[a] + (h / 6.0) * s[a] for a in range(3)]
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
           mask: Optional[np.ndarray] = None, fa_min: float = 0.0, max_turn_deg: float = 90.0):
    """[(forward points, backward points)] per seed, each list starting with the seed (empty when the
    seed is outside the volume)."""
    dims = (vec.shape[3], vec.shape[2], vec.shape[1])
    result = []
    for sd in seeds:
        p = [float(e) for e in sd]
        if any(not (0.0 <= p[a] <= dims[a] - 1) for a in range(3)):
            result.append(([], []))
            continue
        x, y, z = _nearest(p)
        ref = [float(vec[k, z, y, x]) for k in range(3)]
        d0 = direction(vec, p, ref) if all(math.isfinite(e) for e in ref) and any(ref) else None
        if d0 is None:
            result.append(([tuple(p)], [tuple(p)]))
            continue
        fwd = [tuple(p)] + track_one(vec, fa, mask, p, list(d0), h, fa_min, max_turn_deg, max_steps)
        bwd = [tuple(p)] + track_one(vec, fa, mask, p, [-e for e in d0], h, fa_min, max_turn_deg, max_steps)
        result.append((fwd, bwd))
    return result
