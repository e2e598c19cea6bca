"""FP64 transmural HA profile of the oracle's outputs.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by tests
and the benchmark, never by the library.

The paper's analysis module plots the helical angle against depth through
the wall from the HA map of Figure 1(c); the statistic is this histogram:

- depth d = (r - r_in) / (r_out - r_in), where r is the distance of the
  voxel centre from the axis line through ``center`` along ``axis``;
- a voxel counts when it is inside the mask (if any), its HA is finite and
  0 <= d < 1;
- hist[floor(d * n_depth), clamp(floor((HA + 90) * n_ha / 180))] += 1.

``transmural_profile`` evaluates that definition in FP64 with numpy;
``transmural_profile_loops`` is the same definition voxel by voxel in plain
Python, kept as the brute-force check for small inputs.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np


def _frame(center, axis):
    c = np.asarray(center, dtype=np.float64)
    a = np.asarray(axis, dtype=np.float64)
    return c, a / np.linalg.norm(a)


def depth_field(shape_zyx, lo, center, axis, r_in: float, r_out: float) -> np.ndarray:
    """Normalised wall depth of every voxel of the box (lo = (x, y, z), shape [z, y, x])."""
    c, a = _frame(center, axis)
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz) + lo[2], np.arange(ny) + lo[1], np.arange(nx) + lo[0], indexing="ij")
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    h = dx * a[0] + dy * a[1] + dz * a[2]
    r = np.sqrt((dx - h * a[0]) ** 2 + (dy - h * a[1]) ** 2 + (dz - h * a[2]) ** 2)
    return (r - r_in) / (r_out - r_in)


def transmural_profile(ha: np.ndarray, mask: Optional[np.ndarray], lo: Sequence[int], center, axis, r_in: float,
                       r_out: float, n_depth: int, n_ha: int) -> np.ndarray:
    """uint64 [n_depth, n_ha] histogram of HA (degrees, array [z, y, x] over the box at lo)."""
    d = depth_field(ha.shape, lo, center, axis, r_in, r_out)
    h = ha.astype(np.float64)
    keep = np.isfinite(h) & (d >= 0.0) & (d < 1.0)
    if mask is not None:
        keep &= mask.astype(bool)
    kd = np.minimum(np.floor(d[keep] * n_depth).astype(np.int64), n_depth - 1)
    kh = np.clip(np.floor((h[keep] + 90.0) * n_ha / 180.0).astype(np.int64), 0, n_ha - 1)
    out = np.zeros((n_depth, n_ha), dtype=np.uint64)
    np.add.at(out, (kd, kh), 1)
    return out


def transmural_profile_loops(ha, mask, lo, center, axis, r_in, r_out, n_depth, n_ha):
    """The definition voxel by voxel (small inputs only)."""
    c, a = _frame(center, axis)
    out = np.zeros((n_depth, n_ha), dtype=np.uint64)
    nz, ny, nx = ha.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if mask is not None and not mask[k, j, i]:
                    continue
                v = float(ha[k, j, i])
                if not math.isfinite(v):
                    continue
                p = (i + lo[0] - c[0], j + lo[1] - c[1], k + lo[2] - c[2])
                t = p[0] * a[0] + p[1] * a[1] + p[2] * a[2]
                r = math.sqrt(sum((p[q] - t * a[q]) ** 2 for q in range(3)))
                d = (r - r_in) / (r_out - r_in)
                if not (0.0 <= d < 1.0):
                    continue
                kd = min(int(math.floor(d * n_depth)), n_depth - 1)
                kh = min(max(int(math.floor((v + 90.0) * n_ha / 180.0)), 0), n_ha - 1)
                out[kd, kh] += 1
    return out
