"""Seeded synthetic heart-wall volumes.

The method is applied to whole- or partial-heart scans with an optional
myocardial mask (Figure 1a) whose fibres wind helically through the wall, the
helical angle changing from endocardium to epicardium (Figure 1b,c).  No scan
ships with this library, so every volume used by the tests and the benchmark is
made here from a seed: a cylindrical annulus (the left-ventricle wall) filled
with a rod-like grating whose rods run along the local helix direction.

This module is the only code shared by the CUDA path and the CPU oracle, and it
holds none of the method's arithmetic (no filtering, no tensor, no eigen-solve,
no angle extraction).  It draws every random number from a counter-based
generator (SplitMix64 of Steele, Lea & Flood 2014, keyed by seed and voxel
index), so a volume depends only on its spec, never on how it is sliced.

Layout: ``vol[z, y, x]`` uint16, x fastest; positions are voxel-index units.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the finaliser of Steele, Lea & Flood 2014)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _MIX1
        z ^= z >> np.uint64(27)
        z *= _MIX2
        z ^= z >> np.uint64(31)
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x632BE59BD9B4E019 + stream * 0x8CB92BA72F3D8DD7) & _M64], dtype=np.uint64)
    return _mix64(s)[0]


def uniform01(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Uniform in (0, 1) from SplitMix64 at position ``counter`` of the (seed, stream) sequence."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        x = key + (counter.astype(np.uint64) + np.uint64(1)) * _GAMMA
    bits = _mix64(x) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Standard normal by Box-Muller from two uniforms per counter."""
    c = counter.astype(np.uint64)
    u1 = uniform01(seed, stream, c * np.uint64(2))
    u2 = uniform01(seed, stream, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass(frozen=True)
class AnnulusSpec:
    """A left-ventricle-like wall: annulus r_in <= r <= r_out about an axis.

    ``ha_in_deg``/``ha_out_deg``: helical angle at the inner (endocardial) and
    outer (epicardial) radius, linear in between.  ``period``: grating period
    in voxels.  ``ia_std_deg``/``ia_corr``: optional smooth out-of-plane tilt
    of the rods (a radial warp drawn from a low-pass random field).
    ``noise``: ("gauss", std) or ("poisson_like", fraction): per-voxel std =
    fraction * sqrt(background * clean intensity).
    """

    shape: Tuple[int, int, int]  # (nz, ny, nx)
    r_in: float
    r_out: float
    period: float
    ha_in_deg: float
    ha_out_deg: float
    center: Optional[Tuple[float, float, float]] = None  # (x, y, z); default = volume centre
    axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)  # (x, y, z)
    background: float = 1000.0
    amplitude: float = 800.0
    noise: Tuple[str, float] = ("gauss", 50.0)
    ia_std_deg: float = 0.0
    ia_corr: float = 40.0
    seed: int = 1

    def centre_xyz(self) -> Tuple[float, float, float]:
        if self.center is not None:
            return tuple(float(c) for c in self.center)
        nz, ny, nx = self.shape
        return ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)

    def unit_axis(self) -> np.ndarray:
        a = np.asarray(self.axis, dtype=np.float64)
        return a / np.linalg.norm(a)


def _plane_basis(a: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Two unit vectors u, w with (u, w, a) right-handed and orthonormal."""
    ref = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = ref - np.dot(ref, a) * a
    u /= np.linalg.norm(u)
    w = np.cross(a, u)
    return u, w


def _smootherstep(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _value_noise(spec: AnnulusSpec, px, py, pz) -> np.ndarray:
    """C1 value noise: N(0,1) lattice values at spacing ia_corr, quintic-smoothstep blended."""
    L = float(spec.ia_corr)
    fx, fy, fz = px / L, py / L, pz / L
    ix, iy, iz = np.floor(fx), np.floor(fy), np.floor(fz)
    tx, ty, tz = _smootherstep(fx - ix), _smootherstep(fy - iy), _smootherstep(fz - iz)
    ix = ix.astype(np.int64) + 4
    iy = iy.astype(np.int64) + 4
    iz = iz.astype(np.int64) + 4
    out = np.zeros(np.broadcast(px, py, pz).shape)
    for dz in (0, 1):
        wz = tz if dz else 1.0 - tz
        for dy in (0, 1):
            wy = ty if dy else 1.0 - ty
            for dx in (0, 1):
                wx = tx if dx else 1.0 - tx
                idx = ((iz + dz) * 4096 + (iy + dy)) * 4096 + (ix + dx)
                out = out + wx * wy * wz * normal(spec.seed, 7, idx.astype(np.uint64))
    return out


def _clean_and_mask(spec: AnnulusSpec, x, y, z):
    """Noise-free intensity and annulus mask at voxel positions (x, y, z)."""
    c = np.asarray(spec.centre_xyz())
    a = spec.unit_axis()
    u, w = _plane_basis(a)
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    h = dx * a[0] + dy * a[1] + dz * a[2]
    rx, ry, rz = dx - h * a[0], dy - h * a[1], dz - h * a[2]
    r = np.sqrt(rx * rx + ry * ry + rz * rz)
    mask = (r >= spec.r_in) & (r <= spec.r_out)

    if spec.ia_std_deg > 0.0:
        # Radial warp: rods tilt out of the wall's tangent plane by about
        # atan(d delta / d fibre), a smooth field of std ~ ia_std_deg.
        amp = math.tan(math.radians(spec.ia_std_deg)) * spec.ia_corr / 1.3
        delta = amp * _value_noise(spec, x, y, z)
        r = np.maximum(r - delta, 0.0)

    theta = np.arctan2(rx * w[0] + ry * w[1] + rz * w[2], rx * u[0] + ry * u[1] + rz * u[2])
    t = np.clip((r - spec.r_in) / (spec.r_out - spec.r_in), 0.0, 1.0)
    ha = np.radians(spec.ha_in_deg + t * (spec.ha_out_deg - spec.ha_in_deg))
    T = float(spec.period)

    # Rods along f0 = cos(HA) e_theta + sin(HA) e_z: one family of stripes
    # varies with r, the other with a helical phase whose gradient is normal
    # to f0.  A single helical phase cannot stay smooth across the whole wall
    # (its radial derivative grows with the distance from its origin because
    # HA changes with r), so it is taken about local origins on a (theta, h)
    # lattice of spacing 2T and blended with C1 smoothstep weights.
    L = 2.0 * T
    r_mid = 0.5 * (spec.r_in + spec.r_out)
    n_sec = max(4, int(round(2.0 * math.pi * r_mid / L)))
    dth = 2.0 * math.pi / n_sec
    gs = (theta + math.pi) / dth
    g0 = np.floor(gs)
    fs = gs - g0
    fs = fs * fs * (3.0 - 2.0 * fs)
    hs = h / L
    h0 = np.floor(hs)
    fh = hs - h0
    fh = fh * fh * (3.0 - 2.0 * fh)
    sin_ha, cos_ha = np.sin(ha), np.cos(ha)
    helical = np.zeros_like(r)
    for ds in (0, 1):
        ws = fs if ds else 1.0 - fs
        th_j = (g0 + ds) * dth - math.pi
        dtheta = np.angle(np.exp(1j * (theta - th_j)))
        for dh in (0, 1):
            wh = fh if dh else 1.0 - fh
            h_j = (h0 + dh) * L
            phi2 = cos_ha * (h - h_j) - sin_ha * r * dtheta
            helical = helical + ws * wh * np.cos(2.0 * math.pi * phi2 / T)
    grating = np.cos(2.0 * math.pi * r / T) + helical
    clean = spec.background + np.where(mask, 0.5 * spec.amplitude * grating, 0.0)
    return clean, mask


def _generate_slab(spec: AnnulusSpec, zs: int, ze: int):
    nz, ny, nx = spec.shape
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    zz = np.arange(zs, ze, dtype=np.float64)[:, None, None]
    x = np.broadcast_to(xx[None], (ze - zs, ny, nx))
    y = np.broadcast_to(yy[None], (ze - zs, ny, nx))
    z = np.broadcast_to(zz, (ze - zs, ny, nx))
    clean, mask = _clean_and_mask(spec, x, y, z)
    idx = (np.arange(zs, ze, dtype=np.uint64)[:, None, None] * np.uint64(ny * nx)
           + np.arange(ny * nx, dtype=np.uint64).reshape(1, ny, nx))
    n = normal(spec.seed, 1, idx)
    kind, level = spec.noise
    if kind == "gauss":
        std = level
    elif kind == "poisson_like":
        std = level * np.sqrt(spec.background * np.maximum(clean, 0.0))
    else:
        raise ValueError(f"unknown noise kind {kind!r}")
    val = np.rint(np.clip(clean + std * n, 0.0, 65535.0))
    return val.astype(np.uint16), mask.astype(np.uint8)


def generate(spec: AnnulusSpec, z_range: Optional[Tuple[int, int]] = None, slab: int = 4,
             threads: Optional[int] = None):
    """Volume ``vol[z, y, x]`` (uint16) and annulus mask (uint8 0/1) for planes z_range.

    Each voxel is a pure function of (spec, global voxel index): generating a
    z-range gives exactly the planes of the whole volume, and the result does
    not depend on the slab size or thread count.
    """
    import concurrent.futures
    import os

    nz, ny, nx = spec.shape
    z0, z1 = (0, nz) if z_range is None else z_range
    vol = np.empty((z1 - z0, ny, nx), dtype=np.uint16)
    msk = np.empty((z1 - z0, ny, nx), dtype=np.uint8)
    starts = list(range(z0, z1, slab))
    nthr = threads or min(32, os.cpu_count() or 1)

    def work(zs):
        ze = min(z1, zs + slab)
        v, m = _generate_slab(spec, zs, ze)
        vol[zs - z0:ze - z0] = v
        msk[zs - z0:ze - z0] = m

    if nthr <= 1 or len(starts) == 1:
        for zs in starts:
            work(zs)
    else:
        with concurrent.futures.ThreadPoolExecutor(nthr) as ex:
            list(ex.map(work, starts))
    return vol, msk


def truth_fibre(spec: AnnulusSpec, x, y, z) -> np.ndarray:
    """Analytic rod direction f0 at positions (ignores the optional IA warp)."""
    c = np.asarray(spec.centre_xyz())
    a = spec.unit_axis()
    d = np.stack([x - c[0], y - c[1], z - c[2]], axis=-1)
    h = d @ a
    rv = d - h[..., None] * a
    r = np.linalg.norm(rv, axis=-1)
    er = rv / np.maximum(r, 1e-300)[..., None]
    et = np.cross(a, er)
    t = np.clip((r - spec.r_in) / (spec.r_out - spec.r_in), 0.0, 1.0)
    ha = np.radians(spec.ha_in_deg + t * (spec.ha_out_deg - spec.ha_in_deg))
    return np.cos(ha)[..., None] * et + np.sin(ha)[..., None] * a


# Workloads: shapes, scales and structure of whole-heart orientation runs.
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    spec: AnnulusSpec
    sigma: float
    rho: float
    use_mask: bool


def single_chunk_64() -> Workload:
    """64^3 cylinder, radii 10-28, period 4, HA +60 -> -60, IA 0, N(0, 50) noise; sigma 1, rho 3; no mask."""
    spec = AnnulusSpec(shape=(64, 64, 64), r_in=10.0, r_out=28.0, period=4.0, ha_in_deg=60.0,
                       ha_out_deg=-60.0, noise=("gauss", 50.0), seed=1)
    return Workload("annulus64_s1_r3", spec, 1.0, 3.0, False)


def lv_annulus_512(n: int = 512) -> Workload:
    """512^3 LV-like annulus r 120/220, axis tilted 10 deg, period 6, HA +70 -> -70,
    IA field std 5 deg / corr 40, Poisson-like 5% noise, masked; sigma 2, rho 6.

    ``n`` < 512 scales the geometry down for small test cases.
    """
    s = n / 512.0
    tilt = math.radians(10.0)
    spec = AnnulusSpec(shape=(n, n, n), r_in=120.0 * s, r_out=220.0 * s, period=6.0, ha_in_deg=70.0,
                       ha_out_deg=-70.0, axis=(math.sin(tilt), 0.0, math.cos(tilt)),
                       noise=("poisson_like", 0.05), ia_std_deg=5.0, ia_corr=40.0, seed=2)
    return Workload(f"lv_annulus{n}_s2_r6", spec, 2.0, 6.0, True)


def crop_batch(count: int = 200, seed: int = 4, size_range: Tuple[int, int] = (64, 384),
               sigmas: Sequence[float] = (1.0, 1.5, 2.0, 3.0), rhos: Sequence[float] = (2.0, 4.0, 6.0, 8.0)):
    """Uneven crops, each its own small heart-wall volume: every axis uniform in
    size_range, its own sigma and rho, a random LV centre (middle half of the
    crop) and axis (within 20 deg of z), radii 0.2 / 0.42 of the smallest side,
    HA range +-(30..80) deg, Gaussian noise of 2-10% of the background.  All
    draws come from the counter-based generator (seed, stream 11), crop j using
    counters 32 j .. 32 j + 31."""
    out = []
    lo, hi = size_range
    for j in range(count):
        u = uniform01(seed, 11, np.arange(32 * j, 32 * j + 32, dtype=np.uint64))
        nx, ny, nz = (int(lo + min(hi - lo, np.floor(u[k] * (hi - lo + 1)))) for k in range(3))
        sigma = float(sigmas[min(len(sigmas) - 1, int(u[3] * len(sigmas)))])
        rho = float(rhos[min(len(rhos) - 1, int(u[4] * len(rhos)))])
        cx = (0.25 + 0.5 * u[5]) * (nx - 1)
        cy = (0.25 + 0.5 * u[6]) * (ny - 1)
        cz = (0.25 + 0.5 * u[7]) * (nz - 1)
        tilt = math.radians(20.0 * u[8])
        az = 2.0 * math.pi * u[9]
        axis = (math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), math.cos(tilt))
        m = min(nx, ny, nz)
        ha = 30.0 + 50.0 * u[10]
        spec = AnnulusSpec(shape=(nz, ny, nx), r_in=0.2 * m, r_out=0.42 * m, period=6.0, ha_in_deg=ha,
                           ha_out_deg=-ha, center=(cx, cy, cz), axis=axis,
                           noise=("gauss", (0.02 + 0.08 * u[11]) * 1000.0), seed=1000 + j)
        out.append(Workload(f"crop{j}_{nx}x{ny}x{nz}_s{sigma}_r{rho}", spec, sigma, rho, False))
    return out


def frame_of(spec: AnnulusSpec) -> Tuple[Sequence[float], Sequence[float]]:
    """(lv_center, lv_axis) in (x, y, z) voxel units, as the pipeline takes them."""
    return spec.centre_xyz(), tuple(float(v) for v in spec.axis)
