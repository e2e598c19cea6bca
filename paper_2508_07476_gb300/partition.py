"""Host-side partition of one volume into z-slabs across ranks (one GPU each).

Every output voxel depends on its input neighbourhood of radius
R(sigma) + R(rho) only (the Implementation section's chunks with padding), so
a volume splits across GPUs into z-slabs with no exchange on the data path:
rank k computes the output planes [z0_k, z1_k) from the input planes
[max(0, z0_k - h), min(nz, z1_k + h)), h = R(sigma) + R(rho) along z, and the
slabs' outputs tile the volume.  Because edges are clamped at the GLOBAL
volume only and every slab's input holds the full halo inside the volume,
each slab's outputs equal the whole-volume run's (the library's padded-box
call, ct_run_box, takes the boxes in global coordinates).  This module holds
the partition arithmetic only, none of the method's.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple


@dataclass(frozen=True)
class Slab:
    rank: int
    out_lo: Tuple[int, int, int]  # (x, y, z), global
    out_n: Tuple[int, int, int]
    in_lo: Tuple[int, int, int]
    in_n: Tuple[int, int, int]

    @property
    def out_z(self) -> Tuple[int, int]:
        return self.out_lo[2], self.out_lo[2] + self.out_n[2]

    @property
    def in_z(self) -> Tuple[int, int]:
        return self.in_lo[2], self.in_lo[2] + self.in_n[2]


def z_slabs(dims: Tuple[int, int, int], world: int, halo_z: int) -> List[Slab]:
    """Slabs of a volume of size dims (x, y, z) for `world` ranks: output planes
    split as evenly as possible (the first nz % world slabs one plane longer),
    inputs grown by halo_z planes and clipped to the volume.  A rank with no
    planes (world > nz) gets an empty slab."""
    nx, ny, nz = dims
    if world < 1 or halo_z < 0 or min(dims) < 1:
        raise ValueError("bad partition request")
    out = []
    base, extra = divmod(nz, world)
    z = 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        z0, z1 = z, z + n
        i0, i1 = (max(0, z0 - halo_z), min(nz, z1 + halo_z)) if n > 0 else (z0, z0)
        out.append(Slab(k, (0, 0, z0), (nx, ny, n), (0, 0, i0), (nx, ny, i1 - i0)))
        z = z1
    return out
