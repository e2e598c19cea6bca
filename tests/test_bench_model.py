"""The benchmark's algorithmic model, on CPU: the bytes and FMAs each kernel is
charged, from which the roofline fractions are computed."""
import pytest

import bench


def test_kernel_bytes_per_voxel():
    # each input and output once: volume (2 B), partial fields (3 x 4 B),
    # products and smoothed tensors (6 x 4 B), mask (1 B), outputs (6 x 4 B)
    assert bench._kernel_algorithmic("grad_xy", 1, 8, 24) == (0, 2 + 12)
    assert bench._kernel_algorithmic("grad_z", 1, 8, 24) == (0, 12 + 24)
    for k in ("rho_x_tc", "rho_y_tc", "rho_z_tc"):
        assert bench._kernel_algorithmic(k, 1, 8, 24) == (0, 48)


@pytest.mark.parametrize("inside", [0.0, 0.413, 1.0])
def test_eigen_bytes_follow_the_mask(inside):
    # the tensor is read for voxels inside the mask only; the mask and the six
    # outputs (fill outside) everywhere
    _, b = bench._kernel_algorithmic("eig_angles", 1000, 8, 24, inside)
    assert b == pytest.approx(1000 * (1 + 24 + 24 * inside))


def test_launched_sequence_floor():
    # grad_xy + grad_z + three rho passes + eigen on the annulus (41.3% inside)
    seq = ("grad_xy", "grad_z", "rho_x_tc", "rho_y_tc", "rho_z_tc", "eig_angles")
    total = sum(bench._kernel_algorithmic(k, 1, 8, 24, 0.413)[1] for k in seq)
    assert total == pytest.approx(14 + 36 + 3 * 48 + 1 + 24 + 24 * 0.413)
    assert round(total) == 229


def test_stencil_fma_count():
    # 8 sigma passes, 6 products, 18 rho passes of 2R+1 taps: 1024 at sigma 2, rho 6;
    # 1312 at sigma 2, rho 8; 1520 at sigma 3, rho 9
    assert bench._fma_per_voxel(8, 24) == 8 * 17 + 6 + 18 * 49 == 1024
    assert bench._fma_per_voxel(8, 32) == 1312
    assert bench._fma_per_voxel(12, 36) == 1520


def test_grading_exempts_only_ill_conditioned_voxels():
    # a direction error above 0.5 deg passes only where the voxel's own bound
    # eps_S tr S / (l2 - l1) is larger, and is counted either way
    import numpy as np
    ev = np.array([[1.0, 1.0], [1.0 + 1e-4, 2.0], [3.0, 3.0]])[:, :, None, None]  # [3, 2, 1, 1]
    ora = {"fa": np.full((2, 1, 1), 0.5), "ha": np.zeros((2, 1, 1)), "ia": np.zeros((2, 1, 1)), "evals": ev,
           "v": np.zeros((3, 2, 1, 1))}
    ora["v"][0] = 1.0
    t = np.radians(1.0)
    out = {k: ora[k].copy() for k in ("ha", "ia", "fa")}
    out["v"] = np.zeros((3, 2, 1, 1))
    out["v"][0], out["v"][1] = np.cos(t), np.sin(t)  # 1 deg off on both voxels
    r = bench._grade_box(ora, out, np.ones((2, 1, 1), bool), 1)
    assert r["dir_over_05"] == 2 and r["ill"] == 1
    assert r["dir_bound_excess"] > 0  # the well-conditioned voxel fails its 0.5 deg bound
