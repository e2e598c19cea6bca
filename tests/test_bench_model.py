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


def test_stencil_fma_count_and_roofline():
    # 8 sigma passes, 6 products, 18 rho passes of 2R+1 taps: 1024 at sigma 2, rho 6
    assert bench._fma_per_voxel(8, 24) == 8 * 17 + 6 + 18 * 49 == 1024
    fma_peak = 152 * 128 * 2070e6
    assert fma_peak / 1024 == pytest.approx(3.93e10, rel=1e-3)
