"""The transmural HA profile kernel against the FP64 oracle histogram.

A voxel whose depth or HA lies within a rounding distance of a bin edge may
fall on either side (the kernel computes depth in FP32); those voxels are the
only tolerance: each bin may differ by at most the number of such voxels near
its edges, and the totals by the number near the depth range's ends.
"""
import numpy as np
import pytest

from oracle import oracle, profile
from paper_2508_07476_gb300 import _lib, build, synth

from gpu_util import fused

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _gpu_hist(ha, mask, lo, dims, center, axis, r_in, r_out, nd, nh, ha_type):
    spec = _lib.make_profile_spec(center, axis, r_in, r_out, nd, nh, ha_type)
    d_ha = torch.from_numpy(np.ascontiguousarray(ha)).cuda()
    d_mask = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    hist = torch.zeros(nd * nh, dtype=torch.int64, device="cuda")
    nz, ny, nx = ha.shape
    _lib.ct_transmural_profile(spec, dims, lo, (nx, ny, nz), d_ha, d_mask, hist)
    torch.cuda.synchronize()
    return hist.cpu().numpy().astype(np.uint64).reshape(nd, nh)


def _near_edges(values, n_bins, lo, hi, eps):
    """Voxels whose value is within eps of an interior bin edge (or of the range ends)."""
    t = (values - lo) / (hi - lo) * n_bins
    return np.abs(t - np.round(t)) * (hi - lo) / n_bins < eps


def _assert_close(gpu, ora, slack):
    diff = np.abs(gpu.astype(np.int64) - ora.astype(np.int64))
    assert diff.sum() <= 2 * slack, (diff.sum(), slack)
    assert abs(int(gpu.sum()) - int(ora.sum())) <= slack


@pytest.mark.parametrize("nx", [301, 304])
@pytest.mark.parametrize("ha_type", [_lib.CT_OUT_F32, _lib.CT_OUT_F16, _lib.CT_OUT_U8Q])
def test_histogram_of_a_given_field(ha_type, nx):
    rng = np.random.default_rng(5)
    # 301: rows of ragged 8-voxel segments, loaded voxel by voxel; 304: whole
    # segments, one vector load each
    shape = (23, 70, nx)
    lo, dims = (40, 3, 7), (400, 80, 40)
    center, axis = (190.3, 40.7, 12.0), (0.15, -0.2, 1.0)
    r_in, r_out, nd, nh = 10.0, 60.0, 16, 90
    ha = rng.uniform(-90.0, 90.0, size=shape).astype(np.float32)
    mask = (rng.random(shape) < 0.85).astype(np.uint8)
    if ha_type == _lib.CT_OUT_F32:
        ha[rng.random(shape) < 0.05] = np.nan
        field, decoded = ha, ha.astype(np.float64)
    elif ha_type == _lib.CT_OUT_F16:
        field = ha.astype(np.float16)
        field[rng.random(shape) < 0.05] = np.nan
        decoded = field.astype(np.float64)
    else:
        field = (np.rint((ha.astype(np.float64) + 90.0) * 256.0 / 180.0).astype(np.int64) % 256).astype(np.uint8)
        field[rng.random(shape) < 0.05] = 0
        decoded = np.where(field == 0, np.nan, field.astype(np.float64) * 180.0 / 256.0 - 90.0)
    gpu = _gpu_hist(field, mask, lo, dims, center, axis, r_in, r_out, nd, nh, ha_type)
    ora = profile.transmural_profile(decoded, mask, lo, center, axis, r_in, r_out, nd, nh)
    d = profile.depth_field(shape, lo, center, axis, r_in, r_out)
    near = mask.astype(bool) & np.isfinite(decoded) & (
        _near_edges(d, nd, 0.0, 1.0, 1e-5) | _near_edges(decoded, nh, -90.0, 90.0, 1e-4))
    _assert_close(gpu, ora, int(near.sum()))
    assert ora.sum() > 100000


def test_profile_of_the_pipeline_matches_the_oracle_pipeline():
    """HA from the GPU pipeline vs HA from the FP64 oracle pipeline, same volume.
    The histograms may differ only by voxels whose two HA values fall in
    different bins (or whose depth is near an edge), and those must be few."""
    W = synth.lv_annulus_512(96)
    vol, mask = synth.generate(W.spec)
    n = 96
    cen, ax = synth.frame_of(W.spec)
    ora = oracle.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask)
    g = fused(vol, W.sigma, W.rho, cen, ax, mask=mask, precision=_lib.CT_PREC_FP32)
    nd, nh = 10, 36
    r_in, r_out = W.spec.r_in, W.spec.r_out
    gpu = _gpu_hist(g["ha"], mask, (0, 0, 0), (n, n, n), cen, ax, r_in, r_out, nd, nh, _lib.CT_OUT_F32)
    oh = profile.transmural_profile(ora["ha"], mask, (0, 0, 0), cen, ax, r_in, r_out, nd, nh)
    d = profile.depth_field(vol.shape, (0, 0, 0), cen, ax, r_in, r_out)
    counted = mask.astype(bool) & np.isfinite(ora["ha"]) & (d >= 0) & (d < 1)

    def hbin(h):
        return np.clip(np.floor((np.nan_to_num(h.astype(np.float64)) + 90.0) * nh / 180.0), 0, nh - 1)

    moved = counted & (hbin(g["ha"]) != hbin(ora["ha"]))
    near = counted & _near_edges(d, nd, 0.0, 1.0, 1e-5)
    slack = int((moved | near).sum())
    assert slack <= 0.02 * counted.sum(), (slack, int(counted.sum()))
    _assert_close(gpu, oh, slack)
    assert oh.sum() > 10000


def test_invalid_arguments():
    ha = torch.zeros((2, 2, 2), device="cuda")
    hist = torch.zeros(4, dtype=torch.int64, device="cuda")
    for nd, nh, r_in, r_out, ty in [(0, 4, 1.0, 2.0, 0), (200, 100, 1.0, 2.0, 0), (2, 2, 2.0, 2.0, 0),
                                    (2, 2, 1.0, 2.0, 7)]:
        spec = _lib.make_profile_spec((0, 0, 0), (0, 0, 1), r_in, r_out, nd, nh, ty)
        with pytest.raises(_lib.CTError):
            _lib.ct_transmural_profile(spec, (2, 2, 2), (0, 0, 0), (2, 2, 2), ha, None, hist)
    spec = _lib.make_profile_spec((0, 0, 0), (0, 0, 0), 1.0, 2.0, 2, 2)
    with pytest.raises(_lib.CTError):
        _lib.ct_transmural_profile(spec, (2, 2, 2), (0, 0, 0), (2, 2, 2), ha, None, hist)
    spec = _lib.make_profile_spec((0, 0, 0), (0, 0, 1), 1.0, 2.0, 2, 2)
    with pytest.raises(_lib.CTError):
        _lib.ct_transmural_profile(spec, (2, 2, 2), (1, 0, 0), (2, 2, 2), ha, None, hist)
