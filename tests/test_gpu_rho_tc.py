"""The integration-scale passes on the tensor cores (banded Toeplitz products
with TF32 split operands), called through the C ABI, against the FP64 oracle.

CT_TUNE_TC_RHO selects, per plan, which axes run on the tensor cores (bit a
for axis a; the library default is 7, all three, for rho radii of 24 and up
on volumes whose x extent suits 16-byte copies); the oracle cases run each
single axis, all three and none (the FP32 stencils), so a wrong ring slot,
band offset, transpose or clamp on any axis fails.  With all three axes the
default chain stores the gradient (FP16 in the mixed form) and forms the
products in the z pass (then y, then x); CT_TUNE_TC_PRODUCTS=0 keeps the
products in the gradient kernel and runs x, y, z: both are graded.  Tolerances are
the FP32 stage tolerances of test_gpu_parity.py: the split keeps each product
within about 2^-20 of its value, below the stencil's own accumulated rounding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402

FP32, MIXED = _lib.CT_PREC_FP32, _lib.CT_PREC_MIXED
MASKS = [0, 1, 2, 4, 7]  # 0: the FP32 stencil passes


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


@pytest.fixture
def tc(monkeypatch):
    # the library picks the tensor cores for R >= 24 and volumes whose x extent
    # suits the 16-byte copies; these tests force them (or the stencils, mask 0)
    # at every radius and extent
    def use(mask, products=True):
        monkeypatch.setenv("CT_TUNE_TC_RHO", str(mask))
        monkeypatch.setenv("CT_TUNE_TC_MIN_R", "0")
        monkeypatch.setenv("CT_TUNE_TC_ANY_BOX", "1")
        monkeypatch.setenv("CT_TUNE_TC_PRODUCTS", "1" if products else "0")
    return use


def _rand_vol(shape, seed, lo=500, hi=3000):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(seed)
    v = rng.integers(lo, hi, size=shape).astype(np.float64)
    v = ndi.gaussian_filter(v, 1.0) + rng.normal(0, 30, size=shape)
    return np.clip(np.rint(v), 0, 65535).astype(np.uint16)


def _rel(S, S_o):
    return (np.abs(S - S_o) / (S_o[0] + S_o[1] + S_o[2])[None]).max()


# radii of rho: 1.0 -> 4, 1.7 -> 7 (served by 8), 3.0 -> 12, 6.0 -> 24, 9.0 -> 36 (256 TMEM columns)
@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("shape,sigma,rho", [((23, 29, 37), 1.0, 1.0), ((9, 8, 130), 0.8, 1.7),
                                             ((40, 17, 70), 1.5, 3.0), ((70, 33, 45), 2.0, 6.0),
                                             ((20, 150, 11), 1.0, 9.0), ((40, 24, 256), 2.0, 6.0),
                                             ((16, 64, 256), 1.0, 3.0),  # x rows through tensor maps
                                             ((24, 20, 200), 1.0, 6.0)])  # 16-byte y / z copies, ragged group
def test_tc_structure_tensor_ragged(tc, mask, shape, sigma, rho):
    tc(mask)
    vol = _rand_vol(shape, seed=sum(shape))
    g = G.stages(vol, sigma, rho, (10.0, 10.0, 5.0), (0.0, 0.0, 1.0))
    S_o = O.structure_tensor(vol, sigma, rho)
    err = _rel(g["S"], S_o)
    assert err <= 2e-5, (mask, err)


@pytest.mark.parametrize("mask", MASKS + ["7j"])
def test_tc_sub_box_matches_oracle_and_whole(tc, mask):
    # a padded chunk whose line groups, rows and segments are all ragged
    # ("7j": all three axes with the products in the gradient kernel)
    tc(7, False) if mask == "7j" else tc(mask)
    vol = _rand_vol((60, 150, 140), seed=11)
    sigma, rho = 1.0, 3.0
    h = O.radius(sigma) + O.radius(rho)
    out_lo, out_n = (13, 41, 9), (120, 70, 37)
    in_lo = tuple(max(0, a - h) for a in out_lo)
    in_hi = tuple(min(d, a + n + h) for a, n, d in zip(out_lo, out_n, (140, 150, 60)))
    in_n = tuple(b - a for a, b in zip(in_lo, in_hi))
    g = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1), in_box=(in_lo, in_n), out_box=(out_lo, out_n))
    S_o = O.structure_tensor(vol, sigma, rho, lo=out_lo, n=out_n)
    assert _rel(g["S"], S_o) <= 2e-5
    full = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1))
    sl = (slice(None), slice(out_lo[2], out_lo[2] + out_n[2]), slice(out_lo[1], out_lo[1] + out_n[1]),
          slice(out_lo[0], out_lo[0] + out_n[0]))
    np.testing.assert_array_equal(g["S"], full["S"][sl])


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("nx_out", [128, 100, 124])
def test_tc_aligned_sub_box_matches_oracle_and_whole(tc, mask, nx_out):
    # boxes on 16-byte boundaries: the 16-byte copy paths (100: a ragged line
    # group, whose last warps copy line by line; 124: x extents that are
    # multiples of 4 but not 8, where the FP16 gradient rows lose their
    # 16-byte alignment and go line by line)
    tc(mask)
    vol = _rand_vol((48, 60, 192), seed=13)
    sigma, rho = 1.0, 3.0
    h = O.radius(sigma) + O.radius(rho)
    assert h == 16
    out_lo, out_n = (16, 20, 16), (nx_out, 20, 16)
    in_lo = tuple(a - h for a in out_lo)
    in_n = tuple(n + 2 * h for n in out_n)
    g = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1), in_box=(in_lo, in_n), out_box=(out_lo, out_n))
    S_o = O.structure_tensor(vol, sigma, rho, lo=out_lo, n=out_n)
    assert _rel(g["S"], S_o) <= 2e-5
    full = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1))
    sl = (slice(None), slice(out_lo[2], out_lo[2] + out_n[2]), slice(out_lo[1], out_lo[1] + out_n[1]),
          slice(out_lo[0], out_lo[0] + out_n[0]))
    np.testing.assert_array_equal(g["S"], full["S"][sl])


@pytest.mark.parametrize("products", [True, False])
@pytest.mark.parametrize("prec,tol", [(FP32, 2e-5), (MIXED, 2e-3)])
def test_tc_helix64(tc, prec, tol, products):
    tc(7, products)
    W = synth.single_chunk_64()
    vol, _ = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    g = G.stages(vol, W.sigma, W.rho, cen, ax, precision=prec)
    S_o = O.structure_tensor(vol, W.sigma, W.rho)
    assert _rel(g["S"], S_o) <= tol


def test_tc_agrees_with_stencil(tc):
    # the same plan settings with and without the tensor cores: tensors agree
    # to the FP32 stage tolerance on a volume with a 512-long z line
    vol = _rand_vol((512, 12, 130), seed=5)
    out = {}
    for mask in (0, 7):
        tc(mask)
        out[mask] = G.stages(vol, 2.0, 6.0, (0, 0, 0), (0, 0, 1))["S"].astype(np.float64)
    rel = np.abs(out[7] - out[0]) / (out[0][0] + out[0][1] + out[0][2])[None]
    assert rel.max() <= 2e-5, rel.max()


def test_tc_many_units_aligned_matches_oracle(tc):
    # 16-byte copies and many work units per CTA on every axis (the regime of
    # the full-size runs), graded against the oracle on boxes across the 64-
    # position tile seams (x 64 / 128 / 448, y 128, z 64) and the x pass's
    # 128-row groups (y = 128), and against the FP32 stencils everywhere
    vol = _rand_vol((96, 256, 512), seed=17)
    out = {}
    for mask in (0, 7):
        tc(mask)
        out[mask] = G.stages(vol, 2.0, 6.0, (0, 0, 0), (0, 0, 1))["S"].astype(np.float64)
    rel = np.abs(out[7] - out[0]) / (out[0][0] + out[0][1] + out[0][2])[None]
    assert rel.max() <= 2e-5, rel.max()
    b = 12
    for lo in [(58, 122, 58), (122, 250 - b, 0), (442, 0, 90 - b), (500, 122, 40), (0, 122, 84)]:
        S_o = O.structure_tensor(vol, 2.0, 6.0, lo=lo, n=(b, b, b))
        sub = out[7][:, lo[2]:lo[2] + b, lo[1]:lo[1] + b, lo[0]:lo[0] + b]
        assert _rel(sub, S_o) <= 2e-5, lo


@pytest.mark.parametrize("products", [True, False])
@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_tc_fused_and_chunked_match_oracle(tc, prec, products):
    tc(7, products)
    W = synth.single_chunk_64()
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    ora = O.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask)
    whole = G.fused(vol, W.sigma, W.rho, cen, ax, mask=mask, precision=prec)
    G.assert_within(G.compare(whole, ora, mask, precision=prec), f"tc fused prec={prec}")
    for on_host in (False, True):
        ch = G.fused(vol, W.sigma, W.rho, cen, ax, mask=mask, precision=prec, chunk=(40, 24, 20), on_host=on_host)
        for k in ("v", "ha", "ia", "fa"):
            np.testing.assert_array_equal(ch[k], whole[k])


@pytest.mark.parametrize("sp", [(1.0, 1.25, 0.8), (0.6, 0.6, 1.5)])
def test_tc_anisotropic_matches_oracle(tc, sp):
    # per-axis tap sets, zero-padded to the largest radius, on every axis
    tc(7)
    W = synth.single_chunk_64()
    vol, _ = synth.generate(W.spec)
    vol = vol[4:60, 2:62, 0:64].copy()
    sigma, rho = W.sigma * sp[0], W.rho * sp[0]
    nz, ny, nx = vol.shape
    c = ((nx - 1) / 2 * sp[0], (ny - 1) / 2 * sp[1], (nz - 1) / 2 * sp[2])
    ax = (0.05, 0.0, 1.0)
    ora = O.pipeline(vol, sigma, rho, c, ax, spacing=sp)
    gpu = G.fused(vol, sigma, rho, c, ax, spacing=sp)
    G.assert_within(G.compare(gpu, ora, precision=FP32), f"tc aniso {sp}")


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 9), (6, 1, 5), (4, 5, 1), (2, 3, 200)])
def test_tc_degenerate_shapes(tc, shape):
    tc(7)
    vol = _rand_vol(shape, seed=11)
    cen, ax = (0.3, 0.4, 0.5), (0.0, 1.0, 1.0)
    ora = O.pipeline(vol, 1.0, 2.0, cen, ax)
    gpu = G.fused(vol, 1.0, 2.0, cen, ax)
    G.assert_within(G.compare(gpu, ora), f"tc shape {shape}")


def test_tc_constant_volume_gives_zero_tensor(tc):
    tc(7)
    vol = np.full((20, 21, 22), 1500, np.uint16)
    st = G.stages(vol, 1.0, 3.0, (10, 10, 10), (0, 0, 1))
    assert np.all(st["S"] == 0.0)
    assert np.all(st["fa"] == 0.0)


def _kernels_and_outputs(vol, sigma, rho, chunk=(0, 0, 0)):
    nz, ny, nx = vol.shape
    p = _lib.make_params(sigma, rho, (nx / 2, ny / 2, nz / 2), (0, 0, 1), FP32, chunk=chunk)
    plan = _lib.ct_plan_create(p, (nx, ny, nz))
    try:
        _lib.ct_plan_profile(plan, True)
        fa = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
        vec = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        _lib.ct_run_chunks(plan, [_lib.make_item(G.dev_u16(vol), (nx, ny, nz), None, vec, None, None, fa)], False)
        torch.cuda.synchronize()
        _lib.ct_plan_sync(plan)
        names = set(_lib.ct_plan_kernel_times(plan))
    finally:
        _lib.ct_plan_destroy(plan)
    return names, vec.cpu().numpy(), fa.cpu().numpy()


@pytest.mark.parametrize("nx,rho,min_vox,expect_tc", [(128, 6.0, "0", "xyz"), (256, 8.0, "0", "xyz"),
                                                      (100, 6.0, "0", "xyz"), (126, 6.0, "0", ""),
                                                      (128, 3.0, "0", ""), (128, 6.0, None, "")])
def test_default_selection_is_per_volume(monkeypatch, nx, rho, min_vox, expect_tc):
    monkeypatch.setenv("CT_TUNE_CACHE", "")  # the built-in choices
    # the tensor cores take rho radii >= 24 on volumes whose x extent suits their
    # 16-byte copies (a multiple of 4) and, with the library's own settings, of
    # at least 2^24 voxels (None: that default, which sends these small volumes
    # to the stencils); chunks of any shape take the whole volume's passes and
    # match it bit for bit
    if min_vox is not None:
        monkeypatch.setenv("CT_TUNE_TC_MIN_VOX", min_vox)
    vol = _rand_vol((40, 36, nx), seed=nx)
    names, v, fa = _kernels_and_outputs(vol, 1.0, rho)
    tc_axes = "".join(a for a in "xyz" if any(k.startswith(f"rho_{a}_tc") for k in names))
    assert tc_axes == ("xyz" if expect_tc == "xyz" else ""), names
    assert ("rho_xy" in names) == (expect_tc != "xyz"), names
    names_c, v_c, fa_c = _kernels_and_outputs(vol, 1.0, rho, chunk=(44, 20, 16))
    assert {n for n in names_c if n.startswith("rho")} == {n for n in names if n.startswith("rho")}
    np.testing.assert_array_equal(v_c, v)
    np.testing.assert_array_equal(fa_c, fa)


@pytest.mark.parametrize("shape", [(40, 24, 256), (24, 20, 204), (20, 30, 61), (16, 40, 128)])
def test_tc_fp16_gradient_paths(tc, shape):
    # the mixed form's gradient crosses HBM in FP16 and the z pass forms the
    # products from it: 16-byte copies of 8 lines (x extent a multiple of 8),
    # line-by-line loads otherwise (204, 61).  The chain with the products in
    # the gradient kernel uses the same FP16-rounded gradient and the same FP32
    # products, so the two differ only by the order of the three passes
    vol = _rand_vol(shape, seed=sum(shape) + 1)
    S_o = O.structure_tensor(vol, 1.0, 3.0)
    out = {}
    for products in (True, False):
        tc(7, products)
        out[products] = G.stages(vol, 1.0, 3.0, (10.0, 10.0, 5.0), (0.0, 0.0, 1.0), precision=MIXED)["S"]
        assert _rel(out[products], S_o) <= 2e-3, products
    assert _rel(out[True], out[False].astype(np.float64)) <= 2e-5
