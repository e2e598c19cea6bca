"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Stages (structure tensor, eigen-solve, angles) and the fused chunked path are
compared element by element on seeded inputs: the 64^3 helix chunk, ragged
random volumes spanning several tiles, degenerate shapes, masks and output
encodings; and on sampled boxes of the 512^3 annulus in the launch
configuration the benchmark times.  Tolerances: see gpu_util.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402

FP32, MIXED = _lib.CT_PREC_FP32, _lib.CT_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _lib_loaded():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _helix64():
    W = synth.single_chunk_64()
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    return W, vol, mask, cen, ax


def _rand_vol(shape, seed, lo=500, hi=3000):
    rng = np.random.default_rng(seed)
    v = rng.integers(lo, hi, size=shape).astype(np.float64)
    # smooth a little so the tensor has structure, then requantise
    import scipy.ndimage as ndi
    v = ndi.gaussian_filter(v, 1.0) + rng.normal(0, 30, size=shape)
    return np.clip(np.rint(v), 0, 65535).astype(np.uint16)


def _trace(S):
    return S[0] + S[1] + S[2]


# ------------------------------------------------------------------ stages
@pytest.mark.parametrize("prec,tol", [(FP32, 2e-5), (MIXED, 2e-3)])
def test_structure_tensor_stage_helix64(prec, tol):
    W, vol, _, cen, ax = _helix64()
    g = G.stages(vol, W.sigma, W.rho, cen, ax, precision=prec)
    S_o = O.structure_tensor(vol, W.sigma, W.rho)
    err = np.abs(g["S"] - S_o) / _trace(S_o)[None]
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("shape,sigma,rho", [((23, 29, 37), 1.0, 2.0), ((40, 17, 70), 1.5, 3.0),
                                             ((20, 33, 45), 2.0, 6.0), ((9, 8, 130), 0.8, 1.7)])
def test_structure_tensor_stage_ragged(shape, sigma, rho):
    vol = _rand_vol(shape, seed=sum(shape))
    g = G.stages(vol, sigma, rho, (10.0, 10.0, 5.0), (0.0, 0.0, 1.0))
    S_o = O.structure_tensor(vol, sigma, rho)
    err = np.abs(g["S"] - S_o) / _trace(S_o)[None]
    assert err.max() <= 2e-5, err.max()


def test_structure_tensor_stage_sub_box():
    # a padded chunk: output box in the middle, input box = output grown by the halo
    vol = _rand_vol((48, 50, 52), seed=3)
    sigma, rho = 1.0, 2.0
    h = O.radius(sigma) + O.radius(rho)
    out_lo, out_n = (13, 11, 9), (20, 17, 15)
    in_lo = tuple(max(0, a - h) for a in out_lo)
    in_hi = tuple(min(d, a + n + h) for a, n, d in zip(out_lo, out_n, (52, 50, 48)))
    in_n = tuple(b - a for a, b in zip(in_lo, in_hi))
    g = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1), in_box=(in_lo, in_n), out_box=(out_lo, out_n))
    S_o = O.structure_tensor(vol, sigma, rho, lo=out_lo, n=out_n)
    assert (np.abs(g["S"] - S_o) / _trace(S_o)[None]).max() <= 2e-5
    # the whole-volume stage gives the same numbers bit for bit
    full = G.stages(vol, sigma, rho, (0, 0, 0), (0, 0, 1))
    sl = (slice(None), slice(out_lo[2], out_lo[2] + out_n[2]), slice(out_lo[1], out_lo[1] + out_n[1]),
          slice(out_lo[0], out_lo[0] + out_n[0]))
    np.testing.assert_array_equal(g["S"], full["S"][sl])


def test_structure_tensor_rejects_short_halo():
    vol = _rand_vol((20, 20, 20), seed=4)
    with pytest.raises(_lib.CTError) as ei:
        G.stages(vol, 1.0, 2.0, (0, 0, 0), (0, 0, 1), in_box=((5, 5, 5), (10, 10, 10)),
                 out_box=((6, 6, 6), (8, 8, 8)))
    assert ei.value.status == _lib.CT_ERR_INVALID


def _eig_inputs(n=20000, seed=5):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    lam = np.sort(rng.uniform(0.0, 1.0, size=(n, 3)) * 10 ** rng.uniform(-2, 6, size=(n, 1)), axis=1)
    # a quarter with a near-degenerate smallest pair, some exactly equal, some isotropic
    k = n // 4
    lam[:k, 1] = lam[:k, 0] * (1 + 10 ** rng.uniform(-7, -1, size=k))
    lam[k:k + 50, 1] = lam[k:k + 50, 2]
    lam[k + 50:k + 60] = lam[k + 50:k + 60, :1]
    A = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    S = np.stack([A[:, 0, 0], A[:, 1, 1], A[:, 2, 2], A[:, 0, 1], A[:, 0, 2], A[:, 1, 2]])
    S[:, -5:] = 0.0  # zero tensors
    return S.astype(np.float32)


@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_eig_stage_matches_oracle(prec):
    S32 = _eig_inputs()
    n = S32.shape[1]
    ev_o, v_o = O.eig_field(S32.astype(np.float64))
    p = _lib.make_params(1.0, 2.0, (0, 0, 0), (0, 0, 1), prec)
    plan = _lib.ct_plan_create(p, (n, 1, 1))
    try:
        d_S = torch.from_numpy(S32).cuda()
        ev = torch.empty((3, n), device="cuda")
        vec = torch.empty((3, n), device="cuda")
        _lib.ct_eig_smallest(plan, d_S, n, ev, vec)
        torch.cuda.synchronize()
        stats = _lib.ct_plan_stats(plan)
    finally:
        _lib.ct_plan_destroy(plan)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    scale = np.maximum(np.abs(ev_o[2]), 1e-30)
    assert (np.abs(ev - ev_o) / scale).max() <= 3e-4
    # direction: graded where the smallest pair is separated (conditioning bound
    # of the FP32-rounded input: error ~ eps * l3 / (l2 - l1))
    gap = (ev_o[1] - ev_o[0]) / np.maximum(ev_o[2], 1e-300)
    graded = gap > 1e-3
    ang = G.angle_deg(vec[:, graded], v_o[:, graded])
    assert ang.max() <= 0.5, (ang.max(), np.argmax(ang))
    assert stats["fallback_voxels"] > 0  # the near-degenerate quarter went through the re-solve
    # above the listing threshold the FP32 closed form itself decides the direction
    # on the same FP32 input: the FP32 form lists below 2e-2 of the spread, where
    # the closed form is at its floor (a few hundredths of a degree); the mixed
    # form lists below 1e-2 (its FP16-held gradient already bounds such voxels'
    # directions only to eps_S tr S / (l2 - l1) >= 5.7 deg), and just above that
    # the closed form reaches 0.12 deg on these tensors, still well inside 0.5
    gap_list, bound = (2e-2, 0.06) if prec == FP32 else (1e-2, 0.15)
    spread_ = np.maximum(ev_o[2] - ev_o[0], 1e-300)
    rel_ = (ev_o[1] - ev_o[0]) / spread_
    fp32 = rel_ > 1.25 * gap_list
    assert fp32.sum() > 1000
    assert G.angle_deg(vec[:, fp32], v_o[:, fp32]).max() <= bound
    if prec == MIXED:
        # the listed voxels are re-solved in FP64 (closed form down to a gap of 1e-4 of
        # the spread, Jacobi below): on the same FP32 input as the oracle their
        # directions agree to far better than the FP32 outputs resolve
        spread = np.maximum(ev_o[2] - ev_o[0], 1e-300)
        rel = (ev_o[1] - ev_o[0]) / spread
        fp64 = (rel < 0.8 * gap_list) & (rel > 1e-6)  # inside the listing threshold with margin
        assert fp64.sum() > 1000
        ang64 = G.angle_deg(vec[:, fp64], v_o[:, fp64])
        assert ang64.max() <= 1e-3, (ang64.max(), rel[fp64][np.argmax(ang64)])


def test_angles_stage_matches_oracle():
    W, vol, mask, cen, ax = _helix64()
    ora = O.pipeline(vol, W.sigma, W.rho, cen, ax)
    nz, ny, nx = vol.shape
    p = _lib.make_params(W.sigma, W.rho, cen, ax)
    plan = _lib.ct_plan_create(p, (nx, ny, nz))
    try:
        ev = torch.from_numpy(ora["evals"].astype(np.float32)).cuda()
        v1 = torch.from_numpy(ora["v"].astype(np.float32)).cuda()
        vo = torch.empty_like(v1)
        ha, ia, fa = (torch.empty((nz, ny, nx), device="cuda") for _ in range(3))
        _lib.ct_angles(plan, v1, ev, (0, 0, 0), (nx, ny, nz), None, vo, ha, ia, fa)
        torch.cuda.synchronize()
    finally:
        _lib.ct_plan_destroy(plan)
    gpu = {"v": vo.cpu().numpy(), "ha": ha.cpu().numpy(), "ia": ia.cpu().numpy(), "fa": fa.cpu().numpy()}
    m = G.compare(gpu, ora)
    assert m["ha_max"] <= 1e-3 and m["ia_max"] <= 1e-3 and m["fa_max"] <= 1e-5, m


# ------------------------------------------------------------------ fused
@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_fused_helix64_matches_oracle(prec):
    W, vol, _, cen, ax = _helix64()
    ora = O.pipeline(vol, W.sigma, W.rho, cen, ax)
    gpu = G.fused(vol, W.sigma, W.rho, cen, ax, precision=prec)
    m = G.compare(gpu, ora, precision=prec)
    print("helix64", prec, m)
    # the FP32 form meets the HA bound literally on every graded voxel
    G.assert_within(m, f"helix64 prec={prec}", literal_ha=(prec == FP32), precision=prec)


@pytest.mark.parametrize("shape,sigma,rho,prec", [((23, 29, 37), 1.0, 2.0, FP32), ((40, 17, 70), 1.5, 3.0, MIXED),
                                                  ((33, 41, 35), 2.0, 6.0, FP32)])
def test_fused_ragged_masked(shape, sigma, rho, prec):
    vol = _rand_vol(shape, seed=7 + shape[0])
    rng = np.random.default_rng(8)
    mask = (rng.random(shape) > 0.3).astype(np.uint8)
    cen = (shape[2] / 2 + 0.3, shape[1] / 2 - 0.2, 1.0)
    ax = (0.2, -0.1, 1.0)
    ora = O.pipeline(vol, sigma, rho, cen, ax, mask=mask)
    gpu = G.fused(vol, sigma, rho, cen, ax, mask=mask, precision=prec)
    G.assert_within(G.compare(gpu, ora, mask, precision=prec), f"ragged {shape}", literal_ha=(prec == FP32))
    out = ~mask.astype(bool)
    assert np.all(np.isnan(gpu["fa"][out])) and np.all(np.isnan(gpu["ha"][out])) and np.all(np.isnan(gpu["v"][:, out]))


@pytest.mark.parametrize("slab_bytes", [None, "1"])
@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_chunked_and_host_equal_whole_bit_exact(monkeypatch, prec, slab_bytes):
    # host streaming: the chunks of one x run share a slab of copies ("1": every
    # slab a single chunk); z-slab runs start with a short first slab (8 + 12, 20,
    # 20, 4 and 10 + 30, 24 planes here)
    if slab_bytes is not None:
        monkeypatch.setenv("CT_TUNE_SLAB_BYTES", slab_bytes)
    W, vol, _, cen, ax = _helix64()
    whole = G.fused(vol, W.sigma, W.rho, cen, ax, precision=prec)
    for chunk, on_host in [((24, 20, 28), False), ((0, 0, 17), False), ((32, 32, 32), True), ((0, 0, 0), True),
                           ((0, 0, 20), True), ((64, 64, 40), True), ((24, 40, 30), True)]:
        part = G.fused(vol, W.sigma, W.rho, cen, ax, precision=prec, chunk=chunk, on_host=on_host)
        for k in ("v", "ha", "ia", "fa"):
            np.testing.assert_array_equal(part[k], whole[k], err_msg=f"{k} chunk={chunk} host={on_host}")


def test_stage_path_equals_fused_path():
    # same kernels up to the eigen step; the eigen code is compiled into two
    # kernels whose FMA contraction may differ by an ulp
    W, vol, _, cen, ax = _helix64()
    st = G.stages(vol, W.sigma, W.rho, cen, ax)
    fu = G.fused(vol, W.sigma, W.rho, cen, ax)
    np.testing.assert_allclose(st["fa"], fu["fa"], rtol=0, atol=1e-6)
    sel = st["fa"] >= 0.1
    for k in ("ha", "ia"):
        d = np.abs((st[k] - fu[k] + 90.0) % 180.0 - 90.0)
        assert d[sel].max() <= 1e-3, k


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 9), (6, 1, 5), (4, 5, 1), (2, 3, 200)])
def test_degenerate_shapes(shape):
    vol = _rand_vol(shape, seed=11)
    cen, ax = (0.3, 0.4, 0.5), (0.0, 1.0, 1.0)
    ora = O.pipeline(vol, 1.0, 2.0, cen, ax)
    gpu = G.fused(vol, 1.0, 2.0, cen, ax)
    G.assert_within(G.compare(gpu, ora), f"shape {shape}")


def test_constant_volume_gives_zero_tensor_and_fa():
    vol = np.full((20, 21, 22), 1500, np.uint16)
    st = G.stages(vol, 1.0, 3.0, (10, 10, 10), (0, 0, 1))
    assert np.all(st["S"] == 0.0)
    assert np.all(st["fa"] == 0.0)
    fu = G.fused(vol, 1.0, 3.0, (10, 10, 10), (0, 0, 1), precision=MIXED)
    assert np.all(fu["fa"] == 0.0)


def test_output_encodings():
    W, vol, _, cen, ax = _helix64()
    ref = G.fused(vol, W.sigma, W.rho, cen, ax)
    h = G.fused(vol, W.sigma, W.rho, cen, ax, vec_type=_lib.CT_OUT_F16, angle_type=_lib.CT_OUT_F16,
                fa_type=_lib.CT_OUT_F16)
    np.testing.assert_allclose(h["fa"], ref["fa"], atol=1e-3)
    np.testing.assert_allclose(h["ha"], ref["ha"], atol=0.05)
    q = G.fused(vol, W.sigma, W.rho, cen, ax, angle_type=_lib.CT_OUT_U8Q, outputs=("ha", "ia"), raw=True)
    ora = O.pipeline(vol, W.sigma, W.rho, cen, ax)
    sel = ora["fa"] >= 0.1
    for k in ("ha", "ia"):
        code_o = np.rint((ora[k] + 90.0) * 256.0 / 180.0).astype(np.int64) % 256
        d = (q[k].astype(np.int64) - code_o) % 256
        d = np.minimum(d, 256 - d)
        assert d[sel].max() <= 1, k


def test_fill_value_and_on_axis():
    vol = _rand_vol((16, 17, 18), seed=12)
    cen, ax = (0.0, 8.0, 6.0), (1.0, 0.0, 0.0)  # voxels (x, 8, 6) lie on the axis
    gpu = G.fused(vol, 1.0, 2.0, cen, ax, fill=-5.0)
    assert np.all(gpu["ha"][6, 8, :] == -5.0) and np.all(gpu["ia"][6, 8, :] == -5.0)
    assert np.all(gpu["fa"][6, 8, :] >= 0.0)


def test_stats_count_voxels_and_launches():
    W, vol, _, cen, ax = _helix64()
    gpu = G.fused(vol, W.sigma, W.rho, cen, ax)
    assert gpu["stats"]["voxels"] == vol.size
    assert gpu["stats"]["launches"] >= 5


# ------------------------------------------------- full-size, sampled boxes
@pytest.fixture(scope="module")
def annulus512():
    W = synth.lv_annulus_512()
    vol, mask = synth.generate(W.spec)
    return W, vol, mask


def _sample_boxes(shape, R, rng):
    nz, ny, nx = shape
    b = 12
    boxes = [((0, 0, 0), (b, b, b)), ((nx - b, ny - b, nz - b), (b, b, b)), ((0, ny // 2, nz - b), (b, b, b)),
             ((nx // 2 - 120, ny // 2, nz // 2), (16, 16, 16)), ((nx // 2 + 200, ny // 2 - 8, nz // 3), (16, 16, 16))]
    for _ in range(3):
        lo = tuple(int(rng.integers(0, d - b)) for d in (nx, ny, nz))
        boxes.append((lo, (b, b, b)))
    return boxes


@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_full_size_annulus512_sampled(annulus512, prec):
    W, vol, mask = annulus512
    cen, ax = synth.frame_of(W.spec)
    gpu = G.fused(vol, W.sigma, W.rho, cen, ax, mask=mask, precision=prec)
    rng = np.random.default_rng(99)
    for lo, n in _sample_boxes(vol.shape, O.radius(W.sigma) + O.radius(W.rho), rng):
        ora = O.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask, lo=lo, n=n)
        sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
        sub = {k: (gpu[k][(slice(None),) + sl] if k == "v" else gpu[k][sl]) for k in ("v", "ha", "ia", "fa")}
        m = G.compare(sub, ora, mask[sl], precision=prec)
        G.assert_within(m, f"box {lo} {n} prec={prec}", precision=prec)
