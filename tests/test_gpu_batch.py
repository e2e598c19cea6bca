"""Batches of uneven volumes and caller-chunked boxes through the C ABI.

A batch (ct_run_chunks with several device items) runs inside one captured
CUDA graph: the items on the FP32 stencil chain as one persistent launch per
stage and tap set (CTAs taking (item, block) work from a device counter, in
waves that fit the plan's scratch budget), the others as their own launch
sequences on side streams.  Each item's outputs must equal, bit for bit,
those of running the item alone, and match the oracle.  ct_run_box on padded
chunks must reproduce the whole-volume run bit for bit.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _alloc(shape):
    nz, ny, nx = shape
    return (torch.empty((3, nz, ny, nx), device="cuda"), torch.empty((nz, ny, nx), device="cuda"),
            torch.empty((nz, ny, nx), device="cuda"), torch.empty((nz, ny, nx), device="cuda"))


_MODES = {"graph": ("1", "0"), "persistent": ("1", "1"), "per_item": ("0", "0")}  # (graph, persistent)


def _run_batch(crops, vols, precision, mode: str):
    os.environ["CT_TUNE_BATCH_GRAPH"], os.environ["CT_TUNE_BATCH_PERSISTENT"] = _MODES[mode]
    try:
        plan = _lib.ct_plan_create(_lib.make_params(1.0, 2.0, (0, 0, 0), (0, 0, 1), precision), (1, 1, 1))
    finally:
        del os.environ["CT_TUNE_BATCH_GRAPH"]
        del os.environ["CT_TUNE_BATCH_PERSISTENT"]
    outs, items = [], []
    for w, v in zip(crops, vols):
        nz, ny, nx = w.spec.shape
        o = _alloc(w.spec.shape)
        outs.append(o)
        cen, ax = synth.frame_of(w.spec)
        items.append(_lib.make_item(v, (nx, ny, nz), None, *o, sigma=w.sigma, rho=w.rho, lv_center=cen, lv_axis=ax))
    try:
        _lib.ct_run_chunks(plan, items, False)
        torch.cuda.synchronize()
        s1 = _lib.ct_plan_stats(plan, reset=True)
        _lib.ct_run_chunks(plan, items, False)  # same item list: the cached graph replays
        torch.cuda.synchronize()
        s2 = _lib.ct_plan_stats(plan, reset=True)
    finally:
        _lib.ct_plan_destroy(plan)
    res = [{k: t.cpu().numpy() for k, t in zip(("v", "ha", "ia", "fa"), o)} for o in outs]
    return res, s1, s2


@pytest.mark.parametrize("prec", [_lib.CT_PREC_FP32, _lib.CT_PREC_MIXED])
def test_batch_graph_equals_items_alone_and_oracle(prec):
    crops = synth.crop_batch(count=6, seed=9, size_range=(20, 56), sigmas=(1.0, 1.5), rhos=(2.0, 3.0, 4.0))
    host = [synth.generate(w.spec)[0] for w in crops]
    vols = [G.dev_u16(h) for h in host]
    batched, s1, s2 = _run_batch(crops, vols, prec, "graph")
    pers, p1, p2 = _run_batch(crops, vols, prec, "persistent")
    seq, _, _ = _run_batch(crops, vols, prec, "per_item")
    for a, b in ((s1, s2), (p1, p2)):
        assert a["voxels"] == b["voxels"] == sum(h.size for h in host)
        assert b["launches"] == a["launches"] > 0
    assert p1["launches"] < s1["launches"]
    for w, h, b, p, q in zip(crops, host, batched, pers, seq):
        for k in ("v", "ha", "ia", "fa"):
            np.testing.assert_array_equal(b[k], q[k], err_msg=f"{w.name} {k}")
            np.testing.assert_array_equal(p[k], q[k], err_msg=f"{w.name} {k} (persistent)")
        cen, ax = synth.frame_of(w.spec)
        alone = G.fused(h, w.sigma, w.rho, cen, ax, precision=prec)
        for k in ("v", "ha", "ia", "fa"):
            np.testing.assert_array_equal(b[k], alone[k], err_msg=f"{w.name} {k} (alone)")
        ora = O.pipeline(h, w.sigma, w.rho, cen, ax)
        G.assert_within(G.compare(b, ora, precision=prec), w.name, precision=prec)


def test_run_box_chunks_equal_whole():
    W = synth.single_chunk_64()
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    whole = G.fused(vol, W.sigma, W.rho, cen, ax, mask=mask)
    nz, ny, nx = vol.shape
    h = O.radius(W.sigma) + O.radius(W.rho)
    plan = _lib.ct_plan_create(_lib.make_params(W.sigma, W.rho, cen, ax), (nx, ny, nz))
    got = {k: np.full_like(whole[k], -1.0) for k in ("v", "ha", "ia", "fa")}
    try:
        for z0 in range(0, nz, 24):
            for x0 in range(0, nx, 40):
                lo = (x0, 0, z0)
                n = (min(40, nx - x0), ny, min(24, nz - z0))
                ilo = tuple(max(0, a - h) for a in lo)
                ihi = tuple(min(d, a + b + h) for a, b, d in zip(lo, n, (nx, ny, nz)))
                ino = tuple(b - a for a, b in zip(ilo, ihi))
                sub = vol[ilo[2]:ihi[2], ilo[1]:ihi[1], ilo[0]:ihi[0]]
                msub = mask[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
                o = _alloc((n[2], n[1], n[0]))
                _lib.ct_run_box(plan, G.dev_u16(sub), ilo, ino, lo, n, G.dev_u8(msub), *o)
                torch.cuda.synchronize()
                sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
                for k, t in zip(("v", "ha", "ia", "fa"), o):
                    a = t.cpu().numpy()
                    if k == "v":
                        got[k][(slice(None),) + sl] = a
                    else:
                        got[k][sl] = a
    finally:
        _lib.ct_plan_destroy(plan)
    for k in ("v", "ha", "ia", "fa"):
        np.testing.assert_array_equal(got[k], whole[k], err_msg=k)


def _items(crops, vols, outs, with_mask):
    items = []
    for w, v, o in zip(crops, vols, outs):
        nz, ny, nx = w.spec.shape
        cen, ax = synth.frame_of(w.spec)
        m = G.dev_u8(synth.generate(w.spec)[1]) if with_mask else None
        items.append((_lib.make_item(v, (nx, ny, nz), m, *o, sigma=w.sigma, rho=w.rho, lv_center=cen, lv_axis=ax), m))
    return items


PERSISTENT = {"CT_TUNE_BATCH_PERSISTENT": "1"}  # the persistent form is opt-in


def _batch_outputs(monkeypatch, crops, vols, prec, env, types, with_mask=False):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    vt, at, ft = types
    plan = _lib.ct_plan_create(_lib.make_params(1.0, 2.0, (0, 0, 0), (0, 0, 1), prec, vt, at, ft), (1, 1, 1))
    for k in env:
        monkeypatch.delenv(k)
    dt = {_lib.CT_OUT_F32: torch.float32, _lib.CT_OUT_F16: torch.float16, _lib.CT_OUT_U8Q: torch.uint8}
    outs = []
    for w in crops:
        nz, ny, nx = w.spec.shape
        outs.append((torch.full((3, nz, ny, nx), -7, dtype=dt[vt], device="cuda"),
                     torch.full((nz, ny, nx), 7, dtype=dt[at], device="cuda"),
                     torch.full((nz, ny, nx), 7, dtype=dt[at], device="cuda"),
                     torch.full((nz, ny, nx), -7, dtype=dt[ft], device="cuda")))
    pairs = _items(crops, vols, outs, with_mask)
    try:
        _lib.ct_run_chunks(plan, [p[0] for p in pairs], False)
        torch.cuda.synchronize()
        st = _lib.ct_plan_stats(plan, reset=True)
    finally:
        _lib.ct_plan_destroy(plan)
    return [[t.cpu().numpy() for t in o] for o in outs], st


@pytest.mark.parametrize("types", [(_lib.CT_OUT_F32,) * 3, (_lib.CT_OUT_F16,) * 3,
                                   (_lib.CT_OUT_F32, _lib.CT_OUT_U8Q, _lib.CT_OUT_F16)])
@pytest.mark.parametrize("with_mask", [False, True])
def test_persistent_batch_equals_per_item_launches(monkeypatch, types, with_mask):
    # every sigma and rho of the uneven crops (R_sigma 4..12, R_rho 8..32), masks
    # (compacted eigen stage) or none, the three output encodings; waves of
    # several items and of one item each; and, with the tensor cores forced
    # for R_rho >= 24, a batch mixing persistent items with per-item launches
    crops = synth.crop_batch(count=10, seed=21, size_range=(24, 72))
    host = [synth.generate(w.spec)[0] for w in crops]
    vols = [G.dev_u16(h) for h in host]
    prec = _lib.CT_PREC_MIXED
    ref, st_ref = _batch_outputs(monkeypatch, crops, vols, prec, {"CT_TUNE_BATCH_PERSISTENT": "0"}, types, with_mask)
    for env in ({}, {"CT_TUNE_BATCH_BYTES": "1"}, {"CT_TUNE_BATCH_GRAPH": "0"},
                {"CT_TUNE_TC_ANY_BOX": "1", "CT_TUNE_TC_MIN_R": "24", "CT_TUNE_BATCH_BYTES": "20000000"}):
        env = dict(env, **PERSISTENT)
        if "CT_TUNE_TC_ANY_BOX" in env:
            ref_env = dict(env, CT_TUNE_BATCH_PERSISTENT="0")
            ref, _ = _batch_outputs(monkeypatch, crops, vols, prec, ref_env, types, with_mask)
        got, st = _batch_outputs(monkeypatch, crops, vols, prec, env, types, with_mask)
        assert st["voxels"] == st_ref["voxels"]
        for w, a, b in zip(crops, got, ref):
            for k, x, y in zip(("v", "ha", "ia", "fa"), a, b):
                np.testing.assert_array_equal(x, y, err_msg=f"{w.name} {k} {env}")
    # the persistent form launches once per stage, tap set and CTA shape (the x / y
    # pass at two widths, the z pass at up to four shapes) and once per wave for the
    # eigen stage and the re-solve: fewer than a launch sequence per crop
    _, st_p = _batch_outputs(monkeypatch, crops, vols, prec, PERSISTENT, types, with_mask)
    n_sets = len({(w.sigma, w.rho) for w in crops})
    assert st_p["launches"] <= 8 * n_sets + 3 and st_p["launches"] < st_ref["launches"], (st_p, st_ref, n_sets)


def test_persistent_batch_matches_oracle(monkeypatch):
    crops = synth.crop_batch(count=6, seed=33, size_range=(24, 64), sigmas=(1.0, 3.0), rhos=(2.0, 8.0))
    host = [synth.generate(w.spec)[0] for w in crops]
    vols = [G.dev_u16(h) for h in host]
    for prec in (_lib.CT_PREC_FP32, _lib.CT_PREC_MIXED):
        got, _ = _batch_outputs(monkeypatch, crops, vols, prec, PERSISTENT, (_lib.CT_OUT_F32,) * 3)
        for w, h, o in zip(crops, host, got):
            cen, ax = synth.frame_of(w.spec)
            ora = O.pipeline(h, w.sigma, w.rho, cen, ax)
            gpu = dict(zip(("v", "ha", "ia", "fa"), o))
            G.assert_within(G.compare(gpu, ora, precision=prec), f"persistent {w.name} prec={prec}", precision=prec)
