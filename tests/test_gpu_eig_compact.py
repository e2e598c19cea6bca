"""The masked eigen stage over compacted inside voxels (each row segment lists
its inside voxels, then solves them with full warps) against the one-thread-
per-voxel form: the same arithmetic per voxel, so every output agrees bit for
bit, including the fill outside the mask, the re-solved near-degenerate voxels
and every output encoding; and both against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402

F32, F16, U8Q = _lib.CT_OUT_F32, _lib.CT_OUT_F16, _lib.CT_OUT_U8Q


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _both(monkeypatch, *args, **kw):
    out = {}
    for on in (0, 1):
        monkeypatch.setenv("CT_TUNE_EIG_COMPACT", str(on))
        out[on] = G.fused(*args, raw=True, **kw)
    return out[0], out[1]


def _vol_and_mask(shape, seed, density):
    rng = np.random.default_rng(seed)
    import scipy.ndimage as ndi
    v = ndi.gaussian_filter(rng.integers(500, 3000, size=shape).astype(np.float64), 1.2)
    vol = np.clip(np.rint(v + rng.normal(0, 20, size=shape)), 0, 65535).astype(np.uint16)
    vol[:, :, : shape[2] // 5] = 1500  # a constant slab: zero and near-degenerate tensors (the re-solve list)
    mask = (rng.random(shape) < density).astype(np.uint8)
    return vol, mask


@pytest.mark.parametrize("shape", [(9, 7, 600), (5, 11, 512), (6, 5, 37), (3, 4, 1025)])
@pytest.mark.parametrize("density", [0.0, 0.3, 1.0])
def test_compact_equals_per_voxel(monkeypatch, shape, density):
    vol, mask = _vol_and_mask(shape, sum(shape), density)
    cen, ax = (shape[2] / 2 + 0.3, shape[1] / 2 - 0.2, 1.0), (0.1, 0.0, 1.0)
    a, b = _both(monkeypatch, vol, 1.0, 2.0, cen, ax, mask=mask)
    for k in ("v", "ha", "ia", "fa"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["stats"]["fallback_voxels"] == b["stats"]["fallback_voxels"]


@pytest.mark.parametrize("types", [(F16, F16, F16), (-1, U8Q, F16), (F16, F32, F32)])
def test_compact_encodings_and_frames(monkeypatch, types):
    vt, at, ft = types
    vol, mask = _vol_and_mask((8, 9, 300), 3, 0.5)
    outputs = ("ha", "ia", "fa") if vt < 0 else ("v", "ha", "ia", "fa")
    kw = dict(mask=mask, vec_type=max(vt, F32), angle_type=at, fa_type=ft, outputs=outputs)
    cen, ax = (150.0, 4.0, 4.0), (0.0, 0.2, 1.0)
    for extra in ({}, {"spacing": (1.0, 1.2, 0.8)}, {"lv_centres": [(150.0 + 0.1 * k, 4.0) for k in range(8)]}):
        a, b = _both(monkeypatch, vol, 1.0, 2.0, cen, ax, **kw, **extra)
        for k in outputs:
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} {extra}")


def test_compact_matches_oracle_on_the_wall(monkeypatch):
    monkeypatch.setenv("CT_TUNE_EIG_COMPACT", "1")
    W = synth.single_chunk_64()
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    ora = O.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask)
    gpu = G.fused(vol, W.sigma, W.rho, cen, ax, mask=mask)
    G.assert_within(G.compare(gpu, ora, mask), "compact eigen stage")
    out = ~mask.astype(bool)
    assert np.all(np.isnan(gpu["fa"][out])) and np.all(np.isnan(gpu["ha"][out]))
    assert math.isnan(float(gpu["v"][0][out][0]))
