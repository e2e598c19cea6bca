"""The autotuner through the C ABI: ct_autotune times the candidate kernel
choices on a synthetic volume, stores the best under the GPU's name and the
volume's key, and plans created with that cache take the stored choice, with
results still inside the oracle tolerances and chunked runs still equal to the
whole volume bit for bit."""
import json

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


def _names(vol, mask, sigma, rho, cen, ax, prec):
    nz, ny, nx = vol.shape
    plan = _lib.ct_plan_create(_lib.make_params(sigma, rho, cen, ax, prec), (nx, ny, nz))
    try:
        _lib.ct_plan_profile(plan, True)
        fa = torch.empty((nz, ny, nx), device="cuda")
        _lib.ct_run_chunks(plan, [_lib.make_item(G.dev_u16(vol), (nx, ny, nz), G.dev_u8(mask), None, None, None, fa)],
                           False)
        torch.cuda.synchronize()
        return set(_lib.ct_plan_kernel_times(plan))
    finally:
        _lib.ct_plan_destroy(plan)


@pytest.mark.parametrize("prec", [_lib.CT_PREC_MIXED, _lib.CT_PREC_FP32])
def test_autotune_stores_a_choice_that_plans_follow(tmp_path, monkeypatch, prec):
    cache = tmp_path / "cache.json"
    W = synth.single_chunk_64()
    spec = synth.AnnulusSpec(shape=(48, 80, 96), r_in=12.0, r_out=30.0, period=6.0, ha_in_deg=60.0, ha_out_deg=-60.0,
                             noise=("gauss", 50.0), seed=3)
    vol, mask = synth.generate(spec)
    cen, ax = synth.frame_of(spec)
    sigma, rho = 1.0, 6.0
    nz, ny, nx = vol.shape
    p = _lib.make_params(sigma, rho, cen, ax, prec)
    r = _lib.ct_autotune(p, (nx, ny, nz), True, str(cache))
    assert r["candidates"] >= 8
    assert 0 < r["ms"] <= r["default_ms"] * 1.2  # the best candidate is no slower than the defaults, within noise
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    e = entries[0]
    assert e["gpu"] == torch.cuda.get_device_name(0)
    assert (e["precision"], e["rs"], e["rr"], e["xclass"]) == (prec, 4, 24, 8)
    assert (e["rho_path"], e["seg_cap"], e["stream_block"], e["eig_compact"]) == \
        (r["rho_path"], r["seg_cap"], r["stream_block"], r["eig_compact"])
    # tuning the same key again replaces the entry
    _lib.ct_autotune(p, (nx, ny, nz), True, str(cache))
    assert len(json.loads(cache.read_text())) == 1
    # a plan reading the cache takes the stored rho path
    monkeypatch.setenv("CT_TUNE_CACHE", str(cache))
    names = _names(vol, mask, sigma, rho, cen, ax, prec)
    tc = any(k.startswith("rho_") and "_tc" in k for k in names)
    assert tc == (r["rho_path"] > 0), (r, names)
    if r["rho_path"] == 2:
        assert any(k.startswith("rho_z_tc_g") for k in names), names
    # and stays inside the tolerances, chunks equal to the whole
    ora = O.pipeline(vol, sigma, rho, cen, ax, mask=mask)
    whole = G.fused(vol, sigma, rho, cen, ax, mask=mask, precision=prec)
    G.assert_within(G.compare(whole, ora, mask, precision=prec), f"tuned prec={prec}", precision=prec)
    part = G.fused(vol, sigma, rho, cen, ax, mask=mask, precision=prec, chunk=(40, 32, 20))
    for k in ("v", "ha", "ia", "fa"):
        np.testing.assert_array_equal(part[k], whole[k], err_msg=k)


def test_autotune_on_a_chunk_of_a_large_volume(tmp_path):
    # the key is the volume's; only the chunk and its halo are generated and timed
    cache = tmp_path / "c.json"
    p = _lib.make_params(2.0, 8.0, (1023.5, 1023.5, 511.5), (0.0, 0.0, 1.0), _lib.CT_PREC_MIXED, _lib.CT_OUT_F16,
                         _lib.CT_OUT_F16, _lib.CT_OUT_F16)
    r = _lib.ct_autotune(p, (2048, 2048, 1024), True, str(cache), chunk=(128, 128, 128))
    e = json.loads(cache.read_text())[0]
    assert e["vox_log2"] == 32 and e["rr"] == 32 and r["ms"] > 0
