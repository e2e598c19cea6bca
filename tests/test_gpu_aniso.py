"""Anisotropic voxels and a per-slice LV centreline on the GPU, against the
FP64 oracle's anisotropic form (pinned in test_oracle_aniso.py)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402

FP32, MIXED = _lib.CT_PREC_FP32, _lib.CT_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


@pytest.fixture(scope="module")
def helix():
    W = synth.single_chunk_64()
    vol, _ = synth.generate(W.spec)
    return W, vol[4:60, 2:62, 0:64].copy()  # 64 x 60 x 56 (x, y, z)


def _centre(vol, sp):
    nz, ny, nx = vol.shape
    return ((nx - 1) / 2 * sp[0], (ny - 1) / 2 * sp[1], (nz - 1) / 2 * sp[2])


def test_unit_spacing_is_bit_identical(helix):
    W, vol = helix
    c = _centre(vol, (1, 1, 1))
    a = G.fused(vol, W.sigma, W.rho, c, (0, 0, 1))
    b = G.fused(vol, W.sigma, W.rho, c, (0, 0, 1), spacing=(1.0, 1.0, 1.0))
    for k in ("v", "ha", "ia", "fa"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("prec", [FP32, MIXED])
@pytest.mark.parametrize("sp", [(1.0, 1.25, 0.8), (0.6, 0.6, 1.5)])
def test_anisotropic_matches_oracle(helix, prec, sp):
    W, vol = helix
    sigma, rho = W.sigma * sp[0], W.rho * sp[0]  # scales in the spacing's units
    c = _centre(vol, sp)
    ax = (0.05, 0.0, 1.0)
    mask = np.ones(vol.shape, np.uint8)
    mask[:, :5, :] = 0
    ora = O.pipeline(vol, sigma, rho, c, ax, mask=mask, spacing=sp)
    gpu = G.fused(vol, sigma, rho, c, ax, mask=mask, precision=prec, spacing=sp)
    m = G.compare(gpu, ora, mask, precision=prec)
    print("aniso", sp, prec, m)
    G.assert_within(m, f"aniso {sp} prec={prec}")


def test_centreline_matches_oracle_and_chunks(helix):
    W, vol = helix
    sp = (1.0, 1.0, 1.2)
    nz = vol.shape[0]
    base = _centre(vol, sp)
    cen = [(base[0] + 0.08 * (k - nz / 2), base[1] - 0.05 * (k - nz / 2)) for k in range(nz)]
    ora = O.pipeline(vol, W.sigma, W.rho, base, (0, 0, 1), spacing=sp, centres=np.array(cen))
    whole = G.fused(vol, W.sigma, W.rho, base, (0, 0, 1), spacing=sp, lv_centres=cen)
    m = G.compare(whole, ora, precision=FP32)
    G.assert_within(m, "centreline")
    # per-axis halos: chunked = whole, bit for bit (device and host-streamed)
    for on_host in (False, True):
        ch = G.fused(vol, W.sigma, W.rho, base, (0, 0, 1), spacing=sp, lv_centres=cen, chunk=(24, 40, 17),
                     on_host=on_host)
        for k in ("v", "ha", "ia", "fa"):
            np.testing.assert_array_equal(ch[k], whole[k])


def test_invalid_spacing_is_rejected():
    for sp in ((-1.0, 1.0, 1.0), (1.0, float("nan"), 1.0), (1.0, 1.0, float("inf"))):
        with pytest.raises(_lib.CTError):
            _lib.ct_plan_create(_lib.make_params(1.0, 3.0, (0, 0, 0), (0, 0, 1), spacing=sp), (8, 8, 8))
    with pytest.raises(_lib.CTError):
        _lib.ct_plan_create(_lib.make_params(1.0, 3.0, (0, 0, 0), (0, 0, 1),
                                             lv_centres=[(0.0, float("nan"))] * 8), (8, 8, 8))
