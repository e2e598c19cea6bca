"""The device generator against the host generator (synth.py), box by box.

Both implement one seeded definition (SplitMix64 + Box-Muller, helix-rod
annulus, optional IA warp, Gaussian or Poisson-like noise) in FP64; the device
may contract multiply-adds and its transcendentals may differ from the host's
in the last bit, so a voxel may land on the other side of a rounding boundary:
at most 1 intensity unit, on a vanishing fraction of voxels.
"""
import numpy as np
import pytest

from paper_2508_07476_gb300 import _lib, build, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _device_box(spec, lo, n):
    nz, ny, nx = spec.shape
    v = torch.empty((n[2], n[1], n[0]), dtype=torch.int16, device="cuda")
    m = torch.empty((n[2], n[1], n[0]), dtype=torch.uint8, device="cuda")
    _lib.ct_synth_annulus(spec, (nx, ny, nz), lo, n, v, m)
    torch.cuda.synchronize()
    return v.cpu().numpy().view(np.uint16), m.cpu().numpy()


@pytest.mark.parametrize("wl", [synth.single_chunk_64(), synth.lv_annulus_512(96)])
def test_device_generator_matches_host(wl):
    spec = wl.spec
    nz, ny, nx = spec.shape
    ref, mref = synth.generate(spec)
    full, mfull = _device_box(spec, (0, 0, 0), (nx, ny, nz))
    d = np.abs(full.astype(np.int64) - ref.astype(np.int64))
    assert d.max() <= 1 and (d > 0).mean() < 1e-4, (d.max(), (d > 0).mean())
    assert (mfull != mref).mean() < 1e-5
    # a box of the volume equals the same box of the whole
    lo, n = (5, 9, 13), (31, 17, 23)
    box, mbox = _device_box(spec, lo, n)
    sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
    np.testing.assert_array_equal(box, full[sl])
    np.testing.assert_array_equal(mbox, mfull[sl])
