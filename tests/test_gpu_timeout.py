"""A bounded wait that runs out is reported as CT_ERR_TIMEOUT, per plan, and
leaves the context usable.

The tensor-core passes wait on mbarriers for the other roles of their CTA
(staged operands, finished products, freed accumulators).  Each such wait
polls at most the plan's wait limit (CT_TUNE_TC_WAIT_LIMIT, read at plan
creation; 2^20 by default).  With the limit at 0 every such wait gives up at
once: the CTA raises its abort flag, the other roles stop, copies in flight
are drained, the last committed product is waited for, the tensor memory is
released and the plan's timeout word is incremented.  No fault, trap or hang
is involved: the wait simply returns without success and the kernel returns.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_07476_gb300 import _lib, build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import gpu_util as G  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


def _rand_vol(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(800, 2400, size=shape).astype(np.uint16)


def _force_tc(monkeypatch):
    monkeypatch.setenv("CT_TUNE_TC_RHO", "7")
    monkeypatch.setenv("CT_TUNE_TC_MIN_R", "0")
    monkeypatch.setenv("CT_TUNE_TC_ANY_BOX", "1")


def test_wait_limit_zero_reports_timeout_and_context_survives(monkeypatch):
    _force_tc(monkeypatch)
    vol = _rand_vol((24, 40, 64), 3)
    nz, ny, nx = vol.shape
    d_vol = G.dev_u16(vol)
    monkeypatch.setenv("CT_TUNE_TC_WAIT_LIMIT", "0")
    p = _lib.make_params(1.0, 3.0, (nx / 2, ny / 2, 0.0), (0.0, 0.0, 1.0))
    starved = _lib.ct_plan_create(p, (nx, ny, nz))
    bystander = None
    try:
        monkeypatch.delenv("CT_TUNE_TC_WAIT_LIMIT")
        bystander = _lib.ct_plan_create(p, (nx, ny, nz))
        S = torch.empty((6, nz, ny, nx), device="cuda")
        # every tensor-core pass (x form and y / z form) gives up its first wait
        _lib.ct_structure_tensor(starved, d_vol, (0, 0, 0), (nx, ny, nz), (0, 0, 0), (nx, ny, nz), S)
        with pytest.raises(_lib.CTError) as ei:
            _lib.ct_plan_sync(starved)
        assert ei.value.status == _lib.CT_ERR_TIMEOUT
        assert "gave up" in _lib.ct_last_error()
        # the word is per plan: another plan's sync does not see it, and it was cleared
        _lib.ct_plan_sync(bystander)
        _lib.ct_plan_sync(starved)
        # host items: the synchronous call itself reports it
        h_vol = torch.from_numpy(vol.view(np.int16)).pin_memory()
        fa = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
        with pytest.raises(_lib.CTError) as ei:
            _lib.ct_run_chunks(starved, [_lib.make_item(h_vol, (nx, ny, nz), None, None, None, None, fa)], True)
        assert ei.value.status == _lib.CT_ERR_TIMEOUT
        # the context is intact: the bystander plan computes the right tensor
        S2 = torch.empty((6, nz, ny, nx), device="cuda")
        _lib.ct_structure_tensor(bystander, d_vol, (0, 0, 0), (nx, ny, nz), (0, 0, 0), (nx, ny, nz), S2)
        _lib.ct_plan_sync(bystander)
        S_o = O.structure_tensor(vol, 1.0, 3.0)
        err = np.abs(S2.cpu().numpy() - S_o) / (S_o[0] + S_o[1] + S_o[2])[None]
        assert err.max() <= 2e-5
    finally:
        _lib.ct_plan_destroy(starved)
        if bystander is not None:
            _lib.ct_plan_destroy(bystander)
