"""The allocation-free eigen entry point against the allocating one.

ct_eig_smallest_noalloc exists for callers that may not allocate device
memory (their framework owns it, or allocation is forbidden once they run);
it keeps its re-solve list in a fixed array of the library instead of plan
scratch.  Two calls in a row, on different inputs, must agree with
ct_eig_smallest within the tolerances of the eigen-stage parity test; this
also shows that the second call starts from cleared counters.  The file is
named to run last.
"""
import numpy as np
import pytest

from paper_2508_07476_gb300 import _lib, build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_VOXELS = 1 << 20


def _tensors(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    lam = np.sort(rng.uniform(0.0, 1.0, size=(n, 3)) * 10 ** rng.uniform(-1, 5, size=(n, 1)), axis=1)
    k = n // 4  # a quarter with a near-degenerate smallest pair: they take the re-solve list
    lam[:k, 1] = lam[:k, 0] * (1 + 10 ** rng.uniform(-6, -2, size=k))
    A = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    S = np.stack([A[:, 0, 0], A[:, 1, 1], A[:, 2, 2], A[:, 0, 1], A[:, 0, 2], A[:, 1, 2]])
    return S.astype(np.float32)


def _angle_deg(u, v):
    u = u.astype(np.float64)
    v = v.astype(np.float64)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, v, axis=0), axis=0), np.abs((u * v).sum(0))))


@pytest.fixture(scope="module", autouse=True)
def _ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _lib.load()


@pytest.mark.parametrize("prec", [_lib.CT_PREC_FP32, _lib.CT_PREC_MIXED])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    for call, (n, seed) in enumerate([(300000, 21), (MAX_VOXELS, 22)]):
        S = torch.from_numpy(_tensors(n, seed)).cuda()
        ev_ref = torch.empty((3, n), device="cuda")
        v_ref = torch.empty((3, n), device="cuda")
        plan = _lib.ct_plan_create(_lib.make_params(1.0, 2.0, (0, 0, 0), (0, 0, 1), prec), (n, 1, 1))
        try:
            _lib.ct_eig_smallest(plan, S, n, ev_ref, v_ref)
            torch.cuda.synchronize()
        finally:
            _lib.ct_plan_destroy(plan)
        ev = torch.full((3, n), float("nan"), device="cuda")
        v = torch.full((3, n), float("nan"), device="cuda")
        _lib.ct_eig_smallest_noalloc(S, n, ev, v, prec)
        torch.cuda.synchronize()
        ev_r, v_r, ev_n, v_n = (t.cpu().numpy() for t in (ev_ref, v_ref, ev, v))
        scale = np.maximum(np.abs(ev_r[2]), 1e-30)
        assert np.all(np.isfinite(ev_n)) and np.all(np.isfinite(v_n)), f"call {call}"
        assert (np.abs(ev_n - ev_r) / scale).max() <= 3e-4, f"call {call}"
        assert _angle_deg(v_n, v_r).max() <= 0.5, f"call {call}"


def test_noalloc_rejects_more_than_its_limit():
    S = torch.zeros((6, 1), device="cuda")
    with pytest.raises(_lib.CTError) as ei:
        _lib.ct_eig_smallest_noalloc(S, MAX_VOXELS + 1, None, S)
    assert ei.value.status == _lib.CT_ERR_INVALID
    assert "exceeds" in _lib.ct_last_error()
