"""Tractography kernel (ct_track) against the FP64 oracle (oracle/tracks.py).

Fields are written by numpy (analytic), so no oracle input comes from the
CUDA path; the pipeline-driven case feeds each side its own pipeline's
output.  The kernel integrates in FP32: points agree to a small fraction of a
voxel, and a track's length may differ by one step only where a point lands
within rounding of a stopping boundary (checked against the oracle's step
margins).
"""
import math

import numpy as np
import pytest

from oracle import oracle, tracks
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


def _gpu_tracks(vec, seeds, h, max_steps, fa=None, mask=None, fa_min=0.0, max_turn_deg=90.0):
    _, nz, ny, nx = vec.shape
    p = _lib.make_track_params(h, max_steps, fa_min, max_turn_deg)
    d_vec = torch.from_numpy(np.ascontiguousarray(vec, dtype=np.float32)).cuda()
    d_fa = None if fa is None else torch.from_numpy(np.ascontiguousarray(fa, dtype=np.float32)).cuda()
    d_mask = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    s = np.asarray(seeds, dtype=np.float32).reshape(-1, 3)
    d_seeds = torch.from_numpy(s).cuda()
    pts = torch.zeros((len(s), 2, max_steps + 1, 3), dtype=torch.float32, device="cuda")
    cnt = torch.zeros((len(s), 2), dtype=torch.int32, device="cuda")
    _lib.ct_track(p, (nx, ny, nz), d_vec, d_fa, d_mask, d_seeds, len(s), pts, cnt)
    torch.cuda.synchronize()
    return pts.cpu().numpy(), cnt.cpu().numpy()


def _compare(gpu, ora, atol, margins=None):
    """Share of tracks whose lengths agree; every common point within atol.  A
    track may be one step longer on either side only where the oracle's step
    at that point lies within rounding of a stopping threshold: its margin
    (oracle.tracks, in voxels, cosine or FA units) must be below 10 atol."""
    pts, cnt = gpu
    same, worst, n = 0, 0.0, 0
    for i, (fwd, bwd) in enumerate(ora):
        for k, tr in enumerate((fwd, bwd)):
            n += 1
            c = int(cnt[i, k])
            assert abs(c - len(tr)) <= 1, (i, k, c, len(tr))
            m = min(c, len(tr))
            if m:
                worst = max(worst, float(np.abs(pts[i, k, :m] - np.array(tr[:m], dtype=np.float64)).max()))
            same += c == len(tr)
            if margins is not None and c != len(tr):
                mg = margins[i][k][m - 1]  # the step attempted from the last common point
                assert mg < 10 * atol, (i, k, c, len(tr), mg)
    assert worst < atol, worst
    return same / n


def _helix_field(n, c, pitch):
    """Unit field of helices about the z axis through (c, c): e_theta cos a + e_z sin a."""
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    dx, dy = x - c, y - c
    r = np.hypot(dx, dy)
    r[r == 0] = 1.0
    a = np.arctan2(pitch, r)
    f = np.stack([-dy / r * np.cos(a), dx / r * np.cos(a), np.sin(a) * np.ones_like(r)])
    return f


def test_tracks_match_oracle_on_a_helix_field():
    n = 48
    f = _helix_field(n, 23.5, 4.0)
    rng = np.random.default_rng(3)
    seeds = np.column_stack([rng.uniform(8, 40, 60), rng.uniform(8, 40, 60), rng.uniform(4, 44, 60)])
    mg = []
    ora = tracks.tracks(f, seeds, 0.5, 80, margins=mg)
    gpu = _gpu_tracks(f, seeds, 0.5, 80)
    assert _compare(gpu, ora, 2e-3, mg) >= 0.98


def test_stopping_rules_match_oracle():
    n = 40
    f = np.zeros((3, 6, n, n))
    f[0] = 1.0
    f[0, :, :, 25:] = 0.0
    f[1, :, :, 25:] = 1.0  # a 90 degree bend at x = 25
    fa = np.ones((6, n, n))
    fa[:, 30:, :] = 0.0
    mask = np.ones((6, n, n), np.uint8)
    mask[:, :4, :] = 0
    rng = np.random.default_rng(4)
    seeds = np.column_stack([rng.uniform(1, 38, 50), rng.uniform(5, 35, 50), rng.uniform(1, 4, 50)])
    for turn, fa_min in ((20.0, 0.5), (90.0, 0.5), (90.0, 0.0)):
        mg = []
        ora = tracks.tracks(f, seeds, 0.4, 120, fa=fa, mask=mask, fa_min=fa_min, max_turn_deg=turn, margins=mg)
        gpu = _gpu_tracks(f, seeds, 0.4, 120, fa=fa, mask=mask, fa_min=fa_min, max_turn_deg=turn)
        assert _compare(gpu, ora, 1e-3, mg) >= 0.98


def test_orientation_sign_is_ignored_exactly():
    n = 40
    f = _helix_field(n, 19.5, 3.0)
    flips = np.where(np.random.default_rng(5).random((n, n, n)) < 0.5, -1.0, 1.0)
    seeds = [(10.2, 19.0, 5.0), (30.0, 25.5, 20.0)]
    a = _gpu_tracks(f, seeds, 0.5, 60)
    b = _gpu_tracks(f * flips[None], seeds, 0.5, 60)
    # a flip at the seed's nearest voxel swaps which track is called forward
    for i in range(len(seeds)):
        order = (0, 1) if np.array_equal(a[0][i, 0], b[0][i, 0]) else (1, 0)
        for k in range(2):
            assert a[1][i, k] == b[1][i, order[k]] > 10
            np.testing.assert_array_equal(a[0][i, k, :a[1][i, k]], b[0][i, order[k], :a[1][i, k]])


def test_seed_cases_and_invalid_arguments():
    f = np.zeros((3, 4, 4, 4))
    f[0] = 1.0
    f[:, 1, 1, 1] = np.nan
    pts, cnt = _gpu_tracks(f, [(9.0, 1.0, 1.0), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), (float("nan"), 1.0, 1.0)], 0.5, 4)
    assert cnt[0].tolist() == [0, 0] and cnt[1].tolist() == [1, 1] and cnt[3].tolist() == [0, 0]
    assert cnt[2, 0] >= 1 and cnt[2, 1] >= 1
    vec = torch.zeros((3, 4, 4, 4), device="cuda")
    buf = torch.zeros(64, device="cuda")
    c = torch.zeros(2, dtype=torch.int32, device="cuda")
    s = torch.zeros((1, 3), device="cuda")
    for p, dims in ((_lib.make_track_params(0.0, 4), (4, 4, 4)), (_lib.make_track_params(0.5, 0), (4, 4, 4)),
                    (_lib.make_track_params(0.5, 4), (1, 4, 4))):
        with pytest.raises(_lib.CTError):
            _lib.ct_track(p, dims, vec, None, None, s, 1, buf, c)


def test_tracks_through_the_pipeline_output():
    """GPU pipeline + GPU tracks vs oracle pipeline + oracle tracks on the same
    volume: short tracks from seeds in the wall agree closely."""
    W = synth.lv_annulus_512(96)
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    ora = oracle.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask)
    g = fused(vol, W.sigma, W.rho, cen, ax, mask=mask, precision=_lib.CT_PREC_FP32)
    rng = np.random.default_rng(6)
    zz, yy, xx = np.nonzero(mask[10:86, 10:86, 10:86])
    pick = rng.choice(len(xx), 40, replace=False)
    seeds = np.column_stack([xx[pick] + 10.3, yy[pick] + 10.2, zz[pick] + 10.1])
    ot = tracks.tracks(ora["v"], seeds, 0.5, 12, fa=ora["fa"], mask=mask, fa_min=0.1, max_turn_deg=45.0)
    gt = _gpu_tracks(g["v"], seeds, 0.5, 12, fa=g["fa"], mask=mask, fa_min=0.1, max_turn_deg=45.0)
    pts, cnt = gt
    agree, worst = 0, 0.0
    for i, (fwd, bwd) in enumerate(ot):
        for k, tr in enumerate((fwd, bwd)):
            if int(cnt[i, k]) == len(tr):
                agree += 1
                worst = max(worst, float(np.abs(pts[i, k, :len(tr)] - np.array(tr)).max()))
    assert agree >= 0.9 * 2 * len(seeds)
    assert worst < 0.05, worst
