#!/usr/bin/env python
"""Throughput of the per-voxel orientation pipeline on GB300.

One step = the whole hot path (sigma-gradient, rho-smoothed structure tensor,
eigen-solve, HA / IA / FA under the mask) over one 512^3 uint16 volume: the
left-ventricle-like annulus (radii 120/220, axis tilted 10 deg, period 6,
HA +70 -> -70, IA field 5 deg / 40 voxels, Poisson-like 5% noise, annulus mask),
sigma = 2, rho = 6, FP32 outputs.  Inputs are seeded synthetic volumes
(no scan data ships with the library).

Arms
  --impl ours (default): the CUDA library through its C ABI.  Both arithmetic
      forms are timed; the headline `value` is the mixed form (FP16-held
      gradient, FP32 sums, FP32 closed-form eigen with FP64 re-solve), the
      FP32 form is reported beside it.  `e2e` times the same call with host
      buffers (pinned), copies inside the timed region.
  --impl reference: the FP64 CPU oracle on the host cores, each step a bounded
      sample (a box of the same volume), as the baseline arm.

Timing: CUDA events on the launching stream, W warm-up steps, K timed steps,
barrier + synchronize on both sides, max over ranks.  The volume plus the
plan's scratch (6.4 GB per step) exceed the 129 MB L2, so no flush is needed.
Under torchrun every rank runs its own volume (weak scaling, no collective on
the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxels/s for tensor+eigen+HA/IA/FA at 1 GB300, mixed vs FP32 form at ≤0.5°; % roofline"
UNIT = "voxels/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=512, help="cube edge (512 = the measured workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-zchunk", type=int, default=128, help="z extent of the slabs of the e2e call (0 = whole)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", choices=["annulus512", "crops200", "stream2048", "tera4096"], default="annulus512",
                    help="annulus512 (default, the headline line) or one of the other workload shapes")
    ap.add_argument("--crops", type=int, default=200)
    ap.add_argument("--zplanes", type=int, default=0, help="stream2048/tera4096: limit the z extent (0 = full)")
    ap.add_argument("--split", choices=["replicas", "zslab"], default="replicas",
                    help="under torchrun: one volume per rank (replicas, weak scaling) or one volume split in "
                         "z-slabs with their halos (zslab, strong scaling)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def _workload(size: int):
    from paper_2508_07476_gb300 import synth
    W = synth.lv_annulus_512(size)
    return W


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value over the ranks (the step time the job is charged with)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_voxels_per_s(voxels_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank processes its own volume (weak scaling)."""
    return world * voxels_per_rank / (ms_max * 1e-3)


def _fma_per_voxel(rs: int, rr: int) -> int:
    """Algorithmic FMAs per interior voxel: 8 sigma passes, 6 products, 18 rho passes."""
    return 8 * (2 * rs + 1) + 6 + 18 * (2 * rr + 1)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _fma_rate_measured(local: int) -> dict:
    """The device's FP32 FMA rate, measured live (ct_fp32_fma_rate: independent
    FMA chains on every SM, CUDA events), with the SM clock sampled meanwhile."""
    from paper_2508_07476_gb300 import _lib
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    best = None
    for _ in range(3):
        r = _lib.ct_fp32_fma_rate(1_000_000)
        if best is None or r["fma_per_s"] > best["fma_per_s"]:
            best = r
    clocks = sampler.stop()
    return {"fma_per_s": best["fma_per_s"], "sms": best["sms"], "kernel_ms": best["ms"],
            "sm_mhz_median": clocks.get("sm_mhz"), "reasons": clocks.get("reasons"),
            "fma_per_sm_per_clock": best["fma_per_s"] / best["sms"] / (clocks["sm_mhz"] * 1e6)
            if clocks.get("sm_mhz") else None,
            "source": "measured live: ct_fp32_fma_rate (16 independent FMA chains per thread, one full wave of "
                      "CTAs on every SM, best of 3, CUDA events)"}


# ------------------------------------------------------------- accuracy legs
EPS_S = {0: 1e-5, 1: 1e-3}  # worst-case relative tensor error of the FP32 / mixed forms


def _u8q_code(deg):
    return np.rint((np.asarray(deg, dtype=np.float64) + 90.0) * 256.0 / 180.0).astype(np.int64) % 256


def _grade_box(ora: dict, out: dict, inside, prec: int, u8q: bool = False) -> dict:
    """One box of outputs against the oracle: fibre direction on FA >= 0.1 voxels
    inside the mask (literal 0.5 deg, and against the first-order bound
    eps_S tr S / (l2 - l1) where that is larger), HA / IA on the voxels whose
    direction is fixed to 0.5 deg (U8Q: code distance to the oracle's own
    quantisation), FA on every voxel inside."""
    sel = inside & (ora["fa"] >= 0.1) & np.isfinite(ora["ha"])
    r = {"graded": int(sel.sum()), "dir": 0.0, "dir_bound_excess": -1.0, "dir_over_05": 0, "ill": 0,
         "ha": 0.0, "ia": 0.0, "fa": 0.0, "ha_code": 0, "ia_code": 0}
    if inside.any():
        r["fa"] = float(np.abs(out["fa"][inside] - ora["fa"][inside]).max())
    if not sel.any():
        return r
    u, v = out["v"][:, sel].astype(np.float64), ora["v"][:, sel]
    d = np.degrees(np.arctan2(np.linalg.norm(np.cross(u, v, axis=0), axis=0), np.abs((u * v).sum(0))))
    ev = ora["evals"][:, sel]
    bound = np.maximum(0.5, np.degrees(EPS_S[prec] * ev.sum(0) / np.maximum(ev[1] - ev[0], 1e-300)))
    well = bound <= 0.5
    r.update(dir=float(d.max()), dir_bound_excess=float((d - bound).max()), dir_over_05=int((d > 0.5).sum()),
             ill=int((~well).sum()))
    ha_o, ia_o = ora["ha"][sel], ora["ia"][sel]
    flip = np.abs(ha_o) > 89.0
    if u8q:
        def dist(a, b):
            x = (a - b) % 256
            return np.minimum(x, 256 - x)
        ch, ci = out["ha"][sel].astype(np.int64), out["ia"][sel].astype(np.int64)
        dh = dist(ch, _u8q_code(ha_o))
        di = np.where(flip, np.minimum(dist(ci, _u8q_code(ia_o)), dist(ci, _u8q_code(-ia_o))),
                      dist(ci, _u8q_code(ia_o)))
        r["ha_code"] = int(dh[well].max()) if well.any() else 0
        r["ia_code"] = int(di[well].max()) if well.any() else 0
    else:
        dha = np.abs((out["ha"][sel] - ha_o + 90.0) % 180.0 - 90.0)
        dia = np.abs(out["ia"][sel] - ia_o)
        dia = np.where(flip, np.minimum(dia, np.abs(out["ia"][sel] + ia_o)), dia)
        g_ha = well & (np.abs(ia_o) <= 75.0)
        r["ha"] = float(dha[g_ha].max()) if g_ha.any() else 0.0
        r["ia"] = float(dia[well].max()) if well.any() else 0.0
    return r


def _merge(worst: dict, r: dict) -> dict:
    for k in ("dir", "dir_bound_excess", "ha", "ia", "fa", "ha_code", "ia_code"):
        worst[k] = max(worst.get(k, -1.0 if k == "dir_bound_excess" else 0), r[k])
    for k in ("graded", "dir_over_05", "ill"):
        worst[k] = worst.get(k, 0) + r[k]
    worst["boxes"] = worst.get("boxes", 0) + 1
    return worst


def _verdict(worst: dict, u8q: bool = False) -> dict:
    g = max(worst.get("graded", 0), 1)
    ok = worst.get("dir_bound_excess", -1.0) <= 0.0 and worst.get("fa", 0.0) <= 2e-3
    ok = ok and (worst.get("ha_code", 0) <= 1 and worst.get("ia_code", 0) <= 1 if u8q else
                 worst.get("ha", 0.0) <= 0.5 and worst.get("ia", 0.0) <= 0.5)
    worst["dir_over_05_frac"] = worst.get("dir_over_05", 0) / g
    worst["ill_frac"] = worst.get("ill", 0) / g
    worst["within_tolerance"] = bool(ok)
    return worst


def _decode(t) -> np.ndarray:
    a = t.cpu() if hasattr(t, "cpu") else t
    import torch
    return a.numpy() if a.dtype == torch.uint8 else a.float().numpy()


# ------------------------------------------------------------------ reference
def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle
    from paper_2508_07476_gb300 import synth
    W = _workload(args.size)
    n = args.size
    box = (min(128, n), min(128, n), min(64, n))
    h = oracle.radius(W.sigma) + oracle.radius(W.rho)
    rng = np.random.default_rng(2024)
    centre = synth.frame_of(W.spec)
    # one slab of the volume holds every sample box plus its halo
    z0 = max(0, n // 2 - box[2] // 2 - h)
    z1 = min(n, z0 + box[2] + 2 * h)
    vol_slab, mask_slab = synth.generate(W.spec, (z0, z1))
    vol = np.zeros((n, n, n), np.uint16)
    mask = np.zeros((n, n, n), np.uint8)
    vol[z0:z1] = vol_slab
    mask[z0:z1] = mask_slab
    zlo = min(max(0, n // 2 - box[2] // 2), n - box[2])

    def step():
        lo = (int(rng.integers(0, n - box[0] + 1)), int(rng.integers(0, n - box[1] + 1)), zlo)
        t = time.perf_counter()
        oracle.pipeline(vol, W.sigma, W.rho, centre[0], centre[1], mask=mask, lo=lo, n=box)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    per = float(np.mean(ts))
    value = box[0] * box[1] * box[2] / per
    cores = oracle.num_threads()
    sample = f"oracle (FP64, OpenMP) on a {box[0]}x{box[1]}x{box[2]} box of the {n}^3 volume per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded annulus volume)",
        "config": {"workload": W.name, "dims": [n, n, n], "sigma": W.sigma, "rho": W.rho, "mask": True},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------- ours
def _cpu_baseline(W, vol, mask, seconds: float) -> dict:
    """The oracle as it stands on this host's cores: all of them for `seconds`,
    then one core for a quarter of that, on 128 x 128 x 64 boxes of the volume."""
    from oracle import oracle
    from paper_2508_07476_gb300 import synth
    n = vol.shape[0]
    box = (min(128, n), min(128, n), min(64, n))
    cen, ax = synth.frame_of(W.spec)
    rng = np.random.default_rng(7)

    def timed(sec):
        done, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < sec:
            lo = tuple(int(rng.integers(0, d - b + 1)) for d, b in zip((n, n, n), box))
            oracle.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask, lo=lo, n=box)
            done += box[0] * box[1] * box[2]
        return done, time.perf_counter() - t0

    cores = oracle.num_threads()
    done, el = timed(seconds)
    oracle.set_num_threads(1)
    try:
        done1, el1 = timed(seconds / 4)
    finally:
        oracle.set_num_threads(cores)
    nb = box[0] * box[1] * box[2]
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
            "one_core": {"value": done1 / el1, "unit": UNIT, "cores": 1,
                         "sample": f"{done1 // nb} boxes ({el1:.1f} s)"},
            "sample": f"{done // nb} boxes of {box[0]}x{box[1]}x{box[2]} voxels of the {n}^3 volume ({el:.1f} s) "
                      f"on {cores} threads"}


def _accuracy(W, vol, mask, outs, prec: int) -> dict:
    """Sampled parity of the timed outputs against the oracle: boxes at the
    corners, across the tensor-core tiles' seams and on seeded wall points."""
    from oracle import oracle
    from paper_2508_07476_gb300 import synth
    n = vol.shape[0]
    cen, ax = synth.frame_of(W.spec)
    b = min(12, n)
    rng = np.random.default_rng(11)
    boxes = [(0, 0, 0), (n - b, n - b, n - b), (n // 2 - min(120, n // 4), n // 2, n // 2),
             (122, 250, 122), (250, 122, 378)]
    walls = 0
    for _ in range(100000):
        if walls == 5:
            break
        x, y, z = (int(v) for v in rng.integers(0, n, size=3))
        if mask[z, y, x]:
            boxes.append((x - b // 2, y - b // 2, z - b // 2))
            walls += 1
    worst = {}
    for lo in boxes:
        lo = tuple(min(max(0, v), n - b) for v in lo)
        ora = oracle.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask, lo=lo, n=(b, b, b))
        sl = (slice(lo[2], lo[2] + b), slice(lo[1], lo[1] + b), slice(lo[0], lo[0] + b))
        out = {"v": outs["v"][(slice(None),) + sl], "ha": outs["ha"][sl], "ia": outs["ia"][sl], "fa": outs["fa"][sl]}
        _merge(worst, _grade_box(ora, out, mask[sl].astype(bool), prec))
    return _verdict(worst)


def _kernel_algorithmic(name: str, nvox: int, rs: int, rr: int, inside: float = 1.0):
    """(algorithmic FMAs, algorithmic HBM bytes) of one launch over nvox output voxels:
    FMAs count taps unfolded; bytes count each input and output once.  inside is
    the fraction of voxels inside the mask: the eigen stage reads the tensor of
    those voxels only (the others take the fill value), every other stage works
    on the whole box."""
    if name == "grad_products":
        return nvox * (8 * (2 * rs + 1) + 6), nvox * (2 + 24)
    if name in ("rho_x", "rho_y", "rho_z"):
        return nvox * 6 * (2 * rr + 1), nvox * 48
    if name in ("rho_x_tc", "rho_y_tc", "rho_z_tc"):  # tensor-core passes: bound by HBM, 6 planes in and out
        return 0, nvox * 48
    if name == "grad_xy":  # volume in, three x/y-filtered planes out
        return 0, nvox * (2 + 12)
    if name == "grad_z":  # three planes in, six products out
        return 0, nvox * (12 + 24)
    if name in ("grad_z_g32", "grad_z_g16"):  # three planes in, the gradient out (FP32 / FP16)
        return 0, nvox * (12 + (12 if name.endswith("32") else 6))
    if name in ("rho_z_tc_g32", "rho_z_tc_g16"):  # the gradient in (products formed on chip), six planes out
        return 0, nvox * ((12 if name.endswith("32") else 6) + 24)
    if name == "rho_xy":
        return nvox * 12 * (2 * rr + 1), nvox * 48
    if name == "rho_z_eig":
        return nvox * 6 * (2 * rr + 1), nvox * (24 + 1 + 24)
    if name == "eig_angles":  # mask everywhere, tensor inside, six outputs everywhere
        return 0, nvox * (1 + 24 + 24 * inside)
    return 0, 0


# DRAM bytes per output voxel of a kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the launch / voxels of the
# capture); valid only for the kernel version summarised in the named file.
MEASURED_TRAFFIC = {"rho_x_tc": (45.1, "profiles/kernels_annulus256.md"),
                    "rho_y_tc": (44.8, "profiles/kernels_annulus256.md"),
                    "rho_z_tc_g16": (26.6, "profiles/kernels_annulus256.md"),
                    "grad_z_g16": (16.4, "profiles/kernels_annulus256.md"),
                    "grad_xy": (10.4, "profiles/kernels_annulus256.md"),
                    "eig_angles": (36.4, "profiles/kernels_annulus256.md")}


def run_ours(args):
    import torch
    from paper_2508_07476_gb300 import _lib, synth
    import __graft_entry__

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    __graft_entry__.build()
    W = _workload(args.size)
    vol, mask = synth.generate(W.spec)
    n = args.size
    nvox = n ** 3
    cen, ax = synth.frame_of(W.spec)
    inside_frac = float(np.count_nonzero(mask)) / nvox
    d_vol = torch.from_numpy(vol.view(np.int16)).cuda()
    d_mask = torch.from_numpy(mask).cuda()
    outs = {"v": torch.empty((3, n, n, n), device="cuda"), "ha": torch.empty((n, n, n), device="cuda"),
            "ia": torch.empty((n, n, n), device="cuda"), "fa": torch.empty((n, n, n), device="cuda")}
    item = _lib.make_item(d_vol, (n, n, n), d_mask, outs["v"], outs["ha"], outs["ia"], outs["fa"])
    stream = torch.cuda.current_stream()
    rs, rr = _lib.ct_radius(W.sigma), _lib.ct_radius(W.rho)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    forms = {}
    accuracy = {}
    kernels = {}
    clocks = None
    launches_per_step = None
    for name, prec in (("fp32", _lib.CT_PREC_FP32), ("mixed", _lib.CT_PREC_MIXED)):
        plan = _lib.ct_plan_create(_lib.make_params(W.sigma, W.rho, cen, ax, prec), (n, n, n))
        try:
            for _ in range(args.warmup):
                _lib.ct_run_chunks(plan, [item], False, stream)
            torch.cuda.synchronize()
            _lib.ct_plan_stats(plan, reset=True)
            headline = name == "mixed"
            _lib.ct_plan_profile(plan, True)
            sampler = ClockSampler(local) if headline and rank == 0 else None
            barrier()
            torch.cuda.synchronize()
            if sampler:
                sampler.start()
                time.sleep(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                _lib.ct_run_chunks(plan, [item], False, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            if sampler:
                clocks = sampler.stop()
            ms = e0.elapsed_time(e1) / args.steps
            ms = max_over_ranks(ms, world)
            kt = _lib.ct_plan_kernel_times(plan)
            _lib.ct_plan_profile(plan, False)
            st = _lib.ct_plan_stats(plan, reset=True)
            forms[name] = {"ms_per_step": ms, "voxels_per_s": job_voxels_per_s(nvox, world, ms),
                           "fallback_voxels_per_step": st["fallback_voxels"] / args.steps}
            kernels[name] = {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in kt.items()}
            if headline:
                launches_per_step = st["launches"] / args.steps
            host_outs = {k: t.cpu().numpy() for k, t in outs.items()}
            accuracy[name] = _accuracy(W, vol, mask, host_outs, prec) if rank == 0 else None
        finally:
            _lib.ct_plan_destroy(plan)

    # transmural HA profile of the mixed form's HA output (a reduction after the step, timed apart)
    nd_p, nh_p = 20, 180
    pspec = _lib.make_profile_spec(cen, ax, W.spec.r_in, W.spec.r_out, nd_p, nh_p, _lib.CT_OUT_F32)
    hist = torch.zeros(nd_p * nh_p, dtype=torch.int64, device="cuda")
    _lib.ct_transmural_profile(pspec, (n, n, n), (0, 0, 0), (n, n, n), outs["ha"], d_mask, hist, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        _lib.ct_transmural_profile(pspec, (n, n, n), (0, 0, 0), (n, n, n), outs["ha"], d_mask, hist, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    h = hist.cpu().numpy().reshape(nd_p, nh_p) // (reps + 1)
    centres = (np.arange(nh_p) + 0.5) * 180.0 / nh_p - 90.0
    prof_ms = e0.elapsed_time(e1) / reps
    transmural = {"ms": prof_ms, "bins": [nd_p, nh_p], "voxels_counted": int(h.sum()),
                  "gb_per_s": nvox * 5 / (prof_ms * 1e-3) / 1e9,
                  "mean_ha_by_depth": [round(float((r * centres).sum() / max(r.sum(), 1)), 2) for r in h]}

    # streamline tractography through the mixed form's fibre field (timed apart from the step)
    rng_t = np.random.default_rng(9)
    zz, yy, xx = np.nonzero(mask)
    pick = rng_t.choice(len(xx), min(100000, len(xx)), replace=False)
    seeds = np.column_stack([xx[pick], yy[pick], zz[pick]]).astype(np.float32) + \
        rng_t.uniform(-0.4, 0.4, (len(pick), 3)).astype(np.float32)
    d_seeds = torch.from_numpy(seeds).cuda()
    t_steps = 200
    tp = _lib.make_track_params(0.5, t_steps, 0.1, 45.0)
    pts = torch.empty((len(seeds), 2, t_steps + 1, 3), dtype=torch.float32, device="cuda")
    tcnt = torch.empty((len(seeds), 2), dtype=torch.int32, device="cuda")
    _lib.ct_track(tp, (n, n, n), outs["v"], outs["fa"], d_mask, d_seeds, len(seeds), pts, tcnt, stream)
    e0.record(stream)
    _lib.ct_track(tp, (n, n, n), outs["v"], outs["fa"], d_mask, d_seeds, len(seeds), pts, tcnt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    track_ms = e0.elapsed_time(e1)
    nsteps = int(tcnt.sum().item()) - int((tcnt > 0).sum().item())
    tractography = {"ms": track_ms, "seeds": len(seeds), "tracks": 2 * len(seeds), "steps": nsteps,
                    "steps_per_s": nsteps / (track_ms * 1e-3), "mean_points_per_track": float(tcnt.float().mean()),
                    "params": {"step": 0.5, "max_steps": t_steps, "fa_min": 0.1, "max_turn_deg": 45.0,
                               "scheme": "RK4, sign-aligned trilinear field"}}
    del pts

    head = forms["mixed"]
    peaks, peak_kind = _peaks()
    fma_meas = _fma_rate_measured(local)
    fma_peak = fma_meas["fma_per_s"]  # FMA/s, measured on this GPU in this run
    # dominant kernel of the headline form
    km = kernels["mixed"]
    dom = max(km, key=lambda k: km[k]["avg_ms"] * km[k]["launches"])
    fmas, byts = _kernel_algorithmic(dom, nvox, rs, rr, inside_frac)
    avg_s = km[dom]["avg_ms"] * 1e-3
    if fmas > 0:
        ach = 2.0 * fmas / avg_s / 1e12
        peak = 2.0 * fma_peak / 1e12
        tr = MEASURED_TRAFFIC.get(dom)
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None if tr is None else tr[0] * nvox,
                    "traffic_source": None if tr is None else tr[1], "peak_source": fma_meas["source"]}
    else:
        ach = byts / avg_s / 1e9
        tr = MEASURED_TRAFFIC.get(dom)
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None if tr is None else tr[0] * nvox,
                    "traffic_source": None if tr is None else tr[1], "peak_source": f"{peak_kind} hbm_gbs",
                    "algorithmic_bytes_per_voxel": byts / nvox}
    # the launched kernel sequence's own floor: its algorithmic HBM bytes per voxel
    path_bytes = sum(_kernel_algorithmic(k, 1, rs, rr, inside_frac)[1] * km[k]["launches"] / args.steps for k in km)
    path_hbm = {"voxels_per_s_roofline": peaks["hbm_gbs"] * 1e9 / path_bytes, "bytes_per_voxel": path_bytes,
                "frac_mixed": head["voxels_per_s"] / world / (peaks["hbm_gbs"] * 1e9 / path_bytes),
                "bound": "HBM: sum over the launched kernels of their algorithmic bytes"}
    f_vox = _fma_per_voxel(rs, rr)
    path_roof = min(fma_peak / f_vox, peaks["hbm_gbs"] * 1e9 / 27.0)
    pipeline_roofline = {"voxels_per_s_roofline": path_roof, "fma_per_voxel": f_vox,
                         "fma_peak": fma_meas, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peak_kind,
                         "min_bytes_per_voxel": 27, "frac_fp32": forms["fp32"]["voxels_per_s"] / world / path_roof,
                         "frac_mixed": head["voxels_per_s"] / world / path_roof,
                         "bound": "FP32 FMA of the stencil formulation (min of FMA/s / F and HBM / bytes); "
                                  "the rho passes run on the tensor cores, which this bound does not cover",
                         "kernel_sequence_hbm": path_hbm}

    e2e = None
    if not args.no_e2e:
        # z slabs of the volume on two streams, so that one slab's copies overlap another's kernels
        zc = args.e2e_zchunk if args.e2e_zchunk > 0 else n
        plan = _lib.ct_plan_create(_lib.make_params(W.sigma, W.rho, cen, ax, _lib.CT_PREC_MIXED, chunk=(n, n, zc)),
                                   (n, n, n))
        try:
            h_vol = torch.from_numpy(vol.view(np.int16)).pin_memory()
            h_mask = torch.from_numpy(mask).pin_memory()
            h_out = {"v": torch.empty((3, n, n, n)).pin_memory(), "ha": torch.empty((n, n, n)).pin_memory(),
                     "ia": torch.empty((n, n, n)).pin_memory(), "fa": torch.empty((n, n, n)).pin_memory()}
            hitem = _lib.make_item(h_vol, (n, n, n), h_mask, h_out["v"], h_out["ha"], h_out["ia"], h_out["fa"])
            _lib.ct_run_chunks(plan, [hitem], True)
            _lib.ct_plan_stats(plan, reset=True)
            barrier()
            t0 = time.perf_counter()
            k_e2e = max(1, min(args.steps, 5))
            for _ in range(k_e2e):
                _lib.ct_run_chunks(plan, [hitem], True)
            torch.cuda.synchronize()
            el = max_over_ranks((time.perf_counter() - t0) / k_e2e, world)
            st = _lib.ct_plan_stats(plan, reset=True)
            e2e = {"value": world * nvox / el, "unit": UNIT, "h2d_bytes_per_step": st["h2d_bytes"] // k_e2e,
                   "d2h_bytes_per_step": st["d2h_bytes"] // k_e2e, "ms_per_step": el * 1e3,
                   "timing": "wall clock around the synchronous host-buffer call",
                   "chunk": [n, n, zc], "copies": "pinned host buffers, one H2D and one D2H per plane per slab"}
        finally:
            _lib.ct_plan_destroy(plan)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = _cpu_baseline(W, vol, mask, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["voxels_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded annulus volume)",
            "config": {"workload": W.name, "dims": [n, n, n], "sigma": W.sigma, "rho": W.rho, "mask": True,
                       "outputs": "f32 vector, HA, IA, FA", "precision": "mixed (FP16-held gradient)",
                       "l2": "inputs larger than L2 (268 MB volume + 6.4 GB scratch per step)",
                       "parallelism": f"{world} independent volume(s), one per GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "gpu_launches_per_step": launches_per_step, "clocks": clocks, "forms": forms,
            "pipeline_roofline": pipeline_roofline, "accuracy": accuracy, "kernels": kernels,
            "transmural_profile": transmural, "tractography": tractography,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _line(metric, value, unit, args, ms, config, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded, generated on the device)", "config": config}
    line.update(extra)
    print(json.dumps(line))


def _oracle_sub(get_vol, get_mask, dims, lo, b, halo, sigma, rho, cen, ax):
    """Oracle outputs over the box (lo, b^3) of a volume of size dims (x, y, z)
    from the sub-volume the box needs: the box grown by the halo and clipped to
    the volume.  Where the growth is clipped the sub-volume's edge is the
    volume's, so the oracle's edge clamp is the volume's; elsewhere no tap
    reaches the sub-volume's edge.  get_vol / get_mask(lo, n) return the
    uint16 / uint8 [z, y, x] arrays of a global box."""
    from oracle import oracle
    glo = tuple(max(0, a - halo) for a in lo)
    ghi = tuple(min(d, a + b + halo) for a, d in zip(lo, dims))
    gn = tuple(h - l for l, h in zip(glo, ghi))
    sub = get_vol(glo, gn)
    msub = None if get_mask is None else get_mask(glo, gn)
    c = tuple(cc - o for cc, o in zip(cen, glo))
    rel = tuple(a - o for a, o in zip(lo, glo))
    ora = oracle.pipeline(sub, sigma, rho, c, ax, mask=msub, lo=rel, n=(b, b, b))
    inside = np.ones((b, b, b), bool) if msub is None else \
        msub[rel[2]:rel[2] + b, rel[1]:rel[1] + b, rel[0]:rel[0] + b].astype(bool)
    return ora, inside


def _host_box(arr):
    def get(lo, n):
        return np.ascontiguousarray(arr[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]])
    return get


def run_crops(args):
    """Uneven crops, three ways: a graph of per-crop launch sequences on four
    streams (the default, the line's value), persistent batched launches (one
    per stage and tap set over all crops, in a CUDA graph), and per-crop launch
    sequences on one stream."""
    import torch
    from paper_2508_07476_gb300 import _lib, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    crops = synth.crop_batch(args.crops)
    vols, outs, items = [], [], []
    total = 0
    for w in crops:
        nz, ny, nx = w.spec.shape
        v = torch.empty((nz, ny, nx), dtype=torch.int16, device="cuda")
        _lib.ct_synth_annulus(w.spec, (nx, ny, nz), (0, 0, 0), (nx, ny, nz), v, flags=_lib.CT_SYNTH_FP32)
        o = [torch.empty((3, nz, ny, nx), dtype=torch.float16, device="cuda")] + \
            [torch.empty((nz, ny, nx), dtype=torch.float16, device="cuda") for _ in range(3)]
        cen, ax = synth.frame_of(w.spec)
        items.append(_lib.make_item(v, (nx, ny, nz), None, *o, sigma=w.sigma, rho=w.rho, lv_center=cen,
                                    lv_axis=ax))
        vols.append(v)
        outs.append(o)
        total += nx * ny * nz
    torch.cuda.synchronize()
    res = {}
    rng0 = np.random.default_rng(23)
    picks = []  # 8 seed-chosen crops, one 12^3 box each, graded after every mode
    for j in sorted(rng0.choice(len(crops), 8, replace=False)):
        nz, ny, nx = crops[j].spec.shape
        picks.append((int(j), tuple(int(rng0.integers(0, d - 12 + 1)) for d in (nx, ny, nz))))
    ora_cache = {}
    mode_env = {"persistent": {"CT_TUNE_BATCH_GRAPH": "1", "CT_TUNE_BATCH_PERSISTENT": "1"},
                "graph": {"CT_TUNE_BATCH_GRAPH": "1", "CT_TUNE_BATCH_PERSISTENT": "0"},
                "per_crop": {"CT_TUNE_BATCH_GRAPH": "0", "CT_TUNE_BATCH_PERSISTENT": "0"},
                "graph_fp32": {"CT_TUNE_BATCH_GRAPH": "1", "CT_TUNE_BATCH_PERSISTENT": "0"}}
    clocks = None
    for mode in ("persistent", "graph", "per_crop", "graph_fp32"):
        # graph_fp32: the default batch form with the plain FP32 arithmetic, for the mixed / FP32 comparison
        prec = _lib.CT_PREC_FP32 if mode == "graph_fp32" else _lib.CT_PREC_MIXED
        os.environ.update(mode_env[mode])
        plan = _lib.ct_plan_create(_lib.make_params(2.0, 6.0, (0, 0, 0), (0, 0, 1), prec,
                                                    _lib.CT_OUT_F16, _lib.CT_OUT_F16, _lib.CT_OUT_F16), (1, 1, 1))
        for k in mode_env[mode]:
            del os.environ[k]
        try:
            for _ in range(args.warmup):
                _lib.ct_run_chunks(plan, items, False)
            torch.cuda.synchronize()
            _lib.ct_plan_stats(plan, reset=True)
            sampler = ClockSampler(0) if mode == "graph" else None
            if sampler:
                sampler.start()
                time.sleep(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                _lib.ct_run_chunks(plan, items, False)
            e1.record()
            torch.cuda.synchronize()
            if sampler:
                clocks = sampler.stop()
            st = _lib.ct_plan_stats(plan, reset=True)
            ms = e0.elapsed_time(e1) / args.steps
            res[mode] = {"ms_per_step": ms, "voxels_per_s": total / (ms * 1e-3),
                         "launches_per_step": st["launches"] / args.steps,
                         "fallback_voxels_per_step": st["fallback_voxels"] / args.steps}
            if mode not in ("graph", "graph_fp32"):  # where the time goes: one more step with per-kernel events
                _lib.ct_plan_profile(plan, True)
                _lib.ct_run_chunks(plan, items, False)
                torch.cuda.synchronize()
                kt = _lib.ct_plan_kernel_times(plan)
                _lib.ct_plan_profile(plan, False)
                res[mode]["kernel_ms_per_step"] = {k: round(v[1], 3) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][1])}
        finally:
            _lib.ct_plan_destroy(plan)
        # accuracy of this mode's outputs: the 8 seed-chosen crops' boxes against
        # the oracle on the same input bytes (copied back from the device generator)
        worst = {}
        b = 12
        for j, lo in picks:
            w = crops[j]
            nz, ny, nx = w.spec.shape
            if (j, lo) not in ora_cache:
                host = vols[j].cpu().numpy().view(np.uint16)
                halo = _lib.ct_radius(w.sigma) + _lib.ct_radius(w.rho)
                cen, ax = synth.frame_of(w.spec)
                ora_cache[(j, lo)] = _oracle_sub(_host_box(host), None, (nx, ny, nz), lo, b, halo, w.sigma, w.rho,
                                                 cen, ax)
            ora, inside = ora_cache[(j, lo)]
            o = [_decode(t) for t in outs[j]]
            sl = (slice(lo[2], lo[2] + b), slice(lo[1], lo[1] + b), slice(lo[0], lo[0] + b))
            out = {"v": o[0][(slice(None),) + sl], "ha": o[1][sl], "ia": o[2][sl], "fa": o[3][sl]}
            _merge(worst, _grade_box(ora, out, inside, prec))
        res[mode]["accuracy"] = _verdict(worst)
    accuracy = dict(res["graph"]["accuracy"])
    accuracy["sample"] = "one 12^3 box in each of 8 seed-chosen crops, F16 outputs decoded (every mode graded the " \
                         "same way: modes.*.accuracy); input bytes from the device generator copied back"
    _line("voxels/s, 200 uneven crops, one call: the batch's launches in a CUDA graph on 4 streams",
          res["graph"]["voxels_per_s"], UNIT, args, res["graph"]["ms_per_step"],
          {"workload": f"crops{args.crops}", "voxels": total, "sizes": "each axis U[64,384]",
           "sigma": "per crop from {1,1.5,2,3}", "rho": "per crop from {2,4,6,8}", "outputs": "f16 v, HA, IA, FA",
           "precision": "mixed"},
          {"modes": res, "gpu_launches": res["graph"]["launches_per_step"] * args.steps, "clocks": clocks,
           "accuracy": accuracy,
           "mixed_vs_fp32": res["graph"]["voxels_per_s"] / res["graph_fp32"]["voxels_per_s"]})


def run_stream(args):
    """Host-resident volume streamed through the device in padded chunks on two streams."""
    import torch
    from paper_2508_07476_gb300 import _lib, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    W = synth.lv_annulus_512(512)
    # the 4x-scaled annulus of the 2048 x 2048 x 1024 stream
    spec = synth.AnnulusSpec(shape=(1024, 2048, 2048), r_in=480.0, r_out=880.0, period=8.0, ha_in_deg=70.0,
                             ha_out_deg=-70.0, axis=W.spec.axis, noise=("poisson_like", 0.05), ia_std_deg=5.0,
                             ia_corr=40.0, seed=3)
    nz = args.zplanes or 1024
    ny = nx = 2048
    sigma, rho, C = 2.0, 8.0, 256
    t_alloc = time.perf_counter()
    h_vol = torch.empty((nz, ny, nx), dtype=torch.int16, pin_memory=True)
    h_mask = torch.empty((nz, ny, nx), dtype=torch.uint8, pin_memory=True)
    slab = 64
    dv = torch.empty((slab, ny, nx), dtype=torch.int16, device="cuda")
    dm = torch.empty((slab, ny, nx), dtype=torch.uint8, device="cuda")
    for z0 in range(0, nz, slab):
        k = min(slab, nz - z0)
        _lib.ct_synth_annulus(spec, (nx, ny, 1024), (0, 0, z0), (nx, ny, k), dv, dm, flags=_lib.CT_SYNTH_FP32)
        h_vol[z0:z0 + k].copy_(dv[:k])
        h_mask[z0:z0 + k].copy_(dm[:k])
    del dv, dm
    torch.cuda.synchronize()
    outs = [torch.empty((3, nz, ny, nx), dtype=torch.float16, pin_memory=True)] + \
        [torch.empty((nz, ny, nx), dtype=torch.float16, pin_memory=True) for _ in range(3)]
    t_alloc = time.perf_counter() - t_alloc
    cen, ax = synth.frame_of(spec)
    plan = _lib.ct_plan_create(_lib.make_params(sigma, rho, cen, ax, _lib.CT_PREC_MIXED, _lib.CT_OUT_F16,
                                                _lib.CT_OUT_F16, _lib.CT_OUT_F16, chunk=(C, C, C)),
                               (nx, ny, nz))
    try:
        item = _lib.make_item(h_vol, (nx, ny, nz), h_mask, *outs)
        for _ in range(args.warmup):
            _lib.ct_run_chunks(plan, [item], True)
        _lib.ct_plan_stats(plan, reset=True)
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _lib.ct_run_chunks(plan, [item], True)
        el = (time.perf_counter() - t0) / args.steps
        clocks = sampler.stop()
        st = _lib.ct_plan_stats(plan, reset=True)
    finally:
        _lib.ct_plan_destroy(plan)
    vox = nx * ny * nz
    h2d, d2h = st["h2d_bytes"] / args.steps, st["d2h_bytes"] / args.steps
    # accuracy: 8 seed-chosen 12^3 boxes (two corners, the rest across chunk
    # seams at multiples of 256, where a box's voxels come from several chunks)
    hv, hm = h_vol.numpy().view(np.uint16), h_mask.numpy()
    o = [t.numpy() for t in outs]
    rng = np.random.default_rng(29)
    b, halo = 12, _lib.ct_radius(sigma) + _lib.ct_radius(rho)
    boxes = [(0, 0, 0), (nx - b, ny - b, nz - b)]
    while len(boxes) < 8:
        lo = tuple(int(C * rng.integers(1, max(2, d // C))) - b // 2 for d in (nx, ny, nz))
        x, y, z = (a + b // 2 for a in lo)
        if hm[min(z, nz - 1), y, x]:
            boxes.append(tuple(min(max(0, a), d - b) for a, d in zip(lo, (nx, ny, nz))))
    worst = {}
    for lo in boxes:
        ora, inside = _oracle_sub(_host_box(hv), _host_box(hm), (nx, ny, nz), lo, b, halo, sigma, rho, cen, ax)
        sl = (slice(lo[2], lo[2] + b), slice(lo[1], lo[1] + b), slice(lo[0], lo[0] + b))
        out = {"v": o[0][(slice(None),) + sl].astype(np.float32), "ha": o[1][sl].astype(np.float32),
               "ia": o[2][sl].astype(np.float32), "fa": o[3][sl].astype(np.float32)}
        _merge(worst, _grade_box(ora, out, inside, _lib.CT_PREC_MIXED))
    accuracy = _verdict(worst)
    accuracy["sample"] = "8 seed-chosen 12^3 boxes (corners; across 256-voxel chunk seams in the wall), F16 outputs"
    _line(f"voxels/s, host-resident 2048x2048x{nz} volume streamed in 256^3 chunks", vox / el, UNIT, args, el * 1e3,
          {"workload": f"stream2048x2048x{nz}", "chunk": [C, C, C], "halo": halo, "sigma": sigma, "rho": rho,
           "mask": True, "outputs": "f16 v, HA, IA, FA", "precision": "mixed", "host_buffers": "pinned",
           "host_bytes": int(vox * (2 + 1 + 12))},
          {"e2e": {"value": vox / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
           "host_link_gbs": (h2d + d2h) / el / 1e9,
           "host_link_bound": {"voxels_per_s": vox / ((h2d + d2h) / (_HOST_LINK_GBS * 1e9)),
                               "note": f"the step's copies at {_HOST_LINK_GBS:.0f} GB/s (H2D and D2H together, "
                                       f"measured on this box)"},
           "gpu_launches": st["launches"], "setup_s": t_alloc, "clocks": clocks, "accuracy": accuracy})


_HOST_LINK_GBS = 312.0  # host <-> device copies in both directions at once, pinned (measured here)


def run_tera(args):
    """Teravoxel-shaped stream: each padded chunk generated on the device, processed, and its u8 / f16
    outputs copied into a pinned ring that a host sink checksums; two chunks resident at a time.  The
    pipeline's own time is taken with CUDA events around each chunk's ct_run_box (the generator apart)."""
    import torch
    from paper_2508_07476_gb300 import _lib, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    nx = ny = 4096
    nzf = 2048
    nz = args.zplanes or nzf
    spec = synth.AnnulusSpec(shape=(nzf, ny, nx), r_in=1000.0, r_out=1800.0, period=10.0, ha_in_deg=70.0,
                             ha_out_deg=-70.0, axis=(math.sin(math.radians(10.0)), 0.0, math.cos(math.radians(10.0))),
                             noise=("poisson_like", 0.05), ia_std_deg=5.0, ia_corr=40.0, seed=5)
    cen, ax = synth.frame_of(spec)
    sigma, rho, C = 3.0, 9.0, 384
    rs, rr = _lib.ct_radius(sigma), _lib.ct_radius(rho)
    halo = rs + rr
    fma_meas = _fma_rate_measured(0)
    fma_rate = fma_meas["fma_per_s"]
    chunks = [(x, y, z) for z in range(0, nz, C) for y in range(0, ny, C) for x in range(0, nx, C)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = [_lib.ct_plan_create(_lib.make_params(sigma, rho, cen, ax, _lib.CT_PREC_MIXED, _lib.CT_OUT_F32,
                                                  _lib.CT_OUT_U8Q, _lib.CT_OUT_F16), (nx, ny, nzf)) for _ in range(2)]
    cin = C + 2 * halo
    slots = []
    for _ in range(2):
        slots.append({
            "vol": torch.empty(cin ** 3, dtype=torch.int16, device="cuda"),
            "mask": torch.empty(C ** 3, dtype=torch.uint8, device="cuda"),
            "ha": torch.empty(C ** 3, dtype=torch.uint8, device="cuda"),
            "ia": torch.empty(C ** 3, dtype=torch.uint8, device="cuda"),
            "fa": torch.empty(C ** 3, dtype=torch.float16, device="cuda"),
            "h": torch.empty(C ** 3 * 4, dtype=torch.uint8, pin_memory=True),
            "ev": torch.cuda.Event(), "n": 0, "pending": False, "spans": []})
    sink = {"sum": 0, "voxels": 0, "wait_s": 0.0, "read_s": 0.0}
    F32 = _lib.CT_SYNTH_FP32

    def drain(sl):
        # The host consumer: waits for the slot's copies, then reads every byte
        # (a wrapping 64-bit sum), as a writer to storage would.
        if not sl["pending"]:
            return
        t0 = time.perf_counter()
        sl["ev"].synchronize()
        t1 = time.perf_counter()
        n = sl["n"]
        sink["sum"] = (sink["sum"] + int(sl["h"][:4 * n].view(torch.int64).sum())) & ((1 << 64) - 1)
        sink["voxels"] += n
        sink["wait_s"] += t1 - t0
        sink["read_s"] += time.perf_counter() - t1
        sl["pending"] = False

    def boxes_of(x0, y0, z0):
        lo = (x0, y0, z0)
        n = (min(C, nx - x0), min(C, ny - y0), min(C, nz - z0))
        ilo = tuple(max(0, a - halo) for a in lo)
        ihi = tuple(min(d, a + b + halo) for a, b, d in zip(lo, n, (nx, ny, nzf)))
        return lo, n, ilo, tuple(b - a for a, b in zip(ilo, ihi))

    def run_chunks(todo, timed=False, keep=None, serial=False):
        # serial: every chunk's generator, pipeline and copies on one stream, so
        # that no kernel runs beside a timed pipeline span
        for i, (x0, y0, z0) in enumerate(todo):
            sl, st, plan = slots[i & 1], streams[0 if serial else i & 1], plans[i & 1]
            drain(sl)
            lo, n, ilo, ino = boxes_of(x0, y0, z0)
            nv = n[0] * n[1] * n[2]
            assert nv % 2 == 0
            with torch.cuda.stream(st):
                _lib.ct_synth_annulus(spec, (nx, ny, nzf), ilo, ino, sl["vol"], None, st, flags=F32)
                _lib.ct_synth_annulus(spec, (nx, ny, nzf), lo, n, None, sl["mask"], st, flags=F32)
                if timed:
                    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ea.record(st)
                vec = None
                if keep is not None:  # the accuracy re-run also writes the vector, to grade the direction
                    if "vec" not in sl:
                        sl["vec"] = torch.empty(3 * C ** 3, dtype=torch.float32, device="cuda")
                    vec = sl["vec"]
                _lib.ct_run_box(plan, sl["vol"], ilo, ino, lo, n, sl["mask"], vec, sl["ha"], sl["ia"], sl["fa"], st)
                if timed:
                    eb.record(st)
                    sl["spans"].append((ea, eb))
                if keep is not None:
                    keep.append({k: sl[k][:(3 if k == "vec" else 1) * nv].clone() for k in ("vec", "ha", "ia", "fa")})
                h = sl["h"]
                h[:nv].copy_(sl["ha"][:nv], non_blocking=True)
                h[nv:2 * nv].copy_(sl["ia"][:nv], non_blocking=True)
                h[2 * nv:4 * nv].copy_(sl["fa"][:nv].view(torch.uint8), non_blocking=True)
                sl["ev"].record(st)
            sl["n"] = nv
            sl["pending"] = True
        for sl in slots:
            drain(sl)

    try:
        # warm-up: the first chunks (plans size their buffers, streams spin up)
        run_chunks(chunks[:max(3, args.warmup)])
        sink.update({"sum": 0, "voxels": 0, "wait_s": 0.0, "read_s": 0.0})
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run_chunks(chunks, timed=True)
        torch.cuda.synchronize()
        el = (time.perf_counter() - t0) / args.steps
        overlap_ms = sum(a.elapsed_time(b) for sl in slots for a, b in sl["spans"]) / args.steps
        # the pipeline alone: the same chunks with the generator serialised before
        # each chunk's ct_run_box, so that each span times the pipeline only
        for sl in slots:
            sl["spans"] = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run_chunks(chunks, timed=True, serial=True)
        torch.cuda.synchronize()
        serial_s = (time.perf_counter() - t0) / args.steps
        clocks = sampler.stop()
        pipe_ms = sum(a.elapsed_time(b) for sl in slots for a, b in sl["spans"]) / args.steps
        # the generator alone over the same chunks (timed apart, as the stream's input cost)
        t0 = time.perf_counter()
        for i, (x0, y0, z0) in enumerate(chunks):
            sl, st = slots[i & 1], streams[i & 1]
            lo, n, ilo, ino = boxes_of(x0, y0, z0)
            _lib.ct_synth_annulus(spec, (nx, ny, nzf), ilo, ino, sl["vol"], None, st, flags=F32)
            _lib.ct_synth_annulus(spec, (nx, ny, nzf), lo, n, None, sl["mask"], st, flags=F32)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        # accuracy: 8 seed-chosen chunks (two corners, six drawn), run again the same
        # way; in each a 12^3 box on the wall, graded against the oracle on the
        # generator's bytes of the box and its halo (copied back from the device)
        rng = np.random.default_rng(31)
        pick = [0, len(chunks) - 1] + [int(k) for k in rng.choice(np.arange(1, len(chunks) - 1), 6, replace=False)]
        kept = []
        run_chunks([chunks[k] for k in pick], keep=kept)
        torch.cuda.synchronize()

        def gen_box(lo, n, mask=False):
            t = torch.empty(n[0] * n[1] * n[2], dtype=torch.uint8 if mask else torch.int16, device="cuda")
            if mask:
                _lib.ct_synth_annulus(spec, (nx, ny, nzf), lo, n, None, t, flags=F32)
            else:
                _lib.ct_synth_annulus(spec, (nx, ny, nzf), lo, n, t, None, flags=F32)
            a = t.cpu().numpy().reshape(n[2], n[1], n[0])
            return a if mask else a.view(np.uint16)

        worst = {}
        b = 12
        for k, out_dev in zip(pick, kept):
            lo_c, n_c, _, _ = boxes_of(*chunks[k])
            m_c = gen_box(lo_c, n_c, mask=True)
            # a wall point of the chunk, else its centre
            zz, yy, xx = np.nonzero(m_c)
            j = int(rng.integers(0, len(xx))) if len(xx) else None
            c_loc = (xx[j], yy[j], zz[j]) if j is not None else tuple(d // 2 for d in n_c)
            rel = tuple(int(min(max(0, c - b // 2), d - b)) for c, d in zip(c_loc, n_c))
            lo = tuple(a + r for a, r in zip(lo_c, rel))
            ora, inside = _oracle_sub(lambda l, n: gen_box(l, n), lambda l, n: gen_box(l, n, True), (nx, ny, nzf),
                                      lo, b, halo, sigma, rho, cen, ax)
            shp = (n_c[2], n_c[1], n_c[0])
            sl = (slice(rel[2], rel[2] + b), slice(rel[1], rel[1] + b), slice(rel[0], rel[0] + b))
            ha = out_dev["ha"].cpu().numpy().reshape(shp)[sl]
            ia = out_dev["ia"].cpu().numpy().reshape(shp)[sl]
            fa = out_dev["fa"].float().cpu().numpy().reshape(shp)[sl]
            v = out_dev["vec"].cpu().numpy().reshape((3,) + shp)[(slice(None),) + sl]
            out = {"v": v, "ha": ha, "ia": ia, "fa": fa}
            r = _grade_box(ora, out, inside, _lib.CT_PREC_MIXED, u8q=True)
            _merge(worst, r)
        accuracy = _verdict(worst, u8q=True)
        accuracy["sample"] = "one 12^3 wall box in each of 8 seed-chosen chunks (corners included), run again " \
                             "with an F32 vector output as well: U8Q HA / IA codes against the oracle's own " \
                             "quantisation, F16 FA, the vector's direction; input bytes from the device " \
                             "generator copied back"
    finally:
        for p in plans:
            _lib.ct_plan_destroy(p)
    vox = nx * ny * nz
    _line("voxels/s, 4096x4096x2048 device-generated stream in 384^3 chunks (pipeline time; generator timed apart)",
          vox / (pipe_ms * 1e-3), UNIT, args, pipe_ms,
          {"workload": f"tera4096x4096x{nz}", "chunk": [C, C, C], "halo": halo, "sigma": sigma, "rho": rho,
           "mask": True, "outputs": "u8 HA, u8 IA (180/256 deg bins), f16 FA", "precision": "mixed",
           "resident_chunks": 2, "generator": "device, FP32 form, padded chunk + output-box mask per chunk",
           "sink": "two pinned host slots, every byte read by a 64-bit host checksum", "warmup": "first chunks"},
          {"timing": "value: CUDA events around each chunk's ct_run_box, summed, with each chunk's generator run "
                     "before it on the same stream (no other kernel beside a span); clocks sampled over both passes",
           "roofline": {"bound": "alu", "voxels_per_s_roofline": fma_rate / _fma_per_voxel(rs, rr),
                        "fma_per_voxel": _fma_per_voxel(rs, rr), "fma_peak": fma_meas,
                        "frac": vox / (pipe_ms * 1e-3) / (fma_rate / _fma_per_voxel(rs, rr)),
                        "note": "output voxels; the halo of each chunk (R_sigma + R_rho per side) is extra work"},
           "stream_with_generator": {"s_per_step": el, "voxels_per_s": vox / el,
                                     "pipeline_spans_ms": overlap_ms,
                                     "note": "generator of the next chunk on the other stream, beside the pipeline"},
           "serial_pass_s_per_step": serial_s,
           "generator_only": {"s_per_step": gen_s, "voxels_per_s": vox / gen_s,
                              "note": "padded chunks + output-box masks generated alone, same streams"},
           "sink_voxels": sink["voxels"], "sink_checksum": sink["sum"],
           "host_s_per_step": {"waiting_for_gpu": sink["wait_s"] / args.steps, "sink_read": sink["read_s"] / args.steps},
           "e2e": {"value": vox / el, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 4 * vox},
           "clocks": clocks, "accuracy": accuracy})


def run_zslab(args):
    """One annulus volume split across the ranks in z-slabs (strong scaling):
    rank k generates the input planes of its slab plus the halo and runs the
    padded-box call on them; no collective on the data path."""
    import torch
    from paper_2508_07476_gb300 import _lib, partition, synth
    import __graft_entry__

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    W = _workload(args.size)
    n = args.size
    h = _lib.ct_radius(W.sigma) + _lib.ct_radius(W.rho)
    sl = partition.z_slabs((n, n, n), world, h)[rank]
    i0, i1 = sl.in_z
    z0, z1 = sl.out_z
    vol, _ = synth.generate(W.spec, (i0, i1))
    _, mask = synth.generate(W.spec, (z0, z1))
    cen, ax = synth.frame_of(W.spec)
    d_vol = torch.from_numpy(vol.view(np.int16)).cuda()
    d_mask = torch.from_numpy(mask).cuda()
    nzs = z1 - z0
    outs = [torch.empty((3, nzs, n, n), device="cuda")] + [torch.empty((nzs, n, n), device="cuda") for _ in range(3)]
    plan = _lib.ct_plan_create(_lib.make_params(W.sigma, W.rho, cen, ax, _lib.CT_PREC_MIXED), (n, n, n))
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    try:
        for _ in range(args.warmup):
            _lib.ct_run_box(plan, d_vol, sl.in_lo, sl.in_n, sl.out_lo, sl.out_n, d_mask, *outs, stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            _lib.ct_run_box(plan, d_vol, sl.in_lo, sl.in_n, sl.out_lo, sl.out_n, d_mask, *outs, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
        st = _lib.ct_plan_stats(plan)
    finally:
        _lib.ct_plan_destroy(plan)
    if rank == 0:
        line = {"metric": METRIC, "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded annulus volume)",
                "config": {"workload": W.name, "dims": [n, n, n], "sigma": W.sigma, "rho": W.rho, "mask": True,
                           "precision": "mixed", "parallelism": f"one volume in {world} z-slabs, halo {h} planes",
                           "slab_planes": [s.out_n[2] for s in partition.z_slabs((n, n, n), world, h)]},
                "gpu_launches": st["launches"]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.split == "zslab":
        run_zslab(args)
    elif args.workload == "crops200":
        run_crops(args)
    elif args.workload == "stream2048":
        run_stream(args)
    elif args.workload == "tera4096":
        run_tera(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
