"""Thin ctypes binding of the C ABI in ``include/ct.h`` (same names).

Argument marshalling only: every step of the pipeline runs in the CUDA
library.  Arrays are passed as raw pointers taken from torch tensors (device
or host); torch supplies device memory and streams, nothing else.  There is no
fallback of any kind: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Iterable, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libct_gb300.so")

CT_OK = 0
CT_ERR_INVALID = -1
CT_ERR_OOM = -2
CT_ERR_CUDA = -3
CT_ERR_TIMEOUT = -4
CT_ERR_NO_DEVICE = -5
CT_ERR_UNSUPPORTED = -6

CT_PREC_FP32 = 0
CT_PREC_MIXED = 1
CT_OUT_F32 = 0
CT_OUT_F16 = 1
CT_OUT_U8Q = 2

_I64x3 = ctypes.c_int64 * 3
_D3 = ctypes.c_double * 3


class ct_params(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_double), ("rho", ctypes.c_double), ("truncate", ctypes.c_double),
        ("lv_center", _D3), ("lv_axis", _D3),
        ("precision", ctypes.c_int32), ("vec_type", ctypes.c_int32), ("angle_type", ctypes.c_int32),
        ("fa_type", ctypes.c_int32), ("fill_value", ctypes.c_float), ("flags", ctypes.c_int32),
        ("chunk", _I64x3), ("spacing", _D3), ("lv_centres", ctypes.POINTER(ctypes.c_double)),
    ]


class ct_item(ctypes.Structure):
    _fields_ = [
        ("vol", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("dims", _I64x3),
        ("sigma", ctypes.c_double), ("rho", ctypes.c_double), ("lv_center", _D3), ("lv_axis", _D3),
        ("vec", ctypes.c_void_p), ("ha", ctypes.c_void_p), ("ia", ctypes.c_void_p), ("fa", ctypes.c_void_p),
    ]


class ct_stats(ctypes.Structure):
    _fields_ = [("voxels", ctypes.c_int64), ("fallback_voxels", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]


class ct_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class ct_synth_spec(ctypes.Structure):
    _fields_ = [("center", _D3), ("axis", _D3), ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
                ("period", ctypes.c_double), ("ha_in_deg", ctypes.c_double), ("ha_out_deg", ctypes.c_double),
                ("background", ctypes.c_double), ("amplitude", ctypes.c_double), ("noise_kind", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("noise_level", ctypes.c_double), ("ia_std_deg", ctypes.c_double),
                ("ia_corr", ctypes.c_double), ("seed", ctypes.c_uint64)]


class ct_profile_spec(ctypes.Structure):
    _fields_ = [("lv_center", _D3), ("lv_axis", _D3), ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
                ("n_depth", ctypes.c_int32), ("n_ha", ctypes.c_int32), ("ha_type", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ct_tune_result(ctypes.Structure):
    _fields_ = [("rho_path", ctypes.c_int32), ("seg_cap", ctypes.c_int32), ("stream_block", ctypes.c_int32),
                ("eig_compact", ctypes.c_int32), ("ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ct_track_params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_double), ("fa_min", ctypes.c_double), ("max_turn_deg", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class CTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"ct status {status}: {message}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every exported function.
_SIGNATURES = [
    ("ct_plan_create", ctypes.c_int32, [ctypes.POINTER(ct_params), _I64x3, ctypes.POINTER(ctypes.c_void_p)]),
    ("ct_plan_destroy", ctypes.c_int32, [ctypes.c_void_p]),
    ("ct_structure_tensor", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, _I64x3, _I64x3, _I64x3, _I64x3, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_eig_smallest", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_angles", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _I64x3, _I64x3, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_run_chunks", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(ct_item), ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    ("ct_run_box", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, _I64x3, _I64x3, _I64x3, _I64x3, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_plan_sync", ctypes.c_int32, [ctypes.c_void_p]),
    ("ct_plan_stats", ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ct_stats), ctypes.c_int32]),
    ("ct_eig_smallest_noalloc", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("ct_synth_annulus", ctypes.c_int32,
     [ctypes.POINTER(ct_synth_spec), _I64x3, _I64x3, _I64x3, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_transmural_profile", ctypes.c_int32,
     [ctypes.POINTER(ct_profile_spec), _I64x3, _I64x3, _I64x3, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p]),
    ("ct_track", ctypes.c_int32,
     [ctypes.POINTER(ct_track_params), _I64x3, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ct_plan_profile", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    ("ct_plan_kernel_times", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(ct_kernel_time), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("ct_autotune", ctypes.c_int32,
     [ctypes.POINTER(ct_params), _I64x3, ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p,
      ctypes.POINTER(ct_tune_result)]),
    ("ct_fp32_fma_rate", ctypes.c_int32,
     [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
      ctypes.POINTER(ctypes.c_double)]),
    ("ct_last_error", ctypes.c_char_p, []),
    ("ct_radius", ctypes.c_int32, [ctypes.c_double, ctypes.c_double]),
]


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the CUDA library (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None or path is not None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise FileNotFoundError(f"CUDA library not built: {p} (run paper_2508_07476_gb300.build.build())")
        lib = ctypes.CDLL(p)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is not None:
            return lib
        _lib = lib
    return _lib


def exported_names() -> Iterable[str]:
    return [s[0] for s in _SIGNATURES]


def _check(status: int):
    if status != CT_OK:
        raise CTError(status, ct_last_error())


def _i64x3(v: Sequence[int]):
    return _I64x3(*[int(a) for a in v])


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(sigma: float, rho: float, lv_center, lv_axis, precision: int = CT_PREC_FP32,
                vec_type: int = CT_OUT_F32, angle_type: int = CT_OUT_F32, fa_type: int = CT_OUT_F32,
                fill_value: float = math.nan, truncate: float = 4.0, chunk=(0, 0, 0), flags: int = 0,
                spacing=(0.0, 0.0, 0.0), lv_centres=None) -> ct_params:
    """ct_params; ``lv_centres`` (a sequence of (cx, cy) per z slice) is kept alive on the
    returned object until the plan has copied it."""
    p = ct_params()
    p.spacing = _D3(*spacing)
    if lv_centres is not None:
        flat = [float(v) for pair in lv_centres for v in pair]
        buf = (ctypes.c_double * len(flat))(*flat)
        p._centres_keep = buf
        p.lv_centres = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
    p.sigma, p.rho, p.truncate = sigma, rho, truncate
    p.lv_center = _D3(*lv_center)
    p.lv_axis = _D3(*lv_axis)
    p.precision, p.vec_type, p.angle_type, p.fa_type = precision, vec_type, angle_type, fa_type
    p.fill_value = fill_value
    p.flags = flags
    p.chunk = _i64x3(chunk)
    return p


def ct_plan_create(params: ct_params, vol_dims: Sequence[int]) -> ctypes.c_void_p:
    plan = ctypes.c_void_p()
    _check(load().ct_plan_create(ctypes.byref(params), _i64x3(vol_dims), ctypes.byref(plan)))
    return plan


def ct_plan_destroy(plan) -> None:
    _check(load().ct_plan_destroy(plan))


def ct_structure_tensor(plan, vol, in_lo, in_n, out_lo, out_n, S, stream=None) -> None:
    _check(load().ct_structure_tensor(plan, _ptr(vol), _i64x3(in_lo), _i64x3(in_n), _i64x3(out_lo), _i64x3(out_n),
                                      _ptr(S), _stream(stream)))


def ct_eig_smallest(plan, S, n: int, evals, evec, stream=None) -> None:
    _check(load().ct_eig_smallest(plan, _ptr(S), int(n), _ptr(evals), _ptr(evec), _stream(stream)))


def ct_eig_smallest_noalloc(S, n: int, evals, evec, precision: int = CT_PREC_FP32, stream=None) -> None:
    _check(load().ct_eig_smallest_noalloc(_ptr(S), int(n), _ptr(evals), _ptr(evec), int(precision), _stream(stream)))


def ct_angles(plan, evec, evals, out_lo, out_n, mask, vec, ha, ia, fa, stream=None) -> None:
    _check(load().ct_angles(plan, _ptr(evec), _ptr(evals), _i64x3(out_lo), _i64x3(out_n), _ptr(mask), _ptr(vec),
                            _ptr(ha), _ptr(ia), _ptr(fa), _stream(stream)))


def make_item(vol, dims, mask=None, vec=None, ha=None, ia=None, fa=None, sigma: float = 0.0, rho: float = 0.0,
              lv_center=(0.0, 0.0, 0.0), lv_axis=(0.0, 0.0, 0.0)) -> ct_item:
    it = ct_item()
    it.vol, it.mask = _ptr(vol), _ptr(mask)
    it.dims = _i64x3(dims)
    it.sigma, it.rho = sigma, rho
    it.lv_center = _D3(*lv_center)
    it.lv_axis = _D3(*lv_axis)
    it.vec, it.ha, it.ia, it.fa = _ptr(vec), _ptr(ha), _ptr(ia), _ptr(fa)
    return it


def ct_run_chunks(plan, items: Sequence[ct_item], items_on_host: bool, stream=None) -> None:
    arr = (ct_item * len(items))(*items)
    _check(load().ct_run_chunks(plan, arr, len(items), 1 if items_on_host else 0,
                                None if items_on_host else _stream(stream)))


def ct_run_box(plan, vol, in_lo, in_n, out_lo, out_n, mask, vec, ha, ia, fa, stream=None) -> None:
    _check(load().ct_run_box(plan, _ptr(vol), _i64x3(in_lo), _i64x3(in_n), _i64x3(out_lo), _i64x3(out_n), _ptr(mask),
                             _ptr(vec), _ptr(ha), _ptr(ia), _ptr(fa), _stream(stream)))


CT_SYNTH_FP32 = 1


def make_synth_spec(spec, flags: int = 0) -> ct_synth_spec:
    """C description of a synth.AnnulusSpec."""
    c = ct_synth_spec()
    c.flags = flags
    c.center = _D3(*spec.centre_xyz())
    c.axis = _D3(*[float(v) for v in spec.axis])
    c.r_in, c.r_out, c.period = spec.r_in, spec.r_out, spec.period
    c.ha_in_deg, c.ha_out_deg = spec.ha_in_deg, spec.ha_out_deg
    c.background, c.amplitude = spec.background, spec.amplitude
    kind, level = spec.noise
    c.noise_kind = {"gauss": 0, "poisson_like": 1}[kind]
    c.noise_level = level
    c.ia_std_deg, c.ia_corr = spec.ia_std_deg, spec.ia_corr
    c.seed = spec.seed
    return c


def ct_synth_annulus(spec, vol_dims, lo, n, vol, mask=None, stream=None, flags: int = 0) -> None:
    cs = make_synth_spec(spec, flags)
    _check(load().ct_synth_annulus(ctypes.byref(cs), _i64x3(vol_dims), _i64x3(lo), _i64x3(n), _ptr(vol), _ptr(mask),
                                   _stream(stream)))


def make_profile_spec(lv_center, lv_axis, r_in: float, r_out: float, n_depth: int, n_ha: int,
                      ha_type: int = CT_OUT_F32) -> ct_profile_spec:
    p = ct_profile_spec()
    p.lv_center = _D3(*lv_center)
    p.lv_axis = _D3(*lv_axis)
    p.r_in, p.r_out = r_in, r_out
    p.n_depth, p.n_ha, p.ha_type, p.reserved = n_depth, n_ha, ha_type, 0
    return p


def ct_transmural_profile(spec: ct_profile_spec, vol_dims, lo, n, ha, mask, hist, stream=None) -> None:
    _check(load().ct_transmural_profile(ctypes.byref(spec), _i64x3(vol_dims), _i64x3(lo), _i64x3(n), _ptr(ha),
                                        _ptr(mask), _ptr(hist), _stream(stream)))


def make_track_params(step: float, max_steps: int, fa_min: float = 0.0, max_turn_deg: float = 90.0) -> ct_track_params:
    p = ct_track_params()
    p.step, p.fa_min, p.max_turn_deg, p.max_steps, p.reserved = step, fa_min, max_turn_deg, max_steps, 0
    return p


def ct_track(params: ct_track_params, vol_dims, vec, fa, mask, seeds, n_seeds: int, points, count,
             stream=None) -> None:
    _check(load().ct_track(ctypes.byref(params), _i64x3(vol_dims), _ptr(vec), _ptr(fa), _ptr(mask), _ptr(seeds),
                           int(n_seeds), _ptr(points), _ptr(count), _stream(stream)))


def ct_plan_sync(plan) -> None:
    _check(load().ct_plan_sync(plan))


def ct_plan_stats(plan, reset: bool = False) -> dict:
    s = ct_stats()
    _check(load().ct_plan_stats(plan, ctypes.byref(s), 1 if reset else 0))
    return {k: getattr(s, k) for k, _ in ct_stats._fields_}


def ct_plan_profile(plan, enable: bool) -> None:
    _check(load().ct_plan_profile(plan, 1 if enable else 0))


def ct_plan_kernel_times(plan) -> dict:
    """{kernel name: (launches, total ms)} since the last call (clears the records)."""
    buf = (ct_kernel_time * 64)()
    n = ctypes.c_int32(0)
    _check(load().ct_plan_kernel_times(plan, buf, 64, ctypes.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n.value)}


def ct_autotune(params: ct_params, vol_dims, masked: bool, cache_file: Optional[str] = None, chunk=None) -> dict:
    """Time the kernel choices for volumes of this size and scale (on the whole
    volume, or on one chunk of it); store the best in cache_file."""
    r = ct_tune_result()
    path = None if cache_file is None else os.fsencode(cache_file)
    ch = None if chunk is None else ctypes.cast(_i64x3(chunk), ctypes.c_void_p)
    _check(load().ct_autotune(ctypes.byref(params), _i64x3(vol_dims), ch, int(bool(masked)), path, ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in ct_tune_result._fields_ if k != "reserved"}


def ct_fp32_fma_rate(iterations: int = 200000) -> dict:
    """Measured FP32 FMA rate of the current device: {fma_per_s, sms, ms}."""
    rate, sms, ms = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
    _check(load().ct_fp32_fma_rate(int(iterations), ctypes.byref(rate), ctypes.byref(sms), ctypes.byref(ms)))
    return {"fma_per_s": rate.value, "sms": sms.value, "ms": ms.value}


def ct_last_error() -> str:
    return load().ct_last_error().decode()


def ct_radius(s: float, truncate: float = 4.0) -> int:
    return int(load().ct_radius(s, truncate))
