"""Python face of the FP64 CPU oracle (``ct_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares nothing with the
CUDA path; the two meet only through the seeded inputs of ``synth``.

``build()`` compiles ``ct_oracle.c`` with gcc (FP64, OpenMP) into
``oracle/_build/libct_oracle.so``; every other function calls into that
library through ctypes with numpy arrays.  Arrays are ``[z, y, x]``; boxes and
positions are ``(x, y, z)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ct_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libct_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    lib.cto_radius.argtypes = [D, D]
    lib.cto_radius.restype = ctypes.c_int
    lib.cto_kernels.argtypes = [D, D, P, P]
    lib.cto_gradient.argtypes = [P, P, P, P, D, D, P]
    lib.cto_structure_tensor.argtypes = [P, P, P, P, D, D, D, P]
    lib.cto_eig3.argtypes = [P, P, P]
    lib.cto_eig_field.argtypes = [P, ctypes.c_int64, P, P]
    lib.cto_fa.argtypes = [P]
    lib.cto_fa.restype = D
    lib.cto_ha_ia.argtypes = [P, P, P, P, P, P, P]
    lib.cto_angles_field.argtypes = [P, P, P, P, P, P, P, P, D, P, P, P, P]
    lib.cto_angles_field3.argtypes = [P, P, P, P, P, P, P, P, P, P, D, P, P, P, P]
    lib.cto_pipeline.argtypes = [P, P, P, P, D, D, D, P, P, P, D, P, P, P, P, P, P]
    lib.cto_pipeline3.argtypes = [P, P, P, P, D, D, D, P, P, P, P, P, D, P, P, P, P, P, P]
    lib.cto_num_threads.restype = ctypes.c_int
    lib.cto_set_num_threads.argtypes = [ctypes.c_int]
    return lib


class use_library:
    """Temporarily route every call to another build of the oracle (used by the
    tests that plant a mistake in a copy of the source and expect a pin to fail)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile C source text with the oracle's flags (for planted-mistake tests)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", out_path, c_path, "-lm"],
                   check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i64(v: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def _dims(vol: np.ndarray) -> np.ndarray:
    nz, ny, nx = vol.shape
    return _i64([nx, ny, nz])


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(_load().cto_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of later calls (OpenMP); the benchmark times a 1-core figure with it."""
    _load().cto_set_num_threads(int(n))


def radius(s: float, truncate: float = 4.0) -> int:
    return int(_load().cto_radius(s, truncate))


def kernels(s: float, truncate: float = 4.0):
    """(w, c): smoothing taps and derivative-correlation taps, k = -R..R."""
    R = radius(s, truncate)
    w = np.zeros(2 * R + 1)
    c = np.zeros(2 * R + 1)
    _check(_load().cto_kernels(s, truncate, _p(w), _p(c)), "kernels")
    return w, c


def _box(vol, lo, n):
    nz, ny, nx = vol.shape
    lo = (0, 0, 0) if lo is None else tuple(lo)
    n = (nx - lo[0], ny - lo[1], nz - lo[2]) if n is None else tuple(n)
    return _i64(lo), _i64(n)


def gradient(vol: np.ndarray, sigma: float, lo=None, n=None, truncate: float = 4.0) -> np.ndarray:
    """g as array [3, nz, ny, nx] (components x, y, z) over the box (lo, n)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    lo, n = _box(vol, lo, n)
    g = np.zeros((3, n[2], n[1], n[0]))
    _check(_load().cto_gradient(_p(vol), _p(_dims(vol)), _p(lo), _p(n), sigma, truncate, _p(g)), "gradient")
    return g


def structure_tensor(vol: np.ndarray, sigma: float, rho: float, lo=None, n=None, truncate: float = 4.0) -> np.ndarray:
    """S as array [6, nz, ny, nx] (xx, yy, zz, xy, xz, yz) over the box (lo, n)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    lo, n = _box(vol, lo, n)
    S = np.zeros((6, n[2], n[1], n[0]))
    _check(_load().cto_structure_tensor(_p(vol), _p(_dims(vol)), _p(lo), _p(n), sigma, rho, truncate, _p(S)),
           "structure_tensor")
    return S


def eig3(s6: Sequence[float]):
    """(eigenvalues ascending [3], eigenvectors [3, 3] with row k the vector of eigenvalue k)."""
    s6 = np.ascontiguousarray(np.asarray(s6, dtype=np.float64))
    ev = np.zeros(3)
    V = np.zeros(9)
    _check(_load().cto_eig3(_p(s6), _p(ev), _p(V)), "eig3")
    return ev, V.reshape(3, 3)


def eig_field(S: np.ndarray):
    """Eigenvalues [3, ...] and smallest-eigenvalue eigenvectors [3, ...] of S [6, ...]."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    shp = S.shape[1:]
    n = int(np.prod(shp))
    ev = np.zeros((3,) + shp)
    v1 = np.zeros((3,) + shp)
    _check(_load().cto_eig_field(_p(S), n, _p(ev), _p(v1)), "eig_field")
    return ev, v1


def fa(ev: Sequence[float]) -> float:
    ev = np.ascontiguousarray(np.asarray(ev, dtype=np.float64))
    return float(_load().cto_fa(_p(ev)))


def ha_ia(p, center, axis, v):
    """(HA, IA, oriented v) in degrees at position p; (None, None, None) on the axis."""
    arr = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (p, center, axis, v)]
    ha = np.zeros(1)
    ia = np.zeros(1)
    vo = np.zeros(3)
    ok = _load().cto_ha_ia(*[_p(a) for a in arr], _p(ha), _p(ia), _p(vo))
    if not ok:
        return None, None, None
    return float(ha[0]), float(ia[0]), vo


def angles_field(v1, evals, dims_xyz, lo, n, center, axis, mask=None, fill=float("nan"), spacing=None,
                 centres=None):
    """(v oriented [3,...], HA, IA, FA) for a box, from smallest eigenvectors and eigenvalues
    (``spacing`` / ``centres`` as in ``pipeline``)."""
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    evals = np.ascontiguousarray(evals, dtype=np.float64)
    shp = v1.shape[1:]
    vout = np.zeros((3,) + shp)
    ha = np.zeros(shp)
    ia = np.zeros(shp)
    fa_ = np.zeros(shp)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    c = np.ascontiguousarray(np.asarray(center, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(axis, dtype=np.float64))
    if spacing is None and centres is None:
        _check(_load().cto_angles_field(_p(v1), _p(evals), _p(_i64(dims_xyz)), _p(_i64(lo)), _p(_i64(n)), _p(c),
                                         _p(a), _p(m), fill, _p(vout), _p(ha), _p(ia), _p(fa_)), "angles_field")
        return vout, ha, ia, fa_
    sp = np.ascontiguousarray(np.asarray((1.0, 1.0, 1.0) if spacing is None else spacing, dtype=np.float64))
    ce = None if centres is None else np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 2))
    _check(_load().cto_angles_field3(_p(v1), _p(evals), _p(_i64(dims_xyz)), _p(_i64(lo)), _p(_i64(n)), _p(c), _p(a),
                                      _p(sp), _p(ce), _p(m), fill, _p(vout), _p(ha), _p(ia), _p(fa_)), "angles_field")
    return vout, ha, ia, fa_


def pipeline(vol: np.ndarray, sigma: float, rho: float, center, axis, mask: Optional[np.ndarray] = None,
             lo=None, n=None, truncate: float = 4.0, fill: float = float("nan"), spacing=None,
             centres: Optional[np.ndarray] = None) -> dict:
    """All per-voxel outputs over the box (lo, n): S, evals, v (oriented), ha, ia, fa.

    ``spacing`` (x, y, z voxel size; sigma, rho, center and axis then in its
    units) and ``centres`` (per-slice LV centre, [nz, 2] as (cx, cy)) select
    the anisotropic form; S is then in physical units."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    lo, n = _box(vol, lo, n)
    shp = (int(n[2]), int(n[1]), int(n[0]))
    out = {
        "S": np.zeros((6,) + shp), "evals": np.zeros((3,) + shp), "v": np.zeros((3,) + shp),
        "ha": np.zeros(shp), "ia": np.zeros(shp), "fa": np.zeros(shp),
    }
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    c = np.ascontiguousarray(np.asarray(center, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(axis, dtype=np.float64))
    if spacing is None and centres is None:
        _check(_load().cto_pipeline(_p(vol), _p(_dims(vol)), _p(lo), _p(n), sigma, rho, truncate, _p(c), _p(a),
                                    _p(m), fill, _p(out["S"]), _p(out["evals"]), _p(out["v"]), _p(out["ha"]),
                                    _p(out["ia"]), _p(out["fa"])), "pipeline")
        return out
    sp = np.ascontiguousarray(np.asarray((1.0, 1.0, 1.0) if spacing is None else spacing, dtype=np.float64))
    ce = None if centres is None else np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 2))
    if ce is not None and ce.shape[0] != vol.shape[0]:
        raise ValueError("centres needs one (cx, cy) per z slice")
    _check(_load().cto_pipeline3(_p(vol), _p(_dims(vol)), _p(lo), _p(n), sigma, rho, truncate, _p(sp), _p(c), _p(a),
                                 _p(ce), _p(m), fill, _p(out["S"]), _p(out["evals"]), _p(out["v"]), _p(out["ha"]),
                                 _p(out["ia"]), _p(out["fa"])), "pipeline")
    return out
