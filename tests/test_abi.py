"""The C-ABI library builds for sm_103a, loads, exports every function that
include/ct.h declares, lays out its structs as ctypes does, and validates
arguments before touching a device.  No compute call runs here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2508_07476_gb300 import _lib, build
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ct.h")


def header_functions():
    names = []
    with open(HEADER) as f:
        for line in f:
            m = re.match(r"^\s*(?:const\s+)?(?:ct_status|int32_t|char\s*\*|const char\s*\*|void)\s*\**\s*(ct_\w+)\s*\(",
                         line)
            if m:
                names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_lists_the_boundary():
    names = set(header_functions())
    for required in ("ct_plan_create", "ct_plan_destroy", "ct_structure_tensor", "ct_eig_smallest", "ct_angles",
                     "ct_run_chunks", "ct_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) == set(_lib.exported_names())
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(header_functions()) <= exported


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "ct.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu\\n", sizeof(ct_params), offsetof(ct_params, precision),'
        " offsetof(ct_params, fill_value), offsetof(ct_params, chunk), sizeof(ct_item));\n"
        'printf("%zu %zu %zu\\n", offsetof(ct_item, dims), offsetof(ct_item, vec), sizeof(ct_stats));\n'
        'printf("%zu %zu %zu %zu %zu\\n", sizeof(ct_synth_spec), offsetof(ct_synth_spec, flags),'
        " offsetof(ct_synth_spec, seed), sizeof(ct_profile_spec), offsetof(ct_profile_spec, n_depth));\n"
        'printf("%zu %zu\\n", sizeof(ct_track_params), offsetof(ct_track_params, max_steps));\n'
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    a, b, c, d = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:4]
    c_vals = [int(v) for v in (a.split() + b.split() + c.split() + d.split())]
    py_vals = [ctypes.sizeof(_lib.ct_params), _lib.ct_params.precision.offset, _lib.ct_params.fill_value.offset,
               _lib.ct_params.chunk.offset, ctypes.sizeof(_lib.ct_item), _lib.ct_item.dims.offset,
               _lib.ct_item.vec.offset, ctypes.sizeof(_lib.ct_stats), ctypes.sizeof(_lib.ct_synth_spec),
               _lib.ct_synth_spec.flags.offset, _lib.ct_synth_spec.seed.offset, ctypes.sizeof(_lib.ct_profile_spec),
               _lib.ct_profile_spec.n_depth.offset, ctypes.sizeof(_lib.ct_track_params),
               _lib.ct_track_params.max_steps.offset]
    assert c_vals == py_vals


@pytest.mark.parametrize("s", [0.5, 1.0, 1.5, 2.0, 3.0, 6.0, 9.0])
def test_radius_matches_oracle(libpath, s):
    assert _lib.ct_radius(s) == O.radius(s)


def _create(**kw):
    base = dict(sigma=1.0, rho=3.0, lv_center=(1.0, 2.0, 3.0), lv_axis=(0.0, 0.0, 1.0))
    base.update(kw)
    dims = base.pop("dims", (16, 16, 16))
    return _lib.ct_plan_create(_lib.make_params(**base), dims)


@pytest.mark.parametrize("kw,needle", [
    (dict(sigma=0.0), "sigma"),
    (dict(rho=-1.0), "rho"),
    (dict(sigma=float("nan")), "sigma"),
    (dict(lv_axis=(0.0, 0.0, 0.0)), "axis"),
    (dict(lv_center=(float("inf"), 0.0, 0.0)), "lv_center"),
    (dict(precision=7), "precision"),
    (dict(angle_type=9), "angle_type"),
    (dict(vec_type=_lib.CT_OUT_U8Q), "vec_type"),
    (dict(flags=1), "flags"),
    (dict(chunk=(-1, 0, 0)), "chunk"),
    (dict(dims=(0, 4, 4)), "vol_dims"),
])
def test_invalid_arguments_are_rejected(libpath, kw, needle):
    with pytest.raises(_lib.CTError) as ei:
        _create(**kw)
    assert ei.value.status == _lib.CT_ERR_INVALID
    assert needle in _lib.ct_last_error()


def test_unsupported_radius(libpath):
    with pytest.raises(_lib.CTError) as ei:
        _create(rho=12.0)  # R = 48 > 36
    assert ei.value.status == _lib.CT_ERR_UNSUPPORTED


def test_null_plan_calls_are_invalid(libpath):
    lib = _lib.load()
    z = _lib._i64x3((0, 0, 0))
    one = _lib._i64x3((1, 1, 1))
    assert lib.ct_structure_tensor(None, None, z, one, z, one, None, None) == _lib.CT_ERR_INVALID
    assert lib.ct_eig_smallest(None, None, 1, None, None, None) == _lib.CT_ERR_INVALID
    assert lib.ct_run_chunks(None, None, 0, 0, None) == _lib.CT_ERR_INVALID
    assert lib.ct_plan_destroy(None) == _lib.CT_OK


def test_no_device_is_reported_without_fallback(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(_lib.CTError) as ei:
        _create()
    assert ei.value.status == _lib.CT_ERR_NO_DEVICE


def test_noalloc_entry_point_is_exported(libpath):
    assert "ct_eig_smallest_noalloc" in header_functions()
    assert hasattr(ctypes.CDLL(libpath), "ct_eig_smallest_noalloc")


@pytest.mark.parametrize("args,needle", [
    ((None, 4, None, 16, 0), "NULL"),          # no tensors
    ((16, 4, None, None, 0), "NULL"),          # no eigenvector output
    ((16, 4, None, 16, 7), "precision"),
    ((16, -1, None, 16, 0), "n must be"),
    ((16, (1 << 20) + 1, None, 16, 1), "exceeds"),  # above the static scratch's 2^20 tensors
])
def test_noalloc_validates_before_any_cuda_call(libpath, args, needle):
    # the checks run on the host before the device is touched, so they hold
    # without a GPU (the pointers are never dereferenced)
    lib = _lib.load()
    S, n, ev, vec, prec = args
    st = lib.ct_eig_smallest_noalloc(S, n, ev, vec, prec, None)
    assert st == _lib.CT_ERR_INVALID
    assert needle in _lib.ct_last_error()


def test_noalloc_zero_tensors_is_a_no_op(libpath):
    assert _lib.load().ct_eig_smallest_noalloc(16, 0, None, 16, 0, None) == _lib.CT_OK


def test_autotune_validates_before_any_cuda_call(libpath):
    lib = _lib.load()
    p = _lib.make_params(1.0, 3.0, (0, 0, 0), (0, 0, 1))
    res = _lib.ct_tune_result()
    assert lib.ct_autotune(ctypes.byref(p), _lib._i64x3((16, 16, 16)), None, 0, None, None) == _lib.CT_ERR_INVALID
    assert lib.ct_autotune(ctypes.byref(p), _lib._i64x3((0, 16, 16)), None, 0, None,
                           ctypes.byref(res)) == _lib.CT_ERR_INVALID
    bad = _lib.make_params(1.0, 3.0, (0, 0, 0), (0, 0, 0))
    assert lib.ct_autotune(ctypes.byref(bad), _lib._i64x3((16, 16, 16)), None, 0, None,
                           ctypes.byref(res)) == _lib.CT_ERR_INVALID
