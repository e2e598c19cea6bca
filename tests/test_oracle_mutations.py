"""Plant one plausible mistake at a time in a copy of the oracle (CPU only) and
check that at least one pin fails.  A pin set that a dropped term, a wrong
sign or index, or a transposed operand slips through is no pin."""
import numpy as np
import pytest

import test_oracle_eigen_angles as TE
import test_oracle_filters as TF
from conftest import read_golden
from oracle import oracle as O

MUTATIONS = {
    "derivative_sign": ("c[k + R] = ((double)k / (s * s)) * w[k + R];", "c[k + R] = (-(double)k / (s * s)) * w[k + R];"),
    "smoothing_not_normalised": ("w[k + R] /= sum;", "w[k + R] /= (sum * 1.0000001);"),
    "transposed_product": ("static const int cb[6] = {0, 1, 2, 1, 2, 2};", "static const int cb[6] = {0, 1, 2, 2, 1, 2};"),
    "clamp_off_by_one": ("int64_t q = clampi(pa + k, 0, dims[axis] - 1)", "int64_t q = clampi(pa + k, 0, dims[axis] - 2)"),
    "dropped_outer_tap": ("for (int k = 1; k <= R; ++k) {", "for (int k = 1; k < R; ++k) {"),
    "wrong_pass_axis": ("if ((rc = pass1d(t1, &bz, t2, &by, 1, w[1], Rr[1], 0, dims))) goto done;",
                        "if ((rc = pass1d(t1, &bz, t2, &by, 1, w[1], Rr[1] - 1, 0, dims))) goto done;"),
    "theta_cross_reversed": ("double et[3] = {ez[1] * er[2] - ez[2] * er[1],",
                             "double et[3] = {-ez[1] * er[2] + ez[2] * er[1],"),
    "ia_from_wrong_component": ("double s = vr > 1.0 ? 1.0 : (vr < -1.0 ? -1.0 : vr);",
                                "double s = vt > 1.0 ? 1.0 : (vt < -1.0 ? -1.0 : vt);"),
    "fa_missing_half": ("return sqrt(0.5 * num / den);", "return sqrt(num / den);"),
    "eig_sorted_descending": ("if (d[idx[j]] < d[idx[i]]) {", "if (d[idx[j]] > d[idx[i]]) {"),
    "jacobi_rotation_sign": ("A[k][p] = cs * akp - sn * akq;", "A[k][p] = cs * akp + sn * akq;"),
    "fa_no_clamp": ("double l1 = ev[0] > 0.0 ? ev[0] : 0.0,", "double l1 = ev[0],"),
}


def _pins():
    """Every pin of the two pin modules, as (name, callable)."""
    pins = [
        ("kernels", lambda: [TF.test_kernels_normalised_and_match_scipy(s) for s in (1.0, 1.5, 2.0)]),
        ("gradient_scipy", lambda: TF.test_gradient_matches_scipy((16, 18, 20), 1.0)),
        ("tensor_scipy", lambda: TF.test_structure_tensor_matches_scipy((16, 18, 20), 1.0, 3.0)),
        ("brute", TF.test_brute_force_triple_sum_tiny),
        ("ramp", lambda: TF.test_linear_ramp_closed_form(1.0)),
        ("constant", TF.test_constant_volume_is_exactly_zero),
        ("symmetry", TF.test_axis_flip_and_transpose_symmetry),
        ("eig_golden", lambda: [TE.test_eig_golden(r) for r in read_golden("eig3.txt")]),
        ("eig_lapack", TE.test_eig_matches_lapack_and_invariants),
        ("fa_golden", lambda: [TE.test_fa_golden(r) for r in read_golden("fa.txt")]),
        ("ha_ia_golden", lambda: [TE.test_ha_ia_golden(r) for r in read_golden("ha_ia.txt")]),
        ("ha_ia_frame", TE.test_ha_ia_axis_sign_and_orientation),
    ]
    return pins


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = O.source_text()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    lib = O.compile_variant(src.replace(old, new, 1), str(tmp_path / f"libmut_{name}.so"))
    caught = []
    with O.use_library(lib):
        for pin, fn in _pins():
            try:
                fn()
            except (AssertionError, RuntimeError):
                caught.append(pin)
    assert caught, f"no pin failed with planted mistake {name}"


def test_unmutated_oracle_passes_every_pin():
    for pin, fn in _pins():
        fn()
