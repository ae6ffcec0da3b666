"""Planted mistakes: each copy of the oracle with one plausible bug must fail a pin.

The mistake is planted in a temporary copy of the oracle's C source (never in
the product), compiled on the CPU and run against the same pins as the real
oracle.  A mutant that passes every pin would mean the pins cannot see that
kind of error.
"""
import shutil
import subprocess
from pathlib import Path

import pytest

import oracle
import oracle_pins as pins

MUTANTS = {
    "pixel_centre_drops_half": ("((double)i + 0.5)", "((double)i + 0.0)"),
    "tie_on_plane_goes_down": ("return vw->D[b] >= 0;", "return vw->D[b] > 0;"),
    "chord_transposed_denominators": ("i128 num = texit.num * t.den - t.num * texit.den;",
                                      "i128 num = texit.num * texit.den - t.num * t.den;"),
    "exit_picks_latest_face": ("if (!have_exit || time_cmp(e, texit) < 0) texit = e;",
                               "if (!have_exit || time_cmp(e, texit) > 0) texit = e;"),
    "vlos_drops_z_term": ("* cam->w[2];", "* 0.0;"),
    "level_rule_strict": ("<= (double)cam->nx &&", "< (double)cam->nx &&"),
    "midplane_off_by_one_cell": ("((int64_t)tr->coord[3 * oct + b] + 1) << (OR_K - lvl)",
                                 "((int64_t)tr->coord[3 * oct + b]) << (OR_K - lvl)"),
    "box_entry_sign_for_negative_direction": ("en.num = (i128)X0[a] - box;", "en.num = (i128)X0[a];"),
    "max_mode_keeps_minimum": ("if (cnt == 0 || r > M) M = r;", "if (cnt == 0 || r < M) M = r;"),
    "neumaier_wrong_sign": ("a->c += (a->s - t) + x;", "a->c += (a->s - t) - x;"),
    "lambda_off_by_two": ("ldexp(sqrt(s2), -OR_K)", "ldexp(sqrt(s2), -OR_K + 1)"),
    "camera_cut_ignored": ("if (ch < 0 || lvl == vw->L) break;", "if (ch < 0) break;"),
    "direction_truncated": ("llrint(ldexp(cam->w[a] / m, OR_DBITS))", "(int64_t)(ldexp(cam->w[a] / m, OR_DBITS))"),
    "origin_truncated": ("X0[a] = bad ? 0 : llrint(ldexp(x[a], OR_K));", "X0[a] = bad ? 0 : (int64_t)(ldexp(x[a], OR_K));"),
    "value_from_sibling_cell": ("double r = rho[8 * oct + c];", "double r = rho[8 * oct + (c ^ 1)];"),
    "exit_uses_lower_face_going_up": ("(i128)(k + 1) * size - X0[b]", "(i128)k * size - X0[b]"),
    "slice_point_on_face_goes_low": ("c |= (X0[b] >= mid) << b;", "c |= (X0[b] > mid) << b;"),
    "slice_ignores_cut": ("if (ch < 0 || lvl == vw.L) {", "if (ch < 0) {"),
    "mean_level_off_by_one": ("nadd(&N, r * len * (double)lvl);", "nadd(&N, r * len * (double)(lvl + 1));"),
    "touched_marks_sibling_leaf": ("mark_cell(leaf_mark, oct, c);", "mark_cell(leaf_mark, oct, c ^ 1);"),
    "touched_marks_child_not_parent": ("mark_cell(inner_mark, oct, c);", "mark_cell(inner_mark, ch, c);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.SRC.read_text()
    assert src.count(old) == 1, f"mutation site not unique/present: {old!r}"
    msrc = tmp_path / "amr_oracle.c"
    msrc.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mutant.so"
    cmd = oracle.compile_command(lib_path)
    cmd[cmd.index(str(oracle.SRC))] = str(msrc)
    subprocess.run(cmd, check=True, capture_output=True)
    lib = oracle.load(lib_path)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError) as e:
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
