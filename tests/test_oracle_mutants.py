"""Planted mistakes in the oracle must be caught by its pins.

Each case copies oracle/ff_oracle.c, plants one plausible mistake (a dropped term, a wrong sign, index or
operand, a wrong tie rule, wrong wiring of level or direction), compiles the copy with gcc and runs every pin
of tests/oracle_pins.py against it: at least one must fail.  Mistakes are chosen so that the copy stays in
bounds (every access the oracle makes is range-checked or clamped).
"""
import os

import pytest

import oracle
from tests import oracle_pins as P

MUTANTS = {
    "pyr_round_down": ("(a + b + d + e + 2) / 4", "(a + b + d + e + 1) / 4"),
    "pyr_wrong_column": ("x1 = mini(2 * x + 1, w - 1)", "x1 = mini(2 * x, w - 1)"),
    "wht_transposed_basis": ("WALSH8[u][i] * WALSH8[v][j]", "WALSH8[u][j] * WALSH8[v][i]"),
    "wht_anchor_off_by_one": ("int xx = clampi(x - 3 + j, 0, w - 1)", "int xx = clampi(x - 4 + j, 0, w - 1)"),
    "wht_store_transposed": ("out[c * 16 + u * 4 + v]", "out[c * 16 + v * 4 + u]"),
    "wht_wrong_walsh_row": ("{1, 1, -1, -1, -1, -1, 1, 1}", "{1, -1, -1, 1, 1, -1, -1, 1}"),
    "mix_wrong_shift": ("x ^= x >> 15;", "x ^= x >> 14;"),
    "hash_xy_swapped": ("(uint32_t)y * 65536u + (uint32_t)x", "(uint32_t)x * 65536u + (uint32_t)y"),
    "hash_drops_direction_step": ("(uint32_t)(d * 2 + comp)", "(uint32_t)(2 + comp)"),
    "sad_drops_last_coef": ("for (int k = 0; k < FFO_NF; k++) s += abs", "for (int k = 0; k < FFO_NF - 1; k++) s += abs"),
    "sad_wrong_target_column": ("fb + ((long)qy * w + qx)", "fb + ((long)qy * w + x)"),
    "quant_truncates": ("return c >= 0 ? c / 128 : -((-c + 127) / 128);", "return c / 128;"),
    "seed_last_tie_wins": ("if (d2 < best) {", "if (d2 <= best) {"),
    "seed_flow_sign": ("(int16_t)(best_q % w - p % w)", "(int16_t)(p % w - best_q % w)"),
    "upsample_not_doubled": ("int fx = 2 * flow_coarse[2 * pc]", "int fx = flow_coarse[2 * pc]"),
    "neighbour_wrong_quadrant": ("*n1x = (d == 0 || d == 2) ? x - 1 : x + 1;", "*n1x = (d == 0 || d == 1) ? x - 1 : x + 1;"),
    "colour_order_swapped": ("if ((x + y) % 2 != colour) continue;", "if ((x + y) % 2 == colour) continue;"),
    "accept_ties": ("if (cc >= 0 && cc < c) {\n                                fx = cx;", "if (cc >= 0 && cc <= c) {\n                                fx = cx;"),
    "random_accept_ties": ("if (cc >= 0 && cc < c) {\n                                    fx += ox;",
                           "if (cc >= 0 && cc <= c) {\n                                    fx += ox;"),
    "random_search_on_all_steps": ("if (d >= 1) {", "if (d >= 0) {"),
    "random_offset_not_centred": ("% (uint32_t)span) - rs_radius;\n                            int oy",
                                  "% (uint32_t)span);\n                            int oy"),
    "random_cost_wrong_component": ("x, y, fx + ox, fy + oy);", "x, y, fx + ox, fy + ox);"),
    "random_iteration_not_in_hash": ("ffo_hash(seed, dir, level, t, d, lx, ly, 0)", "ffo_hash(seed, dir, level, 0, d, lx, ly, 0)"),
    "random_direction_not_in_hash": ("ffo_hash(seed, dir, level, t, d, lx, ly, 1)", "ffo_hash(seed, 0, level, t, d, lx, ly, 1)"),
    "random_base_before_neighbours": ("int32_t cc = cost_of(cs, x, y, fx + ox, fy + oy);",
                                      "int32_t cc = cost_of(cs, x, y, flow[2 * p] + ox, flow[2 * p + 1] + oy);"),
    "grid_source_not_strided": ("ffo_sad(cs->fa, cs->fb, cs->w, cs->h, cs->g * x, cs->g * y, fx, fy)",
                                "ffo_sad(cs->fa, cs->fb, cs->w, cs->h, x, y, fx, fy)"),
    "grid_hash_in_grid_coordinates": ("int lx = cs->g * x, ly = cs->g * y;", "int lx = x, ly = y;"),
    "grid_handover_not_clamped": ("int fx = clampi(x + flow_parent[2 * pp], 0, cs->w - 1) - x;",
                                  "int fx = flow_parent[2 * pp];"),
    "grid_handover_wrong_parent": ("long pp = (long)mini(v / 2, ph - 1) * pw + mini(u / 2, pw - 1)",
                                   "long pp = (long)mini(v, ph - 1) * pw + mini(u, pw - 1)"),
    "upsample_grid_parent_in_grid_coordinates": ("int x = cs->g * u, y = cs->g * v;\n            int px",
                                                 "int x = u, y = v;\n            int px"),
    "sub_scales_skipped": ("const int k_first = s == L - 1 ? 0 : n_sub;", "const int k_first = 0;"),
    "level_not_in_hash": ("prm->rs_radius, prm->seed, dir, s + 8 * k, -1)", "prm->rs_radius, prm->seed, dir, 8 * k, -1)"),
    "inverse_same_direction_key": ("ws, hs, prm, 1,", "ws, hs, prm, 0,"),
    "consistency_strict": ("<= (long)eps * eps", "< (long)eps * eps"),
    "consistency_sign": ("long ex = fx + bwd[2 * q]", "long ex = fx - bwd[2 * q]"),
    "second_check_same_stream": ("ws, hs, &p2, 2,", "ws, hs, &p2, 1,"),
    "second_check_first_inverse_key": ("ws, hs, p1, 1,", "ws, hs, p1, 0,"),
    "second_check_radius_ignored": ("p2.rs_radius = rs_radius2;", "p2.rs_radius = prm->rs_radius;"),
    "second_check_ignored": ("mask[p] = (uint8_t)(mask[p] & m2[p]);", "mask[p] = (uint8_t)(mask[p] | m2[p]);"),
    "census_not_strict": ("if (v < centre) bits |= (uint64_t)1 << k;", "if (v <= centre) bits |= (uint64_t)1 << k;"),
    "census_reversed": ("if (v < centre) bits |= (uint64_t)1 << k;", "if (v > centre) bits |= (uint64_t)1 << k;"),
    "census_centre_counted": ("if (dy == 0 && dx == 0) continue;", "if (dy == 9) continue;"),
    "census_wrong_window": ("for (int dx = -3; dx <= 3; dx++) {", "for (int dx = -2; dx <= 4; dx++) {"),
    "hamming_drops_channel": ("for (int c = 0; c < 3; c++) s += popcount64(", "for (int c = 0; c < 2; c++) s += popcount64("),
    "sparsify_error_sign": ("long ex = (long)fx + bwd[2 * q]", "long ex = (long)fx - bwd[2 * q]"),
    "sparsify_last_tie_wins": ("if (best_p < 0 || e < best_e) {", "if (best_p < 0 || e <= best_e) {"),
    "sparsify_count_off": ("if (count >= s && best_p >= 0)", "if (count > s && best_p >= 0)"),
    "sparsify_block_4": ("for (int bx = 0; bx < w; bx += 3) {", "for (int bx = 0; bx < w; bx += 4) {"),
    "sparsify_mask_ignored": ("if (keep && !keep[p]) continue;", "(void)keep;"),
}


# Cross-checks that compare the oracle with a restatement of its own loop or a recomposition of its own steps:
# they run, but a planted mistake must also be caught by a pin that comes from outside the oracle.
CROSS_CHECKS = {"check_propagation_schedule", "check_pipeline_composition"}
PINS = [c for c in P.ALL_CHECKS if c.__name__ not in CROSS_CHECKS]

# Mistakes in the random search, its key and the sub-scale grids, with the pin (derived from the definition)
# that must catch each.
EXPECTED_PIN = {
    "random_search_on_all_steps": "check_random_search_moves",
    "random_offset_not_centred": "check_random_search_finds_negative_offset",
    "level_not_in_hash": "check_stream_keys",
    "random_iteration_not_in_hash": "check_random_search_moves",
    "random_direction_not_in_hash": "check_random_search_moves",
    "inverse_same_direction_key": "check_stream_keys",
    "grid_source_not_strided": "check_sub_scale_propagation",
    "grid_hash_in_grid_coordinates": "check_sub_scale_propagation",
    "grid_handover_not_clamped": "check_sub_scale_handovers",
    "grid_handover_wrong_parent": "check_sub_scale_handovers",
    "upsample_grid_parent_in_grid_coordinates": "check_sub_scale_handovers",
    "sub_scales_skipped": "check_sub_scale_translation",
}


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(os.path.dirname(oracle.__file__), "ff_oracle.c")) as f:
        return f.read()


def _fails(check, mutant):
    try:
        check(mutant)
    except Exception:  # an assertion, or the oracle reporting a broken internal assertion
        return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site not unique: {old!r}"
    src = tmp_path / "ff_oracle_mutant.c"
    src.write_text(source.replace(old, new))
    lib = oracle.load_library(oracle.compile_library(str(src), str(tmp_path / f"libffo_{name}.so")))
    mutant = oracle.Oracle(lib)
    caught_by = next((c.__name__ for c in PINS if _fails(c, mutant)), None)
    assert caught_by is not None, f"no pin outside the cross-checks catches the planted mistake {name}"
    if name in EXPECTED_PIN:
        pin = EXPECTED_PIN[name]
        assert _fails(getattr(P, pin), mutant), f"{pin} does not catch {name} (first caught by {caught_by})"
