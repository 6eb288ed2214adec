"""Plants plausible mistakes in a copy of the CPU oracle (on the CPU only) and checks that
at least one pin in test_oracle_pins.py fails for each: a pin that cannot tell a wrong
oracle from the right one pins nothing."""
import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_lit as lpins
from tests import test_oracle_msaa as mpins
from tests import test_oracle_threshold as tpins

MUTANTS = {
    # fill rule: right/bottom edges owned instead of left/top
    "owned_rule_flipped": ("return dy < 0 || (dy == 0 && dx > 0);",
                           "return dy > 0 || (dy == 0 && dx < 0);",
                           [pins.test_rect_coverage_closed_form]),
    # barycentric weights attached to the wrong vertices
    "weights_swapped": ("float l1 = (float)e1 * tri->inv;", "float l1 = (float)e2 * tri->inv;",
                        [pins.test_depth_key_is_screen_linear_inverse_w]),
    # ties resolved with the lower quad index on top
    "tie_direction": ("if (a->j != b->j) return a->j < b->j ? -1 : 1;",
                      "if (a->j != b->j) return a->j < b->j ? 1 : -1;",
                      [pins.test_equal_depth_tie_higher_index_on_top]),
    # nearest drawn first: sorted descending instead of ascending
    "order_reversed": ("if (a->key != b->key) return a->key < b->key ? -1 : 1;",
                       "if (a->key != b->key) return a->key < b->key ? 1 : -1;",
                       [pins.test_two_layers_closed_form_and_order]),
    # snapping by truncation instead of round-half-even
    "snap_truncates": ("out->X[k] = (int32_t)rintf(sx * 256.0f);",
                       "out->X[k] = (int32_t)(sx * 256.0f);",
                       [pins.test_snap_rounds_half_to_even]),
    # screen-space (not perspective-correct) colour interpolation
    "affine_colour": ("double wk = l[k] * (double)tri->q[k];", "double wk = l[k];",
                      [pins.test_perspective_correct_vertex_colour]),
    # backward drops the colour of the fragments behind
    "backward_no_behind": ("ga += g[c] * T * (cc[c] - behind[i * 4 + c]);",
                           "ga += g[c] * T * cc[c];",
                           [pins.test_backward_matches_central_differences]),
    # wrong quad diagonal for the second triangle: leaves holes / overlaps
    "wrong_diagonal": ("static const int corner[2][3] = {{0, 1, 2}, {0, 2, 3}};",
                       "static const int corner[2][3] = {{0, 1, 2}, {1, 2, 3}};",
                       [pins.test_exactly_once_jittered_grid]),
    # composite forgets to attenuate what is behind
    "over_no_attenuation": ("float keep = om * C[c];", "float keep = C[c];",
                            [pins.test_two_layers_closed_form_and_order]),
    # alpha threshold: the stop test made strict (T = t_min keeps blending)
    "threshold_strict": ("if (!(T > job->t_min)) break;", "if (!(T >= job->t_min)) break;",
                         [tpins.test_stack_closed_form]),
    # alpha threshold: fragments weighted by their own alpha only (no transmittance)
    "threshold_no_transmittance": ("float w = T * a;", "float w = a;",
                                   [tpins.test_stack_closed_form]),
    # multisampling: coverage still tested at the pixel centre
    "sample_position_ignored": ("int64_t Px = 256 * (int64_t)px + s->sample_x, Py = 256 * (int64_t)py + s->sample_y;",
                                "int64_t Px = 256 * (int64_t)px + 128, Py = 256 * (int64_t)py + 128;",
                                [mpins.test_partial_coverage_closed_form]),
    # lighting: one-sided Lambert (back faces dark)
    "lit_one_sided": ("fabs(n[0] * L[0] + n[1] * L[1] + n[2] * L[2])", "(n[0] * L[0] + n[1] * L[1] + n[2] * L[2])",
                      [lpins.test_lighting_invariances]),
    # lighting: normals interpolated without the perspective weights
    "lit_affine_normal": ("for (int c = 0; c < 3; ++c) n[c] += wk * (double)ck[4 + c];",
                          "for (int c = 0; c < 3; ++c) n[c] += l[k] * (double)ck[4 + c];",
                          [lpins.test_normal_interpolation_on_a_tilted_quad]),
    # near plane ignored
    "no_near_cull": ("} else if (!(w >= s->near_z && w <= s->far_z)) {",
                     "} else if (!(w <= s->far_z)) {",
                     [pins.test_cull_rules]),
}


def _call(test):
    # parametrised pins: run the default-argument form of each
    if test is pins.test_rect_coverage_closed_form:
        test(False, 0)
    elif test is tpins.test_stack_closed_form:
        test(0.5, 7)
    elif test is mpins.test_partial_coverage_closed_form:
        test(4)
    elif test is lpins.test_lighting_invariances:
        test("negate_normals")
    else:
        test()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_mutant(name, tmp_path):
    old, new, catching = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    lib = oracle.build_variant(src.replace(old, new), str(tmp_path))
    oracle.use_library(lib)
    try:
        for test in catching:
            with pytest.raises(AssertionError):
                _call(test)
    finally:
        oracle.use_library(None)
    # and the unmodified oracle passes the same pins
    for test in catching:
        _call(test)
