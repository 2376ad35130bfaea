"""Plant mistakes in the oracle (on the CPU) and check that the pins catch every one.

Each mutant is an edited copy of the oracle's C source, compiled to a temporary library;
the pin battery of `test_oracle_pins` runs against it and at least one pin must fail.
"""
import pytest

import oracle
import test_oracle_block as blk
import test_oracle_pins as pins

MUTANTS = [
    ("momentum flux drops the pressure", "f = f + P;", "f = f;"),
    ("energy flux drops the pressure", "return (E + P) * v_d;", "return E * v_d;"),
    ("kinetic energy without the 1/2", "double KE = 0.5 *", "double KE = 1.0 *"),
    ("gamma instead of gamma - 1", "double P = (gamma - 1.0)", "double P = (gamma - 0.5)"),
    ("flux difference sign flipped", "flux = flux + (Fp - Fm)", "flux = flux + (Fm - Fp)"),
    ("difference scaled by 1/h, not 1/(2h)", "/ (2.0 * h[d])", "/ (h[d])"),
    ("centre weight 5 instead of 6", "+ 6.0 * Uc[p]", "+ 5.0 * Uc[p]"),
    ("outer dissipation point at +1, not +2", "+ Uc[p + 2 * s];", "+ Uc[p + s];"),
    ("dissipation added instead of subtracted", "= -flux - eps * diss;", "= -flux + eps * diss;"),
    ("velocity always along x", "double v_d = m[d] / rho;", "double v_d = m[0] / rho;"),
    ("momentum flux uses m_d for every component", "double f = m[c - 1] * v_d;", "double f = m[d] * v_d;"),
    ("y and z strides swapped (RHS)", "const i64 stride[3] = {1, isy, isz};\n    const double h[3]",
     "const i64 stride[3] = {1, isz, isy};\n    const double h[3]"),
    ("minus neighbour one cell too far", "euler_flux(U, isc, p - stride[d], d, c, gamma)",
     "euler_flux(U, isc, p - 2 * stride[d], d, c, gamma)"),
    ("grid spacing of the wrong axis", "const double h[3] = {hx, hy, hz};", "const double h[3] = {hy, hz, hx};"),
    ("stencil centre shifted", "- 2.0 * u[p] + u[p - s]", "- 2.0 * u[p + 1] + u[p - s]"),
    ("stencil ignores per-axis weights", "c[4 * d + (o - 1)]", "c[(o - 1)]"),
    ("stencil weights reversed", "c[4 * d + (o - 1)]", "c[4 * d + (4 - o)]"),
    ("stencil coefficient field off by one", "* a[p] *", "* a[p + 1] *"),
    ("stencil minus side at o-1", "+ u[p - s]);", "+ u[p - s + stride[d]]);"),
    ("block: lower block reads the upper plane", "-t2 * A[(i64)q * isc + p - isz]", "-t2 * A[(i64)q * isc + p + isz]"),
    ("block: diagonal G term on every entry", "const double diag = (m == n) ? 1.0 : 0.0;",
     "const double diag = 1.0;"),
    ("block: outputs of L and W swapped", "out[(i64)(50 + q) * osc + o] = t2", "out[(i64)q * osc + o + 0 * osc] = t2"),
    ("block: D uses 2 t2 B", "= 2.0 * t1 * B[(i64)q * isc + p]", "= 2.0 * t2 * B[(i64)q * isc + p]"),
]


def _battery(orc):
    """Run every pin that takes the oracle; return the names of those that failed."""
    checks = [
        (pins.test_constant_dyadic_field_gives_exact_zero, {}),
        (pins.test_constant_arbitrary_field_is_rounding_small, {}),
        (pins.test_linear_energy_at_rest, {"h": (1.0, 0.5, 2.0)}),
        (pins.test_quartic_fields_pin_dissipation, {"d": 0}),
        (pins.test_quartic_fields_pin_dissipation, {"d": 2}),
        (pins.test_reflection_symmetry, {}),
        (pins.test_axis_permutation_symmetry, {}),
        (pins.test_brute_force_exact_rationals_4cubed, {}),
        (pins.test_stencil_constant_is_exact_zero, {}),
        (pins.test_stencil_polynomials_exact_to_degree_9, {"d": 0}),
        (pins.test_stencil_polynomials_exact_to_degree_9, {"d": 1}),
        (pins.test_stencil_single_term_matches_library_correlation, {"d": 1, "o": 3}),
        (pins.test_stencil_full_weights_match_library_correlation, {}),
    ] + [(pins.test_one_dimensional_flow_closed_form, {"d": d}) for d in range(3)] + [
        (blk.test_block_closed_form_exact_on_integers, {}),
        (blk.test_block_zero_blocks_give_identity_structure, {}),
        (blk.test_block_general_params_within_rounding, {}),
    ]
    failed = []
    for fn, kw in checks:
        try:
            fn(orc, **kw)
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(f"{fn.__name__}{kw or ''}")
    return failed


def test_unmodified_oracle_passes_the_battery():
    assert _battery(oracle.default()) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mutant = oracle.variant(src.replace(old, new), str(tmp_path))
    failed = _battery(mutant)
    assert failed, f"no pin caught: {name}"
