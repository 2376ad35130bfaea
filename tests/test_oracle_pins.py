"""Pins for the CPU oracle: each test fixes a value by something other than the oracle's
own formula (closed forms, invariants, symmetries, a library routine, exact rationals),
chosen so that a dropped term, a wrong sign or index, or a swapped axis fails one of them.
"""
from fractions import Fraction as Q

import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import exact
from paper_2306_13002_gb300 import inputs

U53 = 2.0 ** -53


@pytest.fixture
def orc():
    return oracle.default()

G = 1.4
G1 = Q(G) - 1          # fl(1.4) - 1 is exact (Sterbenz), as in the oracle


def _ext_coords(shape_zyx):
    Z, Y, X = shape_zyx
    k, j, i = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)


# ----------------------------------------------------------------------------- RHS pins

def test_constant_dyadic_field_gives_exact_zero(orc):
    """Every difference of a constant field is x - x; with short-mantissa constants the
    5-point dissipation is exact too, so R is bitwise zero."""
    n, h = 6, 2
    U = np.empty((5, n + 2 * h, n + 2 * h, n + 2 * h))
    for c, v in enumerate((1.25, 0.5, -0.25, 0.125, 2.5)):
        U[c] = v
    R = orc.rhs(U, h=(1.0, 0.5, 2.0))
    assert np.all(R == 0.0)


def test_constant_arbitrary_field_is_rounding_small(orc):
    n, h = 5, 2
    rng = np.random.default_rng(1)
    vals = [rng.uniform(0.5, 1.5), *rng.uniform(-0.5, 0.5, 3), rng.uniform(0.5, 1.5)]
    U = np.empty((5, n + 4, n + 4, n + 4))
    for c, v in enumerate(vals):
        U[c] = v
    R = orc.rhs(U)
    assert np.max(np.abs(R)) <= 16 * 0.25 * 1.5 * 4 * U53     # a few ulp of the dissipation terms


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0)])
def test_linear_energy_at_rest(orc, h):
    """m = 0, rho = 2, E linear with dyadic slopes: F_d = [0, P e_d, 0] with P = (gamma-1) E,
    so R = [0, -(gamma-1) g_x/h_x, -(gamma-1) g_y/h_y, -(gamma-1) g_z/h_z, 0]."""
    n, H = 6, 2
    i, j, k = _ext_coords((n + 2 * H,) * 3)
    gx, gy, gz = 0.5, -0.25, 0.125
    U = np.zeros((5, n + 4, n + 4, n + 4))
    U[0] = 2.0
    U[4] = 8.0 + gx * i + gy * j + gz * k
    R = orc.rhs(U, h=h)
    assert np.all(R[0] == 0.0) and np.all(R[4] == 0.0)
    for d, g in enumerate((gx, gy, gz)):
        expect = float(-G1 * Q(g) / Q(h[d]))
        np.testing.assert_allclose(R[1 + d], expect, rtol=0, atol=1e-14)


def _one_d_flow_expect(m, E, b, hd):
    """Closed form for rho = 1, m_d = a + b x (others 0), E constant (derivation:
    d(m^2) = 4bm, dP = -2(gamma-1)bm, d((E+P)m) = 2b(1+(gamma-1))E - (gamma-1)b(3m^2+b^2))."""
    g1 = G1
    r0 = -Q(b) / Q(hd)
    rmom = -Q(b) * m * (2 - g1) / Q(hd)
    re = -(2 * Q(b) * (1 + g1) * E - g1 * Q(b) * (3 * m * m + Q(b) * Q(b))) / (2 * Q(hd))
    return r0, rmom, re


@pytest.mark.parametrize("d", [0, 1, 2])
def test_one_dimensional_flow_closed_form(orc, d):
    n, H = 6, 2
    coords = _ext_coords((n + 2 * H,) * 3)          # (i, j, k)
    a, b, e0 = 0.25, 0.0625, 1.5
    h = (1.0, 0.5, 2.0)
    U = np.zeros((5, n + 4, n + 4, n + 4))
    U[0] = 1.0
    U[1 + d] = a + b * coords[d]
    U[4] = e0
    R = orc.rhs(U, h=h)
    for kk in range(n):
        for jj in range(n):
            for ii in range(n):
                x = (ii, jj, kk)[d] + H
                m = Q(a) + Q(b) * x
                r0, rmom, re = _one_d_flow_expect(m, Q(e0), b, h[d])
                assert R[0, kk, jj, ii] == pytest.approx(float(r0), abs=1e-14)
                assert R[1 + d, kk, jj, ii] == pytest.approx(float(rmom), rel=1e-13, abs=1e-15)
                assert R[4, kk, jj, ii] == pytest.approx(float(re), rel=1e-13, abs=1e-15)
                for other in range(3):
                    if other != d:
                        assert R[1 + other, kk, jj, ii] == 0.0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_quartic_fields_pin_dissipation(orc, d):
    """rho = 1 + s x^4 and E = e0 + s x^4 along axis d, m = 0. The 5-point fourth difference of
    x^4 is 24 exactly; with m = 0 only the pressure flux survives:
    R_0 = -24 eps s, R_{1+d} = -(gamma-1) s ((x+1)^4 - (x-1)^4) / (2h) = -4(gamma-1) s (x^3 + x) / h,
    R_4 = -24 eps s."""
    n, H = 5, 2
    coords = _ext_coords((n + 2 * H,) * 3)
    s, e0, eps = 1.0 / 64.0, 1.0, 0.25
    h = (1.0, 0.5, 2.0)
    U = np.zeros((5, n + 4, n + 4, n + 4))
    U[0] = 1.0 + s * coords[d] ** 4
    U[4] = e0 + s * coords[d] ** 4
    R = orc.rhs(U, eps=eps, h=h)
    np.testing.assert_array_equal(R[0], -24 * eps * s)
    np.testing.assert_array_equal(R[4], -24 * eps * s)
    x = coords[d][H:-H, H:-H, H:-H]
    expect = -4 * float(G1) * s * (x ** 3 + x) / h[d]
    np.testing.assert_allclose(R[1 + d], expect, rtol=1e-13, atol=1e-14)
    for other in range(3):
        if other != d:
            assert np.all(R[1 + other] == 0.0)


def test_reflection_symmetry(orc):
    """Mirroring x and negating m_x maps the RHS onto itself with R_1 negated."""
    U = inputs.rhs_field(7, 6, 5, halo=2, seed=77)
    Um = U[:, :, :, ::-1].copy()
    Um[1] = -Um[1]
    R = orc.rhs(U)
    Rm = orc.rhs(Um)
    expect = R[:, :, :, ::-1].copy()
    expect[1] = -expect[1]
    np.testing.assert_allclose(Rm, expect, rtol=0, atol=1e-13)


def test_axis_permutation_symmetry(orc):
    """Swapping x and y (and m_x with m_y) permutes R the same way."""
    U = inputs.rhs_field(6, 6, 5, halo=2, seed=78)
    Ut = U.transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]].copy()
    R = orc.rhs(U)
    Rt = orc.rhs(Ut)
    expect = R.transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]]
    np.testing.assert_allclose(Rt, expect, rtol=0, atol=1e-13)


def test_translation_and_padding_and_slabs_are_bitwise_stable(orc):
    U = inputs.rhs_field(6, 5, 7, halo=2, seed=79)
    R = orc.rhs(U)
    # row pitch padding
    Up = inputs.pad_rows(U, U.shape[-1] + 3)
    np.testing.assert_array_equal(orc.rhs(Up), R)
    # slab evaluation
    Rs = orc.rhs(U, k_range=(2, 5))
    np.testing.assert_array_equal(Rs[:, 2:5], R[:, 2:5])
    assert np.all(np.isnan(Rs[:, :2]))
    # translation by one cell along z
    R2 = orc.rhs(U[:, 1:])
    np.testing.assert_array_equal(R2, R[:, 1:])


def test_brute_force_exact_rationals_4cubed(orc):
    """Config-1 distributions on a 4^3 interior: the FP64 oracle is within a small multiple of
    the unit roundoff (times the sum of |terms|) of the exact rational value."""
    U = inputs.rhs_field(4, halo=2, seed=inputs.SEED_RHS_SMALL)
    R = orc.rhs(U)
    worst = 0.0
    for k in range(4):
        for j in range(4):
            for i in range(4):
                ex, sc = exact.rhs_point(U, i, j, k)
                for c in range(5):
                    err = abs(Q(float(R[c, k, j, i])) - ex[c])
                    bound = 32 * Q(U53) * sc[c]
                    assert err <= bound, (c, i, j, k, float(err), float(bound))
                    worst = max(worst, float(err / sc[c]))
    assert worst < 32 * U53


def test_saturated_grouping_is_an_exact_identity(orc):
    """The saturated regrouping (one reciprocal, shared off-diagonal products, reassociated
    dissipation, folded 1/(2h)) equals the as-written definition exactly over the rationals."""
    U = inputs.rhs_field(3, halo=2, seed=80)
    for (i, j, k) in [(0, 0, 0), (1, 2, 0), (2, 1, 2)]:
        a, _ = exact.rhs_point(U, i, j, k, h=(1.0, 0.5, 2.0))
        b = exact.saturated_rhs_point(U, i, j, k, h=(1.0, 0.5, 2.0))
        assert a == b


@pytest.mark.parametrize("h", [1.0, 0.37, 3.0])
def test_scaled_flux_grouping_is_an_exact_identity(orc, h):
    """Equal spacing: -1/(2h) folded into the fluxes where they are formed (scaled reciprocal,
    pressure through the folded constant, scaled diagonal pressure) equals the as-written
    definition exactly over the rationals."""
    U = inputs.rhs_field(3, halo=2, seed=81)
    for (i, j, k) in [(0, 0, 0), (1, 2, 0), (2, 1, 2)]:
        a, _ = exact.rhs_point(U, i, j, k, h=(h, h, h))
        b = exact.saturated_rhs_point(U, i, j, k, h=(h, h, h), scaled=True)
        assert a == b


# ----------------------------------------------------------------------------- stencil pins

def test_stencil_constant_is_exact_zero(orc):
    u = np.full((13, 12, 14), 0.7384615)
    a = inputs.stencil_fields(6, 4, 5, seed=5)[1]
    out = orc.stencil(u, a)
    assert np.all(out == 0.0)


def test_taylor_weights_centre_and_moments(orc):
    """The 8th-order weights: 2 sum c_o = 205/72 (centre), sum c_o 2 o^2 / 2! = 1 (second
    derivative), and the 4th, 6th, 8th moments vanish."""
    c = [Q(8, 5), Q(-1, 5), Q(8, 315), Q(-1, 560)]
    assert 2 * sum(c) == Q(205, 72)
    assert sum(co * 2 * o ** 2 for o, co in zip(range(1, 5), c)) == 2
    for m in (4, 6, 8):
        assert sum(co * 2 * o ** m for o, co in zip(range(1, 5), c)) == 0
    assert sum(co * 2 * o ** 10 for o, co in zip(range(1, 5), c)) != 0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_stencil_polynomials_exact_to_degree_9(orc, d):
    """u = x^k along axis d: out = a w_d k (k-1) x^(k-2) for k <= 9, with per-axis scalings
    w = (1, 2, 1/2) of the Taylor weights; degree 10 is visibly not reproduced."""
    n, H = 4, 4
    shape = (n + 2 * H, n + 2 * H + 1, n + 2 * H + 2)
    coords = _ext_coords(shape)
    a = inputs.stencil_fields(n + 2, n + 1, n, seed=6)[1]
    c = oracle.taylor_coeffs() * np.array([[1.0], [2.0], [0.5]])
    w = (1.0, 2.0, 0.5)
    for kdeg in range(0, 11):
        x = coords[d] - (shape[::-1][d] // 2)         # centred coordinate, small magnitudes
        u = x ** kdeg
        out = orc.stencil(u, a, c)
        xi = x[H:-H, H:-H, H:-H]
        ai = a[H:-H, H:-H, H:-H]
        expect = ai * w[d] * kdeg * (kdeg - 1) * xi ** max(kdeg - 2, 0) if kdeg >= 2 else np.zeros_like(ai)
        scale = ai * w[d] * 6.0 * (np.abs(xi) + 4.0) ** kdeg + 1.0
        err = np.abs(out - expect)
        if kdeg <= 9:
            assert np.all(err <= 64 * U53 * scale), (kdeg, err.max())
        else:
            assert np.max(err) > 1.0


@pytest.mark.parametrize("d,o", [(0, 1), (1, 3), (2, 4)])
def test_stencil_single_term_matches_library_correlation(orc, d, o):
    """c = unit weight on one (axis, offset): out = a (u(p+o) - 2u(p) + u(p-o)), the textbook
    second difference, computed here by scipy.ndimage.correlate1d."""
    n, H = 5, 4
    u, a = inputs.stencil_fields(n, n + 1, n + 2, seed=7)
    c = np.zeros((3, 4))
    c[d, o - 1] = 1.0
    out = orc.stencil(u, a, c)
    wts = np.zeros(2 * o + 1)
    wts[0], wts[o], wts[-1] = 1.0, -2.0, 1.0
    axis = 2 - d
    lib = ndimage.correlate1d(u, wts, axis=axis, mode="constant")[H:-H, H:-H, H:-H] * a[H:-H, H:-H, H:-H]
    np.testing.assert_allclose(out, lib, rtol=1e-14, atol=1e-15)


def test_stencil_full_weights_match_library_correlation(orc):
    n, H = 6, 4
    u, a = inputs.stencil_fields(n, n, n, seed=8)
    out = orc.stencil(u, a)
    c = oracle.TAYLOR8
    wts = np.array([c[3], c[2], c[1], c[0], -2 * sum(c), c[0], c[1], c[2], c[3]])
    lib = sum(ndimage.correlate1d(u, wts, axis=ax, mode="constant") for ax in (0, 1, 2))
    lib = lib[H:-H, H:-H, H:-H] * a[H:-H, H:-H, H:-H]
    np.testing.assert_allclose(out, lib, rtol=1e-13, atol=1e-14)


def test_stencil_brute_force_exact_rationals(orc):
    u, a = inputs.stencil_fields(4, seed=inputs.SEED_STENCIL)
    c = oracle.taylor_coeffs()
    out = orc.stencil(u, a, c)
    for k in range(4):
        for j in range(4):
            for i in range(4):
                ex, sc = exact.stencil_point(u, a, c, i, j, k)
                assert abs(Q(float(out[k, j, i])) - ex) <= 32 * Q(U53) * sc
                assert exact.saturated_stencil_point(u, a, c, i, j, k) == ex


def test_stencil_padding_and_slabs_bitwise(orc):
    u, a = inputs.stencil_fields(5, 6, 7, seed=9)
    out = orc.stencil(u, a)
    up, ap = inputs.pad_rows(u, u.shape[-1] + 5), inputs.pad_rows(a, a.shape[-1] + 5)
    np.testing.assert_array_equal(orc.stencil(up, ap), out)
    np.testing.assert_array_equal(orc.stencil(u, a, k_range=(1, 4))[1:4], out[1:4])


def test_openmp_threads_do_not_change_bits(orc):
    U = inputs.rhs_field(8, halo=2, seed=81)
    np.testing.assert_array_equal(orc.rhs(U, threads=1), orc.rhs(U, threads=4))


@pytest.mark.parametrize("rho_exp", [-1010, 1010])
def test_oracle_extreme_density_within_condition_bound_of_exact(rho_exp):
    """rho scaled by 2^+-1010 (momenta by 2^+-505): at every point the FP64 oracle is within
    1e-12 |exact| + 2^-46 sum|terms| of the exact rational value, the per-point bound the GPU
    test of these fields uses."""
    from oracle import exact
    U = inputs.rhs_field(5, 4, 3, halo=2, seed=3200)
    U[0] *= 2.0 ** rho_exp
    U[1:4] *= 2.0 ** (rho_exp // 2)
    ref = oracle.rhs(U)
    for k in range(3):
        for j in range(4):
            for i in range(5):
                ex, sc = exact.rhs_point(U, i, j, k, gamma=1.4, eps=0.25, halo=2)
                for c in range(5):
                    e = float(ex[c])
                    assert abs(ref[c, k, j, i] - e) <= 1e-12 * abs(e) + 2.0 ** -46 * float(sc[c])
