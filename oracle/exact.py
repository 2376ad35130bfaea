"""Exact-rational evaluation of the two loop bodies (TEST INFRASTRUCTURE ONLY).

Every IEEE double is a dyadic rational, and the definitions use only +, -, *, / by
nonzero values, so each output has an exact rational value. `fractions.Fraction` computes
it; the FP64 oracle and both GPU forms are different roundings of this number. It is the
arbiter when two floating-point results disagree, and together with a rounding-error
bound it pins the FP64 oracle on tiny grids.

Definitions (identical in meaning to `acs_oracle.c`):
  RHS  R_c(p) = -sum_d (F_{d,c}(p+e_d) - F_{d,c}(p-e_d)) / (2 h_d)
                - eps * sum_d (U_c(p-2e_d) - 4U_c(p-e_d) + 6U_c(p) - 4U_c(p+e_d) + U_c(p+2e_d))
       with the Euler fluxes F_d of an ideal gas (ratio gamma) at each neighbour.
  Star out(p) = sum_d sum_{o=1..4} c_{d,o} a(p) (u(p+o e_d) - 2u(p) + u(p-o e_d)).

The `saturated_*` functions regroup the same sums the way the saturated form does
(per-point reciprocal, shared off-diagonal products, reassociated dissipation, folded
centre weight). Over the rationals they must equal the as-written value exactly: the
rewrite rules of Table I (FMA, commutativity, associativity, constant folding) preserve
value in exact arithmetic.
"""
from __future__ import annotations

from fractions import Fraction as Q

AXES = ((1, 0, 0), (0, 1, 0), (0, 0, 1))   # e_x, e_y, e_z as (di, dj, dk)


def _at(U, c, i, j, k):
    """Exact value of component c at extended index (i, j, k); U is (5, Z, Y, X) or (Z, Y, X)."""
    v = U[c, k, j, i] if c is not None else U[k, j, i]
    return Q(float(v))


def euler_flux(U, i, j, k, d, gamma):
    """Exact flux vector F_d (5 Fractions) at extended index (i, j, k)."""
    rho = _at(U, 0, i, j, k)
    m = [_at(U, 1, i, j, k), _at(U, 2, i, j, k), _at(U, 3, i, j, k)]
    E = _at(U, 4, i, j, k)
    g = Q(float(gamma))
    v_d = m[d] / rho
    KE = Q(1, 2) * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho
    P = (g - 1) * (E - KE)
    F = [m[d], m[0] * v_d, m[1] * v_d, m[2] * v_d, (E + P) * v_d]
    F[1 + d] += P
    return F


def rhs_point(U, i, j, k, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2):
    """Exact R_c (c = 0..4) at interior point (i, j, k). Also returns the per-component
    condition scale sum |terms| (every addend of the as-written sums, in absolute value)."""
    I, J, K = i + halo, j + halo, k + halo
    e = Q(float(eps))
    out, scale = [], []
    fp = [euler_flux(U, I + a[0], J + a[1], K + a[2], d, gamma) for d, a in enumerate(AXES)]
    fm = [euler_flux(U, I - a[0], J - a[1], K - a[2], d, gamma) for d, a in enumerate(AXES)]
    for c in range(5):
        flux = Q(0)
        diss = Q(0)
        s = Q(0)
        for d, a in enumerate(AXES):
            tw = Q(2) * Q(float(h[d]))
            flux += (fp[d][c] - fm[d][c]) / tw
            s += (abs(fp[d][c]) + abs(fm[d][c])) / tw
            w = [1, -4, 6, -4, 1]
            for o, wo in zip(range(-2, 3), w):
                val = _at(U, c, I + o * a[0], J + o * a[1], K + o * a[2])
                diss += wo * val
                s += abs(e * wo * val)
        out.append(-flux - e * diss)
        scale.append(s)
    return out, scale


def stencil_point(u, a, c, i, j, k, halo=4):
    """Exact out(p) at interior point (i, j, k) and its condition scale sum |terms|."""
    I, J, K = i + halo, j + halo, k + halo
    ap = _at(a, None, I, J, K)
    u0 = _at(u, None, I, J, K)
    acc = Q(0)
    s = Q(0)
    for d, ax in enumerate(AXES):
        for o in range(1, 5):
            cf = Q(float(c[d][o - 1]))
            up = _at(u, None, I + o * ax[0], J + o * ax[1], K + o * ax[2])
            um = _at(u, None, I - o * ax[0], J - o * ax[1], K - o * ax[2])
            acc += cf * ap * (up - 2 * u0 + um)
            s += abs(cf * ap) * (abs(up) + 2 * abs(u0) + abs(um))
    return acc, s


# ---------------------------------------------------------------------------------------
# The saturated regrouping, over the rationals.

def saturated_flux_point(U, i, j, k, gamma):
    """Per-point flux set computed once (one reciprocal, shared off-diagonal products).

    Returns {(d, c): value} for the 15 flux values at extended index (i, j, k).
    """
    rho = _at(U, 0, i, j, k)
    mx, my, mz = (_at(U, c, i, j, k) for c in (1, 2, 3))
    E = _at(U, 4, i, j, k)
    g1 = Q(float(gamma)) - 1
    r = 1 / rho
    vx, vy, vz = mx * r, my * r, mz * r
    mxvx = mx * vx
    twoKE = mz * vz + (my * vy + mxvx)
    P = g1 * E + (-g1 / 2) * twoKE
    EP = E + P
    mxvy, mxvz, myvz = mx * vy, mx * vz, my * vz     # = my*vx, mz*vx, mz*vy
    return {
        (0, 0): mx, (0, 1): mxvx + P, (0, 2): mxvy, (0, 3): mxvz, (0, 4): EP * vx,
        (1, 0): my, (1, 1): mxvy, (1, 2): my * vy + P, (1, 3): myvz, (1, 4): EP * vy,
        (2, 0): mz, (2, 1): mxvz, (2, 2): myvz, (2, 3): mz * vz + P, (2, 4): EP * vz,
    }


def scaled_flux_point(U, i, j, k, gamma, s):
    """The flux set with the common scale s = -1/(2h) of equal spacing folded in where it is
    formed: r' = s / rho, v' = m r' (= s v), the pressure from sum m v' with the folded
    constant -(gamma-1) / (2 s), the diagonal fluxes m_d v'_d + s P and the energy fluxes
    (E + P) v'_d. Components 1..4 come out as s F; component 0 (m_d) is not scaled.
    """
    rho = _at(U, 0, i, j, k)
    mx, my, mz = (_at(U, c, i, j, k) for c in (1, 2, 3))
    E = _at(U, 4, i, j, k)
    g1 = Q(float(gamma)) - 1
    r = (1 / rho) * s
    vx, vy, vz = mx * r, my * r, mz * r
    mxvx = mx * vx
    twoKE = mz * vz + (my * vy + mxvx)
    P = g1 * E + ((-g1 / 2) / s) * twoKE
    Pd = P * s
    EP = E + P
    mxvy, mxvz, myvz = mx * vy, mx * vz, my * vz
    return {
        (0, 0): mx, (0, 1): mxvx + Pd, (0, 2): mxvy, (0, 3): mxvz, (0, 4): EP * vx,
        (1, 0): my, (1, 1): mxvy, (1, 2): my * vy + Pd, (1, 3): myvz, (1, 4): EP * vy,
        (2, 0): mz, (2, 1): mxvz, (2, 2): myvz, (2, 3): mz * vz + Pd, (2, 4): EP * vz,
    }


def saturated_rhs_point(U, i, j, k, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2, scaled=False):
    """R_c via the saturated grouping: flux sum scaled once, dissipation as
    S2 - 4 S1 + 18 U(p) summed over all three axes, combined last. With `scaled` (equal
    spacing only) the fluxes of components 1..4 carry s = -1/(2h) from `scaled_flux_point`
    and their three differences are summed unscaled."""
    I, J, K = i + halo, j + halo, k + halo
    e = Q(float(eps))
    out = []
    fl = {}
    if scaled:
        assert h[0] == h[1] == h[2], "the scaled grouping needs equal spacing"
        s = -1 / (2 * Q(float(h[0])))
        point_flux = lambda a, b, c_: scaled_flux_point(U, a, b, c_, gamma, s)  # noqa: E731
    else:
        point_flux = lambda a, b, c_: saturated_flux_point(U, a, b, c_, gamma)  # noqa: E731
    for d, ax in enumerate(AXES):
        fl[(d, +1)] = point_flux(I + ax[0], J + ax[1], K + ax[2])
        fl[(d, -1)] = point_flux(I - ax[0], J - ax[1], K - ax[2])
    for c in range(5):
        fsum = Q(0)
        for d in range(3):
            diff = fl[(d, +1)][(d, c)] - fl[(d, -1)][(d, c)]
            fsum += diff if (scaled and c > 0) else diff * (-1 / (2 * Q(float(h[d]))))
        s1 = Q(0)
        s2 = Q(0)
        for ax in AXES:
            s1 += _at(U, c, I + ax[0], J + ax[1], K + ax[2]) + _at(U, c, I - ax[0], J - ax[1], K - ax[2])
            s2 += _at(U, c, I + 2 * ax[0], J + 2 * ax[1], K + 2 * ax[2]) + \
                _at(U, c, I - 2 * ax[0], J - 2 * ax[1], K - 2 * ax[2])
        diss = s2 + (-4) * s1 + 18 * _at(U, c, I, J, K)
        out.append(fsum + (-e) * diss)
    return out


def saturated_stencil_point(u, a, c, i, j, k, halo=4):
    """out = a(p) * (C0 u(p) + sum_d sum_o c_{d,o} (u(p+o e_d) + u(p-o e_d))), C0 = -2 sum c."""
    I, J, K = i + halo, j + halo, k + halo
    cq = [[Q(float(c[d][o])) for o in range(4)] for d in range(3)]
    C0 = -2 * sum(sum(row) for row in cq)
    acc = C0 * _at(u, None, I, J, K)
    for d, ax in enumerate(AXES):
        for o in range(1, 5):
            acc += cq[d][o - 1] * (_at(u, None, I + o * ax[0], J + o * ax[1], K + o * ax[2]) +
                                   _at(u, None, I - o * ax[0], J - o * ax[1], K - o * ax[2]))
    return _at(a, None, I, J, K) * acc
