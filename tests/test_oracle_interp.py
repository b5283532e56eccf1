"""Pins of the oracle's prolongation and restriction (Sec. 2.1, Tab. "amr"
interpolation types 0, 1, 2 and 4) against exact polynomial cell averages,
and of the limited type 1 against its worked cases, bounds and monotonicity."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import interp


def _avg_poly(coef, lo, hi):
    """Exact average of sum_p coef[p] x^p over [lo, hi]."""
    return sum(c * (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo)) for p, c in enumerate(coef))


def _eval_poly(coef, x):
    return sum(c * x ** p for p, c in enumerate(coef))


def test_quartic_weights_reproduce_exact_averages_1d():
    W = interp.weights_1d(4)
    rng = np.random.default_rng(0)
    half = Fr(1, 2)
    for _ in range(20):
        coef = [Fr(int(v), 7) for v in rng.integers(-20, 20, size=5)]
        I = int(rng.integers(-5, 5))
        cavg = {j: _avg_poly(coef, Fr(I + j) - half, Fr(I + j) + half) for j in range(-2, 3)}
        for child, (lo, hi) in ((0, (Fr(I) - half, Fr(I))), (1, (Fr(I), Fr(I) + half))):
            offs, w = W[child]
            got = sum(wj * cavg[o] for o, wj in zip(offs, w))
            assert got == _avg_poly(coef, lo, hi)
    # the weights are not exact on degree 5 (the reading is quartic)
    coef = [0, 0, 0, 0, 0, Fr(1)]
    offs, w = W[1]
    got = sum(wj * _avg_poly(coef, Fr(o) - half, Fr(o) + half) for o, wj in zip(offs, w))
    assert got != _avg_poly(coef, Fr(0), half)


def test_quartic_weights_conservative_and_mirrored():
    W = interp.weights_1d(4)
    (o0, w0), (o1, w1) = W[0], W[1]
    assert sum(w0) == 1 and sum(w1) == 1
    assert tuple(reversed(w0)) == w1
    # the two children average back to the parent: (w0 + w1) / 2 = delta_0
    assert [(a + b) / 2 for a, b in zip(w0, w1)] == [0, 0, 1, 0, 0]


def test_quadratic_weights_pointwise_exact():
    W = interp.weights_1d(2)
    rng = np.random.default_rng(1)
    for _ in range(10):
        coef = [Fr(int(v), 3) for v in rng.integers(-9, 9, size=3)]
        I = int(rng.integers(-4, 4))
        for child, x in ((0, Fr(I) - Fr(1, 4)), (1, Fr(I) + Fr(1, 4))):
            offs, w = W[child]
            assert sum(wj * _eval_poly(coef, Fr(I + o)) for o, wj in zip(offs, w)) == _eval_poly(coef, x)


def _poly3(rng, deg):
    return [[float(v) / 4 for v in rng.integers(-8, 8, size=deg + 1)] for _ in range(3)]


def test_prolong_points_exact_for_tensor_quartic_3d():
    rng = np.random.default_rng(2)
    px, py, pz = _poly3(rng, 4)
    qx, qy, qz = _poly3(rng, 2)

    def avg3(lo, hi):
        return (_avg_f(px, lo[0], hi[0]) * _avg_f(py, lo[1], hi[1]) * _avg_f(pz, lo[2], hi[2])
                + _avg_f(qx, lo[0], hi[0]) * _avg_f(qy, lo[1], hi[1]) * _avg_f(qz, lo[2], hi[2]))

    def coarse_at(Kz, Ky, Kx):
        out = np.empty(Kz.shape)
        for idx in np.ndindex(Kz.shape):
            k = (Kx[idx], Ky[idx], Kz[idx])
            out[idx] = avg3([k[d] - 0.5 for d in range(3)], [k[d] + 0.5 for d in range(3)])
        return out

    fz, fy, fx = np.meshgrid(np.arange(-3, 4), np.arange(-2, 3), np.arange(-4, 2), indexing="ij")
    got = interp.prolong_points(coarse_at, (fz, fy, fx), 4)
    for idx in np.ndindex(fz.shape):
        f = (fx[idx], fy[idx], fz[idx])
        # coarse cell K spans [K - 1/2, K + 1/2]; its children 2K, 2K+1 span
        # [K - 1/2, K] and [K, K + 1/2], i.e. fine cell f spans [f/2 - 1/2, f/2]
        lo = [f[d] / 2 - 0.5 for d in range(3)]
        hi = [f[d] / 2 for d in range(3)]
        exp = avg3(lo, hi)
        assert abs(got[idx] - exp) <= 1e-12 * max(1.0, abs(exp))


def _avg_f(coef, lo, hi):
    return sum(c * (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo)) for p, c in enumerate(coef))


@pytest.mark.parametrize("itype", [0, 1, 2, 4])
def test_restrict_of_prolong_is_identity_and_constants_exact(itype):
    nc = 6
    C = np.random.default_rng(itype).standard_normal((nc, nc, nc))

    def coarse_at(Kz, Ky, Kx):
        return C[Kz % nc, Ky % nc, Kx % nc]

    fz, fy, fx = np.meshgrid(*(np.arange(2 * nc),) * 3, indexing="ij")
    Fv = interp.prolong_points(coarse_at, (fz, fy, fx), itype)
    back = interp.restrict_block(Fv)
    if itype != 2:   # conservative types
        assert np.max(np.abs(back - C)) < 1e-14
    const = interp.prolong_points(lambda a, b, c: np.full(a.shape, 1.375), (fz, fy, fx), itype)
    assert np.all(const == 1.375)


def test_restriction_constants_and_linear():
    f = np.full((4, 6, 8), -2.5)
    assert np.all(interp.restrict_block(f) == -2.5)
    Z, Y, X = np.meshgrid(np.arange(4.0), np.arange(6.0), np.arange(8.0), indexing="ij")
    lin = 0.5 * X - 0.25 * Y + 2.0 * Z + 1.0
    R = interp.restrict_block(lin)
    Zc, Yc, Xc = np.meshgrid(np.arange(2.0), np.arange(3.0), np.arange(4.0), indexing="ij")
    exp = 0.5 * (2 * Xc + 0.5) - 0.25 * (2 * Yc + 0.5) + 2.0 * (2 * Zc + 0.5) + 1.0
    assert np.max(np.abs(R - exp)) < 1e-14


def test_time_lerp_endpoints_exact():
    a, b = np.array([0.1, -3.7]), np.array([2.9, 1e-9])
    assert np.array_equal(interp.time_lerp(a, b, 0.0), a)
    assert np.array_equal(interp.time_lerp(a, b, 1.0), b)


# -- type 1: linear conservative (limited slopes) ----------------------------

@pytest.mark.parametrize("dm,dp,s", [(1.0, 3.0, 2.0), (1.0, 0.2, 0.4), (3.0, 1.0, 2.0), (2.0, 2.0, 2.0),
                                     (-1.0, -3.0, -2.0), (1e-3, 1.0, 2e-3), (1.0, -1.0, 0.0), (0.0, 5.0, 0.0),
                                     (-2.0, 0.5, 0.0)])
def test_mc_slope_worked_cases(dm, dp, s):
    """min(2|dm|, 2|dp|, |dm + dp| / 2) with the sign of the differences,
    zero at an extremum or a flat side."""
    assert interp.mc_slope(dm, dp) == pytest.approx(s, rel=1e-15, abs=0.0)


def _neighbours_range(C, nc):
    stack = [C] + [np.roll(C, sh, axis=ax) for ax in range(3) for sh in (1, -1)]
    return np.max(stack, axis=0), np.min(stack, axis=0)


def test_linear_conservative_bounds_and_conservation_on_random_data():
    """Every child within [m, M] of its parent and the parent's face
    neighbours, and the 8 children average to the parent."""
    nc = 8
    C = np.random.default_rng(4).standard_normal((nc, nc, nc))

    def coarse_at(Kz, Ky, Kx):
        return C[Kz % nc, Ky % nc, Kx % nc]

    fz, fy, fx = np.meshgrid(*(np.arange(2 * nc),) * 3, indexing="ij")
    Fv = interp.prolong_points(coarse_at, (fz, fy, fx), 1)
    M, m = _neighbours_range(C, nc)
    up = lambda a: np.repeat(np.repeat(np.repeat(a, 2, 0), 2, 1), 2, 2)
    Mf, mf = up(M), up(m)
    assert np.all(Fv <= Mf + 1e-15) and np.all(Fv >= mf - 1e-15)
    assert np.max(np.abs(interp.restrict_block(Fv) - C)) < 1e-14
    # on this data the per-axis slopes alone overshoot, so the joint scale is exercised
    sgn = lambda f: 2.0 * (f % 2) - 1.0
    c = up(C)
    slope = lambda ax: up(interp.mc_slope(C - np.roll(C, 1, axis=ax), np.roll(C, -1, axis=ax) - C))
    raw = c + 0.25 * (sgn(fx) * slope(2) + sgn(fy) * slope(1) + sgn(fz) * slope(0))
    assert np.max(np.maximum(raw - Mf, mf - raw)) > 0.05


def test_linear_conservative_exact_for_linear_fields():
    """Coarse cell averages of a linear function (its values at cell
    centres) give children equal to the fine cell averages."""
    a = np.array([0.7, -1.3, 0.4])                         # (x, y, z)

    def coarse_at(Kz, Ky, Kx):
        return a[0] * Kx + a[1] * Ky + a[2] * Kz + 2.5      # no wrap: a linear field

    fz, fy, fx = np.meshgrid(*(np.arange(4, 12),) * 3, indexing="ij")
    Fv = interp.prolong_points(coarse_at, (fz, fy, fx), 1)
    # fine cell f spans [f/2 - 1/2, f/2] in coarse units, centre f/2 - 1/4
    exp = a[0] * (fx / 2 - 0.25) + a[1] * (fy / 2 - 0.25) + a[2] * (fz / 2 - 0.25) + 2.5
    assert np.max(np.abs(Fv - exp)) < 1e-13


def test_linear_conservative_joint_scale_worked_case():
    """Parent 0 with neighbours -1 / +3 along every axis: each slope is 2,
    the corner excursion E = 1.5 would reach -1.5 < m = -1, so alpha = 2/3:
    the lowest child is exactly m and the highest +1."""
    vals = {(0, 0, 0): 0.0}
    for d in range(3):
        e = [0, 0, 0]
        e[d] = -1
        vals[tuple(e)] = -1.0
        e[d] = 1
        vals[tuple(e)] = 3.0

    def coarse_at(Kz, Ky, Kx):
        out = np.empty(Kz.shape)
        for idx in np.ndindex(Kz.shape):
            out[idx] = vals[(int(Kz[idx]), int(Ky[idx]), int(Kx[idx]))]
        return out

    fz, fy, fx = np.meshgrid(*(np.arange(2),) * 3, indexing="ij")
    Fv = interp.prolong_points(coarse_at, (fz, fy, fx), 1)
    assert Fv[0, 0, 0] == pytest.approx(-1.0, abs=1e-15)
    assert Fv[1, 1, 1] == pytest.approx(1.0, abs=1e-15)
    assert np.mean(Fv) == pytest.approx(0.0, abs=1e-15)


def test_linear_conservative_step_is_monotone():
    """A coarse step along x: the children keep the step's values (slopes
    vanish at the cells on either side of the jump), no over- or undershoot."""
    nc = 8
    C = np.zeros((nc, nc, nc))
    C[:, :, nc // 2:] = 1.0

    def coarse_at(Kz, Ky, Kx):
        return C[Kz % nc, Ky % nc, Kx % nc]

    fz, fy, fx = np.meshgrid(*(np.arange(2 * nc),) * 3, indexing="ij")
    Fv = interp.prolong_points(coarse_at, (fz, fy, fx), 1)
    assert np.array_equal(Fv, np.repeat(np.repeat(np.repeat(C, 2, 0), 2, 1), 2, 2))
