"""Ratio-2 inter-level transfer (Sec. 2.1 and the ``interpolation_type``
entry of Tab. "amr").

Prolongation (coarse -> fine).  The paper names the types (0 piecewise
constant, 1 linear conservative, 2 quadratic polynomial, 4 quartic polynomial
conservative, the default) and calls the ghost interpolation fourth order; it
prints no weights.  Readings used here, per axis, tensor product over x, y, z:

* type 4: the fine value is the average over the fine cell of the unique
  degree-4 polynomial whose averages over the five coarse cells I-2..I+2
  equal the coarse values.
* type 2: the fine value is the degree-2 polynomial through the three coarse
  cell-centre values I-1..I+1, evaluated at the fine cell centre (+-1/4).
* type 0: the parent value.
* type 1 (linear conservative): the parent value plus, per axis, a quarter of
  a limited slope signed by the child's side, f = c + (s_x sx + s_y sy +
  s_z sz) / 4 with s = +-1.  The slope along an axis is the monotonized
  central one (van Leer) from the one-sided differences dm = c - c(-1),
  dp = c(+1) - c: zero where dm dp <= 0 (an extremum), else
  sign(dp) min(2|dm|, 2|dp|, |dm + dp| / 2).  Per-axis limiting alone lets a
  corner child leave the range of its neighbours (three axis terms add up),
  so the three slopes are then scaled by one factor alpha = min(1,
  (M - c) / E, (c - m) / E), E = (|sx| + |sy| + |sz|) / 4 the largest excursion
  of a child, M and m the largest and smallest of the parent and its six face
  neighbours.  Conservative (the 8 children average to the parent), exact
  for linear fields (alpha = 1 there), and no child leaves [m, M].  This is
  not a fixed-weight stencil, so it has its own evaluation below.

The 1D weights are derived below from those definitions with exact rational
arithmetic (no table is typed in).  Coarse cell I spans [I-1/2, I+1/2] in
coarse units; its children 2I and 2I+1 span [I-1/2, I] and [I, I+1/2].

Time interpolation (Sec. 2.1): the coarse value at fraction alpha of the
coarse step is (1 - alpha) * old + alpha * new, applied to each coarse value
before the spatial weights.

Restriction (Sec. 2.1, level synchronisation): a coarse cell covered by the
fine level becomes the mean of its 8 children, summed in the order
x fastest, then y, then z, and multiplied by 1/8.

Parity: pinned (exact fine averages of polynomials of per-axis degree <= 4,
restriction(prolongation) = identity, constants and linear functions; for
type 1 also the limiter's cases worked by hand, bounds on random data and a
monotone step) -- tests/test_oracle_interp.py.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np


def _solve(A, b):
    """Exact Gauss-Jordan on Fractions."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [x / pv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def _mean_monomial(p, lo, hi):
    """Average of x^p over [lo, hi]."""
    return (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo))


def weights_1d(interp_type: int):
    """{child: (offsets, weights)} with child 0 = lower half, 1 = upper half."""
    if interp_type == 0:
        return {0: ((0,), (Fr(1),)), 1: ((0,), (Fr(1),))}
    if interp_type == 4:
        offs = (-2, -1, 0, 1, 2)
        half = Fr(1, 2)
        A = [[_mean_monomial(p, Fr(j) - half, Fr(j) + half) for p in range(5)]
             for j in offs]
        out = {}
        for child, (lo, hi) in ((0, (-half, Fr(0))), (1, (Fr(0), half))):
            m = [_mean_monomial(p, lo, hi) for p in range(5)]
            # weight_j = m^T A^{-1} e_j  <=>  solve A^T w = m
            At = [[A[r][c] for r in range(5)] for c in range(5)]
            out[child] = (offs, tuple(_solve(At, m)))
        return out
    if interp_type == 2:
        offs = (-1, 0, 1)
        A = [[Fr(j) ** p for p in range(3)] for j in offs]
        out = {}
        for child, x in ((0, Fr(-1, 4)), (1, Fr(1, 4))):
            m = [x ** p for p in range(3)]
            At = [[A[r][c] for r in range(3)] for c in range(3)]
            out[child] = (offs, tuple(_solve(At, m)))
        return out
    raise ValueError("interpolation type must be 0, 2 or 4 (type 1 has no fixed weights)")


def mc_slope(dm, dp):
    """Monotonized-central slope from the one-sided differences dm = c - c(-1)
    and dp = c(+1) - c (type 1)."""
    dm, dp = np.asarray(dm, dtype=np.float64), np.asarray(dp, dtype=np.float64)
    mag = np.minimum(np.minimum(2.0 * np.abs(dm), 2.0 * np.abs(dp)), 0.5 * np.abs(dm + dp))
    return np.where(dm * dp > 0.0, np.where(dp > 0.0, mag, -mag), 0.0)


def _prolong_linear_limited(coarse_at, fine_idx):
    """Type 1 at fine cells: parent value and its six face neighbours
    gathered in one call, the three limited slopes and their common scale,
    then the children's sum ((c + s_x sx / 4) + s_y sy / 4) + s_z sz / 4."""
    fz, fy, fx = (np.asarray(a, dtype=np.int64).ravel() for a in fine_idx)
    shape = np.shape(fine_idx[0])
    P = (fz // 2, fy // 2, fx // 2)
    sgn = [2.0 * (f - 2 * q) - 1.0 for f, q in zip((fz, fy, fx), P)]    # -1 lower child, +1 upper
    # offsets (z, y, x): centre, then -x, +x, -y, +y, -z, +z
    oz = np.array([0, 0, 0, 0, 0, -1, 1])
    oy = np.array([0, 0, 0, -1, 1, 0, 0])
    ox = np.array([0, -1, 1, 0, 0, 0, 0])
    V = coarse_at(P[0][:, None] + oz[None, :], P[1][:, None] + oy[None, :], P[2][:, None] + ox[None, :])
    c = V[..., 0]
    sx = mc_slope(c - V[..., 1], V[..., 2] - c)
    sy = mc_slope(c - V[..., 3], V[..., 4] - c)
    sz = mc_slope(c - V[..., 5], V[..., 6] - c)
    e = 0.25 * ((np.abs(sx) + np.abs(sy)) + np.abs(sz))
    hi, lo = np.max(V, axis=-1), np.min(V, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        alpha = np.where(e > 0.0, np.minimum(1.0, np.minimum((hi - c) / e, (c - lo) / e)), 1.0)
    sx, sy, sz = alpha * sx, alpha * sy, alpha * sz
    out = ((c + 0.25 * (sgn[2] * sx)) + 0.25 * (sgn[1] * sy)) + 0.25 * (sgn[0] * sz)
    return out.reshape(V.shape[:-2] + shape)


def prolong_points(coarse_at, fine_idx, interp_type: int):
    """Prolonged values at fine cells.

    coarse_at(kz, ky, kx) -> array of coarse values at integer coarse indices
    (the caller resolves periodicity, boxes and time interpolation).
    fine_idx = (fz, fy, fx) integer arrays of fine indices.
    All stencil values are gathered in one call; the weighted sum then runs
    over offsets z (outer), y, x (inner) in increasing order.
    """
    if interp_type == 1:
        return _prolong_linear_limited(coarse_at, fine_idx)
    fz, fy, fx = (np.asarray(a, dtype=np.int64).ravel() for a in fine_idx)
    shape = np.shape(fine_idx[0])
    W = weights_1d(interp_type)
    Pz, Py, Px = fz // 2, fy // 2, fx // 2
    rz, ry, rx = fz - 2 * Pz, fy - 2 * Py, fx - 2 * Px
    offs = W[0][0]
    no = len(offs)
    wz = [np.where(rz == 0, float(W[0][1][a]), float(W[1][1][a])) for a in range(no)]
    wy = [np.where(ry == 0, float(W[0][1][a]), float(W[1][1][a])) for a in range(no)]
    wx = [np.where(rx == 0, float(W[0][1][a]), float(W[1][1][a])) for a in range(no)]
    oz, oy, ox = np.meshgrid(offs, offs, offs, indexing="ij")
    oz, oy, ox = oz.ravel(), oy.ravel(), ox.ravel()
    V = coarse_at(Pz[:, None] + oz[None, :], Py[:, None] + oy[None, :], Px[:, None] + ox[None, :])
    # V may carry leading axes (several components): (..., n, no^3)
    acc = np.zeros(V.shape[:-1])
    j = 0
    for a in range(no):
        for b in range(no):
            for c in range(no):
                acc = acc + (wz[a] * wy[b] * wx[c]) * V[..., j]
                j += 1
    return acc.reshape(V.shape[:-2] + shape)


def restrict_block(fine):
    """Restrict a fine [z, y, x] array (even extents) to the coarse grid."""
    f = np.asarray(fine, dtype=np.float64)
    s = (f[0::2, 0::2, 0::2] + f[0::2, 0::2, 1::2] + f[0::2, 1::2, 0::2]
         + f[0::2, 1::2, 1::2] + f[1::2, 0::2, 0::2] + f[1::2, 0::2, 1::2]
         + f[1::2, 1::2, 0::2] + f[1::2, 1::2, 1::2])
    return s * 0.125


def time_lerp(old, new, alpha: float):
    return (1.0 - alpha) * old + alpha * new
