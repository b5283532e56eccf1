"""Pins of the oracle's finite-difference operators (App. A) against what
mathematics fixes: Taylor moment conditions, the exact discrete dispersion
relation on lattice Fourier modes, and a dense-matrix brute force whose
weights are re-derived from the moment conditions."""
from fractions import Fraction as Fr
import itertools

import numpy as np
import pytest

from oracle import stencil


def _derive_weights(h, deriv):
    """Weights on offsets -h..h exact on x^q for q <= 2h (solve Vandermonde)."""
    n = 2 * h + 1
    offs = list(range(-h, h + 1))
    A = [[Fr(m) ** q for m in offs] for q in range(n)]
    rhs = [Fr(0)] * n
    rhs[deriv] = Fr(1) * (1 if deriv == 0 else (2 if deriv == 2 else 1))
    # Gauss-Jordan
    M = [row[:] + [rhs[i]] for i, row in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        pv = M[c][c]
        M[c] = [x / pv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return tuple(M[i][n] for i in range(n))


@pytest.mark.parametrize("order", [2, 4, 6])
def test_laplacian_weights_moment_conditions(order):
    h = order // 2
    w = stencil.LAPLACIAN_WEIGHTS[order]
    assert len(w) == 2 * h + 1
    for q in range(0, order + 2):
        s = sum(w[m + h] * Fr(m) ** q for m in range(-h, h + 1))
        assert s == (2 if q == 2 else 0), (order, q, s)
    # accuracy is exactly `order`: the next even moment does not vanish
    q = order + 2
    assert sum(w[m + h] * Fr(m) ** q for m in range(-h, h + 1)) != 0


@pytest.mark.parametrize("order", [2, 4, 6])
def test_gradient_weights_moment_conditions(order):
    h = order // 2
    w = stencil.GRADIENT_WEIGHTS[order]
    for q in range(0, order + 1):
        s = sum(w[m + h] * Fr(m) ** q for m in range(-h, h + 1))
        assert s == (1 if q == 1 else 0), (order, q)


def _symbol(order, theta):
    """Closed-form -(1D symbol) * dx^2 of the order-p Laplacian on e^{i theta j}."""
    if order == 2:
        return 4.0 * np.sin(theta / 2) ** 2
    if order == 4:
        return 2.5 - (8.0 / 3.0) * np.cos(theta) + (1.0 / 6.0) * np.cos(2 * theta)
    if order == 6:
        return (49.0 / 18.0 - 3.0 * np.cos(theta) + 0.3 * np.cos(2 * theta)
                - (1.0 / 45.0) * np.cos(3 * theta))
    raise ValueError


@pytest.mark.parametrize("order", [2, 4, 6])
def test_laplacian_dispersion_exact(order):
    n, dx = 16, 0.37
    rng = np.random.default_rng(order)
    ax = np.arange(n)
    kz, ky, kx = np.meshgrid(ax, ax, ax, indexing="ij")
    for _ in range(4):
        m = rng.integers(-n // 2, n // 2, size=3)
        th = 2 * np.pi * m / n
        phase = th[0] * kx + th[1] * ky + th[2] * kz
        lam = sum(_symbol(order, t) for t in th) / dx ** 2
        for f in (np.cos(phase), np.sin(phase)):
            L = stencil.laplacian_periodic(f, dx, order)
            err = np.max(np.abs(L + lam * f))
            assert err <= 1e-12 * max(lam, 1.0), (order, m, err)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_gradient_dispersion_exact(order):
    n, dx = 16, 0.5
    ax = np.arange(n)
    kz, ky, kx = np.meshgrid(ax, ax, ax, indexing="ij")
    m = np.array([3, -2, 5])
    th = 2 * np.pi * m / n
    phase = th[0] * kx + th[1] * ky + th[2] * kz
    h = order // 2
    w = [float(x) for x in stencil.GRADIENT_WEIGHTS[order]]
    for d, name in enumerate("xyz"):
        # symbol of sum_m w_m e^{i m theta} is i * sum_m w_m sin(m theta)
        s = sum(w[j + h] * np.sin(j * th[d]) for j in range(-h, h + 1)) / dx
        G = stencil.gradient_periodic(np.sin(phase), dx, order, name)
        assert np.max(np.abs(G - s * np.cos(phase))) < 1e-12


@pytest.mark.parametrize("order", [2, 4, 6])
def test_laplacian_dense_matrix_bruteforce_8cube(order):
    n, dx = 8, 0.25
    h = order // 2
    w = _derive_weights(h, 2)
    # 1D circulant with independently derived weights, then Kronecker sum
    C = np.zeros((n, n))
    for i in range(n):
        for m in range(-h, h + 1):
            C[i, (i + m) % n] += float(w[m + h])
    I = np.eye(n)
    Lx = np.kron(np.kron(I, I), C)
    Ly = np.kron(np.kron(I, C), I)
    Lz = np.kron(np.kron(C, I), I)
    Lmat = (Lx + Ly + Lz) / dx ** 2
    f = np.random.default_rng(1).standard_normal((n, n, n))
    ref = (Lmat @ f.ravel()).reshape(n, n, n)
    got = stencil.laplacian_periodic(f, dx, order)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("order", [2, 4, 6])
def test_padded_matches_periodic(order):
    n, g = 10, 3
    f = np.random.default_rng(2).standard_normal((n, n + 2, n + 4))
    fp = np.pad(f, g, mode="wrap")
    a = stencil.laplacian_periodic(f, 0.3, order)
    b = stencil.laplacian_padded(fp, g, 0.3, order)
    assert np.array_equal(a, b)
    for d in "xyz":
        assert np.array_equal(stencil.gradient_periodic(f, 0.3, order, d),
                              stencil.gradient_padded(fp, g, 0.3, order, d))


def test_quadratic_exact_on_polynomials():
    # The Laplacian of x^2 + 2 y^2 - z^2 is 2 + 4 - 2 = 4 for every order
    n, g = 12, 3
    ax = np.arange(n + 2 * g, dtype=np.float64) * 0.5
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    f = X ** 2 + 2 * Y ** 2 - Z ** 2
    for order in (2, 4, 6):
        L = stencil.laplacian_padded(f, g, 0.5, order)
        assert np.max(np.abs(L - 4.0)) < 1e-9


def test_stencil_sizes_are_the_printed_ones():
    """App. A: order p (the ghost width) gives the 7/13/19-point Laplacian and
    the 3/5/7-point gradient; the oracle's order-2p stencils have half width p
    and those point counts."""
    from tests.helpers import golden
    G = golden("app_a_stencils.json")
    for p in (1, 2, 3):
        lap = stencil.LAPLACIAN_WEIGHTS[2 * p]
        assert stencil.half_width(2 * p) == p and len(lap) == 2 * p + 1
        assert all(w != 0 for w in lap)
        assert 1 + 3 * (len(lap) - 1) == G["laplacian_points_3d"][str(p)]     # centre shared by the 3 axes
        assert len(stencil.GRADIENT_WEIGHTS[2 * p]) == G["gradient_points_1d"][str(p)]
