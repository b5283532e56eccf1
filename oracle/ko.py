"""Kreiss-Oliger dissipation (Sec. 2.4).  Test infrastructure: imported only
by tests/, __graft_entry__.smoke() and bench.py's CPU baseline.

The small-scale operator added to the evolution of each scalar field
component is

    Q_l = (-1)^((p+3)/2) eps dx_l^p / 2^(p+1) sum_d d^(p+1)/dx_d^(p+1),

p odd (the dissipation order), eps the strength.  The (p+1)-st derivative is
the central difference of p+2 points (binomial weights):

    d^(p+1) f ~ dx^-(p+1) sum_{j=0..p+1} (-1)^j C(p+1, j) f(x + ((p+1)/2 - j) dx),

so Q f = (-1)^((p+3)/2) eps / (2^(p+1) dx) sum_d delta_d^(p+1) f.  Its symbol on
a lattice wave e^{i theta . x} is -(eps/dx) sum_d sin^(p+1)(theta_d / 2): real,
never positive, largest at the Nyquist frequency.

App. C checks the operator on a propagating discontinuity of the advection
equation du/dt + c . grad u = 0; app_c_advection runs that experiment (classic
RK4, central gradient, dissipation added to the right-hand side).

Parity: pinned (the symbol on lattice plane waves for p = 1, 3, 5; constants
and polynomials of degree <= p are annihilated; a free lattice mode with
dissipation follows the closed-form RK4 amplification; the App. C run equals
its closed-form modal solution, conserves energy to the O(0.1-0.3) % the
paper prints without dissipation, and eps ~ 1e-2 damps the high-frequency
content while eps ~ 1 leaks energy) -- tests/test_oracle_ko.py.
"""
from __future__ import annotations

from math import comb

import numpy as np


def weights(p: int):
    """(offset, weight) pairs of delta^(p+1), offsets -(p+1)/2 .. (p+1)/2."""
    if p < 1 or p % 2 == 0:
        raise ValueError("dissipation order p must be odd and >= 1")
    n = p + 1
    return [(n // 2 - j, (-1) ** j * comb(n, j)) for j in range(n + 1)]


def coefficient(p: int, eps: float, dx: float) -> float:
    """(-1)^((p+3)/2) eps / (2^(p+1) dx)."""
    return (-1.0) ** ((p + 3) // 2) * eps / (2.0 ** (p + 1) * dx)


def ko_periodic(f, dx: float, p: int, eps: float):
    """Q f on a periodic [z, y, x] lattice."""
    out = np.zeros_like(np.asarray(f, dtype=np.float64))
    for axis in (2, 1, 0):
        acc = np.zeros_like(out)
        for off, w in weights(p):
            acc = acc + float(w) * np.roll(f, -off, axis=axis)
        out = out + acc
    return coefficient(p, eps, dx) * out


def ko_padded(fp, g: int, dx: float, p: int, eps: float):
    """Q f on the valid cells of a ghost-padded [z, y, x] array (g >= (p+1)/2)."""
    h = (p + 1) // 2
    if g < h:
        raise ValueError("ghost width smaller than the dissipation stencil")
    nz, ny, nx = (s - 2 * g for s in fp.shape)
    out = np.zeros((nz, ny, nx))
    for dz, dy, dxx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
        acc = np.zeros((nz, ny, nx))
        for off, w in weights(p):
            acc = acc + float(w) * fp[g + off * dz:g + off * dz + nz, g + off * dy:g + off * dy + ny,
                                      g + off * dxx:g + off * dxx + nx]
        out = out + acc
    return coefficient(p, eps, dx) * out


def app_c_advection(n: int, eps: float, p: int = 5, c=(2.0, 2.0, 2.0), box_side: float = 10.0, t_end: float = 5.0,
                    dt_over_dx: float = 0.3, grad_order: int = 4, ny: int = 4):
    """The App. C experiment on an n x ny x ny periodic lattice of cells of
    side box_side / n: u = 1 on the slab x < box_side / 2 (cell centres), 0
    elsewhere; round(t_end / dt) classic RK4 steps of
        du/dt = -(c_x D_x + c_y D_y + c_z D_z) u + Q u
    with D the central first difference of accuracy grad_order (App. A) and Q
    the dissipation of order p and strength eps.  Returns (u0, u, dt, steps)."""
    from .stencil import gradient_periodic

    dx = box_side / n
    dt = dt_over_dx * dx
    steps = int(round(t_end / dt))
    x = (np.arange(n) + 0.5) * dx
    u0 = np.broadcast_to((x < 0.5 * box_side).astype(np.float64), (ny, ny, n)).copy()

    def f(u):
        r = -(c[0] * gradient_periodic(u, dx, grad_order, "x") + c[1] * gradient_periodic(u, dx, grad_order, "y")
              + c[2] * gradient_periodic(u, dx, grad_order, "z"))
        if eps > 0.0:
            r = r + ko_periodic(u, dx, p, eps)
        return r

    u = u0
    for _ in range(steps):
        k1 = f(u)
        k2 = f(u + (0.5 * dt) * k1)
        k3 = f(u + (0.5 * dt) * k2)
        k4 = f(u + dt * k3)
        u = u + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return u0, u, dt, steps

