"""Gravitational-wave auxiliary tensor (Sec. 5).

The paper evolves auxiliary fields u_ij (components xx, yy, zz, xy, xz, yz,
Eq. GWEOM) whose source is problem specific.  The form used here for the
axion string field, in conformal time with the radiation-era friction of
Sec. 3.1, is

    u_ij'' + (2/eta) u_ij' - lap u_ij = 2 sum_a d_i psi_a d_j psi_a,

split into first-order form with v_ij = u_ij':

    u_ij' = v_ij
    v_ij' = -(2/eta) v_ij + lap u_ij + 2 (d_i psi1 d_j psi1 + d_i psi2 d_j psi2)

The Laplacian is the same FD operator as the scalars' (accuracy ``order``);
the gradients are the central differences of the same accuracy (App. A,
``Gradient<order>``).  The full state is 16 fields: psi1, psi2, Pi1, Pi2,
then u_xx..u_yz, then v_xx..v_yz.

Parity: pinned (the source against the closed-form gradient symbol on a
lattice plane wave; a source-free lattice mode of u against the closed-form
RK4 amplification) -- tests/test_oracle_gw.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams, coefficients
from .rk4 import f_periodic as scalar_f_periodic
from .stencil import gradient_padded, gradient_periodic, laplacian_padded, laplacian_periodic

# (i, j) direction pairs of the six components
PAIRS = (("x", "x"), ("y", "y"), ("z", "z"), ("x", "y"), ("x", "z"), ("y", "z"))


def source(psi1, psi2, dx, order, grad=None):
    """2 sum_a d_i psi_a d_j psi_a for the six pairs (periodic lattice unless
    ``grad`` supplies the gradient function)."""
    if grad is None:
        def grad(f, d):
            return gradient_periodic(f, dx, order, d)
    g1 = {d: grad(psi1, d) for d in "xyz"}
    g2 = {d: grad(psi2, d) for d in "xyz"}
    return [2.0 * (g1[i] * g1[j] + g2[i] * g2[j]) for i, j in PAIRS]


def rhs_gw(u, v, lap_u, src, eta, p: EOMParams):
    """(du, dv) for the six components; dv = (-c_fric) v + lap u + src."""
    c_fric, _ = coefficients(eta, p)
    du = [vk.copy() for vk in v]
    dv = [(-c_fric) * vk + lk + sk for vk, lk, sk in zip(v, lap_u, src)]
    return du, dv


def f_periodic(y, eta, dx, p: EOMParams):
    """Time derivative of the 16-field state on a periodic lattice."""
    psi1, psi2, pi1, pi2 = y[:4]
    u, v = list(y[4:10]), list(y[10:16])
    ds = scalar_f_periodic((psi1, psi2, pi1, pi2), eta, dx, p)
    lap_u = [laplacian_periodic(uk, dx, p.order) for uk in u]
    du, dv = rhs_gw(u, v, lap_u, source(psi1, psi2, dx, p.order), eta, p)
    return tuple(ds) + tuple(du) + tuple(dv)


def rk4_step_periodic(y, eta: float, dt: float, dx: float, p: EOMParams):
    """Classic RK4 (integrator type 4) of the 16-field state."""
    y = tuple(np.asarray(a, dtype=np.float64) for a in y)
    k1 = f_periodic(y, eta, dx, p)
    k2 = f_periodic(tuple(a + (0.5 * dt) * k for a, k in zip(y, k1)), eta + 0.5 * dt, dx, p)
    k3 = f_periodic(tuple(a + (0.5 * dt) * k for a, k in zip(y, k2)), eta + 0.5 * dt, dx, p)
    k4 = f_periodic(tuple(a + dt * k for a, k in zip(y, k3)), eta + dt, dx, p)
    return tuple(a + (dt / 6.0) * (q1 + 2.0 * q2 + 2.0 * q3 + q4)
                 for a, q1, q2, q3, q4 in zip(y, k1, k2, k3, k4))


def rhs_box_gw(arr, g, dx, eta, p: EOMParams):
    """Time derivatives of the 12 GW fields on the valid cells of a
    ghost-padded 16-field box array (psi and u ghosts filled)."""
    v = (slice(g, arr.shape[1] - g), slice(g, arr.shape[2] - g), slice(g, arr.shape[3] - g))

    def grad(f, d):
        return gradient_padded(f, g, dx, p.order, d)

    src = source(arr[0], arr[1], dx, p.order, grad=grad)
    lap_u = [laplacian_padded(arr[4 + k], g, dx, p.order) for k in range(6)]
    du, dv = rhs_gw([arr[4 + k][v] for k in range(6)], [arr[10 + k][v] for k in range(6)], lap_u, src, eta, p)
    return du + dv
