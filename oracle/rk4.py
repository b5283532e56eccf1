"""Classic fourth-order Runge-Kutta (integrator type 4 of Tab. "integrator")
on a uniform periodic lattice.

Butcher tableau c = (0, 1/2, 1/2, 1), a_21 = a_32 = 1/2, a_43 = 1,
b = (1/6, 1/3, 1/3, 1/6).  Stage s is evaluated at eta_n + c_s dt, so the
eta-dependent coefficients 2/eta and lambda eta^2 take the stage time.

    k1 = f(eta_n,        y)
    k2 = f(eta_n + dt/2, y + (dt/2) k1)
    k3 = f(eta_n + dt/2, y + (dt/2) k2)
    k4 = f(eta_n + dt,   y + dt k3)
    y' = y + (dt/6) (k1 + 2 k2 + 2 k3 + k4),     eta' = eta_n + dt

Parity: pinned (closed-form RK4 amplification of a lattice Fourier mode,
energy drift O(dt^4) in the frozen-coefficient friction-free limit, the
App. B plane-wave energy convergence) -- tests/test_oracle_rk4.py.
"""
from __future__ import annotations

import numpy as np

from . import ko
from .eom import EOMParams, rhs
from .stencil import laplacian_periodic

C = (0.0, 0.5, 0.5, 1.0)


def f_periodic(y, eta, dx, p: EOMParams):
    psi1, psi2, pi1, pi2 = y
    lap1 = laplacian_periodic(psi1, dx, p.order)
    lap2 = laplacian_periodic(psi2, dx, p.order)
    d = rhs(psi1, psi2, pi1, pi2, lap1, lap2, eta, p)
    if p.ko_order:
        # Kreiss-Oliger dissipation of every scalar component (Sec. 2.4)
        d = tuple(dc + ko.ko_periodic(f, dx, p.ko_order, p.ko_eps) for dc, f in zip(d, y))
    return d


def rk4_step_periodic(y, eta: float, dt: float, dx: float, p: EOMParams):
    """One RK4 step of the four fields ``y`` = (psi1, psi2, Pi1, Pi2)."""
    y = tuple(np.asarray(a, dtype=np.float64) for a in y)
    k1 = f_periodic(y, eta, dx, p)
    y2 = tuple(a + (0.5 * dt) * k for a, k in zip(y, k1))
    k2 = f_periodic(y2, eta + 0.5 * dt, dx, p)
    y3 = tuple(a + (0.5 * dt) * k for a, k in zip(y, k2))
    k3 = f_periodic(y3, eta + 0.5 * dt, dx, p)
    y4 = tuple(a + dt * k for a, k in zip(y, k3))
    k4 = f_periodic(y4, eta + dt, dx, p)
    return tuple(a + (dt / 6.0) * (q1 + 2.0 * q2 + 2.0 * q3 + q4)
                 for a, q1, q2, q3, q4 in zip(y, k1, k2, k3, k4))


def evolve_periodic(y, eta0: float, dt: float, dx: float, nsteps: int, p: EOMParams,
                    callback=None):
    """``nsteps`` RK4 steps; eta advances by repeated FP64 addition of dt.
    ``callback(step, y, eta)`` runs before each step (step = 0..nsteps-1)."""
    eta = eta0
    for s in range(nsteps):
        if callback is not None:
            callback(s, y, eta)
        y = rk4_step_periodic(y, eta, dt, dx, p)
        eta = eta + dt
    return y, eta
