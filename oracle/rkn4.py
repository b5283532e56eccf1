"""Fourth-order Runge-Kutta-Nystrom (integrator type 21 of Tab.
"integrator", "RKN4") on a uniform periodic lattice.  Test infrastructure:
imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline.

The paper names the method and prints no tableau.  It is read as Nystrom's
classical fourth-order method for second-order systems x'' = a(t, x, x')
whose acceleration may depend on the velocity (the Hubble friction does):
with positions x (psi, and u_ij with the tensor fields) and velocities
v = x' (Pi, v_ij),

    a1 = a(t,        x,                               v)
    a2 = a(t + dt/2, x + dt/2 v + dt^2/8 a1,          v + dt/2 a1)
    a3 = a(t + dt/2, x + dt/2 v + dt^2/8 a1,          v + dt/2 a2)
    a4 = a(t + dt,   x + dt v + dt^2/2 a3,            v + dt a3)
    x' = x + dt v + dt^2/6 (a1 + a2 + a3)
    v' = v + dt/6 (a1 + 2 a2 + 2 a3 + a4)

Stages 2 and 3 share their position, so the stage times are those of the
classic RK4 (c = 0, 1/2, 1/2, 1).  The scheme needs x' = v exactly, so it is
not combined with the Kreiss-Oliger term (which acts on x' too).

Parity: pinned (exact on polynomial solutions of degree <= 4; fourth-order
convergence to the closed form (A sin w eta + B cos w eta)/eta of a lattice
Fourier mode with the 2/eta friction; energy drift O(dt^4) of the nonlinear
friction-free system with frozen coefficients) -- tests/test_oracle_rkn4.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams
from .rk4 import f_periodic

C = (0.0, 0.5, 0.5, 1.0)
POS, VEL = (0, 1), (2, 3)                              # the scalar system
POS_GW, VEL_GW = (0, 1, 4, 5, 6, 7, 8, 9), (2, 3, 10, 11, 12, 13, 14, 15)   # with the tensor fields


def stage_states(x, v, dt, acc_prev, s):
    """Positions and velocities of stage s (1..3, 0-based after the first)
    from the step's start (x, v) and the previous stages' accelerations."""
    if s == 1:
        a1 = acc_prev[0]
        return ([xi + (0.5 * dt) * vi + (dt * dt / 8.0) * ai for xi, vi, ai in zip(x, v, a1)],
                [vi + (0.5 * dt) * ai for vi, ai in zip(v, a1)])
    if s == 2:
        a1, a2 = acc_prev[0], acc_prev[1]
        return ([xi + (0.5 * dt) * vi + (dt * dt / 8.0) * ai for xi, vi, ai in zip(x, v, a1)],
                [vi + (0.5 * dt) * ai for vi, ai in zip(v, a2)])
    a3 = acc_prev[2]
    return ([xi + dt * vi + (dt * dt / 2.0) * ai for xi, vi, ai in zip(x, v, a3)],
            [vi + dt * ai for vi, ai in zip(v, a3)])


def final_state(x, v, dt, acc):
    a1, a2, a3, a4 = acc
    xn = [xi + dt * vi + (dt * dt / 6.0) * (p1 + p2 + p3) for xi, vi, p1, p2, p3 in zip(x, v, a1, a2, a3)]
    vn = [vi + (dt / 6.0) * (p1 + 2.0 * p2 + 2.0 * p3 + p4) for vi, p1, p2, p3, p4 in zip(v, a1, a2, a3, a4)]
    return xn, vn


def rkn4_step(y, eta: float, dt: float, dx: float, p: EOMParams, f=f_periodic, pos=POS, vel=VEL):
    """One RKN4 step of the fields ``y``; ``f(y, eta, dx, p)`` gives the time
    derivatives of every field (positions' derivatives must be the
    velocities), of which the accelerations (at ``vel``) are used."""
    if getattr(p, "ko_order", 0):
        raise ValueError("RKN4 needs x' = v: no Kreiss-Oliger term")
    y = [np.asarray(a, dtype=np.float64) for a in y]
    x = [y[i] for i in pos]
    v = [y[i] for i in vel]

    def assemble(xs, vs):
        out = list(y)
        for i, a in zip(pos, xs):
            out[i] = a
        for i, a in zip(vel, vs):
            out[i] = a
        return out

    acc = []
    state = y
    for s in range(4):
        if s > 0:
            state = assemble(*stage_states(x, v, dt, acc, s))
        d = f(state, eta + C[s] * dt, dx, p)
        acc.append([np.asarray(d[i], dtype=np.float64) for i in vel])
    return tuple(assemble(*final_state(x, v, dt, acc)))


def rkn4_step_periodic(y, eta: float, dt: float, dx: float, p: EOMParams):
    """One RKN4 step of the scalar system (psi1, psi2, Pi1, Pi2)."""
    return rkn4_step(y, eta, dt, dx, p)
