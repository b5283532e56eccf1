"""Fifth-order Runge-Kutta-Nystrom (integrator type 22 of Tab.
"integrator", "RKN5") on a uniform periodic lattice.  Test infrastructure:
imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline.

The paper names the method and prints no tableau.  It is read as Nystrom's
classical four-stage fifth-order method for second-order systems
x'' = a(t, x) whose acceleration does not depend on the velocity: with
positions x (psi) and velocities v = x' (Pi), step h,

    k_i = a(t + c_i h,  x + c_i h v + h^2 sum_{j<i} abar_ij k_j)
    x'  = x + h v + h^2 sum_i bbar_i k_i
    v'  = v + h sum_i b_i k_i

    c    = (0, 1/5, 2/3, 1)
    abar = [[    0,     0,    0],
            [ 1/50,     0,    0],
            [-1/27,  7/27,    0],
            [ 3/10, -2/35, 9/35]]
    bbar = (14, 100, 54, 0) / 336
    b    = (14, 125, 162, 35) / 336

The fifth-order conditions for x'' = a(t, x) hold for these weights; a
velocity-dependent acceleration (the 2/eta friction, the Kreiss-Oliger term
acting on x') is outside the method, so the step rejects both.  The paper's
own use of the method is the friction-free wave of App. B.

Parity: pinned (exact on polynomial solutions of degree <= 5 and not on
degree 6; fifth-order convergence against an independent ODE integrator on a
nonlinear, explicitly time-dependent system; fifth-order convergence to the
closed form cos/sin of a friction-free lattice Fourier mode; App. B energy
slope against the paper's printed value) -- tests/test_oracle_rkn5.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams
from .rk4 import f_periodic

C = (0.0, 1.0 / 5.0, 2.0 / 3.0, 1.0)
ABAR = ((),
        (1.0 / 50.0,),
        (-1.0 / 27.0, 7.0 / 27.0),
        (3.0 / 10.0, -2.0 / 35.0, 9.0 / 35.0))
BBAR = (14.0 / 336.0, 100.0 / 336.0, 54.0 / 336.0, 0.0)
B = (14.0 / 336.0, 125.0 / 336.0, 162.0 / 336.0, 35.0 / 336.0)
POS, VEL = (0, 1), (2, 3)


def rkn5_step(y, eta: float, dt: float, dx: float, p: EOMParams, f=f_periodic, pos=POS, vel=VEL):
    """One RKN5 step of the fields ``y``; ``f(y, eta, dx, p)`` gives the time
    derivatives of every field, of which the accelerations (at ``vel``) are
    used.  The stage states carry the step's starting velocities (the
    acceleration must not depend on them)."""
    if getattr(p, "friction", False):
        raise ValueError("RKN5 needs an acceleration independent of the velocities: friction off")
    if getattr(p, "ko_order", 0):
        raise ValueError("RKN5 needs x' = v: no Kreiss-Oliger term")
    y = [np.asarray(a, dtype=np.float64) for a in y]
    x = [y[i] for i in pos]
    v = [y[i] for i in vel]
    k = []
    for s in range(4):
        state = list(y)
        for n, i in enumerate(pos):
            xs = x[n] + (C[s] * dt) * v[n]
            for j in range(s):
                xs = xs + (dt * dt * ABAR[s][j]) * k[j][n]
            state[i] = xs
        d = f(state, eta + C[s] * dt, dx, p)
        k.append([np.asarray(d[i], dtype=np.float64) for i in vel])
    out = list(y)
    for n, i in enumerate(pos):
        out[i] = x[n] + dt * v[n] + (dt * dt) * sum(BBAR[s] * k[s][n] for s in range(4))
    for n, i in enumerate(vel):
        out[i] = v[n] + dt * sum(B[s] * k[s][n] for s in range(4))
    return tuple(out)


def rkn5_step_periodic(y, eta: float, dt: float, dx: float, p: EOMParams):
    """One RKN5 step of the scalar system (psi1, psi2, Pi1, Pi2)."""
    return rkn5_step(y, eta, dt, dx, p)
