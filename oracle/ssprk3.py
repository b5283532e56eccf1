"""Low-storage third-order strong-stability-preserving Runge-Kutta
(integrator type 10 of Tab. "integrator", the paper's example default; type
3 is the same scheme with more storage) on a uniform periodic lattice.  Test
infrastructure: imported only by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline.

The paper names the method only.  It is read as the three-stage, third-order
SSP scheme in Shu-Osher form, whose low-storage implementation keeps y_n and
one stage value:

    Y1 = y_n + dt f(eta_n,          y_n)
    Y2 = 3/4 y_n + 1/4 (Y1 + dt f(eta_n + dt,   Y1))
    y' = 1/3 y_n + 2/3 (Y2 + dt f(eta_n + dt/2, Y2))

so stage s evaluates f at eta_n + c_s dt with c = (0, 1, 1/2) and combines
a_s y_n + b_s (Y_s + dt k_s) with (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3).

Parity: pinned (the closed-form amplification 1 + z + z^2/2 + z^3/6 of a
lattice Fourier mode; third-order convergence of the homogeneous field with
the eta-dependent coefficients; the App. B plane-wave energy error falls
like N^-3, the paper's RK3 slope being -3.0) -- tests/test_oracle_ssprk3.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams
from .rk4 import f_periodic

C = (0.0, 1.0, 0.5)
A = (0.0, 0.75, 1.0 / 3.0)
B = (1.0, 0.25, 2.0 / 3.0)


def ssprk3_step_periodic(y, eta: float, dt: float, dx: float, p: EOMParams, f=f_periodic):
    """One SSPRK3 step of the fields ``y`` (f: the time derivative on a
    periodic lattice, the scalar system by default)."""
    y0 = tuple(np.asarray(a, dtype=np.float64) for a in y)
    u = y0
    for s in range(3):
        k = f(u, eta + C[s] * dt, dx, p)
        u = tuple(A[s] * a + B[s] * (ui + dt * ki) for a, ui, ki in zip(y0, u, k))
    return u
