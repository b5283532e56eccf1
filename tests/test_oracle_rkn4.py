"""Pins of the oracle's fourth-order Runge-Kutta-Nystrom step (integrator
type 21, oracle/rkn4.py) against polynomial solutions, the closed form of a
damped lattice mode with the 2/eta friction, an independent ODE integrator,
and energy conservation of the nonlinear friction-free system."""
import numpy as np
import pytest

from oracle import energy, rkn4
from oracle.eom import EOMParams
from oracle.stencil import laplacian_periodic


def _ode(acc):
    """A scalar second-order ODE x'' = acc(t, x, v) in the f(y, t, dx, p)
    form the step takes: y = (x, v), derivatives (v, acc)."""
    return lambda y, t, dx, p: (y[1], acc(t, y[0], y[1]))


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_polynomial_solutions_are_exact(deg):
    """A fourth-order Nystrom step reproduces x(t) = sum c_k t^k, k <= 4
    (x'' then depends on t alone), in position and velocity."""
    c = np.array([0.7, -1.3, 0.4, 2.1, -0.9])[:deg + 1]
    x = np.polynomial.Polynomial(c)
    a = x.deriv(2)
    f = _ode(lambda t, xx, vv: a(t) + 0.0 * xx)
    t0, dt = 0.3, 0.37
    out = rkn4.rkn4_step((np.array(x(t0)), np.array(x.deriv(1)(t0))), t0, dt, 1.0, EOMParams(),
                         f=f, pos=(0,), vel=(1,))
    assert abs(out[0] - x(t0 + dt)) <= 1e-13 * max(1.0, abs(x(t0 + dt)))
    assert abs(out[1] - x.deriv(1)(t0 + dt)) <= 1e-13 * max(1.0, abs(x.deriv(1)(t0 + dt)))


def test_quintic_is_not_exact():
    """... and no further: x = t^5 leaves an O(dt^5) position error, which
    falls by ~32 per halving of dt (the local error of a fourth-order
    method)."""
    f = _ode(lambda t, xx, vv: 20.0 * t ** 3 + 0.0 * xx)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        out = rkn4.rkn4_step((np.array(1.0 ** 5), np.array(5.0)), 1.0, dt, 1.0, EOMParams(), f=f, pos=(0,), vel=(1,))
        errs.append(abs(out[0] - (1.0 + dt) ** 5))
    assert errs[0] > 1e-8
    for e0, e1 in zip(errs, errs[1:]):
        assert 25 < e0 / e1 < 40, errs


def test_damped_lattice_mode_converges_at_fourth_order():
    """Massless, with the 2/eta friction: a lattice Fourier mode obeys
    psi'' + (2/eta) psi' + w^2 psi = 0, whose solutions are
    (A sin w eta + B cos w eta)/eta (eta psi is a free oscillator).  From
    eta = 1 to 3 the error falls by ~16 per halving of dt."""
    n, dx = 8, 0.5
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    mode = np.cos(2 * np.pi * (1 * X + 2 * Y - 1 * Z) / n)
    p = EOMParams(lam=0.0, a=0.0, friction=True, eta_power=2, order=4)
    w2 = -laplacian_periodic(mode, dx, 4)[0, 0, 0] / mode[0, 0, 0]
    w = np.sqrt(w2)
    # psi(1) = 1, psi'(1) = 0 fixes A, B
    eta0, eta1 = 1.0, 3.0
    M = np.array([[np.sin(w * eta0) / eta0, np.cos(w * eta0) / eta0],
                  [w * np.cos(w * eta0) / eta0 - np.sin(w * eta0) / eta0 ** 2,
                   -w * np.sin(w * eta0) / eta0 - np.cos(w * eta0) / eta0 ** 2]])
    A, B = np.linalg.solve(M, [1.0, 0.0])
    exact = (A * np.sin(w * eta1) + B * np.cos(w * eta1)) / eta1
    z = np.zeros((n, n, n))
    errs = []
    for nst in (20, 40, 80):
        dt = (eta1 - eta0) / nst
        y, eta = (mode, 0.5 * mode, z, z), eta0
        for _ in range(nst):
            y = rkn4.rkn4_step_periodic(y, eta, dt, dx, p)
            eta += dt
        errs.append(np.max(np.abs(y[0] - exact * mode)))
        assert np.max(np.abs(y[1] - 0.5 * exact * mode)) <= 0.5 * errs[-1] + 1e-14
    for e0, e1 in zip(errs, errs[1:]):
        assert 13 < e0 / e1 < 19, errs


def test_homogeneous_field_matches_independent_integrator():
    """A spatially constant field obeys the ODE of Sec. 3.1 without the
    Laplacian; RKN4 with 2/eta and lambda eta^2 at the stage times approaches
    a high-accuracy solution at fourth order."""
    from scipy.integrate import solve_ivp
    p = EOMParams(lam=1.0, a=0.3, friction=True, eta_power=2, order=4)
    psi0, pi0 = np.array([0.6, -0.5]), np.array([0.2, 0.1])
    eta0, T = 0.5, 1.0

    def f(eta, s):
        ps, pi = s[:2], s[2:]
        pot = p.lam * eta ** 2 * (ps @ ps - 1.0) + p.a
        return np.concatenate([pi, -(2.0 / eta) * pi - ps * pot])

    ref = solve_ivp(f, (eta0, eta0 + T), np.concatenate([psi0, pi0]), method="DOP853",
                    rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for nst in (40, 80, 160):
        dt = T / nst
        y = tuple(np.full((4, 4, 4), v) for v in np.concatenate([psi0, pi0]))
        eta = eta0
        for _ in range(nst):
            y = rkn4.rkn4_step_periodic(y, eta, dt, 1.0, p)
            eta += dt
        errs.append(max(abs(y[c][0, 0, 0] - ref[c]) for c in range(4)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 12 < e0 / e1 < 20, errs


def test_energy_drift_is_fourth_order():
    """Flat, friction-free, frozen coefficients (lambda eta^2 -> lambda): the
    lattice energy is conserved by the semi-discrete system; RKN4's drift
    over a fixed time falls by ~16 per halving of dt."""
    from paper_2404_02950_gb300 import inputs
    n, dx = 16, 0.5
    p = EOMParams(lam=1.0, a=0.0, friction=False, eta_power=0, order=4)
    y0 = inputs.gaussian_field(n, 3.0, 4)
    E0 = energy.energy_periodic(y0, 1.0, dx, p)[3]
    drifts = []
    for nst in (16, 32, 64):
        dt = 0.8 / nst
        y = y0
        for _ in range(nst):
            y = rkn4.rkn4_step_periodic(y, 1.0, dt, dx, p)
        drifts.append(abs(energy.energy_periodic(y, 1.0, dx, p)[3] - E0))
    for d0, d1 in zip(drifts, drifts[1:]):
        assert 10 < d0 / d1 < 24, drifts


def test_rejects_dissipation():
    with pytest.raises(ValueError):
        rkn4.rkn4_step_periodic([np.zeros((4, 4, 4))] * 4, 1.0, 0.1, 1.0, EOMParams(ko_order=3, ko_eps=0.1))


def test_tensor_fields_follow_the_damped_closed_form():
    """The 16-field state (positions psi and u_ij, velocities Pi and v_ij):
    with a homogeneous psi on the vacuum circle there is no source, and a
    lattice mode of u_xy alone is the damped oscillator of the scalar case,
    (A sin w eta + B cos w eta)/eta, reached at fourth order; psi stays put."""
    from oracle import gw as ogw
    n, dx = 8, 0.5
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    mode = np.cos(2 * np.pi * (2 * X - 1 * Y + 1 * Z) / n)
    p = EOMParams(lam=1.0, a=0.0, friction=True, eta_power=2, order=4)
    w = np.sqrt(-laplacian_periodic(mode, dx, 4)[0, 0, 0] / mode[0, 0, 0])
    eta0, eta1 = 1.0, 2.0
    # u(1) = 1, u'(1) = 0
    M = np.array([[np.sin(w * eta0) / eta0, np.cos(w * eta0) / eta0],
                  [w * np.cos(w * eta0) / eta0 - np.sin(w * eta0) / eta0 ** 2,
                   -w * np.sin(w * eta0) / eta0 - np.cos(w * eta0) / eta0 ** 2]])
    A, B = np.linalg.solve(M, [1.0, 0.0])
    exact = (A * np.sin(w * eta1) + B * np.cos(w * eta1)) / eta1
    one, z = np.ones((n, n, n)), np.zeros((n, n, n))
    errs = []
    for nst in (32, 64, 128):
        dt = (eta1 - eta0) / nst
        y = [np.sqrt(0.5) * one, np.sqrt(0.5) * one, z, z] + [z] * 3 + [mode] + [z] * 2 + [z] * 6
        eta = eta0
        for _ in range(nst):
            y = rkn4.rkn4_step(y, eta, dt, dx, p, f=ogw.f_periodic, pos=rkn4.POS_GW, vel=rkn4.VEL_GW)
            eta += dt
        errs.append(np.max(np.abs(y[7] - exact * mode)))
        for c in (4, 5, 6, 8, 9, 10, 11, 12, 14, 15):
            assert np.max(np.abs(y[c])) < 1e-28, c        # rounding of the (vanishing) source only
        assert np.max(np.abs(y[0] - np.sqrt(0.5))) < 1e-14 and np.max(np.abs(y[2])) < 1e-14
    for e0, e1 in zip(errs, errs[1:]):
        assert 13 < e0 / e1 < 19, errs
