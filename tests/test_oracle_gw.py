"""Pins of the oracle's gravitational-wave tensor (Sec. 5 form in oracle/gw.py)."""
import numpy as np
import pytest

from oracle import gw
from oracle.eom import EOMParams


def _sigma(order, theta, dx):
    """Closed-form symbol of the central first derivative: d/dx e^{i theta j}
    = i sigma e^{i theta j}."""
    if order == 2:
        return np.sin(theta) / dx
    if order == 4:
        return ((4.0 / 3.0) * np.sin(theta) - (1.0 / 6.0) * np.sin(2 * theta)) / dx
    return (1.5 * np.sin(theta) - 0.3 * np.sin(2 * theta) + (1.0 / 30.0) * np.sin(3 * theta)) / dx


def _mode(n, m):
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    th = 2 * np.pi * np.asarray(m) / n
    return th, th[0] * X + th[1] * Y + th[2] * Z


@pytest.mark.parametrize("order", [2, 4, 6])
def test_source_closed_form_on_lattice_mode(order):
    n, dx = 12, 0.3
    th, ph = _mode(n, (1, -2, 3))
    psi1, psi2 = np.cos(ph), 0.5 * np.sin(ph)
    sig = {d: _sigma(order, th[i], dx) for i, d in enumerate("xyz")}
    got = gw.source(psi1, psi2, dx, order)
    for (i, j), S in zip(gw.PAIRS, got):
        exp = 2.0 * sig[i] * sig[j] * (np.sin(ph) ** 2 + 0.25 * np.cos(ph) ** 2)
        assert np.max(np.abs(S - exp)) < 1e-12 * max(1.0, np.max(np.abs(exp)))


def test_axis_exchange_permutes_components():
    n, dx = 8, 0.5
    rng = np.random.default_rng(0)
    psi1, psi2 = rng.standard_normal((2, n, n, n))
    S = gw.source(psi1, psi2, dx, 4)
    St = gw.source(np.swapaxes(psi1, 1, 2), np.swapaxes(psi2, 1, 2), dx, 4)   # swap x <-> y
    perm = {0: 1, 1: 0, 2: 2, 3: 3, 4: 5, 5: 4}                                 # xx<->yy, xz<->yz
    for k, kt in perm.items():
        assert np.allclose(np.swapaxes(S[k], 1, 2), St[kt], rtol=0, atol=1e-12)


def _lap_symbol(order, th):
    if order == 2:
        return 4.0 * np.sin(th / 2) ** 2
    if order == 4:
        return 2.5 - (8.0 / 3.0) * np.cos(th) + (1.0 / 6.0) * np.cos(2 * th)
    return 49.0 / 18.0 - 3.0 * np.cos(th) + 0.3 * np.cos(2 * th) - np.cos(3 * th) / 45.0


@pytest.mark.parametrize("order", [2, 4])
def test_source_free_mode_rk4_amplification(order):
    """Homogeneous psi (no gradients, no source) and a lattice mode in u_xy:
    the step is the closed-form RK4 amplification of (u, v)."""
    n, dx, dt, nst = 8, 0.5, 0.05, 20
    th, ph = _mode(n, (1, 2, -1))
    lam = sum(_lap_symbol(order, t) for t in th) / dx ** 2
    one = np.ones((n, n, n))
    y = [0.6 * one, 0.3 * one, 0 * one, 0 * one] + [0 * one] * 12
    y[4 + 3] = np.cos(ph)
    p = EOMParams(lam=1.0, a=0.0, friction=False, eta_power=0, order=order)
    eta = 1.0
    for _ in range(nst):
        y = gw.rk4_step_periodic(y, eta, dt, dx, p)
        eta += dt
    M = np.array([[0.0, 1.0], [-lam, 0.0]]) * dt
    R = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    A, B = np.linalg.matrix_power(R, nst) @ np.array([1.0, 0.0])
    assert np.max(np.abs(y[4 + 3] - A * np.cos(ph))) < 1e-12
    assert np.max(np.abs(y[10 + 3] - B * np.cos(ph))) < 1e-12 * max(1.0, lam)
    for k in (0, 1, 2, 4, 5):
        assert np.max(np.abs(y[4 + k])) < 1e-25 and np.max(np.abs(y[10 + k])) < 1e-25


def test_friction_ode_fourth_order():
    """Homogeneous u with u' = v0 at eta0 and no source: v = v0 (eta0/eta)^2,
    u = u0 + v0 eta0^2 (1/eta0 - 1/eta); RK4 error falls ~16x per halving."""
    one = np.ones((4, 4, 4))
    eta0, T, u0, v0 = 0.5, 1.0, 0.2, 0.7
    errs = []
    for nst in (10, 20, 40):
        dt = T / nst
        y = [0.6 * one, 0.3 * one, 0 * one, 0 * one] + [u0 * one] * 6 + [v0 * one] * 6
        p = EOMParams(lam=0.0, a=0.0, friction=True, eta_power=0, order=4)
        eta = eta0
        for _ in range(nst):
            y = gw.rk4_step_periodic(y, eta, dt, 0.5, p)
            eta += dt
        ue = u0 + v0 * eta0 ** 2 * (1.0 / eta0 - 1.0 / (eta0 + T))
        ve = v0 * (eta0 / (eta0 + T)) ** 2
        errs.append(max(abs(y[4][0, 0, 0] - ue), abs(y[10][0, 0, 0] - ve)))
    assert 12.0 < errs[0] / errs[1] < 20.0 and 12.0 < errs[1] / errs[2] < 20.0, errs
