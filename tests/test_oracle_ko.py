"""Pins of the oracle's Kreiss-Oliger dissipation (Sec. 2.4, oracle/ko.py)."""
from math import factorial

import numpy as np
import pytest

from oracle import ko, rk4
from oracle.eom import EOMParams


def _mode(n, m):
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    th = 2 * np.pi * np.asarray(m) / n
    return th, th[0] * X + th[1] * Y + th[2] * Z


@pytest.mark.parametrize("p", [1, 3, 5])
def test_symbol_on_lattice_waves(p):
    n, dx, eps = 12, 0.4, 0.07
    for m in ((1, 0, 0), (2, -3, 5), (6, 6, 6)):
        th, ph = _mode(n, m)
        q = -(eps / dx) * sum(np.sin(t / 2) ** (p + 1) for t in th)
        got = ko.ko_periodic(np.cos(ph), dx, p, eps)
        assert np.max(np.abs(got - q * np.cos(ph))) < 1e-13
    # the Nyquist mode along all three axes is damped at the largest rate
    th, ph = _mode(n, (6, 6, 6))
    assert np.allclose(ko.ko_periodic(np.cos(ph), dx, p, eps), -3 * eps / dx * np.cos(ph), atol=1e-12)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_polynomials_up_to_degree_p_are_annihilated(p):
    g, n, dx, eps = 3, 6, 0.5, 0.2
    x = (np.arange(n + 2 * g) - g) * dx
    for k in range(p + 2):
        fp = np.broadcast_to(x ** k, (n + 2 * g,) * 3).copy()   # varies along x only
        got = ko.ko_padded(fp, g, dx, p, eps)
        exp = ko.coefficient(p, eps, dx) * (factorial(p + 1) * dx ** (p + 1) if k == p + 1 else 0.0)
        assert np.allclose(got, exp, rtol=1e-9, atol=1e-9), k


def test_free_mode_with_dissipation_rk4_closed_form():
    """Flat, massless, friction-free, with dissipation on psi and Pi: each
    lattice mode obeys (psi, Pi)' = [[q, 1], [-w^2, q]] (psi, Pi) and one RK4
    step multiplies it by the truncated exponential of that matrix."""
    n, dx, dt, nst, p_ko, eps = 12, 0.5, 0.1, 6, 3, 0.3
    th, ph = _mode(n, (2, -1, 3))
    w2 = sum(2.5 - (8.0 / 3.0) * np.cos(t) + (1.0 / 6.0) * np.cos(2 * t) for t in th) / dx ** 2
    q = -(eps / dx) * sum(np.sin(t / 2) ** (p_ko + 1) for t in th)
    p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=4, ko_order=p_ko, ko_eps=eps)
    z = np.zeros((n, n, n))
    y = (np.cos(ph), z, 0.2 * np.cos(ph), z)
    eta = 1.0
    for _ in range(nst):
        y = rk4.rk4_step_periodic(y, eta, dt, dx, p)
        eta += dt
    M = np.array([[q, 1.0], [-w2, q]]) * dt
    R = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    A, B = np.linalg.matrix_power(R, nst) @ np.array([1.0, 0.2])
    assert np.max(np.abs(y[0] - A * np.cos(ph))) < 1e-12
    assert np.max(np.abs(y[2] - B * np.cos(ph))) < 1e-12 * max(1.0, w2)
    assert abs(A) < 1.0                      # damped


# ---------------------------------------------------------------------------
# App. C: a propagating discontinuity of the advection equation

def _app_c():
    from tests.helpers import golden
    return golden("app_c_ko.json")


def _upper_half_power(u):
    """Share of the spectral power of the x profile above half the Nyquist
    wavenumber (the high-frequency content)."""
    s = np.abs(np.fft.rfft(u[0, 0])) ** 2
    return float(s[len(s) // 2:].sum() / s.sum())


@pytest.mark.parametrize("eps", [0.0, 0.01, 1.0])
def test_app_c_run_equals_its_modal_closed_form(eps):
    """The run is linear and translation invariant: every lattice mode theta
    of the profile is multiplied by R(z)^steps with R the RK4 polynomial and
    z = dt (-i c_x (8 sin theta - sin 2 theta) / (6 dx) - eps / dx sin^6(theta/2))."""
    a = _app_c()
    n = 64
    u0, u, dt, steps = ko.app_c_advection(n, eps, p=a["dissipation_order_p"], c=tuple(a["wave_speed"]),
                                          box_side=a["box_side"], t_end=a["t_end"], dt_over_dx=a["dt_over_dx"])
    dx = a["box_side"] / n
    th = 2 * np.pi * np.arange(n // 2 + 1) / n
    z = dt * (-1j * a["wave_speed"][0] * (8 * np.sin(th) - np.sin(2 * th)) / (6 * dx)
              - eps / dx * np.sin(th / 2) ** 6)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    exp = np.fft.irfft(np.fft.rfft(u0[0, 0]) * R ** steps, n)
    assert np.max(np.abs(u[0, 0] - exp)) < 1e-12
    assert np.array_equal(u, np.broadcast_to(u[0, 0], u.shape))   # the slab stays a slab


@pytest.mark.slow
def test_app_c_energy_and_high_frequency_noise():
    """Without dissipation the energy (sum of u^2) changes by the O(0.1-0.3) %
    App. C prints for the static grids; eps = 1e-2 lowers the high-frequency
    content at every resolution and keeps the energy change below twice the
    undamped one; eps = 1 removes the high frequencies almost entirely and
    leaks visibly more energy."""
    a = _app_c()
    lo, hi = a["energy_change_static_no_dissipation_percent"]
    for n in (64, 128, 256):
        res = {}
        for eps in (0.0, a["eps_small"], a["eps_large"]):
            u0, u, _, _ = ko.app_c_advection(n, eps, p=a["dissipation_order_p"], c=tuple(a["wave_speed"]),
                                             box_side=a["box_side"], t_end=a["t_end"],
                                             dt_over_dx=a["dt_over_dx"])
            dE = abs(float(np.sum(u * u) - np.sum(u0 * u0))) / float(np.sum(u0 * u0))
            res[eps] = (dE, _upper_half_power(u))
        dE0, hf0 = res[0.0]
        dEs, hfs = res[a["eps_small"]]
        dEl, hfl = res[a["eps_large"]]
        assert lo / 100 <= dE0 <= 1.2 * hi / 100, (n, dE0)
        assert hfs < 0.75 * hf0, (n, hfs, hf0)
        assert dEs < 2.0 * dE0, (n, dEs, dE0)
        assert hfl < 1e-4 * hf0 and dEl > 2.5 * dE0, (n, hfl, dEl)
