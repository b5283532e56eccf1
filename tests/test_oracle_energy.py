"""Pins of the oracle's energy reduction: closed forms on a lattice plane
wave and a homogeneous field, the force of the equations of motion being
minus the gradient of the energy (so the flat friction-free flow conserves
it), and the loop's string length."""
import numpy as np

from oracle import energy, eom, rk4
from oracle.eom import EOMParams
from paper_2404_02950_gb300 import inputs


def test_plane_wave_kinetic_and_gradient_closed_form():
    n, dx, order = 12, 0.4, 4
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    th = 2 * np.pi * np.array([2, -1, 3]) / n
    ph = th[0] * X + th[1] * Y + th[2] * Z
    lam = sum(2.5 - (8 / 3) * np.cos(t) + (1 / 6) * np.cos(2 * t) for t in th) / dx ** 2
    w = 1.7
    y = (np.cos(ph), np.zeros_like(ph), -w * np.sin(ph), np.zeros_like(ph))
    p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=order)
    E = energy.energy_periodic(y, 1.0, dx, p)
    vol = n ** 3 * dx ** 3
    assert abs(E[0] - 0.5 * w * w * 0.5 * vol) < 1e-12 * vol
    assert abs(E[1] - 0.5 * lam * 0.5 * vol) < 1e-12 * vol * lam
    assert E[2] == 0.0 and E[4] == 0.0


def test_homogeneous_potential_closed_form():
    y = tuple(np.full((4, 4, 4), v) for v in (0.6, 0.3, 0.0, 0.0))
    p = EOMParams(lam=1.5, a=0.2, friction=True, eta_power=2, order=2)
    eta, dx = 2.0, 0.5
    E = energy.energy_periodic(y, eta, dx, p)
    r2 = 0.45
    exp = 64 * dx ** 3 * ((1.5 * 4.0 / 4) * (r2 - 1) ** 2 + 0.1 * r2)
    assert abs(E[2] - exp) < 1e-13 and E[0] == 0.0 and E[1] == 0.0


def test_rhs_force_is_minus_energy_gradient():
    """d/de E(y + e f(y)) = 0 at e = 0 for the frozen friction-free flow
    (central difference), while a perturbed potential factor breaks it."""
    n, dx = 6, 0.7
    rng = np.random.default_rng(2)
    y = tuple(0.6 * rng.standard_normal((n, n, n)) for _ in range(4))
    p = EOMParams(lam=1.3, a=0.4, friction=False, eta_power=0, order=6)
    f = rk4.f_periodic(y, 1.0, dx, p)
    eps = 1e-5

    def E_at(e):
        return energy.energy_periodic(tuple(a + e * b for a, b in zip(y, f)), 1.0, dx, p)[3]

    deriv = (E_at(eps) - E_at(-eps)) / (2 * eps)
    scale = sum(np.sum(b * b) for b in f) * dx ** 3
    assert abs(deriv) < 1e-7 * scale
    # sanity: with friction on, energy decreases at rate 2/eta * sum Pi^2
    pf = EOMParams(lam=1.3, a=0.4, friction=True, eta_power=0, order=6)
    ff = rk4.f_periodic(y, 1.0, dx, pf)

    def Ef(e):
        return energy.energy_periodic(tuple(a + e * b for a, b in zip(y, ff)), 1.0, dx, pf)[3]

    d2 = (Ef(eps) - Ef(-eps)) / (2 * eps)
    exp = -2.0 * (np.sum(y[2] ** 2) + np.sum(y[3] ** 2)) * dx ** 3
    assert abs(d2 - exp) < 1e-6 * abs(exp)


def test_loop_string_length():
    n, R, dx = 40, 11.0, 0.5
    y = inputs.string_loop(n, R, 1.0, dx)
    E = energy.energy_periodic(y, 1.0, dx, EOMParams())
    cx = n / 2.0 - 0.5 + 0.25
    cy = n / 2.0 - 0.5 + 0.125
    cnt = 2 * sum(1 for i in range(n) if abs(i - cx) < R) + 2 * sum(1 for j in range(n) if abs(j - cy) < R)
    assert E[4] == cnt * dx
