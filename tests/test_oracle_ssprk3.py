"""Pins of the oracle's low-storage SSPRK3 step (integrator type 10,
oracle/ssprk3.py) against closed forms, an independent ODE integrator and
the paper's App. B convergence slope for RK3."""
import numpy as np
import pytest

from oracle import ssprk3
from oracle.eom import EOMParams


def _symbol4(theta):
    return 2.5 - (8.0 / 3.0) * np.cos(theta) + (1.0 / 6.0) * np.cos(2 * theta)


def test_linear_mode_closed_form():
    """Flat, massless, friction-free: every lattice Fourier mode is a linear
    oscillator, and any three-stage third-order RK step multiplies it by
    1 + M + M^2/2 + M^3/6."""
    n, dx, dt, nst = 12, 0.5, 0.1, 7
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    th = 2 * np.pi * np.array([2, -1, 3]) / n
    ph = th[0] * X + th[1] * Y + th[2] * Z
    lam = sum(_symbol4(t) for t in th) / dx ** 2
    p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=4)
    z = np.zeros((n, n, n))
    y = (np.cos(ph), 0.3 * np.cos(ph), z, z)
    eta = 1.0
    for _ in range(nst):
        y = ssprk3.ssprk3_step_periodic(y, eta, dt, dx, p)
        eta += dt
    M = np.array([[0.0, 1.0], [-lam, 0.0]]) * dt
    R = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6
    Rn = np.linalg.matrix_power(R, nst)
    for c0, s in ((0, 1.0), (1, 0.3)):
        A, B = Rn @ np.array([s, 0.0])
        assert np.max(np.abs(y[c0] - A * np.cos(ph))) < 1e-12
        assert np.max(np.abs(y[c0 + 2] - B * np.cos(ph))) < 1e-12 * max(1.0, lam)


def test_homogeneous_field_is_third_order_with_stage_times():
    """A spatially constant field obeys the ODE of Sec. 3.1 without the
    Laplacian; with 2/eta and lambda eta^2 at the stage times (0, 1, 1/2) the
    error falls by ~8 per halving of dt."""
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
        y = tuple(np.full((4, 4, 4), v) for v in (psi0[0], psi0[1], pi0[0], pi0[1]))
        eta = eta0
        for _ in range(nst):
            y = ssprk3.ssprk3_step_periodic(y, eta, dt, 0.5, p)
            eta += dt
        errs.append(np.max(np.abs(np.array([y[c][1, 2, 3] for c in range(4)]) - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, errs


@pytest.mark.slow
def test_plane_wave_energy_convergence_app_b():
    """App. B (tests/app_b.py): the third-order scheme's energy error falls
    like N^-3, the paper's printed index for RK3 within 0.3 (fitted where the
    error is not O(1))."""
    from tests import app_b
    Ns = [192, 256, 384]
    dE, _ = app_b.energy_errors(ssprk3.ssprk3_step_periodic, Ns)
    assert np.all(dE < 0) and abs(dE[-1]) < 0.05 * app_b.APP_B["E_exact"]
    sl = app_b.slope(Ns, dE)
    assert abs(sl - app_b.APP_B["slopes"]["RK3"]) < 0.3, (sl, dE)
