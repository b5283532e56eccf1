"""The App. B plane-wave validation on the oracle, shared by the integrator
pins: setup and printed slopes from tests/golden/app_b_plane_wave.json."""
from math import gcd

import numpy as np

from oracle import energy
from oracle.eom import EOMParams
from paper_2404_02950_gb300 import inputs
from tests.helpers import golden

APP_B = golden("app_b_plane_wave.json")


def energy_errors(step, Ns):
    """Energy error of the App. B run against E_exact for each N, and the
    part of it the Laplacian alone makes (the semi-discrete system conserves
    the lattice energy, so that part is the initial state's lattice energy
    minus E_exact).  The wave sees only its phase increment per cell along
    each axis, so the one-step map of the N^3 run is built on the smallest
    periodic lattice with the same increments (N / gcd(N, m_d) cells along
    axis d, m the whole wavelengths per box side); the evolution over the
    printed number of periods is that map's power."""
    wv = APP_B["wave"]
    m, w = wv["wavelengths_xyz"], wv["omega"]
    k = inputs.plane_wave_vector()
    dE, dE_space = [], []
    for n in Ns:
        dx = wv["box_side"] / n
        shp = tuple(n // gcd(n, md) for md in m)
        Z, Y, X = np.meshgrid(*(np.arange(c) * dx for c in shp[::-1]), indexing="ij")
        ph = k[0] * X + k[1] * Y + k[2] * Z
        cs, sn = np.cos(ph), np.sin(ph)
        nc, ns = np.sum(cs * cs), np.sum(sn * sn)
        p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=APP_B["laplacian_order"])
        dt = APP_B["dt_over_dx"] * dx
        zero = np.zeros_like(cs)
        Mx = np.zeros((4, 4))
        for j, (u0, v0) in enumerate([(cs, zero), (sn, zero), (zero, cs), (zero, sn)]):
            y = step((u0, zero, v0, zero), 1.0, dt, dx, p)
            for r, f in enumerate((y[0], y[2])):
                a, b = np.sum(f * cs) / nc, np.sum(f * sn) / ns
                Mx[2 * r, j], Mx[2 * r + 1, j] = a, b
                assert np.max(np.abs(f - a * cs - b * sn)) < 1e-12
        nsteps = int(round(APP_B["periods"] * 2 * np.pi / w / dt))
        s = np.linalg.matrix_power(Mx, nsteps) @ np.array([1.0, 0.0, 0.0, -w])
        uu, vv = s[0] * cs + s[1] * sn, s[2] * cs + s[3] * sn
        vol = cs.size * dx ** 3
        dE.append(energy.energy_periodic((uu, zero, vv, zero), 1.0, dx, p)[3] / vol - APP_B["E_exact"])
        dE_space.append(energy.energy_periodic((cs, zero, -w * sn, zero), 1.0, dx, p)[3] / vol - APP_B["E_exact"])
    return np.array(dE), np.array(dE_space)


def slope(Ns, dE):
    """Fitted power-law index of |dE| against N."""
    return np.polyfit(np.log(Ns), np.log(np.abs(dE)), 1)[0]
