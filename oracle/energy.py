"""Energy components and string length of a field state.

The paper measures convergence through the total energy of its validation
wave (App. B, E = udot^2/2 + (grad u)^2/2 averaged over the box) and names no
estimator for the axion system; the reduction used here is the discrete
Hamiltonian of the first-order system of Sec. 3.1 at frozen time:

    e_kin  = 1/2 (Pi1^2 + Pi2^2)
    e_grad = -1/2 (psi1 * L psi1 + psi2 * L psi2)     (L = the FD Laplacian)
    e_pot  = (c_pot / 4) (r2 - 1)^2 + (a / 2) r2,      r2 = psi1^2 + psi2^2

each summed over cells and multiplied by dx^3; on a periodic lattice
-sum psi L psi = sum |grad_h psi|^2 (summation by parts), and d/dpsi of e_pot is
psi * pot of the equations of motion, so with friction off and c_pot frozen the
sum is conserved by the semi-discrete system.  String length = number of
pierced plaquettes * dx (winding module).

Parity: pinned (plane-wave energy against the closed-form symbol, exact
conservation of the semi-discrete energy under the flat friction-free flow) --
tests/test_oracle_rk4.py, tests/test_oracle_energy.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams, coefficients
from .stencil import laplacian_padded, laplacian_periodic
from .winding import pierced_count_padded, plaquette_winding


def densities(psi1, psi2, pi1, pi2, lap1, lap2, eta, p: EOMParams):
    _, c_pot = coefficients(eta, p)
    r2 = psi1 * psi1 + psi2 * psi2
    e_kin = 0.5 * (pi1 * pi1 + pi2 * pi2)
    e_grad = -0.5 * (psi1 * lap1 + psi2 * lap2)
    d = r2 - 1.0
    e_pot = (0.25 * c_pot) * (d * d) + (0.5 * p.a) * r2
    return e_kin, e_grad, e_pot


def energy_periodic(y, eta, dx, p: EOMParams):
    """[kin, grad, pot, total, string_length] of a uniform periodic lattice."""
    psi1, psi2, pi1, pi2 = y
    lap1 = laplacian_periodic(psi1, dx, p.order)
    lap2 = laplacian_periodic(psi2, dx, p.order)
    ek, eg, ep = densities(psi1, psi2, pi1, pi2, lap1, lap2, eta, p)
    vol = dx * dx * dx
    K, G, P = float(ek.sum()) * vol, float(eg.sum()) * vol, float(ep.sum()) * vol
    W = plaquette_winding(psi1, psi2, periodic=True)
    nstr = sum(int(np.count_nonzero(W[w])) for w in W)
    return np.array([K, G, P, K + G + P, nstr * dx])


def energy_box(arr, g, dx, eta, p: EOMParams, uncovered=None):
    """Partial sums over the valid cells of one ghost-padded box ``arr``
    (shape (4, nz+2g, ny+2g, nx+2g)), restricted to ``uncovered`` cells when
    given.  Returns (kin, grad, pot, pierced_plaquettes) without the dx
    factors."""
    psi1p, psi2p = arr[0], arr[1]
    nz, ny, nx = (s - 2 * g for s in psi1p.shape)
    v = (slice(g, g + nz), slice(g, g + ny), slice(g, g + nx))
    lap1 = laplacian_padded(psi1p, g, dx, p.order)
    lap2 = laplacian_padded(psi2p, g, dx, p.order)
    ek, eg, ep = densities(psi1p[v], psi2p[v], arr[2][v], arr[3][v], lap1, lap2, eta, p)
    m = np.ones((nz, ny, nx), dtype=bool) if uncovered is None else uncovered
    n = pierced_count_padded(psi1p, psi2p, g, owner_mask=m)
    return float(ek[m].sum()), float(eg[m].sum()), float(ep[m].sum()), n
