"""Right-hand side of the axion-string system (Sec. 3.1).

The second-order equation of Sec. 3.1 for psi_i (i = 1, 2),

    psi_i'' + (2/eta) psi_i' - lap psi_i + eta^2 psi_i (psi1^2 + psi2^2 - 1)
        + a psi_i = 0,

is split (Eqs. EOM1, EOM2) into

    psi_i' = Pi_i,
    Pi_i'  = -(2/eta) Pi_i + lap psi_i - psi_i * pot,
    pot    = lambda eta^p (psi1^2 + psi2^2 - 1) + a.

The paper's form is lambda = 1, p = 2.  Its ``Rhs`` listing declares the
constant ``a`` as an ``int`` initialised from 0.56233, so a = 0 there; ``a``
is kept as a parameter.  ``friction = False`` drops the 2/eta term and
``eta_power = 0`` freezes the potential coefficient (flat, friction-free
limit used by the energy-conservation pin).

Evaluation order (fixed, no fused multiply-add):
    r2  = psi1*psi1 + psi2*psi2
    pot = c_pot*(r2 - 1) + a             with c_pot = lambda * eta^p
    dPi = (-c_fric)*Pi + lap - psi*pot   with c_fric = 2/eta (or 0)

Parity: pinned through the RK4 pins (closed-form amplification, energy
conservation order) in tests/test_oracle_rk4.py.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class EOMParams:
    lam: float = 1.0
    a: float = 0.0
    friction: bool = True
    eta_power: int = 2
    order: int = 2          # Laplacian accuracy order: 2, 4 or 6
    ko_order: int = 0       # Kreiss-Oliger dissipation order p (odd; 0: off), oracle/ko.py
    ko_eps: float = 0.0     # its strength


def coefficients(eta: float, p: EOMParams):
    """(c_fric, c_pot) at conformal time ``eta``, in FP64."""
    c_fric = 2.0 / eta if p.friction else 0.0
    if p.eta_power == 2:
        c_pot = p.lam * (eta * eta)
    elif p.eta_power == 0:
        c_pot = p.lam
    else:
        raise ValueError("eta_power must be 0 or 2")
    return c_fric, c_pot


def rhs(psi1, psi2, pi1, pi2, lap1, lap2, eta: float, p: EOMParams):
    """Time derivatives (dpsi1, dpsi2, dpi1, dpi2) cell by cell."""
    c_fric, c_pot = coefficients(eta, p)
    r2 = psi1 * psi1 + psi2 * psi2
    pot = c_pot * (r2 - 1.0) + p.a
    dpi1 = (-c_fric) * pi1 + lap1 - psi1 * pot
    dpi2 = (-c_fric) * pi2 + lap2 - psi2 * pot
    return pi1.copy(), pi2.copy(), dpi1, dpi2
