"""Truncation-error-estimate (TEE) tagging (Sec. 2.2, "Tagging cells for
refinement").  Test infrastructure: imported only by tests/,
__graft_entry__.smoke() and bench.py's CPU baseline.

The TEE compares one state advanced over the same time span at two
resolutions: Delta phi_cf = |phi_coarse - phi_fine|, taken on the coarse
cells with the fine values averaged over their 2^3 children (the restriction
of Sec. 2.1).  A refined level l >= 1 gets it for free just before it is
synchronised with l-1 (the self-shadow method: l-1 advanced by dt_{l-1}, l by
two steps of dt_l); level 0 needs a shadow level, level 0 coarsened by 2^3
and advanced by one step of 2 dt_0 while level 0 takes two.  Every fine cell
whose parent has f(Delta phi_cf) > eps_phi for some scalar component phi in
(psi1, psi2, Pi1, Pi2) is tagged, with f the identity (the default modifier).
A component whose threshold is not positive takes no part.

Parity: pinned (a stationary state has a TEE of zero up to rounding; on a
smooth wave the shadow TEE, a local error over one coarse step, falls by 2^5
per halving of dx at fixed dt/dx; the shadow TEE of a uniform fine run equals
the self-shadow TEE of a two-level hierarchy whose fine level covers the
domain) -- tests/test_oracle_tee.py.
"""
from __future__ import annotations

import numpy as np

from .eom import EOMParams
from .interp import restrict_block
from .rk4 import rk4_step_periodic

NSCALAR = 4


def te_on_coarse(coarse, fine):
    """Per-component |coarse - restrict(fine)|: coarse (4, nz, ny, nx), fine
    (4, 2nz, 2ny, 2nx); returns (4, nz, ny, nx)."""
    return np.stack([np.abs(np.asarray(coarse[c], dtype=np.float64) - restrict_block(fine[c]))
                     for c in range(NSCALAR)])


def tags_from_te(te, eps):
    """Fine-cell tags (2nz, 2ny, 2nx) uint8 from coarse-cell TEEs (4, nz, ny, nx)."""
    hit = np.zeros(te.shape[1:], dtype=bool)
    for c in range(NSCALAR):
        if eps[c] > 0:
            hit |= te[c] > eps[c]
    return np.repeat(np.repeat(np.repeat(hit, 2, axis=0), 2, axis=1), 2, axis=2).astype(np.uint8)


def coarsen(fields):
    """2^3 restriction of dense periodic fields (each [z, y, x], even extents)."""
    return [restrict_block(f) for f in fields]


def shadow_tags(y_t0, eta0, dt0, dx0, p: EOMParams, y_t2, eps):
    """Level-0 TEE tags from the shadow level: y_t0 the level-0 state at eta0,
    y_t2 the same level after two steps of dt0.  The shadow is coarsen(y_t0)
    advanced one classic RK4 step of 2 dt0 at spacing 2 dx0.  Returns (tags,
    te) with tags on the level-0 cells and te on the shadow cells."""
    sh = rk4_step_periodic(tuple(coarsen(list(y_t0)[:NSCALAR])), eta0, 2.0 * dt0, 2.0 * dx0, p)
    te = te_on_coarse(sh, list(y_t2)[:NSCALAR])
    return tags_from_te(te, eps), te
