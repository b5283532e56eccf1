"""Finite-difference operators of App. A ("Utility Functions").

The paper names the operators by the number of ghost cells they need:
Laplacian order 1/2/3 is the 7/13/19-point stencil; gradient order 1/2/3 the
3/5/7-point stencil.  It prints no coefficients.  Reading: the standard
central-difference weights of accuracy O(dx^2), O(dx^4), O(dx^6), i.e. the
unique symmetric stencils of that width that are exact on polynomials of the
highest possible degree.  Here ``order`` means the accuracy order (2, 4, 6);
the half width is order/2 (= the paper's ``order``).

Parity: pinned (exact discrete dispersion relation per order, polynomial
exactness, dense-matrix brute force on 8^3 -- tests/test_oracle_stencil.py).
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

# Second-derivative weights w_m for m = -h..h (h = order/2), unit spacing.
LAPLACIAN_WEIGHTS = {
    2: (Fr(1), Fr(-2), Fr(1)),
    4: (Fr(-1, 12), Fr(4, 3), Fr(-5, 2), Fr(4, 3), Fr(-1, 12)),
    6: (Fr(1, 90), Fr(-3, 20), Fr(3, 2), Fr(-49, 18), Fr(3, 2), Fr(-3, 20),
        Fr(1, 90)),
}

# First-derivative weights for m = -h..h.
GRADIENT_WEIGHTS = {
    2: (Fr(-1, 2), Fr(0), Fr(1, 2)),
    4: (Fr(1, 12), Fr(-2, 3), Fr(0), Fr(2, 3), Fr(-1, 12)),
    6: (Fr(-1, 60), Fr(3, 20), Fr(-3, 4), Fr(0), Fr(3, 4), Fr(-3, 20),
        Fr(1, 60)),
}

# numpy axis of each spatial direction for [z, y, x] arrays
AXIS = {"x": 2, "y": 1, "z": 0}


def half_width(order: int) -> int:
    if order not in LAPLACIAN_WEIGHTS:
        raise ValueError(f"Laplacian order must be 2, 4 or 6, got {order}")
    return order // 2


def laplacian_periodic(f: np.ndarray, dx: float, order: int) -> np.ndarray:
    """sum_d sum_m w_m f(x + m e_d) / dx^2 on a periodic [z, y, x] lattice."""
    h = half_width(order)
    w = LAPLACIAN_WEIGHTS[order]
    out = np.zeros_like(f)
    for axis in (2, 1, 0):
        acc = np.zeros_like(f)
        for m in range(-h, h + 1):
            acc = acc + float(w[m + h]) * np.roll(f, -m, axis=axis)
        out = out + acc
    return out * (1.0 / (dx * dx))


def laplacian_padded(fp: np.ndarray, g: int, dx: float, order: int) -> np.ndarray:
    """The same operator on a ghost-padded [z, y, x] array with ``g`` ghost
    layers on every side; returns the valid (unpadded) region."""
    h = half_width(order)
    if g < h:
        raise ValueError("ghost width smaller than stencil half width")
    w = LAPLACIAN_WEIGHTS[order]
    nz, ny, nx = (s - 2 * g for s in fp.shape)

    def sl(dz, dy, dx_):
        return fp[g + dz:g + dz + nz, g + dy:g + dy + ny, g + dx_:g + dx_ + nx]

    out = np.zeros((nz, ny, nx))
    for d in ("x", "y", "z"):
        acc = np.zeros((nz, ny, nx))
        for m in range(-h, h + 1):
            off = {"x": (0, 0, m), "y": (0, m, 0), "z": (m, 0, 0)}[d]
            acc = acc + float(w[m + h]) * sl(*off)
        out = out + acc
    return out * (1.0 / (dx * dx))


def gradient_periodic(f: np.ndarray, dx: float, order: int, direction: str) -> np.ndarray:
    """Central first derivative along ``direction`` ('x', 'y' or 'z')."""
    h = order // 2
    w = GRADIENT_WEIGHTS[order]
    axis = AXIS[direction]
    acc = np.zeros_like(f)
    for m in range(-h, h + 1):
        if w[m + h] != 0:
            acc = acc + float(w[m + h]) * np.roll(f, -m, axis=axis)
    return acc * (1.0 / dx)


def gradient_padded(fp: np.ndarray, g: int, dx: float, order: int, direction: str) -> np.ndarray:
    h = order // 2
    w = GRADIENT_WEIGHTS[order]
    nz, ny, nx = (s - 2 * g for s in fp.shape)
    acc = np.zeros((nz, ny, nx))
    for m in range(-h, h + 1):
        if w[m + h] == 0:
            continue
        dz, dy, dxx = {"x": (0, 0, m), "y": (0, m, 0), "z": (m, 0, 0)}[direction]
        acc = acc + float(w[m + h]) * fp[g + dz:g + dz + nz, g + dy:g + dy + ny,
                                          g + dxx:g + dxx + nx]
    return acc * (1.0 / dx)
