"""Seeded synthetic initial states.

This module only draws random numbers and lays out initial data; it holds none
of the scheme's arithmetic (no stencil, no potential, no integrator).  Both the
CUDA path and the CPU oracle are fed from here, so a parity test hands the two
sides bit-identical FP64 snapshots.

The paper reads its initial state from HDF5 files (Sec. 6) and ships none, so
every workload here is synthetic:

* ``gaussian_field``: each of psi1, psi2 an independent real Gaussian random
  field, flat power for lattice modes |m| <= m_max and zero above (spherical
  cut), normalised so that <psi1^2 + psi2^2> = 1; momenta zero.
* ``string_loop``: one circular axion string of radius R in the plane
  z = N/2, psi = tanh(eta0 d / sqrt 2) e^{i theta} with d the distance to the
  circle and theta the angle around it; momenta zero.
* ``plane_wave``: u = cos(k.x), du/dt = -omega sin(k.x) on an N^3 box of side
  L (the validation wave of App. B).

Arrays are C-ordered ``[z, y, x]`` (x fastest), float64.
"""
from __future__ import annotations

import numpy as np


def _irfftn(a, shape):
    try:
        import scipy.fft as sf  # multithreaded when available
        return sf.irfftn(a, s=shape, workers=-1)
    except Exception:  # pragma: no cover - scipy absent
        return np.fft.irfftn(a, s=shape)


def gaussian_field(n: int, m_max: float, seed: int):
    """Two independent Gaussian random fields on an n^3 periodic lattice.

    Modes with integer wave numbers |m| <= m_max carry independent N(0,1)
    complex amplitudes (Hermitian symmetry is imposed by the inverse real FFT);
    all other modes are zero.  The pair is scaled so that
    mean(psi1^2 + psi2^2) == 1.  With k = 2 pi m / (n dx), a cut at
    k_max = pi / (c dx) is m_max = n / (2 c).

    Returns (psi1, psi2, pi1, pi2) as float64 arrays of shape (n, n, n).
    """
    rng = np.random.default_rng(seed)
    mz = np.fft.fftfreq(n, 1.0 / n)
    mx = np.fft.rfftfreq(n, 1.0 / n)
    m2 = mz[:, None, None] ** 2 + mz[None, :, None] ** 2 + mx[None, None, :] ** 2
    mask = m2 <= m_max * m_max
    fields = []
    for _ in range(2):
        re = rng.standard_normal(mask.shape)
        im = rng.standard_normal(mask.shape)
        spec = np.where(mask, re + 1j * im, 0.0)
        spec[0, 0, 0] = 0.0
        fields.append(_irfftn(spec, (n, n, n)))
    p1, p2 = fields
    norm = np.sqrt(np.mean(p1 * p1 + p2 * p2))
    p1 = np.ascontiguousarray(p1 / norm)
    p2 = np.ascontiguousarray(p2 / norm)
    z = np.zeros_like(p1)
    return p1, p2, z, z.copy()


def _loop_center(n: int):
    return (n / 2.0 - 0.5 + 0.25, n / 2.0 - 0.5 + 0.125, n / 2.0 - 0.5 + 0.0625)


def _loop_fields(i, j, k, radius, eta0, dx, c):
    rho = np.hypot(i - c[0], j - c[1])
    dz = k - c[2]
    dr = rho - radius
    d = np.hypot(dr, dz)
    theta = np.arctan2(dz, dr) - np.arctan2(dz, rho + radius)
    amp = np.tanh(eta0 * d * dx / np.sqrt(2.0))
    p1 = np.ascontiguousarray(amp * np.cos(theta))
    p2 = np.ascontiguousarray(amp * np.sin(theta))
    z = np.zeros_like(p1)
    return p1, p2, z, z.copy()


def string_loop(n: int, radius: float, eta0: float, dx: float, center=None):
    """A circular string loop of ``radius`` lattice cells in the plane z = n/2.

    Cell (i, j, k) sits at (i, j, k) in lattice units.  With rho the distance
    from the loop's axis (parallel to z through ``center``), d = hypot(rho - R,
    z - z_c) is the distance to the core and the phase is
    theta = atan2(z - z_c, rho - R) - atan2(z - z_c, rho + R) (the ring and its
    mirror image across the axis), which winds once around the core and tends
    to zero far from the loop, so the periodic wrap adds no spurious string.
    psi = tanh(eta0 d dx / sqrt 2) e^{i theta}.
    """
    c = _loop_center(n) if center is None else center
    k, j, i = np.meshgrid(np.arange(n, dtype=np.float64),
                          np.arange(n, dtype=np.float64),
                          np.arange(n, dtype=np.float64), indexing="ij")
    return _loop_fields(i, j, k, radius, eta0, dx, c)


def string_loop_boxes(n0: int, level: int, boxes, radius: float, eta0: float, dx0: float):
    """The loop of ``string_loop(n0, radius, eta0, dx0)`` sampled at the cell
    centres of refinement level ``level`` (ratio 2 per level) inside
    ``boxes`` (inclusive (lo, hi) in that level's index space).  A level-l cell
    i sits at (i + 1/2) / 2^l - 1/2 in level-0 lattice units.  Returns one
    (4, nz, ny, nx) float64 array per box."""
    c = _loop_center(n0)
    r = float(1 << level)
    out = []
    for lo, hi in boxes:
        ax = [(np.arange(lo[d], hi[d] + 1, dtype=np.float64) + 0.5) / r - 0.5 for d in range(3)]
        k, j, i = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        out.append(np.stack(_loop_fields(i, j, k, radius, eta0, dx0, c)))
    return out


def plane_wave_vector():
    """Wave vector of the App. B validation wave (read as pi(cos t cos p,
    sin t, -cos t sin p) with tan t = 1/2, sin p = 3/5: |k| = pi and exactly
    8, 5, 6 wavelengths along x, y, z in a box of side 10 sqrt 5)."""
    ct, st = 2.0 / np.sqrt(5.0), 1.0 / np.sqrt(5.0)
    cp, sp = 4.0 / 5.0, 3.0 / 5.0
    return np.pi * np.array([ct * cp, st, -ct * sp])


def plane_wave(n: int, box: float = 10.0 * np.sqrt(5.0), k=None, omega=np.pi):
    """u = cos(k.x) and du/dt = -omega sin(k.x) at t = 0 on cell centres
    x = i * dx, dx = box / n.  Returns (u, udot, dx)."""
    k = plane_wave_vector() if k is None else np.asarray(k, dtype=np.float64)
    dx = box / n
    ax = np.arange(n, dtype=np.float64) * dx
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    ph = k[0] * xx + k[1] * yy + k[2] * zz
    return np.cos(ph), -omega * np.sin(ph), dx


def random_snapshot(n, seed, amp=1.0, shape=None):
    """Uniform random fields in [-amp, amp) for the four components (used for
    brute-force and parity cases where no physical structure is needed)."""
    rng = np.random.default_rng(seed)
    shp = (n, n, n) if shape is None else tuple(shape)
    return tuple(rng.uniform(-amp, amp, size=shp) for _ in range(4))
