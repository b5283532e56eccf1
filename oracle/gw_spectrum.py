"""Gravitational-wave spectrum of the coarse level (Sec. 7.4, Eq. gw_spectrum,
with the projector of Sec. 5, Eq. Lambda_ijlm).  Test infrastructure:
imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline.

Unbinned spectrum of the auxiliary-field velocities v_ij = u_ij':

    G(n^2) = N^-6 sum_{k : |n(k)|^2 = n^2} Lambda_ij,lm(k) v~_ij(k) v~*_lm(k)

with v~ the unnormalised discrete Fourier transform over the N^3 coarse
cells, n(k) the signed integer frequency vector, summation over repeated
indices i, j, l, m in {x, y, z} (v symmetric), and

    Lambda_ij,lm = P_il P_jm - P_ij P_lm / 2,   P_ij = delta_ij - khat_i khat_j,

khat the unit vector of the effective lattice momentum k_eff, per axis the
symbol of the central first difference the source uses: projection type 1
(second order) k_eff = sin(theta)/dx, type 2 (fourth order) k_eff =
(8 sin(theta) - sin(2 theta))/(6 dx), theta = 2 pi n/N.  Where k_eff = 0
(the zero mode, and for type 1 the Nyquist planes) khat = 0, so P = delta.

Parity: pinned (the projector's algebra; a transverse-traceless plane wave
gives the closed-form bin value and nothing elsewhere; longitudinal and pure
trace waves give zero; the sum over bins is bounded by the field's mean
square, with equality for transverse-traceless fields) --
tests/test_oracle_gw_spectrum.py.
"""
from __future__ import annotations

import numpy as np

# storage order of the six components and their (i, j)
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def k_eff_1d(n: int, dx: float, ptype: int) -> np.ndarray:
    """k_eff of the FFT indexes 0..n-1 along one axis."""
    th = 2.0 * np.pi * np.arange(n) / n
    if ptype == 1:
        return np.sin(th) / dx
    if ptype == 2:
        return (8.0 * np.sin(th) - np.sin(2.0 * th)) / (6.0 * dx)
    raise ValueError("projection type must be 1 or 2")


def lambda_tensor(khat) -> np.ndarray:
    """Lambda_ij,lm (shape (..., 3, 3, 3, 3)) for unit (or zero) vectors khat (..., 3)."""
    khat = np.asarray(khat, dtype=np.float64)
    P = np.eye(3) - khat[..., :, None] * khat[..., None, :]
    return (np.einsum("...il,...jm->...ijlm", P, P) - 0.5 * np.einsum("...ij,...lm->...ijlm", P, P))


def spectrum(v6, dx: float, ptype: int):
    """(n2, G): the integer |n|^2 values that occur on the lattice (sorted)
    and the spectrum there.  v6: the six v_ij fields, each [z, y, x] of N^3."""
    v6 = [np.asarray(a, dtype=np.float64) for a in v6]
    n = v6[0].shape[0]
    vt = [np.fft.fftn(a) for a in v6]               # axes (z, y, x)
    V = np.empty((n, n, n, 3, 3), dtype=np.complex128)
    for c, (i, j) in enumerate(PAIRS):
        V[..., i, j] = vt[c]
        V[..., j, i] = vt[c]
    ke = k_eff_1d(n, dx, ptype)
    kz, ky, kx = np.meshgrid(ke, ke, ke, indexing="ij")
    kvec = np.stack([kx, ky, kz], axis=-1)          # (x, y, z) components
    norm = np.linalg.norm(kvec, axis=-1)
    khat = np.where(norm[..., None] > 0, kvec / np.where(norm > 0, norm, 1.0)[..., None], 0.0)
    lam = lambda_tensor(khat)
    val = np.einsum("...ijlm,...ij,...lm->...", lam, V, np.conj(V)).real
    sidx = np.arange(n)
    sidx = np.where(sidx <= n // 2, sidx, sidx - n)
    nz, ny, nx = np.meshgrid(sidx, sidx, sidx, indexing="ij")
    n2 = (nx * nx + ny * ny + nz * nz).ravel()
    tot = np.bincount(n2, weights=val.ravel())
    cnt = np.bincount(n2)
    keep = np.nonzero(cnt)[0]
    return keep.astype(np.int64), tot[keep] / float(n) ** 6
