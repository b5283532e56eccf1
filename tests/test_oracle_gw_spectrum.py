"""Pins of the oracle's gravitational-wave spectrum (oracle/gw_spectrum.py)."""
import numpy as np
import pytest

from oracle import gw_spectrum as gs


def test_projector_algebra():
    rng = np.random.default_rng(0)
    k = rng.standard_normal((20, 3))
    khat = k / np.linalg.norm(k, axis=1, keepdims=True)
    L = gs.lambda_tensor(khat)
    assert np.allclose(L, np.transpose(L, (0, 3, 4, 1, 2)))                    # (ij) <-> (lm)
    M = rng.standard_normal((20, 3, 3))
    M = M + np.swapaxes(M, 1, 2)
    LM = np.einsum("nijlm,nlm->nij", L, M)                                     # acting on symmetric M
    assert np.allclose(LM, np.swapaxes(LM, 1, 2), atol=1e-14)
    assert np.allclose(np.einsum("nijlm,nlm->nij", L, LM), LM, atol=1e-14)
    assert np.allclose(np.einsum("ni,nijlm->njlm", khat, L), 0, atol=1e-14)    # transverse
    assert np.allclose(np.einsum("niilm->nlm", L), 0, atol=1e-14)              # traceless
    assert np.allclose(np.einsum("nijab,nablm->nijlm", L, L), L, atol=1e-14)   # idempotent


def _field(n, m, e):
    """v_ij = e_ij cos(2 pi m.x / n) on the [z, y, x] lattice, six components."""
    ax = np.arange(n)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    c = np.cos(2 * np.pi * (m[0] * X + m[1] * Y + m[2] * Z) / n)
    return [e[i, j] * c for i, j in gs.PAIRS]


@pytest.mark.parametrize("ptype", [1, 2])
def test_tt_plane_wave_closed_form(ptype):
    """Along x the effective momentum is along x for both types: e with only
    yy = -zz and yz entries is transverse-traceless, both +-m modes carry
    |v~|^2 = (N^3/2)^2 e:e and G(m^2) = e:e / 2."""
    n, dx = 16, 0.7
    e = np.zeros((3, 3))
    e[1, 1], e[2, 2], e[1, 2], e[2, 1] = 0.3, -0.3, 0.2, 0.2
    n2, G = gs.spectrum(_field(n, (3, 0, 0), e), dx, ptype)
    ee = float(np.sum(e * e))
    assert np.isclose(G[n2 == 9][0], 0.5 * ee, rtol=1e-13)
    assert np.max(np.abs(G[n2 != 9])) < 1e-26


@pytest.mark.parametrize("ptype", [1, 2])
def test_longitudinal_and_trace_waves_project_to_zero(ptype):
    n, dx = 16, 0.5
    m = (2, 1, -3)
    kh = gs.k_eff_1d(n, dx, ptype)[[m[0] % n, m[1] % n, m[2] % n]]
    kh = kh / np.linalg.norm(kh)
    for e in (np.outer(kh, kh), np.eye(3)):
        _, G = gs.spectrum(_field(n, m, e), dx, ptype)
        assert np.max(np.abs(G)) < 1e-15          # against O(0.1) for a TT wave of the same amplitude


def test_spectrum_bounded_by_mean_square():
    """Lambda is an orthogonal projector on symmetric tensors, so the sum of
    the spectrum is at most the Frobenius mean square (Parseval); the
    transverse-traceless plane wave above meets it with equality (e:e / 2)."""
    n, dx = 12, 0.5
    rng = np.random.default_rng(1)
    v = [rng.standard_normal((n, n, n)) for _ in range(6)]
    n2, G = gs.spectrum(v, dx, 2)
    ms = sum((1.0 if i == j else 2.0) * np.sum(v[c] ** 2) for c, (i, j) in enumerate(gs.PAIRS)) / n ** 3
    assert 0 < G.sum() < ms
    assert np.all(G >= -1e-12)
    assert len(n2) == len(set(n2.tolist())) and n2[0] == 0
