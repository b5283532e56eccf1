"""Pins of the oracle's truncation-error estimate (Sec. 2.2, oracle/tee.py)."""
import numpy as np
import pytest

from oracle import amr as oamr
from oracle import tee
from oracle.eom import EOMParams
from oracle.rk4 import rk4_step_periodic


def test_stationary_state_has_zero_tee():
    """psi = (0, -1) on the vacuum circle (|psi|^2 = 1 exactly), Pi = 0: every
    RHS term vanishes at any resolution (the Laplacian of a constant up to the
    rounding of its weights), so both estimates are zero to rounding."""
    n, dx, dt = 16, 0.5, 0.125
    one = np.ones((n, n, n))
    y0 = [0 * one, -one, 0 * one, 0 * one]
    p = EOMParams(lam=1.0, a=0.0, friction=True, eta_power=2, order=4)
    y2 = rk4_step_periodic(rk4_step_periodic(y0, 1.0, dt, dx, p), 1.0 + dt, dt, dx, p)
    tags, te = tee.shadow_tags(y0, 1.0, dt, dx, p, y2, [1e-13] * 4)
    assert np.max(te) < 1e-14 and not tags.any()
    h = oamr.make_hierarchy(8, 2 * dx, 2 * dt, 3, 4, [[((0, 0, 0), (7, 7, 7))], [((0, 0, 0), (15, 15, 15))]],
                            p, eta0=1.0)
    h.levels[0].set_dense(tee.coarsen(y0))
    h.levels[1].set_dense(y0)
    h.te_eps = [1e-13] * 4
    h.step()
    assert not any(t.any() for t in h.te_tags[1])


def _wave(n, L=8.0, m=(1, 0, 0)):
    dx = L / n
    ax = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    k = 2 * np.pi * np.asarray(m) / L
    ph = k[0] * X + k[1] * Y + k[2] * Z
    z = np.zeros_like(ph)
    return [np.cos(ph), 0.5 * np.sin(ph), z, z.copy()], dx


def test_shadow_tee_is_a_fifth_order_local_error():
    """Flat, friction-free, massless limit (the wave equation): the shadow
    estimate of a smooth wave is the difference of two local errors over one
    coarse step, spatial O(dx^4) times a duration O(dt) plus the RK4 local
    error O(dt^5); at fixed dt/dx it falls by about 2^5 per halving of dx."""
    p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=4)
    tes = []
    for n in (16, 32, 64):
        y0, dx = _wave(n, m=(1, 1, 0))
        dt = 0.25 * dx
        y2 = rk4_step_periodic(rk4_step_periodic(y0, 1.0, dt, dx, p), 1.0 + dt, dt, dx, p)
        _, te = tee.shadow_tags(y0, 1.0, dt, dx, p, y2, [1.0] * 4)
        tes.append(np.max(te))
    assert 26.0 < tes[0] / tes[1] < 38.0 and 26.0 < tes[1] / tes[2] < 38.0, tes


def test_self_shadow_equals_shadow_of_a_uniform_fine_run():
    """A two-level hierarchy whose fine level covers the domain, with level 0
    the coarsened fine state: at synchronisation the self-shadow estimate of
    level 1 is the shadow estimate of the uniform fine run."""
    nf, dxf, dtf = 16, 0.5, 0.125
    rng = np.random.default_rng(3)
    base, _ = _wave(nf, L=nf * dxf, m=(1, 2, 0))
    y0 = [b + 0.05 * rng.standard_normal(b.shape) for b in base]
    p = EOMParams(lam=1.0, a=0.0, friction=True, eta_power=2, order=4)
    y2 = rk4_step_periodic(rk4_step_periodic(y0, 1.0, dtf, dxf, p), 1.0 + dtf, dtf, dxf, p)
    tags_s, te_s = tee.shadow_tags(y0, 1.0, dtf, dxf, p, y2, [1.0] * 4)
    eps = [float(np.median(te_s[c])) for c in range(4)]
    tags_s = tee.tags_from_te(te_s, eps)
    h = oamr.make_hierarchy(nf // 2, 2 * dxf, 2 * dtf, 3, 4,
                            [[((0, 0, 0), (nf // 2 - 1,) * 3)], [((0, 0, 0), (nf - 1,) * 3)]], p, eta0=1.0)
    h.levels[0].set_dense(tee.coarsen(y0))
    h.levels[1].set_dense(y0)
    h.te_eps = eps
    h.step()
    assert np.array_equal(h.te_tags[1][0], tags_s)
    assert 0 < tags_s.mean() < 1


def test_threshold_semantics():
    te = np.zeros((4, 2, 2, 2))
    te[2, 1, 0, 1] = 0.5
    te[0, 0, 0, 0] = 0.1
    t = tee.tags_from_te(te, [0.0, 1.0, 0.4, 1.0])   # psi1 ignored (threshold 0), Pi1 above 0.4
    assert t.shape == (4, 4, 4) and t.sum() == 8
    assert t[2:4, 0:2, 2:4].all()
    with pytest.raises(Exception):
        tee.tags_from_te(te[:3], [1.0] * 4)
