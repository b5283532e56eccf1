"""Gravitational-wave tensor on the GPU vs the oracle (Sec. 5, oracle/gw.py):
the 16-field classic RK4 step on a periodic level (FP64 within 1e-12 relative
L2 per field after 5 steps for Laplacian orders 2/4/6; FP32 + Kahan within
1e-4), the 16-field hierarchy (ghost fill of psi and u by copy and
prolongation, restriction and regrid of every field), and the spectrum of
Sec. 7.4 (oracle/gw_spectrum.py)."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import gw as ogw
from oracle import gw_spectrum as ogs
from oracle import ssprk3 as ossp
from paper_2404_02950_gb300 import inputs
from tests.helpers import oparams, rel_l2

pytestmark = pytest.mark.gpu

N, DX, DT, ETA0, G, BF = 32, 0.5, 0.125, 1.0, 3, 8
FULL = [((0, 0, 0), (N - 1, N - 1, N - 1))]


def _initial(n=N, dx=DX):
    """String loop in psi (a source with strong gradients) plus smooth random
    u_ij, v_ij of amplitude ~0.1."""
    p1, p2, z, _ = inputs.string_loop(n, 4.0 * (n / N), 2.0, dx)
    tens = []
    for s in range(6):
        a, b, _, _ = inputs.gaussian_field(n, 3.0, 100 + s)
        tens += [0.1 * a, 0.1 * b]
    u = tens[0::2]
    v = tens[1::2]
    return [p1, p2, z, z.copy()] + u + v


def _gpu(y, p, prec, nsteps):
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec=prec, max_levels=1, gw=True)
    h.init_level(0, FULL)
    h.set_state(0, slh.dense_from_boxes(y, FULL))
    h.set_eta(ETA0)
    for _ in range(nsteps):
        h.rk_step(0, DT, p)
    return slh.boxes_from_dense(h.get_state(0), FULL, 16)[0]


def _oracle(y, p, nsteps):
    y = tuple(np.asarray(a, dtype=np.float64) for a in y)
    eta = ETA0
    for _ in range(nsteps):
        y = ogw.rk4_step_periodic(y, eta, DT, DX, oparams(p))
        eta += DT
    return y


@pytest.mark.parametrize("order", [2, 4, 6])
def test_uniform_f64_matches_oracle(order):
    p = slh.EOMParams(order=order)
    y = _initial()
    exp = _oracle(y, p, 5)
    got = _gpu(y, p, "f64", 5)
    for c in range(16):
        e = rel_l2(got[c], exp[c])
        assert e <= 1e-12, (order, c, e)
    # the source moved u away from its initial value
    assert rel_l2(exp[4], y[4]) > 1e-3


@pytest.mark.parametrize("order,integrator", [(2, 4), (4, 4), (6, 4), (2, 10), (4, 10)])
def test_uniform_f32_within_bound(order, integrator):
    """FP32 (Kahan at RK4's last stage) for every Laplacian order and both
    integrators: orders 2 and 4 run the TMA-fed GW kernel, order 6 the
    column kernel."""
    p = slh.EOMParams(order=order, integrator=integrator)
    y = _initial()
    if integrator == 4:
        exp = _oracle(y, p, 5)
    else:
        exp, eta = tuple(np.asarray(a, dtype=np.float64) for a in y), ETA0
        for _ in range(5):
            exp = ossp.ssprk3_step_periodic(exp, eta, DT, DX, oparams(p), f=ogw.f_periodic)
            eta += DT
    got = _gpu([a.astype(np.float32) for a in y], p, "f32", 5)
    for c in range(16):
        e = rel_l2(got[c].astype(np.float64), exp[c])
        assert e <= 1e-4, (order, integrator, c, e)


def test_no_source_without_gradients_and_free_mode():
    """Homogeneous psi: no source; u_xy a lattice mode evolves by the closed
    form of the free RK4 step (the oracle's pin, here on the GPU)."""
    p = slh.EOMParams(order=4, friction=False, eta_power=0)
    one = np.ones((N, N, N))
    ax = np.arange(N)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    th = 2 * np.pi * np.array([1, 2, -1]) / N
    ph = th[0] * X + th[1] * Y + th[2] * Z
    y = [0.6 * one, 0.3 * one, 0 * one, 0 * one] + [0 * one] * 12
    y[4 + 3] = np.cos(ph)
    got = _gpu(y, p, "f64", 4)
    lam = sum(2.5 - (8.0 / 3.0) * np.cos(t) + (1.0 / 6.0) * np.cos(2 * t) for t in th) / DX ** 2
    M = np.array([[0.0, 1.0], [-lam, 0.0]]) * DT
    R = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    A, B = np.linalg.matrix_power(R, 4) @ np.array([1.0, 0.0])
    assert np.max(np.abs(got[4 + 3] - A * np.cos(ph))) < 1e-12
    assert np.max(np.abs(got[10 + 3] - B * np.cos(ph))) < 1e-12 * max(1.0, lam)
    for k in (0, 1, 2, 4, 5):
        assert np.max(np.abs(got[4 + k])) == 0.0 and np.max(np.abs(got[10 + k])) == 0.0


# ---------------------------------------------------------------------------
# hierarchy

N0 = 32
LEVEL_BOXES = [
    [((0, 0, 0), (31, 31, 31))],
    [((16, 16, 16), (31, 47, 47)), ((32, 16, 16), (47, 47, 47))],
]


def _dense16(level):
    parts = []
    for b in range(len(level.boxes)):
        v = level.data[b][level.valid(b)]
        for c in range(16):
            parts.append(v[c].ravel())
    return np.concatenate(parts)


def _compare(h, oh, tol):
    for l, L in enumerate(oh.levels):
        got = slh.boxes_from_dense(h.get_state(l), L.boxes, 16)
        for b in range(len(L.boxes)):
            exp = L.data[b][L.valid(b)]
            for c in range(16):
                e = rel_l2(got[b][c], exp[c])
                assert e <= tol, (l, b, c, e)


def test_hierarchy_subcycled_step_and_regrid_match_oracle():
    p = slh.EOMParams(order=4, interp_type=4)
    oh = oamr.make_hierarchy(N0, DX, DT, G, BF, LEVEL_BOXES, oparams(p), interp_type=4, eta0=ETA0, gw=True)
    oh.levels[0].set_dense(_initial())
    oamr.prolong_level_from_coarse(oh.levels[1], oh.levels[0], 4)
    oh.levels[0].old = None
    h = slh.Hierarchy(N0, DX, nghost=G, bf=BF, prec="f64", max_levels=2, gw=True)
    for l in range(2):
        h.init_level(l, LEVEL_BOXES[l])
        h.set_state(l, _dense16(oh.levels[l]))
    h.set_eta(ETA0)
    oh.step()
    h.advance(DT, p)
    _compare(h, oh, 1e-12)
    # regrid level 1: copy where the old boxes cover, prolong every field elsewhere
    new = [((16, 16, 24), (47, 47, 55))]
    oamr.regrid_level(oh, 1, new)
    h.regrid_level(1, new)
    _compare(h, oh, 1e-12)
    oh.step()
    h.advance(DT, p)
    _compare(h, oh, 1e-12)


# ---------------------------------------------------------------------------
# spectrum (Sec. 7.4)


@pytest.mark.parametrize("ptype", [1, 2])
@pytest.mark.parametrize("boxes", [FULL, [((0, 0, 0), (15, 31, 31)), ((16, 0, 0), (31, 31, 31))]])
def test_spectrum_matches_oracle_f64(ptype, boxes):
    y = _initial()
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f64", max_levels=1, gw=True)
    h.init_level(0, boxes)
    h.set_state(0, slh.dense_from_boxes(y, boxes))
    n2, g = h.gw_spectrum(ptype)
    en2, eg = ogs.spectrum(y[10:16], DX, ptype)
    assert np.array_equal(n2, en2)
    assert np.max(np.abs(g - eg)) <= 1e-12 * np.max(np.abs(eg))


def test_spectrum_f32_and_tt_wave():
    """FP32 storage: within 1e-5 of the FP64 oracle's largest bin; a
    transverse-traceless wave lands in its own bin with G = e:e / 2."""
    y = _initial()
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f32", max_levels=1, gw=True)
    h.init_level(0, FULL)
    h.set_state(0, slh.dense_from_boxes([a.astype(np.float32) for a in y], FULL))
    n2, g = h.gw_spectrum(2)
    en2, eg = ogs.spectrum(y[10:16], DX, 2)
    assert np.array_equal(n2, en2) and np.max(np.abs(g - eg)) <= 1e-5 * np.max(np.abs(eg))
    ax = np.arange(N)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    c = np.cos(2 * np.pi * 3 * X / N)
    e = {(1, 1): 0.3, (2, 2): -0.3, (1, 2): 0.2}
    v = [e.get((i, j), 0.0) * c for i, j in ogs.PAIRS]
    z = np.zeros_like(c)
    h2 = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f64", max_levels=1, gw=True)
    h2.init_level(0, FULL)
    h2.set_state(0, slh.dense_from_boxes([z, z, z, z] + [z] * 6 + v, FULL))
    n2, g = h2.gw_spectrum(2)
    assert np.isclose(g[n2 == 9][0], 0.5 * (0.09 + 0.09 + 2 * 0.04), rtol=1e-12)
    assert np.max(np.abs(g[n2 != 9])) < 1e-15


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spectrum_is_bit_reproducible(prec):
    """The bins are summed in a fixed order (no atomics): two calls on the
    same state agree bit for bit."""
    y = _initial()
    if prec == "f32":
        y = [a.astype(np.float32) for a in y]
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec=prec, max_levels=1, gw=True)
    h.init_level(0, FULL)
    h.set_state(0, slh.dense_from_boxes(y, FULL))
    runs = [h.gw_spectrum(ptype) for ptype in (2, 2, 1, 1)]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[2][0], runs[3][0]) and np.array_equal(runs[2][1], runs[3][1])
    h.close()


def test_spectrum_needs_tensor_fields():
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f64", max_levels=1)
    h.init_level(0, FULL)
    with pytest.raises(slh.SlhError) as e:
        h.gw_spectrum(2)
    assert e.value.code == -7


def test_f32_graph_replay_matches_direct_steps():
    """The TMA-fed GW kernel inside the captured coarse-step graph (tensor
    maps prepared before capture) gives the direct launches' result bit for
    bit."""
    p = slh.EOMParams(order=4)
    y = [a.astype(np.float32) for a in _initial()]
    outs = []
    for use_graph in (False, True):
        h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f32", max_levels=1, gw=True)
        h.init_level(0, FULL)
        h.set_state(0, slh.dense_from_boxes(y, FULL))
        h.set_eta(ETA0)
        for _ in range(3):
            if use_graph:
                h.advance(DT, p)
            else:
                h.rk_step(0, DT, p)
        outs.append(h.get_state(0))
        h.close()
    assert np.array_equal(outs[0], outs[1])
