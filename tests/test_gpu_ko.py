"""Kreiss-Oliger dissipation on the GPU vs the oracle (Sec. 2.4, oracle/ko.py):
the per-stage dissipation kernel with classic RK4 and with SSPRK3 on a
uniform lattice (FP64 within 1e-12 relative L2; FP32 + Kahan within 1e-4),
and on a subcycled hierarchy, where the momenta's ghosts are prolonged too."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import rk4 as ork4
from oracle import ssprk3 as ossp
from paper_2404_02950_gb300 import inputs
from tests.helpers import download_domain, oparams, rel_l2, uniform_hierarchy, upload

pytestmark = pytest.mark.gpu

N, DX, ETA0 = 48, 0.125, 0.1
DT = DX / 4


@pytest.mark.parametrize("integrator,ko_order,order", [(4, 5, 4), (4, 3, 6), (10, 3, 4), (4, 1, 2)])
def test_uniform_f64(integrator, ko_order, order):
    p = slh.EOMParams(order=order, integrator=integrator, ko_order=ko_order, ko_eps=0.05)
    y0 = inputs.gaussian_field(N, N / 8.0, 3)
    h, boxes = uniform_hierarchy(N, DX, prec="f64", nghost=3, bf=8)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    step = ork4.rk4_step_periodic if integrator == 4 else ossp.ssprk3_step_periodic
    y, eta = y0, ETA0
    for _ in range(40):
        h.rk_step(0, DT, p)
        y = step(y, eta, DT, DX, oparams(p))
        eta += DT
    g = download_domain(h, 0, boxes, N)
    for c in range(4):
        assert rel_l2(g[c], y[c]) <= 1e-12, (c, rel_l2(g[c], y[c]))
    # the dissipation did something: the run without it differs
    y2, eta = y0, ETA0
    for _ in range(40):
        y2 = step(y2, eta, DT, DX, oparams(slh.EOMParams(order=order, integrator=integrator)))
        eta += DT
    assert rel_l2(y[2], y2[2]) > 1e-6


def test_uniform_f32_kahan_within_bound():
    p = slh.EOMParams(order=4, ko_order=5, ko_eps=0.05)
    y0 = inputs.gaussian_field(N, N / 8.0, 4)
    h, boxes = uniform_hierarchy(N, DX, prec="f32", nghost=3, bf=8)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    y, eta = y0, ETA0
    for _ in range(100):
        h.rk_step(0, DT, p)
        y = ork4.rk4_step_periodic(y, eta, DT, DX, oparams(p))
        eta += DT
    g = download_domain(h, 0, boxes, N)
    for c in range(4):
        assert rel_l2(g[c].astype(np.float64), y[c]) <= 1e-4, c


BOXES = [
    [((0, 0, 0), (31, 31, 31))],
    [((16, 16, 16), (31, 47, 47)), ((32, 16, 16), (47, 47, 47))],
]


def _dense(level):
    parts = []
    for b in range(len(level.boxes)):
        v = level.data[b][level.valid(b)]
        for c in range(4):
            parts.append(v[c].ravel())
    return np.concatenate(parts)


@pytest.mark.parametrize("integrator", [4, 10])
def test_subcycled_hierarchy(integrator):
    p = slh.EOMParams(order=4, interp_type=4, integrator=integrator, ko_order=5, ko_eps=0.1)
    oh = oamr.make_hierarchy(32, 0.5, 0.125, 3, 8, BOXES, oparams(p), interp_type=4, eta0=1.0,
                             integrator=integrator)
    y0 = list(inputs.string_loop(32, 3.0, 2.0, 0.5))
    y0[2] = 0.3 * y0[1]                                   # momenta with structure, so their ghosts matter
    oh.levels[0].set_dense(y0)
    oamr.prolong_level_from_coarse(oh.levels[1], oh.levels[0], 4)
    oh.levels[0].old = None
    h = slh.Hierarchy(32, 0.5, nghost=3, bf=8, prec="f64", max_levels=2)
    for l in range(2):
        h.init_level(l, BOXES[l])
        h.set_state(l, _dense(oh.levels[l]))
    h.set_eta(1.0)
    for _ in range(2):
        oh.step()
        h.advance(0.125, p)
    for l, L in enumerate(oh.levels):
        got = slh.boxes_from_dense(h.get_state(l), L.boxes)
        for b in range(len(L.boxes)):
            exp = L.data[b][L.valid(b)]
            for c in range(4):
                assert rel_l2(got[b][c], exp[c]) <= 1e-12, (l, b, c)


def test_dissipation_width_needs_ghosts():
    h, boxes = uniform_hierarchy(16, DX, prec="f64", nghost=2, bf=8)
    with pytest.raises(slh.SlhError) as e:
        h.rk_step(0, DT, slh.EOMParams(order=4, ko_order=5, ko_eps=0.1))
    assert e.value.code == -1
    with pytest.raises(slh.SlhError) as e:
        h.rk_step(0, DT, slh.EOMParams(order=4, ko_order=2, ko_eps=0.1))
    assert e.value.code == -1


def test_app_c_discontinuity_on_the_wave_equation():
    """App. C's check on this repository's own system: the free wave equation
    (friction and potential off) with a box profile psi1 = 1 on the slab
    x < L/2 (half the volume), L = 10, classic RK4 with dt = 0.3 dx to t = 5,
    4th-order Laplacian, dissipation of order 5 (7 points).  With eps = 0 and
    eps = 1e-2 the GPU run equals the oracle (FP64 <= 1e-12 relative L2), and
    the dissipation lowers the high-frequency content of the profile (the
    share of spectral power above half the Nyquist wavenumber) behind the
    two fronts."""
    from tests.helpers import golden
    a = golden("app_c_ko.json")
    n = 64
    L = a["box_side"]
    dx = L / n
    dt = a["dt_over_dx"] * dx
    steps = int(round(a["t_end"] / dt))
    x = (np.arange(n) + 0.5) * dx
    slab = np.broadcast_to((x < 0.5 * L).astype(np.float64), (n, n, n)).copy()
    z = np.zeros_like(slab)
    y0 = (slab, z, z, z.copy())
    hf = {}
    for eps in (0.0, a["eps_small"]):
        p = slh.EOMParams(lam=0.0, friction=False, eta_power=0, order=4, ko_order=a["dissipation_order_p"],
                          ko_eps=eps)
        h, boxes = uniform_hierarchy(n, dx, prec="f64", nghost=3, bf=8)
        upload(h, 0, y0, boxes)
        h.set_eta(1.0)
        y, eta = y0, 1.0
        for _ in range(steps):
            h.rk_step(0, dt, p)
            y = ork4.rk4_step_periodic(y, eta, dt, dx, oparams(p))
            eta += dt
        g = download_domain(h, 0, boxes, n)
        for c in (0, 2):
            assert rel_l2(g[c], y[c]) <= 1e-12, (eps, c, rel_l2(g[c], y[c]))
        assert np.max(np.abs(g[1])) == 0.0 and np.max(np.abs(g[3])) == 0.0
        s = np.abs(np.fft.rfft(g[0][0, 0])) ** 2
        hf[eps] = float(s[len(s) // 2:].sum() / s.sum())
        h.close()
    assert hf[a["eps_small"]] < 0.75 * hf[0.0], hf
