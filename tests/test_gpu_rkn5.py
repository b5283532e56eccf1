"""RKN5 (integrator type 22, friction off) on the GPU vs the oracle
(oracle/rkn5.py): the four-stage Nystrom schedule of both stage kernels on a
uniform lattice (FP64 within 1e-12 relative L2 after 100 steps with fused
tags bit-exact, Laplacian orders 2/4/6 on ragged boxes; FP32 + Kahan within
1e-4), the subcycled hierarchy with graph replay, the autotuner in RKN5 form,
and the rejection of friction, of the Kreiss-Oliger term and of the tensor
fields."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import rkn5 as orkn5
from oracle import winding as owinding
from paper_2404_02950_gb300 import inputs
from tests.helpers import download_domain, oparams, rel_l2, tags_domain, uniform_hierarchy, upload

pytestmark = pytest.mark.gpu

N0, DX0, ETA0 = 64, 0.125, 0.1
DT0 = DX0 / 4


def _p(**kw):
    return slh.EOMParams(integrator=22, friction=False, **kw)


def test_uniform_f64_100_steps_fields_and_tags():
    p = _p(order=4)
    y0 = inputs.gaussian_field(N0, N0 / 8.0, 0)
    h, boxes = uniform_hierarchy(N0, DX0, prec="f64", nghost=2, bf=8, fused_tags=True)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    op = oparams(p)
    y, eta = y0, ETA0
    for step in range(100):
        snap = download_domain(h, 0, boxes, N0) if step % 25 == 0 else None
        h.rk_step(0, DT0, p, flags=slh.SLH_FUSE_TAG)
        if snap is not None:
            assert np.array_equal(tags_domain(h.fused_tags(0), boxes, N0),
                                  owinding.cell_tags_periodic(snap[0], snap[1])), step
        y = orkn5.rkn5_step_periodic(y, eta, DT0, DX0, op)
        eta = eta + DT0
    g = download_domain(h, 0, boxes, N0)
    for c in range(4):
        assert rel_l2(g[c], y[c]) <= 1e-12, (c, rel_l2(g[c], y[c]))
    assert h.get_eta(0) == eta


@pytest.mark.parametrize("order", [2, 6])
def test_uniform_f64_orders_ragged_boxes(order):
    p = _p(order=order)
    n = 40
    y0 = inputs.gaussian_field(n, 5.0, 3)
    boxes = [((0, 0, 0), (39, 39, 19)), ((0, 0, 20), (39, 39, 39))]
    h, _ = uniform_hierarchy(n, DX0, prec="f64", nghost=3, bf=4, boxes=boxes)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    y, eta = y0, ETA0
    for _ in range(40):
        h.rk_step(0, DT0, p)
        y = orkn5.rkn5_step_periodic(y, eta, DT0, DX0, oparams(p))
        eta += DT0
    g = download_domain(h, 0, boxes, n)
    for c in range(4):
        assert rel_l2(g[c], y[c]) <= 1e-12, (order, c)


def test_uniform_f32_kahan_within_bound():
    p = _p(order=6)
    n = 48
    y0 = inputs.gaussian_field(n, n / 8.0, 1)
    h, boxes = uniform_hierarchy(n, DX0, prec="f32", nghost=3, bf=8)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    y, eta = y0, ETA0
    for _ in range(100):
        h.rk_step(0, DT0, p)
        y = orkn5.rkn5_step_periodic(y, eta, DT0, DX0, oparams(p))
        eta += DT0
    g = download_domain(h, 0, boxes, n)
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


def test_subcycled_hierarchy_and_graph_replay():
    p = _p(order=4, interp_type=4)
    oh = oamr.make_hierarchy(32, 0.5, 0.125, 3, 8, BOXES, oparams(p), interp_type=4, eta0=1.0, integrator=22)
    oh.levels[0].set_dense(inputs.string_loop(32, 3.0, 2.0, 0.5))
    oamr.prolong_level_from_coarse(oh.levels[1], oh.levels[0], 4)
    oh.levels[0].old = None
    hs = []
    for graph in (False, True):
        h = slh.Hierarchy(32, 0.5, nghost=3, bf=8, prec="f64", max_levels=2)
        for l in range(2):
            h.init_level(l, BOXES[l])
            h.set_state(l, _dense(oh.levels[l]))
        h.set_eta(1.0)
        for _ in range(2):
            h.advance(0.125, p, flags=slh.SLH_USE_GRAPH if graph else 0)
        hs.append(h)
    for _ in range(2):
        oh.step()
    for l, L in enumerate(oh.levels):
        got = slh.boxes_from_dense(hs[0].get_state(l), L.boxes)
        for b in range(len(L.boxes)):
            exp = L.data[b][L.valid(b)]
            for c in range(4):
                assert rel_l2(got[b][c], exp[c]) <= 1e-12, (l, b, c)
        assert np.array_equal(hs[0].get_state(l), hs[1].get_state(l)), l


def test_autotune_in_rkn5_form_keeps_state():
    p = _p(order=6)
    n = 64
    y0 = inputs.gaussian_field(n, 8.0, seed=6)
    h, boxes = uniform_hierarchy(n, DX0, prec="f32", nghost=3, bf=16)
    upload(h, 0, y0, boxes)
    h.set_eta(0.3)
    before = h.get_state(0)
    chosen, ms = h.autotune(0, p, reps=2)
    assert 0 <= chosen < len(ms) and ms[chosen] == min(ms) and all(m > 0 for m in ms)
    assert np.array_equal(before, h.get_state(0))


def test_friction_dissipation_and_tensor_fields_are_rejected():
    h, _ = uniform_hierarchy(16, DX0, prec="f64", nghost=3, bf=8)
    for bad in (slh.EOMParams(order=4, integrator=22),                                   # friction on
                _p(order=4, ko_order=3, ko_eps=0.1)):
        with pytest.raises(slh.SlhError) as e:
            h.rk_step(0, DT0, bad)
        assert e.value.code == -1
    full = [((0, 0, 0), (15, 15, 15))]
    hg = slh.Hierarchy(16, 0.5, nghost=3, bf=8, prec="f64", max_levels=1, gw=True)
    hg.init_level(0, full)
    with pytest.raises(slh.SlhError) as e:
        hg.rk_step(0, DT0, _p(order=4))
    assert e.value.code == -1
