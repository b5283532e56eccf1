"""GPU vs oracle parity on a static level hierarchy (Sec. 2.1): ghost fill by
same-level copy and quartic prolongation with time interpolation, 2^3
restriction at synchronisation, Berger-Oliger subcycling, tags and energy
over the hierarchy.  FP64 within 1e-12 relative L2 of the oracle; tags
bit-exact on identical (ghost-filled) snapshots."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import interp as ointerp
from oracle import winding as owinding
from paper_2404_02950_gb300 import inputs
from tests.helpers import box_padded_views, oparams, rel_l2

pytestmark = pytest.mark.gpu

N0, DX0, DT0, ETA0, G, BF = 32, 0.5, 0.125, 1.0, 3, 8
LEVEL_BOXES = [
    [((0, 0, 0), (31, 31, 31))],
    [((16, 16, 16), (31, 47, 47)), ((32, 16, 16), (47, 47, 47))],
    [((48, 48, 48), (79, 79, 71)), ((48, 48, 72), (79, 79, 79))],
]


def _dense(level):
    parts = []
    for b in range(len(level.boxes)):
        v = level.data[b][level.valid(b)]
        for c in range(4):
            parts.append(v[c].ravel())
    return np.concatenate(parts)


def _oracle_hierarchy(p, nlev=3, itype=4, g=G):
    h = oamr.make_hierarchy(N0, DX0, DT0, g, BF, LEVEL_BOXES[:nlev], oparams(p), interp_type=itype, eta0=ETA0)
    y = inputs.string_loop(N0, 3.0, 2.0, DX0)
    h.levels[0].set_dense(y)
    for l in range(1, nlev):
        oamr.prolong_level_from_coarse(h.levels[l], h.levels[l - 1], itype)
        h.levels[l - 1].old = None
    return h


def _gpu_hierarchy(oh, prec="f64", fused_tags=False):
    nlev = len(oh.levels)
    h = slh.Hierarchy(N0, DX0, nghost=oh.levels[0].g, bf=BF, prec=prec, max_levels=nlev)
    for l in range(nlev):
        h.init_level(l, LEVEL_BOXES[l], fused_tags=fused_tags)
        h.set_state(l, _dense(oh.levels[l]))
    h.set_eta(ETA0)
    return h


def _gpu_levels(h, lev):
    return slh.boxes_from_dense(h.get_state(lev), LEVEL_BOXES[lev])


def _ghosted(h, lev, g=G):
    """GPU per-box arrays with ghost layers, in the oracle's (4, nz+2g, ny+2g, nx+2g) form."""
    h.sync()
    out = []
    for (lo, hi), v in zip(LEVEL_BOXES[lev], box_padded_views(h, lev)):
        nx = hi[0] - lo[0] + 1
        a = v.double().cpu().numpy()
        out.append(a[:, :, :, 4 - g:4 + nx + g])
    return out


@pytest.mark.parametrize("nlev,g", [(2, 3), (3, 3), (3, 2)])
def test_subcycled_hierarchy_f64_matches_oracle(nlev, g):
    """g = 2: ghost layers equal to the 4th-order stencil's radius."""
    p = slh.EOMParams(order=4, interp_type=4)
    oh = _oracle_hierarchy(p, nlev, g=g)
    h = _gpu_hierarchy(oh)
    for _ in range(2):
        oh.step()
        h.advance(DT0, p)
    for l in range(nlev):
        got = _gpu_levels(h, l)
        for b in range(len(LEVEL_BOXES[l])):
            exp = oh.levels[l].data[b][oh.levels[l].valid(b)]
            for c in range(4):
                assert rel_l2(got[b][c], exp[c]) <= 1e-12, (l, b, c, rel_l2(got[b][c], exp[c]))
        assert h.get_eta(l) == oh.levels[l].eta
    # energy over the uncovered cells of every level
    E = h.reduce_energy(p)
    Eo = oh.energy()
    for k in range(4):
        assert abs(E[k] - Eo[k]) <= 1e-12 * max(abs(Eo[k]), 1.0), (k, E[k], Eo[k])
    assert E[4] == Eo[4]


def test_tags_on_every_level_bit_exact_with_ghosts():
    p = slh.EOMParams(order=4)
    oh = _oracle_hierarchy(p, 3)
    h = _gpu_hierarchy(oh)
    h.advance(DT0, p)
    for l in range(3):
        t, cnt = h.tag(l)           # fills ghosts at alpha = 1, then tags
        snap = _ghosted(h, l)       # the exact ghost-filled state the tags saw
        exp = np.concatenate([owinding.cell_tags_padded(a[0], a[1], G).ravel() for a in snap])
        assert np.array_equal(t.cpu().numpy(), exp), l
        assert cnt == int(exp.sum())
    assert sum(int(h.tag(l)[1]) for l in range(3)) > 0


@pytest.mark.parametrize("itype", [2, 4])
def test_ghost_prolongation_with_time_interpolation(itype):
    p = slh.EOMParams(order=4, interp_type=itype)
    oh = _oracle_hierarchy(p, 2, itype)
    h = _gpu_hierarchy(oh)
    h.rk_step(0, DT0, p)             # coarse old != new
    C = oamr.Level(0, LEVEL_BOXES[0], N0, DX0, DT0, G, BF)
    F = oamr.Level(1, LEVEL_BOXES[1], 2 * N0, DX0 / 2, DT0 / 2, G, BF)
    prev = box_padded_views(h, 0, role=slh.SLH_BUF_Y)     # before the step (rotated away)
    h.sync()
    C.old = [v.double().cpu().numpy()[:, :, :, 4 - G:4 + N0 + G].copy() for v in prev]
    C.data = _ghosted(h, 0)
    alpha = 0.25
    h.fill_ghosts(1, alpha=alpha, interp_type=itype)
    got = _ghosted(h, 1)
    arrs = [g.copy() for g in got]
    oamr.fill_ghosts(F, arrs, C, alpha, itype)
    for b in range(len(arrs)):
        assert np.max(np.abs(arrs[b][:2] - got[b][:2])) <= 1e-13, b


def test_restriction_is_exact_mean_of_children():
    p = slh.EOMParams(order=4)
    oh = _oracle_hierarchy(p, 2)
    h = _gpu_hierarchy(oh)
    h.rk_step(1, DT0, p, sub=0)
    fine = _gpu_levels(h, 1)
    h.fill_ghosts(1, mode=slh.SLH_RESTRICT)
    coarse = _gpu_levels(h, 0)[0]
    for (lo, hi), fb in zip(LEVEL_BOXES[1], fine):
        clo = [v // 2 for v in lo]
        for c in range(4):
            exp = ointerp.restrict_block(fb[c])
            got = coarse[c][clo[2]:clo[2] + exp.shape[0], clo[1]:clo[1] + exp.shape[1], clo[0]:clo[0] + exp.shape[2]]
            assert np.array_equal(got, exp)


def test_f32_hierarchy_within_bound_of_f64_oracle():
    p = slh.EOMParams(order=4, interp_type=4)
    oh = _oracle_hierarchy(p, 3)
    h = _gpu_hierarchy(oh, prec="f32")
    for _ in range(2):
        oh.step()
        h.advance(DT0, p)
    for l in range(3):
        got = _gpu_levels(h, l)
        for b in range(len(LEVEL_BOXES[l])):
            exp = oh.levels[l].data[b][oh.levels[l].valid(b)]
            for c in range(4):
                assert rel_l2(got[b][c], exp[c]) <= 1e-4, (l, b, c)


def test_graph_replay_on_hierarchy_matches_direct():
    p = slh.EOMParams(order=4)
    oh = _oracle_hierarchy(p, 3)
    ha = _gpu_hierarchy(oh)
    hb = _gpu_hierarchy(oh)
    for _ in range(3):
        ha.advance(DT0, p)
        hb.advance(DT0, p, flags=slh.SLH_USE_GRAPH)
    for l in range(3):
        assert np.array_equal(ha.get_state(l), hb.get_state(l))


@pytest.mark.parametrize("prec,integrator,ko", [("f32", 4, 0), ("f64", 4, 0), ("f32", 10, 0), ("f32", 21, 0),
                                                 ("f32", 22, 0), ("f32", 4, 3)])
def test_advance_equals_single_level_steps_bit_for_bit(prec, integrator, ko):
    """slh_advance copies prolonged ghost values a fill already computed in the
    same step of the coarser level (same coarse states, same time fraction)
    instead of prolonging again; the same subcycled order built from single
    level steps and restrictions, where every fill prolongs afresh, gives the
    same bits on every level, for each integrator and with dissipation."""
    p = slh.EOMParams(order=4, interp_type=4, integrator=integrator, friction=integrator != 22,
                      ko_order=ko, ko_eps=0.02 if ko else 0.0)
    oh = _oracle_hierarchy(p, 3)
    a = _gpu_hierarchy(oh, prec=prec)
    b = _gpu_hierarchy(oh, prec=prec)

    def level_step(lev, sub):
        b.rk_step(lev, DT0, p, sub=sub)
        if lev + 1 < 3:
            for i in range(2):
                level_step(lev + 1, i)
            b.fill_ghosts(lev + 1, 1.0, p.interp_type, mode=slh.SLH_RESTRICT)

    for _ in range(2):
        a.advance(DT0, p)
        level_step(0, 0)
    for l in range(3):
        assert np.array_equal(a.get_state(l), b.get_state(l)), l
    a.advance(DT0, p, flags=slh.SLH_USE_GRAPH)
    level_step(0, 0)
    for l in range(3):
        assert np.array_equal(a.get_state(l), b.get_state(l)), l


def test_nonfinite_coarse_value_is_not_a_nesting_error():
    """A NaN in a covered coarse cell is a field value, not a box-layout
    error: the ghost fill returns OK and carries the NaN into the ghost cells
    whose stencil reads it; every other ghost cell stays finite."""
    import torch
    p = slh.EOMParams(order=4, interp_type=4)
    oh = _oracle_hierarchy(p, 2)
    h = _gpu_hierarchy(oh)
    h.sync()
    # coarse cell (x, y, z) = (7, 12, 12): outside level 1's footprint
    # (coarse 8..23) but under the quartic stencils of its lower-x ghost
    # shell (level-1 x = 13..15 -> coarse parents 6..7, radius 2)
    v = box_padded_views(h, 0)[0]
    with torch.no_grad():
        v[0, 12 + G, 12 + G, 7 + 4] = float("nan")
    h.fill_ghosts(1, alpha=1.0, interp_type=4)
    h.sync()   # no latched error
    got = _ghosted(h, 1)
    nan_cells = sum(int(np.isnan(a[0]).sum()) for a in got)
    assert nan_cells > 0
    assert all(np.isfinite(a[1]).all() for a in got)   # psi2's ghosts never read the NaN


def test_nesting_violation_is_rejected_on_host():
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=3)
    h.init_level(0, LEVEL_BOXES[0])
    h.init_level(1, LEVEL_BOXES[1])
    with pytest.raises(slh.SlhError) as e:
        # its coarse footprint (16..23 on level 1) plus the one-block gap
        # reaches level-1 cell 12, outside level 1's boxes (16..47)
        h.init_level(2, [((32, 32, 32), (47, 47, 47))])
    assert e.value.code == -2
    # a level-0 that does not cover the domain is rejected too
    h2 = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=1)
    with pytest.raises(slh.SlhError):
        h2.init_level(0, [((0, 0, 0), (15, 31, 31))])
