"""Dynamic AMR on the GPU vs the oracle (Sec. 2.2-2.3): device tags grown and
coarsened to blocks, host clustering in block units, live-level regrid
(copy where the old level covers, prolongation elsewhere), and subcycled
steps across regrids.  Box lists bit-exact; FP64 fields within 1e-12
relative L2 of the oracle."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import regrid as oregrid
from paper_2404_02950_gb300 import inputs
from tests.helpers import oparams, rel_l2

pytestmark = pytest.mark.gpu

N0, DX0, DT0, ETA0, G, BF = 32, 0.5, 0.125, 1.0, 3, 8
NBUF, MAX_BOX, MAXLEV = 2, 32, 3


def _dense_tags(oh, lev):
    L = oh.levels[lev]
    t = np.zeros((L.n, L.n, L.n), dtype=np.uint8)
    for (lo, hi), tb in zip(L.boxes, oh.tags(lev)):
        t[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = tb
    return t


def _oracle_regrid(oh):
    out = []
    for l in range(MAXLEV - 1):
        if l >= len(oh.levels):
            break
        parent = None if l == 0 else oh.levels[l].boxes
        boxes = oregrid.regrid_boxes(_dense_tags(oh, l), BF, NBUF, MAX_BOX, parent_boxes=parent)
        oamr.regrid_level(oh, l + 1, boxes)
        out.append(boxes)
        if not boxes:
            break
    return out


def _dense(level):
    parts = []
    for b in range(len(level.boxes)):
        v = level.data[b][level.valid(b)]
        for c in range(4):
            parts.append(v[c].ravel())
    return np.concatenate(parts)


def _compare(h, oh, tol):
    assert sorted(h.levels) == list(range(len(oh.levels)))
    for l, L in enumerate(oh.levels):
        assert [tuple(map(tuple, b)) for b in h.levels[l]["boxes"]] == L.boxes, l
        got = slh.boxes_from_dense(h.get_state(l), L.boxes)
        for b in range(len(L.boxes)):
            exp = L.data[b][L.valid(b)]
            for c in range(4):
                e = rel_l2(got[b][c], exp[c])
                assert e <= tol, (l, b, c, e)


@pytest.mark.parametrize("tile", [0, 2])
def test_regrid_then_subcycle_matches_oracle(tile):
    """tile: the stage tile of every level before the second regrid, which
    the regridded levels keep."""
    p = slh.EOMParams(order=4, interp_type=4)
    y0 = inputs.string_loop(N0, 4.0, 2.0, DX0)
    oh = oamr.make_hierarchy(N0, DX0, DT0, G, BF, [[((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))]], oparams(p),
                             interp_type=4, eta0=ETA0)
    oh.levels[0].set_dense(y0)
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=MAXLEV)
    h.init_level(0, [((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))])
    h.set_state(0, _dense(oh.levels[0]))
    h.set_eta(ETA0)
    # first regrid creates levels 1 and 2 by prolongation
    ob = _oracle_regrid(oh)
    gb = h.regrid(MAXLEV, NBUF, MAX_BOX)
    assert gb == ob and len(ob) == 2 and all(len(b) > 0 for b in ob)
    _compare(h, oh, 1e-13)
    for _ in range(2):
        oh.step()
        h.advance(DT0, p)
    _compare(h, oh, 1e-12)
    for l in sorted(h.levels):
        h.set_tile(l, tile)
    # second regrid: copies from the old levels where they overlap
    ob = _oracle_regrid(oh)
    gb = h.regrid(MAXLEV, NBUF, MAX_BOX)
    assert gb == ob
    _compare(h, oh, 1e-12)
    oh.step()
    h.advance(DT0, p)
    _compare(h, oh, 1e-12)


def test_tag_blocks_equal_grown_coarsened_oracle_tags():
    p = slh.EOMParams(order=4)
    y0 = inputs.string_loop(N0, 4.0, 2.0, DX0)
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=1)
    boxes = [((0, 0, 0), (15, 31, 31)), ((16, 0, 0), (31, 31, 31))]
    h.init_level(0, boxes)
    h.set_state(0, slh.dense_from_boxes(y0, boxes))
    h.set_eta(ETA0)
    from oracle import winding
    tags = winding.cell_tags_periodic(y0[0], y0[1])
    for nbuf in (0, 1, 3):
        got = h.tag_blocks(0, nbuf)
        exp = oregrid.coarsen_any(oregrid.dilate_periodic(tags != 0, nbuf), BF // 2)
        assert np.array_equal(got.astype(bool), exp), nbuf


def test_regrid_errors_and_removal():
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=3)
    h.init_level(0, [((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))])
    with pytest.raises(slh.SlhError) as e:
        h.regrid_level(2, [((48, 48, 48), (63, 63, 63))])     # level 1 missing
    assert e.value.code == -7
    h.regrid_level(1, [((16, 16, 16), (47, 47, 47))])
    h.regrid_level(2, [((48, 48, 48), (79, 79, 79))])
    h.regrid_level(1, [((16, 16, 16), (47, 47, 31))])        # level 2 now stale
    with pytest.raises(slh.SlhError) as e:
        h.advance(DT0, slh.EOMParams(order=4))
    assert e.value.code == -7
    # its ghost plan refers to the old level-1 boxes: no ghost-filling call runs
    for call in (lambda: h.fill_ghosts(2), lambda: h.tag(2), lambda: h.tag_blocks(2, 1),
                 lambda: h.reduce_energy(slh.EOMParams(order=4))):
        with pytest.raises(slh.SlhError) as e:
            call()
        assert e.value.code == -7
    h.regrid_level(2, [])                                     # remove it
    h.advance(DT0, slh.EOMParams(order=4))
    assert sorted(h.levels) == [0, 1]


def test_local_regrid_matches_oracle():
    """Local regrid (Sec. 2.3) on the GPU hierarchy: the block masks of the
    device tags, the host box update (slh_local_regrid_boxes) and the level
    rebuild, against the oracle's local regrid and data transfer."""
    from oracle import local_regrid as olr
    p = slh.EOMParams(order=4, interp_type=4)
    y0 = inputs.string_loop(N0, 4.0, 2.0, DX0)
    oh = oamr.make_hierarchy(N0, DX0, DT0, G, BF, [[((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))]], oparams(p),
                             interp_type=4, eta0=ETA0)
    oh.levels[0].set_dense(y0)
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=MAXLEV)
    h.init_level(0, [((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))])
    h.set_state(0, _dense(oh.levels[0]))
    h.set_eta(ETA0)
    # a global regrid with a small buffer, then the string moves and local regrids follow
    _oracle_regrid_nbuf(oh, 1)
    h.regrid(MAXLEV, 1, MAX_BOX)
    for _ in range(3):
        oh.step()
        h.advance(DT0, p)
    masks = [oregrid.coarsen_any(oregrid.dilate_periodic(_dense_tags(oh, l) != 0, NBUF), BF // 2)
             for l in range(len(oh.levels) - 1)]
    exp = olr.local_regrid([L.boxes for L in oh.levels], N0, BF, masks)
    cur = [list(L.boxes) for L in oh.levels]
    added = h.regrid_local(NBUF)
    got = [[tuple(map(tuple, b)) for b in h.levels[l]["boxes"]] for l in sorted(h.levels)]
    assert got == [[(tuple(int(v) for v in lo), tuple(int(v) for v in hi)) for lo, hi in lb] for lb in exp]
    assert any(a > 0 for a in added)
    first = next(l for l in range(1, len(exp)) if exp[l] != cur[l])
    for l in range(first, len(exp)):
        oamr.regrid_level(oh, l, exp[l])
    _compare(h, oh, 1e-12)
    oh.step()
    h.advance(DT0, p)
    _compare(h, oh, 1e-12)


def _oracle_regrid_nbuf(oh, nbuf):
    for l in range(MAXLEV - 1):
        if l >= len(oh.levels):
            break
        parent = None if l == 0 else oh.levels[l].boxes
        boxes = oregrid.regrid_boxes(_dense_tags(oh, l), BF, nbuf, MAX_BOX, parent_boxes=parent)
        oamr.regrid_level(oh, l + 1, boxes)
        if not boxes:
            break


def _volume(boxes):
    return sum((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) for lo, hi in boxes)


def _loop_hierarchy(prec="f64"):
    y0 = inputs.string_loop(N0, 4.0, 2.0, DX0)
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec=prec, max_levels=MAXLEV)
    full = [((0, 0, 0), (N0 - 1, N0 - 1, N0 - 1))]
    h.init_level(0, full)
    h.set_state(0, slh.dense_from_boxes(y0, full))
    h.set_eta(ETA0)
    return h


def test_auto_regrid_follows_the_fallback_rule():
    """slh_regrid in auto mode (the library decides, Sec. 2.3) against the
    oracle's RegridPolicy fed with the hierarchy's own volumes: the same kind
    of regrid every time, the same added-volume fractions after each local
    one, and a global one that leaves the levels below its start level alone."""
    from oracle import local_regrid as olr
    p = slh.EOMParams(order=4, interp_type=4)
    eps_s, eps_w, cap = 0.02, 0.01, 3
    h = _loop_hierarchy()
    pol = olr.RegridPolicy(MAXLEV, eps_strong=eps_s, eps_weak=eps_w, max_local=cap)
    kinds = []
    for _ in range(9):
        before = [list(h.levels[l]["boxes"]) for l in sorted(h.levels)]
        exp_kind, exp_start = pol.next_regrid([_volume(b) for b in before])
        kind, res = h.regrid_auto(MAXLEV, NBUF, MAX_BOX, eps_strong=eps_s, eps_weak=eps_w, max_local=cap)
        assert kind == exp_kind, (kinds, kind)
        after = [list(h.levels[l]["boxes"]) for l in sorted(h.levels)]
        if kind == "local":
            assert len(after) == len(before)
            frac = pol.after_local([_volume(a) - _volume(b) for a, b in zip(after, before)])
            assert res == frac
        else:
            pol.after_global()
            for l in range(exp_start + 1):
                assert after[l] == before[l], l
        kinds.append(kind)
        for _ in range(2):
            h.advance(DT0, p)
    assert kinds.count("local") >= 3 and kinds.count("global") >= 2, kinds
    h.close()


def test_graph_replay_across_regrids_matches_direct():
    """The coarse-step CUDA graph is captured again after every regrid (the
    levels' boxes and buffers change): replayed steps across two global and
    one local regrid equal the direct launches bit for bit."""
    p = slh.EOMParams(order=4, interp_type=4)
    ha, hb = _loop_hierarchy(), _loop_hierarchy()
    for rnd in range(3):
        if rnd < 2:
            la = ha.regrid(MAXLEV, NBUF, MAX_BOX)
            lb = hb.regrid(MAXLEV, NBUF, MAX_BOX)
        else:
            la = ha.regrid_local(NBUF)
            lb = hb.regrid_local(NBUF)
        assert la == lb
        for _ in range(3):
            ha.advance(DT0, p)
            hb.advance(DT0, p, flags=slh.SLH_USE_GRAPH)
        assert sorted(ha.levels) == sorted(hb.levels) and len(ha.levels) == MAXLEV
        for l in sorted(ha.levels):
            assert ha.levels[l]["boxes"] == hb.levels[l]["boxes"]
            assert np.array_equal(ha.get_state(l), hb.get_state(l)), (rnd, l)
    ha.close()
    hb.close()
