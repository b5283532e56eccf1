"""Truncation-error-estimate tagging on the GPU vs the oracle (Sec. 2.2,
oracle/tee.py): the self-shadow estimate fused into the restriction of a
two-level hierarchy, and the level-0 shadow context.  The estimates of the
two sides agree to rounding; thresholds are put in a gap of the oracle's
estimates so that the tags must agree bit for bit."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import regrid as oregrid
from oracle import tee as otee
from oracle.rk4 import rk4_step_periodic
from paper_2404_02950_gb300 import inputs
from tests.helpers import oparams

pytestmark = pytest.mark.gpu

N0, DX0, DT0, ETA0, G, BF = 32, 0.5, 0.125, 1.0, 3, 8
BOXES = [
    [((0, 0, 0), (31, 31, 31))],
    [((16, 16, 16), (31, 47, 47)), ((32, 16, 16), (47, 47, 47))],
]


def _gap_thresholds(te):
    """Per component: the midpoint of the widest gap between consecutive
    sorted estimates in their middle half."""
    eps = []
    for c in range(4):
        v = np.sort(np.concatenate([t[c].ravel() for t in te]))
        lo, hi = len(v) // 4, 3 * len(v) // 4
        gaps = np.diff(v[lo:hi])
        i = int(np.argmax(gaps))
        eps.append(0.5 * (v[lo + i] + v[lo + i + 1]))
    return eps


def _dense(level):
    parts = []
    for b in range(len(level.boxes)):
        v = level.data[b][level.valid(b)]
        for c in range(4):
            parts.append(v[c].ravel())
    return np.concatenate(parts)


def test_self_shadow_tags_at_synchronisation_match_oracle():
    p = slh.EOMParams(order=4, interp_type=4)
    oh = oamr.make_hierarchy(N0, DX0, DT0, G, BF, BOXES, oparams(p), interp_type=4, eta0=ETA0)
    oh.levels[0].set_dense(inputs.string_loop(N0, 3.0, 2.0, DX0))
    oamr.prolong_level_from_coarse(oh.levels[1], oh.levels[0], 4)
    oh.levels[0].old = None
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=2)
    for l in range(2):
        h.init_level(l, BOXES[l])
        h.set_state(l, _dense(oh.levels[l]))
    h.set_eta(ETA0)
    oh.te_eps = [1.0] * 4
    oh.step()
    eps = _gap_thresholds(oh.te_vals[1])
    exp = np.concatenate([otee.tags_from_te(t, eps).ravel() for t in oh.te_vals[1]])
    assert 0.05 < exp.mean() < 0.95
    h.set_tagging(winding=True, te_crit=eps)
    h.advance(DT0, p)
    assert np.array_equal(h.tee_tags(1), exp)
    # a component left out (threshold 0) no longer tags
    h2eps = [eps[0], 0.0, 0.0, 0.0]
    exp0 = np.concatenate([otee.tags_from_te(t, h2eps).ravel() for t in oh.te_vals[1]])
    assert exp0.sum() < exp.sum()


def test_shadow_level_tags_and_block_mask_match_oracle():
    p = slh.EOMParams(order=4)
    y0 = inputs.gaussian_field(N0, N0 / 8.0, seed=5)
    y1 = rk4_step_periodic(y0, ETA0, DT0, DX0, oparams(p))
    y2 = rk4_step_periodic(y1, ETA0 + DT0, DT0, DX0, oparams(p))
    _, te = otee.shadow_tags(y0, ETA0, DT0, DX0, oparams(p), y2, [1.0] * 4)
    eps = _gap_thresholds([te])
    exp, _ = otee.shadow_tags(y0, ETA0, DT0, DX0, oparams(p), y2, eps)
    assert 0.05 < exp.mean() < 0.95
    full = [((0, 0, 0), (N0 - 1,) * 3)]
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=1)
    h.init_level(0, full)
    h.set_state(0, slh.dense_from_boxes(y0, full))
    h.set_eta(ETA0)
    h.set_tagging(winding=False, te_crit=eps)
    sh = h.make_shadow()
    h.shadow_init(sh)
    sh.rk_step(0, 2 * DT0, p)
    for _ in range(2):
        h.advance(DT0, p)
    h.shadow_compare(sh)
    assert np.array_equal(h.tee_tags(0), exp.ravel())
    masks = {}
    for nbuf in (0, 2):
        masks[nbuf] = h.tag_blocks(0, nbuf)
        want = oregrid.coarsen_any(oregrid.dilate_periodic(exp != 0, nbuf), BF // 2)
        assert np.array_equal(masks[nbuf].astype(bool), want), nbuf
    # both criteria: the union of the two block masks
    h.set_tagging(winding=True, te_crit=eps)
    both = h.tag_blocks(0, 0)
    h.set_tagging(winding=True)
    wind = h.tag_blocks(0, 0)
    assert wind.any() and np.array_equal(both.astype(bool), wind.astype(bool) | masks[0].astype(bool))


def test_tagging_errors():
    h = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=1)
    h.init_level(0, [((0, 0, 0), (N0 - 1,) * 3)])
    with pytest.raises(slh.SlhError) as e:
        h.tee_tags(0)                                   # not enabled
    assert e.value.code == -7
    with pytest.raises(slh.SlhError) as e:
        h.set_tagging(winding=False, te_crit=None)      # no criterion
    assert e.value.code == -1
    other = slh.Hierarchy(N0, DX0, nghost=G, bf=BF, prec="f64", max_levels=1)
    other.init_level(0, [((0, 0, 0), (N0 - 1,) * 3)])
    h.set_tagging(winding=True, te_crit=[1e-3] * 4)
    with pytest.raises(slh.SlhError) as e:
        h.shadow_init(other)                            # not half resolution
    assert e.value.code == -1
