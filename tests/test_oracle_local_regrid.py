"""Pins of the oracle's local regrid (Sec. 2.3, oracle/local_regrid.py):
properties the paper fixes, checked cell by cell on random hierarchies."""
import numpy as np
import pytest

from oracle import local_regrid as olr


def _cells(boxes, n):
    m = np.zeros((n, n, n), dtype=np.int32)
    for lo, hi in boxes:
        m[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += 1
    return m


def _nested(fine_boxes, coarse_boxes, nc, r):
    """Every fine box's coarse footprint grown by r coarse cells (periodic)
    lies in the coarse level: checked cell by cell."""
    cov = _cells(coarse_boxes, nc) > 0
    for lo, hi in fine_boxes:
        for z in range(lo[2] // 2 - r, (hi[2] + 1) // 2 + r):
            for y in range(lo[1] // 2 - r, (hi[1] + 1) // 2 + r):
                for x in range(lo[0] // 2 - r, (hi[0] + 1) // 2 + r):
                    if not cov[z % nc, y % nc, x % nc]:
                        return False
    return True


def _random_case(seed, n0=16, bf=4):
    rng = np.random.default_rng(seed)
    r = bf // 2
    L = 3
    boxes = [[((0, 0, 0), (n0 - 1,) * 3)]]
    # level 1: a few bf-aligned boxes well inside level 0; level 2 nested in level 1
    lo1 = rng.integers(1, 3, size=3) * bf
    boxes.append([(tuple(int(v) for v in lo1), tuple(int(v + 2 * bf - 1) for v in lo1))])
    c = [(lo1[d] + bf) * 2 for d in range(3)]   # inside level 1, away from its edge
    boxes.append([(tuple(c), tuple(v + bf - 1 for v in c))])
    assert _nested(boxes[1], boxes[0], n0, r) and _nested(boxes[2], boxes[1], 2 * n0, r)
    masks = []
    for l in range(L - 1):
        nb = (n0 << l) // r
        masks.append(rng.random((nb, nb, nb)) < 0.03)
    return boxes, masks, n0, bf


@pytest.mark.parametrize("seed", range(6))
def test_grows_covers_and_nests(seed):
    boxes, masks, n0, bf = _random_case(seed)
    r = bf // 2
    out = olr.local_regrid(boxes, n0, bf, masks)
    for l in range(len(boxes)):
        n = n0 << l
        assert out[l][:len(boxes[l])] == boxes[l]                 # old boxes kept as they are
        cov = _cells(out[l], n)
        assert cov.max() <= 1                                      # no overlap
        assert np.all(cov[_cells(boxes[l], n) > 0] == 1)           # only grows
        for lo, hi in out[l][len(boxes[l]):]:
            assert all(lo[d] % bf == 0 and (hi[d] + 1) % bf == 0 for d in range(3))
    for l in range(len(boxes) - 1):
        fine = _cells(out[l + 1], n0 << (l + 1)) > 0
        nb = masks[l].shape[0]
        for bz, by, bx in zip(*np.nonzero(masks[l])):
            # the r-block of level l = a bf-block of level l+1
            blk = fine[bz * bf:(bz + 1) * bf, by * bf:(by + 1) * bf, bx * bf:(bx + 1) * bf]
            assert blk.all(), (l, bz, by, bx)
        assert nb == (n0 << l) // r
    for l in range(1, len(boxes)):
        assert _nested(out[l], out[l - 1], n0 << (l - 1), r), l


def test_no_change_when_covered_and_idempotent():
    boxes, masks, n0, bf = _random_case(7)
    none = [np.zeros_like(m) for m in masks]
    assert olr.local_regrid(boxes, n0, bf, none) == boxes
    out = olr.local_regrid(boxes, n0, bf, masks)
    assert olr.local_regrid(out, n0, bf, masks) == out
    # tags inside the already refined region change nothing
    inner = [np.zeros_like(m) for m in masks]
    lo, hi = boxes[1][0]
    inner[0][lo[2] // bf, lo[1] // bf, lo[0] // bf] = True      # level-1 cell c lies in level-0 block c // bf
    assert olr.local_regrid(boxes, n0, bf, inner) == boxes


def _brute_force_cells(boxes, n0, bf, masks):
    """The least refined region per level that keeps the old boxes, covers
    every tagged block of M_l by level l+1 and nests every level in the one
    below with a gap of r = bf/2 coarse cells, with additions in whole blocks
    of bf cells: cell by cell, iterated to a fixed point (no block algebra)."""
    L = len(boxes)
    r = bf // 2
    cells = [_cells(boxes[l], n0 << l) > 0 for l in range(L)]
    for l in range(L - 1):
        for bz, by, bx in zip(*np.nonzero(np.asarray(masks[l], dtype=bool))):
            # r cells of level l along an axis = 2r = bf cells of level l+1
            cells[l + 1][bz * bf:(bz + 1) * bf, by * bf:(by + 1) * bf, bx * bf:(bx + 1) * bf] = True
    changed = True
    while changed:
        changed = False
        for j in range(L - 1, 0, -1):
            nc = n0 << (j - 1)
            foot = cells[j].reshape(nc, 2, nc, 2, nc, 2).any(axis=(1, 3, 5))
            req = np.zeros_like(foot)
            for dz in range(-r, r + 1):
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        req |= np.roll(foot, (dz, dy, dx), axis=(0, 1, 2))
            nb = nc // bf
            blk = req.reshape(nb, bf, nb, bf, nb, bf).any(axis=(1, 3, 5))
            req = np.repeat(np.repeat(np.repeat(blk, bf, 0), bf, 1), bf, 2)
            if (req & ~cells[j - 1]).any():
                cells[j - 1] |= req
                changed = True
    return cells


@pytest.mark.parametrize("seed", range(6))
def test_adds_exactly_the_required_blocks(seed):
    """Minimality: the refined region of every level equals, cell for cell,
    the least region the tags and the nesting rule force (a local regrid that
    grows one block too many, or a nesting shell one block too wide, fails)."""
    boxes, masks, n0, bf = _random_case(seed)
    out = olr.local_regrid(boxes, n0, bf, masks)
    want = _brute_force_cells(boxes, n0, bf, masks)
    for l in range(len(boxes)):
        assert np.array_equal(_cells(out[l], n0 << l) > 0, want[l]), l


def test_worked_case_one_tag_block_at_the_fine_edge():
    """Level 1 = [4, 11]^3 and level 2 = [12, 19]^3 (bf = 4, r = 2); one tagged
    block of level 1 at cells (10..11, 8..9, 8..9), just outside level 2.
    Level 2 gains exactly that block ([20, 23] x [16, 19]^2); its footprint
    grown by 2 reaches level-1 x = 12..13, so level 1 gains exactly the four
    blocks x in [12, 15], y and z in [4, 7] or [8, 11]; level 0 is unchanged."""
    n0, bf = 16, 4
    boxes = [[((0, 0, 0), (15, 15, 15))], [((4, 4, 4), (11, 11, 11))], [((12, 12, 12), (19, 19, 19))]]
    masks = [np.zeros((8, 8, 8), dtype=bool), np.zeros((16, 16, 16), dtype=bool)]
    masks[1][4, 4, 5] = True       # [z, y, x] r-block of level 1: cells x 10..11, y 8..9, z 8..9
    out = olr.local_regrid(boxes, n0, bf, masks)
    assert out[0] == boxes[0]
    assert out[2] == boxes[2] + [((20, 16, 16), (23, 19, 19))]
    assert out[1] == boxes[1] + [((12, 4, 4), (15, 7, 7)), ((12, 8, 4), (15, 11, 7)),
                                 ((12, 4, 8), (15, 7, 11)), ((12, 8, 8), (15, 11, 11))]


def test_policy_worked_sequences():
    """The fallback rule of Sec. 2.3 on hand-worked volume sequences."""
    # a hierarchy short of its levels is regridded globally from level 0
    pol = olr.RegridPolicy(3)
    assert pol.next_regrid([4096, 1000]) == ("global", 0)
    pol.after_global()
    # local regrids accumulate dV_l against the volumes at the last global regrid
    assert pol.next_regrid([4096, 1000, 2000]) == ("local", None)
    assert pol.after_local([0, 40, 90]) == [0.0, 0.04, 0.045]
    assert pol.next_regrid([4096, 1040, 2090]) == ("local", None)
    frac = pol.after_local([0, 70, 10])          # level 1 reaches 11 % >= eps_s
    assert frac == [0.0, 0.11, 0.05]
    # both levels reach eps_w: the global regrid starts at level 1 (from level 0's tags)
    assert pol.next_regrid([4096, 1110, 2100]) == ("global", 0)
    pol.after_global()
    # the counters start again from the new volumes
    assert pol.next_regrid([4096, 1200, 2400]) == ("local", None)
    frac = pol.after_local([0, 12, 250])          # only level 2 is above eps_w (and eps_s)
    assert frac == [0.0, 0.01, 250 / 2400]
    assert pol.next_regrid([4096, 1212, 2650]) == ("global", 1)
    # the cap on consecutive local regrids, with every fraction small
    pol = olr.RegridPolicy(2, max_local=3)
    assert pol.next_regrid([4096, 1000]) == ("local", None)
    for k in range(3):
        assert pol.next_regrid([4096, 1000 + k]) == ("local", None)
        pol.after_local([0, 1])
    assert pol.next_regrid([4096, 1003]) == ("global", 0)
    # eps_s is reached on a level while a finer one is below eps_w
    pol = olr.RegridPolicy(3, eps_strong=0.2, eps_weak=0.1)
    pol.next_regrid([100, 100, 100])
    pol.after_local([0, 5, 25])
    assert pol.next_regrid([100, 105, 125]) == ("global", 1)
