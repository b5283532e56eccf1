"""Pins of the oracle's regrid (Sec. 2.2-2.3 reading in oracle/regrid.py):
invariants any valid clustering must satisfy, brute-force dilation, and
small cases whose answer follows from the rules by hand."""
import numpy as np
import pytest

from oracle import regrid


def _brute_dilate(mask, nbuf):
    n = mask.shape
    out = np.zeros_like(mask, dtype=bool)
    for k, j, i in np.argwhere(mask):
        for dz in range(-nbuf, nbuf + 1):
            for dy in range(-nbuf, nbuf + 1):
                for dx in range(-nbuf, nbuf + 1):
                    out[(k + dz) % n[0], (j + dy) % n[1], (i + dx) % n[2]] = True
    return out


def test_dilation_bruteforce():
    rng = np.random.default_rng(0)
    m = rng.random((8, 12, 10)) < 0.02
    for nb in (0, 1, 2, 4):
        assert np.array_equal(regrid.dilate_periodic(m, nb), _brute_dilate(m, nb))


def _check_invariants(tags, bf, nbuf, max_box, boxes, parent=None):
    nz, ny, nx = tags.shape
    D = regrid.dilate_periodic(tags != 0, nbuf)
    r = bf // 2
    if parent is not None:
        P = regrid.parent_block_mask(parent, (nx, ny, nz), r)
        allowed = ~regrid.dilate_periodic(~P, 1)
    else:
        allowed = np.ones((nz // r, ny // r, nx // r), dtype=bool)
    cover = np.zeros((2 * nz, 2 * ny, 2 * nx), dtype=np.int32)
    for lo, hi in boxes:
        for d in range(3):
            assert lo[d] % bf == 0 and (hi[d] + 1) % bf == 0
            assert bf <= hi[d] - lo[d] + 1 <= max_box
        cover[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += 1
        # nested: every block of the box allowed
        blk = allowed[lo[2] // bf:(hi[2] + 1) // bf, lo[1] // bf:(hi[1] + 1) // bf,
                      lo[0] // bf:(hi[0] + 1) // bf]
        assert blk.all()
    assert cover.max() <= 1          # disjoint
    # every dilated tag inside the allowed region is refined
    Ab = np.repeat(np.repeat(np.repeat(allowed, r, 0), r, 1), r, 2)
    need = D & Ab
    for k, j, i in np.argwhere(need):
        assert cover[2 * k, 2 * j, 2 * i] == 1
    keys = [(b[0][2], b[0][1], b[0][0]) for b in boxes]
    assert keys == sorted(keys)


@pytest.mark.parametrize("seed", range(6))
def test_random_masks_invariants(seed):
    rng = np.random.default_rng(seed)
    n = 32
    tags = np.zeros((n, n, n), dtype=np.uint8)
    for _ in range(int(rng.integers(1, 6))):
        c = rng.integers(0, n, size=3)
        L = int(rng.integers(1, 10))
        ax = int(rng.integers(0, 3))
        for t in range(L):
            p = c.copy()
            p[ax] = (p[ax] + t) % n
            tags[tuple(p)] = 1
    for bf, nbuf, mb in ((8, 2, 16), (4, 1, 8), (16, 4, 32)):
        boxes = regrid.regrid_boxes(tags, bf, nbuf, mb)
        _check_invariants(tags, bf, nbuf, mb, boxes)


def test_nesting_with_parent():
    n = 32
    tags = np.zeros((n, n, n), dtype=np.uint8)
    tags[12:20, 12:14, 10:22] = 1
    tags[2, 2, 2] = 1                 # outside the parent's interior: dropped
    parent = [((8, 8, 8), (23, 23, 23))]
    boxes = regrid.regrid_boxes(tags, 8, 1, 32, parent_boxes=parent)
    _check_invariants(tags, 8, 1, 32, boxes, parent=parent)
    for lo, hi in boxes:
        for d in range(3):
            assert lo[d] >= 2 * 8 + 8 and hi[d] <= 2 * 24 - 8 - 1


def test_single_tag_gives_one_block():
    tags = np.zeros((16, 16, 16), dtype=np.uint8)
    tags[5, 9, 2] = 1
    boxes = regrid.regrid_boxes(tags, 8, 0, 64)
    assert boxes == [((0, 16, 8), (7, 23, 15))]


def test_full_domain_halved_to_max_box():
    tags = np.ones((16, 16, 16), dtype=np.uint8)
    boxes = regrid.regrid_boxes(tags, 8, 0, 16)
    # 16^3 level cells = 4^3 blocks of 4, max box 2 blocks: eight 16^3 boxes
    assert len(boxes) == 8
    assert all(tuple(h - l + 1 for l, h in zip(*b)) == (16, 16, 16) for b in boxes)


def test_two_clusters_split_at_hole():
    M = np.zeros((1, 1, 10), dtype=bool)
    M[0, 0, [0, 1, 2, 7, 8]] = True
    out = regrid.br_cluster(M, np.ones_like(M), 100)
    assert out == [((0, 0, 0), (2, 0, 0)), ((7, 0, 0), (8, 0, 0))]


def test_inflection_cut():
    # signature 3 3 3 1 1 1 along x (no holes, low efficiency): second
    # difference 0 -2 2 0 changes sign between i = 2 and 3 -> cut at c = 3
    M = np.zeros((3, 1, 6), dtype=bool)
    M[:, 0, 0:3] = True
    M[0, 0, 3:6] = True
    assert regrid.choose_cut(M) == (0, 3)
    out = regrid.br_cluster(M, np.ones_like(M), 100)
    assert out == [((0, 0, 0), (2, 0, 2)), ((3, 0, 0), (5, 0, 0))]
