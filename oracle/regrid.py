"""Regrid: tagged cells -> box list of the next finer level (Sec. 2.2-2.3).

The paper tags cells, grows the tags by a buffer of ``n_error_buf`` cells,
and clusters them with the Berger-Rigoutsos algorithm through AMReX, boxes
being multiples of the blocking factor and the new level nested inside the
old one with a gap of one fine blocking factor.  It prints no clustering
parameters.  The deterministic reading used here (the library implements the
same steps independently):

1. D = tags dilated by ``nbuf`` cells (cube, periodic wrap).
2. Blocks of r = bf/2 cells of the tagged level (= bf cells of the new
   level); a block is tagged when any of its cells is in D.
3. Allowed blocks: all when there is no parent box list; otherwise the blocks
   inside the parent level's boxes, eroded by one block (cube, periodic).
   M = tagged blocks AND allowed.
4. Clustering of M, recursively on boxes of blocks starting from the whole
   block domain; each box is first shrunk to the bounding box of its tags
   (dropped when empty).  A box is accepted when 10*tags >= 7*volume, every
   side is <= max_box/bf blocks and all its blocks are allowed.  Otherwise it
   is cut in two at plane c (left [0, c), right [c, n)):
     a. at a plane with zero signature (tag count) nearest the centre
        (smallest |2c - n|), over all axes;
     b. else at the strongest sign change of the signature's second
        difference lap[i] = sig[i-1] - 2 sig[i] + sig[i+1]: for
        lap[i] * lap[i+1] < 0 the cut is c = i + 1 with strength
        |lap[i+1] - lap[i]|; largest strength, then smallest |2c - n|;
     c. else in the middle (c = n // 2) of the longest side.
   Remaining ties go to the lowest axis (x < y < z), then the lowest c.
   Accepted boxes are emitted left part first.
5. Boxes in new-level cells: lo = lo_block * bf, hi = (hi_block + 1) * bf - 1,
   sorted by (lo_z, lo_y, lo_x).

Parity: pinned by invariants (every buffered tag covered, disjoint,
blocking-factor aligned, sides within bounds, nested, efficiency met) and by
brute force on small masks -- tests/test_oracle_regrid.py.
"""
from __future__ import annotations

import numpy as np


def dilate_periodic(mask, nbuf: int):
    out = np.asarray(mask, dtype=bool).copy()
    for axis in range(3):
        acc = out.copy()
        for s in range(1, nbuf + 1):
            acc |= np.roll(out, s, axis=axis) | np.roll(out, -s, axis=axis)
        out = acc
    return out


def coarsen_any(mask, r: int):
    nz, ny, nx = mask.shape
    if nz % r or ny % r or nx % r:
        raise ValueError("level extent not divisible by the block size")
    return np.asarray(mask, dtype=bool).reshape(nz // r, r, ny // r, r, nx // r, r).any(axis=(1, 3, 5))


def _shrink(M, lo, hi):
    sub = M[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
    if not sub.any():
        return None
    zs = np.nonzero(sub.any(axis=(1, 2)))[0]
    ys = np.nonzero(sub.any(axis=(0, 2)))[0]
    xs = np.nonzero(sub.any(axis=(0, 1)))[0]
    nlo = (lo[0] + int(xs[0]), lo[1] + int(ys[0]), lo[2] + int(zs[0]))
    nhi = (lo[0] + int(xs[-1]), lo[1] + int(ys[-1]), lo[2] + int(zs[-1]))
    return nlo, nhi


def _signatures(sub):
    # sub is [z, y, x]; axis d = 0 (x), 1 (y), 2 (z)
    return [sub.sum(axis=(0, 1)).astype(np.int64),
            sub.sum(axis=(0, 2)).astype(np.int64),
            sub.sum(axis=(1, 2)).astype(np.int64)]


def choose_cut(sub):
    """(axis, c) for a box whose tags are given by ``sub`` ([z, y, x])."""
    sig = _signatures(sub)
    n = [len(s) for s in sig]
    holes = [(abs(2 * c - n[d]), d, c)
             for d in range(3) for c in range(1, n[d] - 1) if sig[d][c] == 0]
    if holes:
        _, d, c = min(holes)
        return d, c
    infl = []
    for d in range(3):
        if n[d] < 4:
            continue
        s = sig[d]
        lap = [0] * n[d]
        for i in range(1, n[d] - 1):
            lap[i] = int(s[i - 1]) - 2 * int(s[i]) + int(s[i + 1])
        for i in range(1, n[d] - 2):
            if lap[i] * lap[i + 1] < 0:
                c = i + 1
                infl.append((-abs(lap[i + 1] - lap[i]), abs(2 * c - n[d]), d, c))
    if infl:
        _, _, d, c = min(infl)
        return d, c
    d = int(np.argmax(n))      # first maximum = lowest axis on ties
    return d, n[d] // 2


def br_cluster(M, allowed, max_blocks: int, eff_num: int = 7, eff_den: int = 10):
    """Boxes ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)) in block units."""
    M = np.asarray(M, dtype=bool)
    allowed = np.asarray(allowed, dtype=bool)
    out = []

    def rec(lo, hi):
        b = _shrink(M, lo, hi)
        if b is None:
            return
        lo, hi = b
        sub = M[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        vol = n[0] * n[1] * n[2]
        ntag = int(np.count_nonzero(sub))
        ok = (eff_den * ntag >= eff_num * vol and max(n) <= max_blocks and
              bool(allowed[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].all()))
        if ok:
            out.append((lo, hi))
            return
        d, c = choose_cut(sub)
        lhi = list(hi)
        lhi[d] = lo[d] + c - 1
        rlo = list(lo)
        rlo[d] = lo[d] + c
        rec(lo, tuple(lhi))
        rec(tuple(rlo), hi)

    nz, ny, nx = M.shape
    rec((0, 0, 0), (nx - 1, ny - 1, nz - 1))
    return out


def parent_block_mask(parent_boxes, dims, r: int):
    """Blocks (of r cells) lying inside the parent boxes; dims = (nx, ny, nz)."""
    P = np.zeros((dims[2] // r, dims[1] // r, dims[0] // r), dtype=bool)
    for lo, hi in parent_boxes:
        for d in range(3):
            if lo[d] % r or (hi[d] + 1) % r:
                raise ValueError("parent box not aligned to the block size")
        P[lo[2] // r:(hi[2] + 1) // r, lo[1] // r:(hi[1] + 1) // r,
          lo[0] // r:(hi[0] + 1) // r] = True
    return P


def regrid_boxes(tags, bf: int, nbuf: int, max_box: int, parent_boxes=None):
    """New-level boxes from uint8 tags over the tagged level's index domain
    ([z, y, x] array).  ``parent_boxes`` = the tagged level's own boxes (None
    when it covers the periodic domain)."""
    if bf < 2 or bf & (bf - 1):
        raise ValueError("blocking factor must be a power of two >= 2")
    if max_box % bf:
        raise ValueError("max_box must be a multiple of the blocking factor")
    r = bf // 2
    tags = np.asarray(tags)
    B = coarsen_any(dilate_periodic(tags != 0, nbuf), r)
    if parent_boxes is None:
        allowed = np.ones_like(B)
    else:
        P = parent_block_mask(parent_boxes, (tags.shape[2], tags.shape[1], tags.shape[0]), r)
        allowed = ~dilate_periodic(~P, 1)
    M = B & allowed
    blocks = br_cluster(M, allowed, max_box // bf)
    fine = [(tuple(l * bf for l in lo), tuple((h + 1) * bf - 1 for h in hi)) for lo, hi in blocks]
    fine.sort(key=lambda b: (b[0][2], b[0][1], b[0][0]))
    return fine
