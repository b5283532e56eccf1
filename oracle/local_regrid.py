"""Local regrid (Sec. 2.3).  Test infrastructure: imported only by tests/,
__graft_entry__.smoke() and bench.py's CPU baseline.

The paper describes the behaviour, not an algorithm: the existing grid is
kept, tagged cells closer than n_error_buf cells to a coarse/fine boundary
make the finer grid expand around them, coarser levels expand where nesting
needs it, and refined volume is never removed.  Reading, on the block
structure of the global regrid (oracle/regrid.py), with r = bf/2:

1. M_l (l < L-1): the blocks of r cells of level l met by the tags of l grown
   by n_error_buf cells (the global regrid's block mask, slh_tag_blocks).
2. C_l: the blocks of r cells of level l covered by level l+1.
3. New blocks of level l+1: M_l and not C_l; one block of r cells of l is one
   block of bf cells of l+1.
4. Nesting closure, for j = L-1 down to 1: every block of level j (old and
   new) needs the r-blocks of level j-1 around it (3 x 3 x 3, periodic)
   inside level j-1; the bf-blocks of level j-1 that hold them and that level
   j-1 lacks are added to it.  Level 0 covers the domain.
5. Each level's box list is its old boxes, unchanged and in their order,
   followed by its new blocks merged along x into runs (runs ordered by z,
   then y, then x; no run crosses the periodic boundary).

RegridPolicy states the paper's rule for falling back from local to global
regrids (the volume thresholds eps_s, eps_w and the cap on consecutive local
regrids).

Parity: pinned (the refined region only grows; every block of M_l ends up
covered by level l+1; nesting holds on every level afterwards; nothing changes
when every grown tag is already covered; minimality: each level's region
equals, cell for cell, the least region the tags and the nesting rule force,
found by a cell-level fixed-point iteration, plus a worked case where one
block too many fails; the policy by worked sequences of volumes) --
tests/test_oracle_local_regrid.py.
"""
from __future__ import annotations

import numpy as np


def _cover(boxes, nbd: int, unit: int) -> np.ndarray:
    """Blocks of ``unit`` cells (nbd per axis, [z, y, x]) inside the boxes."""
    m = np.zeros((nbd, nbd, nbd), dtype=bool)
    for lo, hi in boxes:
        m[lo[2] // unit:(hi[2] + 1) // unit, lo[1] // unit:(hi[1] + 1) // unit, lo[0] // unit:(hi[0] + 1) // unit] = True
    return m


def _runs(new: np.ndarray, unit: int):
    """x-runs of the new blocks as boxes in cells (blocks of ``unit`` cells)."""
    out = []
    nz, ny, nx = new.shape
    for z in range(nz):
        for y in range(ny):
            x = 0
            while x < nx:
                if not new[z, y, x]:
                    x += 1
                    continue
                x0 = x
                while x < nx and new[z, y, x]:
                    x += 1
                out.append(((x0 * unit, y * unit, z * unit), (x * unit - 1, (y + 1) * unit - 1, (z + 1) * unit - 1)))
    return out


def local_regrid(level_boxes, n0: int, bf: int, masks):
    """New box lists of every level.  level_boxes[l]: boxes of level l (level 0
    covers the domain of n0 cells); masks[l] for l < L-1: M_l as a [z, y, x]
    array of blocks of bf/2 cells of level l."""
    L = len(level_boxes)
    r = bf // 2
    n = [n0 << l for l in range(L)]
    # blocks of bf cells per level: existing ones and additions
    have = [_cover(level_boxes[l], n[l] // bf, bf) for l in range(L)]
    new = [np.zeros_like(h) for h in have]
    for l in range(L - 1):
        M = np.asarray(masks[l], dtype=bool)
        C = _cover([((lo[0] // 2, lo[1] // 2, lo[2] // 2), ((hi[0] + 1) // 2 - 1, (hi[1] + 1) // 2 - 1, (hi[2] + 1) // 2 - 1))
                    for lo, hi in level_boxes[l + 1]], n[l] // r, r)
        new[l + 1] |= M & ~C               # r-blocks of l = bf-blocks of l+1
    for j in range(L - 1, 0, -1):
        blocks = have[j] | new[j]           # bf-blocks of j = r-blocks of j-1
        nr = blocks.shape[0]
        need = np.zeros_like(blocks)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    need |= np.roll(blocks, (dz, dy, dx), axis=(0, 1, 2))
        # r-blocks of j-1 -> bf-blocks of j-1 (pairs of r-blocks per axis)
        nb = nr // 2
        needc = need.reshape(nb, 2, nb, 2, nb, 2).any(axis=(1, 3, 5))
        new[j - 1] |= needc & ~have[j - 1]
    new[0][:] = False                        # level 0 covers the domain
    return [list(level_boxes[l]) + _runs(new[l] & ~have[l], bf) for l in range(L)]


class RegridPolicy:
    """When a local regrid gives way to a global one (Sec. 2.3): the volume
    that local regrids added to each level since the last global regrid is
    tracked as a fraction dV_l of the level's volume at that global regrid.
    Once dV_l >= eps_strong on some level (or max_local local regrids have
    run in a row), the next regrid is global, starting at the lowest level
    l >= 1 with dV_l >= eps_weak (that level and the finer ones are rebuilt,
    from the tags of level l - 1); with no such level it starts at level 1.
    A hierarchy with fewer levels than it may have is regridded globally
    (a local regrid never creates a level).  The paper's defaults are
    eps_strong = 10 % and eps_weak = 5 % (its parameter table writes them as
    the volume ratios 1.1 and 1.05) and at most 10 local regrids in a row.

    next_regrid(volumes) -> ("global", l0) or ("local", None), where l0 is the
    level whose tags the global regrid starts from; then after_local(added)
    with the cells each level gained, or after_global()."""

    def __init__(self, max_levels, eps_strong=0.1, eps_weak=0.05, max_local=10):
        self.max_levels = max_levels
        self.eps_strong, self.eps_weak, self.max_local = eps_strong, eps_weak, max_local
        self.base = None

    def next_regrid(self, volumes):
        if self.base is None or len(self.base) != len(volumes):
            self.base = [max(1, int(v)) for v in volumes]
            self.added = [0] * len(volumes)
            self.count = 0
            self.pending = None
        if self.pending is not None:
            return "global", self.pending
        if len(volumes) < self.max_levels:
            return "global", 0
        return "local", None

    def after_local(self, added):
        self.count += 1
        self.added = [a + int(b) for a, b in zip(self.added, added)]
        frac = [a / b for a, b in zip(self.added, self.base)]
        if any(f >= self.eps_strong for f in frac) or (self.max_local and self.count >= self.max_local):
            weak = [l for l in range(1, len(frac)) if frac[l] >= self.eps_weak]
            self.pending = (min(weak) - 1) if weak else 0
        return frac

    def after_global(self):
        self.base = None

