"""String-winding refinement tags (the problem-specific tagging hook of
Sec. 4.2, ``TagCellForRefinement``).

The paper provides the hook but not the axion-string criterion.  Reading used
here (integer, sign-only, so both implementations agree bit for bit):

* A plaquette is the unit square with lower corner p and normal e_w, its
  corners z0 = p, z1 = p + e_u, z2 = p + e_u + e_v, z3 = p + e_v traversed
  counter-clockwise about +e_w, with (u, v, w) cyclic: (x, y, z), (y, z, x),
  (z, x, y).  It is owned by cell p.
* For an edge a -> b of psi = psi1 + i psi2, with up(z) = (Im z >= 0) and
  X = Re a * Im b - Im a * Re b (two rounded products and one subtraction):
      delta = +1  if up(a) and not up(b) and X > 0
      delta = -1  if not up(a) and up(b) and X < 0
      delta =  0  otherwise.
  W = sum of delta over the four edges is the number of times the phase,
  taking the shorter way along each edge, crosses the negative real axis
  counter-clockwise -- the winding number whenever no edge is exactly
  antipodal (X = 0 with opposite signs counts 0).
* A cell is tagged when any of the 12 plaquettes it is a corner of has W != 0.
* String length = (number of plaquettes with W != 0) * dx.

For FP32 fields the products of two FP32 numbers are exact in FP64, so X is
formed in FP64 from the FP32 values and its sign is exact.

Parity: pinned (straight string through an off-lattice point gives +1 on the
one pierced plaquette per layer and 0 elsewhere, -1 reversed; circular loop;
brute force against wrapped atan2 phase sums on 8^3) --
tests/test_oracle_winding.py.
"""
from __future__ import annotations

import numpy as np

# (u, v) axes of numpy [z, y, x] arrays for each plaquette normal w
_ORIENT = {
    "z": (2, 1),   # normal z: u = x, v = y
    "x": (1, 0),   # normal x: u = y, v = z
    "y": (0, 2),   # normal y: u = z, v = x
}


def edge_delta(ar, ai, br, bi):
    ar = np.asarray(ar, dtype=np.float64)
    ai = np.asarray(ai, dtype=np.float64)
    br = np.asarray(br, dtype=np.float64)
    bi = np.asarray(bi, dtype=np.float64)
    X = ar * bi - ai * br
    ua = ai >= 0.0
    ub = bi >= 0.0
    plus = ua & ~ub & (X > 0.0)
    minus = ~ua & ub & (X < 0.0)
    return plus.astype(np.int32) - minus.astype(np.int32)


def _shift(f, axis, periodic):
    if periodic:
        return np.roll(f, -1, axis=axis)
    sl = [slice(None)] * 3
    sl[axis] = slice(1, None)
    return f[tuple(sl)]


def _crop(f, shape):
    return f[:shape[0], :shape[1], :shape[2]]


def plaquette_winding(psi1, psi2, periodic=True):
    """W for the three plaquette normals, indexed by owner cell.

    periodic=True: arrays of the full lattice shape (wrap-around corners).
    periodic=False: owners are the cells whose plaquette corners all lie in
    the array, i.e. shape (n-1) along the two in-plane axes (all along the
    normal axis is kept, then cropped to n-1 on every axis for uniformity).
    Returns a dict {'x': Wx, 'y': Wy, 'z': Wz} of int32 arrays.
    """
    psi1 = np.asarray(psi1, dtype=np.float64)
    psi2 = np.asarray(psi2, dtype=np.float64)
    out = {}
    for w, (u, v) in _ORIENT.items():
        c0r, c0i = psi1, psi2
        c1r, c1i = _shift(psi1, u, periodic), _shift(psi2, u, periodic)
        c3r, c3i = _shift(psi1, v, periodic), _shift(psi2, v, periodic)
        c2r = _shift(_shift(psi1, u, periodic), v, periodic)
        c2i = _shift(_shift(psi2, u, periodic), v, periodic)
        if not periodic:
            shp = tuple(s - 1 for s in psi1.shape)
            c0r, c0i, c1r, c1i, c2r, c2i, c3r, c3i = (
                _crop(a, shp) for a in (c0r, c0i, c1r, c1i, c2r, c2i, c3r, c3i))
        W = (edge_delta(c0r, c0i, c1r, c1i) + edge_delta(c1r, c1i, c2r, c2i)
             + edge_delta(c2r, c2i, c3r, c3i) + edge_delta(c3r, c3i, c0r, c0i))
        out[w] = W
    return out


def cell_tags_periodic(psi1, psi2):
    """uint8 tag per lattice cell (periodic lattice)."""
    W = plaquette_winding(psi1, psi2, periodic=True)
    tag = np.zeros(np.shape(psi1), dtype=bool)
    for w, (u, v) in _ORIENT.items():
        nz = W[w] != 0
        # cell c is a corner of the plaquettes owned by c, c-e_u, c-e_v, c-e_u-e_v
        tag |= nz
        tag |= np.roll(nz, 1, axis=u)
        tag |= np.roll(nz, 1, axis=v)
        tag |= np.roll(np.roll(nz, 1, axis=u), 1, axis=v)
    return tag.astype(np.uint8)


def cell_tags_padded(psi1p, psi2p, g):
    """Tags of the valid cells of a ghost-padded box (g >= 1 ghost layers).

    Uses the plaquettes owned by the valid cells and by their lower
    neighbours (which reach one ghost layer below and above)."""
    if g < 1:
        raise ValueError("winding tags need at least one ghost layer")
    W = plaquette_winding(psi1p, psi2p, periodic=False)   # owners 0..n_pad-2
    nz, ny, nx = (s - 2 * g for s in np.shape(psi1p))
    tag = np.zeros((nz, ny, nx), dtype=bool)
    for w, (u, v) in _ORIENT.items():
        nzw = W[w] != 0
        for du in (0, 1):
            for dv in (0, 1):
                off = [g, g, g]
                off[u] -= du
                off[v] -= dv
                tag |= nzw[off[0]:off[0] + nz, off[1]:off[1] + ny, off[2]:off[2] + nx]
    return tag.astype(np.uint8)


def pierced_count_padded(psi1p, psi2p, g, owner_mask=None):
    """Number of plaquettes with W != 0 owned by valid cells of a padded box
    (optionally only owners where ``owner_mask`` is True)."""
    W = plaquette_winding(psi1p, psi2p, periodic=False)
    nz, ny, nx = (s - 2 * g for s in np.shape(psi1p))
    total = 0
    for w in ("x", "y", "z"):
        nzw = W[w][g:g + nz, g:g + ny, g:g + nx] != 0
        if owner_mask is not None:
            nzw = nzw & owner_mask
        total += int(np.count_nonzero(nzw))
    return total


def string_length_periodic(psi1, psi2, dx):
    W = plaquette_winding(psi1, psi2, periodic=True)
    return sum(int(np.count_nonzero(W[w])) for w in W) * dx
