"""Parity at the full sizes of the workloads, where the oracle cannot follow
the whole run.  The GPU runs the workload in full and every result is checked
against what the oracle computes from the same snapshots:

* static 2-level AMR (128^3 base plus two ratio-2 levels on fixed boxes around
  a string loop of radius 32 coarse cells, 4th-order Laplacian, quartic
  prolongation, 200 coarse steps, FP64): winding tags of every level bit-exact
  with the oracle's on the ghost-filled state each level holds; every covered
  coarse cell the exact mean of its 8 children; energies and string length
  within 1e-12 of the oracle's on the final snapshot.  The FP32 + Kahan form
  of the same hierarchy, after 100 coarse steps, within 1e-4 relative L2 per
  field and 1 % in string length of the FP64 result (itself pinned to the
  oracle element by element on the smaller hierarchies of test_gpu_amr.py);
* dynamic AMR (256^3 base, blocking factor 16, buffer 4, max box 128, two
  refinement levels, the relaxed c0-style Gaussian field of the dynamic-AMR
  benchmark, FP64): at every regrid the device tags of each level bit-exact
  with the oracle's winding on the snapshot, and the box lists of the next
  level bit-exact with the oracle's regrid (Sec. 2.2-2.3) of those tags;
  restriction exact after the subcycled steps in between;
* the 16-field gravitational-wave lattice on a 128^3 crop (Gaussian psi,
  u = v = 0, 4th order): FP64 within 1e-12 and FP32 + Kahan within 1e-4
  relative L2 of the oracle per field after 3 steps."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import amr as oamr
from oracle import gw as ogw
from oracle import interp as ointerp
from oracle import regrid as oregrid
from oracle import winding as owinding
from paper_2404_02950_gb300 import inputs
from tests.helpers import box_padded_views, oparams, rel_l2

pytestmark = pytest.mark.gpu

G = 3

# ---------------------------------------------------------------------------
# static hierarchy around a string loop

# dx0 = 1/4, dt0 = dx0/4 from eta = 1: after 200 coarse steps (eta = 13.5)
# the radial mode's frequency sqrt(2 lambda) eta times dt0 is 1.2, inside
# RK4's stability interval (with dx0 = 1 it would leave it near eta ~ 11)
C1_N0, C1_DX0, C1_BF, C1_R, C1_ETA0 = 128, 0.25, 8, 32.0, 1.0
C1_DT0 = C1_DX0 / 4
# square rings of 4 boxes around the loop (centre ~(63.75, 63.63, 63.56)
# coarse cells, radius 32): level 1 covers |rho - R| <= 8 and |z - z_c| <= 8
# coarse cells, level 2 |rho - R| <= 4 and |z - z_c| <= 4, both rounded
# outward to the blocking factor (the inner holes inward)
C1_BOXES = [
    [((0, 0, 0), (127, 127, 127))],
    [((40, 40, 104), (207, 95, 143)), ((40, 160, 104), (207, 207, 143)),
     ((40, 96, 104), (95, 159, 143)), ((160, 96, 104), (207, 159, 143))],
    [((104, 104, 232), (399, 175, 271)), ((104, 328, 232), (399, 399, 271)),
     ((104, 176, 232), (175, 327, 271)), ((328, 176, 232), (399, 327, 271))],
]


def _c1_hierarchy(prec):
    h = slh.Hierarchy(C1_N0, C1_DX0, nghost=G, bf=C1_BF, prec=prec, max_levels=3)
    for l in range(3):
        h.init_level(l, C1_BOXES[l])
        vals = inputs.string_loop_boxes(C1_N0, l, C1_BOXES[l], C1_R, C1_ETA0, C1_DX0)
        h.set_state(l, np.concatenate([v.ravel() for v in vals]).astype(h.np_dtype))
    h.set_eta(C1_ETA0)
    return h


def _ghosted(h, lev):
    """Per-box GPU arrays with G ghost layers, (4, nz+2G, ny+2G, nx+2G) FP64."""
    h.sync()
    out = []
    for (lo, hi), v in zip(h.levels[lev]["boxes"], box_padded_views(h, lev)):
        nx = hi[0] - lo[0] + 1
        out.append(v[:4].double().cpu().numpy()[:, :, :, 4 - G:4 + nx + G])
    return out


def _check_tags(h, lev):
    """Device tags (ghosts filled at the synchronised time) against the
    oracle's winding on the very state they saw; returns the count."""
    t, cnt = h.tag(lev)
    exp = np.concatenate([owinding.cell_tags_padded(a[0], a[1], G).ravel() for a in _ghosted(h, lev)])
    assert np.array_equal(t.cpu().numpy(), exp), lev
    assert cnt == int(exp.sum())
    return cnt


def _check_restriction(h, fine_lev, every=1):
    """Every coarse cell under the fine level equals the exact mean of its 8
    children (the oracle's restriction of the fine data)."""
    fb = h.levels[fine_lev]["boxes"]
    cb = h.levels[fine_lev - 1]["boxes"]
    fine = slh.boxes_from_dense(h.get_state(fine_lev), fb)
    coarse = slh.boxes_from_dense(h.get_state(fine_lev - 1), cb)
    checked = 0
    for k in range(0, len(fb), every):
        lo, hi = fb[k]
        red = np.stack([ointerp.restrict_block(fine[k][c]) for c in range(4)])
        clo = [v // 2 for v in lo]
        chi = [(v + 1) // 2 - 1 for v in hi]
        for (blo, bhi), cv in zip(cb, coarse):
            ilo = [max(clo[d], blo[d]) for d in range(3)]
            ihi = [min(chi[d], bhi[d]) for d in range(3)]
            if any(ilo[d] > ihi[d] for d in range(3)):
                continue
            got = cv[:, ilo[2] - blo[2]:ihi[2] - blo[2] + 1, ilo[1] - blo[1]:ihi[1] - blo[1] + 1,
                     ilo[0] - blo[0]:ihi[0] - blo[0] + 1]
            exp = red[:, ilo[2] - clo[2]:ihi[2] - clo[2] + 1, ilo[1] - clo[1]:ihi[1] - clo[1] + 1,
                      ilo[0] - clo[0]:ihi[0] - clo[0] + 1]
            assert np.array_equal(got, exp), (fine_lev, k)
            checked += got.size
    assert checked > 0


def _oracle_from_gpu(h, level_boxes, n0, dx0, dt0, bf, p):
    """An oracle hierarchy holding the GPU's valid cells (ghosts are the
    oracle's own business)."""
    oh = oamr.make_hierarchy(n0, dx0, dt0, G, bf, level_boxes, oparams(p), interp_type=p.interp_type,
                             eta0=h.get_eta(0))
    for l, L in enumerate(oh.levels):
        got = slh.boxes_from_dense(h.get_state(l), L.boxes)
        for b in range(len(L.boxes)):
            L.data[b][L.valid(b)] = got[b]
        L.eta = h.get_eta(l)
    return oh


def test_static_loop_hierarchy_full_size():
    p = slh.EOMParams(order=4, interp_type=4)
    h64 = _c1_hierarchy("f64")
    h32 = _c1_hierarchy("f32")
    for _ in range(100):
        h64.advance(C1_DT0, p)
        h32.advance(C1_DT0, p)
    # FP32 + Kahan against FP64 after 100 coarse steps
    for l in range(3):
        a = slh.boxes_from_dense(h64.get_state(l), C1_BOXES[l])
        b = slh.boxes_from_dense(h32.get_state(l), C1_BOXES[l])
        for k in range(len(C1_BOXES[l])):
            for c in range(4):
                e = rel_l2(b[k][c].astype(np.float64), a[k][c])
                assert e <= 1e-4, (l, k, c, e)
    s64 = h64.reduce_energy(p)[4]
    s32 = h32.reduce_energy(p)[4]
    assert s64 > 0 and abs(s32 - s64) <= 0.01 * s64, (s32, s64)
    h32.close()
    for _ in range(100):
        h64.advance(C1_DT0, p)
    assert h64.get_eta(0) == C1_ETA0 + 200 * C1_DT0
    for l in (1, 2):
        _check_restriction(h64, l)
    for l in range(3):
        _check_tags(h64, l)
    E = h64.reduce_energy(p)
    Eo = _oracle_from_gpu(h64, C1_BOXES, C1_N0, C1_DX0, C1_DT0, C1_BF, p).energy()
    for k in range(4):
        assert abs(E[k] - Eo[k]) <= 1e-12 * max(abs(Eo[k]), 1.0), (k, E[k], Eo[k])
    assert E[4] == Eo[4]
    h64.close()


# ---------------------------------------------------------------------------
# dynamic hierarchy at the dynamic-AMR benchmark's sizes

C3_N, C3_DX, C3_BF, C3_NBUF, C3_MAXBOX, C3_ETA0 = 256, 0.125, 16, 4, 128, 0.1
C3_DT = C3_DX / 4


def _dense_tags(h, lev):
    """Device tags of a level over its whole index domain (after checking them
    against the oracle's winding on the snapshot)."""
    _check_tags(h, lev)
    t, _ = h.tag(lev)
    t = t.cpu().numpy()
    n = C3_N << lev
    out = np.zeros((n, n, n), dtype=np.uint8)
    off = 0
    for lo, hi in h.levels[lev]["boxes"]:
        s = [hi[d] - lo[d] + 1 for d in range(3)]
        out[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = t[off:off + s[0] * s[1] * s[2]].reshape(s[2], s[1], s[0])
        off += s[0] * s[1] * s[2]
    return out


def test_dynamic_hierarchy_full_size_regrids():
    p = slh.EOMParams(order=4, interp_type=4)
    full = [((0, 0, 0), (C3_N - 1,) * 3)]
    y0 = inputs.gaussian_field(C3_N, C3_N / 8.0, 0)
    h = slh.Hierarchy(C3_N, C3_DX, nghost=G, bf=C3_BF, prec="f64", max_levels=3)
    h.init_level(0, full)
    h.set_state(0, slh.dense_from_boxes(y0, full))
    h.set_eta(C3_ETA0)
    for _ in range(100):              # the benchmark's relaxation on the base level
        h.advance(C3_DT, p)
    nboxes = []
    for rnd in range(2):
        for l in range(2):
            tags = _dense_tags(h, l)
            parent = None if l == 0 else [tuple(map(tuple, b)) for b in h.levels[l]["boxes"]]
            exp = oregrid.regrid_boxes(tags, C3_BF, C3_NBUF, C3_MAXBOX, parent_boxes=parent)
            got = h.regrid(l + 2, C3_NBUF, C3_MAXBOX, start=l)
            assert got[0] == exp, (rnd, l)
            nboxes.append(len(exp))
        for _ in range(4):
            h.advance(C3_DT, p)
        _check_restriction(h, 1)
        _check_restriction(h, 2, every=7)
    assert min(nboxes) > 0, nboxes
    h.close()


# ---------------------------------------------------------------------------
# the 16-field lattice on a 128^3 crop

def test_gw_lattice_128_crop():
    n, dx, eta0, steps = 128, 0.125, 0.1, 3
    dt = dx / 4
    p = slh.EOMParams(order=4)
    p1, p2, z, _ = inputs.gaussian_field(n, n / 8.0, 3)
    y = [p1, p2, z, z.copy()] + [np.zeros_like(p1) for _ in range(12)]
    full = [((0, 0, 0), (n - 1,) * 3)]
    exp, eta = tuple(y), eta0
    for _ in range(steps):
        exp = ogw.rk4_step_periodic(exp, eta, dt, dx, oparams(p))
        eta += dt
    for prec, tol in (("f64", 1e-12), ("f32", 1e-4)):
        h = slh.Hierarchy(n, dx, nghost=G, bf=16, prec=prec, max_levels=1, gw=True)
        h.init_level(0, full)
        h.set_state(0, slh.dense_from_boxes(y, full).astype(h.np_dtype))
        h.set_eta(eta0)
        for _ in range(steps):
            h.rk_step(0, dt, p)
        got = slh.boxes_from_dense(h.get_state(0), full, 16)[0]
        for c in range(16):
            assert np.abs(exp[c]).max() > 0, c
            e = rel_l2(got[c].astype(np.float64), exp[c])
            assert e <= tol, (prec, c, e)
        h.close()
