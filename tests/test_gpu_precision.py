"""Error of the FP32 + Kahan form against FP64, per result, at the sizes the
benchmark measures (the FP64 GPU path is itself pinned to the oracle: element
by element on small cases, on sampled cells at 512^3, and on the stored
oracle values of the 128^3 crop below).  Bound: 1e-4 relative L2 per field
and 1 % in total string length after 100 or more steps.

* uniform 512^3, 6th-order Laplacian, classic RK4, Gaussian init
  (k_max = pi/(8 dx)), tags and energy fused in stage 1 every step with the
  autotuned tiles: 100 steps;
* the dynamic hierarchy (256^3 base, blocking factor 16, buffer 4, max box
  128, two refinement levels, 4th order, quartic prolongation): 100 coarse
  steps on the base level, then 6 rounds of a global regrid and 4 subcycled
  coarse steps; both forms take the box lists the FP64 run's tags give, so
  that tags which differ near ties cannot make the hierarchies diverge;
* the 16-field gravitational-wave crop (128^3, 4th order, Gaussian psi,
  u = v = 0): 100 steps; the FP64 run against the oracle's stored values
  (tests/golden/gw_crop_128_order4_100steps.json), the FP32 run against the
  FP64 run."""
import json
import os

import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from paper_2404_02950_gb300 import inputs

pytestmark = pytest.mark.gpu

FLAGS = slh.SLH_FUSE_TAG | slh.SLH_FUSE_ENERGY


def _field_errors(h32, h64, lev, ncomp):
    """Relative L2 error per field of level lev (all boxes), on the device."""
    import torch
    a = h32.get_state_device(lev).double()
    b = h64.get_state_device(lev)
    nv = h64.levels[lev]["nvalid"]
    errs = []
    per = [(lo, hi) for lo, hi in h64.levels[lev]["boxes"]]
    # dense layout [box][comp][cells]: gather every box's part of component c
    offs, o = [], 0
    for lo, hi in per:
        v = (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1)
        offs.append((o, v))
        o += ncomp * v
    assert o == ncomp * nv
    for c in range(ncomp):
        num = torch.zeros((), dtype=torch.float64, device=b.device)
        den = torch.zeros((), dtype=torch.float64, device=b.device)
        for o0, v in offs:
            x = a[o0 + c * v:o0 + (c + 1) * v]
            y = b[o0 + c * v:o0 + (c + 1) * v]
            num += torch.sum((x - y) ** 2)
            den += torch.sum(y ** 2)
        errs.append(float(torch.sqrt(num / den)) if float(den) > 0 else float(torch.sqrt(num)))
    return errs


@pytest.mark.slow
def test_uniform_512_order6_f32_vs_f64_100_steps():
    import torch
    n, dx, eta0 = 512, 0.125, 0.1
    dt = dx / 4
    p = slh.EOMParams(order=6)
    full = [((0, 0, 0), (n - 1,) * 3)]
    dense = slh.dense_from_boxes(inputs.gaussian_field(n, n / 16.0, seed=0), full)
    hs = {}
    for prec in ("f64", "f32"):
        h = slh.Hierarchy(n, dx, nghost=3, bf=16, prec=prec, max_levels=1)
        h.init_level(0, full, fused_tags=True)
        h.set_state(0, dense.astype(h.np_dtype))
        h.set_eta(eta0)
        h.autotune(0, p, reps=2)
        h.autotune(0, p, reps=2, diag=True)
        for _ in range(100):
            h.advance(dt, p, flags=FLAGS)
        hs[prec] = h
    del dense
    errs = _field_errors(hs["f32"], hs["f64"], 0, 4)
    assert max(errs) <= 1e-4, errs
    s64 = hs["f64"].reduce_energy(p)[4]
    s32 = hs["f32"].reduce_energy(p)[4]
    assert s64 > 0 and abs(s32 - s64) <= 0.01 * s64, (s32, s64)
    for h in hs.values():
        h.close()
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_dynamic_hierarchy_f32_vs_f64():
    import torch
    n, dx, eta0, bf, nbuf, maxbox = 256, 0.125, 0.1, 16, 4, 128
    dt = dx / 4
    p = slh.EOMParams(order=4, interp_type=4)
    full = [((0, 0, 0), (n - 1,) * 3)]
    dense = slh.dense_from_boxes(inputs.gaussian_field(n, n / 8.0, 0), full)
    hs = {}
    for prec in ("f64", "f32"):
        h = slh.Hierarchy(n, dx, nghost=2, bf=bf, prec=prec, max_levels=3)
        h.init_level(0, full)
        h.set_state(0, dense.astype(h.np_dtype))
        h.set_eta(eta0)
        for _ in range(100):
            h.advance(dt, p)
        hs[prec] = h
    nboxes = []
    for _ in range(6):
        lists = hs["f64"].regrid(3, nbuf, maxbox)
        for l, boxes in enumerate(lists):
            hs["f32"].regrid_level(l + 1, boxes)
        nboxes.append([len(b) for b in lists])
        for _ in range(4):
            for h in hs.values():
                h.advance(dt, p)
    assert all(len(nb) == 2 and min(nb) > 0 for nb in nboxes), nboxes
    for lev in range(3):
        assert hs["f32"].levels[lev]["boxes"] == hs["f64"].levels[lev]["boxes"]
        errs = _field_errors(hs["f32"], hs["f64"], lev, 4)
        assert max(errs) <= 1e-4, (lev, errs)
    s64 = hs["f64"].reduce_energy(p)[4]
    s32 = hs["f32"].reduce_energy(p)[4]
    assert s64 > 0 and abs(s32 - s64) <= 0.01 * s64, (s32, s64)
    for h in hs.values():
        h.close()
    torch.cuda.empty_cache()


def _gw_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "gw_crop_128_order4_100steps.json")) as f:
        return json.load(f)


@pytest.mark.slow
def test_gw_crop_128_100_steps():
    gold = _gw_golden()
    n, dx, eta0, steps = gold["n"], gold["dx"], gold["eta0"], gold["steps"]
    dt = dx / 4
    p = slh.EOMParams(order=gold["order"])
    p1, p2, z, _ = inputs.gaussian_field(n, n / 8.0, gold["seed"])
    full = [((0, 0, 0), (n - 1,) * 3)]
    dense = slh.dense_from_boxes([p1, p2, z, z.copy()] + [np.zeros_like(p1) for _ in range(12)], full)
    hs = {}
    for prec in ("f64", "f32"):
        h = slh.Hierarchy(n, dx, nghost=2, bf=16, prec=prec, max_levels=1, gw=True)
        h.init_level(0, full)
        h.set_state(0, dense.astype(h.np_dtype))
        h.set_eta(eta0)
        for _ in range(steps):
            h.advance(dt, p)
        hs[prec] = h
    # FP64 against the oracle's stored cells and sums of squares
    y = slh.boxes_from_dense(hs["f64"].get_state(0), full, 16)[0]
    vals = np.array(gold["values"])
    scale = [np.sqrt(s / n ** 3) for s in gold["sumsq"]]
    for (cz, cy, cx), v in zip(gold["cells_zyx"], vals):
        for c in range(16):
            assert abs(y[c, cz, cy, cx] - v[c]) <= 1e-12 * max(scale[c], 1e-300), (c, cz, cy, cx)
    for c in range(16):
        assert gold["sumsq"][c] > 0, c
        s = float(np.sum(y[c] ** 2))
        assert abs(s - gold["sumsq"][c]) <= 1e-11 * gold["sumsq"][c], (c, s, gold["sumsq"][c])
    # FP32 + Kahan against FP64, every field
    errs = _field_errors(hs["f32"], hs["f64"], 0, 16)
    assert max(errs) <= 1e-4, errs
    for h in hs.values():
        h.close()
