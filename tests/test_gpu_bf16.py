"""BF16 storage of the gravitational-wave tensor (precision SLH_F32_BF16, the
form of the largest single-GPU workload): psi, Pi in FP32, u_ij and v_ij
stored as BF16 pairs, FP32 arithmetic, SSPRK3 on three level buffers.

* psi, Pi equal bit for bit those of the 16-field FP32 run (the scalar stage
  never reads the tensor fields), which the oracle pins to 1e-4;
* u_ij, v_ij within the BF16 bound of the FP64 oracle (uniform lattice) and
  of the FP32 run (subcycled hierarchy with ghost prolongation, restriction
  and regrid of the packed pairs);
* graph replay across the three-buffer rotation equals direct steps;
* the 128^3 crop after 100 steps against the oracle's stored values;
* the spectrum of a BF16 level against the oracle's spectrum of the stored
  (exactly widened) values.
The bound: every stored tensor value carries a relative rounding error of
at most 2^-9; u, v are rounded three times per SSPRK3 step, so after n
steps the relative L2 error stays below 2^-9 sqrt(3 n) times a safety factor
of 4 (errors of successive roundings are uncorrelated and partly damped)."""
import json
import math
import os

import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import gw as ogw
from oracle import gw_spectrum as ogs
from oracle import ssprk3 as ossp
from paper_2404_02950_gb300 import inputs
from tests.helpers import oparams, rel_l2

pytestmark = pytest.mark.gpu

N, DX, DT, ETA0, G, BF = 32, 0.5, 0.125, 1.0, 2, 8
FULL = [((0, 0, 0), (N - 1, N - 1, N - 1))]
P = slh.EOMParams(order=4, integrator=10)


def bf16_bound(steps):
    return 4.0 * 2.0 ** -9 * math.sqrt(3.0 * steps)


def _initial(n=N, dx=DX):
    p1, p2, z, _ = inputs.string_loop(n, 4.0 * (n / N), 2.0, dx)
    tens = []
    for s in range(6):
        a, b, _, _ = inputs.gaussian_field(n, 3.0, 100 + s)
        tens += [0.1 * a, 0.1 * b]
    return [p1, p2, z, z.copy()] + tens[0::2] + tens[1::2]


def _fields(h, lev, boxes):
    """Per-box (16, nz, ny, nx) float64 arrays of a level."""
    nsl = h.nslots
    per = slh.boxes_from_dense(h.get_state(lev), boxes, nsl)
    out = []
    for a in per:
        f = slh.unpack_bf16_fields(list(a)) if h.prec == slh.SLH_F32_BF16 else list(a)
        out.append([np.asarray(x, dtype=np.float64) for x in f])
    return out


def _load(h, lev, fields16, boxes):
    f = slh.pack_bf16_fields(fields16) if h.prec == slh.SLH_F32_BF16 else [np.asarray(a, np.float32) for a in fields16]
    h.set_state(lev, slh.dense_from_boxes(f, boxes))


def _stored(fields16):
    """The values a BF16 level holds for these fields (tensor fields rounded)."""
    return [np.asarray(a, np.float64) for a in slh.unpack_bf16_fields(slh.pack_bf16_fields(fields16))]


def test_uniform_against_fp32_run_and_oracle():
    y = _initial()
    steps = 6
    exp, eta = tuple(np.asarray(a, dtype=np.float64) for a in _stored(y)), ETA0
    for _ in range(steps):
        exp = ossp.ssprk3_step_periodic(exp, eta, DT, DX, oparams(P), f=ogw.f_periodic)
        eta += DT
    got = {}
    for prec in ("f32", "f32bf16"):
        h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec=prec, max_levels=1, gw=True)
        h.init_level(0, FULL)
        _load(h, 0, _stored(y), FULL)
        h.set_eta(ETA0)
        for _ in range(steps):
            h.rk_step(0, DT, P)
        got[prec] = _fields(h, 0, FULL)[0]
        h.close()
    for c in range(4):
        assert np.array_equal(got["f32bf16"][c], got["f32"][c]), c
        assert rel_l2(got["f32bf16"][c], exp[c]) <= 1e-4, c
    errs = [rel_l2(got["f32bf16"][c], exp[c]) for c in range(4, 16)]
    assert max(errs) <= bf16_bound(steps), errs
    assert min(errs) > 0.0                      # the tensor fields really are rounded
    assert rel_l2(exp[4], _stored(y)[4]) > 1e-3     # and moved


LEVEL_BOXES = [
    [((0, 0, 0), (31, 31, 31))],
    [((16, 16, 16), (31, 47, 47)), ((32, 16, 16), (47, 47, 47))],
]
NEW_L1 = [((16, 16, 16), (47, 31, 47)), ((16, 32, 16), (47, 47, 47)), ((48, 16, 16), (55, 47, 47))]


@pytest.mark.parametrize("use_graph", [False, True])
def test_hierarchy_regrid_against_fp32_run(use_graph):
    """Two levels, subcycled SSPRK3 steps, a regrid of level 1 (copy where the
    old boxes cover, prolongation elsewhere), more steps: scalars bit for bit
    with the FP32 run, tensor fields within the bound."""
    y = _stored(_initial())
    res = {}
    for prec in ("f32", "f32bf16"):
        h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec=prec, max_levels=2, gw=True)
        h.init_level(0, LEVEL_BOXES[0])
        _load(h, 0, y, LEVEL_BOXES[0])
        h.set_eta(ETA0)
        h.regrid_level(1, LEVEL_BOXES[1])
        flags = slh.SLH_USE_GRAPH if use_graph else 0
        for _ in range(3):
            h.advance(DT, P, flags=flags)
        h.regrid_level(1, NEW_L1)
        for _ in range(3):
            h.advance(DT, P, flags=flags)
        res[prec] = [_fields(h, l, h.levels[l]["boxes"]) for l in (0, 1)]
        h.close()
    for l in (0, 1):
        for a, b in zip(res["f32bf16"][l], res["f32"][l]):
            for c in range(4):
                assert np.array_equal(a[c], b[c]), (l, c)
            for c in range(4, 16):
                assert rel_l2(a[c], b[c]) <= bf16_bound(6 * 2 ** l), (l, c, rel_l2(a[c], b[c]))


def test_graph_replay_equals_direct_steps():
    y = _stored(_initial())
    outs = []
    for use_graph in (False, True):
        h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f32bf16", max_levels=2, gw=True)
        h.init_level(0, LEVEL_BOXES[0])
        _load(h, 0, y, LEVEL_BOXES[0])
        h.set_eta(ETA0)
        h.regrid_level(1, LEVEL_BOXES[1])
        for _ in range(4):   # more than one turn of the three-buffer rotation
            h.advance(DT, P, flags=slh.SLH_USE_GRAPH if use_graph else 0)
        outs.append([h.get_state(l) for l in (0, 1)])
        h.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_three_buffers_only():
    """A BF16 level holds three buffers; integrators other than SSPRK3 are
    refused."""
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f32bf16", max_levels=1, gw=True)
    info = h.init_level(0, FULL)
    assert info["bufs"][slh.SLH_BUF_D] is None and info["bufs"][slh.SLH_BUF_C] is None
    with pytest.raises(slh.SlhError) as e:
        h.rk_step(0, DT, slh.EOMParams(order=4, integrator=4))
    assert e.value.code == -1
    h.close()


def test_spectrum_of_bf16_level():
    y = _initial()
    st = _stored(y)
    h = slh.Hierarchy(N, DX, nghost=G, bf=BF, prec="f32bf16", max_levels=1, gw=True)
    h.init_level(0, FULL)
    _load(h, 0, y, FULL)
    n2, g = h.gw_spectrum(2)
    en2, eg = ogs.spectrum(st[10:16], DX, 2)
    assert np.array_equal(n2, en2) and np.max(np.abs(g - eg)) <= 1e-5 * np.max(np.abs(eg))
    h.close()


@pytest.mark.slow
def test_crop_128_100_steps_against_stored_oracle():
    with open(os.path.join(os.path.dirname(__file__), "golden", "gw_crop_128_order4_100steps_ssprk3.json")) as f:
        gold = json.load(f)
    n, dx, eta0, steps = gold["n"], gold["dx"], gold["eta0"], gold["steps"]
    p = slh.EOMParams(order=gold["order"], integrator=10)
    p1, p2, z, _ = inputs.gaussian_field(n, n / 8.0, gold["seed"])
    full = [((0, 0, 0), (n - 1,) * 3)]
    h = slh.Hierarchy(n, dx, nghost=2, bf=16, prec="f32bf16", max_levels=1, gw=True)
    h.init_level(0, full)
    _load(h, 0, [p1, p2, z, z.copy()] + [np.zeros_like(p1)] * 12, full)
    h.set_eta(eta0)
    for _ in range(steps):
        h.advance(dx / 4, p)
    y = _fields(h, 0, full)[0]
    cells = gold["cells_zyx"]
    vals = np.array(gold["values"])
    for c in range(16):
        got = np.array([y[c][cz, cy, cx] for cz, cy, cx in cells])
        scale = math.sqrt(gold["sumsq"][c] / n ** 3)
        err = np.linalg.norm(got - vals[:, c]) / (scale * math.sqrt(len(cells)))
        bound = 1e-4 if c < 4 else bf16_bound(steps)
        assert err <= bound, (c, err, bound)
        s = float(np.sum(y[c] ** 2))
        assert abs(s - gold["sumsq"][c]) <= (1e-4 if c < 4 else 2 * bf16_bound(steps)) * gold["sumsq"][c], c
    h.close()
