"""GPU vs oracle parity on uniform periodic lattices (one level): the fused
RK4 stage kernels (Laplacian + RHS of Sec. 3.1 + RK4), the fused and
standalone winding tags, and the energy reduction.

Tolerances: FP64 fields within 1e-12 relative L2 of the oracle after 100
steps (the two sides differ only in rounding order and FMA contraction);
tags bit-exact on identical snapshots; FP32 + Kahan fields within 1e-4
relative L2 of the FP64 oracle and string length within 1%."""
import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import energy as oenergy
from oracle import rk4 as ork4
from oracle import winding as owinding
from paper_2404_02950_gb300 import inputs
from tests.helpers import (box_padded_views, download_domain, oparams, rel_l2, tags_domain, uniform_hierarchy,
                           upload)

pytestmark = pytest.mark.gpu

# the 64^3 plain-method workload with dx read as 1/8 (dt = dx/4, eta 0.1 -> 3.225)
N0, DX0, ETA0 = 64, 0.125, 0.1
DT0 = DX0 / 4


def _config0_fields(n=N0, seed=0):
    return inputs.gaussian_field(n, n / 8.0, seed)


def test_config0_f64_100_steps_fields_and_tags():
    p = slh.EOMParams(order=2)
    y0 = _config0_fields()
    h, boxes = uniform_hierarchy(N0, DX0, prec="f64", nghost=1, bf=8, fused_tags=True)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    op = oparams(p)
    y, eta = y0, ETA0
    tag_checks = 0
    for step in range(100):
        snap = download_domain(h, 0, boxes, N0) if step % 10 == 0 else None
        h.rk_step(0, DT0, p, flags=slh.SLH_FUSE_TAG)
        if snap is not None:
            gtags = tags_domain(h.fused_tags(0), boxes, N0)
            assert np.array_equal(gtags, owinding.cell_tags_periodic(snap[0], snap[1])), step
            tag_checks += 1
        y = ork4.rk4_step_periodic(y, eta, DT0, DX0, op)
        eta = eta + DT0
    g = download_domain(h, 0, boxes, N0)
    for c in range(4):
        assert rel_l2(g[c], y[c]) <= 1e-12, (c, rel_l2(g[c], y[c]))
    assert h.get_eta(0) == eta
    assert tag_checks == 10


@pytest.mark.parametrize("order", [4, 6])
def test_high_order_f64_multibox_ragged(order):
    """A 48^3 level split into uneven boxes (ragged tiles, same-level ghost
    copies across boxes and the periodic wrap)."""
    n, dx = 48, 0.2
    boxes = [((0, 0, 0), (15, 47, 47)), ((16, 0, 0), (47, 15, 47)), ((16, 16, 0), (47, 47, 15)),
             ((16, 16, 16), (47, 47, 47))]
    p = slh.EOMParams(order=order, lam=1.0, a=0.05)
    y0 = inputs.gaussian_field(n, 6.0, seed=3)
    y0 = (y0[0], y0[1], 0.3 * y0[1], -0.2 * y0[0])
    h, _ = uniform_hierarchy(n, dx, prec="f64", nghost=3, bf=16, boxes=boxes)
    upload(h, 0, y0, boxes)
    h.set_eta(0.7)
    y, eta = y0, 0.7
    for _ in range(10):
        h.rk_step(0, 0.05, p)
        y = ork4.rk4_step_periodic(y, eta, 0.05, dx, oparams(p))
        eta += 0.05
    g = download_domain(h, 0, boxes, n)
    for c in range(4):
        assert rel_l2(g[c], y[c]) <= 1e-12


def test_frozen_friction_free_energy_conservation_on_gpu():
    n, dx = 32, 0.25
    p = slh.EOMParams(order=4, friction=False, eta_power=0, lam=1.0)
    y0 = inputs.gaussian_field(n, 4.0, seed=9)
    h, boxes = uniform_hierarchy(n, dx, prec="f64")
    upload(h, 0, y0, boxes)
    h.set_eta(1.0)
    E0 = h.reduce_energy(p)
    assert abs(E0[3] - oenergy.energy_periodic(y0, 1.0, dx, oparams(p))[3]) <= 1e-12 * abs(E0[3])
    drift = []
    for dt in (0.04, 0.02):
        upload(h, 0, y0, boxes)
        for _ in range(int(round(0.8 / dt))):
            h.rk_step(0, dt, p)
        drift.append(abs(h.reduce_energy(p)[3] - E0[3]))
    assert 10.0 < drift[0] / drift[1] < 40.0, drift


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_energy_and_tags_match_oracle_on_snapshot(prec):
    n, dx = 40, 0.125
    p = slh.EOMParams(order=6, a=0.1)
    y0 = inputs.gaussian_field(n, 5.0, seed=1)
    y0 = (y0[0], y0[1], 0.5 * y0[0], 0.25 * y0[1])
    boxes = [((0, 0, 0), (39, 39, 19)), ((0, 0, 20), (39, 39, 39))]
    h, _ = uniform_hierarchy(n, dx, prec=prec, nghost=3, bf=4, boxes=boxes, fused_tags=True)
    upload(h, 0, y0, boxes)
    h.set_eta(2.5)
    snap = download_domain(h, 0, boxes, n)      # exactly what the GPU holds (FP32 rounded)
    E = h.reduce_energy(p)
    Eo = oenergy.energy_periodic(snap, 2.5, dx, oparams(p))
    tol = 1e-12 if prec == "f64" else 2e-6
    for k in range(4):
        assert abs(E[k] - Eo[k]) <= tol * max(abs(Eo[k]), 1e-300), (k, E[k], Eo[k])
    assert E[4] == Eo[4]
    t, cnt = h.tag(0)
    otags = owinding.cell_tags_periodic(snap[0], snap[1])
    assert np.array_equal(tags_domain(t.cpu().numpy(), boxes, n), otags)
    assert cnt == int(otags.sum())
    # fused energy of stage 1 equals the standalone reduction of the same state
    h.rk_step(0, 0.01, p, flags=slh.SLH_FUSE_ENERGY)
    Ef = h.reduce_energy(p, mode=1)
    for k in range(4):
        assert abs(Ef[k] - E[k]) <= (1e-13 if prec == "f64" else 2e-6) * abs(E[k])
    assert Ef[4] == E[4]


def test_config0_f32_kahan_within_bounds():
    p = slh.EOMParams(order=2)
    y0 = _config0_fields()
    h, boxes = uniform_hierarchy(N0, DX0, prec="f32", nghost=1, bf=8)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    y, eta = y0, ETA0
    for _ in range(100):
        h.rk_step(0, DT0, p)
        y = ork4.rk4_step_periodic(y, eta, DT0, DX0, oparams(p))
        eta += DT0
    g = download_domain(h, 0, boxes, N0)
    errs = [rel_l2(g[c], y[c]) for c in range(4)]
    assert max(errs) <= 1e-4, errs
    Lg = owinding.string_length_periodic(g[0], g[1], DX0)
    Lo = owinding.string_length_periodic(y[0], y[1], DX0)
    assert abs(Lg - Lo) <= 0.01 * Lo


def test_graph_replay_matches_direct_steps():
    n, dx = 32, 0.25
    p = slh.EOMParams(order=4)
    y0 = inputs.gaussian_field(n, 4.0, seed=2)
    ha, boxes = uniform_hierarchy(n, dx, prec="f64")
    hb, _ = uniform_hierarchy(n, dx, prec="f64")
    for h in (ha, hb):
        upload(h, 0, y0, boxes)
        h.set_eta(0.5)
    for _ in range(5):
        ha.advance(0.05, p)
        hb.advance(0.05, p, flags=slh.SLH_USE_GRAPH)
    a = ha.get_state(0)
    b = hb.get_state(0)
    assert np.array_equal(a, b)
    assert ha.get_eta(0) == hb.get_eta(0)


def _local_rk4_center(y, idx, half, eta, dt, dx, op):
    """The oracle's RK4 step at one cell from a periodic patch of the global
    snapshot (the patch is wide enough that its wrap does not reach the centre)."""
    k, j, i = idx
    n = y[0].shape[0]
    rz = np.arange(k - half, k + half + 1) % n
    ry = np.arange(j - half, j + half + 1) % n
    rx = np.arange(i - half, i + half + 1) % n
    patch = tuple(a[np.ix_(rz, ry, rx)] for a in y)
    out = ork4.rk4_step_periodic(patch, eta, dt, dx, op)
    return np.array([o[half, half, half] for o in out])


def _local_tag(y, idx):
    """The oracle's winding tag of one cell from a periodic 5^3 patch."""
    k, j, i = idx
    n = y[0].shape[0]
    r = [np.arange(c - 2, c + 3) % n for c in (k, j, i)]
    t = owinding.cell_tags_padded(y[0][np.ix_(*r)], y[1][np.ix_(*r)], 2)
    return int(t[0, 0, 0])


def _check_sampled(get, y0, n_field, idx, dt, dx, p, prec, tags=None):
    """Sampled cells of one RK4 step (and their tags) against the oracle;
    ``get(c3)`` returns the 4 GPU values at lattice cell c3 and the snapshot
    is periodic with period n_field."""
    half = 4 * 3 + 1
    tol = 1e-12 if prec == "f64" else 1e-5
    for c3 in idx:
        cm = tuple(v % n_field for v in c3)
        exp = _local_rk4_center(y0, cm, half, ETA0, dt, dx, oparams(p))
        got = get(c3)
        scale = max(1.0, float(np.max(np.abs(exp))))
        assert np.max(np.abs(got - exp)) <= tol * scale, (c3, got, exp)
        if tags is not None:
            assert tags(c3) == _local_tag(y0, cm), c3


def _bench_launch(h, p):
    """The launch configuration of the benchmark: both autotuners, then one
    RK4 step with the winding tags and energy fused in stage 1."""
    h.autotune(0, p, reps=2)
    h.autotune(0, p, reps=2, diag=True)
    h.rk_step(0, DX_FULL / 4, p, flags=slh.SLH_FUSE_TAG | slh.SLH_FUSE_ENERGY)


DX_FULL = 0.125


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_512_order6_sampled(prec):
    """512^3, 6th-order Laplacian, one RK4 step in the benchmark's launch
    configuration (autotuned tiles, tags and energy fused in stage 1); 48
    sampled cells computed one by one by the oracle, their tags too."""
    import torch
    n, dx = 512, DX_FULL
    p = slh.EOMParams(order=6)
    y0 = inputs.gaussian_field(n, n / 16.0, seed=0)
    h, boxes = uniform_hierarchy(n, dx, prec=prec, nghost=3, bf=16, fused_tags=True)
    upload(h, 0, y0, boxes)
    h.set_eta(ETA0)
    _bench_launch(h, p)
    g = h.get_state(0).reshape(4, n, n, n)
    tg = h.fused_tags(0).reshape(n, n, n)
    rng = np.random.default_rng(5)
    idx = [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(44)]
    idx += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 3, 0)]
    _check_sampled(lambda c3: g[:, c3[0], c3[1], c3[2]].astype(np.float64), y0, n, idx, dx / 4, dx, p, prec,
                   tags=lambda c3: int(tg[c3]))
    del h
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_max_size_1024_f32_sampled():
    """1024^3 FP32 + Kahan, the largest uniform scalar lattice one GPU holds
    in this form (5 level buffers, 86 GB): the 512^3 Gaussian field tiled
    twice per axis (periodic, so the oracle's patches come from the 512^3
    arrays), written into the level on the device; one RK4 step in the
    benchmark's launch configuration; 24 sampled cells and their tags against
    the oracle, read back one by one."""
    import torch
    n, m, dx = 1024, 512, DX_FULL
    p = slh.EOMParams(order=6)
    y0 = inputs.gaussian_field(m, m / 16.0, seed=2)
    h, boxes = uniform_hierarchy(n, dx, prec="f32", nghost=3, bf=16, fused_tags=True)
    v = box_padded_views(h, 0)[0]
    for c in range(4):
        t = torch.from_numpy(y0[c].astype(np.float32)).to(v.device)
        v[c, 3:3 + n, 3:3 + n, 4:4 + n] = t.repeat(2, 2, 2)
        del t
    torch.cuda.synchronize()
    h.set_eta(ETA0)
    _bench_launch(h, p)
    h.sync()
    out = box_padded_views(h, 0)[0]
    tg = h.fused_tags(0).reshape(n, n, n)
    rng = np.random.default_rng(9)
    idx = [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(20)]
    idx += [(0, 0, 0), (n - 1, n - 1, n - 1), (511, 512, 1023), (1023, 0, 512)]
    _check_sampled(lambda c3: out[:, 3 + c3[0], 3 + c3[1], 4 + c3[2]].double().cpu().numpy(), y0, m, idx,
                   dx / 4, dx, p, "f32", tags=lambda c3: int(tg[c3]))
    del out, v, h
    torch.cuda.empty_cache()


@pytest.mark.parametrize("which", ["both", "diag_only"])
@pytest.mark.parametrize("prec,nvar", [("f64", 3), ("f32", 7)])
def test_every_tile_variant_matches_oracle(prec, nvar, which):
    """Each stage-kernel tile shape the autotuner may pick gives the oracle's
    result (ragged 40-cell boxes, 6th order, fused tags in stage 1), set for
    every stage or for the diagnostics stage 1 alone (plain stages on
    variant 0)."""
    n, dx = 40, 0.125
    p = slh.EOMParams(order=6)
    y0 = inputs.gaussian_field(n, 5.0, seed=4)
    boxes = [((0, 0, 0), (39, 39, 19)), ((0, 0, 20), (39, 39, 39))]
    ref, eta = y0, 0.5
    for _ in range(3):
        ref = ork4.rk4_step_periodic(ref, eta, 0.02, dx, oparams(p))
        eta += 0.02
    otags = owinding.cell_tags_periodic(y0[0], y0[1])
    tol = 1e-12 if prec == "f64" else 1e-5
    for v in range(nvar):
        h, _ = uniform_hierarchy(n, dx, prec=prec, nghost=3, bf=4, boxes=boxes, fused_tags=True)
        if which == "both":
            h.set_tile(0, v)
        else:
            h.set_diag_tile(0, v)
        upload(h, 0, y0, boxes)
        h.set_eta(0.5)
        snap = download_domain(h, 0, boxes, n)
        h.rk_step(0, 0.02, p, flags=slh.SLH_FUSE_TAG)
        assert np.array_equal(tags_domain(h.fused_tags(0), boxes, n),
                              owinding.cell_tags_periodic(snap[0], snap[1])), v
        if prec == "f64":
            assert np.array_equal(tags_domain(h.fused_tags(0), boxes, n), otags)
        for _ in range(2):
            h.rk_step(0, 0.02, p)
        g = download_domain(h, 0, boxes, n)
        for c in range(4):
            assert rel_l2(g[c], ref[c]) <= tol, (v, c, rel_l2(g[c], ref[c]))
        h.close()


def test_autotune_keeps_state_and_picks_a_variant():
    n, dx = 64, 0.125
    p = slh.EOMParams(order=6)
    y0 = inputs.gaussian_field(n, 8.0, seed=6)
    h, boxes = uniform_hierarchy(n, dx, prec="f32", nghost=3, bf=16)
    upload(h, 0, y0, boxes)
    h.set_eta(0.3)
    before = h.get_state(0)
    chosen, ms = h.autotune(0, p, reps=2)
    assert 0 <= chosen < len(ms) and len(ms) == 7 and all(m > 0 for m in ms)   # the FP32 tile variants
    assert ms[chosen] == min(ms)
    assert np.array_equal(before, h.get_state(0))
    # the diagnostics stage is tuned on its own; the fused partials it
    # overwrites are no longer reported
    h.rk_step(0, 0.02, p, flags=slh.SLH_FUSE_ENERGY)
    h.reduce_energy(p, mode=1)
    before = h.get_state(0)
    chosen_d, ms_d = h.autotune(0, p, reps=2, diag=True)
    assert 0 <= chosen_d < len(ms_d) and len(ms_d) == 7 and all(m > 0 for m in ms_d)
    assert ms_d[chosen_d] == min(ms_d)
    assert np.array_equal(before, h.get_state(0))
    with pytest.raises(slh.SlhError) as e:
        h.reduce_energy(p, mode=1)
    assert e.value.code == -7          # STATE


def test_bounded_wait_expiry_is_reported_and_context_survives():
    """A device wait that nothing completes gives up after its poll limit,
    the host reads SLH_ERR_TIMEOUT, and the context keeps working."""
    n, dx = 32, 0.25
    p = slh.EOMParams(order=4)
    y0 = inputs.gaussian_field(n, 4.0, seed=12)
    h, boxes = uniform_hierarchy(n, dx, prec="f32")
    upload(h, 0, y0, boxes)
    h.set_eta(0.5)
    slh._check(slh.lib().slh_selftest_wait_timeout(h.h, 1000))
    with pytest.raises(slh.SlhError) as e:
        h.sync()
    assert e.value.code == -4
    h.sync()                                   # cleared
    h.rk_step(0, 0.05, p)
    ref = ork4.rk4_step_periodic(y0, 0.5, 0.05, dx, oparams(p))
    g = download_domain(h, 0, boxes, n)
    assert max(rel_l2(g[c], ref[c]) for c in range(4)) <= 1e-5


def test_f64_tags_bit_exact_with_extreme_magnitudes():
    """FP64 winding tags where the sign classes of the values cannot stand in
    for the sign of X: products that underflow (subnormal and tiny values) or
    magnitudes outside the range the shortcut trusts, mixed with ordinary
    values and signed zeros.  On every FP64 diagnostics tile the fused tags of
    the state and the standalone tags equal the oracle's on the same snapshot."""
    n, dx = 24, 0.125
    rng = np.random.default_rng(13)
    # a smooth field (about one string per few hundred cells) with 12 % of its
    # values rescaled, signs kept: tiny, subnormal, huge or (signed) zero
    y = inputs.gaussian_field(n, 3.0, seed=5)
    p1, p2 = y[0].copy(), y[1].copy()
    for a in (p1, p2):
        m = rng.random((n, n, n)) < 0.12
        f = rng.choice([1e-200, 1e-320, 1e160, 0.0], size=(n, n, n))
        a[m] = a[m] * f[m]
    z = np.zeros((n, n, n))
    y0 = [p1, p2, z, z.copy()]
    boxes = [((0, 0, 0), (23, 11, 23)), ((0, 12, 0), (23, 23, 23))]
    p = slh.EOMParams(order=4)
    for v in range(3):
        h, _ = uniform_hierarchy(n, dx, prec="f64", nghost=3, bf=4, boxes=boxes, fused_tags=True)
        h.set_diag_tile(0, v)
        upload(h, 0, y0, boxes)
        h.set_eta(0.5)
        snap = download_domain(h, 0, boxes, n)
        with np.errstate(all="ignore"):   # X overflows (inf - inf) on some edges, as on the GPU
            exp = owinding.cell_tags_periodic(snap[0], snap[1])
        assert 0 < int(exp.sum()) < exp.size
        t, cnt = h.tag(0)
        assert np.array_equal(tags_domain(t.cpu().numpy(), boxes, n), exp), v
        assert cnt == int(exp.sum())
        with np.errstate(all="ignore"):
            h.rk_step(0, 0.02, p, flags=slh.SLH_FUSE_TAG)   # the stepped state may overflow; its input's tags count
        assert np.array_equal(tags_domain(h.fused_tags(0), boxes, n), exp), v
        h.close()


@pytest.mark.parametrize("prec,nvar", [("f32", 7), ("f64", 3)])
def test_tags_bit_exact_on_ties_signed_zeros_and_near_ties(prec, nvar):
    """Winding tags where the method meets its degenerate cases: values from a
    small set with signed zeros (Im = +-0 counts as upper, X = 0 on many
    edges), neighbours that are exact multiples of each other (X = 0 across
    crossing edges) and near ties (X tiny but nonzero, the FP32 form's exact
    fallback).  Fused in stage 1 and standalone, on every diagnostics tile,
    bit-exact with the oracle on the same snapshot; ragged boxes."""
    n, dx = 24, 0.125
    rng = np.random.default_rng(11)
    vals = np.array([-2.0, -1.0, -0.5, -0.0, 0.0, 0.5, 1.0, 2.0])
    p1 = rng.choice(vals, size=(n, n, n))
    p2 = rng.choice(vals, size=(n, n, n))
    sh1, sh2 = np.roll(p1, 1, axis=2), np.roll(p2, 1, axis=2)
    m = rng.random((n, n, n)) < 0.25
    s = rng.choice([-1.0, 2.0, 0.5, -0.5], size=(n, n, n))
    p1, p2 = np.where(m, s * sh1, p1), np.where(m, s * sh2, p2)
    q = rng.random((n, n, n)) < 0.15
    p1 = np.where(q, np.roll(p1, 1, axis=1) * (1.0 + 2.0 ** -20), p1)
    p2 = np.where(q, np.roll(p2, 1, axis=1), p2)
    z = np.zeros((n, n, n))
    y0 = [p1, p2, z, z.copy()]
    boxes = [((0, 0, 0), (23, 11, 23)), ((0, 12, 0), (11, 23, 23)), ((12, 12, 0), (23, 23, 15)),
             ((12, 12, 16), (23, 23, 23))]
    p = slh.EOMParams(order=4)
    for v in range(nvar):
        h, _ = uniform_hierarchy(n, dx, prec=prec, nghost=3, bf=4, boxes=boxes, fused_tags=True)
        h.set_diag_tile(0, v)
        upload(h, 0, y0, boxes)
        h.set_eta(0.5)
        snap = download_domain(h, 0, boxes, n)       # the values as stored (FP32: rounded)
        exp = owinding.cell_tags_periodic(snap[0], snap[1])
        assert 0 < int(exp.sum()) < exp.size
        h.rk_step(0, 0.02, p, flags=slh.SLH_FUSE_TAG)
        assert np.array_equal(tags_domain(h.fused_tags(0), boxes, n), exp), v
        # standalone tags of the stepped state
        snap2 = download_domain(h, 0, boxes, n)
        t, cnt = h.tag(0)
        exp2 = owinding.cell_tags_periodic(snap2[0], snap2[1])
        assert np.array_equal(tags_domain(t.cpu().numpy(), boxes, n), exp2), v
        assert cnt == int(exp2.sum())
        h.close()
