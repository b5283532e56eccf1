"""Pins of the oracle's level hierarchy (Sec. 2.1): subcycling of a fine
level that covers the whole domain must reproduce a uniform fine run bit for
bit and restrict exactly onto the coarse level; ghost cells prolonged from a
polynomial coarse field must equal its exact fine cell averages."""
import numpy as np
import pytest

from oracle import amr, interp, rk4, rkn4, rkn5, ssprk3
from oracle.eom import EOMParams
from paper_2404_02950_gb300 import inputs


@pytest.mark.parametrize("order,integrator,ko_order", [(2, 4, 0), (4, 4, 0), (4, 10, 0), (4, 4, 5), (4, 21, 0),
                                                           (4, 22, 0)])
def test_full_cover_fine_level_equals_uniform_fine_run(order, integrator, ko_order):
    n0, dx0, dt0, g, bf = 8, 0.25, 1.0 / 16, 3, 4
    p = EOMParams(order=order, ko_order=ko_order, ko_eps=0.05 if ko_order else 0.0,
                  friction=integrator != 22)    # RKN5: velocity-independent acceleration
    eta0 = 0.5                       # dyadic times keep eta sums exact
    fine0 = inputs.random_snapshot(16, seed=4, amp=0.8)
    coarse0 = [interp.restrict_block(f) for f in fine0]
    h = amr.make_hierarchy(n0, dx0, dt0, g, bf,
                           [[((0, 0, 0), (7, 7, 7))],
                            [((0, 0, 0), (7, 15, 15)), ((8, 0, 0), (15, 7, 15)),
                             ((8, 8, 0), (15, 15, 15))]],
                           p, interp_type=4, eta0=eta0, integrator=integrator)
    h.levels[0].set_dense(coarse0)
    h.levels[1].set_dense(fine0)
    nsteps = 2
    for _ in range(nsteps):
        h.step()
    if integrator == 4:
        ref, _ = rk4.evolve_periodic(fine0, eta0, dt0 / 2, dx0 / 2, 2 * nsteps, p)
    else:
        step = {21: rkn4.rkn4_step_periodic, 22: rkn5.rkn5_step_periodic}.get(integrator, ssprk3.ssprk3_step_periodic)
        ref, eta = fine0, eta0
        for _ in range(2 * nsteps):
            ref = step(ref, eta, dt0 / 2, dx0 / 2, p)
            eta += dt0 / 2
    L1 = h.levels[1]
    for b, (lo, hi) in enumerate(L1.boxes):
        got = L1.data[b][L1.valid(b)]
        for c in range(4):
            exp = ref[c][lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
            assert np.array_equal(got[c], exp)
    L0 = h.levels[0]
    got0 = L0.data[0][L0.valid(0)]
    for c in range(4):
        assert np.array_equal(got0[c], interp.restrict_block(ref[c]))
    assert L0.eta == L1.eta == eta0 + nsteps * dt0


def _avg_poly(coef, lo, hi):
    return sum(c * (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo)) for p, c in enumerate(coef))


def test_ghost_prolongation_exact_for_polynomials_with_time_interp():
    n0, g, bf = 16, 3, 4
    p = EOMParams(order=6)
    h = amr.make_hierarchy(n0, 1.0, 0.25, g, bf,
                           [[((0, 0, 0), (15, 15, 15))], [((12, 8, 12), (19, 23, 19))]],
                           p, interp_type=4, eta0=1.0)
    rng = np.random.default_rng(7)
    polys = [[[float(v) / 8 for v in rng.integers(-8, 8, size=5)] for _ in range(3)] for _ in range(2)]

    def coarse_avgs(P):
        px, py, pz = P
        ax = np.arange(n0, dtype=np.float64)
        ax_ = [_avg_poly(px, i - 0.5, i + 0.5) for i in ax]
        ay_ = [_avg_poly(py, i - 0.5, i + 0.5) for i in ax]
        az_ = [_avg_poly(pz, i - 0.5, i + 0.5) for i in ax]
        return np.einsum("k,j,i->kji", az_, ay_, ax_)

    C0 = h.levels[0]
    old = coarse_avgs(polys[0])
    new = coarse_avgs(polys[1])
    C0.set_dense([old, old, old, old])
    C0.old = [a.copy() for a in C0.data]
    C0.set_dense([new, new, new, new])
    alpha = 0.25
    F = h.levels[1]
    arrs = [a.copy() for a in F.data]
    amr.fill_ghosts(F, arrs, C0, alpha, 4)
    lo, hi = F.boxes[0]
    a = arrs[0]
    checked = 0
    for pz_ in range(a.shape[1]):
        for py_ in range(a.shape[2]):
            for px_ in range(a.shape[3]):
                if g <= pz_ < a.shape[1] - g and g <= py_ < a.shape[2] - g and g <= px_ < a.shape[3] - g:
                    continue
                f = (px_ + lo[0] - g, py_ + lo[1] - g, pz_ + lo[2] - g)
                exp = 0.0
                for wgt, P in ((1 - alpha, polys[0]), (alpha, polys[1])):
                    e = 1.0
                    for d in range(3):
                        e *= _avg_poly(P[d], f[d] / 2 - 0.5, f[d] / 2)
                    exp += wgt * e
                assert abs(a[0][pz_, py_, px_] - exp) <= 1e-12 * max(1.0, abs(exp))
                checked += 1
    assert checked == a.shape[1] * a.shape[2] * a.shape[3] - 8 * 16 * 8


def test_nesting_violation_raises():
    h = amr.make_hierarchy(8, 1.0, 0.25, 3, 4,
                           [[((0, 0, 0), (3, 7, 7))], [((0, 0, 0), (3, 3, 3))]],
                           EOMParams(), interp_type=4, eta0=1.0)
    arrs = [a.copy() for a in h.levels[1].data]
    h.levels[0].old = h.levels[0].data
    with pytest.raises(ValueError):
        amr.fill_ghosts(h.levels[1], arrs, h.levels[0], 0.0, 4)


# Exact symmetries of the subcycled hierarchy (no closed form exists for it):
# a lattice translation of boxes and data by whole blocks, and the rotation
# (psi1, psi2) -> (-psi2, psi1) in field space, under which the equations of
# Sec. 3.1 are invariant.  Both commute with every rounding the scheme does
# (relabelled cells; exact negation, commutative sums), so the shifted or
# rotated run equals the shifted or rotated original bit for bit.
SYM_BOXES = [[((0, 0, 0), (15, 15, 15))],
             [((8, 8, 4), (19, 23, 23)), ((20, 8, 4), (23, 15, 23))],
             [((24, 24, 20), (31, 39, 27))]]
SYM_CASES = [(4, 0, True, 4), (10, 0, True, 4), (21, 0, True, 4), (22, 0, False, 4), (4, 3, True, 4),
             (4, 0, True, 1)]


def _sym_run(boxes, fields, integrator, ko_order, friction, itype, nsteps=2):
    p = EOMParams(order=4, ko_order=ko_order, ko_eps=0.05 if ko_order else 0.0, friction=friction)
    h = amr.make_hierarchy(16, 0.5, 0.125, 3, 4, boxes, p, interp_type=itype, eta0=0.75, integrator=integrator)
    for L, f in zip(h.levels, fields):
        L.set_dense(f)
    for _ in range(nsteps):
        h.step()
    return h


def _sym_fields(seed):
    return [inputs.random_snapshot(16 * 2 ** l, seed=seed + l, amp=0.8) for l in range(3)]


@pytest.mark.parametrize("integrator,ko_order,friction,itype", SYM_CASES)
def test_hierarchy_translation_invariance(integrator, ko_order, friction, itype):
    s0 = (4, 4, 0)                                    # (x, y, z) coarse cells: whole blocks on every level
    fields = _sym_fields(21)
    ref = _sym_run(SYM_BOXES, fields, integrator, ko_order, friction, itype)
    boxes, moved = [], []
    for l, (bl, fl) in enumerate(zip(SYM_BOXES, fields)):
        s = [c * 2 ** l for c in s0]
        boxes.append(bl if l == 0 else [(tuple(a + d for a, d in zip(lo, s)), tuple(a + d for a, d in zip(hi, s)))
                                        for lo, hi in bl])
        moved.append([np.roll(a, shift=(s[2], s[1], s[0]), axis=(0, 1, 2)) for a in fl])
    got = _sym_run(boxes, moved, integrator, ko_order, friction, itype)
    for l, (Lr, Lg) in enumerate(zip(ref.levels, got.levels)):
        s = [c * 2 ** l for c in s0]
        for b in range(len(Lr.boxes)):
            vr, vg = Lr.data[b][Lr.valid(b)], Lg.data[b][Lg.valid(b)]
            if l == 0:                                # the one periodic box: compare rolled
                vr = np.stack([np.roll(a, shift=(s[2], s[1], s[0]), axis=(0, 1, 2)) for a in vr])
            assert np.array_equal(vr, vg), (l, b)


@pytest.mark.parametrize("integrator,ko_order,friction,itype", SYM_CASES)
def test_hierarchy_field_rotation_invariance(integrator, ko_order, friction, itype):
    fields = _sym_fields(33)
    ref = _sym_run(SYM_BOXES, fields, integrator, ko_order, friction, itype)
    rot = [(-f[1], f[0], -f[3], f[2]) for f in fields]
    got = _sym_run(SYM_BOXES, rot, integrator, ko_order, friction, itype)
    for l, (Lr, Lg) in enumerate(zip(ref.levels, got.levels)):
        for b in range(len(Lr.boxes)):
            vr, vg = Lr.data[b][Lr.valid(b)], Lg.data[b][Lg.valid(b)]
            for a, e in ((vg[0], -vr[1]), (vg[1], vr[0]), (vg[2], -vr[3]), (vg[3], vr[2])):
                assert np.array_equal(a, e), (l, b)


@pytest.mark.parametrize("integrator", [4, 10, 21, 22])
def test_linear_in_time_field_pins_the_stage_time_fractions(integrator):
    """With lambda = a = 0 and no friction, psi = psi0 + v t (constant in
    space) solves the equations, and prolongation of constants and linear
    time interpolation are exact: every level of a three-level hierarchy
    stays at psi0 + v t through the subcycled steps.  A fine ghost taken at
    the wrong fraction of the coarse step differs from the interior by v
    times the time error, which the Laplacian turns into a visible error."""
    p = EOMParams(lam=0.0, a=0.0, friction=False, eta_power=0, order=4)
    h = amr.make_hierarchy(16, 0.5, 0.125, 3, 4, SYM_BOXES, p, interp_type=4, eta0=0.75, integrator=integrator)
    psi0, v = (0.3, -0.2), (1.25, 0.5)
    for L in h.levels:
        n = L.n
        L.set_dense([np.full((n, n, n), psi0[0]), np.full((n, n, n), psi0[1]),
                     np.full((n, n, n), v[0]), np.full((n, n, n), v[1])])
    t = 0.0
    for _ in range(2):
        h.step()
        t += 0.125
    for L in h.levels:
        for b in range(len(L.boxes)):
            got = L.data[b][L.valid(b)]
            for c in range(2):
                assert np.max(np.abs(got[c] - (psi0[c] + v[c] * t))) < 1e-14, (L, b, c)
                assert np.max(np.abs(got[2 + c] - v[c])) < 1e-14


def _set_level_fields(h, fn):
    """Fields from fn(x, y, z) at the cell centres of each level, in level-0
    lattice units (a level-l cell i sits at (i + 1/2) / 2^l - 1/2)."""
    for lev, L in enumerate(h.levels):
        r = float(1 << lev)
        ax = (np.arange(L.n, dtype=np.float64) + 0.5) / r - 0.5
        z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
        L.set_dense(fn(x, y, z))


def test_hierarchy_energy_of_a_constant_field_is_density_times_volume():
    """Every cell of the domain counted once, whatever the box layout: the
    energy of a constant state is the closed-form density times the domain
    volume (the gradient part vanishes)."""
    p = EOMParams(lam=1.0, a=0.3, friction=True, eta_power=2, order=4)
    h = amr.make_hierarchy(16, 0.5, 0.125, 3, 4, SYM_BOXES, p, interp_type=4, eta0=0.75)
    psi, pi = (0.6, -0.3), (0.2, 0.1)
    _set_level_fields(h, lambda x, y, z: [np.full(x.shape, v) for v in psi + pi])
    K, G, P, T, S = h.energy()
    r2 = psi[0] ** 2 + psi[1] ** 2
    vol = (16 * 0.5) ** 3
    kin = 0.5 * (pi[0] ** 2 + pi[1] ** 2) * vol
    pot = ((p.lam * 0.75 ** 2 / 4.0) * (r2 - 1.0) ** 2 + 0.5 * p.a * r2) * vol
    assert abs(K - kin) < 1e-12 * kin and abs(P - pot) < 1e-12 * pot
    assert abs(G) < 1e-12 and S == 0.0 and abs(T - (kin + pot)) < 1e-12 * (kin + pot)


def test_hierarchy_string_length_of_straight_strings_is_exact():
    """psi = sin(2 pi (x - x0) / 16) + i sin(2 pi (y - y0) / 16) has four
    straight strings along z, one pierced plaquette per layer of whichever
    level owns the region: one string runs through levels 1 and 2, three
    through the coarse level only.  The string length is 4 x 16 dx_0 exactly
    (a layer of level l counts dx_l, and level l has 2^l layers per coarse
    one)."""
    p = EOMParams(order=4)
    h = amr.make_hierarchy(16, 0.5, 0.125, 3, 4, SYM_BOXES, p, interp_type=4, eta0=0.75)
    x0, y0 = 7.1, 7.3
    _set_level_fields(h, lambda x, y, z: [np.sin(2 * np.pi * (x - x0) / 16), np.sin(2 * np.pi * (y - y0) / 16),
                                          np.zeros(x.shape), np.zeros(x.shape)])
    S = h.energy()[4]
    assert S == 4 * 16 * 0.5, S


def _level_cells(L):
    """{(x, y, z): values of the four fields} over the valid cells of a level."""
    out = {}
    for b, (lo, hi) in enumerate(L.boxes):
        v = L.data[b][L.valid(b)]
        for k in range(hi[2] - lo[2] + 1):
            for j in range(hi[1] - lo[1] + 1):
                for i in range(hi[0] - lo[0] + 1):
                    out[(lo[0] + i, lo[1] + j, lo[2] + k)] = tuple(v[:, k, j, i])
    return out


def test_regrid_level_copies_old_cells_and_prolongs_new_ones():
    """Sec. 2.3's rebuild of a level: the same cells chopped into other boxes
    keep their values bit for bit; a superset keeps the old cells bit for
    bit and takes, in the new cells, the prolongation of the coarse level,
    here the exact fine averages of the coarse level's quartic polynomial
    (type 4 is exact for those); no boxes remove the level and every finer one."""
    p = EOMParams(order=4)
    boxes0 = [((0, 0, 0), (15, 15, 15))]
    old1 = [((8, 8, 8), (15, 15, 15)), ((16, 8, 8), (23, 15, 15))]
    h = amr.make_hierarchy(16, 0.5, 0.125, 3, 4, [boxes0, old1, [((20, 20, 20), (27, 27, 27))]], p, interp_type=4)
    coef = [0.3, -0.2, 0.05, 0.01, -0.002]                  # quartic in x, constant in y and z

    def avg(lo, hi):                                         # exact average over [lo, hi] (level-0 units)
        return sum(c * (hi ** (q + 1) - lo ** (q + 1)) / ((q + 1) * (hi - lo)) for q, c in enumerate(coef))

    xs = np.arange(16.0)
    row = np.array([avg(x - 0.5, x + 0.5) for x in xs])
    h.levels[0].set_dense([np.broadcast_to(row, (16, 16, 16)).copy()] * 4)
    rng = np.random.default_rng(9)
    h.levels[1].set_dense([rng.standard_normal((32, 32, 32)) for _ in range(4)])
    before = _level_cells(h.levels[1])
    # same cells, other boxes
    amr.regrid_level(h, 1, [((8, 8, 8), (23, 11, 15)), ((8, 12, 8), (23, 15, 15))])
    assert _level_cells(h.levels[1]) == before
    # a superset: the old cells and new cells along x
    amr.regrid_level(h, 1, [((4, 8, 8), (27, 15, 15))])
    after = _level_cells(h.levels[1])
    for key, val in after.items():
        if key in before:
            assert val == before[key], key
        else:
            x = key[0]                                       # fine cell x spans [x/2 - 1/2, x/2] in level-0 units
            exp = avg(x / 2 - 0.5, x / 2)
            assert all(abs(c - exp) < 1e-13 for c in val), (key, val, exp)
    assert len(after) == 24 * 8 * 8 and len(h.levels) == 3
    amr.regrid_level(h, 1, [])
    assert len(h.levels) == 1


def test_full_cover_with_tensor_fields_equals_uniform_fine_run():
    """The 16-field state (Sec. 5): a fine level covering the whole domain
    reproduces a uniform fine run of psi, Pi, u_ij, v_ij bit for bit and
    restricts onto the coarse level exactly, all 16 fields."""
    from oracle import gw as ogw
    n0, dx0, dt0 = 8, 0.25, 1.0 / 16
    p = EOMParams(order=4)
    rng = np.random.default_rng(14)
    fine0 = [rng.uniform(-0.8, 0.8, size=(16, 16, 16)) for _ in range(4)]
    fine0 += [0.1 * rng.standard_normal((16, 16, 16)) for _ in range(12)]
    h = amr.make_hierarchy(n0, dx0, dt0, 3, 4,
                           [[((0, 0, 0), (7, 7, 7))],
                            [((0, 0, 0), (7, 15, 15)), ((8, 0, 0), (15, 7, 15)), ((8, 8, 0), (15, 15, 15))]],
                           p, interp_type=4, eta0=0.5, gw=True)
    h.levels[0].set_dense([interp.restrict_block(f) for f in fine0])
    h.levels[1].set_dense(fine0)
    for _ in range(2):
        h.step()
    ref, eta = fine0, 0.5
    for _ in range(4):
        ref = ogw.rk4_step_periodic(ref, eta, dt0 / 2, dx0 / 2, p)
        eta += dt0 / 2
    L1 = h.levels[1]
    for b, (lo, hi) in enumerate(L1.boxes):
        got = L1.data[b][L1.valid(b)]
        for c in range(16):
            assert np.array_equal(got[c], ref[c][lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]), (b, c)
    got0 = h.levels[0].data[0][h.levels[0].valid(0)]
    for c in range(16):
        assert np.array_equal(got0[c], interp.restrict_block(ref[c])), c
