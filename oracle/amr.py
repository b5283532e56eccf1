"""Block-structured level hierarchy with recursive time subcycling
(Sec. 2 and 2.1, Fig. 2).

* Level l has spacing dx_l = dx_0 / 2^l and step dt_l = dt_0 / 2^l (Eqs. 1-3).
* Each level is a list of disjoint boxes (inclusive lo/hi in the level's index
  space, aligned to and multiples of the blocking factor); only level 0 covers
  the periodic domain.  Every box carries ``g`` ghost layers.
* Ghost fill of a box (psi components, the only ones the stencil reads):
  a ghost cell, wrapped periodically, that lies in a box of the same level is
  copied from it; otherwise it is prolonged from the next coarser level with
  the spatial weights of ``interp`` applied to coarse values interpolated in
  time between the coarse states at the start and end of the coarse step
  (fraction alpha of that step).
* One step of level l (classic RK4, SSPRK3, RKN4 or RKN5) fills ghosts before every stage at the
  stage time: the fine sub-step i in {0, 1} of the coarse step has stage fractions
  alpha = (i + c_s) / 2 with the integrator's stage times c (c = (0, 1/2, 1/2, 1) for RK4).
* advance(l): keep the level's state as "old", take one step; if a finer
  level exists, advance it twice, then synchronise: every coarse cell covered
  by the finer level becomes the mean of its 8 children (all four fields).
* eta: level 0 advances by repeated addition of dt_0; the finer level's
  sub-step i starts at eta_parent_start + i * dt_l.

Parity: the ingredients are pinned individually (stencil, rk4, interp,
winding); the hierarchy itself has no closed form.  Pins here: a fine level
covering the whole domain reproduces a uniform fine-lattice run bit for bit
and restricts onto the coarse level exactly; a polynomial coarse field is
prolonged exactly into fine ghosts; a field constant in space and linear in
time stays exact through the subcycled steps (the stage-time fractions); a
three-level run is invariant bit for bit under lattice translations by whole
blocks and under the rotation (psi1, psi2) -> (-psi2, psi1) in field space --
tests/test_oracle_amr.py.
"""
from __future__ import annotations

import numpy as np

from . import gw as ogw
from . import ko, rkn4, rkn5, ssprk3, tee
from . import interp, winding
from .eom import EOMParams, rhs
from .energy import energy_box
from .stencil import laplacian_padded

C_RK = (0.0, 0.5, 0.5, 1.0)
A_RK = (0.0, 0.5, 0.5, 1.0)


class Level:
    def __init__(self, lev, boxes, n, dx, dt, g, bf, ncomp=4):
        self.lev, self.n, self.dx, self.dt, self.g, self.bf = lev, n, dx, dt, g, bf
        self.ncomp = ncomp
        self.boxes = [(tuple(int(v) for v in lo), tuple(int(v) for v in hi)) for lo, hi in boxes]
        if n % bf:
            raise ValueError("domain not a multiple of the blocking factor")
        nb = n // bf
        self.owner = -np.ones((nb, nb, nb), dtype=np.int64)
        for b, (lo, hi) in enumerate(self.boxes):
            for d in range(3):
                if lo[d] % bf or (hi[d] + 1) % bf or lo[d] < 0 or hi[d] >= n or hi[d] < lo[d]:
                    raise ValueError(f"box {b} not aligned to blocking factor / outside domain")
            blk = self.owner[lo[2] // bf:(hi[2] + 1) // bf, lo[1] // bf:(hi[1] + 1) // bf,
                             lo[0] // bf:(hi[0] + 1) // bf]
            if (blk >= 0).any():
                raise ValueError("boxes overlap")
            blk[...] = b
        self.data = [np.zeros((ncomp,) + self.padded_shape(b)) for b in range(len(self.boxes))]
        self.old = None
        self.eta = None

    def padded_shape(self, b):
        lo, hi = self.boxes[b]
        g = self.g
        return (hi[2] - lo[2] + 1 + 2 * g, hi[1] - lo[1] + 1 + 2 * g, hi[0] - lo[0] + 1 + 2 * g)

    def valid(self, b):
        g = self.g
        nz, ny, nx = (s - 2 * g for s in self.padded_shape(b))
        return (slice(None), slice(g, g + nz), slice(g, g + ny), slice(g, g + nx))

    def owners_of(self, kz, ky, kx):
        """Box index owning (already wrapped) cells, -1 where uncovered."""
        bf = self.bf
        return self.owner[kz // bf, ky // bf, kx // bf]

    def gather(self, sources, comps, kz, ky, kx):
        """Values of valid cells (wrapped indices) from each list of per-box
        arrays in ``sources``: shape (len(sources), len(comps)) + kz.shape."""
        own = self.owners_of(kz, ky, kx)
        if (own < 0).any():
            raise ValueError("coarse stencil reaches outside the coarser level (nesting)")
        out = np.empty((len(sources), len(comps)) + kz.shape)
        g = self.g
        for s in range(len(self.boxes)):
            sel = own == s
            if not sel.any():
                continue
            lo = self.boxes[s][0]
            iz, iy, ix = kz[sel] - lo[2] + g, ky[sel] - lo[1] + g, kx[sel] - lo[0] + g
            for si, arrays in enumerate(sources):
                for ci, c in enumerate(comps):
                    out[si, ci][sel] = arrays[s][c][iz, iy, ix]
        return out

    def dense(self, arrays, comps):
        """The level's valid cells of ``comps`` as arrays over its whole
        periodic domain, NaN where no box of the level lies."""
        out = np.full((len(comps), self.n, self.n, self.n), np.nan)
        for b, (lo, hi) in enumerate(self.boxes):
            v = self.valid(b)
            for ci, c in enumerate(comps):
                out[ci, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = arrays[b][c][v[1:]]
        return out

    def set_dense(self, fields):
        """Fill valid cells from dense arrays (one per field) over the level domain."""
        for b, (lo, hi) in enumerate(self.boxes):
            v = self.valid(b)
            for c in range(len(fields)):
                self.data[b][c][v[1:]] = fields[c][lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]

    def covered_mask(self, b, finer):
        """True where a valid cell of box b is covered by the finer level."""
        lo, hi = self.boxes[b]
        shp = tuple(hi[d] - lo[d] + 1 for d in (2, 1, 0))
        m = np.zeros(shp, dtype=bool)
        if finer is None:
            return m
        for flo, fhi in finer.boxes:
            clo = [flo[d] // 2 for d in range(3)]
            chi = [(fhi[d] + 1) // 2 - 1 for d in range(3)]
            ilo = [max(clo[d], lo[d]) for d in range(3)]
            ihi = [min(chi[d], hi[d]) for d in range(3)]
            if all(ilo[d] <= ihi[d] for d in range(3)):
                m[ilo[2] - lo[2]:ihi[2] - lo[2] + 1, ilo[1] - lo[1]:ihi[1] - lo[1] + 1,
                  ilo[0] - lo[0]:ihi[0] - lo[0] + 1] = True
        return m


def fill_ghosts(level: Level, arrays, coarse: Level | None, alpha: float, interp_type: int,
                comps=(0, 1)):
    """Fill the ghost layers of ``arrays`` (one padded array per box of
    ``level``) for the given components; see the module docstring."""
    g, n = level.g, level.n
    for b, (lo, hi) in enumerate(level.boxes):
        arr = arrays[b]
        shp = level.padded_shape(b)
        pz, py, px = np.indices(shp)
        kz, ky, kx = pz + lo[2] - g, py + lo[1] - g, px + lo[0] - g
        interior = ((pz >= g) & (pz < shp[0] - g) & (py >= g) & (py < shp[1] - g)
                    & (px >= g) & (px < shp[2] - g))
        gh = ~interior
        gpz, gpy, gpx = pz[gh], py[gh], px[gh]
        wz, wy, wx = kz[gh] % n, ky[gh] % n, kx[gh] % n
        own = level.owners_of(wz, wy, wx)
        for s in np.unique(own[own >= 0]):
            sel = own == s
            slo = level.boxes[s][0]
            for c in comps:
                arr[c][gpz[sel], gpy[sel], gpx[sel]] = arrays[s][c][
                    wz[sel] - slo[2] + g, wy[sel] - slo[1] + g, wx[sel] - slo[0] + g]
        sel = own < 0
        if sel.any():
            if coarse is None:
                raise ValueError("uncovered ghost cell on a level without a coarser level")
            nc = coarse.n

            # coarse state at fraction alpha of its step, over its whole domain
            Da = interp.time_lerp(coarse.dense(coarse.old, comps), coarse.dense(coarse.data, comps),
                                  alpha).reshape(len(comps), -1)

            def coarse_at(Kz, Ky, Kx):
                v = Da[:, ((Kz % nc) * nc + Ky % nc) * nc + Kx % nc]
                if np.isnan(v).any():
                    raise ValueError("coarse stencil reaches outside the coarser level (nesting)")
                return v

            vals = interp.prolong_points(coarse_at, (wz[sel], wy[sel], wx[sel]), interp_type)
            for ci, c in enumerate(comps):
                arr[c][gpz[sel], gpy[sel], gpx[sel]] = vals[ci]


def rhs_box(arr, g, dx, eta, p: EOMParams):
    v = (slice(g, arr.shape[1] - g), slice(g, arr.shape[2] - g), slice(g, arr.shape[3] - g))
    lap1 = laplacian_padded(arr[0], g, dx, p.order)
    lap2 = laplacian_padded(arr[1], g, dx, p.order)
    d = rhs(arr[0][v], arr[1][v], arr[2][v], arr[3][v], lap1, lap2, eta, p)
    if p.ko_order:
        # Kreiss-Oliger dissipation of every scalar component (Sec. 2.4)
        d = [dc + ko.ko_padded(arr[c], g, dx, p.ko_order, p.ko_eps) for c, dc in enumerate(d)]
    return np.stack(d)


class Hierarchy:
    """Levels 0..L-1 with fixed (or externally regridded) boxes.  With
    ``gw`` the state carries the 12 gravitational-wave fields of oracle.gw
    (16 fields; ghosts of psi and u are filled)."""

    def __init__(self, levels, params: EOMParams, interp_type: int = 4, gw: bool = False, integrator: int = 4):
        self.levels = levels
        self.p = params
        self.interp_type = interp_type
        if integrator not in (4, 10, 21, 22):
            raise ValueError("integrator must be 4 (classic RK4), 10 (low-storage SSPRK3), 21 (RKN4) or 22 (RKN5)")
        if integrator in (21, 22) and params.ko_order:
            raise ValueError("RKN needs x' = v: no Kreiss-Oliger term")
        if integrator == 22 and (params.friction or gw):
            raise ValueError("RKN5 needs an acceleration independent of the velocities: "
                             "friction off, scalar fields only")
        self.integrator = integrator
        self.gw = gw
        # ghosts of psi (stencil), of Pi under dissipation, and of u_ij
        self.ghost_comps = (0, 1) + ((2, 3) if params.ko_order else ()) + ((4, 5, 6, 7, 8, 9) if gw else ())
        self.tag_log = []          # optional (lev, eta, [tags per box]) at stage 1
        self.record_tags = False
        self.te_eps = None         # TEE thresholds of (psi1, psi2, Pi1, Pi2): self-shadow tags at sync
        self.te_tags = {}          # lev -> [tags per box] from the last synchronisation of lev
        self.te_vals = {}          # lev -> [(4, nz, ny, nx) estimates on the parent cells, per box]

    def coarse_of(self, lev):
        return self.levels[lev - 1] if lev > 0 else None

    def rk4_level(self, lev, sub):
        L = self.levels[lev]
        C = self.coarse_of(lev)
        g, dt, eta = L.g, L.dt, L.eta
        y0 = [a.copy() for a in L.data]
        Y = [a.copy() for a in y0]
        ks = []
        for s in range(4):
            alpha = (sub + C_RK[s]) / 2.0
            if s > 0:
                for b in range(len(Y)):
                    v = L.valid(b)
                    Y[b][v] = y0[b][v] + (A_RK[s] * dt) * ks[s - 1][b]
            fill_ghosts(L, Y, C, alpha, self.interp_type, comps=self.ghost_comps)
            if s == 0 and self.record_tags:
                self.tag_log.append((lev, eta, [winding.cell_tags_padded(a[0], a[1], g) for a in Y]))
            ks.append([self._rhs(Y[b], g, L.dx, eta + C_RK[s] * dt) for b in range(len(Y))])
        for b in range(len(Y)):
            v = L.valid(b)
            L.data[b][v] = y0[b][v] + (dt / 6.0) * (ks[0][b] + 2.0 * ks[1][b] + 2.0 * ks[2][b] + ks[3][b])

    def ssprk3_level(self, lev, sub):
        """One low-storage SSPRK3 step of level ``lev`` (oracle/ssprk3.py): stage
        s evaluates at eta + c_s dt, c = (0, 1, 1/2), with ghosts at time
        fraction (sub + c_s)/2 of the coarser step."""
        L = self.levels[lev]
        C = self.coarse_of(lev)
        g, dt, eta = L.g, L.dt, L.eta
        y0 = [a.copy() for a in L.data]
        U = [a.copy() for a in y0]
        for s in range(3):
            alpha = (sub + ssprk3.C[s]) / 2.0
            fill_ghosts(L, U, C, alpha, self.interp_type, comps=self.ghost_comps)
            if s == 0 and self.record_tags:
                self.tag_log.append((lev, eta, [winding.cell_tags_padded(a[0], a[1], g) for a in U]))
            k = [self._rhs(U[b], g, L.dx, eta + ssprk3.C[s] * dt) for b in range(len(U))]
            for b in range(len(U)):
                v = L.valid(b)
                U[b][v] = ssprk3.A[s] * y0[b][v] + ssprk3.B[s] * (U[b][v] + dt * k[b])
        for b in range(len(U)):
            v = L.valid(b)
            L.data[b][v] = U[b][v]

    def rkn4_level(self, lev, sub):
        """One RKN4 step of level ``lev`` (oracle/rkn4.py): stage s from the
        positions and velocities the previous stages' accelerations give,
        ghosts at time fraction (sub + c_s)/2 of the coarser step."""
        L = self.levels[lev]
        C = self.coarse_of(lev)
        g, dt, eta = L.g, L.dt, L.eta
        pos, vel = (rkn4.POS_GW, rkn4.VEL_GW) if self.gw else (rkn4.POS, rkn4.VEL)
        y0 = [a.copy() for a in L.data]
        Y = [a.copy() for a in y0]
        acc = []                              # per stage: per box, the accelerations (len(vel), nz, ny, nx)
        for s in range(4):
            alpha = (sub + rkn4.C[s]) / 2.0
            if s > 0:
                for b in range(len(Y)):
                    v = L.valid(b)
                    x0 = [y0[b][i][v[1:]] for i in pos]
                    v0 = [y0[b][i][v[1:]] for i in vel]
                    xs, vs = rkn4.stage_states(x0, v0, dt, [a[b] for a in acc], s)
                    for i, a in zip(pos, xs):
                        Y[b][i][v[1:]] = a
                    for i, a in zip(vel, vs):
                        Y[b][i][v[1:]] = a
            fill_ghosts(L, Y, C, alpha, self.interp_type, comps=self.ghost_comps)
            if s == 0 and self.record_tags:
                self.tag_log.append((lev, eta, [winding.cell_tags_padded(a[0], a[1], g) for a in Y]))
            acc.append([[k[i] for i in vel] for k in
                        (self._rhs(Y[b], g, L.dx, eta + rkn4.C[s] * dt) for b in range(len(Y)))])
        for b in range(len(Y)):
            v = L.valid(b)
            x0 = [y0[b][i][v[1:]] for i in pos]
            v0 = [y0[b][i][v[1:]] for i in vel]
            xn, vn = rkn4.final_state(x0, v0, dt, [a[b] for a in acc])
            for i, a in zip(pos, xn):
                L.data[b][i][v[1:]] = a
            for i, a in zip(vel, vn):
                L.data[b][i][v[1:]] = a

    def rkn5_level(self, lev, sub):
        """One RKN5 step of level ``lev`` (oracle/rkn5.py): stage s at the
        positions x + c_s h v + h^2 sum_j abar_sj k_j (velocities left at the
        step's start: the acceleration does not read them), ghosts at time
        fraction (sub + c_s)/2 of the coarser step."""
        L = self.levels[lev]
        C = self.coarse_of(lev)
        g, dt, eta = L.g, L.dt, L.eta
        pos, vel = rkn5.POS, rkn5.VEL
        y0 = [a.copy() for a in L.data]
        Y = [a.copy() for a in y0]
        acc = []                              # per stage: per box, the accelerations
        for s in range(4):
            if s > 0:
                for b in range(len(Y)):
                    v = L.valid(b)
                    for n, i in enumerate(pos):
                        xs = y0[b][i][v[1:]] + (rkn5.C[s] * dt) * y0[b][vel[n]][v[1:]]
                        for j in range(s):
                            xs = xs + (dt * dt * rkn5.ABAR[s][j]) * acc[j][b][n]
                        Y[b][i][v[1:]] = xs
            fill_ghosts(L, Y, C, (sub + rkn5.C[s]) / 2.0, self.interp_type, comps=self.ghost_comps)
            if s == 0 and self.record_tags:
                self.tag_log.append((lev, eta, [winding.cell_tags_padded(a[0], a[1], g) for a in Y]))
            acc.append([[k[i] for i in vel] for k in
                        (self._rhs(Y[b], g, L.dx, eta + rkn5.C[s] * dt) for b in range(len(Y)))])
        for b in range(len(Y)):
            v = L.valid(b)
            for n, i in enumerate(pos):
                L.data[b][i][v[1:]] = (y0[b][i][v[1:]] + dt * y0[b][vel[n]][v[1:]]
                                       + (dt * dt) * sum(rkn5.BBAR[q] * acc[q][b][n] for q in range(4)))
            for n, i in enumerate(vel):
                L.data[b][i][v[1:]] = y0[b][i][v[1:]] + dt * sum(rkn5.B[q] * acc[q][b][n] for q in range(4))

    def _rhs(self, arr, g, dx, eta):
        k = rhs_box(arr, g, dx, eta, self.p)
        if not self.gw:
            return k
        return np.concatenate([k, np.stack(ogw.rhs_box_gw(arr, g, dx, eta, self.p))])

    def restrict(self, fine_lev):
        F = self.levels[fine_lev]
        Cl = self.levels[fine_lev - 1]
        gc = Cl.g
        for b, (flo, fhi) in enumerate(F.boxes):
            fv = F.data[b][F.valid(b)]
            red = np.stack([interp.restrict_block(fv[c]) for c in range(F.ncomp)])
            clo = [flo[d] // 2 for d in range(3)]
            nz, ny, nx = red.shape[1:]
            kz, ky, kx = np.indices((nz, ny, nx))
            kz, ky, kx = kz + clo[2], ky + clo[1], kx + clo[0]
            own = Cl.owners_of(kz, ky, kx)
            if (own < 0).any():
                raise ValueError("fine level not covered by the coarse level")
            if self.te_eps is not None:
                # self-shadow TEE (Sec. 2.2): the coarse values before they are replaced
                cval = Cl.gather([Cl.data], range(tee.NSCALAR), kz, ky, kx)[0]
                te = tee.te_on_coarse(cval, fv[:tee.NSCALAR])
                self.te_tags.setdefault(fine_lev, [None] * len(F.boxes))[b] = tee.tags_from_te(te, self.te_eps)
                self.te_vals.setdefault(fine_lev, [None] * len(F.boxes))[b] = te
            for s in np.unique(own):
                sel = own == s
                slo = Cl.boxes[s][0]
                for c in range(F.ncomp):
                    Cl.data[s][c][kz[sel] - slo[2] + gc, ky[sel] - slo[1] + gc,
                                  kx[sel] - slo[0] + gc] = red[c][sel]

    def advance(self, lev=0, sub=0, parent_eta=None):
        L = self.levels[lev]
        if lev > 0:
            L.eta = parent_eta + sub * L.dt
        eta_start = L.eta
        L.old = [a.copy() for a in L.data]
        if self.integrator == 4:
            self.rk4_level(lev, sub)
        elif self.integrator == 21:
            self.rkn4_level(lev, sub)
        elif self.integrator == 22:
            self.rkn5_level(lev, sub)
        else:
            self.ssprk3_level(lev, sub)
        L.eta = eta_start + L.dt
        if lev + 1 < len(self.levels):
            for i in (0, 1):
                self.advance(lev + 1, i, eta_start)
            self.restrict(lev + 1)

    def step(self):
        """One coarse step (level 0 by dt_0, every finer level subcycled)."""
        self.advance(0, 0)

    # -- diagnostics at the synchronised time -------------------------------
    def _filled(self, lev):
        L = self.levels[lev]
        arrs = [a.copy() for a in L.data]
        C = self.coarse_of(lev)
        if C is not None and C.old is None:
            C.old = [a.copy() for a in C.data]
        fill_ghosts(L, arrs, C, 1.0, self.interp_type, comps=self.ghost_comps)
        return arrs

    def tags(self, lev):
        L = self.levels[lev]
        arrs = self._filled(lev)
        return [winding.cell_tags_padded(a[0], a[1], L.g) for a in arrs]

    def energy(self):
        """[kin, grad, pot, total, string_length] over the uncovered cells of
        every level (each level at its own eta, equal after a coarse step)."""
        K = G = P = S = 0.0
        for lev, L in enumerate(self.levels):
            arrs = self._filled(lev)
            finer = self.levels[lev + 1] if lev + 1 < len(self.levels) else None
            vol = L.dx ** 3
            for b in range(len(L.boxes)):
                unc = ~L.covered_mask(b, finer)
                k, gr, po, nst = energy_box(arrs[b], L.g, L.dx, L.eta, self.p, uncovered=unc)
                K += k * vol
                G += gr * vol
                P += po * vol
                S += nst * L.dx
        return np.array([K, G, P, K + G + P, S])


def make_hierarchy(n0, dx0, dt0, g, bf, level_boxes, params: EOMParams, interp_type=4, eta0=0.1, gw=False,
                   integrator=4):
    """level_boxes[l] = list of (lo, hi) for level l (level 0 usually the one
    box covering the domain)."""
    levels = []
    for l, boxes in enumerate(level_boxes):
        L = Level(l, boxes, n0 * 2 ** l, dx0 / 2 ** l, dt0 / 2 ** l, g, bf, ncomp=16 if gw else 4)
        L.eta = eta0
        levels.append(L)
    return Hierarchy(levels, params, interp_type, gw=gw, integrator=integrator)


def prolong_level_from_coarse(fine: Level, coarse: Level, interp_type: int, comps=None):
    """Initialise every valid cell of ``fine`` by prolongation of the coarse
    level's current state (used to create refined levels from a coarse
    initial state)."""
    if coarse.old is None:
        coarse.old = [a.copy() for a in coarse.data]
    comps = tuple(range(fine.ncomp)) if comps is None else comps
    nc = coarse.n
    for b, (lo, hi) in enumerate(fine.boxes):
        kz, ky, kx = np.indices(tuple(hi[d] - lo[d] + 1 for d in (2, 1, 0)))
        kz, ky, kx = kz + lo[2], ky + lo[1], kx + lo[0]
        v = fine.valid(b)
        def coarse_at(Kz, Ky, Kx):
            return coarse.gather([coarse.data], comps, Kz % nc, Ky % nc, Kx % nc)[0]
        vals = interp.prolong_points(coarse_at, (kz, ky, kx), interp_type)
        for ci, c in enumerate(comps):
            fine.data[b][c][v[1:]] = vals[ci]


def regrid_level(h: Hierarchy, lev: int, new_boxes):
    """Give level ``lev`` (>= 1) the boxes ``new_boxes`` (Sec. 2.3 global
    regrid): every valid cell of the new boxes takes the old level's value
    where an old box of that level covers it, otherwise the prolongation of
    the coarser level's current state (all four fields, the hierarchy's
    interpolation type).  With no boxes the level and every finer one are
    removed; ``lev == len(h.levels)`` creates a new finest level."""
    C = h.levels[lev - 1]
    old = h.levels[lev] if lev < len(h.levels) else None
    if not new_boxes:
        del h.levels[lev:]
        return
    L = Level(lev, new_boxes, C.n * 2, C.dx / 2, C.dt / 2, C.g, C.bf, ncomp=C.ncomp)
    L.eta = C.eta
    prolong_level_from_coarse(L, C, h.interp_type)
    if old is not None:
        g = L.g
        for b, (lo, hi) in enumerate(L.boxes):
            kz, ky, kx = np.indices(tuple(hi[d] - lo[d] + 1 for d in (2, 1, 0)))
            kz, ky, kx = kz + lo[2], ky + lo[1], kx + lo[0]
            own = old.owners_of(kz, ky, kx)
            for s_ in range(len(old.boxes)):
                sel = own == s_
                if not sel.any():
                    continue
                olo = old.boxes[s_][0]
                for c in range(L.ncomp):
                    L.data[b][c][kz[sel] - lo[2] + g, ky[sel] - lo[1] + g, kx[sel] - lo[0] + g] = \
                        old.data[s_][c][kz[sel] - olo[2] + g, ky[sel] - olo[1] + g, kx[sel] - olo[0] + g]
    if old is None:
        h.levels.append(L)
    else:
        h.levels[lev] = L

