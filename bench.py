"""Benchmark of the fused RK4 hot path on GB300.

Default workload: the uniform 512^3 periodic lattice (6th-order Laplacian,
classic RK4, Gaussian random initial field with k_max = pi/(8 dx), dx = 1/8,
dt = dx/4, eta from 0.1) with winding tags and energy partials fused into
stage 1.  The headline ``value`` is the FP32 + Kahan form in cell-updates/s
(one update = one valid cell advanced one full RK4 step); the FP64 form is
timed on the same field and reported under ``fp64_plain``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank advances its own
replica (the path needs no exchange on one level): value = all ranks'
updates / max-over-ranks time, scaling "weak".  ``--impl reference`` times
the CPU FP64 oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 512
DX = 0.125
DT = DX / 4
ETA0 = 0.1
ORDER = 6
KAHAN_VALUES = 76          # field values moved per cell-update, FP32 + Kahan (fused schedule)
F64_VALUES = 68            # FP64


def fp64_ops_per_cell_update(order):
    """FP64 pipe operations (an add, a multiply or a fused multiply-add each
    take one issue slot) per cell-update of the classic RK4 stage kernel,
    diagnostics excluded: per stage and component, the textbook Laplacian
    w0-term (1), G pair sums of 6 neighbours (5 adds + 1 FMA each) and the
    1/dx^2 scale (1); |psi|^2 (2), the potential factor (2) and Pi' for two
    components (2 each); the stage combine adds 8 per stage."""
    g = order // 2
    lap = 2 * (2 + 6 * g)
    return 4 * (lap + 8) + 4 * 8
WORKLOAD = ("uniform 512^3 periodic lattice, 6th-order Laplacian, classic RK4, Gaussian init "
            "k_max=pi/(8dx), dx=1/8, dt=dx/4, eta0=0.1, tags+energy fused in stage 1")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _stage_source_sha():
    """Hash of the stage kernel's source (the kernel header and its host side)."""
    csrc = os.path.join(ROOT, "paper_2404_02950_gb300", "csrc")
    m = hashlib.sha256()
    for name in ("stage_kernel.cuh", "stage.cu"):
        m.update(open(os.path.join(csrc, name), "rb").read())
    return m.hexdigest()[:16]


def _stage_traffic():
    """DRAM bytes per stage-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source (else None)."""
    f = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(f):
        return None
    d = json.load(open(f))
    h = _stage_source_sha()
    e = d.get("stage_kernel_f32_g3")
    if e and e.get("source_sha") == h:
        return e.get("bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--id={self.gpu_index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def max_over_ranks(dist, values, device):
    """Each value's maximum over the ranks of the job (the slowest replica
    sets the time); the values themselves on a single rank."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(world, cells, steps, ms):
    """Whole-job throughput: every rank advances its own replica of ``cells``
    cells ``steps`` times; the job takes the slowest rank's ``ms``."""
    return world * float(cells) * steps / (ms / 1e3)


def cpu_oracle_sample(budget_s=12.0, n=96):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload:
    an n^3 periodic lattice with the same dx, dt, order and init recipe."""
    from oracle import rk4
    from oracle.eom import EOMParams
    from paper_2404_02950_gb300 import inputs
    y = inputs.gaussian_field(n, n / 16.0, seed=0)
    p = EOMParams(order=ORDER)
    eta = ETA0
    steps = 0
    t0 = time.perf_counter()
    while True:
        y = rk4.rk4_step_periodic(y, eta, DT, DX, p)
        eta += DT
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 50:
            break
    return {"value": n ** 3 * steps / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} RK4 step(s) of a {n}^3 periodic lattice (same dx, dt, order 6, init recipe), "
                      f"numpy FP64, {el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_step = []
    base = None
    for _ in range(args.warmup + args.steps):
        r = cpu_oracle_sample(budget_s=max(2.0, 20.0 / max(1, args.steps + args.warmup)), n=64)
        per_step.append(r)
        base = r
    vals = [r["value"] for r in per_step[args.warmup:]]
    v = float(np.mean(vals))
    line = {"metric": "cell-updates/s (one valid cell advanced one full RK4 step)", "value": v,
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 64 ** 3 / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "64^3 crop of the same recipe"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _error_vs_f64(st32, st64, cells, len32, len64, steps):
    """Relative L2 error per field (psi1, psi2, Pi1, Pi2) and relative
    string-length error of the FP32 + Kahan state against the FP64 state
    after the same steps from the same field."""
    import torch
    out = {}
    for c, name in enumerate(("psi1", "psi2", "Pi1", "Pi2")):
        a = st32[c * cells:(c + 1) * cells].double()
        b = st64[c * cells:(c + 1) * cells]
        out[name] = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    out["string_length"] = abs(len32 - len64) / len64 if len64 > 0 else None
    out["steps"] = steps
    out["bound"] = "1e-4 relative L2 per field, 1 % string length (tests/test_gpu_precision.py checks 100 steps)"
    return out


def _time_form(slh, torch, prec, y0_dense, n, K, W, dist, flags, gw=False, order=ORDER, integrator=4, tile=None,
               diag_tile=None, friction=True):
    """Warm up, then time K steps of one precision; returns a dict."""
    # ghost layers = the Laplacian's stencil radius (the paper's "order")
    h = slh.Hierarchy(n, DX, nghost=order // 2, bf=16, prec=prec, max_levels=1, gw=gw)
    boxes = [((0, 0, 0), (n - 1, n - 1, n - 1))]
    h.init_level(0, boxes, fused_tags=True)
    h.set_state(0, y0_dense.astype(h.np_dtype))
    h.set_eta(ETA0)
    p = slh.EOMParams(order=order, integrator=integrator, friction=friction)
    if tile is None:
        chosen, tune_ms = h.autotune(0, p, reps=3)
        chosen_d, tune_d_ms = h.autotune(0, p, reps=3, diag=True) if flags else (chosen, [])
    else:
        h.set_tile(0, tile)
        chosen, tune_ms, chosen_d, tune_d_ms = tile, [], tile, []
        if diag_tile is not None:
            h.set_diag_tile(0, diag_tile)
            chosen_d = diag_tile
    for _ in range(W):
        h.advance(DT, p, flags=flags)
    h.sync()
    h.profile(True, True)
    stream = h.stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(K):
        h.advance(DT, p, flags=flags)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    per_stage = [h.profile_read(k)[0] for k in (slh.SLH_PROF_S1, slh.SLH_PROF_S2, slh.SLH_PROF_S3,
                                                 slh.SLH_PROF_S4)]
    stage = h.profile_read(slh.SLH_PROF_STAGE)
    ghost = h.profile_read(slh.SLH_PROF_GHOST)
    tim = h.profile_read(slh.SLH_PROF_TIME)
    gwk = h.profile_read(slh.SLH_PROF_GW)
    h.profile(False, True)
    E = h.reduce_energy(p, mode=1) if flags & slh.SLH_FUSE_ENERGY else None
    out = dict(ms=ms, stage_ms=stage[0], stage_launches=stage[1], stage_bytes=stage[2],
               ghost_ms=ghost[0], ghost_launches=ghost[1], time_launches=tim[1],
               energy=None if E is None else E.tolist(),
               per_stage_ms=[m / K for m in per_stage], tile_variant=chosen, tune_ms=tune_ms,
               diag_tile_variant=chosen_d, diag_tune_ms=tune_d_ms,
               gw_ms=gwk[0], gw_launches=gwk[1], gw_bytes=gwk[2],
               buffer_bytes=sum(b.numel() * b.element_size() for b in h.levels[0]["bufs"] if b is not None))
    return h, out


GW_N, GW_ORDER, GW_K = 512, 4, 5
GW_WORKLOAD = ("gravitational-wave tensor (16 fields: psi, Pi, u_ij, v_ij): uniform 512^3 periodic lattice, "
               "4th-order Laplacian and gradients, classic RK4, FP32 + Kahan, Gaussian psi init "
               "k_max=pi/(4dx), u = v = 0, dx=1/8, dt=dx/4, eta0=0.1, tags+energy fused in stage 1")
GW_VALUES = 236            # tensor-field values moved per cell-update by the GW kernel (FP32 + Kahan)


def _gw_form(slh, torch, n, dist, peak, K=GW_K):
    """Uniform 16-field lattice: whole-step throughput and the GW stage
    kernel's achieved HBM bandwidth."""
    from paper_2404_02950_gb300 import inputs
    y = [a.astype(np.float32) for a in inputs.gaussian_field(n, n / 8.0, seed=7)]
    zero = np.zeros_like(y[0])
    dense = slh.dense_from_boxes(y + [zero] * 12, [((0, 0, 0), (n - 1,) * 3)])
    del y, zero
    flags = slh.SLH_FUSE_TAG | slh.SLH_FUSE_ENERGY
    h, r = _time_form(slh, torch, "f32", dense, n, K, 3, dist, flags, gw=True, order=GW_ORDER)
    h.close()
    del h, dense
    torch.cuda.empty_cache()
    ach = r["gw_bytes"] / (r["gw_ms"] / 1e3) / 1e9
    return {"workload": GW_WORKLOAD, "unit": "cell-updates/s",
            "value": float(n) ** 3 * K / (r["ms"] / 1e3), "ms_per_step": r["ms"] / K,
            "gw_kernel": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                          "ms_per_step": r["gw_ms"] / K, "launches": r["gw_launches"],
                          "alg_bytes_per_cell_update": GW_VALUES * 4},
            "scalar_stage_ms_per_step": r["stage_ms"] / K, "ghost_ms_per_step": r["ghost_ms"] / K,
            "hbm_footprint_gb": r["buffer_bytes"] / 1e9,
            "footprint_note": ("5 level buffers x 16 FP32 fields = 320 B per cell: 1024^3 would need 344 GB "
                               "(over the 288 GB of HBM); the largest lattice under 150 GB is 768^3")}


C4_N, C4_K, C4_W = 1024, 4, 2
C4_WORKLOAD = ("largest single-GPU run: 1024^3 periodic base + 2 ratio-2 levels (each a 256^3 cube of eight 128^3 "
               "boxes at the centre of the level below), 16 fields: psi, Pi in FP32, u_ij, v_ij stored BF16 and "
               "accumulated FP32, low-storage SSPRK3 (integrator type 10) on three level buffers, 4th-order "
               "Laplacian and gradients, quartic prolongation, Gaussian psi (k_max = pi/(4 dx) on a 512^3 lattice, "
               "tiled twice per axis), u = v = 0, dx0 = 1/8, dt0 = dx0/4, eta0 = 0.1; subcycled coarse steps "
               "replayed from CUDA graphs")
C4_GW_SLOTS = (14, 20, 20)   # 4-byte slots the BF16 GW stage moves per cell at SSPRK3 stages 1..3


def _c4_level_boxes(n0, side=128):
    """Fixed refined levels 1 and 2: a cube of 2 side cells at the centre of
    the level's index space, cut into eight boxes of side^3 (nested in the
    level below with room to spare for n0 >= 4 side)."""
    out = []
    for lev in (1, 2):
        lo = (n0 << lev) // 2 - side
        out.append([((lo + side * i, lo + side * j, lo + side * k),
                     (lo + side * (i + 1) - 1, lo + side * (j + 1) - 1, lo + side * (k + 1) - 1))
                    for k in range(2) for j in range(2) for i in range(2)])
    return out


def _c4_form(slh, torch, peak, n=C4_N, K=C4_K, W=C4_W):
    """The largest single-GPU workload with BF16 tensor storage: footprint,
    whole-step throughput and the BF16 GW stage kernel's HBM fraction."""
    from paper_2404_02950_gb300 import inputs
    n_small = n // 2
    y = inputs.gaussian_field(n_small, n_small / 4.0, seed=11)
    h = slh.Hierarchy(n, DX, nghost=2, bf=16, prec="f32bf16", max_levels=3, gw=True)
    h.init_level(0, [((0, 0, 0), (n - 1,) * 3)])    # every buffer zeroed: Pi = u = v = 0
    # psi1, psi2: the n/2 lattice tiled twice per axis, written into the padded
    # state buffer on the device (slots 0 and 1)
    offs, geom, _, _ = slh.slh_level_layout(2, [((0, 0, 0), (n - 1,) * 3)], slh.SLH_SLOTS_BF16)
    pitch, pny, pnz, cs = (int(v) for v in geom[0])
    buf = h.state_buffer(0)
    for c in range(2):
        v = buf[int(offs[0]) + c * cs:int(offs[0]) + c * cs + pitch * pny * pnz].view(pnz, pny, pitch)
        t = torch.from_numpy(y[c].astype(np.float32)).cuda()
        v[2:2 + n, 2:2 + n, 4:4 + n].copy_(t.repeat(2, 2, 2))
        del t
    del y
    h.set_eta(ETA0)
    for lev, boxes in enumerate(_c4_level_boxes(n), start=1):
        h.regrid_level(lev, boxes)
    p = slh.EOMParams(order=4, interp_type=4, integrator=10)
    footprint = sum(b.numel() * b.element_size() for info in h.levels.values() for b in info["bufs"] if b is not None)
    for _ in range(W):
        h.advance(DT, p, flags=slh.SLH_USE_GRAPH)
    h.sync()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(h.stream)
    for _ in range(K):
        h.advance(DT, p, flags=slh.SLH_USE_GRAPH)
    ev1.record(h.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    updates = sum(info["nvalid"] * 2 ** lev for lev, info in h.levels.items())
    # the same steps launched directly with the per-kernel profile on
    h.profile(True, True)
    for _ in range(K):
        h.advance(DT, p)
    h.sync()
    gwk = h.profile_read(slh.SLH_PROF_GW)
    stg = h.profile_read(slh.SLH_PROF_STAGE)
    gho = h.profile_read(slh.SLH_PROF_GHOST)
    h.profile(False, True)
    E = h.reduce_energy(p)
    levels = {str(l): {"boxes": len(info["boxes"]), "cells": info["nvalid"]} for l, info in h.levels.items()}
    h.close()
    del h
    torch.cuda.empty_cache()
    ach = gwk[2] / (gwk[0] / 1e3) / 1e9 if gwk[0] > 0 else None
    return {"workload": C4_WORKLOAD, "unit": "cell-updates/s", "value": updates * K / (ms / 1e3),
            "ms_per_coarse_step": ms / K, "coarse_steps_timed": K, "levels": levels,
            "hbm_footprint_gb": footprint / 1e9,
            "footprint_note": ("3 level buffers x (4 FP32 + 6 BF16-pair slots) = 120 B per cell; the < 150 GB "
                               "target of the 1024^3 + 2-level run"),
            "gw_kernel": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": (ach / peak) if ach else None,
                          "ms_per_coarse_step_direct": gwk[0] / K, "launches": gwk[1],
                          "alg_slots_per_cell_update": sum(C4_GW_SLOTS), "slot_bytes": 4},
            "scalar_stage_ms_per_coarse_step_direct": stg[0] / K, "ghost_ms_per_coarse_step_direct": gho[0] / K,
            "string_length_end": E[4],
            "error_vs_f64": "tests/test_gpu_bf16.py: the 128^3 crop after 100 steps against the FP64 oracle"}


AMR_N, AMR_LEVELS, AMR_NBUF, AMR_BF, AMR_MAXBOX, AMR_RELAX, AMR_EVERY = 256, 4, 4, 16, 128, 300, 4
AMR_ORDER = 4
AMR_K32, AMR_K64 = 16, 4   # coarse steps timed (FP32 batched, FP64 plain)
AMR_WORKLOAD = ("dynamic AMR: 256^3 base + up to 3 ratio-2 levels, c0-style Gaussian init (k_max=pi/(4dx)) relaxed "
                f"{AMR_RELAX} coarse steps on the base level, then global regrids every {AMR_EVERY} coarse steps from "
                "string tags (buffer 4, blocking factor 16, max box 128), 4th-order Laplacian, quartic prolongation, "
                "subcycled RK4 replayed as one CUDA graph per coarse step (captured again after every regrid); "
                "regrid and capture time included")


def _amr_form(slh, torch, prec, y0_dense, K, n=AMR_N, peak=None, relax=AMR_RELAX):
    """Dynamic-AMR timing: K coarse steps with a global regrid every
    AMR_EVERY steps, every coarse step replayed from its CUDA graph, then K
    more steps launched directly with the per-kernel profile on.  Returns
    (cell-updates/s of the graph pass, details)."""
    h = slh.Hierarchy(n, DX, nghost=AMR_ORDER // 2, bf=AMR_BF, prec=prec, max_levels=AMR_LEVELS)
    h.init_level(0, [((0, 0, 0), (n - 1, n - 1, n - 1))])
    h.set_state(0, y0_dense.astype(h.np_dtype))
    h.set_eta(ETA0)
    p = slh.EOMParams(order=AMR_ORDER, interp_type=4)
    for _ in range(relax):
        h.advance(DT, p, flags=slh.SLH_USE_GRAPH)
    h.sync()
    h.regrid(AMR_LEVELS, AMR_NBUF, AMR_MAXBOX)
    tiles = {}
    for lev in sorted(h.levels):
        ch, ms_t = h.autotune(lev, p, reps=2)
        tiles[str(lev)] = {"chosen": ch, "ms": [round(v, 3) for v in ms_t]}
    # x extents of the refined levels' boxes (the tiles the autotuner weighs them against)
    widths = {str(lev): {str(w): n for w, n in sorted(collections.Counter(
        hi[0] - lo[0] + 1 for lo, hi in info["boxes"]).items())} for lev, info in sorted(h.levels.items()) if lev > 0}
    h.advance(DT, p, flags=slh.SLH_USE_GRAPH)   # first capture outside the timed pass
    h.sync()
    h.profile(False, True)                       # clears the host-phase counters
    # pass 1: graph replay, regrids and re-captures included
    updates = 0
    regrid_s = 0.0
    boxes_seen = []
    t0 = time.perf_counter()
    for k in range(K):
        if k and k % AMR_EVERY == 0:
            h.sync()
            tr = time.perf_counter()
            h.regrid(AMR_LEVELS, AMR_NBUF, AMR_MAXBOX)
            regrid_s += time.perf_counter() - tr
            boxes_seen.append([len(info["boxes"]) for _, info in sorted(h.levels.items())])
        updates += sum(info["nvalid"] * 2 ** lev for lev, info in h.levels.items())
        h.advance(DT, p, flags=slh.SLH_USE_GRAPH)
    h.sync()
    el = time.perf_counter() - t0
    phases = {name: h.profile_read(kind)[:2] for name, kind in
              (("regrid_tags", slh.SLH_PROF_REGRID_TAGS), ("regrid_cluster", slh.SLH_PROF_REGRID_CLUSTER),
               ("regrid_build", slh.SLH_PROF_REGRID_BUILD), ("graph_capture", slh.SLH_PROF_GRAPH_CAPTURE))}
    cap_ms, ncap = phases["graph_capture"]
    # pass 2: the same kind of steps launched directly, per-kernel device time
    h.profile(True, True)
    upd2 = 0
    for k in range(K):
        upd2 += sum(info["nvalid"] * 2 ** lev for lev, info in h.levels.items())
        h.advance(DT, p)
    h.sync()
    kinds = {"stage": slh.SLH_PROF_STAGE, "ghost": slh.SLH_PROF_GHOST, "restrict": slh.SLH_PROF_RESTRICT,
             "diag": slh.SLH_PROF_DIAG, "time": slh.SLH_PROF_TIME}
    prof = {k: round(h.profile_read(v)[0], 3) for k, v in kinds.items()}
    st = h.profile_read(slh.SLH_PROF_STAGE)
    h.profile(False, True)
    stage_gbs = st[2] / (st[0] / 1e3) / 1e9 if st[0] > 0 else None
    det = {"levels": {str(l): {"boxes": len(info["boxes"]), "cells": info["nvalid"]} for l, info in h.levels.items()},
           "boxes_per_regrid": boxes_seen, "coarse_steps": K, "relax_coarse_steps": relax,
           "horizon": f"{relax} relaxation + {K} timed + {K} profiled coarse steps (config 3 states 400)",
           "seconds": el, "regrid_seconds": regrid_s,
           "regrid_phases_ms": {k: round(v[0], 2) for k, v in phases.items() if k != "graph_capture"},
           "graph": {"captures": ncap, "capture_ms_total": round(cap_ms, 2),
                     "capture_ms_per_regrid": round(cap_ms / max(1, ncap), 2),
                     "step_ms_excl_regrid_capture": round((el - regrid_s - cap_ms / 1e3) / K * 1e3, 3)},
           "device_ms_direct": prof, "direct_pass_cell_updates": upd2,
           "autotune_after_first_regrid": tiles, "box_x_extents_after_first_regrid": widths,
           "stage_kernels": {"achieved_gbs": stage_gbs, "frac": (stage_gbs / peak) if (stage_gbs and peak) else None,
                             "peak": peak},
           "cell_updates": updates, "eta_end": h.get_eta(0)}
    h.close()
    return updates / el, det


def run_ours(args, rank, world, local_rank, dist):
    import torch
    import paper_2404_02950_gb300 as slh
    from paper_2404_02950_gb300 import inputs
    if not os.path.exists(slh.LIB_PATH):
        from paper_2404_02950_gb300 import build
        build.build()
    torch.cuda.set_device(local_rank)
    n, K, W = args.cells, args.steps, args.warmup
    peak, peak_kind = _peaks()
    if args.profile_only == "amr":
        # short dynamic-AMR run for profilers (base n^3, K coarse steps)
        ya = inputs.gaussian_field(n, n / 8.0, seed=rank)
        _amr_form(slh, torch, "f32", slh.dense_from_boxes(ya, [((0, 0, 0), (n - 1,) * 3)]), K, n=n, peak=peak,
                  relax=args.amr_relax)
        return
    if args.profile_only == "gw":
        _gw_form(slh, torch, n, dist, peak, K=K)
        return
    if args.profile_only == "gw4":
        _c4_form(slh, torch, peak, n=n, K=K, W=W)
        return
    if args.profile_only == "alu":
        # FMA issue rates with the clocks sampled over the measurement
        with ClockSampler(_gpu_index(local_rank)) as clk:
            fma64 = slh.slh_alu_rate(slh.SLH_F64, 12)
            fma32 = slh.slh_alu_rate(slh.SLH_F32_KAHAN, 12)
        print(json.dumps({"fp64_fma_per_s": fma64, "fp64_tflops": 2 * fma64 / 1e12,
                          "fp32_fma_per_s": fma32, "fp32_tflops": 2 * fma32 / 1e12,
                          "sms": torch.cuda.get_device_properties(local_rank).multi_processor_count,
                          "clocks": clk.summary()}), flush=True)
        return
    y0 = inputs.gaussian_field(n, n / 16.0, seed=rank)
    boxes = [((0, 0, 0), (n - 1, n - 1, n - 1))]
    dense = slh.dense_from_boxes(y0, boxes)
    del y0
    flags = slh.SLH_FUSE_TAG | slh.SLH_FUSE_ENERGY

    # FP32 + Kahan (headline), with clock sampling over its timed region
    with ClockSampler(_gpu_index(local_rank)) as clk:
        h32, r32 = _time_form(slh, torch, "f32", dense, n, K, W, dist, flags,
                              tile=args.tile if args.profile_only else None,
                              diag_tile=args.diag_tile if args.profile_only else None)
    clocks = clk.summary()
    if args.profile_only:
        # short run for profilers: no e2e leg, no FP64 form, no JSON line
        h32.close()
        return
    # the FP32 state after the timed steps, kept on the device for the error
    # against the FP64 form on the same field and step count
    p6 = slh.EOMParams(order=ORDER)
    st32 = h32.get_state_device(0)
    len32 = float(h32.reduce_energy(p6, mode=0)[4])

    # end to end through the C ABI with host buffers: upload the step's input
    # from pinned memory, advance, read the step's energy back
    pinned = torch.from_numpy(dense.astype(np.float32)).pin_memory()
    p = slh.EOMParams(order=ORDER)
    h32.set_state(0, pinned)
    h32.advance(DT, p, flags=flags)
    h32.reduce_energy(p, mode=1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        h32.set_state(0, pinned)
        h32.advance(DT, p, flags=flags)
        h32.reduce_energy(p, mode=1)
    torch.cuda.synchronize()
    e2e_serial_s = time.perf_counter() - t0
    # the same steps with the uploads pipelined: step k's input goes from
    # pinned memory into one of two device staging buffers on a copy stream
    # while step k-1 computes, then slh_set_state moves it into the level
    # (device to device, on the library's stream)
    cstream = torch.cuda.Stream()
    staging = [torch.empty(pinned.shape, dtype=pinned.dtype, device="cuda") for _ in range(2)]
    uploaded = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def upload(i):
        with torch.cuda.stream(cstream):
            cstream.wait_event(consumed[i])
            staging[i].copy_(pinned, non_blocking=True)
            uploaded[i].record(cstream)

    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    upload(0)
    for k in range(K):
        i = k % 2
        h32.stream.wait_event(uploaded[i])
        h32.set_state(0, staging[i])
        consumed[i].record(h32.stream)
        if k + 1 < K:
            upload(1 - i)
        h32.advance(DT, p, flags=flags)
        h32.reduce_energy(p, mode=1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = pinned.numel() * 4
    h32.close()
    del h32, pinned, staging
    torch.cuda.empty_cache()

    # FP64 plain on the same field
    h64, r64 = _time_form(slh, torch, "f64", dense, n, K, W, dist, flags)
    err = _error_vs_f64(st32, h64.get_state_device(0), n ** 3, len32, float(h64.reduce_energy(p6, mode=0)[4]),
                        W + K)
    h64.close()
    del h64, st32
    torch.cuda.empty_cache()
    # the FP64 form's ALU roofline: the device's measured FP64 FMA rate
    fma64 = slh.slh_alu_rate(slh.SLH_F64, 5)
    fma32 = slh.slh_alu_rate(slh.SLH_F32_KAHAN, 5)

    # dynamic AMR (config 3 workload), FP32 batched and FP64 plain
    amr = None
    if not args.no_amr:
        ya = inputs.gaussian_field(AMR_N, AMR_N / 8.0, seed=rank)
        yad = slh.dense_from_boxes(ya, [((0, 0, 0), (AMR_N - 1,) * 3)])
        del ya
        v32, d32 = _amr_form(slh, torch, "f32", yad, AMR_K32, peak=peak)
        torch.cuda.empty_cache()
        v64, d64 = _amr_form(slh, torch, "f64", yad, AMR_K64, peak=peak)
        torch.cuda.empty_cache()
        amr = {"workload": AMR_WORKLOAD, "unit": "cell-updates/s",
               "f32": {"value": world * v32, **d32}, "f64": {"value": world * v64, **d64}}

    # the same workload with the low-storage SSPRK3 integrator (type 10)
    ssp = None
    if not args.no_ssp:
        hs, rs = _time_form(slh, torch, "f32", dense, n, K, W, dist, flags, integrator=10)
        hs.close()
        del hs
        torch.cuda.empty_cache()
        ach_s = rs["stage_bytes"] / (rs["stage_ms"] / 1e3) / 1e9
        ssp = {"workload": WORKLOAD.replace("classic RK4", "low-storage SSPRK3 (integrator type 10)"),
               "unit": "cell-updates/s", "value": world * float(n) ** 3 * K / (rs["ms"] / 1e3),
               "ms_per_step": rs["ms"] / K, "per_stage_ms": rs["per_stage_ms"][:3],
               "stage_achieved_gbs": ach_s, "hbm_frac": ach_s / peak, "alg_bytes_per_cell_update": 32 * 4,
               "precision": "FP32 (no compensation)"}

    # the same workload with RKN4 (integrator type 21)
    rkn = None
    if not args.no_rkn:
        hr, rr = _time_form(slh, torch, "f32", dense, n, K, W, dist, flags, integrator=21)
        hr.close()
        del hr
        torch.cuda.empty_cache()
        ach_r = rr["stage_bytes"] / (rr["stage_ms"] / 1e3) / 1e9
        rkn = {"workload": WORKLOAD.replace("classic RK4", "RKN4 (integrator type 21)"),
               "unit": "cell-updates/s", "value": world * float(n) ** 3 * K / (rr["ms"] / 1e3),
               "ms_per_step": rr["ms"] / K, "per_stage_ms": rr["per_stage_ms"],
               "stage_achieved_gbs": ach_r, "hbm_frac": ach_r / peak, "alg_bytes_per_cell_update": 72 * 4,
               "precision": "FP32 + Kahan"}

    # RKN5 (integrator type 22) needs an acceleration independent of Pi: the
    # same lattice and init with the friction term off
    rkn5 = None
    if not args.no_rkn:
        h5, r5 = _time_form(slh, torch, "f32", dense, n, K, W, dist, flags, integrator=22, friction=False)
        h5.close()
        del h5
        torch.cuda.empty_cache()
        ach_5 = r5["stage_bytes"] / (r5["stage_ms"] / 1e3) / 1e9
        rkn5 = {"workload": WORKLOAD.replace("classic RK4", "RKN5 (integrator type 22), friction off"),
                "unit": "cell-updates/s", "value": world * float(n) ** 3 * K / (r5["ms"] / 1e3),
                "ms_per_step": r5["ms"] / K, "per_stage_ms": r5["per_stage_ms"],
                "stage_achieved_gbs": ach_5, "hbm_frac": ach_5 / peak, "alg_bytes_per_cell_update": 66 * 4,
                "precision": "FP32 + Kahan"}

    # the same RK4 steps without the fused tags and energy (the paper tags at
    # regrid time only): what the diagnostics cost, and the stencil stages'
    # own share of the HBM roofline
    plain = None
    if not args.no_plain:
        hp, rp = _time_form(slh, torch, "f32", dense, n, K, W, dist, 0)
        hp.close()
        del hp
        torch.cuda.empty_cache()
        ach_p = rp["stage_bytes"] / (rp["stage_ms"] / 1e3) / 1e9
        plain = {"workload": WORKLOAD.replace(", tags+energy fused in stage 1", ", no fused tags or energy"),
                 "unit": "cell-updates/s", "value": world * float(n) ** 3 * K / (rp["ms"] / 1e3),
                 "ms_per_step": rp["ms"] / K, "per_stage_ms": rp["per_stage_ms"],
                 "stage_achieved_gbs": ach_p, "hbm_frac": ach_p / peak}

    # gravitational-wave tensor fields
    gw = None
    c4 = None
    if not args.no_gw:
        gw = _gw_form(slh, torch, GW_N, dist, peak)
        gw["value"] *= world
        c4 = _c4_form(slh, torch, peak)
        c4["value"] *= world

    ms = r32["ms"]
    e2e_ms = e2e_s * 1e3
    e2e_serial_ms = e2e_serial_s * 1e3
    ms, e2e_ms, e2e_serial_ms, ms64 = max_over_ranks(dist, [ms, e2e_ms, e2e_serial_ms, r64["ms"]], "cuda")
    cells = float(n) ** 3
    value = job_value(world, cells, K, ms)
    launches = r32["stage_launches"] + r32["ghost_launches"] + r32["time_launches"]
    achieved = r32["stage_bytes"] / (r32["stage_ms"] / 1e3) / 1e9
    ach64 = r64["stage_bytes"] / (r64["stage_ms"] / 1e3) / 1e9
    ops64 = fp64_ops_per_cell_update(ORDER) * cells * K / (r64["stage_ms"] / 1e3)
    if rank != 0:
        return
    line = {
        "metric": "cell-updates/s (one valid cell advanced one full RK4 step)",
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_CELLS else WORKLOAD.replace("512^3", f"{n}^3"), "cells": n ** 3, "order": ORDER, "precision": "FP32 + Kahan",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (10.9 GB of level buffers)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _stage_traffic(),
                     "kernel": "stage_kernel<float,3> (4 RK4 stages; tags + energy fused in stage 1)",
                     "peak_kind": peak_kind,
                     "alg_bytes_per_cell_update": KAHAN_VALUES * 4},
        "error_vs_f64": err,
        "fp64_plain": {"value": job_value(world, cells, K, ms64), "unit": "cell-updates/s",
                       "ms_per_step": ms64 / K, "stage_achieved_gbs": ach64,
                       "hbm_frac": ach64 / peak, "alg_bytes_per_cell_update": F64_VALUES * 8,
                       "alu_roofline": {"bound": "alu", "achieved": ops64 / 1e12, "peak": fma64 / 1e12,
                                        "unit": "T FP64 op/s", "frac": ops64 / fma64,
                                        "ops_per_cell_update": fp64_ops_per_cell_update(ORDER),
                                        "peak_kind": "measured live (slh_alu_rate: FP64 FMA issue rate)",
                                        "fp32_fma_per_s": fma32}},
        "stage_share": r32["stage_ms"] / ms,
        "per_stage_ms": {"f32": r32["per_stage_ms"], "f64": r64["per_stage_ms"]},
        "autotune": {"f32": {"chosen": r32["tile_variant"], "ms": r32["tune_ms"],
                             "diag_chosen": r32["diag_tile_variant"], "diag_ms": r32["diag_tune_ms"]},
                     "f64": {"chosen": r64["tile_variant"], "ms": r64["tune_ms"],
                             "diag_chosen": r64["diag_tile_variant"], "diag_ms": r64["diag_tune_ms"]}},
        "energy_f32": r32["energy"], "energy_f64": r64["energy"],
        "e2e": {"value": job_value(world, cells, K, e2e_ms), "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4 * 8,
                "method": "each step's input uploaded from pinned host memory on a copy stream while the "
                          "previous step computes (two device staging buffers), then slh_set_state, "
                          "slh_advance and the energy read back (slh_reduce_energy mode 1)",
                "serial": {"value": job_value(world, cells, K, e2e_serial_ms),
                           "method": "slh_set_state from pinned host memory, slh_advance, energy read back, "
                                     "one after the other"}},
        "amr": amr,
        "ssprk3": ssp,
        "rkn4": rkn,
        "rkn5": rkn5,
        "plain_step": plain,
        "gw": gw,
        "gw_1024_bf16": c4,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=N_CELLS, help="lattice cells per axis (default 512)")
    ap.add_argument("--no-amr", action="store_true", help="skip the dynamic-AMR line")
    ap.add_argument("--no-gw", action="store_true", help="skip the gravitational-wave tensor line")
    ap.add_argument("--no-ssp", action="store_true", help="skip the SSPRK3 line")
    ap.add_argument("--no-plain", action="store_true", help="skip the line without fused diagnostics")
    ap.add_argument("--no-rkn", action="store_true", help="skip the RKN4 and RKN5 lines")
    ap.add_argument("--tile", type=int, default=None,
                    help="with --profile-only: use this stage-kernel tile variant instead of autotuning")
    ap.add_argument("--amr-relax", type=int, default=AMR_RELAX,
                    help="--profile-only amr: coarse steps of the base level before the first regrid")
    ap.add_argument("--diag-tile", type=int, default=None,
                    help="with --profile-only --tile: the diagnostics stage-1 tile variant (default: --tile)")
    ap.add_argument("--profile-only", nargs="?", const="uniform", default=None, choices=["uniform", "amr", "gw", "gw4", "alu"],
                    help="short run for ncu captures of a small case, printing nothing: the FP32 uniform form "
                         "(default), the dynamic-AMR form (base --cells^3, --steps coarse steps), the "
                         "16-field lattice or the BF16 16-field hierarchy (base --cells^3); 'alu' prints "
                         "the device's measured FP64 and FP32 FMA rates with the clocks seen")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
        dist = td
    run_ours(args, rank, world, local_rank, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
