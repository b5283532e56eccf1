"""GB300-native AMR axion-string stepper (arXiv:2404.02950, sledgehamr).

Thin Python binding of the C ABI declared in ``include/slh.h``: every
function below marshals arguments and calls the CUDA library
``lib/libslh.so``; every step of the computation runs in its kernels.
PyTorch provides device memory (the level buffers) and the CUDA stream.
There is no CPU fallback: a missing library raises.

Low-level names mirror the ABI (``slh_create``, ``slh_init_level``,
``slh_rk_step``, ``slh_advance``, ``slh_tag``, ``slh_tag_blocks``,
``slh_fill_ghosts``, ``slh_regrid_boxes``, ``slh_reduce_energy`` ...);
``Hierarchy`` bundles a context with the torch buffers it needs.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libslh.so")

SLH_OK = 0
SLH_F64 = 0
SLH_F32_KAHAN = 2
SLH_F32_BF16 = 3
SLH_SLOTS_BF16 = 10   # 4 FP32 slots (psi, Pi) + 6 slots of BF16 pairs (u_ij, v_ij)
SLH_NBUF = 5
SLH_BUF_Y, SLH_BUF_YA, SLH_BUF_YB, SLH_BUF_D, SLH_BUF_C = range(5)
SLH_FUSE_TAG = 1
SLH_FUSE_ENERGY = 2
SLH_USE_GRAPH = 4
SLH_GHOSTS = 0
SLH_RESTRICT = 1
SLH_TAG_WINDING, SLH_TAG_TEE = 1, 2
SLH_REGRID_GLOBAL, SLH_REGRID_LOCAL, SLH_REGRID_AUTO = 0, 1, 2
(SLH_PROF_STAGE, SLH_PROF_GHOST, SLH_PROF_RESTRICT, SLH_PROF_DIAG, SLH_PROF_TIME,
 SLH_PROF_S1, SLH_PROF_S2, SLH_PROF_S3, SLH_PROF_S4, SLH_PROF_GW, SLH_PROF_KO,
 SLH_PROF_REGRID_TAGS, SLH_PROF_REGRID_CLUSTER, SLH_PROF_REGRID_BUILD, SLH_PROF_GRAPH_CAPTURE) = range(15)
NFIELDS, NFIELDS_GW = 4, 16   # psi1, psi2, Pi1, Pi2 (+ u_xx..u_yz, v_xx..v_yz)

ERRORS = {-1: "INVALID_ARG", -2: "OUT_OF_RANGE", -3: "CUDA", -4: "TIMEOUT", -5: "NOMEM",
          -6: "DEVICE", -7: "STATE"}

# every entry point declared in include/slh.h
ABI_SYMBOLS = (
    "slh_last_error", "slh_create", "slh_destroy", "slh_level_layout", "slh_init_level",
    "slh_set_state", "slh_get_state", "slh_set_eta", "slh_get_eta", "slh_rk_step",
    "slh_advance", "slh_fill_ghosts", "slh_tag", "slh_tag_blocks", "slh_regrid_boxes",
    "slh_reduce_energy", "slh_sync", "slh_profile", "slh_profile_read", "slh_set_tile", "slh_set_diag_tile",
    "slh_autotune", "slh_autotune_diag",
    "slh_energy_noalloc", "slh_regrid_level", "slh_selftest_wait_timeout",
    "slh_set_tagging", "slh_shadow_init", "slh_shadow_compare", "slh_tee_tags", "slh_gw_spectrum",
    "slh_local_regrid_boxes", "slh_regrid", "slh_level_roles", "slh_alu_rate",
)


class SlhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"slh error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class slh_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int32 * 3), ("hi", ctypes.c_int32 * 3)]


class slh_eom_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("a", ctypes.c_double), ("friction", ctypes.c_int32),
                ("eta_power", ctypes.c_int32), ("lap_order", ctypes.c_int32),
                ("interp_type", ctypes.c_int32), ("integrator", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("ko_eps", ctypes.c_double), ("ko_order", ctypes.c_int32), ("pad2_", ctypes.c_int32)]


class slh_regrid_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("start", ctypes.c_int32),
                ("n_error_buf", ctypes.c_int32), ("max_box", ctypes.c_int32), ("interp_type", ctypes.c_int32),
                ("max_local", ctypes.c_int32), ("pad_", ctypes.c_int32), ("eps_strong", ctypes.c_double),
                ("eps_weak", ctypes.c_double)]


# the caller's allocator slh_regrid calls for every level it rebuilds
SLH_LEVEL_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(slh_box),
                                      ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p))


@dataclass(frozen=True)
class EOMParams:
    """Coefficients of Sec. 3.1: lambda, a, friction on/off, eta power of the
    potential coefficient, Laplacian accuracy order, ghost interpolation,
    the integrator type (4 classic RK4, 10 low-storage SSPRK3, 21 RKN4, 22 RKN5
    with friction off) and the
    Kreiss-Oliger dissipation order (0 off, 1/3/5) and strength (Sec. 2.4)."""
    lam: float = 1.0
    a: float = 0.0
    friction: bool = True
    eta_power: int = 2
    order: int = 2
    interp_type: int = 4
    integrator: int = 4
    ko_order: int = 0
    ko_eps: float = 0.0

    def c(self):
        return slh_eom_params(self.lam, self.a, int(self.friction), self.eta_power, self.order,
                              self.interp_type, self.integrator, 0, self.ko_eps, self.ko_order, 0)


_lib = None


def lib():
    """Load ``libslh.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_02950_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "slh_last_error": (ctypes.c_char_p, []),
        "slh_create": (i32, [P(vp), i32, dbl, i32, i32, i32, i32, i32, vp]),
        "slh_destroy": (None, [vp]),
        "slh_level_layout": (i32, [i32, i32, P(slh_box), i32, P(i64), P(i64), P(i64), P(i64)]),
        "slh_init_level": (i32, [vp, i32, P(slh_box), i32, P(vp), vp]),
        "slh_set_state": (i32, [vp, i32, vp, i32]),
        "slh_get_state": (i32, [vp, i32, vp, i32]),
        "slh_set_eta": (i32, [vp, dbl]),
        "slh_get_eta": (i32, [vp, i32, P(dbl)]),
        "slh_rk_step": (i32, [vp, i32, i32, dbl, P(slh_eom_params), ctypes.c_uint32]),
        "slh_advance": (i32, [vp, dbl, P(slh_eom_params), ctypes.c_uint32]),
        "slh_fill_ghosts": (i32, [vp, i32, dbl, i32, i32]),
        "slh_tag": (i32, [vp, i32, vp, P(i64)]),
        "slh_tag_blocks": (i32, [vp, i32, i32, vp]),
        "slh_regrid_boxes": (i32, [vp, P(i32), i32, i32, i32, P(slh_box), i32, P(slh_box), i32, P(i32)]),
        "slh_reduce_energy": (i32, [vp, P(slh_eom_params), i32, P(dbl)]),
        "slh_sync": (i32, [vp]),
        "slh_profile": (i32, [vp, i32, i32]),
        "slh_profile_read": (i32, [vp, i32, P(dbl), P(i64), P(dbl)]),
        "slh_set_tile": (i32, [vp, i32, i32]),
        "slh_autotune": (i32, [vp, i32, P(slh_eom_params), i32, P(i32), P(dbl)]),
        "slh_set_diag_tile": (i32, [vp, i32, i32]),
        "slh_autotune_diag": (i32, [vp, i32, P(slh_eom_params), i32, P(i32), P(dbl)]),
        "slh_energy_noalloc": (i32, [vp, i32, i32, dbl, dbl, P(slh_eom_params), vp, vp]),
        "slh_regrid_level": (i32, [vp, i32, P(slh_box), i32, P(vp), vp, i32]),
        "slh_selftest_wait_timeout": (i32, [vp, i64]),
        "slh_set_tagging": (i32, [vp, ctypes.c_uint32, P(dbl)]),
        "slh_shadow_init": (i32, [vp, vp]),
        "slh_shadow_compare": (i32, [vp, vp]),
        "slh_tee_tags": (i32, [vp, i32, vp, i32]),
        "slh_gw_spectrum": (i32, [vp, i32, P(i64), P(dbl), i32, P(i32)]),
        "slh_local_regrid_boxes": (i32, [i32, i32, i32, P(vp), P(slh_box), P(i32), P(slh_box), i32, P(i32)]),
        "slh_regrid": (i32, [vp, P(slh_regrid_params), SLH_LEVEL_ALLOC_FN, vp, P(i32), P(dbl)]),
        "slh_level_roles": (i32, [vp, i32, P(i32)]),
        "slh_alu_rate": (i32, [i32, i32, P(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != SLH_OK:
        msg = lib().slh_last_error().decode(errors="replace")
        raise SlhError(status, msg)


def _boxes(boxes):
    arr = (slh_box * max(1, len(boxes)))()
    for i, (lo, hi) in enumerate(boxes):
        arr[i].lo[:] = [int(v) for v in lo]
        arr[i].hi[:] = [int(v) for v in hi]
    return arr


# ---------------------------------------------------------------------------
# ABI-named wrappers

def slh_level_layout(nghost, boxes, nfields=NFIELDS):
    """(box_offsets, box_geom (n,4), total_elems, nvalid) of a level layout."""
    n = len(boxes)
    offs = (ctypes.c_int64 * max(1, n))()
    geom = (ctypes.c_int64 * max(1, 4 * n))()
    tot, nv = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().slh_level_layout(nghost, nfields, _boxes(boxes), n, offs, geom, ctypes.byref(tot),
                                  ctypes.byref(nv)))
    return (np.array(offs[:n], dtype=np.int64), np.array(geom[:4 * n], dtype=np.int64).reshape(n, 4),
            tot.value, nv.value)


def slh_regrid_boxes(tags, blocking_factor, n_error_buf, max_box, parent=None):
    """Host-only regrid of a dense uint8 tag array [z, y, x] (Sec. 2.2-2.3);
    returns [((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)), ...] of the finer level."""
    t = np.ascontiguousarray(np.asarray(tags, dtype=np.uint8))
    dims = (ctypes.c_int32 * 3)(t.shape[2], t.shape[1], t.shape[0])
    par = _boxes(parent) if parent else None
    npar = len(parent) if parent else 0
    nout = ctypes.c_int32(0)
    cap = 64
    while True:
        out = (slh_box * cap)()
        st = lib().slh_regrid_boxes(t.ctypes.data, dims, blocking_factor, n_error_buf, max_box, par, npar,
                                    out, cap, ctypes.byref(nout))
        if st == -2 and nout.value > cap:
            cap = nout.value
            continue
        _check(st)
        return [(tuple(out[i].lo), tuple(out[i].hi)) for i in range(nout.value)]


def slh_local_regrid_boxes(level_boxes, n0, blocking_factor, masks):
    """Local regrid (Sec. 2.3), host only: every level's boxes kept, new blocks
    of level l+1 where the block mask of level l (grown tags in blocks of
    blocking_factor/2 cells, as from slh_tag_blocks) is not covered by level
    l+1, coarser levels grown where nesting needs it.  Returns the new box
    lists (old boxes first)."""
    L = len(level_boxes)
    flat = [b for lb in level_boxes for b in lb]
    nb = (ctypes.c_int32 * L)(*[len(lb) for lb in level_boxes])
    keep = [np.ascontiguousarray(np.asarray(m, dtype=np.uint8)) for m in masks]
    mp = (ctypes.c_void_p * max(1, L))(*([m.ctypes.data for m in keep] + [None] * (max(1, L) - len(keep))))
    cap = max(64, 4 * len(flat))
    counts = (ctypes.c_int32 * L)()
    while True:
        out = (slh_box * cap)()
        st = lib().slh_local_regrid_boxes(L, n0, blocking_factor, mp, _boxes(flat), nb, out, cap, counts)
        if st == -2 and sum(counts) > cap:
            cap = sum(counts)
            continue
        _check(st)
        res, o = [], 0
        for l in range(L):
            res.append([(tuple(out[o + i].lo), tuple(out[o + i].hi)) for i in range(counts[l])])
            o += counts[l]
        return res


def slh_energy_noalloc(fields_dev, n, dx, eta, params: EOMParams, out_dev, stream=None):
    """Energy and string length of a dense periodic lattice without any
    device allocation (for callers that cannot allocate; the library keeps
    the reduction scratch in a fixed device array, lattice side <= 4096).
    fields_dev: CUDA tensor (4, n, n, n) float64 or float32; out_dev: CUDA
    float64 tensor of 5 elements, written asynchronously on ``stream``
    (default: the current torch stream)."""
    import torch
    # the C call sees raw pointers only: every size and type is checked here
    n = int(n)
    if not (isinstance(fields_dev, torch.Tensor) and fields_dev.is_cuda):
        raise ValueError("fields_dev must be a CUDA tensor")
    if fields_dev.dtype not in (torch.float64, torch.float32):
        raise ValueError(f"fields_dev must be float64 or float32, not {fields_dev.dtype}")
    if not fields_dev.is_contiguous():
        raise ValueError("fields_dev must be contiguous")
    if n < 1 or fields_dev.numel() < 4 * n ** 3:
        raise ValueError(f"fields_dev holds {fields_dev.numel()} values, fewer than 4 n^3 = {4 * n ** 3}")
    if not (isinstance(out_dev, torch.Tensor) and out_dev.is_cuda and out_dev.dtype == torch.float64
            and out_dev.is_contiguous() and out_dev.numel() >= 5):
        raise ValueError("out_dev must be a contiguous CUDA float64 tensor of at least 5 values")
    if out_dev.device != fields_dev.device:
        raise ValueError("fields_dev and out_dev must be on the same device")
    prec = SLH_F64 if fields_dev.dtype == torch.float64 else SLH_F32_KAHAN
    p = params.c()
    # the library looks up its scratch array on the current device
    with torch.cuda.device(fields_dev.device):
        st = torch.cuda.current_stream(fields_dev.device) if stream is None else stream
        _check(lib().slh_energy_noalloc(ctypes.c_void_p(fields_dev.data_ptr()), n, prec, float(dx), float(eta),
                                        ctypes.byref(p), ctypes.c_void_p(out_dev.data_ptr()),
                                        ctypes.c_void_p(st.cuda_stream)))


def slh_alu_rate(prec=SLH_F64, reps=5):
    """Measured fused multiply-adds per second of the current device, FP64
    (``SLH_F64``) or FP32 (``SLH_F32_KAHAN``): the ALU roofline of the FP64
    form.  Synchronises the device."""
    out = ctypes.c_double(0.0)
    _check(lib().slh_alu_rate(int(prec), int(reps), ctypes.byref(out)))
    return out.value


def _bf16_bits(a):
    """float32 -> BF16 bit patterns (uint32, low 16 bits), rounded to
    nearest even (finite values)."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32)


def pack_bf16_fields(fields):
    """The 16 fields (psi1, psi2, Pi1, Pi2, u_xx..u_yz, v_xx..v_yz) as the
    10 slots of an SLH_F32_BF16 level: the scalar fields in FP32, the tensor
    fields rounded to BF16 and paired, (u_xx, u_yy), (u_zz, u_xy), (u_xz, u_yz),
    (v_xx, v_yy), ... with the first field of a pair in the low half.  Returns
    float32 arrays (the pairs as raw bit patterns)."""
    assert len(fields) == 16
    out = [np.asarray(f, dtype=np.float32) for f in fields[:4]]
    for k in range(4, 16, 2):
        w = _bf16_bits(fields[k]) | (_bf16_bits(fields[k + 1]) << 16)
        out.append(w.astype(np.uint32).view(np.float32))
    return out


def unpack_bf16_fields(slots):
    """Inverse of pack_bf16_fields: the 16 fields as float32 arrays (the
    tensor fields widened exactly from BF16)."""
    assert len(slots) == SLH_SLOTS_BF16
    out = [np.asarray(s, dtype=np.float32) for s in slots[:4]]
    for s in slots[4:]:
        w = np.ascontiguousarray(np.asarray(s, dtype=np.float32)).view(np.uint32)
        out.append((w << 16).astype(np.uint32).view(np.float32))
        out.append((w & 0xFFFF0000).astype(np.uint32).view(np.float32))
    return out


def dense_from_boxes(fields, boxes):
    """Pack the [z, y, x] domain arrays of the fields (4 or 16) into the
    dense valid-cell layout [box][comp][z][y][x] (host numpy)."""
    parts = []
    for lo, hi in boxes:
        for c in range(len(fields)):
            parts.append(np.asarray(fields[c])[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].ravel())
    return np.concatenate(parts)


def boxes_from_dense(dense, boxes, nfields=NFIELDS):
    """Split a dense valid-cell array into per-box (nfields, nz, ny, nx) arrays."""
    out, off = [], 0
    for lo, hi in boxes:
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        vol = n[0] * n[1] * n[2]
        out.append(np.asarray(dense[off:off + nfields * vol]).reshape(nfields, n[2], n[1], n[0]))
        off += nfields * vol
    return out


class Hierarchy:
    """A context plus the torch-allocated buffers of its levels.

    n0: level-0 cells per axis; dx0: level-0 spacing; nghost: ghost layers;
    bf: blocking factor; prec: 'f64' or 'f32' (FP32 + Kahan); gw: also evolve
    the gravitational-wave tensor (16 fields per cell instead of 4)."""

    def __init__(self, n0, dx0, nghost=3, bf=8, prec="f64", max_levels=1, device="cuda:0", stream=None,
                 gw=False):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.prec = {"f64": SLH_F64, "f32": SLH_F32_KAHAN, "f32bf16": SLH_F32_BF16}[prec]
        if self.prec == SLH_F32_BF16 and not gw:
            raise ValueError("BF16 storage is for the tensor fields: prec='f32bf16' needs gw=True")
        self.dtype = torch.float64 if self.prec == SLH_F64 else torch.float32
        self.np_dtype = np.float64 if self.prec == SLH_F64 else np.float32
        # a stream of its own: CUDA graphs cannot capture the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.nghost, self.bf, self.n0, self.dx0 = nghost, bf, n0, dx0
        self.ncomp = NFIELDS_GW if gw else NFIELDS
        # storage slots per cell (elements of the buffers' dtype)
        self.nslots = SLH_SLOTS_BF16 if self.prec == SLH_F32_BF16 else self.ncomp
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().slh_create(ctypes.byref(h), n0, dx0, nghost, bf, self.prec, max_levels, self.ncomp,
                                    ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self.levels = {}

    def close(self):
        if self.h:
            lib().slh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _needs(self, i):
        """Whether level buffer i is allocated: three for BF16 storage
        (SSPRK3), no Kahan compensation in FP64."""
        if self.prec == SLH_F32_BF16:
            return i in (SLH_BUF_Y, SLH_BUF_YA, SLH_BUF_YB)
        return not (i == SLH_BUF_C and self.prec == SLH_F64)

    def init_level(self, lev, boxes, fused_tags=False):
        torch = self.torch
        _, geom, total, nvalid = slh_level_layout(self.nghost, boxes, self.nslots)
        bufs = [torch.empty(int(total), dtype=self.dtype, device=self.device) if self._needs(i) else None
                for i in range(SLH_NBUF)]
        tags = torch.zeros(int(nvalid), dtype=torch.uint8, device=self.device) if fused_tags else None
        ptrs = (ctypes.c_void_p * SLH_NBUF)(*[b.data_ptr() if b is not None else None for b in bufs])
        _check(lib().slh_init_level(self.h, lev, _boxes(boxes), len(boxes), ptrs,
                                    ctypes.c_void_p(tags.data_ptr()) if tags is not None else None))
        for l in list(self.levels):
            if l >= lev:
                del self.levels[l]
        self.levels[lev] = dict(boxes=list(boxes), bufs=bufs, tags=tags, nvalid=int(nvalid), total=int(total),
                                steps=0)
        return self.levels[lev]

    def roles(self, lev):
        """(state, previous state, stage scratch) buffer indices of the level
        (they rotate from step to step)."""
        r = (ctypes.c_int32 * 3)()
        _check(lib().slh_level_roles(self.h, lev, r))
        return tuple(r)

    def state_buffer(self, lev):
        """The torch buffer currently holding the level's state."""
        return self.levels[lev]["bufs"][self.roles(lev)[0]]

    def _alloc_level(self, boxes, fused_tags):
        torch = self.torch
        _, geom, total, nvalid = slh_level_layout(self.nghost, boxes, self.nslots)
        bufs = [torch.empty(int(total), dtype=self.dtype, device=self.device) if self._needs(i) else None
                for i in range(SLH_NBUF)]
        tags = torch.zeros(int(nvalid), dtype=torch.uint8, device=self.device) if fused_tags else None
        return bufs, tags, int(total), int(nvalid)

    def regrid_level(self, lev, boxes, interp_type=4, fused_tags=None):
        """Give level ``lev`` new boxes (copy where the old level covers,
        prolong elsewhere); empty ``boxes`` removes it and every finer level."""
        if not boxes:
            _check(lib().slh_regrid_level(self.h, lev, None, 0, None, None, interp_type))
            for l in list(self.levels):
                if l >= lev:
                    del self.levels[l]
            return None
        old = self.levels.get(lev)
        if fused_tags is None:
            fused_tags = old is not None and old["tags"] is not None
        bufs, tags, total, nvalid = self._alloc_level(boxes, fused_tags)
        ptrs = (ctypes.c_void_p * SLH_NBUF)(*[b.data_ptr() if b is not None else None for b in bufs])
        _check(lib().slh_regrid_level(self.h, lev, _boxes(boxes), len(boxes), ptrs,
                                      ctypes.c_void_p(tags.data_ptr()) if tags is not None else None, interp_type))
        self.levels[lev] = dict(boxes=list(boxes), bufs=bufs, tags=tags, nvalid=nvalid, total=total, steps=0)
        return self.levels[lev]

    def _regrid(self, mode, max_levels, n_error_buf, max_box, interp_type=4, start=0, eps_strong=0.1,
                eps_weak=0.05, max_local=10):
        """One slh_regrid call; this side only allocates the buffers the
        library asks for.  Returns (kind, [(level, boxes) rebuilt, in order],
        per-level values of slh_regrid's frac output)."""
        rp = slh_regrid_params(mode, max_levels, start, n_error_buf, max_box, interp_type,
                               0 if max_local is None else max_local, 0, eps_strong, eps_weak)
        done = []

        def alloc(user, lev, boxes, nboxes, total, nvalid, bufs, tags):
            try:
                if nboxes == 0:
                    done.append((lev, None))
                    return 0
                bl = [(tuple(boxes[i].lo), tuple(boxes[i].hi)) for i in range(nboxes)]
                old = self.levels.get(lev)
                fused = old is not None and old["tags"] is not None
                nb, nt, tot, nv = self._alloc_level(bl, fused)
                assert tot == total and nv == nvalid
                for i in range(SLH_NBUF):
                    bufs[i] = nb[i].data_ptr() if nb[i] is not None else None
                tags[0] = nt.data_ptr() if nt is not None else None
                done.append((lev, dict(boxes=bl, bufs=nb, tags=nt, nvalid=nv, total=tot, steps=0)))
                return 0
            except Exception:   # the library reports SLH_ERR_NOMEM
                return -5

        cb = SLH_LEVEL_ALLOC_FN(alloc)
        kind = ctypes.c_int32(-1)
        nl = len(self.levels)
        frac = (ctypes.c_double * max(1, nl))()
        st = lib().slh_regrid(self.h, ctypes.byref(rp), cb, None, ctypes.byref(kind), frac)
        # the levels rebuilt before a failure stay in place: keep their buffers
        for lev, info in done:
            if info is None:
                for l in list(self.levels):
                    if l >= lev:
                        del self.levels[l]
            else:
                self.levels[lev] = info
        _check(st)
        return kind.value, [(lev, info["boxes"] if info else []) for lev, info in done], list(frac[:nl])

    def regrid(self, max_levels, n_error_buf, max_box, interp_type=4, start=0):
        """Global regrid of every level above ``start`` (Sec. 2.2-2.3, one
        slh_regrid call).  Returns the new box lists in order."""
        _, lists, _ = self._regrid(SLH_REGRID_GLOBAL, max_levels, n_error_buf, max_box, interp_type, start)
        return [b for _, b in lists]

    def regrid_local(self, n_error_buf, interp_type=4, max_box=None):
        """Local regrid of every level (Sec. 2.3, one slh_regrid call).
        Returns the cells added per level."""
        mb = max_box if max_box is not None else self.bf
        _, _, added = self._regrid(SLH_REGRID_LOCAL, len(self.levels), n_error_buf, mb, interp_type)
        return [int(a) for a in added]

    def regrid_auto(self, max_levels, n_error_buf, max_box, interp_type=4, eps_strong=0.1, eps_weak=0.05,
                    max_local=10):
        """Local regrids with the paper's fallback to a global one (Sec. 2.3,
        decided by the library).  Returns ("global", box lists) or ("local",
        per-level added-volume fractions)."""
        kind, lists, frac = self._regrid(SLH_REGRID_AUTO, max_levels, n_error_buf, max_box, interp_type,
                                         eps_strong=eps_strong, eps_weak=eps_weak, max_local=max_local)
        if kind == SLH_REGRID_GLOBAL:
            return "global", [b for _, b in lists]
        return "local", frac

    def set_state(self, lev, dense):
        """dense: host numpy array (or CUDA tensor) in the dense valid-cell
        layout of the context precision."""
        torch = self.torch
        if isinstance(dense, torch.Tensor):
            t = dense.to(self.dtype).contiguous()
            _check(lib().slh_set_state(self.h, lev, ctypes.c_void_p(t.data_ptr()), 0 if t.is_cuda else 1))
            if not t.is_cuda:
                self.sync()
            self._keep = t
        else:
            a = np.ascontiguousarray(np.asarray(dense, dtype=self.np_dtype))
            _check(lib().slh_set_state(self.h, lev, ctypes.c_void_p(a.ctypes.data), 1))
            self.sync()

    def get_state(self, lev):
        n = self.nslots * self.levels[lev]["nvalid"]
        out = np.empty(n, dtype=self.np_dtype)
        _check(lib().slh_get_state(self.h, lev, ctypes.c_void_p(out.ctypes.data), 1))
        return out

    def get_state_device(self, lev):
        """The level's valid cells in the dense layout, as a CUDA tensor
        (device-to-device copy on the library's stream)."""
        out = self.torch.empty(self.nslots * self.levels[lev]["nvalid"], dtype=self.dtype, device=self.device)
        _check(lib().slh_get_state(self.h, lev, ctypes.c_void_p(out.data_ptr()), 0))
        self.sync()
        return out

    def set_eta(self, eta):
        _check(lib().slh_set_eta(self.h, float(eta)))

    def get_eta(self, lev=0):
        v = ctypes.c_double()
        _check(lib().slh_get_eta(self.h, lev, ctypes.byref(v)))
        return v.value

    def rk_step(self, lev, dt0, params: EOMParams, sub=0, flags=0):
        p = params.c()
        _check(lib().slh_rk_step(self.h, lev, sub, float(dt0), ctypes.byref(p), flags))
        self.levels[lev]["steps"] += 1

    def advance(self, dt0, params: EOMParams, flags=0):
        p = params.c()
        _check(lib().slh_advance(self.h, float(dt0), ctypes.byref(p), flags))
        for l, info in self.levels.items():
            info["steps"] += 2 ** l

    def fill_ghosts(self, lev, alpha=1.0, interp_type=4, mode=SLH_GHOSTS):
        _check(lib().slh_fill_ghosts(self.h, lev, float(alpha), interp_type, mode))

    def tag(self, lev):
        t = self.torch.zeros(self.levels[lev]["nvalid"], dtype=self.torch.uint8, device=self.device)
        n = ctypes.c_int64()
        _check(lib().slh_tag(self.h, lev, ctypes.c_void_p(t.data_ptr()), ctypes.byref(n)))
        return t, n.value

    def tag_blocks(self, lev, n_error_buf):
        nb = (self.n0 << lev) // (self.bf // 2)
        m = np.zeros((nb, nb, nb), dtype=np.uint8)
        _check(lib().slh_tag_blocks(self.h, lev, n_error_buf, ctypes.c_void_p(m.ctypes.data)))
        return m

    def reduce_energy(self, params: EOMParams, mode=0):
        p = params.c()
        out = (ctypes.c_double * 5)()
        _check(lib().slh_reduce_energy(self.h, ctypes.byref(p), mode, out))
        return np.array(out[:])

    def sync(self):
        _check(lib().slh_sync(self.h))

    def set_tile(self, lev, variant):
        _check(lib().slh_set_tile(self.h, lev, variant))

    def set_diag_tile(self, lev, variant):
        _check(lib().slh_set_diag_tile(self.h, lev, variant))

    def autotune(self, lev, params: EOMParams, reps=3, nvariants=8, diag=False):
        """Time every stage-kernel tile variant on this level; keep the fastest.
        diag: tune the diagnostics stage 1 (fused tags and energy) instead of
        the plain stages.  Returns (chosen index, [ms per variant])."""
        p = params.c()
        ch = ctypes.c_int32()
        ms = (ctypes.c_double * nvariants)(*([-1.0] * nvariants))
        fn = lib().slh_autotune_diag if diag else lib().slh_autotune
        _check(fn(self.h, lev, ctypes.byref(p), reps, ctypes.byref(ch), ms))
        return ch.value, [v for v in ms[:] if v >= 0]

    def fused_tags(self, lev):
        """Host copy of the tags written by the last SLH_FUSE_TAG stage 1."""
        self.sync()
        return self.levels[lev]["tags"].cpu().numpy()

    def set_tagging(self, winding=True, te_crit=None):
        """Refinement criteria of slh_tag_blocks / regrid: the string winding
        and/or the truncation-error estimate with thresholds te_crit of
        (psi1, psi2, Pi1, Pi2) (Sec. 2.2)."""
        crit = (SLH_TAG_WINDING if winding else 0) | (SLH_TAG_TEE if te_crit is not None else 0)
        eps = (ctypes.c_double * 4)(*[float(v) for v in te_crit]) if te_crit is not None else None
        _check(lib().slh_set_tagging(self.h, crit, eps))

    def make_shadow(self):
        """The shadow context of level 0 (n0/2 cells of spacing 2 dx0, one
        box), for the level-0 truncation-error estimate."""
        n = self.n0 // 2
        bf = self.bf if n % self.bf == 0 else max(2, self.bf // 2)
        sh = Hierarchy(n, 2.0 * self.dx0, nghost=self.nghost, bf=bf,
                       prec="f64" if self.prec == SLH_F64 else "f32", max_levels=1, device=self.device,
                       gw=self.ncomp == NFIELDS_GW)
        sh.init_level(0, [((0, 0, 0), (self.n0 // 2 - 1,) * 3)])
        return sh

    def shadow_init(self, shadow):
        _check(lib().slh_shadow_init(self.h, shadow.h))

    def shadow_compare(self, shadow):
        _check(lib().slh_shadow_compare(self.h, shadow.h))

    def tee_tags(self, lev):
        """Host copy of level lev's truncation-error-estimate tags (dense)."""
        out = np.empty(self.levels[lev]["nvalid"], dtype=np.uint8)
        _check(lib().slh_tee_tags(self.h, lev, ctypes.c_void_p(out.ctypes.data), 1))
        return out

    def gw_spectrum(self, ptype=2):
        """(n2, G): the unbinned gravitational-wave spectrum of level 0
        (Sec. 7.4) for projection type 1 or 2."""
        cap = 3 * (self.n0 // 2) ** 2 + 1
        n2 = np.empty(cap, dtype=np.int64)
        g = np.empty(cap, dtype=np.float64)
        nout = ctypes.c_int32()
        _check(lib().slh_gw_spectrum(self.h, ptype, n2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap, ctypes.byref(nout)))
        return n2[:nout.value].copy(), g[:nout.value].copy()

    def profile(self, enable=True, reset=True):
        _check(lib().slh_profile(self.h, int(enable), int(reset)))

    def profile_read(self, kind):
        ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().slh_profile_read(self.h, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
        return ms.value, n.value, b.value
