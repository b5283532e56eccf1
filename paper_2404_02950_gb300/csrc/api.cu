// C ABI of the GB300 AMR stepper: context and level management, state I/O,
// the RK4 step of one level (Tab. "integrator", type 4), the subcycled
// coarse step (Sec. 2.1, Fig. 2) with optional CUDA-graph replay, and the
// synchronising diagnostics (tags, energy, regrid block mask).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "slh_internal.cuh"

namespace slh {

// NVTX range over a host-side phase (a level step, a ghost fill, a regrid):
// a profiler that records NVTX can select one by name; without one the push
// and pop are no-ops
struct NvtxRange {
  NvtxRange(const char* fmt, int a, int b = 0) {
    char buf[64];
    snprintf(buf, sizeof buf, fmt, a, b);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

static thread_local std::string g_last_error;

slh_status fail(slh_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

slh_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SLH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

bool make_layout(int g, int ncomp, const slh_box* boxes, int nboxes, Layout* out, std::string* why) {
  out->boxes.clear();
  long long off = 0, voff = 0;
  for (int b = 0; b < nboxes; ++b) {
    BoxDev B;
    memset(&B, 0, sizeof(B));
    for (int d = 0; d < 3; ++d) {
      B.lo[d] = boxes[b].lo[d];
      B.n[d] = boxes[b].hi[d] - boxes[b].lo[d] + 1;
      if (B.n[d] <= 0) {
        if (why) *why = "box " + std::to_string(b) + " has hi < lo";
        return false;
      }
    }
    B.pitch = (int)round_up(XPAD + B.n[0] + g, 8);
    B.pny = B.n[1] + 2 * g;
    B.pnz = B.n[2] + 2 * g;
    B.cs = round_up((long long)B.pitch * B.pny * B.pnz, 32);
    off = round_up(off, 64);
    B.off = off;
    off += ncomp * B.cs;
    B.voff = voff;
    voff += (long long)B.n[0] * B.n[1] * B.n[2];
    out->boxes.push_back(B);
  }
  out->total = round_up(off, 64);
  out->nvalid = voff;
  return true;
}

void prof_begin(slh_ctx* c, int kind, double bytes) {
  if (!c->prof) return;
  ProfRec r;
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  r.kind = kind;
  r.bytes = bytes;
  cudaEventRecord(r.a, c->stream);
  c->prof_open.push_back(r);
}

void prof_end(slh_ctx* c) {
  if (!c->prof || c->prof_open.empty()) return;
  cudaEventRecord(c->prof_open.back().b, c->stream);
}

static double host_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

HostPhase::HostPhase(slh_ctx* cc, int k) : c(cc), kind(k), t0(host_ms()) {}
HostPhase::~HostPhase() {
  c->prof_ms[kind] += host_ms() - t0;
  c->prof_n[kind] += 1;
}

static void free_level(Level& L) {
  free_tmaps(L);
  cudaFree(L.tile.d_items);
  cudaFree(L.dtile.d_items);
  cudaFree(L.d_col_items);
  cudaFree(L.d_boxes);
  cudaFree(L.d_bmap);
  cudaFree(L.d_gregions);
  cudaFree(L.d_pieces);
  cudaFree(L.d_covered);
  cudaFree(L.d_ritems);
  cudaFree(L.d_rchunks);
  cudaFree(L.d_epart);
  cudaFree(L.d_tagtmp);
  cudaFree(L.d_tee);
  L = Level();
}

static void drop_graphs(slh_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

template <typename V>
static slh_status upload(V** dptr, const std::vector<V>& h) {
  cudaFree(*dptr);
  *dptr = nullptr;
  if (h.empty()) return SLH_OK;
  cudaError_t e = cudaMalloc((void**)dptr, sizeof(V) * h.size());
  if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "cudaMalloc of %zu bytes: %s", sizeof(V) * h.size(), cudaGetErrorString(e));
  SLH_CUDA(cudaMemcpy(*dptr, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
  return SLH_OK;
}

static int ilog2(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}

static size_t elem_size(const slh_ctx* c) { return c->prec == SLH_F64 ? 8 : 4; }
static bool bf16(const slh_ctx* c) { return c->prec == SLH_F32_BF16; }

// fields whose ghost cells are filled: psi1, psi2 (+ the six u_ij)
static int ghost_fields(const slh_ctx* c) { return c->ncomp == NCOMP_GW ? 8 : 2; }

// mark, for the coarser level lev-1, the blocks of bf/2 cells covered by lev
static slh_status build_covered(slh_ctx* c, int lev) {
  Level& C = c->lev[lev - 1];
  Level& F = c->lev[lev];
  const int r = c->bf / 2;
  const int nb = C.n_dom / r;
  std::vector<uint8_t> m((size_t)nb * nb * nb, 0);
  for (const slh_box& b : F.boxes) {
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = (b.lo[d] / 2) / r;
      hi[d] = ((b.hi[d] + 1) / 2) / r - 1;
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) m[((size_t)z * nb + y) * nb + x] = 1;
  }
  C.ncov = nb;
  return upload(&C.d_covered, m);
}

// Stage work items of a tile variant: box by box, z chunk outer, then y,
// then x tiles (consecutive CTAs share halo planes in L2).  which: 1 the
// plain stages, 2 the diagnostics stage, 3 both.
static slh_status set_tile(slh_ctx* c, Level& L, const TileVariant& v, int which = 3) {
  (void)c;
  std::vector<int4> items;
  for (size_t b = 0; b < L.lay.boxes.size(); ++b) {
    const BoxDev& B = L.lay.boxes[b];
    for (int z0 = 0; z0 < B.n[2]; z0 += v.zlen)
      for (int y0 = 0; y0 < B.n[1]; y0 += v.ty)
        for (int x0 = 0; x0 < B.n[0]; x0 += v.tx) items.push_back(make_int4((int)b, x0, y0, z0));
  }
  for (int k = 0; k < 2; ++k) {
    if (!(which & (1 << k))) continue;
    Tile& t = k == 0 ? L.tile : L.dtile;
    slh_status st = upload(&t.d_items, items);
    if (st != SLH_OK) return st;
    t.v = v;
    t.nitems = (int)items.size();
    t.zlen = v.zlen;
  }
  return SLH_OK;
}

}  // namespace slh

using namespace slh;

extern "C" {

const char* slh_last_error(void) { return g_last_error.c_str(); }

slh_status slh_level_layout(int32_t nghost, int32_t nfields, const slh_box* boxes, int32_t nboxes,
                            int64_t* box_offsets, int64_t* box_geom, int64_t* total_elems, int64_t* nvalid) {
  if (!boxes || nboxes < 0 || nghost < 1 || nghost > 4) return fail(SLH_ERR_INVALID_ARG, "layout: bad arguments");
  if (nfields != NCOMP && nfields != NCOMP_GW && nfields != SLH_SLOTS_BF16)
    return fail(SLH_ERR_INVALID_ARG, "layout: nfields must be 4, 16 or %d (BF16 tensor slots)", SLH_SLOTS_BF16);
  Layout lay;
  std::string why;
  if (!make_layout(nghost, nfields, boxes, nboxes, &lay, &why))
    return fail(SLH_ERR_INVALID_ARG, "layout: %s", why.c_str());
  for (int b = 0; b < nboxes; ++b) {
    if (box_offsets) box_offsets[b] = lay.boxes[b].off;
    if (box_geom) {
      box_geom[4 * b + 0] = lay.boxes[b].pitch;
      box_geom[4 * b + 1] = lay.boxes[b].pny;
      box_geom[4 * b + 2] = lay.boxes[b].pnz;
      box_geom[4 * b + 3] = lay.boxes[b].cs;
    }
  }
  if (total_elems) *total_elems = lay.total;
  if (nvalid) *nvalid = lay.nvalid;
  return SLH_OK;
}

slh_status slh_create(slh_ctx** out, int32_t n0, double dx0, int32_t nghost, int32_t bf, int32_t prec,
                      int32_t max_levels, int32_t nfields, void* stream) {
  if (!out) return fail(SLH_ERR_INVALID_ARG, "create: ctx pointer is null");
  *out = nullptr;
  if (nghost < 1 || nghost > 4) return fail(SLH_ERR_INVALID_ARG, "create: nghost must be in [1,4]");
  if (bf < 2 || (bf & (bf - 1))) return fail(SLH_ERR_INVALID_ARG, "create: blocking factor must be a power of two >= 2");
  if (n0 < bf || n0 % bf) return fail(SLH_ERR_INVALID_ARG, "create: n0 must be a positive multiple of the blocking factor");
  if (prec != SLH_F64 && prec != SLH_F32_KAHAN && prec != SLH_F32_BF16)
    return fail(SLH_ERR_INVALID_ARG, "create: unknown precision %d", prec);
  if (prec == SLH_F32_BF16 && nfields != NCOMP_GW)
    return fail(SLH_ERR_INVALID_ARG, "create: SLH_F32_BF16 stores the 16-field state (nfields 16)");
  if (max_levels < 1 || max_levels > MAX_LEVELS) return fail(SLH_ERR_INVALID_ARG, "create: max_levels must be in [1,8]");
  if (!(dx0 > 0.0)) return fail(SLH_ERR_INVALID_ARG, "create: dx0 must be positive");
  if (nfields != NCOMP && nfields != NCOMP_GW) return fail(SLH_ERR_INVALID_ARG, "create: nfields must be 4 or 16");
  slh_ctx* c = new (std::nothrow) slh_ctx();
  if (!c) return fail(SLH_ERR_NOMEM, "create: out of host memory");
  c->n0 = n0;
  c->dx0 = dx0;
  c->g = nghost;
  c->bf = bf;
  c->prec = prec;
  c->ncomp = nfields;
  c->nslots = prec == SLH_F32_BF16 ? SLH_SLOTS_BF16 : nfields;
  c->max_levels = max_levels;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_time, sizeof(double) * 2 * MAX_LEVELS);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_levsum, sizeof(double) * 4 * MAX_LEVELS);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_count, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_time, 0, sizeof(double) * 2 * MAX_LEVELS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) {
    slh_destroy(c);
    return cuda_fail(e, "create");
  }
  *out = c;
  return SLH_OK;
}

void slh_destroy(slh_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (int l = 0; l < MAX_LEVELS; ++l) free_level(c->lev[l]);
  for (auto& r : c->prof_open) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaFree(c->d_time);
  cudaFree(c->d_err);
  cudaFree(c->d_levsum);
  cudaFree(c->d_count);
  cudaFree(c->d_blockmask);
  delete c;
}

}  // extern "C"

namespace slh {

// Validate a level's boxes (alignment, overlap, level-0 coverage, nesting in
// lev-1) and build its block owner map.
static slh_status validate_boxes(slh_ctx* c, int lev, const slh_box* boxes, int nboxes, void* const* bufs,
                                 std::vector<int>* bmap_out, const char* who) {
  for (int i = 0; i < SLH_NBUF; ++i) {
    // SLH_F32_BF16 levels hold three buffers (SSPRK3); the others need D,
    // and the Kahan compensation with SLH_F32_KAHAN
    const bool need = bf16(c) ? (i == SLH_BUF_Y || i == SLH_BUF_YA || i == SLH_BUF_YB)
                              : ((i != SLH_BUF_C) || c->prec == SLH_F32_KAHAN);
    if (need && !bufs[i]) return fail(SLH_ERR_INVALID_ARG, "%s: buffer %d is null", who, i);
  }
  const int ndom = c->n0 << lev;
  const int bf = c->bf;
  const int nbd = ndom / bf;
  std::vector<int>& bmap = *bmap_out;
  bmap.assign((size_t)nbd * nbd * nbd, -1);
  for (int b = 0; b < nboxes; ++b) {
    const slh_box& B = boxes[b];
    for (int d = 0; d < 3; ++d) {
      if (B.lo[d] < 0 || B.hi[d] >= ndom || B.hi[d] < B.lo[d])
        return fail(SLH_ERR_OUT_OF_RANGE, "%s: box %d outside the level domain [0,%d)", who, b, ndom);
      if (B.lo[d] % bf || (B.hi[d] + 1) % bf)
        return fail(SLH_ERR_INVALID_ARG, "%s: box %d not aligned to the blocking factor %d", who, b, bf);
    }
    for (int z = B.lo[2] / bf; z <= B.hi[2] / bf; ++z)
      for (int y = B.lo[1] / bf; y <= B.hi[1] / bf; ++y)
        for (int x = B.lo[0] / bf; x <= B.hi[0] / bf; ++x) {
          int& o = bmap[((size_t)z * nbd + y) * nbd + x];
          if (o >= 0) return fail(SLH_ERR_INVALID_ARG, "%s: boxes %d and %d overlap", who, o, b);
          o = b;
        }
  }
  if (lev == 0) {
    for (int v : bmap)
      if (v < 0) return fail(SLH_ERR_INVALID_ARG, "%s: level 0 must cover the periodic domain", who);
    return SLH_OK;
  }
  // nesting: the coarse projection grown by one block of bf/2 coarse cells
  // must lie inside level lev-1 (periodic).  A block of bf/2 coarse cells
  // lies inside a coarse box iff its enclosing block of bf cells does
  // (coarse boxes are aligned to bf).
  Level& C = c->lev[lev - 1];
  const int r = bf / 2;
  const int nbc = C.n_dom / r;
  for (int b = 0; b < nboxes; ++b) {
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = (boxes[b].lo[d] / 2) / r - 1;
      hi[d] = ((boxes[b].hi[d] + 1) / 2) / r;
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int wx = ((x % nbc) + nbc) % nbc, wy = ((y % nbc) + nbc) % nbc, wz = ((z % nbc) + nbc) % nbc;
          const int own = C.h_bmap[((size_t)(wz / 2) * C.nb_dom + wy / 2) * C.nb_dom + wx / 2];
          if (own < 0)
            return fail(SLH_ERR_OUT_OF_RANGE,
                        "%s: box %d of level %d is not nested in level %d with a gap of %d coarse cells", who, b, lev,
                        lev - 1, r);
        }
  }
  return SLH_OK;
}

// Split [a, b] (inclusive) at multiples of `step` relative to `base` and at
// the domain boundaries 0 and n (so that one periodic image applies).
static void split_axis(int a, int b, int base, int step, int n, std::vector<std::pair<int, int>>* out) {
  out->clear();
  int s0 = a;
  while (s0 <= b) {
    int e = b;
    const int nextb = base + ((s0 - base) / step + 1) * step;   // next chunk boundary above s0 (s0 >= base)
    if (s0 >= base && nextb - 1 < e) e = nextb - 1;
    if (s0 < base && base - 1 < e) e = base - 1;
    if (s0 < 0 && -1 < e) e = -1;
    if (s0 < n && n - 1 < e) e = n - 1;
    out->push_back({s0, e});
    s0 = e + 1;
  }
}

// Pieces of the coarse patch of a prolongation region (fine cells flo..fhi
// inclusive, unwrapped): the radius-PROLONG_RAD_MAX footprint [plo, plo+pn)
// split at the coarse domain boundaries into periodic images, each image
// intersected with the coarse boxes it meets (found from the coarse block
// map).  Returns whether the pieces tile the whole footprint.
static bool plan_patch(const Level& C, int bf, const int flo[3], const int fhi[3], std::vector<PatchPiece>* pieces) {
  int plo[3], pn[3];
  for (int d = 0; d < 3; ++d) {
    plo[d] = (flo[d] >> 1) - PROLONG_RAD_MAX;
    pn[d] = (fhi[d] >> 1) + PROLONG_RAD_MAX - plo[d] + 1;
  }
  const int nc = C.n_dom, nbd = C.nb_dom;
  long long got = 0;
  // per axis: up to three segments [a, b] of the footprint, each under one image
  std::vector<std::pair<int, int>> seg[3];
  for (int d = 0; d < 3; ++d) {
    int a = plo[d];
    const int e = plo[d] + pn[d] - 1;
    while (a <= e) {
      const int img = a >= 0 ? a / nc : -((-a + nc - 1) / nc);   // floor(a / nc)
      const int b = std::min(e, (img + 1) * nc - 1);
      seg[d].push_back({a, b});
      a = b + 1;
    }
  }
  std::vector<int> owners;
  for (auto& sz : seg[2])
    for (auto& sy : seg[1])
      for (auto& sx : seg[0]) {
        const int lo[3] = {sx.first, sy.first, sz.first}, hi[3] = {sx.second, sy.second, sz.second};
        int wlo[3], shift[3];
        for (int d = 0; d < 3; ++d) {
          const int img = lo[d] >= 0 ? lo[d] / nc : -((-lo[d] + nc - 1) / nc);
          shift[d] = img * nc;
          wlo[d] = lo[d] - shift[d];
        }
        owners.clear();
        for (int bz = wlo[2] / bf; bz <= (hi[2] - shift[2]) / bf; ++bz)
          for (int by = wlo[1] / bf; by <= (hi[1] - shift[1]) / bf; ++by)
            for (int bx = wlo[0] / bf; bx <= (hi[0] - shift[0]) / bf; ++bx) {
              const int o = C.h_bmap[((size_t)bz * nbd + by) * nbd + bx];
              if (o >= 0 && std::find(owners.begin(), owners.end(), o) == owners.end()) owners.push_back(o);
            }
        std::sort(owners.begin(), owners.end());
        for (int o : owners) {
          const slh_box& cb = C.boxes[o];
          PatchPiece P;
          P.cbox = o;
          bool empty = false;
          for (int d = 0; d < 3; ++d) {
            const int a = std::max(wlo[d], cb.lo[d]), b = std::min(hi[d] - shift[d], cb.hi[d]);
            if (a > b) empty = true;
            P.src[d] = a - cb.lo[d];
            P.dst[d] = a + shift[d] - plo[d];
            P.ext[d] = b - a + 1;
          }
          if (empty) continue;
          got += (long long)P.ext[0] * P.ext[1] * P.ext[2];
          pieces->push_back(P);
        }
      }
  return got == (long long)pn[0] * pn[1] * pn[2];
}

// Ghost regions of every box: each of the six ghost slabs is cut at the box
// bounds, every GHOST_CHUNK cells and at the domain boundaries; each piece is
// classified from the host block map (blocks of bf >= g cells, so a piece
// meets few blocks).  A piece that meets several owners (or owners and
// uncovered blocks) is cut further at the block boundaries, where ownership
// is constant, and neighbouring cuts of one kind and source merged again, so
// that every region is a pure copy or a pure prolongation.  For a level > 0,
// regions that prolong get the pieces of their coarse patch.  Copy regions
// come first in the list (a kernel of their own fills them).
static slh_status plan_ghost_regions(slh_ctx* c, int lev, Level& L, std::vector<GhostRegion>* out,
                                     std::vector<PatchPiece>* pieces, long long* total, int* ncopy) {
  const int g = c->g, bf = c->bf, n = L.n_dom, nbd = L.nb_dom;
  out->clear();
  pieces->clear();
  *total = 0;
  std::vector<GhostRegion> copies, others;
  // classification of cells glo..ghi (unwrapped, inclusive, one periodic image)
  auto classify = [&](const BoxDev& B, int b, const int glo[3], const int ghi[3], GhostRegion* R) {
    int wl[3], k[3];
    R->box = b;
    for (int d = 0; d < 3; ++d) {
      R->lo[d] = glo[d] - B.lo[d];
      R->ext[d] = ghi[d] - glo[d] + 1;
      k[d] = glo[d] < 0 ? -1 : (glo[d] >= n ? 1 : 0);
      wl[d] = glo[d] - k[d] * n;
    }
    int own = -2;
    bool same = true, any_cov = false, any_unc = false;
    for (int bz = wl[2] / bf; bz <= (wl[2] + R->ext[2] - 1) / bf; ++bz)
      for (int by = wl[1] / bf; by <= (wl[1] + R->ext[1] - 1) / bf; ++by)
        for (int bx = wl[0] / bf; bx <= (wl[0] + R->ext[0] - 1) / bf; ++bx) {
          const int o = L.h_bmap[((size_t)bz * nbd + by) * nbd + bx];
          if (o >= 0) any_cov = true; else any_unc = true;
          if (own == -2) own = o;
          else if (o != own) same = false;
        }
    R->src = -1;
    R->d[0] = R->d[1] = R->d[2] = 0;
    if (!any_cov) {
      R->kind = GHOST_PROLONG;
    } else if (!any_unc && same) {
      R->kind = GHOST_COPY;
      R->src = own;
      const BoxDev& S = L.lay.boxes[own];
      for (int d = 0; d < 3; ++d) R->d[d] = B.lo[d] - k[d] * n - S.lo[d];
    } else {
      R->kind = GHOST_MIXED;
    }
  };
  // each box is planned on its own (host threads); piece indexes are local
  // to the box until the plans are joined in box order
  struct BoxPlan {
    std::vector<GhostRegion> copies, others;
    std::vector<PatchPiece> pieces;
    long long total = 0;
  };
  std::vector<BoxPlan> plans(L.lay.boxes.size());
  auto emit = [&](BoxPlan& bp, const BoxDev& B, int b, const int glo[3], const int ghi[3]) {
    GhostRegion R;
    classify(B, b, glo, ghi, &R);
    R.p0 = (int)bp.pieces.size();
    R.np = 0;
    R.covered = 0;
    if (lev > 0 && R.kind != GHOST_COPY) {
      int flo[3], fhi[3];
      for (int d = 0; d < 3; ++d) {
        flo[d] = glo[d];
        fhi[d] = ghi[d];
      }
      R.covered = plan_patch(c->lev[lev - 1], bf, flo, fhi, &bp.pieces) ? 1 : 0;
      R.np = (int)bp.pieces.size() - R.p0;
    }
    (R.kind == GHOST_COPY ? bp.copies : bp.others).push_back(R);
    bp.total += (long long)R.ext[0] * R.ext[1] * R.ext[2];
  };
  auto same_key = [](const GhostRegion& a, const GhostRegion& b) {
    return a.kind == b.kind && a.kind != GHOST_MIXED && a.src == b.src && a.d[0] == b.d[0] && a.d[1] == b.d[1] &&
           a.d[2] == b.d[2];
  };
  parallel_for((int)L.lay.boxes.size(), 4096, [&](int b) {
    std::vector<std::pair<int, int>> sx, sy, sz, cut[3];
    std::vector<GhostRegion> sub;
    BoxPlan& bp = plans[b];
    const BoxDev& B = L.lay.boxes[b];
    const int nn[3] = {B.n[0], B.n[1], B.n[2]};
    // six slabs: (lo, hi) valid-relative, inclusive
    int slabs[6][2][3] = {
        {{-g, -g, -g}, {nn[0] + g - 1, nn[1] + g - 1, -1}},
        {{-g, -g, nn[2]}, {nn[0] + g - 1, nn[1] + g - 1, nn[2] + g - 1}},
        {{-g, -g, 0}, {nn[0] + g - 1, -1, nn[2] - 1}},
        {{-g, nn[1], 0}, {nn[0] + g - 1, nn[1] + g - 1, nn[2] - 1}},
        {{-g, 0, 0}, {-1, nn[1] - 1, nn[2] - 1}},
        {{nn[0], 0, 0}, {nn[0] + g - 1, nn[1] - 1, nn[2] - 1}},
    };
    for (auto& sl : slabs) {
      // split in global coordinates so domain boundaries are seen
      split_axis(B.lo[0] + sl[0][0], B.lo[0] + sl[1][0], B.lo[0], GHOST_CHUNK, n, &sx);
      split_axis(B.lo[1] + sl[0][1], B.lo[1] + sl[1][1], B.lo[1], GHOST_CHUNK, n, &sy);
      split_axis(B.lo[2] + sl[0][2], B.lo[2] + sl[1][2], B.lo[2], GHOST_CHUNK, n, &sz);
      for (auto& zz : sz)
        for (auto& yy : sy)
          for (auto& xx : sx) {
            const int glo[3] = {xx.first, yy.first, zz.first}, ghi[3] = {xx.second, yy.second, zz.second};
            GhostRegion R;
            classify(B, (int)b, glo, ghi, &R);
            if (R.kind != GHOST_MIXED) {
              emit(bp, B, b, glo, ghi);
              continue;
            }
            // cut at the block boundaries (of the wrapped coordinates)
            for (int d = 0; d < 3; ++d) {
              cut[d].clear();
              const int k = glo[d] < 0 ? -1 : (glo[d] >= n ? 1 : 0);
              int a = glo[d];
              while (a <= ghi[d]) {
                const int w = a - k * n;
                const int e = std::min(ghi[d], a + (bf - w % bf) - 1);
                cut[d].push_back({a, e});
                a = e + 1;
              }
            }
            const int nx = (int)cut[0].size(), ny = (int)cut[1].size(), nz = (int)cut[2].size();
            sub.assign((size_t)nx * ny * nz, GhostRegion());
            for (int iz = 0; iz < nz; ++iz)
              for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                  const int l[3] = {cut[0][ix].first, cut[1][iy].first, cut[2][iz].first};
                  const int h[3] = {cut[0][ix].second, cut[1][iy].second, cut[2][iz].second};
                  classify(B, (int)b, l, h, &sub[((size_t)iz * ny + iy) * nx + ix]);
                }
            // merge runs along x of one key, then rows along y with the same
            // runs; z (the slab's thickness, or a 32-cell chunk) stays cut
            for (int iz = 0; iz < nz; ++iz) {
              int iy = 0;
              while (iy < ny) {
                // runs of row iy
                std::vector<std::pair<int, int>> runs;
                for (int ix = 0; ix < nx;) {
                  int jx = ix;
                  while (jx + 1 < nx && same_key(sub[((size_t)iz * ny + iy) * nx + ix], sub[((size_t)iz * ny + iy) * nx + jx + 1])) ++jx;
                  runs.push_back({ix, jx});
                  ix = jx + 1;
                }
                // extend every run along y while the next row holds its key
                // over the run's whole width (each rectangle stays uniform)
                int jy = iy;
                while (jy + 1 < ny) {
                  bool ok = true;
                  for (auto& r : runs)
                    for (int q = r.first; q <= r.second && ok; ++q)
                      ok = same_key(sub[((size_t)iz * ny + iy) * nx + r.first], sub[((size_t)iz * ny + jy + 1) * nx + q]);
                  if (!ok) break;
                  ++jy;
                }
                for (auto& r : runs) {
                  const int l[3] = {cut[0][r.first].first, cut[1][iy].first, cut[2][iz].first};
                  const int h[3] = {cut[0][r.second].second, cut[1][jy].second, cut[2][iz].second};
                  emit(bp, B, b, l, h);
                }
                iy = jy + 1;
              }
            }
          }
    }
  });
  for (BoxPlan& bp : plans) {
    const int off = (int)pieces->size();
    for (GhostRegion& R : bp.copies) {
      R.p0 += off;
      copies.push_back(R);
    }
    for (GhostRegion& R : bp.others) {
      R.p0 += off;
      others.push_back(R);
    }
    pieces->insert(pieces->end(), bp.pieces.begin(), bp.pieces.end());
    *total += bp.total;
  }
  *ncopy = (int)copies.size();
  out->reserve(copies.size() + others.size());
  out->insert(out->end(), copies.begin(), copies.end());
  out->insert(out->end(), others.begin(), others.end());
  return SLH_OK;
}

// Fill the metadata of level lev (boxes already validated) into L.
static slh_status build_level(slh_ctx* c, int lev, Level& L, const slh_box* boxes, int nboxes, void* const* bufs,
                              uint8_t* tags_dev, const std::vector<int>& bmap) {
  L.n_dom = c->n0 << lev;
  L.nb_dom = L.n_dom / c->bf;
  L.dx = c->dx0 / (double)(1 << lev);
  L.boxes.assign(boxes, boxes + nboxes);
  std::string why;
  if (!make_layout(c->g, c->nslots, boxes, nboxes, &L.lay, &why))
    return fail(SLH_ERR_INVALID_ARG, "level %d: %s", lev, why.c_str());
  for (int i = 0; i < SLH_NBUF; ++i) L.buf[i] = bufs[i];
  if (c->prec != SLH_F32_KAHAN) L.buf[SLH_BUF_C] = nullptr;
  if (bf16(c)) L.buf[SLH_BUF_D] = nullptr;
  L.tags_dev = tags_dev;
  L.role_y = SLH_BUF_Y;
  L.role_prev = SLH_BUF_YB;
  L.role_s = SLH_BUF_YA;
  slh_status st;
  if ((st = upload(&L.d_boxes, L.lay.boxes)) != SLH_OK) return st;
  if ((st = upload(&L.d_bmap, bmap)) != SLH_OK) return st;
  L.h_bmap = bmap;

  // ghost shell regions, classified from the block map
  {
    std::vector<GhostRegion> regs;
    std::vector<PatchPiece> pcs;
    long long tot = 0;
    int ncopy = 0;
    if ((st = plan_ghost_regions(c, lev, L, &regs, &pcs, &tot, &ncopy)) != SLH_OK) return st;
    L.ngregions = (int)regs.size();
    L.ncopyregions = ncopy;
    L.nghost_cells = tot;
    L.npieces = (int)pcs.size();
    if ((st = upload(&L.d_gregions, regs)) != SLH_OK) return st;
    if ((st = upload(&L.d_pieces, pcs)) != SLH_OK) return st;
  }

  {
    int nv = 0;
    const TileVariant* vs = tile_variants(c->prec, &nv);
    if ((st = set_tile(c, L, vs[0])) != SLH_OK) return st;
  }
  {   // column items of the GW and dissipation kernels
    std::vector<int4> items;
    for (size_t b = 0; b < L.lay.boxes.size(); ++b) {
      const BoxDev& B = L.lay.boxes[b];
      for (int z0 = 0; z0 < B.n[2]; z0 += COL_ZLEN)
        for (int y0 = 0; y0 < B.n[1]; y0 += COL_TY)
          for (int x0 = 0; x0 < B.n[0]; x0 += COL_TX) items.push_back(make_int4((int)b, x0, y0, z0));
    }
    if ((st = upload(&L.d_col_items, items)) != SLH_OK) return st;
    L.ncol_items = (int)items.size();
  }

  // restriction items onto lev-1
  if (lev > 0) {
    std::vector<RestrictItem> ri;
    std::vector<int2> chunks;
    long long rt = 0;
    for (int b = 0; b < nboxes; ++b) {
      RestrictItem it;
      it.fbox = b;
      for (int d = 0; d < 3; ++d) it.n[d] = L.lay.boxes[b].n[d] / 2;
      const int ncell = it.n[0] * it.n[1] * it.n[2];
      for (int c0 = 0; c0 < ncell; c0 += RESTRICT_CHUNK) chunks.push_back(make_int2((int)ri.size(), c0));
      ri.push_back(it);
      rt += ncell;
    }
    L.nritems = (int)ri.size();
    L.nrchunks = (int)chunks.size();
    L.nrcells = rt;
    if ((st = upload(&L.d_ritems, ri)) != SLH_OK) return st;
    if ((st = upload(&L.d_rchunks, chunks)) != SLH_OK) return st;
  }

  // truncation-error-estimate tags
  if (c->tag_criteria & SLH_TAG_TEE) {
    cudaError_t e = cudaMalloc(&L.d_tee, (size_t)std::max<long long>(1, L.lay.nvalid));
    if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "level %d: TEE tags: %s", lev, cudaGetErrorString(e));
    SLH_CUDA(cudaMemsetAsync(L.d_tee, 0, (size_t)std::max<long long>(1, L.lay.nvalid), c->stream));
  }

  // energy partials
  L.epart_cap = c->num_sms * 32;
  {
    cudaError_t e = cudaMalloc(&L.d_epart, sizeof(double) * 4 * L.epart_cap);
    if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "level %d: energy partials: %s", lev, cudaGetErrorString(e));
  }
  L.defined = true;
  return SLH_OK;
}

}  // namespace slh

extern "C" {

slh_status slh_init_level(slh_ctx* c, int32_t lev, const slh_box* boxes, int32_t nboxes, void* const* bufs,
                          uint8_t* tags_dev) {
  if (!c || !boxes || !bufs || nboxes < 1) return fail(SLH_ERR_INVALID_ARG, "init_level: null argument or no boxes");
  if (lev < 0 || lev >= c->max_levels) return fail(SLH_ERR_OUT_OF_RANGE, "init_level: level %d outside [0,%d)", lev, c->max_levels);
  if (lev > c->nlevels) return fail(SLH_ERR_STATE, "init_level: level %d defined before level %d", lev, c->nlevels);
  std::vector<int> bmap;
  slh_status st = validate_boxes(c, lev, boxes, nboxes, bufs, &bmap, "init_level");
  if (st != SLH_OK) return st;
  // drop this level and every finer one
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (int l = lev; l < MAX_LEVELS; ++l) free_level(c->lev[l]);
  if (lev > 0) {
    cudaFree(c->lev[lev - 1].d_covered);
    c->lev[lev - 1].d_covered = nullptr;
  }
  c->nlevels = lev;
  c->stale_from = MAX_LEVELS;
  Level& L = c->lev[lev];
  if ((st = build_level(c, lev, L, boxes, nboxes, bufs, tags_dev, bmap)) != SLH_OK) return st;
  c->nlevels = lev + 1;
  if (lev > 0 && (st = build_covered(c, lev)) != SLH_OK) return st;
  const size_t bytes = (size_t)L.lay.total * elem_size(c);
  for (int i = 0; i < SLH_NBUF; ++i)
    if (L.buf[i]) SLH_CUDA(cudaMemsetAsync(L.buf[i], 0, bytes, c->stream));
  return SLH_OK;
}

slh_status slh_regrid_level(slh_ctx* c, int32_t lev, const slh_box* boxes, int32_t nboxes, void* const* bufs,
                            uint8_t* tags_dev, int32_t interp_type) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "regrid_level: null ctx");
  if (lev < 1 || lev >= c->max_levels) return fail(SLH_ERR_OUT_OF_RANGE, "regrid_level: level %d outside [1,%d)", lev, c->max_levels);
  if (lev > c->nlevels) return fail(SLH_ERR_STATE, "regrid_level: level %d below it is not defined", lev - 1);
  NvtxRange range("slh regrid level %d (%d boxes)", lev, nboxes);
  if (lev - 1 >= c->stale_from) return fail(SLH_ERR_STATE, "regrid_level: regrid level %d first", c->stale_from);
  if (interp_type != 0 && interp_type != 2 && interp_type != 4)
    return fail(SLH_ERR_INVALID_ARG, "regrid_level: interp_type must be 0, 2 or 4");
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  if (nboxes <= 0) {
    // the level disappears, and every finer one with it
    for (int l = lev; l < MAX_LEVELS; ++l) free_level(c->lev[l]);
    cudaFree(c->lev[lev - 1].d_covered);
    c->lev[lev - 1].d_covered = nullptr;
    c->nlevels = lev;
    c->stale_from = MAX_LEVELS;
    return SLH_OK;
  }
  if (!boxes || !bufs) return fail(SLH_ERR_INVALID_ARG, "regrid_level: null argument");
  std::vector<int> bmap;
  slh_status st = validate_boxes(c, lev, boxes, nboxes, bufs, &bmap, "regrid_level");
  if (st != SLH_OK) return st;
  Level fresh;
  if ((st = build_level(c, lev, fresh, boxes, nboxes, bufs, tags_dev, bmap)) != SLH_OK) {
    free_level(fresh);
    return st;
  }
  const size_t bytes = (size_t)fresh.lay.total * elem_size(c);
  for (int i = 0; i < SLH_NBUF; ++i)
    if (fresh.buf[i]) SLH_CUDA(cudaMemsetAsync(fresh.buf[i], 0, bytes, c->stream));
  Level* old = lev < c->nlevels ? &c->lev[lev] : nullptr;
  if (old) {
    // a level that is regridded keeps the tiles its autotuners chose
    if ((st = set_tile(c, fresh, old->tile.v, 1)) != SLH_OK || (st = set_tile(c, fresh, old->dtile.v, 2)) != SLH_OK) {
      free_level(fresh);
      return st;
    }
  }
  c->regrid_itype = interp_type;
  if ((st = launch_regrid_fill(c, lev, fresh, old)) != SLH_OK) {
    free_level(fresh);
    return st;
  }
  SLH_CUDA(cudaMemcpyAsync(fresh.buf[fresh.role_prev], fresh.buf[fresh.role_y], bytes, cudaMemcpyDeviceToDevice,
                           c->stream));
  // the new level starts at its coarser level's (synchronised) time
  SLH_CUDA(cudaMemcpyAsync(c->d_time + 2 * lev, c->d_time + 2 * (lev - 1), 2 * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
  st = slh_sync(c);
  if (old) free_level(*old);
  c->lev[lev] = fresh;
  fresh = Level();   // ownership moved (avoid freeing twice)
  if (st != SLH_OK) return st;
  if (lev + 1 > c->nlevels) c->nlevels = lev + 1;
  if ((st = build_covered(c, lev)) != SLH_OK) return st;
  if (lev + 1 < c->nlevels) {
    c->stale_from = lev + 1;
    if ((st = build_covered(c, lev + 1)) != SLH_OK) return st;
  } else {
    c->stale_from = MAX_LEVELS;
  }
  return SLH_OK;
}

static slh_status copy_state(slh_ctx* c, int lev, void* host_or_dev, bool to_device) {
  Level& L = c->lev[lev];
  const size_t s = elem_size(c);
  char* dense = static_cast<char*>(host_or_dev);
  char* buf = static_cast<char*>(L.buf[L.role_y]);
  for (size_t b = 0; b < L.lay.boxes.size(); ++b) {
    const BoxDev& B = L.lay.boxes[b];
    const long long vol = (long long)B.n[0] * B.n[1] * B.n[2];
    for (int comp = 0; comp < c->nslots; ++comp) {
      cudaMemcpy3DParms p;
      memset(&p, 0, sizeof(p));
      cudaPitchedPtr dptr =
          make_cudaPitchedPtr(dense + (size_t)(c->nslots * B.voff + comp * vol) * s, B.n[0] * s, B.n[0], B.n[1]);
      cudaPitchedPtr bptr = make_cudaPitchedPtr(buf + (size_t)(B.off + comp * B.cs) * s, (size_t)B.pitch * s, B.pitch, B.pny);
      if (to_device) {
        p.srcPtr = dptr;
        p.dstPtr = bptr;
        p.dstPos = make_cudaPos(XPAD * s, c->g, c->g);
      } else {
        p.srcPtr = bptr;
        p.srcPos = make_cudaPos(XPAD * s, c->g, c->g);
        p.dstPtr = dptr;
      }
      p.extent = make_cudaExtent(B.n[0] * s, B.n[1], B.n[2]);
      p.kind = cudaMemcpyDefault;
      SLH_CUDA(cudaMemcpy3DAsync(&p, c->stream));
    }
  }
  return SLH_OK;
}

slh_status slh_set_state(slh_ctx* c, int32_t lev, const void* src, int32_t src_is_host) {
  (void)src_is_host;
  if (!c || !src) return fail(SLH_ERR_INVALID_ARG, "set_state: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "set_state: level %d not defined", lev);
  Level& L = c->lev[lev];
  slh_status st = copy_state(c, lev, const_cast<void*>(src), true);
  if (st != SLH_OK) return st;
  const size_t bytes = (size_t)L.lay.total * elem_size(c);
  SLH_CUDA(cudaMemcpyAsync(L.buf[L.role_prev], L.buf[L.role_y], bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (L.buf[SLH_BUF_C]) SLH_CUDA(cudaMemsetAsync(L.buf[SLH_BUF_C], 0, bytes, c->stream));
  return SLH_OK;
}

slh_status slh_get_state(slh_ctx* c, int32_t lev, void* dst, int32_t dst_is_host) {
  if (!c || !dst) return fail(SLH_ERR_INVALID_ARG, "get_state: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "get_state: level %d not defined", lev);
  slh_status st = copy_state(c, lev, dst, false);
  if (st != SLH_OK) return st;
  if (dst_is_host) return slh_sync(c);
  return SLH_OK;
}

}  // extern "C"

__global__ void set_eta_kernel(double* t, double eta) {
  const int i = threadIdx.x;
  if (i < 2 * MAX_LEVELS) t[i] = eta;
}

extern "C" {

slh_status slh_set_eta(slh_ctx* c, double eta) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "set_eta: null ctx");
  set_eta_kernel<<<1, 32, 0, c->stream>>>(c->d_time, eta);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status slh_level_roles(slh_ctx* c, int32_t lev, int32_t roles[3]) {
  if (!c || !roles) return fail(SLH_ERR_INVALID_ARG, "level_roles: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "level_roles: level %d not defined", lev);
  roles[0] = c->lev[lev].role_y;
  roles[1] = c->lev[lev].role_prev;
  roles[2] = c->lev[lev].role_s;
  return SLH_OK;
}

slh_status slh_get_eta(slh_ctx* c, int32_t lev, double* eta) {
  if (!c || !eta) return fail(SLH_ERR_INVALID_ARG, "get_eta: null argument");
  if (lev < 0 || lev >= MAX_LEVELS) return fail(SLH_ERR_OUT_OF_RANGE, "get_eta: level %d", lev);
  SLH_CUDA(cudaMemcpyAsync(eta, c->d_time + 2 * lev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  return SLH_OK;
}

static slh_status check_params(const slh_eom_params* p) {
  if (!p) return fail(SLH_ERR_INVALID_ARG, "null eom params");
  if (p->lap_order != 2 && p->lap_order != 4 && p->lap_order != 6)
    return fail(SLH_ERR_INVALID_ARG, "lap_order must be 2, 4 or 6 (got %d)", p->lap_order);
  if (p->eta_power != 0 && p->eta_power != 2) return fail(SLH_ERR_INVALID_ARG, "eta_power must be 0 or 2");
  if (p->interp_type != 0 && p->interp_type != 2 && p->interp_type != 4)
    return fail(SLH_ERR_INVALID_ARG, "interp_type must be 0, 2 or 4");
  if (p->integrator != 4 && p->integrator != 10 && p->integrator != 3 && p->integrator != 21 && p->integrator != 22)
    return fail(SLH_ERR_INVALID_ARG,
                "integrator must be 4 (classic RK4), 10 / 3 (SSPRK3), 21 (RKN4) or 22 (RKN5), got %d", p->integrator);
  if (p->ko_order != 0 && p->ko_order != 1 && p->ko_order != 3 && p->ko_order != 5)
    return fail(SLH_ERR_INVALID_ARG, "ko_order must be 0 (off), 1, 3 or 5 (got %d)", p->ko_order);
  if (!(p->ko_eps >= 0.0) || p->ko_eps > 1e30) return fail(SLH_ERR_INVALID_ARG, "ko_eps must be finite and >= 0");
  if ((p->integrator == 21 || p->integrator == 22) && p->ko_order > 0 && p->ko_eps > 0.0)
    return fail(SLH_ERR_INVALID_ARG, "RKN%d takes no Kreiss-Oliger term (it needs psi' = Pi)", p->integrator - 17);
  if (p->integrator == 22 && p->friction)
    return fail(SLH_ERR_INVALID_ARG, "RKN5 needs an acceleration independent of Pi: friction must be off");
  return SLH_OK;
}

static slh_status rk_step_impl(slh_ctx* c, int lev, int sub, double dt0, const slh_eom_params& p, uint32_t flags) {
  NvtxRange range("slh level %d step (sub %d)", lev, sub);
  Level& L = c->lev[lev];
  if (p.integrator == 22 && c->ncomp == NCOMP_GW)
    return fail(SLH_ERR_INVALID_ARG, "RKN5 is built for the scalar fields only (not the tensor fields)");
  if (bf16(c) && p.integrator != 10 && p.integrator != 3)
    return fail(SLH_ERR_INVALID_ARG, "SLH_F32_BF16 levels hold three buffers: integrator SSPRK3 (10 or 3) only");
  if (c->g < p.lap_order / 2) return fail(SLH_ERR_INVALID_ARG, "nghost %d < Laplacian half width %d", c->g, p.lap_order / 2);
  if (p.ko_order > 0 && c->g < (p.ko_order + 1) / 2)
    return fail(SLH_ERR_INVALID_ARG, "nghost %d < dissipation half width %d", c->g, (p.ko_order + 1) / 2);
  const bool ko = p.ko_order > 0 && p.ko_eps > 0.0;
  const double dt = std::ldexp(dt0, -lev);
  const double cRK[4] = {0.0, 0.5, 0.5, 1.0};
  const double aRK[4] = {0.5, 0.5, 1.0, 0.0};
  const double bRK[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const size_t s = elem_size(c);
  const double V = (double)L.lay.nvalid;
  slh_status st;
  prof_begin(c, SLH_PROF_TIME, 0.0);
  st = launch_time_begin(c, lev, sub, dt);
  prof_end(c);
  if (st != SLH_OK) return st;
  const int ybuf = L.role_y, nbuf = L.role_prev, sbuf = L.role_s;
  const bool rkn5 = p.integrator == 22;
  const bool rkn = p.integrator == 21 || rkn5;
  const bool ssp = p.integrator != 4 && !rkn;
  // classic RK4: Y -> S -> prev -> S -> prev with the increment in D (state
  // and previous state swap);
  // SSPRK3: Y -> S -> prev -> S, three buffers (the new state in S, the old
  // one the previous state, prev the next scratch);
  // RKN4: Y -> prev -> prev (velocities only, in place: stages 2 and 3 share
  // their positions) -> S -> prev, the position and velocity sums in D
  int in_role[4] = {ybuf, sbuf, nbuf, sbuf};
  int out_role[4] = {sbuf, nbuf, sbuf, nbuf};
  double vals[4] = {ssp ? 8.0 : 12.0, ssp ? 12.0 : 20.0, ssp ? 12.0 : 20.0, c->prec == SLH_F32_KAHAN ? 24.0 : 16.0};
  // RKN5: Y -> YA (stage-2 positions, k1) -> prev (stage-3 positions, A4;
  // D = position and velocity sums) -> YA (stage-4 positions; D = position
  // increment, velocity sum) -> prev
  if (rkn5) {
    const int ir[4] = {ybuf, sbuf, nbuf, sbuf}, orr[4] = {sbuf, nbuf, sbuf, nbuf};
    const double vr[4] = {8.0, 16.0, 18.0, c->prec == SLH_F32_KAHAN ? 24.0 : 16.0};
    for (int k = 0; k < 4; ++k) {
      in_role[k] = ir[k];
      out_role[k] = orr[k];
      vals[k] = vr[k];
    }
  } else if (rkn) {
    const int ir[4] = {ybuf, nbuf, nbuf, sbuf}, orr[4] = {nbuf, nbuf, sbuf, nbuf};
    const double vr[4] = {12.0, 16.0, 20.0, c->prec == SLH_F32_KAHAN ? 24.0 : 16.0};
    for (int k = 0; k < 4; ++k) {
      in_role[k] = ir[k];
      out_role[k] = orr[k];
      vals[k] = vr[k];
    }
  }
  // RKN4 stage coefficients: (Pi_n in the positions, a in the positions,
  // a in the velocities, a into the position sum, a into the velocity sum)
  const double h = dt;
  const double rknc[4][5] = {{0.5 * h, h * h / 8.0, 0.5 * h, h * h / 6.0, h / 6.0},
                             {0.0, 0.0, 0.5 * h, h * h / 6.0, h / 3.0},
                             {h, h * h / 2.0, h, h * h / 6.0, h / 3.0},
                             {h, 0.0, 0.0, 0.0, h / 6.0}};
  // RKN5 (Nystrom's fifth-order tableau: c, abar, bbar, b):
  // per stage the coefficients the stage kernel's combine takes
  const double c5[4] = {0.0, 1.0 / 5.0, 2.0 / 3.0, 1.0};
  const double h2 = h * h;
  const double rq5[4][9] = {
      {h / 5.0, h2 / 50.0},
      {2.0 * h / 3.0, -h2 / 27.0, 7.0 * h2 / 27.0, 3.0 * h2 / 10.0, -2.0 * h2 / 35.0, 14.0 * h2 / 336.0,
       100.0 * h2 / 336.0, 14.0 * h / 336.0, 125.0 * h / 336.0},
      {h, 9.0 * h2 / 35.0, 54.0 * h2 / 336.0, 162.0 * h / 336.0},
      {35.0 * h / 336.0}};
  const double cSSP[3] = {0.0, 1.0, 0.5}, aSSP[3] = {0.0, 0.75, 1.0 / 3.0}, bSSP[3] = {1.0, 0.25, 2.0 / 3.0};
  const int nstage = ssp ? 3 : 4;
  for (int k = 0; k < nstage; ++k) {
    const double cs = ssp ? cSSP[k] : (rkn5 ? c5[k] : cRK[k]);
    const double alpha = lev > 0 ? (sub + cs) / 2.0 : 1.0;
    prof_begin(c, SLH_PROF_GHOST, (double)L.nghost_cells * ghost_fields(c) * 2 * s);
    if (c->ghost_reuse && lev > 0) {
      // within one step of the coarser level its old and new states are
      // fixed, so a fill at a time fraction an earlier fill of this step
      // used (RK4: stages 2 and 3; the last stage of the first substep and
      // the first of the second) repeats its prolonged values bit for bit:
      // copy them from the buffer that holds them
      if (sub == 0 && k == 0)
        for (int b = 0; b < SLH_NBUF; ++b) L.gc_key[b] = -1;
      const int key = (ko ? 8 : 0) | p.interp_type;
      const int dst = in_role[k];
      int src = -1;
      for (int b = 0; b < SLH_NBUF; ++b)
        if (L.gc_key[b] == key && L.gc_alpha[b] == alpha && (src < 0 || b == dst)) src = b;
      st = src >= 0 ? launch_ghosts_reuse(c, lev, dst, src, ko) : launch_ghosts(c, lev, dst, alpha, p.interp_type, ko);
      L.gc_key[dst] = key;
      L.gc_alpha[dst] = alpha;
    } else {
      st = launch_ghosts(c, lev, in_role[k], alpha, p.interp_type, ko);
    }
    prof_end(c);
    if (st != SLH_OK) return st;
    StageLaunch sl;
    memset(&sl, 0, sizeof(sl));
    sl.stage = k + 1;
    sl.in_buf = in_role[k];
    sl.yn_buf = ybuf;
    sl.d_buf = SLH_BUF_D;
    sl.out_buf = out_role[k];
    sl.c_buf = (!ssp && k == 3 && L.buf[SLH_BUF_C]) ? SLH_BUF_C : -1;
    sl.c_stage = cs * dt;
    sl.ha = ssp ? dt : aRK[k] * dt;
    sl.hb = ssp ? 0.0 : bRK[k] * dt;
    sl.ssp = ssp ? 1 : 0;
    sl.rkn = rkn ? 1 : 0;
    if (rkn5) {
      sl.ha = sl.hb = 0.0;
      sl.rkn5 = 1;
      for (int q = 0; q < 9; ++q) sl.rq[q] = rq5[k][q];
    } else if (rkn) {
      sl.ha = rknc[k][0];
      sl.hb = rknc[k][1];
      sl.hc = rknc[k][2];
      sl.hd = rknc[k][3];
      sl.he = rknc[k][4];
    }
    sl.sa = ssp ? aSSP[k] : 0.0;
    sl.sb = ssp ? bSSP[k] : 0.0;
    sl.lev = lev;
    double extra = 0.0;
    if (k == 0 && (flags & SLH_FUSE_TAG)) {
      if (!L.tags_dev) return fail(SLH_ERR_STATE, "rk_step: SLH_FUSE_TAG needs tags_dev at init_level");
      sl.tags = L.tags_dev;
      extra = 1.0;
    }
    if (k == 0 && (flags & SLH_FUSE_ENERGY)) {
      sl.epart = L.d_epart;
      sl.covered = L.d_covered;
      sl.cov_shift = ilog2(c->bf / 2);
      sl.cov_nb = L.ncov;
    }
    if (ko && !ssp && k == 3) {
      // the last RK4 stage's share goes into the increment before the
      // compensated final sum: D += b_4 dt Q(Y_4)
      prof_begin(c, SLH_PROF_KO, V * 12.0 * s);
      st = launch_ko(c, L, p, in_role[k], out_role[k], SLH_BUF_D, 0.0, bRK[k] * dt);
      prof_end(c);
      if (st != SLH_OK) return st;
    }
    prof_begin(c, SLH_PROF_S1 + k, V * (vals[k] * s + extra));
    int used = 0;
    st = launch_stage(c, L, p, sl, &used);
    prof_end(c);
    if (st != SLH_OK) return st;
    if (ko && (ssp || k < 3)) {
      // out += a dt Q(Y_s), D += b dt Q(Y_s) (classic RK4); out += b_s dt Q(Y_s) (SSPRK3)
      prof_begin(c, SLH_PROF_KO, V * (ssp ? 12.0 : 20.0) * s);
      st = ssp ? launch_ko(c, L, p, in_role[k], out_role[k], -1, bSSP[k] * dt, 0.0)
               : launch_ko(c, L, p, in_role[k], out_role[k], SLH_BUF_D, aRK[k] * dt, bRK[k] * dt);
      prof_end(c);
      if (st != SLH_OK) return st;
    }
    if (k == 0 && (flags & SLH_FUSE_ENERGY)) L.fused_energy_ctas = used;
    if (c->ncomp == NCOMP_GW) {
      // the 12 tensor fields: reads psi (2) + u, v (12) of the stage input,
      // and as the scalar stage y_n, D, C of its 12 fields
      double gvals[4] = {ssp ? 26.0 : 38.0, ssp ? 38.0 : 62.0, ssp ? 38.0 : 62.0,
                         c->prec == SLH_F32_KAHAN ? 74.0 : 50.0};
      if (bf16(c)) {   // 4-byte slots: psi (2) + u, v pairs (6) in, u, v pairs (6) out, + y_n pairs (6)
        gvals[0] = 14.0;
        gvals[1] = gvals[2] = 20.0;
      }
      if (rkn) {   // RKN4: stage 2 writes the velocities only (no y_n positions read)
        gvals[1] = 50.0;
        gvals[3] = c->prec == SLH_F32_KAHAN ? 74.0 : 50.0;
      }
      prof_begin(c, SLH_PROF_GW, V * gvals[k] * s);
      st = launch_gw_stage(c, L, p, sl);
      prof_end(c);
      if (st != SLH_OK) return st;
    }
  }
  if (ssp) {
    L.role_y = sbuf;
    L.role_prev = ybuf;
    L.role_s = nbuf;
  } else {
    L.role_y = nbuf;
    L.role_prev = ybuf;
  }
  return SLH_OK;
}

slh_status slh_rk_step(slh_ctx* c, int32_t lev, int32_t sub, double dt0, const slh_eom_params* p, uint32_t flags) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "rk_step: null ctx");
  slh_status st = check_params(p);
  if (st != SLH_OK) return st;
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "rk_step: level %d not defined", lev);
  if (lev >= c->stale_from) return fail(SLH_ERR_STATE, "rk_step: level %d must be regridded first", c->stale_from);
  if (sub != 0 && sub != 1) return fail(SLH_ERR_INVALID_ARG, "rk_step: sub must be 0 or 1");
  if (!(dt0 > 0.0)) return fail(SLH_ERR_INVALID_ARG, "rk_step: dt0 must be positive");
  return rk_step_impl(c, lev, sub, dt0, *p, flags);
}

static slh_status fill_impl(slh_ctx* c, int lev, double alpha, int itype, int mode) {
  NvtxRange range(mode == SLH_RESTRICT ? "slh level %d restrict + ghost fill" : "slh level %d ghost fill", lev);
  Level& L = c->lev[lev];
  for (int b = 0; b < SLH_NBUF; ++b) L.gc_key[b] = -1;   // the coarser level may have changed
  const size_t s = elem_size(c);
  if (mode == SLH_RESTRICT) {
    prof_begin(c, SLH_PROF_RESTRICT, (double)L.nrcells * c->nslots * 9 * s);
    slh_status st = launch_restrict(c, lev);
    prof_end(c);
    if (st != SLH_OK) return st;
    alpha = 1.0;
  }
  prof_begin(c, SLH_PROF_GHOST, (double)L.nghost_cells * ghost_fields(c) * 2 * s);
  slh_status st = launch_ghosts(c, lev, L.role_y, alpha, itype);
  prof_end(c);
  return st;
}

static slh_status advance_rec(slh_ctx* c, int lev, int sub, double dt0, const slh_eom_params& p, uint32_t flags) {
  slh_status st = rk_step_impl(c, lev, sub, dt0, p, flags);
  if (st != SLH_OK) return st;
  if (lev + 1 < c->nlevels) {
    for (int i = 0; i < 2; ++i)
      if ((st = advance_rec(c, lev + 1, i, dt0, p, flags)) != SLH_OK) return st;
    if ((st = fill_impl(c, lev + 1, 1.0, p.interp_type, SLH_RESTRICT)) != SLH_OK) return st;
  }
  return SLH_OK;
}

static unsigned long long graph_key(slh_ctx* c, double dt0, const slh_eom_params& p, uint32_t flags) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](const void* d, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(d);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  mix(&dt0, sizeof(dt0));
  mix(&p, sizeof(p));
  mix(&flags, sizeof(flags));
  mix(&c->tag_criteria, sizeof(c->tag_criteria));
  mix(c->te_crit, sizeof(c->te_crit));
  mix(&c->nlevels, sizeof(int));
  for (int l = 0; l < c->nlevels; ++l) {
    mix(&c->lev[l].d_boxes, sizeof(void*));
    mix(c->lev[l].buf, sizeof(c->lev[l].buf));
    mix(&c->lev[l].role_y, sizeof(int));
    mix(&c->lev[l].role_prev, sizeof(int));
    mix(&c->lev[l].role_s, sizeof(int));
  }
  return h | 1ull;
}

slh_status slh_advance(slh_ctx* c, double dt0, const slh_eom_params* p, uint32_t flags) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "advance: null ctx");
  slh_status st = check_params(p);
  if (st != SLH_OK) return st;
  if (c->nlevels < 1) return fail(SLH_ERR_STATE, "advance: no level defined");
  if (c->stale_from < c->nlevels) return fail(SLH_ERR_STATE, "advance: level %d must be regridded first", c->stale_from);
  if (!(dt0 > 0.0)) return fail(SLH_ERR_INVALID_ARG, "advance: dt0 must be positive");
  NvtxRange range("slh coarse step (%d levels)", c->nlevels);
  // prolonged ghosts are reused only inside one coarse step, whose order of
  // level steps advance_rec fixes
  struct ReuseScope {
    slh_ctx* c;
    explicit ReuseScope(slh_ctx* cc) : c(cc) {
      for (int l = 0; l < MAX_LEVELS; ++l)
        for (int b = 0; b < SLH_NBUF; ++b) c->lev[l].gc_key[b] = -1;
      c->ghost_reuse = true;
    }
    ~ReuseScope() { c->ghost_reuse = false; }
  } reuse_scope(c);
  if (!(flags & SLH_USE_GRAPH) || c->prof) return advance_rec(c, 0, 0, dt0, *p, flags);

  // graph replay: one graph per buffer-role configuration of the levels at
  // the start of the step (the key covers them with the parameters, boxes
  // and buffers); a replay leaves the roles the captured step left
  const uint32_t f = flags & ~SLH_USE_GRAPH;
  const unsigned long long key = graph_key(c, dt0, *p, f);
  slh_ctx::Graph* hit = nullptr;
  for (auto& g : c->graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    HostPhase phase(c, SLH_PROF_GRAPH_CAPTURE);   // preparation, capture and instantiation
    if (c->graphs.size() >= 4) drop_graphs(c);      // parameters or levels changed: start afresh
    // everything a launch sets up lazily (tensor maps, kernel attributes) is
    // prepared before capture: allocations are not allowed while capturing
    for (int l = 0; l < c->nlevels; ++l) {
      for (int diag = 0; diag < 2; ++diag) {
        StageLaunch sl;
        memset(&sl, 0, sizeof(sl));
        sl.dry = true;
        sl.stage = 1;
        sl.lev = l;
        sl.c_buf = -1;
        if (diag) sl.tags = reinterpret_cast<uint8_t*>(1);
        if ((st = launch_stage(c, c->lev[l], *p, sl, nullptr)) != SLH_OK) return st;
      }
      if (c->ncomp == NCOMP_GW) {
        StageLaunch sl;
        memset(&sl, 0, sizeof(sl));
        sl.dry = true;
        sl.stage = 1;
        sl.lev = l;
        sl.c_buf = -1;
        if ((st = launch_gw_stage(c, c->lev[l], *p, sl)) != SLH_OK) return st;
      }
    }
    int saved[MAX_LEVELS][3];
    for (int l = 0; l < c->nlevels; ++l) {
      saved[l][0] = c->lev[l].role_y;
      saved[l][1] = c->lev[l].role_prev;
      saved[l][2] = c->lev[l].role_s;
    }
    slh_ctx::Graph g;
    memset(&g, 0, sizeof(g));
    g.key = key;
    cudaGraph_t gr;
    SLH_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    slh_status cst = advance_rec(c, 0, 0, dt0, *p, f);
    cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
    for (int l = 0; l < c->nlevels; ++l) {
      g.roles_after[l][0] = c->lev[l].role_y;
      g.roles_after[l][1] = c->lev[l].role_prev;
      g.roles_after[l][2] = c->lev[l].role_s;
      c->lev[l].role_y = saved[l][0];
      c->lev[l].role_prev = saved[l][1];
      c->lev[l].role_s = saved[l][2];
    }
    if (cst != SLH_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(gr);
      return cst;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->graphs.push_back(g);
    hit = &c->graphs.back();
  }
  SLH_CUDA(cudaGraphLaunch(hit->exec, c->stream));
  for (int l = 0; l < c->nlevels; ++l) {
    c->lev[l].role_y = hit->roles_after[l][0];
    c->lev[l].role_prev = hit->roles_after[l][1];
    c->lev[l].role_s = hit->roles_after[l][2];
  }
  return SLH_OK;
}

slh_status slh_fill_ghosts(slh_ctx* c, int32_t lev, double alpha, int32_t itype, int32_t mode) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "fill_ghosts: null ctx");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "fill_ghosts: level %d not defined", lev);
  if (lev >= c->stale_from) return fail(SLH_ERR_STATE, "fill_ghosts: level %d must be regridded first", c->stale_from);
  if (mode != SLH_GHOSTS && mode != SLH_RESTRICT) return fail(SLH_ERR_INVALID_ARG, "fill_ghosts: bad mode");
  if (mode == SLH_RESTRICT && lev == 0) return fail(SLH_ERR_INVALID_ARG, "fill_ghosts: level 0 has no coarser level");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(SLH_ERR_INVALID_ARG, "fill_ghosts: alpha outside [0,1]");
  if (itype != 0 && itype != 2 && itype != 4) return fail(SLH_ERR_INVALID_ARG, "fill_ghosts: interp_type must be 0, 2 or 4");
  return fill_impl(c, lev, alpha, itype, mode);
}

slh_status slh_selftest_wait_timeout(slh_ctx* c, int64_t polls) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "selftest: null ctx");
  if (polls < 1 || polls > (1ll << 22)) return fail(SLH_ERR_INVALID_ARG, "selftest: polls must be in [1, 2^22]");
  return launch_expired_wait(c, polls);
}

slh_status slh_sync(slh_ctx* c) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "sync: null ctx");
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  int err = 0;
  SLH_CUDA(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    SLH_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    if (err == DERR_TIMEOUT) return fail(SLH_ERR_TIMEOUT, "device: a bounded wait gave up");
    if (err == DERR_NESTING) return fail(SLH_ERR_DEVICE, "device: ghost prolongation reached a cell the coarser level does not cover");
    if (err == DERR_RESTRICT) return fail(SLH_ERR_DEVICE, "device: restriction target outside the coarser level");
    return fail(SLH_ERR_DEVICE, "device error %d", err);
  }
  return SLH_OK;
}

static slh_status diag_pass(slh_ctx* c, int lev, const slh_eom_params& p, uint8_t* tags, bool energy, int* used) {
  Level& L = c->lev[lev];
  slh_status st;
  if ((st = fill_impl(c, lev, 1.0, p.interp_type, SLH_GHOSTS)) != SLH_OK) return st;
  StageLaunch sl;
  memset(&sl, 0, sizeof(sl));
  sl.stage = 0;
  sl.in_buf = L.role_y;
  sl.yn_buf = L.role_y;
  sl.d_buf = SLH_BUF_D;
  sl.out_buf = L.role_s;   // the diagnostics-only pass writes no field
  sl.c_buf = -1;
  sl.lev = lev;
  sl.c_stage = 0.0;
  sl.tags = tags;
  if (tags) {
    SLH_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->stream));
    sl.tagcount = c->d_count;
  }
  if (energy) {
    sl.epart = L.d_epart;
    sl.covered = L.d_covered;
    sl.cov_shift = ilog2(c->bf / 2);
    sl.cov_nb = L.ncov;
  }
  sl.cur_eta = true;   // diagnostics evaluate at the level's current eta
  prof_begin(c, SLH_PROF_DIAG, (double)L.lay.nvalid * 4 * elem_size(c));
  st = launch_stage(c, L, p, sl, used);
  prof_end(c);
  return st;
}

slh_status slh_tag(slh_ctx* c, int32_t lev, uint8_t* tags_dev, int64_t* n_tagged) {
  if (!c || !tags_dev) return fail(SLH_ERR_INVALID_ARG, "tag: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "tag: level %d not defined", lev);
  if (lev >= c->stale_from) return fail(SLH_ERR_STATE, "tag: level %d must be regridded first", c->stale_from);
  // the winding tags read psi only; the cheapest stencil variant runs them
  const slh_eom_params p = {1.0, 0.0, 1, 2, 2, 4, 4, 0, 0.0, 0, 0};
  int used = 0;
  slh_status st = diag_pass(c, lev, p, tags_dev, false, &used);
  if (st != SLH_OK) return st;
  if (n_tagged) {
    unsigned long long cnt = 0;
    SLH_CUDA(cudaMemcpyAsync(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    st = slh_sync(c);
    if (st != SLH_OK) return st;
    *n_tagged = (int64_t)cnt;
  }
  return SLH_OK;
}

slh_status slh_tag_blocks(slh_ctx* c, int32_t lev, int32_t nbuf, uint8_t* mask_host) {
  if (!c || !mask_host) return fail(SLH_ERR_INVALID_ARG, "tag_blocks: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "tag_blocks: level %d not defined", lev);
  if (lev >= c->stale_from) return fail(SLH_ERR_STATE, "tag_blocks: level %d must be regridded first", c->stale_from);
  if (nbuf < 0) return fail(SLH_ERR_INVALID_ARG, "tag_blocks: n_error_buf < 0");
  Level& L = c->lev[lev];
  slh_status st;
  const uint8_t* winding = nullptr;
  if (c->tag_criteria & SLH_TAG_WINDING) {
    if (!L.d_tagtmp) {
      cudaError_t e = cudaMalloc(&L.d_tagtmp, (size_t)L.lay.nvalid);
      if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "tag_blocks: %s", cudaGetErrorString(e));
    }
    if ((st = slh_tag(c, lev, L.d_tagtmp, nullptr)) != SLH_OK) return st;
    winding = L.d_tagtmp;
  }
  const uint8_t* tee = (c->tag_criteria & SLH_TAG_TEE) ? L.d_tee : nullptr;
  const int r = c->bf / 2;
  const int nb = L.n_dom / r;
  const size_t nmask = (size_t)nb * nb * nb;
  if (c->blockmask_cap < nmask) {
    cudaFree(c->d_blockmask);
    c->d_blockmask = nullptr;
    cudaError_t e = cudaMalloc(&c->d_blockmask, nmask);
    if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "tag_blocks: %s", cudaGetErrorString(e));
    c->blockmask_cap = nmask;
  }
  SLH_CUDA(cudaMemsetAsync(c->d_blockmask, 0, nmask, c->stream));
  if ((st = launch_tag_blocks(c, L, winding, tee, nbuf, r, c->d_blockmask, nb)) != SLH_OK) return st;
  SLH_CUDA(cudaMemcpyAsync(mask_host, c->d_blockmask, nmask, cudaMemcpyDeviceToHost, c->stream));
  return slh_sync(c);
}

slh_status slh_set_tagging(slh_ctx* c, uint32_t criteria, const double* te_crit) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "set_tagging: null ctx");
  if (criteria == 0 || (criteria & ~(SLH_TAG_WINDING | SLH_TAG_TEE)))
    return fail(SLH_ERR_INVALID_ARG, "set_tagging: criteria must be a nonzero combination of SLH_TAG_WINDING and SLH_TAG_TEE");
  if ((criteria & SLH_TAG_TEE) && !te_crit) return fail(SLH_ERR_INVALID_ARG, "set_tagging: SLH_TAG_TEE needs te_crit[4]");
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  drop_graphs(c);   // the restriction's arguments change
  c->tag_criteria = criteria;
  for (int q = 0; q < 4; ++q) c->te_crit[q] = (criteria & SLH_TAG_TEE) ? te_crit[q] : 0.0;
  if (criteria & SLH_TAG_TEE) {
    for (int l = 0; l < c->nlevels; ++l) {
      Level& L = c->lev[l];
      if (L.d_tee) continue;
      const size_t nb = (size_t)std::max<long long>(1, L.lay.nvalid);
      cudaError_t e = cudaMalloc(&L.d_tee, nb);
      if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "set_tagging: TEE tags: %s", cudaGetErrorString(e));
      SLH_CUDA(cudaMemsetAsync(L.d_tee, 0, nb, c->stream));
    }
  }
  return SLH_OK;
}

slh_status slh_tee_tags(slh_ctx* c, int32_t lev, uint8_t* dst, int32_t dst_is_host) {
  if (!c || !dst) return fail(SLH_ERR_INVALID_ARG, "tee_tags: null argument");
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "tee_tags: level %d not defined", lev);
  Level& L = c->lev[lev];
  if (!(c->tag_criteria & SLH_TAG_TEE) || !L.d_tee) return fail(SLH_ERR_STATE, "tee_tags: SLH_TAG_TEE is not enabled");
  SLH_CUDA(cudaMemcpyAsync(dst, L.d_tee, (size_t)L.lay.nvalid, cudaMemcpyDefault, c->stream));
  if (dst_is_host) return slh_sync(c);
  return SLH_OK;
}

// shadow checks shared by init and compare
static slh_status check_shadow(slh_ctx* c, slh_ctx* s, const char* who) {
  if (!c || !s || c == s) return fail(SLH_ERR_INVALID_ARG, "%s: need two distinct contexts", who);
  if (s->prec != c->prec || s->ncomp != c->ncomp)
    return fail(SLH_ERR_INVALID_ARG, "%s: shadow precision / field count differ", who);
  if (bf16(c)) return fail(SLH_ERR_INVALID_ARG, "%s: the shadow level is not built for BF16 tensor storage", who);
  if (2 * s->n0 != c->n0 || s->dx0 != 2.0 * c->dx0)
    return fail(SLH_ERR_INVALID_ARG, "%s: shadow must have n0/2 cells of spacing 2 dx0", who);
  if (s->device != c->device) return fail(SLH_ERR_INVALID_ARG, "%s: shadow on another device", who);
  if (c->nlevels < 1 || s->nlevels < 1) return fail(SLH_ERR_STATE, "%s: level 0 not defined", who);
  return SLH_OK;
}

// make `later` wait for the work queued so far on `earlier`
static slh_status stream_after(cudaStream_t later, cudaStream_t earlier) {
  if (later == earlier) return SLH_OK;
  cudaEvent_t e;
  SLH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaError_t r = cudaEventRecord(e, earlier);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(later, e, 0);
  cudaEventDestroy(e);
  SLH_CUDA(r);
  return SLH_OK;
}

slh_status slh_shadow_init(slh_ctx* c, slh_ctx* s) {
  slh_status st = check_shadow(c, s, "shadow_init");
  if (st != SLH_OK) return st;
  if ((st = stream_after(c->stream, s->stream)) != SLH_OK) return st;
  if ((st = launch_shadow(c, s, false)) != SLH_OK) return st;
  Level& S = s->lev[0];
  const size_t bytes = (size_t)S.lay.total * elem_size(s);
  SLH_CUDA(cudaMemcpyAsync(S.buf[S.role_prev], S.buf[S.role_y], bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (S.buf[SLH_BUF_C]) SLH_CUDA(cudaMemsetAsync(S.buf[SLH_BUF_C], 0, bytes, c->stream));
  // the shadow starts at level 0's (synchronised) time
  SLH_CUDA(cudaMemcpyAsync(s->d_time, c->d_time, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  SLH_CUDA(cudaMemcpyAsync(s->d_time + 1, c->d_time, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return stream_after(s->stream, c->stream);
}

slh_status slh_shadow_compare(slh_ctx* c, slh_ctx* s) {
  slh_status st = check_shadow(c, s, "shadow_compare");
  if (st != SLH_OK) return st;
  if (!(c->tag_criteria & SLH_TAG_TEE) || !c->lev[0].d_tee)
    return fail(SLH_ERR_STATE, "shadow_compare: SLH_TAG_TEE is not enabled");
  if ((st = stream_after(c->stream, s->stream)) != SLH_OK) return st;
  if ((st = launch_shadow(c, s, true)) != SLH_OK) return st;
  return stream_after(s->stream, c->stream);
}

slh_status slh_gw_spectrum(slh_ctx* c, int32_t ptype, int64_t* n2_out, double* g_out, int32_t cap, int32_t* nout) {
  if (!c || !nout) return fail(SLH_ERR_INVALID_ARG, "gw_spectrum: null argument");
  if (ptype != 1 && ptype != 2) return fail(SLH_ERR_INVALID_ARG, "gw_spectrum: projection type must be 1 or 2");
  if (c->ncomp != NCOMP_GW) return fail(SLH_ERR_STATE, "gw_spectrum: the context carries no gravitational-wave fields");
  if (c->nlevels < 1) return fail(SLH_ERR_STATE, "gw_spectrum: level 0 not defined");
  std::vector<double> bins;
  std::vector<unsigned long long> counts;
  slh_status st = gw_spectrum_impl(c, ptype, &bins, &counts);
  if (st != SLH_OK) return st;
  int need = 0;
  for (unsigned long long k : counts) need += k ? 1 : 0;
  *nout = need;
  if (cap < need || (need > 0 && (!n2_out || !g_out)))
    return fail(SLH_ERR_OUT_OF_RANGE, "gw_spectrum: capacity %d < %d entries", cap, need);
  const double n = (double)c->lev[0].n_dom;
  const double norm = 1.0 / (n * n * n * n * n * n);
  int o = 0;
  for (size_t k = 0; k < counts.size(); ++k)
    if (counts[k]) {
      n2_out[o] = (int64_t)k;
      g_out[o] = bins[k] * norm;
      ++o;
    }
  return slh_sync(c);
}

slh_status slh_reduce_energy(slh_ctx* c, const slh_eom_params* p, int32_t mode, double out[5]) {
  if (!c || !out) return fail(SLH_ERR_INVALID_ARG, "reduce_energy: null argument");
  slh_status st = check_params(p);
  if (st != SLH_OK) return st;
  if (c->nlevels < 1) return fail(SLH_ERR_STATE, "reduce_energy: no level defined");
  if (c->stale_from < c->nlevels)
    return fail(SLH_ERR_STATE, "reduce_energy: level %d must be regridded first", c->stale_from);
  double sums[MAX_LEVELS][4];
  int nl = c->nlevels;
  if (mode == 1) {
    Level& L = c->lev[0];
    if (c->nlevels != 1 || L.fused_energy_ctas <= 0)
      return fail(SLH_ERR_STATE, "reduce_energy: no fused energy partials (single level, SLH_FUSE_ENERGY)");
    if ((st = launch_energy_final(c, L.d_epart, L.fused_energy_ctas, c->d_levsum)) != SLH_OK) return st;
    nl = 1;
  } else if (mode == 0) {
    for (int l = 0; l < nl; ++l) {
      int used = 0;
      if ((st = diag_pass(c, l, *p, nullptr, true, &used)) != SLH_OK) return st;
      if ((st = launch_energy_final(c, c->lev[l].d_epart, used, c->d_levsum + 4 * l)) != SLH_OK) return st;
    }
  } else {
    return fail(SLH_ERR_INVALID_ARG, "reduce_energy: mode must be 0 or 1");
  }
  SLH_CUDA(cudaMemcpyAsync(sums, c->d_levsum, sizeof(double) * 4 * nl, cudaMemcpyDeviceToHost, c->stream));
  if ((st = slh_sync(c)) != SLH_OK) return st;
  double K = 0, G = 0, P = 0, S = 0;
  for (int l = 0; l < nl; ++l) {
    const double dx = c->lev[l].dx, vol = dx * dx * dx;
    K += sums[l][0] * vol;
    G += sums[l][1] * vol;
    P += sums[l][2] * vol;
    S += sums[l][3] * dx;
  }
  out[0] = K;
  out[1] = G;
  out[2] = P;
  out[3] = K + G + P;
  out[4] = S;
  return SLH_OK;
}

static slh_status set_tile_api(slh_ctx* c, int32_t lev, int32_t variant, int which, const char* what) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "%s: null ctx", what);
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "%s: level %d not defined", what, lev);
  int nv = 0;
  const TileVariant* vs = tile_variants(c->prec, &nv);
  if (variant < 0 || variant >= nv) return fail(SLH_ERR_OUT_OF_RANGE, "%s: variant %d outside [0,%d)", what, variant, nv);
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  return set_tile(c, c->lev[lev], vs[variant], which);
}

slh_status slh_set_tile(slh_ctx* c, int32_t lev, int32_t variant) {
  return set_tile_api(c, lev, variant, 3, "set_tile");
}

slh_status slh_set_diag_tile(slh_ctx* c, int32_t lev, int32_t variant) {
  return set_tile_api(c, lev, variant, 2, "set_diag_tile");
}

// Time every tile variant of the plain stage (diag = false: a stage-2 launch
// with the traffic of a real one, three distinct input buffers, writing only
// the scratch buffers YA and D) or of the diagnostics stage 1 (reads the
// state, writes YA, D and the energy partials), keep the fastest.
static slh_status autotune_impl(slh_ctx* c, int32_t lev, const slh_eom_params* p, int32_t reps, int32_t* chosen,
                                double* ms_out, bool diag) {
  const char* what = diag ? "autotune_diag" : "autotune";
  if (!c) return fail(SLH_ERR_INVALID_ARG, "%s: null ctx", what);
  NvtxRange range(diag ? "slh autotune (diagnostics) level %d" : "slh autotune level %d", lev);
  slh_status st = check_params(p);
  if (st != SLH_OK) return st;
  if (lev < 0 || lev >= c->nlevels) return fail(SLH_ERR_STATE, "%s: level %d not defined", what, lev);
  if (reps < 1) reps = 3;
  Level& L = c->lev[lev];
  const int which = diag ? 2 : 1;
  int nv = 0;
  const TileVariant* vs = tile_variants(c->prec, &nv);
  const bool was_prof = c->prof;
  c->prof = false;
  // the winding's near-tie fallback depends on the values it reads, so the
  // diagnostics stage is timed on the state with its ghosts filled, as in a step
  if (diag && (st = fill_impl(c, lev, 1.0, p->interp_type, SLH_GHOSTS)) != SLH_OK) {
    c->prof = was_prof;
    return st;
  }
  cudaEvent_t e0, e1;
  SLH_CUDA(cudaEventCreate(&e0));
  SLH_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < nv; ++v) {
    if ((st = set_tile(c, L, vs[v], which)) != SLH_OK) break;
    StageLaunch sl;
    memset(&sl, 0, sizeof(sl));
    if (diag) {
      sl.stage = 1;
      sl.in_buf = L.role_y;
      sl.yn_buf = L.role_y;
      sl.epart = L.d_epart;
    } else {
      // a middle stage in the form the integrator runs it (its pointwise
      // operands differ: 5 boxes for classic RK4, RKN4 and RKN5, 3 for SSPRK3)
      const bool rk_n = p->integrator == 21 || p->integrator == 22;
      sl.stage = rk_n ? 3 : 2;
      sl.in_buf = L.role_s;
      sl.yn_buf = L.role_y;
      sl.ssp = (p->integrator != 4 && !rk_n) ? 1 : 0;
      sl.rkn = rk_n ? 1 : 0;
      sl.rkn5 = p->integrator == 22 ? 1 : 0;
      sl.sa = sl.ssp ? 0.75 : 0.0;
      sl.sb = sl.ssp ? 0.25 : 0.0;
    }
    sl.d_buf = SLH_BUF_D;
    sl.out_buf = L.role_s;   // the level's scratch buffers only (S and D)
    sl.c_buf = -1;
    sl.ha = sl.hb = 0.0;
    sl.lev = lev;
    if ((st = launch_stage(c, L, *p, sl, nullptr)) != SLH_OK) break;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps; ++r)
      if ((st = launch_stage(c, L, *p, sl, nullptr)) != SLH_OK) break;
    if (st != SLH_OK) break;
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[v] = ms / reps;
    if (v == 0 || ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof = was_prof;
  if (st != SLH_OK) return st;
  drop_graphs(c);
  if (diag) L.fused_energy_ctas = 0;   // the partials now hold a timing launch's sums
  if ((st = set_tile(c, L, vs[best], which)) != SLH_OK) return st;
  if (chosen) *chosen = best;
  return slh_sync(c);
}

slh_status slh_autotune(slh_ctx* c, int32_t lev, const slh_eom_params* p, int32_t reps, int32_t* chosen,
                        double* ms_out) {
  return autotune_impl(c, lev, p, reps, chosen, ms_out, false);
}

slh_status slh_autotune_diag(slh_ctx* c, int32_t lev, const slh_eom_params* p, int32_t reps, int32_t* chosen,
                             double* ms_out) {
  return autotune_impl(c, lev, p, reps, chosen, ms_out, true);
}

slh_status slh_profile(slh_ctx* c, int32_t enable, int32_t reset) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "profile: null ctx");
  if (reset) {
    cudaStreamSynchronize(c->stream);
    for (auto& r : c->prof_open) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    c->prof_open.clear();
    for (int k = 0; k < SLH_PROF_NKINDS; ++k) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
      c->prof_bytes[k] = 0;
    }
  }
  c->prof = enable != 0;
  return SLH_OK;
}

slh_status slh_profile_read(slh_ctx* c, int32_t kind, double* ms, int64_t* launches, double* bytes) {
  if (!c) return fail(SLH_ERR_INVALID_ARG, "profile_read: null ctx");
  if (kind < 0 || kind >= SLH_PROF_NKINDS) return fail(SLH_ERR_INVALID_ARG, "profile_read: bad kind");
  SLH_CUDA(cudaStreamSynchronize(c->stream));
  for (auto& r : c->prof_open) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.kind] += t;
      c->prof_n[r.kind] += 1;
      c->prof_bytes[r.kind] += r.bytes;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->prof_open.clear();
  if (kind == SLH_PROF_STAGE) {
    double m = 0, b = 0;
    long long n = 0;
    for (int k = SLH_PROF_S1; k <= SLH_PROF_S4; ++k) {
      m += c->prof_ms[k];
      n += c->prof_n[k];
      b += c->prof_bytes[k];
    }
    if (ms) *ms = m;
    if (launches) *launches = n;
    if (bytes) *bytes = b;
    return SLH_OK;
  }
  if (ms) *ms = c->prof_ms[kind];
  if (launches) *launches = c->prof_n[kind];
  if (bytes) *bytes = c->prof_bytes[kind];
  return SLH_OK;
}

}  // extern "C"
