// Internal structures of the GB300 AMR stepper (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "slh.h"

struct CUtensorMap_st;   // cuda.h: the driver's tensor-map type

namespace slh {

// x padding in front of the first valid cell of every row: keeps the first
// valid cell 16-byte aligned for FP32 and FP64 and is >= every ghost width.
constexpr int XPAD = 4;
constexpr int NCOMP = 4;        // psi1, psi2, Pi1, Pi2
constexpr int NCOMP_GW = 16;    // + u_xx..u_yz (4..9), v_xx..v_yz (10..15)
constexpr int GW_U0 = 4, GW_V0 = 10;
constexpr int SLOT_U0 = 4, SLOT_V0 = 7;   // SLH_F32_BF16: first slot of the u and v pairs
constexpr int MAX_LEVELS = 8;

// Per-box geometry as the kernels see it.
struct BoxDev {
  int lo[3];        // first valid cell, level index space
  int n[3];         // valid extents
  int pitch;        // padded x row length (elements)
  int pny, pnz;     // padded y / z extents (n + 2 g)
  int pad_;
  long long off;    // element offset of component 0
  long long cs;     // component stride (elements)
  long long voff;   // offset of the box's first valid cell in dense valid-cell arrays
};

// A rectangular piece of a box's ghost shell (at most 32 cells along its two
// long axes): cells lo..lo+ext-1 in valid-relative coordinates (-g .. n+g-1),
// classified on the host from the level's block map:
//   GHOST_COPY     every cell lies in box `src` of the same level under one
//                  periodic image: source valid-relative = cell + d
//   GHOST_PROLONG  no cell lies in a box of the same level
//   GHOST_MIXED    anything else (per-cell lookup)
constexpr int GHOST_COPY = 0;
constexpr int GHOST_PROLONG = 1;
constexpr int GHOST_MIXED = 2;
constexpr int GHOST_CHUNK = 32;
constexpr int PROLONG_RAD_MAX = 2;   // widest prolongation stencil (type 4)
struct GhostRegion {
  int box;
  int lo[3];
  int ext[3];
  int kind;
  int src;
  int d[3];
  // prolongation / mixed regions of a level > 0: the coarse patch (the
  // radius-2 stencil footprint of the region) as pieces [p0, p0+np), each in
  // one coarse box under one periodic image; covered = 1 iff they tile it
  int p0, np, covered;
};

// One rectangular piece of a region's coarse patch: ext cells starting at
// valid-relative cell src of coarse box cbox go to patch cell dst.
struct PatchPiece {
  int cbox;
  int src[3];
  int dst[3];
  int ext[3];
};

// Restriction work: one fine box, its coarse region.
struct RestrictItem {
  int fbox;
  int n[3];         // coarse extents = fine extents / 2
};
constexpr int RESTRICT_CHUNK = 256;   // coarse cells per restriction CTA step

// A stage-kernel tile shape: x and y extent of the CTA's cell column, the
// TMA pipeline depth (planes in flight) and the z-march length of one item.
struct TileVariant {
  int tx, ty, p, zlen;
};

struct Tile {
  TileVariant v{32, 16, 2, 64};
  int4* d_items = nullptr;       // work items (box, x0, y0, z0)
  int nitems = 0;
  int zlen = 64;
};

struct Layout {
  std::vector<BoxDev> boxes;
  long long total = 0;
  long long nvalid = 0;
};

bool make_layout(int g, int ncomp, const slh_box* boxes, int nboxes, Layout* out, std::string* why);

struct Level {
  bool defined = false;
  int n_dom = 0;                 // cells per axis of the level's periodic domain
  double dx = 0, dtfac = 1;      // dt_l = dt0 * dtfac
  std::vector<slh_box> boxes;
  Layout lay;
  void* buf[SLH_NBUF] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int role_y = SLH_BUF_Y;        // buffer currently holding y_n
  int role_prev = SLH_BUF_YB;    // buffer holding the previous state
  int role_s = SLH_BUF_YA;       // stage scratch (rotates with the other two under SSPRK3)
  uint8_t* tags_dev = nullptr;   // caller-owned (fused tags)
  // device metadata (owned)
  BoxDev* d_boxes = nullptr;
  int* d_bmap = nullptr;         // block owner map, blocks of bf cells
  std::vector<int> h_bmap;       // host mirror of the block owner map
  int nb_dom = 0;
  GhostRegion* d_gregions = nullptr;
  int ngregions = 0;
  int ncopyregions = 0;          // regions [0, ncopyregions) are copies
  PatchPiece* d_pieces = nullptr;
  int npieces = 0;
  long long nghost_cells = 0;
  Tile tile;                     // stage work items for the chosen tile variant
  Tile dtile;                    // the same for the diagnostics stage 1 (tags, energy)
  int4* d_col_items = nullptr;   // column work items (box, x0, y0, z0) of the GW and dissipation kernels
  int ncol_items = 0;
  std::map<unsigned long long, void*> tmaps;   // device tensor maps per (G, TX, TY)
  uint8_t* d_covered = nullptr;  // covered by the finer level, blocks of bf/2 cells
  int ncov = 0;
  RestrictItem* d_ritems = nullptr;  // restriction of this level onto lev-1, per fine box
  int2* d_rchunks = nullptr;         // (item, first coarse cell) chunks of RESTRICT_CHUNK cells
  int nritems = 0, nrchunks = 0;
  long long nrcells = 0;
  double* d_epart = nullptr;     // energy partials (per CTA x 4)
  int epart_cap = 0;
  int fused_energy_ctas = 0;     // CTAs of the last fused-energy stage 1
  uint8_t* d_tagtmp = nullptr;   // internal tags for slh_tag_blocks
  uint8_t* d_tee = nullptr;      // truncation-error-estimate tags (per valid cell)
  // Within one step of the coarser level, the prolonged ghost cells a fill
  // wrote into buffer b (time fraction alpha, key = fields and interpolation
  // type) stay valid until the coarser level changes: a later fill with the
  // same alpha copies them instead of prolonging again (slh_advance only).
  double gc_alpha[SLH_NBUF] = {0, 0, 0, 0, 0};
  int gc_key[SLH_NBUF] = {-1, -1, -1, -1, -1};   // -1: nothing cached
};

struct ProfRec {
  cudaEvent_t a, b;
  int kind;
  double bytes;
};

}  // namespace slh

struct slh_ctx {
  int n0 = 0;
  double dx0 = 0;
  int g = 0;
  int bf = 0;
  int prec = SLH_F64;
  int ncomp = slh::NCOMP;        // fields per cell: 4, or 16 with the GW tensor
  int nslots = slh::NCOMP;       // storage slots per cell: ncomp, or 10 with BF16 tensor pairs
  int max_levels = 1;
  int nlevels = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  slh::Level lev[slh::MAX_LEVELS];
  double* d_time = nullptr;      // [2*MAX_LEVELS]: eta[l], eta_start[l]
  int* d_err = nullptr;          // latched device error code
  double* d_levsum = nullptr;    // [MAX_LEVELS][4] per-level energy sums
  unsigned long long* d_count = nullptr;
  uint8_t* d_blockmask = nullptr;
  size_t blockmask_cap = 0;
  // profiling
  bool prof = false;
  bool ghost_reuse = false;       // set while slh_advance steps the hierarchy
  std::vector<slh::ProfRec> prof_open;
  double prof_ms[SLH_PROF_NKINDS] = {0};
  long long prof_n[SLH_PROF_NKINDS] = {0};
  double prof_bytes[SLH_PROF_NKINDS] = {0};
  // CUDA graphs of one coarse step, one per buffer-role configuration the
  // levels start it in (two for the integrators that swap state and previous
  // state, three for SSPRK3's rotation of three buffers)
  struct Graph {
    unsigned long long key;
    cudaGraphExec_t exec;
    int roles_after[slh::MAX_LEVELS][3];   // (y, prev, s) of every level after the step
  };
  std::vector<Graph> graphs;
  int stale_from = slh::MAX_LEVELS;   // levels >= this must be regridded before stepping
  int regrid_itype = 4;
  uint32_t tag_criteria = SLH_TAG_WINDING;
  double te_crit[4] = {0.0, 0.0, 0.0, 0.0};
  // regrid policy (Sec. 2.3): each level's volume at the last global regrid
  // and the volume local regrids added to it since
  bool rp_valid = false;
  int rp_nlev = 0;
  double rp_base[slh::MAX_LEVELS] = {0};
  double rp_added[slh::MAX_LEVELS] = {0};
  int rp_count = 0;
  int rp_pending = -1;
};

namespace slh {

// error reporting (thread-local message)
slh_status fail(slh_status code, const char* fmt, ...);

// Host helper: f(i) for i in [0, n) on up to 16 threads in contiguous chunks
// (a plain loop below about 64K units of work, work_per_i units per i).
// Every caller writes disjoint data per i, so results do not depend on the
// thread count.
template <typename F>
void parallel_for(int n, size_t work_per_i, F f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<size_t>({(size_t)hw, (size_t)16, (size_t)std::max(n, 1), (size_t)n * work_per_i / 65536 + 1});
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  auto chunk = [&](int t) {
    const int a = (int)((long long)n * t / nt), b = (int)((long long)n * (t + 1) / nt);
    for (int i = a; i < b; ++i) f(i);
  };
  for (int t = 1; t < nt; ++t) th.emplace_back(chunk, t);
  chunk(0);
  for (std::thread& x : th) x.join();
}
slh_status cuda_fail(cudaError_t e, const char* what);

#define SLH_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return slh::cuda_fail(e_, #call); \
  } while (0)

// device error codes latched in ctx->d_err
constexpr int DERR_NESTING = 1;   // prolongation stencil reached an uncovered coarse cell
constexpr int DERR_RESTRICT = 2;  // fine cell projected outside the coarse level
constexpr int DERR_TIMEOUT = 3;   // a bounded wait gave up

// launchers (stage.cu, ghost.cu, diag.cu)
struct StageLaunch {
  int stage;            // 0 = diagnostics only, 1..4
  int in_buf, yn_buf, d_buf, out_buf, c_buf;   // physical buffer indices (-1: unused)
  double c_stage;       // c_s * dt
  double ha, hb;        // a_{s+1} dt, b_s dt (classic RK4); dt (SSPRK3)
  int ssp;              // 1: low-storage SSPRK3 stage, out = sa y_n + sb (Y + ha k)
  double sa, sb;
  int rkn;              // 1: RKN4 stage; ha, hb, hc, hd, he its coefficients of Pi_n in the
  double hc, hd, he;    // positions, a in the positions, a in the velocities, a into the
                        // position sum, a into the velocity sum (a = this stage's Pi')
  uint8_t* tags;
  double* epart;        // per CTA x 4 (kin, grad, pot, pierced count)
  unsigned long long* tagcount;
  const uint8_t* covered;
  int cov_shift, cov_nb;
  int lev;
  bool cur_eta;         // evaluate at eta[lev] (diagnostics) instead of eta_start[lev] + c_stage
  bool dry;             // set up tensor maps and kernel attributes only, launch nothing
  int rkn5;             // 1 (with rkn): RKN5 stage, rq its coefficients (see stage_kernel.cuh)
  double rq[9];
};
slh_status launch_stage(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s,
                        int* ctas_used);
const TileVariant* tile_variants(int prec, int* n);
void free_tmaps(Level& L);
slh_status launch_expired_wait(slh_ctx* c, long long polls);

slh_status launch_gw_stage(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s);
slh_status build_gw_tmaps(slh_ctx* c, Level& L, int G, int TX, int TY, ::CUtensorMap_st** out);
slh_status build_tmaps(slh_ctx* c, Level& L, int G, int TX, int TY, ::CUtensorMap_st** out);
slh_status launch_stage_rkn(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used);
slh_status launch_stage_diag(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used,
                             bool rkn);
// Kreiss-Oliger dissipation of the stage input in_buf: out += cout Q, D += cd Q (psi, Pi)
slh_status launch_ko(slh_ctx* c, Level& L, const slh_eom_params& p, int in_buf, int out_buf, int d_buf, double cout,
                     double cd);
constexpr int COL_TX = 32, COL_TY = 8, COL_ZLEN = 32;

slh_status launch_ghosts(slh_ctx* c, int lev, int role, double alpha, int itype, bool with_pi = false);
// Ghost fill of buffer `role` whose prolonged cells are copied from buffer
// `src` of the same level (filled earlier with the same coarse data and time
// fraction; src == role: they are in place); same-level copies as usual.
slh_status launch_ghosts_reuse(slh_ctx* c, int lev, int role, int src, bool with_pi = false);
slh_status launch_restrict(slh_ctx* c, int fine_lev);
slh_status launch_energy_final(slh_ctx* c, const double* epart, int n, double* out4);
slh_status launch_tag_blocks(slh_ctx* c, Level& L, const uint8_t* tags, const uint8_t* tags2, int nbuf, int r,
                             uint8_t* mask, int nb);
slh_status launch_shadow(slh_ctx* c, slh_ctx* shadow, bool compare);
slh_status gw_spectrum_impl(slh_ctx* c, int ptype, std::vector<double>* bins, std::vector<unsigned long long>* counts);
slh_status launch_time_begin(slh_ctx* c, int lev, int sub, double dt_l);
slh_status launch_regrid_fill(slh_ctx* c, int lev, Level& fresh, Level* old);

// profiling helpers
void prof_begin(slh_ctx* c, int kind, double bytes);
void prof_end(slh_ctx* c);
// host wall-clock phase timer: adds its lifetime to kind (always recorded)
struct HostPhase {
  slh_ctx* c;
  int kind;
  double t0;
  HostPhase(slh_ctx* cc, int k);
  ~HostPhase();
  HostPhase(const HostPhase&) = delete;
  HostPhase& operator=(const HostPhase&) = delete;
};

// host regrid
slh_status regrid_boxes_impl(const uint8_t* tags, const int dims[3], int bf, int nbuf, int max_box,
                             const slh_box* parent, int nparent, std::vector<slh_box>* out);
slh_status local_regrid_impl(int L, int n0, int bf, const uint8_t* const* masks, const slh_box* boxes,
                             const int32_t* nboxes, std::vector<std::vector<slh_box>>* out);

}  // namespace slh
