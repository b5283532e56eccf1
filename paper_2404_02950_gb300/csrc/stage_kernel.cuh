// Fused stage kernel: finite-difference Laplacian (App. A), right-hand side
// of the axion-string system (Sec. 3.1, Eqs. EOM1-EOM2), the stage
// combination of classic RK4 (integrator type 4), low-storage SSPRK3 (type 10)
// or RKN4 (type 21, a compile-time flag), and -- in the diagnostics variant
// (stage 1 with fused tags/energy, or the diagnostics-only pass) -- the
// string-winding tags and the energy partials of the stage input.
//
// Work decomposition.  A persistent grid walks a list of (box, x0, y0, z0)
// tiles; each CTA marches along z through a TX x TY column of cells.  The
// z-planes a CTA needs form one continuous stream of "load steps" across all
// its tiles; one elected thread issues, P steps ahead of the consumers, TMA
// tensor copies (cp.async.bulk.tensor) of
//   - the halo'd psi1/psi2 plane (TX+8 by TY+2G cells, 16-byte aligned in x),
//   - the pointwise operands of the plane G below it (momenta of the stage
//     input, y_n, the increment accumulator, the Kahan compensation),
// into shared-memory rings whose completion is tracked by mbarrier
// transaction counts.  Consumers read the 2G+1 psi planes of the stencil from
// the ring and write outputs with coalesced stores.  In the plain variant the
// copies come from a producer warp of their own, and each consumer warp
// releases a load step on a "consumed" mbarrier when it is done with it, so
// the warps run without a CTA barrier per plane (the producer reuses the ring
// slots of step u - P - 1 for step u once all warps have released it); the
// diagnostics variant exchanges its winding data through shared memory, keeps
// thread 0 as the producer and one CTA barrier per plane.  Every waiting loop
// is bounded; on expiry the CTA latches DERR_TIMEOUT, drains its copies with a
// bounded wait and leaves.
//
// The kernel and its launch templates are shared by the translation units
// that instantiate them: stage.cu (classic RK4 and SSPRK3) and stage_rkn.cu
// (RKN4), compiled in parallel.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdio.h>
#include <string.h>

#include "slh_internal.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace slh {

constexpr int NPW_MAX = 7;   // pointwise boxes: Pi | y_n(0,1) y_n(2,3) | D(0,1) D(2,3) | C(0,1) C(2,3)

template <typename T>
struct StageArgs {
  const BoxDev* boxes;
  const int4* items;
  int nitems;
  int zlen;
  int gl;                   // ghost layers of the level layout
  const CUtensorMap* tmaps; // [box][buffer][kind 0 = halo'd psi, 1 = pointwise]
  int in_buf, yn_buf, d_buf, out_buf, c_buf;   // physical buffer indices (-1: none)
  T* bufs[SLH_NBUF];
  int stage;                // 0 = diagnostics only, 1..4 (classic RK4) or 1..3 (SSPRK3)
  int ssp;                  // 1: low-storage SSPRK3 combine a y_n + b (Y + h k)
  double sa, sb;            // its a_s, b_s (h is ha)
  const double* eta_start;  // device eta at the start of the step (or current eta)
  double c_stage;           // c_s * dt
  double lambda, a;
  int friction, eta_power;
  double inv_dx2;
  double ha, hb;
  uint8_t* tags;
  double* epart;
  unsigned long long* tagcount;
  const uint8_t* covered;
  int cov_shift, cov_nb;
  int* err;
  double hc, hd, he;        // RKN4 coefficients (with ha, hb; see StageLaunch)
  int rkn5;                 // RKN5 stage (RKN instantiations only), coefficients rq
  double rq[9];
};


// ---------------------------------------------------------------------------
// Winding contribution of the edge a -> b: +1 when it leaves the upper half
// plane (Im >= 0) turning counter-clockwise, -1 when it enters it turning
// clockwise, by the exact sign of X = Re a Im b - Im a Re b.  edge_terms
// gives delta + 1 (0..2) for N edges at once.

// FP64 inputs: X from two correctly rounded products and one correctly
// rounded difference, the form the oracle uses.  The sign classes of the
// four values decide most edges without X, in integer arithmetic on the bit
// patterns (GB300 issues FP64 at 1/64 of the FP32 rate):
//  - Im a >= 0 and Im b >= 0, or both < 0: delta = 0 whatever X is;
//  - the sign of Im changes and Re a, Re b >= 0 (-0 included): the two
//    rounded products have the signs that make X <= 0 on the way down and
//    X >= 0 on the way up (rounding keeps signs), so delta = 0;
//  - the sign of Im changes and Re a, Re b < 0: X > 0 down, X < 0 up, when
//    neither product underflows to zero, which holds for magnitudes in
//    [2^-500, 2^501) or zero ("safe" below);
//  - otherwise (mixed signs of Re, unsafe magnitudes, Inf or NaN) X itself
//    decides, out of line.
__device__ __forceinline__ unsigned dclass(double v) {
  // bit 0: v < 0 (sign bit set, nonzero); bit 1: v is zero or safe
  const int hi = __double2hiint(v);
  const unsigned mag = (unsigned)hi & 0x7FFFFFFFu;
  const bool zero = (mag | (unsigned)__double2loint(v)) == 0u;
  const bool safe = zero || ((mag >> 20) - 0x20Bu <= 0x3E8u);   // exponent field 0x20B .. 0x5F3
  return (unsigned)(hi < 0 && !zero) | ((unsigned)safe << 1);
}

static __device__ __noinline__ unsigned exact_edge_term_f64(double ar, double ai, double br, double bi) {
  const bool ua = ai >= 0.0, ub = bi >= 0.0;
  const double X = __dsub_rn(__dmul_rn(ar, bi), __dmul_rn(ai, br));
  return 1u + (unsigned)(ua && !ub && X > 0.0) - (unsigned)(!ua && ub && X < 0.0);
}

template <int N>
__device__ __forceinline__ void edge_terms(const double (&ar)[N], const double (&ai)[N], const double (&br)[N],
                                           const double (&bi)[N], unsigned (&out)[N]) {
  unsigned need[N], any = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const unsigned ca = dclass(ai[k]), cb = dclass(bi[k]), ra = dclass(ar[k]), rb = dclass(br[k]);
    const unsigned dI = (ca ^ cb) & 1u;                 // the sign of Im changes
    const unsigned both_neg = ra & rb & 1u;
    const unsigned safe = (ca & cb & ra & rb) >> 1;
    const unsigned fast = dI & both_neg;                // +1 down (Im a >= 0), -1 up
    out[k] = 1u + (fast & ~ca & 1u) - (fast & ca & 1u);
    need[k] = dI & (((ra ^ rb) & 1u) | (both_neg & ~safe & 1u));
    any |= need[k];
  }
  if (any) {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (need[k]) out[k] = exact_edge_term_f64(ar[k], ai[k], br[k], bi[k]);
  }
}

// FP32 near-tie fallback: the products, exact in FP64, formed in FP64.  Kept
// out of line so that FP64 work is never if-converted into the common path.
static __device__ __noinline__ unsigned exact_edge_term(float ar, float ai, float br, float bi) {
  const double X = __dsub_rn(__dmul_rn((double)ar, (double)bi), __dmul_rn((double)ai, (double)br));
  const bool ua = ai >= 0.0f, ub = bi >= 0.0f;
  return 1u + (unsigned)(ua && !ub && X > 0.0) - (unsigned)(!ua && ub && X < 0.0);
}

// FP32 inputs, in integer arithmetic on the bit patterns (no predicates, of
// which a thread has few).  Half-plane flags: bit 31 of fl(v + 0) is set iff
// v < 0 (the sum maps -0 to +0).  q = fl(Im a Re b), s = fma(Re a, Im b, -q)
// = fl(X + dq) with |dq| <= max(2^-24 |q|, 2^-150) the rounding error of q.
// When |s| > max(2^-23 |q|, 2^-126), s is normal (so |X + dq| >=
// |s| / (1 + 2^-24)) and exceeds |dq| with room to spare, so X has the sign
// of s.  The bound's bit pattern is max(bits|q| - 23 * 2^23, bits 2^-126)
// (scaling a normal number by 2^-23 subtracts 23 from its exponent field;
// where that leaves the normal range the 2^-126 term wins), and for
// non-negative floats the order of bit patterns is the numeric order.  An
// edge that crosses the real axis without such a certificate takes the
// exact fallback; with one, the sign bit of s is the sign of X.
template <int N>
__device__ __forceinline__ void edge_terms(const float (&ar)[N], const float (&ai)[N], const float (&br)[N],
                                           const float (&bi)[N], unsigned (&out)[N]) {
  unsigned need[N], any = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const unsigned na = __float_as_uint(__fadd_rn(ai[k], 0.0f)), nb = __float_as_uint(__fadd_rn(bi[k], 0.0f));
    const float q = __fmul_rn(ai[k], br[k]);
    const unsigned ns = __float_as_uint(__fmaf_rn(ar[k], bi[k], -q));
    const int bound = max((int)(__float_as_uint(q) & 0x7FFFFFFFu) - 0x0B800000, 0x00800000);
    const unsigned cert = (unsigned)(bound - (int)(ns & 0x7FFFFFFFu));   // bit 31: |s| above the bound
    const unsigned pos = ~na & nb & ~ns, neg = na & ~nb & ns;
    out[k] = 1u + (pos >> 31) - (neg >> 31);
    need[k] = (na ^ nb) & ~cert;
    any |= need[k];
  }
  if ((int)any < 0) {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if ((int)need[k] < 0) out[k] = exact_edge_term(ar[k], ai[k], br[k], bi[k]);
  }
}

// FP32 inputs, whether the winding term is nonzero (bit 31 of nz[k] set iff
// delta != 0), from the sign classes s = bit 31 of fl(v + 0) (set iff v < 0):
//  - the endpoints share the sign of Im: delta = 0;
//  - the sign of Im changes and both Re < 0: the edge crosses the negative
//    real axis (X = Re a Im b - Im a Re b is then > 0 on the way down and
//    < 0 on the way up), delta != 0;
//  - the sign of Im changes and both Re >= 0: X <= 0 on the way down and
//    >= 0 on the way up, delta = 0;
//  - the signs of Im and of Re both change: the sign of X decides (delta != 0
//    iff X > 0 on the way down, X < 0 on the way up), by the certificate of
//    edge_terms or, without one, exactly in FP64.  That last case is rare on
//    a smooth field (a few per thousand edges), so it runs in a branch that is
//    taken only by warps that need it.
template <int N>
__device__ __forceinline__ void edge_nonzero(const float (&ar)[N], const float (&ai)[N], const float (&br)[N],
                                             const float (&bi)[N], unsigned (&nz)[N]) {
  unsigned need[N], any = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const unsigned sra = __float_as_uint(__fadd_rn(ar[k], 0.0f)), sia = __float_as_uint(__fadd_rn(ai[k], 0.0f));
    const unsigned srb = __float_as_uint(__fadd_rn(br[k], 0.0f)), sib = __float_as_uint(__fadd_rn(bi[k], 0.0f));
    const unsigned dI = sia ^ sib;
    nz[k] = dI & sra & srb;
    need[k] = dI & (sra ^ srb);
    any |= need[k];
  }
  if (__any_sync(0xffffffffu, (int)any < 0)) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if ((int)need[k] >= 0) continue;
      const unsigned nb = __float_as_uint(__fadd_rn(bi[k], 0.0f));   // set: the way down
      const float q = __fmul_rn(ai[k], br[k]);
      const unsigned ns = __float_as_uint(__fmaf_rn(ar[k], bi[k], -q));
      const int bound = max((int)(__float_as_uint(q) & 0x7FFFFFFFu) - 0x0B800000, 0x00800000);
      const bool cert = (int)(ns & 0x7FFFFFFFu) > bound;
      if (cert) nz[k] = (nb & ~ns) | (~nb & ns);              // X > 0 down, X < 0 up
      else nz[k] = exact_edge_term(ar[k], ai[k], br[k], bi[k]) != 1u ? 0x80000000u : 0u;
    }
  }
}

// shared-memory geometry of one kernel variant (the diagnostics variant runs
// stage 0 or 1 only, whose pointwise ring holds just the momenta)
template <typename T, int G, int TX, int TY, int P, bool DIAG>
struct Geo {
  static constexpr int SXL = TX + 8;
  static constexpr int SY = TY + 2 * G;
  static constexpr int RPSI = 2 * G + 1 + P;
  static constexpr int RPW = P + 1;
  static constexpr int PSI_BYTES = 2 * SY * SXL * (int)sizeof(T);
  static constexpr int PSI_STRIDE = (PSI_BYTES + 127) / 128 * 128;
  static constexpr int PW2 = 2 * TY * TX * (int)sizeof(T);
  static constexpr int NPW = DIAG ? 1 : (sizeof(T) == 4 ? NPW_MAX : NPW_MAX - 2);
  static constexpr int PW_STRIDE = (NPW * PW2 + 127) / 128 * 128;
  static constexpr bool WS = !DIAG;     // producer warp + per-step release barriers
  static constexpr int NTHREADS = TX * TY + (WS ? 32 : 0);
  static constexpr int BAR_BYTES = 128;  // RPSI "loaded" + (P + 1) "consumed" mbarriers
  static_assert(RPSI + P + 1 <= BAR_BYTES / 8, "mbarrier area too small");
  static constexpr int SMEM = BAR_BYTES + RPSI * PSI_STRIDE + RPW * PW_STRIDE;
};

struct Cursor {
  int item, q, box, x0, y0, z0, z1;
  bool valid;
};

template <int G>
__device__ __forceinline__ void cursor_load(Cursor& c, const int4* items, const BoxDev* boxes, int nitems, int zlen) {
  c.valid = c.item < nitems;
  if (!c.valid) return;
  const int4 it = items[c.item];
  c.box = it.x;
  c.x0 = it.y;
  c.y0 = it.z;
  c.z0 = it.w;
  c.z1 = min(it.w + zlen, boxes[it.x].n[2]);
  c.q = c.z0 - G;
}

template <int G>
__device__ __forceinline__ void cursor_next(Cursor& c, const int4* items, const BoxDev* boxes, int nitems, int zlen) {
  if (++c.q <= c.z1 + G - 1) return;
  c.item += gridDim.x;
  cursor_load<G>(c, items, boxes, nitems, zlen);
}

template <typename T, int G, int TX, int TY, int P, bool DIAG, bool RKN>
__global__ void __launch_bounds__(Geo<T, G, TX, TY, P, DIAG>::NTHREADS, (DIAG && TX * TY <= 256) ? (sizeof(T) == 4 ? 3 : 2) : 1)
    stage_kernel(const StageArgs<T> A) {
  using GE = Geo<T, G, TX, TY, P, DIAG>;
  constexpr int SXL = GE::SXL, SY = GE::SY, RPSI = GE::RPSI, RPW = GE::RPW;
  constexpr int PLANE = SY * SXL;   // elements of one psi component plane
  constexpr int TXY = TX * TY;
  // producer warp (plain variant): consumer warps release each load step on
  // an mbarrier instead of meeting at a CTA barrier per plane
  constexpr bool WS = GE::WS;
  // diagnostics in bit-sliced form: FP32 fields, rows of 32 cells (one warp)
  constexpr bool BITS = DIAG && sizeof(T) == 4 && TX == 32;
  constexpr int RD = P + 1;         // "step consumed" barriers
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);
  unsigned char* psi_base = smem + GE::BAR_BYTES;
  unsigned char* pw_base = psi_base + RPSI * GE::PSI_STRIDE;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int gl = A.gl;

  const double eta = *A.eta_start + A.c_stage;
  const double cfd = A.friction ? 2.0 / eta : 0.0;
  const double cpd = A.eta_power == 2 ? A.lambda * (eta * eta) : A.lambda;
  const T c_fric = (T)cfd, c_pot = (T)cpd, a_c = (T)A.a;
  const T ha = (T)A.ha, hb = (T)A.hb, idx2 = (T)A.inv_dx2;
  const int stage = A.stage;
  const bool has_c = A.c_buf >= 0;
  // pointwise boxes this stage needs: Pi always; y_n and D from stage 2; C in stage 4
  const bool ssp = A.ssp != 0;
  // RKN5's stage 2 writes D without reading it
  const bool rkn5 = RKN && A.rkn5 != 0;
  const bool read_d = !ssp && !(rkn5 && stage == 2);
  const int npw = stage >= 2 ? (!read_d ? 3 : ((stage == 4 && has_c) ? 7 : 5)) : 1;
  const unsigned step_bytes_pw = (unsigned)(npw * GE::PW2);

  unsigned long long* done_bars = bars + RPSI;
  __shared__ int s_abort, s_issued;
  if (tid == 0) {
    for (int i = 0; i < RPSI; ++i) mbar_init(smem_u32(&bars[i]), 1);
    if (WS)
      for (int i = 0; i < RD; ++i) mbar_init(smem_u32(&done_bars[i]), TXY / 32);
    fence_mbar_init();
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();

  Cursor cc, pc;
  cc.item = blockIdx.x;
  cursor_load<G>(cc, A.items, A.boxes, A.nitems, A.zlen);
  pc = cc;

  // issue the copies of load step t (cursor c) -- elected thread only
  // (slot = load step mod RPSI, pslot = load step mod RPW)
  auto issue = [&](const Cursor& c, int slot, int pslot) {
    const unsigned bar = smem_u32(&bars[slot]);
    const bool pw = (c.q - G >= c.z0);
    mbar_expect_tx(bar, (unsigned)GE::PSI_BYTES + (pw ? step_bytes_pw : 0u));
    const CUtensorMap* mb = A.tmaps + (size_t)c.box * SLH_NBUF * 2;
    tma_load4(smem_u32(psi_base + slot * GE::PSI_STRIDE), mb + 2 * A.in_buf + 0, c.x0, c.y0 - G + gl, c.q + gl, 0,
              bar);
    if (pw) {
      unsigned char* dst = pw_base + pslot * GE::PW_STRIDE;
      const int xp = c.x0 + XPAD, yp = c.y0 + gl, zp = c.q - G + gl;
      tma_load4(smem_u32(dst), mb + 2 * A.in_buf + 1, xp, yp, zp, 2, bar);
      if (stage >= 2) {
        tma_load4(smem_u32(dst + 1 * GE::PW2), mb + 2 * A.yn_buf + 1, xp, yp, zp, 0, bar);
        tma_load4(smem_u32(dst + 2 * GE::PW2), mb + 2 * A.yn_buf + 1, xp, yp, zp, 2, bar);
      }
      if (stage >= 2 && read_d) {
        tma_load4(smem_u32(dst + 3 * GE::PW2), mb + 2 * A.d_buf + 1, xp, yp, zp, 0, bar);
        tma_load4(smem_u32(dst + 4 * GE::PW2), mb + 2 * A.d_buf + 1, xp, yp, zp, 2, bar);
        if (stage == 4 && has_c) {
          tma_load4(smem_u32(dst + 5 * GE::PW2), mb + 2 * A.c_buf + 1, xp, yp, zp, 0, bar);
          tma_load4(smem_u32(dst + 6 * GE::PW2), mb + 2 * A.c_buf + 1, xp, yp, zp, 2, bar);
        }
      }
    }
  };

  // ring positions are tracked incrementally in 32-bit registers:
  // consumer step t -> (slot, pslot, parity), producer step t+P -> (islot, ipslot)
  int issued = 0, islot = 0, ipslot = 0;
  if (WS && tid >= TXY) {
    // producer: load step u may overwrite the ring slots of step u - P - 1
    // once every consumer warp has released that step
    if (tid == TXY) {
      int dslot = 0;
      unsigned dpar = 0;
      while (pc.valid) {
        if (issued >= RD) {
          if (!mbar_wait(smem_u32(&done_bars[dslot]), dpar) || *(volatile int*)&s_abort) {
            atomicExch(&s_abort, 1);
            break;
          }
          if (++dslot == RD) {
            dslot = 0;
            dpar ^= 1u;
          }
        }
        fence_proxy_async();
        issue(pc, islot, ipslot);
        ++issued;
        if (++islot == RPSI) islot = 0;
        if (++ipslot == RPW) ipslot = 0;
        cursor_next<G>(pc, A.items, A.boxes, A.nitems, A.zlen);
      }
      s_issued = issued;
    }
    cc.valid = false;   // the producer warp consumes nothing
  }
  if (!WS && tid == 0) {
    for (int i = 0; i < P && pc.valid; ++i) {
      issue(pc, islot, ipslot);
      ++issued;
      if (++islot == RPSI) islot = 0;
      if (++ipslot == RPW) ipslot = 0;
      cursor_next<G>(pc, A.items, A.boxes, A.nitems, A.zlen);
    }
  }

  // per-thread energy partials in the field precision, FP32 ones with a
  // compensation term each (Kahan), so that no FP64 work remains inside the
  // plane loop of the FP32 form (FP64 runs at 1/64 of the FP32 rate here);
  // FP64 from the block reduction on
  // per-thread counts stay far below 2^32: at most 3 per cell a thread visits,
  // and a persistent CTA visits (cells of the level) / (CTAs) of them
  unsigned n_pierced = 0, n_tagged = 0;
  T i_kin = 0, i_grad = 0, i_pot = 0, c_kin = 0, c_grad = 0, c_pot_ = 0;
  // (FP64 partials need no compensation: a thread sums some thousands of
  // terms, whose rounding stays near 1e-13 relative, and every FP64 add
  // costs as much as 64 FP32 ones here)
  auto kahan = [](T& sum, T& comp, T v) {
    if constexpr (sizeof(T) == 8) {
      (void)comp;
      sum += v;
    } else {
      const T y_ = v - comp;
      const T t_ = sum + y_;
      comp = (t_ - sum) - y_;
      sum = t_;
    }
  };
  int cur_box = -1;
  BoxDev B;
  bool aborted = false;
  const int thread_off = (ty + G) * SXL + 4 + tx;
  constexpr int PSI_T = GE::PSI_STRIDE / (int)sizeof(T);

  // fixed per-thread assignment of the diagnostics work: extended-tile cells
  // (edges) and mask cells, with their shared-memory offsets.  Interior
  // columns first, TX consecutive items per row, so that a warp reads and
  // writes whole rows (no bank conflicts); the side columns after them.
  constexpr int NEK = ((TX + 2) * (TY + 2) + TXY - 1) / TXY;
  constexpr int NMK = ((TX + 1) * (TY + 1) + TXY - 1) / TXY;
  int e_x[NEK], e_y[NEK], e_off[NEK], m_x[NMK], m_y[NMK];
#pragma unroll
  for (int k = 0; k < NEK; ++k) {
    const int j = k * TXY + tid;
    if (j < (TY + 2) * TX) {
      e_x[k] = j % TX;
      e_y[k] = j / TX - 1;
    } else {
      const int r = j - (TY + 2) * TX;
      e_x[k] = (r & 1) ? TX : -1;
      e_y[k] = r / 2 - 1;
    }
    e_off[k] = e_y[k] * SXL + e_x[k];
  }
#pragma unroll
  for (int k = 0; k < NMK; ++k) {
    const int j = k * TXY + tid;
    if (j < (TY + 1) * TX) {
      m_x[k] = j % TX + 1;
      m_y[k] = j / TX;
    } else {
      m_x[k] = 0;
      m_y[k] = j - (TY + 1) * TX;
    }
  }
  // values carried from one plane to the next (diagnostics): corner values
  // of plane z and biased in-plane edge terms of each edge cell, the masks
  // of plane z-1 of each mask cell
  T c_r[NEK], c_i[NEK];
  unsigned e_pl[NEK], m_pl[NMK];
#pragma unroll
  for (int k = 0; k < NEK; ++k) {
    c_r[k] = 0;
    c_i[k] = 0;
    e_pl[k] = 0x0101u;
  }
#pragma unroll
  for (int k = 0; k < NMK; ++k) m_pl[k] = 0;
  (void)e_x; (void)e_y; (void)e_off; (void)m_x; (void)m_y; (void)c_r; (void)c_i; (void)e_pl; (void)m_pl;

  int t = 0, slot = 0, pslot = 0;
  unsigned parity = 0;
  int dslot = 0;
  for (; cc.valid; ++t) {
    if (!WS && tid == 0 && pc.valid) {
      fence_proxy_async();
      issue(pc, islot, ipslot);
      ++issued;
      if (++islot == RPSI) islot = 0;
      if (++ipslot == RPW) ipslot = 0;
      cursor_next<G>(pc, A.items, A.boxes, A.nitems, A.zlen);
    }
    bool ok = mbar_wait(smem_u32(&bars[slot]), parity);
    if (WS) {
      // warp-uniform: a warp leaves together, before its release
      ok = __all_sync(0xffffffffu, ok) && !*(volatile int*)&s_abort;
      if (!ok) {
        atomicExch(&s_abort, 1);
        aborted = true;
        break;
      }
    }

    const int z = cc.q - G;
    const bool compute = ok && z >= cc.z0;
    // diagnostics need the plaquette masks of plane z0-1 too: the last
    // prologue step of an item computes them
    const bool premask = DIAG && ok && z == cc.z0 - 1;
    if ((compute || premask) && cc.box != cur_box) {
      B = A.boxes[cc.box];
      cur_box = cc.box;
    }
    const int x = cc.x0 + tx, y = cc.y0 + ty;
    const bool active = (compute || premask) && x < B.n[0] && y < B.n[1];
    // the 2G+1 planes z-G..z+G of the ring as 32-bit element offsets into
    // the shared array (plb: tile origin, plane + thread_off: this thread's cell)
    const T* psi = reinterpret_cast<const T*>(psi_base);
    int plb[2 * G + 1];
#pragma unroll
    for (int k = 0; k <= 2 * G; ++k) {
      int sl = slot - 2 * G + k;
      if (sl < 0) sl += RPSI;
      plb[k] = sl * PSI_T + G * SXL + 4;
    }
    const int tcell = thread_off - (G * SXL + 4);
    auto S = [&](int c, int dx, int dy, int dz) -> T { return psi[plb[dz + G] + tcell + c * PLANE + dy * SXL + dx]; };
    T p1 = 0, p2 = 0, l1 = 0, l2 = 0, P1 = 0, P2 = 0, r2 = 0;
    if (compute && active) {
      const T* pwp = reinterpret_cast<const T*>(pw_base + pslot * GE::PW_STRIDE);
      auto PWv = [&](int box, int comp) -> T { return pwp[box * 2 * TXY + comp * TXY + ty * TX + tx]; };
      p1 = S(0, 0, 0, 0);
      p2 = S(1, 0, 0, 0);
      if (sizeof(T) == 8) {
        // textbook form sum_m w_m (f(+m) + f(-m)) + 3 w_0 f(0): fewest FP64 operations
        T a1 = (T)(3.0 * lap_w<G>(0)) * p1, a2 = (T)(3.0 * lap_w<G>(0)) * p2;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)lap_w<G>(m);
          a1 += w * (((S(0, m, 0, 0) + S(0, -m, 0, 0)) + (S(0, 0, m, 0) + S(0, 0, -m, 0))) +
                     (S(0, 0, 0, m) + S(0, 0, 0, -m)));
          a2 += w * (((S(1, m, 0, 0) + S(1, -m, 0, 0)) + (S(1, 0, m, 0) + S(1, 0, -m, 0))) +
                     (S(1, 0, 0, m) + S(1, 0, 0, -m)));
        }
        l1 = a1 * idx2;
        l2 = a2 * idx2;
      } else {
        // difference form sum_m w_m ((f(+m) - f0) + (f(-m) - f0)): the
        // differences of neighbouring values are exact, which keeps FP32
        // cancellation error at the level of the curvature itself
        T a1 = 0, a2 = 0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)lap_w<G>(m);
          a1 += w * ((((S(0, m, 0, 0) - p1) + (S(0, -m, 0, 0) - p1)) + ((S(0, 0, m, 0) - p1) + (S(0, 0, -m, 0) - p1))) +
                     ((S(0, 0, 0, m) - p1) + (S(0, 0, 0, -m) - p1)));
          a2 += w * ((((S(1, m, 0, 0) - p2) + (S(1, -m, 0, 0) - p2)) + ((S(1, 0, m, 0) - p2) + (S(1, 0, -m, 0) - p2))) +
                     ((S(1, 0, 0, m) - p2) + (S(1, 0, 0, -m) - p2)));
        }
        l1 = a1 * idx2;
        l2 = a2 * idx2;
      }
      P1 = PWv(0, 0);
      P2 = PWv(0, 1);
      r2 = p1 * p1 + p2 * p2;
      const T pot = c_pot * (r2 - (T)1) + a_c;
      const T kP1 = (-c_fric) * P1 + l1 - p1 * pot;
      const T kP2 = (-c_fric) * P2 + l2 - p2 * pot;
      if (DIAG && A.epart != nullptr) {
        // energy of the stage input, accumulated where its terms are formed;
        // the pierced-plaquette count follows the tags (three planes later)
        bool cov = false;
        if (A.covered != nullptr) {
          const int gx = (B.lo[0] + x) >> A.cov_shift, gy = (B.lo[1] + y) >> A.cov_shift,
                    gz = (B.lo[2] + z) >> A.cov_shift;
          cov = A.covered[((long long)gz * A.cov_nb + gy) * A.cov_nb + gx] != 0;
        }
        if (!cov) {
          const T dd = r2 - (T)1;
          kahan(i_kin, c_kin, (T)0.5 * (P1 * P1 + P2 * P2));
          kahan(i_grad, c_grad, (T)(-0.5) * (p1 * l1 + p2 * l2));
          kahan(i_pot, c_pot_, ((T)0.25 * c_pot) * (dd * dd) + ((T)0.5 * a_c) * r2);
        }
      }
      const long long e0 = B.off + (long long)(z + gl) * B.pny * B.pitch + (long long)(y + gl) * B.pitch + x + XPAD;
      const long long cs = B.cs;
      if (ssp) {
        // low-storage SSPRK3: out = a_s y_n + b_s (Y + h k), Y + h k alone at stage 1
        T* yo = A.bufs[A.out_buf];
        const T f0 = p1 + ha * P1, f1 = p2 + ha * P2, f2 = P1 + ha * kP1, f3 = P2 + ha * kP2;
        if (stage == 1) {
          yo[e0] = f0;
          yo[e0 + cs] = f1;
          yo[e0 + 2 * cs] = f2;
          yo[e0 + 3 * cs] = f3;
        } else {
          const T sa = (T)A.sa, sb = (T)A.sb;
          yo[e0] = sa * PWv(1, 0) + sb * f0;
          yo[e0 + cs] = sa * PWv(1, 1) + sb * f1;
          yo[e0 + 2 * cs] = sa * PWv(2, 0) + sb * f2;
          yo[e0 + 3 * cs] = sa * PWv(2, 1) + sb * f3;
        }
      } else if (RKN) {
        // RKN4 (positions psi, velocities Pi, a = kP this stage's Pi'):
        //   stage 1 (input y_n): psi + ha Pi + hb a, Pi + hc a; D = (hd a, he a)
        //   stage 2: Pi_n + hc a over the input's own velocities (its
        //            positions are stage 3's); D += (hd a, he a)
        //   stage 3: psi_n + ha Pi_n + hb a, Pi_n + hc a; D += (hd a, he a)
        //   stage 4: psi_n + (ha Pi_n + D_psi), Pi_n + (D_Pi + he a)
        // RKN5 (a independent of Pi; q = rq, k = a; the input's velocity
        // slots carry k1 into stage 2, the partial sum A4 into stage 3):
        //   stage 1 (input y_n): psi_n + q0 Pi_n + q1 k | k1
        //   stage 2: psi_n + q0 Pi_n + (q1 k1 + q2 k) | A4 = q3 k1 + q4 k;
        //            D = (q5 k1 + q6 k, q7 k1 + q8 k)
        //   stage 3: positions psi_n + q0 Pi_n + (A4 + q1 k);
        //            D = (q0 Pi_n + (D_psi + q2 k), D_Pi + q3 k)
        //   stage 4: psi_n + D_psi, Pi_n + (D_Pi + q0 k)
        T* yo = A.bufs[A.out_buf];
        T* dd = A.bufs[A.d_buf];
        const T hc = (T)A.hc, hd = (T)A.hd, he = (T)A.he;
        if (rkn5 && stage < 4) {
          const T q0 = (T)A.rq[0], q1 = (T)A.rq[1];
          if (stage == 1) {
            yo[e0] = p1 + q0 * P1 + q1 * kP1;
            yo[e0 + cs] = p2 + q0 * P2 + q1 * kP2;
            yo[e0 + 2 * cs] = kP1;
            yo[e0 + 3 * cs] = kP2;
          } else if (stage == 2) {
            const T q2 = (T)A.rq[2], q3 = (T)A.rq[3], q4 = (T)A.rq[4], q5 = (T)A.rq[5], q6 = (T)A.rq[6],
                    q7 = (T)A.rq[7], q8 = (T)A.rq[8];
            yo[e0] = PWv(1, 0) + q0 * PWv(2, 0) + (q1 * P1 + q2 * kP1);
            yo[e0 + cs] = PWv(1, 1) + q0 * PWv(2, 1) + (q1 * P2 + q2 * kP2);
            yo[e0 + 2 * cs] = q3 * P1 + q4 * kP1;
            yo[e0 + 3 * cs] = q3 * P2 + q4 * kP2;
            dd[e0] = q5 * P1 + q6 * kP1;
            dd[e0 + cs] = q5 * P2 + q6 * kP2;
            dd[e0 + 2 * cs] = q7 * P1 + q8 * kP1;
            dd[e0 + 3 * cs] = q7 * P2 + q8 * kP2;
          } else {
            const T q2 = (T)A.rq[2], q3 = (T)A.rq[3];
            yo[e0] = PWv(1, 0) + q0 * PWv(2, 0) + (P1 + q1 * kP1);
            yo[e0 + cs] = PWv(1, 1) + q0 * PWv(2, 1) + (P2 + q1 * kP2);
            dd[e0] = q0 * PWv(2, 0) + (PWv(3, 0) + q2 * kP1);
            dd[e0 + cs] = q0 * PWv(2, 1) + (PWv(3, 1) + q2 * kP2);
            dd[e0 + 2 * cs] = PWv(4, 0) + q3 * kP1;
            dd[e0 + 3 * cs] = PWv(4, 1) + q3 * kP2;
          }
        } else if (stage == 1) {
          yo[e0] = p1 + ha * P1 + hb * kP1;
          yo[e0 + cs] = p2 + ha * P2 + hb * kP2;
          yo[e0 + 2 * cs] = P1 + hc * kP1;
          yo[e0 + 3 * cs] = P2 + hc * kP2;
          dd[e0] = hd * kP1;
          dd[e0 + cs] = hd * kP2;
          dd[e0 + 2 * cs] = he * kP1;
          dd[e0 + 3 * cs] = he * kP2;
        } else if (stage <= 3) {
          if (stage == 3) {
            yo[e0] = PWv(1, 0) + ha * PWv(2, 0) + hb * kP1;
            yo[e0 + cs] = PWv(1, 1) + ha * PWv(2, 1) + hb * kP2;
          }
          yo[e0 + 2 * cs] = PWv(2, 0) + hc * kP1;
          yo[e0 + 3 * cs] = PWv(2, 1) + hc * kP2;
          dd[e0] = PWv(3, 0) + hd * kP1;
          dd[e0 + cs] = PWv(3, 1) + hd * kP2;
          dd[e0 + 2 * cs] = PWv(4, 0) + he * kP1;
          dd[e0 + 3 * cs] = PWv(4, 1) + he * kP2;
        } else {
          const T y0v = PWv(1, 0), y1v = PWv(1, 1), y2v = PWv(2, 0), y3v = PWv(2, 1);
          const T ka = rkn5 ? (T)A.rq[0] : he;
          const T inc0 = rkn5 ? PWv(3, 0) : ha * y2v + PWv(3, 0), inc1 = rkn5 ? PWv(3, 1) : ha * y3v + PWv(3, 1);
          const T inc2 = PWv(4, 0) + ka * kP1, inc3 = PWv(4, 1) + ka * kP2;
          if (has_c) {
            T* cc_ = A.bufs[A.c_buf];
            T v, sm;
            v = inc0 - PWv(5, 0); sm = y0v + v; cc_[e0] = (sm - y0v) - v; yo[e0] = sm;
            v = inc1 - PWv(5, 1); sm = y1v + v; cc_[e0 + cs] = (sm - y1v) - v; yo[e0 + cs] = sm;
            v = inc2 - PWv(6, 0); sm = y2v + v; cc_[e0 + 2 * cs] = (sm - y2v) - v; yo[e0 + 2 * cs] = sm;
            v = inc3 - PWv(6, 1); sm = y3v + v; cc_[e0 + 3 * cs] = (sm - y3v) - v; yo[e0 + 3 * cs] = sm;
          } else {
            yo[e0] = y0v + inc0;
            yo[e0 + cs] = y1v + inc1;
            yo[e0 + 2 * cs] = y2v + inc2;
            yo[e0 + 3 * cs] = y3v + inc3;
          }
        }
      } else if (stage == 1) {
        T* yo = A.bufs[A.out_buf];
        T* dd = A.bufs[A.d_buf];
        yo[e0] = p1 + ha * P1;
        yo[e0 + cs] = p2 + ha * P2;
        yo[e0 + 2 * cs] = P1 + ha * kP1;
        yo[e0 + 3 * cs] = P2 + ha * kP2;
        dd[e0] = hb * P1;
        dd[e0 + cs] = hb * P2;
        dd[e0 + 2 * cs] = hb * kP1;
        dd[e0 + 3 * cs] = hb * kP2;
      } else if (stage == 2 || stage == 3) {
        T* yo = A.bufs[A.out_buf];
        T* dd = A.bufs[A.d_buf];
        yo[e0] = PWv(1, 0) + ha * P1;
        yo[e0 + cs] = PWv(1, 1) + ha * P2;
        yo[e0 + 2 * cs] = PWv(2, 0) + ha * kP1;
        yo[e0 + 3 * cs] = PWv(2, 1) + ha * kP2;
        dd[e0] = PWv(3, 0) + hb * P1;
        dd[e0 + cs] = PWv(3, 1) + hb * P2;
        dd[e0 + 2 * cs] = PWv(4, 0) + hb * kP1;
        dd[e0 + 3 * cs] = PWv(4, 1) + hb * kP2;
      } else if (stage == 4) {
        T* yo = A.bufs[A.out_buf];
        const T y0v = PWv(1, 0), y1v = PWv(1, 1), y2v = PWv(2, 0), y3v = PWv(2, 1);
        const T inc0 = PWv(3, 0) + hb * P1, inc1 = PWv(3, 1) + hb * P2;
        const T inc2 = PWv(4, 0) + hb * kP1, inc3 = PWv(4, 1) + hb * kP2;
        if (has_c) {
          // compensated sum y + inc, the rounding error carried in C
          T* cc_ = A.bufs[A.c_buf];
          T v, sm;
          v = inc0 - PWv(5, 0); sm = y0v + v; cc_[e0] = (sm - y0v) - v; yo[e0] = sm;
          v = inc1 - PWv(5, 1); sm = y1v + v; cc_[e0 + cs] = (sm - y1v) - v; yo[e0 + cs] = sm;
          v = inc2 - PWv(6, 0); sm = y2v + v; cc_[e0 + 2 * cs] = (sm - y2v) - v; yo[e0 + 2 * cs] = sm;
          v = inc3 - PWv(6, 1); sm = y3v + v; cc_[e0 + 3 * cs] = (sm - y3v) - v; yo[e0 + 3 * cs] = sm;
        } else {
          yo[e0] = y0v + inc0;
          yo[e0 + cs] = y1v + inc1;
          yo[e0 + 2 * cs] = y2v + inc2;
          yo[e0 + 3 * cs] = y3v + inc3;
        }
      }
    }
    if constexpr (BITS) {
      // Plaquette windings, bit-sliced (FP32, 32-cell rows: one warp per row).
      // A plaquette's winding W is the signed sum of its four edge terms, and
      // a quadrilateral winds at most once around the origin: the angle each
      // edge turns through is below pi in magnitude, and where the sign of X
      // is exact (X in FP64 from FP32 values) the half-plane rule counts those
      // turns (proof by contradiction: two crossings of one sign would chain
      // the corners' angles into a < a).  So |W| <= 1, and W != 0 exactly
      // when an odd number of its edges have a nonzero term: the masks are
      // XORs of "edge nonzero" bits, 32 cells per operation.  Steps, one CTA
      // barrier apart (software-pipelined over the planes of an item):
      //  edges(z):      every edge cell of the tile grown by one cell
      //                 evaluates its z edge of plane z and its x, y edges of
      //                 plane z+1 (plane z0-1's own x, y edges in the
      //                 premask step); a warp (one row of 32 cells) packs
      //                 them with ballots, side columns into words of their
      //                 own;
      //  masks(z-2):    the last warp, one lane per owner row -1..TY-1, from the
      //                 edge words of planes z-2 and z-1;
      //  words(z-3):    the warp before it, one lane per row, the tag word (OR of the 12
      //                 plaquettes around each cell) from the masks of planes
      //                 z-3 and z-4, with the pierced-plaquette and tag counts;
      //  stores(z-4):   every thread stores its cell's tag byte.
      // Words hold cell x at bit x+1 (x = -1 .. 32).
      constexpr int NE = (TY + 2) * TX + 2 * (TY + 2);
      constexpr int SIDEW = (2 * (TY + 2) + 31) / 32;
      __shared__ unsigned bw[4][3][TY + 2];              // interior edge bits (plane & 3, x/y/z, row + 1)
      __shared__ unsigned bs[4][3][SIDEW];               // side columns: bit 2 (row + 1) + (x == TX)
      __shared__ unsigned long long mw[4][3][TY + 1];    // masks (plane & 3, normal z/x/y, owner row + 1)
      __shared__ unsigned long long tw[2][TY];           // tag words (plane & 1, row)
      const int lane = tid & 31, warp = tid >> 5;
      // the edge cells beyond one per thread (the last rows and the side
      // columns) fall to the first warps, so masks and tag words go to the last
      constexpr int MASK_WARP = TXY / 32 - 1, WORD_WARP = TXY / 32 - 2;
      static_assert(TXY / 32 >= 3, "bit-sliced winding needs at least 3 warps");
      auto row_word = [&](int slot, int dir, int rr) -> unsigned long long {
        unsigned long long w = (unsigned long long)bw[slot][dir][rr] << 1;
        // the row's two side bits, 2 rr and 2 rr + 1, share one word
        const unsigned sw = bs[slot][dir][rr >> 4] >> ((2 * rr) & 31);
        w |= (unsigned long long)(sw & 1u) | ((unsigned long long)((sw >> 1) & 1u) << 33);
        return w;
      };
      auto masks = [&](int pm) {
        if (warp != MASK_WARP) return;
        const int s0 = pm & 3, s1 = (pm + 1) & 3;
        constexpr unsigned long long OWN = (1ull << (TX + 1)) - 1;   // owners x = -1 .. TX-1
        // one lane per (owner row r - 1, orientation o):
        // xy: C.ex X.ey Y.ex C.ey;  yz: C.ey Y.ez Z.ey C.ez;  zx: C.ez Z.ex X.ez C.ex
        for (int idx = lane; idx < 3 * (TY + 1); idx += 32) {
          const int r = idx / 3, o = idx - 3 * r;
          unsigned long long m;
          if (o == 0) {
            const unsigned long long ex = row_word(s0, 0, r), ey = row_word(s0, 1, r);
            m = ex ^ (ey >> 1) ^ row_word(s0, 0, r + 1) ^ ey;
          } else if (o == 1) {
            m = row_word(s0, 1, r) ^ row_word(s0, 2, r + 1) ^ row_word(s1, 1, r) ^ row_word(s0, 2, r);
          } else {
            const unsigned long long ez = row_word(s0, 2, r);
            m = ez ^ row_word(s1, 0, r) ^ (ez >> 1) ^ row_word(s0, 0, r);
          }
          mw[pm & 3][o][r] = m & OWN;
        }
      };
      auto words = [&](int pt) {
        if (warp != WORD_WARP || lane >= TY) return;
        const int a = pt & 3, b = (pt - 1) & 3, r = lane + 1, rm = lane;   // owner rows y and y-1
        const unsigned long long xy0 = mw[a][0][r], xy1 = mw[a][0][rm], zx0 = mw[a][2][r], zx1 = mw[b][2][r];
        const unsigned long long tg = xy0 | (xy0 << 1) | xy1 | (xy1 << 1) | mw[a][1][r] | mw[a][1][rm] | mw[b][1][r] |
                                      mw[b][1][rm] | zx0 | (zx0 << 1) | zx1 | (zx1 << 1);
        tw[pt & 1][lane] = tg;
        const int yv = cc.y0 + lane;
        if (yv >= B.n[1]) return;
        const int nx = min(TX, B.n[0] - cc.x0);
        unsigned long long valid = ((1ull << nx) - 1) << 1;
        if (A.tags != nullptr) n_tagged += __popcll(tg & valid);
        if (A.epart != nullptr) {
          if (A.covered != nullptr) {
            // owners in blocks covered by the finer level do not count
            const int gy = (B.lo[1] + yv) >> A.cov_shift, gz = (B.lo[2] + pt) >> A.cov_shift;
            const uint8_t* crow = A.covered + ((long long)gz * A.cov_nb + gy) * A.cov_nb;
            for (int xx = 0; xx < nx;) {
              const int gx = (B.lo[0] + cc.x0 + xx) >> A.cov_shift;
              const int xe = min(nx, ((gx + 1) << A.cov_shift) - B.lo[0] - cc.x0);   // end of this block
              if (crow[gx]) valid &= ~((((1ull << (xe - xx)) - 1)) << (xx + 1));
              xx = xe;
            }
          }
          n_pierced += __popcll(mw[a][0][r] & valid) + __popcll(mw[a][1][r] & valid) + __popcll(mw[a][2][r] & valid);
        }
      };
      auto stores = [&](int ps) {
        if (A.tags == nullptr || !(x < B.n[0] && y < B.n[1])) return;
        A.tags[B.voff + ((long long)ps * B.n[1] + y) * B.n[0] + x] = (uint8_t)((tw[ps & 1][ty] >> (tx + 1)) & 1u);
      };
      if (compute || premask) {
#pragma unroll
        for (int k = 0; k < NEK; ++k) {
          if (k * TXY >= NE) break;                  // uniform over the CTA
          if (k * TXY + (warp << 5) >= NE) continue;   // uniform over the warp: no edge cell left
          const int j = k * TXY + tid;
          const bool act = j < NE;
          const int ey = e_y[k];
          auto SE = [&](int c, int dx, int dy, int dz) -> T { return psi[plb[dz + G] + c * PLANE + e_off[k] + dy * SXL + dx]; };
          // every lane runs the edge tests (they vote); lanes past the last
          // edge cell read nothing and test zeros
          T r0 = 0, i0 = 0, rz = 0, iz = 0, xr = 0, xi = 0, yr = 0, yi = 0;
          if (act) {
            r0 = premask ? SE(0, 0, 0, 0) : c_r[k];   // plane z0-1 from the ring in the premask step
            i0 = premask ? SE(1, 0, 0, 0) : c_i[k];
            rz = SE(0, 0, 0, 1);
            iz = SE(1, 0, 0, 1);
            xr = SE(0, 1, 0, 1);
            xi = SE(1, 1, 0, 1);
            yr = ey < TY ? SE(0, 0, 1, 1) : rz;
            yi = ey < TY ? SE(1, 0, 1, 1) : iz;
          }
          unsigned px = 0, py = 0;
          if (premask) {   // uniform over the CTA: the x and y edges of plane z0-1
            T br2[2] = {0, 0}, bi2[2] = {0, 0};
            if (act) {
              br2[0] = SE(0, 1, 0, 0);
              bi2[0] = SE(1, 1, 0, 0);
              br2[1] = ey < TY ? SE(0, 0, 1, 0) : r0;
              bi2[1] = ey < TY ? SE(1, 0, 1, 0) : i0;
            }
            const T ar2[2] = {r0, r0}, ai2[2] = {i0, i0};
            unsigned nz2[2];
            edge_nonzero<2>(ar2, ai2, br2, bi2, nz2);
            px = __ballot_sync(0xffffffffu, act && (int)nz2[0] < 0);
            py = __ballot_sync(0xffffffffu, act && (int)nz2[1] < 0);
          }
          // the z edge of plane z, the x and y edges of plane z+1
          const T ar3[3] = {r0, rz, rz}, ai3[3] = {i0, iz, iz}, br3[3] = {rz, xr, yr}, bi3[3] = {iz, xi, yi};
          unsigned nz3[3];
          edge_nonzero<3>(ar3, ai3, br3, bi3, nz3);
          const unsigned nzz = nz3[0], nzx = nz3[1], nzy = nz3[2];
          c_r[k] = rz;
          c_i[k] = iz;
          const unsigned bz = __ballot_sync(0xffffffffu, act && (int)nzz < 0);
          const unsigned bx = __ballot_sync(0xffffffffu, act && (int)nzx < 0);
          const unsigned by = __ballot_sync(0xffffffffu, act && (int)nzy < 0);
          if (lane == 0) {
            if (k * TXY + (warp << 5) < (TY + 2) * TX) {
              const int rr = ey + 1;   // one row per warp
              if (premask) {
                bw[z & 3][0][rr] = px;
                bw[z & 3][1][rr] = py;
              }
              bw[z & 3][2][rr] = bz;
              bw[(z + 1) & 3][0][rr] = bx;
              bw[(z + 1) & 3][1][rr] = by;
            } else {
              const int sw = (k * TXY + (warp << 5) - (TY + 2) * TX) >> 5;
              if (sw < SIDEW) {
                if (premask) {
                  bs[z & 3][0][sw] = px;
                  bs[z & 3][1][sw] = py;
                }
                bs[z & 3][2][sw] = bz;
                bs[(z + 1) & 3][0][sw] = bx;
                bs[(z + 1) & 3][1][sw] = by;
              }
            }
          }
        }
      }
      // planes z-2, z-3, z-4: their inputs were written before the last barrier
      if (compute && z - 2 >= cc.z0 - 1) masks(z - 2);
      if (compute && z - 3 >= cc.z0) words(z - 3);
      if (compute && z - 4 >= cc.z0) stores(z - 4);
      if (cc.valid && z == cc.z1 - 1) {   // the item's last plane: drain (uniform over the CTA)
        __syncthreads();
        if (z - 1 >= cc.z0 - 1) masks(z - 1);
        if (z - 2 >= cc.z0) words(z - 2);
        if (z - 3 >= cc.z0) stores(z - 3);
        __syncthreads();
        masks(z);
        if (z - 1 >= cc.z0) words(z - 1);
        if (z - 2 >= cc.z0) stores(z - 2);
        __syncthreads();
        words(z);
        if (z - 1 >= cc.z0) stores(z - 1);
        __syncthreads();
        stores(z);
      }
    }
    if constexpr (DIAG && !BITS) {
      // Plaquette windings.  The edge term is antisymmetric (delta(b,a) =
      // -delta(a,b)), so a plaquette's winding is the signed sum of the edges
      // leaving its corners along +x, +y, +z.  Three steps, software-pipelined
      // over the planes of an item so that one CTA barrier per plane (the
      // ring barrier below) separates them:
      //  edges(z):   every edge of the tile grown by one cell is evaluated
      //              once, spread over the CTA, and stored biased (delta + 1)
      //              as bytes 0-2 (e_x, e_y, e_z) of one word per cell: the
      //              vertical edges of plane z and the in-plane edges of
      //              plane z+1 (plane z0-1's own in-plane edges in the
      //              premask step);
      //  masks(z-2): the 3-bit "winding != 0" mask of each cell of the tile
      //              and of its low halo, from four words by byte-wise sums;
      //  tags(z-3):  a cell's tag is the OR over the 12 plaquettes it is a
      //              corner of (owners c, c-u, c-v, c-u-v), from the masks
      //              of two planes, which share one byte.
      // After an item's last plane the pipeline drains in three more
      // barrier-separated steps.  Each thread keeps the same edge and mask
      // cells on every plane, so the corner values of plane z, its in-plane
      // edge terms and the masks of the plane below stay in registers.
      constexpr int EXW = TX + 2, EXH = TY + 2, NE = EXW * EXH;
      constexpr int MW = TX + 1, MH = TY + 1, NM = MW * MH;
      __shared__ unsigned ew[4][EXH][EXW];     // edge words of planes z-2..z+1 (plane & 3)
      __shared__ unsigned char mk[2][MH][MW];  // by plane parity; bits 0-2: plane p, 3-5: plane p-1
      const bool in_box = x < B.n[0] && y < B.n[1];
      auto masks = [&](int pm) {
        const int s0 = pm & 3, s1 = (pm + 1) & 3, mo = pm & 1;
#pragma unroll
        for (int k = 0; k < NMK; ++k) {
          if (k * TXY + tid >= NM) break;
          const int mx = m_x[k], my = m_y[k];   // cell offset (mx-1, my-1) from (x0, y0)
          // windings in bytes 0, 1, 2 (normals z, x, y):
          //   xy: C.ex + X.ey - Y.ex - C.ey   (c, c+x, c+x+y, c+y)
          //   yz: C.ey + Y.ez - Z.ey - C.ez   (c, c+y, c+y+z, c+z)
          //   zx: C.ez + Z.ex - X.ez - C.ex   (c, c+z, c+z+x, c+x)
          // each term in 0..2, so every byte of s = W + 4 lies in 0..8 and no
          // carry or borrow crosses a byte
          const unsigned C = ew[s0][my][mx], X = ew[s0][my][mx + 1], Y = ew[s0][my + 1][mx], Z = ew[s1][my][mx];
          const unsigned plus = __byte_perm(__byte_perm(X, Y, 0x0061u), Z, 0x0410u);    // X.ey, Y.ez, Z.ex
          const unsigned minus = __byte_perm(__byte_perm(Y, Z, 0x0050u), X, 0x0610u);   // Y.ex, Z.ey, X.ez
          const unsigned rot = __byte_perm(C, 0u, 0x0021u);                              // C.ey, C.ez, C.ex
          const unsigned sw = (C + plus + 0x00040404u) - (minus + rot);
          const unsigned nz = ((sw ^ 0x00040404u) + 0x007F7F7Fu) & 0x00808080u;         // bit 7: W != 0
          const unsigned m = ((nz >> 7) & 1u) | ((nz >> 14) & 2u) | ((nz >> 21) & 4u);
          mk[mo][my][mx] = (unsigned char)(m | (m_pl[k] << 3));
          m_pl[k] = m;
        }
      };
      auto tags = [&](int pt) {
        if (!in_box) return;
        const int mo = pt & 1;
        const unsigned a00 = mk[mo][ty + 1][tx + 1], a0x = mk[mo][ty + 1][tx], a0y = mk[mo][ty][tx + 1],
                       a0xy = mk[mo][ty][tx];
        const unsigned u = a00 | a0y, v = a00 | a0x;
        const unsigned tg = ((u | a0x | a0xy) & 1u) | ((u | (u >> 3)) & 2u) | ((v | (v >> 3)) & 4u);
        const bool tagged = tg != 0;
        if (A.tags != nullptr) {
          A.tags[B.voff + ((long long)pt * B.n[1] + y) * B.n[0] + x] = tagged ? 1 : 0;
          n_tagged += tagged ? 1u : 0u;
        }
        if (A.epart != nullptr) {
          bool cov = false;
          if (A.covered != nullptr) {
            const int gx = (B.lo[0] + x) >> A.cov_shift, gy = (B.lo[1] + y) >> A.cov_shift,
                      gz = (B.lo[2] + pt) >> A.cov_shift;
            cov = A.covered[((long long)gz * A.cov_nb + gy) * A.cov_nb + gx] != 0;
          }
          if (!cov) n_pierced += __popc(a00 & 7u);
        }
      };
      if (compute || premask) {
#pragma unroll
        for (int k = 0; k < NEK; ++k) {
          if (k * TXY + tid >= NE) break;
          const int ey = e_y[k];
          auto SE = [&](int c, int dx, int dy, int dz) -> T { return psi[plb[dz + G] + c * PLANE + e_off[k] + dy * SXL + dx]; };
          T r0, i0;
          if (premask) {
            // plane z0-1: its corner values and in-plane edges from the ring
            r0 = SE(0, 0, 0, 0);
            i0 = SE(1, 0, 0, 0);
            const T xr = SE(0, 1, 0, 0), xi = SE(1, 1, 0, 0);
            const T yr = ey < TY ? SE(0, 0, 1, 0) : r0, yi = ey < TY ? SE(1, 0, 1, 0) : i0;
            const T ar2[2] = {r0, r0}, ai2[2] = {i0, i0}, br2[2] = {xr, yr}, bi2[2] = {xi, yi};
            unsigned b2[2];
            edge_terms<2>(ar2, ai2, br2, bi2, b2);
            e_pl[k] = b2[0] | (b2[1] << 8);
          } else {
            r0 = c_r[k];
            i0 = c_i[k];
          }
          const T rz = SE(0, 0, 0, 1), iz = SE(1, 0, 0, 1);
          const T xr = SE(0, 1, 0, 1), xi = SE(1, 1, 0, 1);
          const T yr = ey < TY ? SE(0, 0, 1, 1) : rz, yi = ey < TY ? SE(1, 0, 1, 1) : iz;
          // e_z of plane z, e_x and e_y of plane z+1
          const T ar3[3] = {r0, rz, rz}, ai3[3] = {i0, iz, iz}, br3[3] = {rz, xr, yr}, bi3[3] = {iz, xi, yi};
          unsigned b3[3];
          edge_terms<3>(ar3, ai3, br3, bi3, b3);
          const unsigned nxt = b3[1] | (b3[2] << 8);
          ew[z & 3][ey + 1][e_x[k] + 1] = e_pl[k] | (b3[0] << 16);
          ew[(z + 1) & 3][ey + 1][e_x[k] + 1] = nxt | (1u << 16);
          c_r[k] = rz;
          c_i[k] = iz;
          e_pl[k] = nxt;
        }
      }
      // planes z-2 and z-3: their inputs were written before the last barrier
      if (compute && z - 2 >= cc.z0 - 1) masks(z - 2);
      if (compute && z - 3 >= cc.z0) tags(z - 3);
      if (cc.valid && z == cc.z1 - 1) {   // the item's last plane: drain (uniform over the CTA)
        __syncthreads();
        if (z - 1 >= cc.z0 - 1) masks(z - 1);
        if (z - 2 >= cc.z0) tags(z - 2);
        __syncthreads();
        masks(z);
        if (z - 1 >= cc.z0) tags(z - 1);
        __syncthreads();
        tags(z);
      }
    }
    if (WS) {
      // this warp is done with the step's ring slots
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(smem_u32(&done_bars[dslot]));
      if (++dslot == RD) dslot = 0;
    } else if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    if (++slot == RPSI) {
      slot = 0;
      parity ^= 1u;
    }
    if (++pslot == RPW) pslot = 0;
    cursor_next<G>(cc, A.items, A.boxes, A.nitems, A.zlen);
  }

  if (WS) {
    // every copy the producer issued has been waited for by the consumers,
    // unless a wait gave up: then latch the error and drain (bounded) the
    // last phase issued on each ring slot
    __syncthreads();
    if (s_abort) {
      if (tid == TXY) {
        atomicCAS(A.err, 0, DERR_TIMEOUT);
        const int n = s_issued;
        for (int u = n > RPSI ? n - RPSI : 0; u < n; ++u)
          mbar_wait(smem_u32(&bars[u % RPSI]), (unsigned)((u / RPSI) & 1));
      }
      __syncthreads();
    }
    return;
  }
  if (aborted) {
    // latch the error and drain every copy still in flight (bounded)
    if (tid == 0) {
      atomicCAS(A.err, 0, DERR_TIMEOUT);
      for (int u = t; u < issued; ++u) mbar_wait(smem_u32(&bars[u % RPSI]), (unsigned)((u / RPSI) & 1));
    }
    __syncthreads();
    return;
  }

  if (DIAG && (A.epart != nullptr || A.tagcount != nullptr)) {
    // fixed-order block reduction: warp shuffles, then thread 0 over warps
    constexpr int NW = TXY / 32;
    __shared__ double red[4][NW];
    __shared__ unsigned long long redt[NW];
    double v0 = (double)i_kin - (double)c_kin, v1 = (double)i_grad - (double)c_grad,
           v2 = (double)i_pot - (double)c_pot_, v3 = (double)n_pierced;
    unsigned long long vt = (unsigned long long)n_tagged;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, o);
      v1 += __shfl_down_sync(0xffffffffu, v1, o);
      v2 += __shfl_down_sync(0xffffffffu, v2, o);
      v3 += __shfl_down_sync(0xffffffffu, v3, o);
      vt += __shfl_down_sync(0xffffffffu, vt, o);
    }
    const int wid = tid >> 5, lane = tid & 31;
    if (lane == 0) {
      red[0][wid] = v0;
      red[1][wid] = v1;
      red[2][wid] = v2;
      red[3][wid] = v3;
      redt[wid] = vt;
    }
    __syncthreads();
    if (tid == 0) {
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      unsigned long long at = 0;
      for (int w = 0; w < NW; ++w) {
        a0 += red[0][w];
        a1 += red[1][w];
        a2 += red[2][w];
        a3 += red[3][w];
        at += redt[w];
      }
      if (A.epart != nullptr) {
        A.epart[blockIdx.x * 4 + 0] = a0;
        A.epart[blockIdx.x * 4 + 1] = a1;
        A.epart[blockIdx.x * 4 + 2] = a2;
        A.epart[blockIdx.x * 4 + 3] = a3;
      }
      if (A.tagcount != nullptr && at) atomicAdd(A.tagcount, at);
    }
  }
}

// ---------------------------------------------------------------------------
// launch templates (the tensor maps come from build_tmaps in stage.cu)

template <typename T, int G, int TX, int TY, int P, bool DIAG, bool RKN>
static slh_status launch_v(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used) {
  using GE = Geo<T, G, TX, TY, P, DIAG>;
  if (DIAG && s.stage >= 2) return fail(SLH_ERR_INVALID_ARG, "diagnostics variant launched for stage %d", s.stage);
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(stage_kernel<T, G, TX, TY, P, DIAG, RKN>, cudaFuncAttributeMaxDynamicSharedMemorySize, GE::SMEM);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, stage_kernel<T, G, TX, TY, P, DIAG, RKN>, GE::NTHREADS, GE::SMEM);
    occ = o > 0 ? o : 1;
  }
  CUtensorMap* maps = nullptr;
  slh_status st = build_tmaps(c, L, G, TX, TY, &maps);
  if (st != SLH_OK) return st;
  if (s.dry) return SLH_OK;   // preparation only (before stream capture)
  const Tile& tile = DIAG ? L.dtile : L.tile;
  StageArgs<T> A;
  A.boxes = L.d_boxes;
  A.items = tile.d_items;
  A.nitems = tile.nitems;
  A.zlen = tile.zlen;
  A.gl = c->g;
  A.tmaps = maps;
  A.in_buf = s.in_buf;
  A.yn_buf = s.yn_buf;
  A.d_buf = s.d_buf;
  A.out_buf = s.out_buf;
  A.c_buf = s.c_buf;
  for (int k = 0; k < SLH_NBUF; ++k) A.bufs[k] = static_cast<T*>(L.buf[k]);
  A.stage = s.stage;
  A.eta_start = c->d_time + 2 * s.lev + (s.cur_eta ? 0 : 1);
  A.c_stage = s.c_stage;
  A.lambda = p.lambda;
  A.a = p.a;
  A.friction = p.friction;
  A.eta_power = p.eta_power;
  A.inv_dx2 = 1.0 / (L.dx * L.dx);
  A.ha = s.ha;
  A.ssp = s.ssp;
  A.sa = s.sa;
  A.sb = s.sb;
  A.hc = s.hc;
  A.hd = s.hd;
  A.he = s.he;
  A.rkn5 = s.rkn5;
  for (int q = 0; q < 9; ++q) A.rq[q] = s.rq[q];
  A.hb = s.hb;
  A.tags = s.tags;
  A.epart = s.epart;
  A.tagcount = s.tagcount;
  A.covered = s.covered;
  A.cov_shift = s.cov_shift;
  A.cov_nb = s.cov_nb;
  A.err = c->d_err;
  int grid = occ * c->num_sms;
  if (grid > tile.nitems) grid = tile.nitems;
  if (grid < 1) grid = 1;
  if (s.epart != nullptr && grid > L.epart_cap) grid = L.epart_cap;
  if (ctas_used) *ctas_used = grid;
  if (tile.nitems == 0) return SLH_OK;
  stage_kernel<T, G, TX, TY, P, DIAG, RKN><<<grid, GE::NTHREADS, GE::SMEM, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

template <typename T, int TX, int TY, int P, bool DIAG, bool RKN>
static slh_status by_order(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* u) {
  switch (p.lap_order) {
    case 2: return launch_v<T, 1, TX, TY, P, DIAG, RKN>(c, L, p, s, u);
    case 4: return launch_v<T, 2, TX, TY, P, DIAG, RKN>(c, L, p, s, u);
    case 6: return launch_v<T, 3, TX, TY, P, DIAG, RKN>(c, L, p, s, u);
    default: return fail(SLH_ERR_INVALID_ARG, "lap_order must be 2, 4 or 6 (got %d)", p.lap_order);
  }
}

template <bool DIAG, bool RKN>
static slh_status launch_tile(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* u) {
  const TileVariant& v = DIAG ? L.dtile.v : L.tile.v;
  if (c->prec == SLH_F64) {
    if (v.tx == 32 && v.ty == 8 && v.p == 2) return by_order<double, 32, 8, 2, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 32 && v.ty == 4 && v.p == 3) return by_order<double, 32, 4, 3, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 16 && v.ty == 8 && v.p == 2) return by_order<double, 16, 8, 2, DIAG, RKN>(c, L, p, s, u);
  } else {
    if (v.tx == 32 && v.ty == 16 && v.p == 2) return by_order<float, 32, 16, 2, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 32 && v.ty == 8 && v.p == 3) return by_order<float, 32, 8, 3, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 32 && v.ty == 16 && v.p == 3) return by_order<float, 32, 16, 3, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 16 && v.ty == 16 && v.p == 2) return by_order<float, 16, 16, 2, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 64 && v.ty == 8 && v.p == 2) return by_order<float, 64, 8, 2, DIAG, RKN>(c, L, p, s, u);
    if (v.tx == 128 && v.ty == 4 && v.p == 2) return by_order<float, 128, 4, 2, DIAG, RKN>(c, L, p, s, u);
  }
  return fail(SLH_ERR_STATE, "no stage kernel for tile %dx%d depth %d", v.tx, v.ty, v.p);
}

}  // namespace slh
