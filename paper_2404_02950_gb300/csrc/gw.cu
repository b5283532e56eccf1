// Gravitational-wave tensor stage kernel (Sec. 5).  With 16 fields per cell
// the state carries, besides psi and Pi, six tensor components u_ij (ij =
// xx, yy, zz, xy, xz, yz) and their conformal-time derivatives v_ij, evolved
// by the string-network form of Eq. GWEOM in conformal time:
//   u_ij' = v_ij
//   v_ij' = -c_fric v_ij + lap u_ij + 2 (d_i psi1 d_j psi1 + d_i psi2 d_j psi2)
// with the same Laplacian as the scalar field and central first differences
// of the same accuracy for the source (App. A).  One launch per RK4 stage,
// after the scalar stage kernel and with the same buffer roles, so that the
// two together advance all 16 fields by classic RK4.
//
// Work decomposition: one CTA of COL_TX x COL_TY threads per (box, x0, y0, z0)
// item, each thread a cell column marching up to COL_ZLEN planes in z.  The
// stencil operands are plain global loads: x and y neighbours come from the
// lines the CTA's own rows bring into L1, z neighbours from planes read a few
// iterations earlier (L1/L2), so DRAM sees each value about once.
#include <cuda.h>
#include <cuda_bf16.h>

#include "slh_internal.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace slh {

template <typename T>
struct GwArgs {
  const BoxDev* boxes;
  const int4* items;
  int gl;
  const T* in;              // stage input (psi and u ghosts filled)
  const T* yn;              // y_n
  T* d;                     // increment accumulator
  T* out;                   // next stage input, or y_{n+1} at stage 4
  T* cc;                    // Kahan compensation (stage 4, FP32 form) or null
  int stage;                // 1..4 (classic RK4) or 1..3 (SSPRK3)
  int ssp;                  // 1: low-storage SSPRK3 combine sa y_n + sb (Y + ha k)
  double sa, sb;
  const double* eta_start;  // device eta at the start of the step
  double c_stage;           // c_s * dt
  int friction;
  double inv_dx, inv_dx2;
  double ha, hb;            // a_{s+1} dt, b_s dt
  const CUtensorMap* tmaps; // TMA form: [box][buffer] maps of the 16-field view
  int in_buf;               // TMA form: physical index of the stage input buffer
  int* err;
  int rkn;                  // 1: RKN4 stage, coefficients ha, hb, hc, hd, he (as the scalar stage)
  double hc, hd, he;
};

// (i, j) direction pairs of the six tensor components
__device__ __forceinline__ constexpr int pair_i(int k) { return k < 3 ? k : (k == 5 ? 1 : 0); }
__device__ __forceinline__ constexpr int pair_j(int k) { return k < 3 ? k : (k == 3 ? 1 : 2); }

template <typename T, int G>
__global__ void __launch_bounds__(COL_TX * COL_TY, sizeof(T) == 4 ? 4 : 3) gw_stage_kernel(const GwArgs<T> A) {
  const int4 it = A.items[blockIdx.x];
  const BoxDev B = A.boxes[it.x];
  const int x = it.y + threadIdx.x, y = it.z + threadIdx.y;
  if (x >= B.n[0] || y >= B.n[1]) return;
  const int z1 = min(it.w + COL_ZLEN, B.n[2]);
  const double eta = *A.eta_start + A.c_stage;
  const T c_fric = (T)(A.friction ? 2.0 / eta : 0.0);
  const T ha = (T)A.ha, hb = (T)A.hb, idx = (T)A.inv_dx, idx2 = (T)A.inv_dx2;
  const long long sy = B.pitch, sz = (long long)B.pitch * B.pny, cs = B.cs;
  const long long st[3] = {1, sy, sz};
  // the buffers of one launch never overlap: every pointer is restricted so
  // that the loads of later components may be issued before earlier stores
  const T* __restrict__ in = A.in;
  const T* __restrict__ yn = A.yn;
  T* __restrict__ dd = A.d;
  T* __restrict__ out = A.out;
  T* __restrict__ cc = A.cc;
  const int stage = A.stage;
  const bool ssp = A.ssp != 0;
  const T sa = (T)A.sa, sb = (T)A.sb;
  long long e = B.off + ((long long)(it.w + A.gl) * B.pny + (y + A.gl)) * B.pitch + x + XPAD;
#pragma unroll 1
  for (int z = it.w; z < z1; ++z, e += sz) {
    // gradients of psi1, psi2: all 12 G operands loaded first
    T n1[3][2 * G], n2[3][2 * G];
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int m = 1; m <= G; ++m) {
        const long long o = m * st[dir];
        n1[dir][2 * m - 2] = __ldg(in + e + o);
        n1[dir][2 * m - 1] = __ldg(in + e - o);
        n2[dir][2 * m - 2] = __ldg(in + e + cs + o);
        n2[dir][2 * m - 1] = __ldg(in + e + cs - o);
      }
    T g1[3], g2[3];
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      T a1 = 0, a2 = 0;
#pragma unroll
      for (int m = 1; m <= G; ++m) {
        const T w = (T)grad_w<G>(m);
        a1 += w * (n1[dir][2 * m - 2] - n1[dir][2 * m - 1]);
        a2 += w * (n2[dir][2 * m - 2] - n2[dir][2 * m - 1]);
      }
      g1[dir] = a1 * idx;
      g2[dir] = a2 * idx;
    }
    // one component at a time for the 7-point stencil (unrolled, its loads
    // would all be hoisted and overflow the register budget)
#pragma unroll (G == 1 ? 1 : 6)
    for (int k = 0; k < 6; ++k) {
      const long long eu = e + (GW_U0 + k) * cs, ev = e + (GW_V0 + k) * cs;
      const T* f = in + eu;
      // operands of this component
      T nb[3][2 * G];
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          nb[dir][2 * m - 2] = __ldg(f + m * st[dir]);
          nb[dir][2 * m - 1] = __ldg(f - m * st[dir]);
        }
      const T u0 = __ldg(f);
      const T v = __ldg(in + ev);
      T yu = 0, yv = 0, du = 0, dv = 0, cu = 0, cv = 0;
      if (stage >= 2) {
        yu = __ldg(yn + eu);
        yv = __ldg(yn + ev);
        if (!ssp) {
          du = dd[eu];
          dv = dd[ev];
        }
      }
      if (stage == 4 && cc != nullptr) {
        cu = cc[eu];
        cv = cc[ev];
      }
      T lap;
      if (sizeof(T) == 8) {
        // textbook form, as the scalar FP64 stage
        T a = (T)(3.0 * lap_w<G>(0)) * u0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)lap_w<G>(m);
          a += w * (((nb[0][2 * m - 2] + nb[0][2 * m - 1]) + (nb[1][2 * m - 2] + nb[1][2 * m - 1])) +
                    (nb[2][2 * m - 2] + nb[2][2 * m - 1]));
        }
        lap = a * idx2;
      } else {
        // difference form, as the scalar FP32 stage
        T a = 0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)lap_w<G>(m);
          a += w * ((((nb[0][2 * m - 2] - u0) + (nb[0][2 * m - 1] - u0)) +
                     ((nb[1][2 * m - 2] - u0) + (nb[1][2 * m - 1] - u0))) +
                    ((nb[2][2 * m - 2] - u0) + (nb[2][2 * m - 1] - u0)));
        }
        lap = a * idx2;
      }
      const int i = pair_i(k), j = pair_j(k);
      const T g1i = i == 0 ? g1[0] : (i == 1 ? g1[1] : g1[2]), g1j = j == 0 ? g1[0] : (j == 1 ? g1[1] : g1[2]);
      const T g2i = i == 0 ? g2[0] : (i == 1 ? g2[1] : g2[2]), g2j = j == 0 ? g2[0] : (j == 1 ? g2[1] : g2[2]);
      const T src = (T)2 * (g1i * g1j + g2i * g2j);
      const T ku = v;
      const T kv = ((-c_fric) * v + lap) + src;
      if (ssp) {
        const T fu = u0 + ha * ku, fv = v + ha * kv;
        if (stage == 1) {
          out[eu] = fu;
          out[ev] = fv;
        } else {
          out[eu] = sa * yu + sb * fu;
          out[ev] = sa * yv + sb * fv;
        }
      } else if (A.rkn) {
        // RKN4 with positions u, velocities v (see the scalar stage kernel)
        const T hc = (T)A.hc, hd = (T)A.hd, he = (T)A.he;
        if (stage == 1) {
          out[eu] = u0 + ha * v + hb * kv;
          out[ev] = v + hc * kv;
          dd[eu] = hd * kv;
          dd[ev] = he * kv;
        } else if (stage <= 3) {
          if (stage == 3) out[eu] = yu + ha * yv + hb * kv;
          out[ev] = yv + hc * kv;
          dd[eu] = du + hd * kv;
          dd[ev] = dv + he * kv;
        } else {
          const T iu = ha * yv + du, iv = dv + he * kv;
          if (cc != nullptr) {
            T w, sm;
            w = iu - cu; sm = yu + w; cc[eu] = (sm - yu) - w; out[eu] = sm;
            w = iv - cv; sm = yv + w; cc[ev] = (sm - yv) - w; out[ev] = sm;
          } else {
            out[eu] = yu + iu;
            out[ev] = yv + iv;
          }
        }
      } else if (stage == 1) {
        out[eu] = u0 + ha * ku;
        out[ev] = v + ha * kv;
        dd[eu] = hb * ku;
        dd[ev] = hb * kv;
      } else if (stage == 2 || stage == 3) {
        out[eu] = yu + ha * ku;
        out[ev] = yv + ha * kv;
        dd[eu] = du + hb * ku;
        dd[ev] = dv + hb * kv;
      } else {
        const T iu = du + hb * ku, iv = dv + hb * kv;
        if (cc != nullptr) {
          // compensated sum y + inc, the rounding error carried in C
          T w, sm;
          w = iu - cu; sm = yu + w; cc[eu] = (sm - yu) - w; out[eu] = sm;
          w = iv - cv; sm = yv + w; cc[ev] = (sm - yv) - w; out[ev] = sm;
        } else {
          out[eu] = yu + iu;
          out[ev] = yv + iv;
        }
      }
    }
  }
}

// BF16 storage (SLH_F32_BF16): the SSPRK3 stage of the tensor fields with
// u_ij and v_ij held as BF16 pairs, (u_xx, u_yy), (u_zz, u_xy), (u_xz, u_yz)
// in slots SLOT_U0 .. SLOT_U0 + 2 and the v_ij likewise from SLOT_V0, the
// first field of a pair in the low half.  Every value is widened to FP32
// (exactly), the stage is computed and combined in FP32 as in
// gw_stage_kernel, and the results are rounded to BF16 (to nearest even)
// once, when stored.  Same items and threads as gw_stage_kernel.
__device__ __forceinline__ float bf_lo(float w) { return __uint_as_float(__float_as_uint(w) << 16); }
__device__ __forceinline__ float bf_hi(float w) { return __uint_as_float(__float_as_uint(w) & 0xFFFF0000u); }
__device__ __forceinline__ float bf_pack(float lo, float hi) {
  return __uint_as_float((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
                         ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16));
}

template <int G>
__global__ void __launch_bounds__(COL_TX * COL_TY, 4) gw_bf16_kernel(const GwArgs<float> A) {
  using T = float;
  const int4 it = A.items[blockIdx.x];
  const BoxDev B = A.boxes[it.x];
  const int x = it.y + threadIdx.x, y = it.z + threadIdx.y;
  if (x >= B.n[0] || y >= B.n[1]) return;
  const int z1 = min(it.w + COL_ZLEN, B.n[2]);
  const double eta = *A.eta_start + A.c_stage;
  const T c_fric = (T)(A.friction ? 2.0 / eta : 0.0);
  const T ha = (T)A.ha, idx = (T)A.inv_dx, idx2 = (T)A.inv_dx2;
  const long long sy = B.pitch, sz = (long long)B.pitch * B.pny, cs = B.cs;
  const long long st[3] = {1, sy, sz};
  const T* __restrict__ in = A.in;
  const T* __restrict__ yn = A.yn;
  T* __restrict__ out = A.out;
  const int stage = A.stage;
  const T sa = (T)A.sa, sb = (T)A.sb;
  long long e = B.off + ((long long)(it.w + A.gl) * B.pny + (y + A.gl)) * B.pitch + x + XPAD;
  // psi1, psi2 on planes z-G .. z+G of the column, rolled one plane per step
  // (the z differences of the gradients come from registers)
  T w1[2 * G + 1], w2[2 * G + 1];
#pragma unroll
  for (int k = 0; k < 2 * G; ++k) {
    w1[k] = __ldg(in + e + (k - G) * sz);
    w2[k] = __ldg(in + e + cs + (k - G) * sz);
  }
#pragma unroll 1
  for (int z = it.w; z < z1; ++z, e += sz) {
    w1[2 * G] = __ldg(in + e + G * sz);
    w2[2 * G] = __ldg(in + e + cs + G * sz);
    // gradients of psi1, psi2 (FP32 slots 0 and 1)
    T g1[3], g2[3];
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      T a1 = 0, a2 = 0;
#pragma unroll
      for (int m = 1; m <= G; ++m) {
        const long long o = m * st[dir];
        const T w = (T)grad_w<G>(m);
        a1 += w * (__ldg(in + e + o) - __ldg(in + e - o));
        a2 += w * (__ldg(in + e + cs + o) - __ldg(in + e + cs - o));
      }
      g1[dir] = a1 * idx;
      g2[dir] = a2 * idx;
    }
    {
      T a1 = 0, a2 = 0;
#pragma unroll
      for (int m = 1; m <= G; ++m) {
        const T w = (T)grad_w<G>(m);
        a1 += w * (w1[G + m] - w1[G - m]);
        a2 += w * (w2[G + m] - w2[G - m]);
      }
      g1[2] = a1 * idx;
      g2[2] = a2 * idx;
    }
#pragma unroll
    for (int k = 0; k < 2 * G; ++k) {
      w1[k] = w1[k + 1];
      w2[k] = w2[k + 1];
    }
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
      const long long eu = e + (SLOT_U0 + q) * cs, ev = e + (SLOT_V0 + q) * cs;
      const T* f = in + eu;
      const T uc = __ldg(f);
      const T u0[2] = {bf_lo(uc), bf_hi(uc)};
      T acc[2] = {(T)(3.0 * lap_w<G>(0)) * u0[0], (T)(3.0 * lap_w<G>(0)) * u0[1]};
#pragma unroll
      for (int m = 1; m <= G; ++m) {
        const T w = (T)lap_w<G>(m);
        T sm[2] = {0, 0};
#pragma unroll
        for (int dir = 0; dir < 3; ++dir) {
          const T pv = __ldg(f + m * st[dir]), mv = __ldg(f - m * st[dir]);
          sm[0] += bf_lo(pv) + bf_lo(mv);
          sm[1] += bf_hi(pv) + bf_hi(mv);
        }
        acc[0] += w * sm[0];
        acc[1] += w * sm[1];
      }
      const T vc = __ldg(in + ev);
      const T v[2] = {bf_lo(vc), bf_hi(vc)};
      T yu[2] = {0, 0}, yv[2] = {0, 0};
      if (stage >= 2) {
        const T a = __ldg(yn + eu), b = __ldg(yn + ev);
        yu[0] = bf_lo(a);
        yu[1] = bf_hi(a);
        yv[0] = bf_lo(b);
        yv[1] = bf_hi(b);
      }
      T ou[2], ov[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * q + h, i = pair_i(k), j = pair_j(k);
        const T g1i = i == 0 ? g1[0] : (i == 1 ? g1[1] : g1[2]), g1j = j == 0 ? g1[0] : (j == 1 ? g1[1] : g1[2]);
        const T g2i = i == 0 ? g2[0] : (i == 1 ? g2[1] : g2[2]), g2j = j == 0 ? g2[0] : (j == 1 ? g2[1] : g2[2]);
        const T src = (T)2 * (g1i * g1j + g2i * g2j);
        const T kv = ((-c_fric) * v[h] + acc[h] * idx2) + src;
        const T fu = u0[h] + ha * v[h], fv = v[h] + ha * kv;
        ou[h] = stage == 1 ? fu : sa * yu[h] + sb * fu;
        ov[h] = stage == 1 ? fv : sa * yv[h] + sb * fv;
      }
      out[eu] = bf_pack(ou[0], ou[1]);
      out[ev] = bf_pack(ov[0], ov[1]);
    }
  }
}

// TMA-fed form (FP32, Laplacian radius G <= 2).  The same items, threads and
// arithmetic as gw_stage_kernel, but the stencil operands -- psi1, psi2 and
// the six u_ij of every plane of the column with its x/y halo -- stream into
// a shared-memory ring of 2G+1+P planes by tensor copies (four 2-component
// boxes of (32+8) x (8+2G) cells per plane, 16-byte aligned in x), issued P
// planes ahead by one thread and tracked by mbarrier transaction counts.
// Only the pointwise operands (v_ij of the input, y_n, D, C) are read from
// global memory, coalesced, each value once.  Every wait is bounded; on
// expiry the CTA latches DERR_TIMEOUT, drains its copies (bounded) and leaves.
constexpr int GWT_P = 2;

template <int G>
struct GwTmaGeo {
  static constexpr int SXL = COL_TX + 8;        // x halo of 4 cells each side (G <= 4)
  static constexpr int SY = COL_TY + 2 * G;
  static constexpr int RU = 2 * G + 1 + GWT_P;  // ring planes
  static constexpr int PLANE = SY * SXL;        // floats of one component plane
  static constexpr int PAIR = 2 * PLANE;        // one tensor copy (2 components)
  static constexpr int SLOT = 4 * PAIR;         // psi pair + three u pairs
  static constexpr int BAR_BYTES = 128;
  static constexpr int SMEM = BAR_BYTES + RU * SLOT * 4;
  static_assert((PAIR * 4) % 128 == 0, "tensor copy destinations must stay 128-byte aligned");
};

template <int G>
__global__ void __launch_bounds__(COL_TX * COL_TY, 2) gw_tma_kernel(const GwArgs<float> A) {
  using GE = GwTmaGeo<G>;
  using T = float;
  constexpr int SXL = GE::SXL, PLANE = GE::PLANE, RU = GE::RU;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);
  T* ring = reinterpret_cast<T*>(smem + GE::BAR_BYTES);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * COL_TX + tx;
  const int4 it = A.items[blockIdx.x];
  const BoxDev B = A.boxes[it.x];
  const int x = it.y + tx, y = it.z + ty;
  const bool active = x < B.n[0] && y < B.n[1];
  const int z0 = it.w, z1 = min(it.w + COL_ZLEN, B.n[2]);
  const int nplanes = (z1 - z0) + 2 * G;
  const CUtensorMap* map = A.tmaps + (size_t)it.x * SLH_NBUF + A.in_buf;

  if (tid == 0) {
    for (int i = 0; i < RU; ++i) mbar_init(smem_u32(&bars[i]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  // plane z0 - G + t of the input into slot t % RU (one thread)
  auto issue = [&](int t) {
    const int slot = t % RU;
    const unsigned bar = smem_u32(&bars[slot]);
    mbar_expect_tx(bar, (unsigned)(GE::SLOT * 4));
    T* dst = ring + slot * GE::SLOT;
    const int cy = it.z - G + A.gl, cz = z0 - G + t + A.gl;
    tma_load4(smem_u32(dst), map, it.y, cy, cz, 0, bar);
    tma_load4(smem_u32(dst + GE::PAIR), map, it.y, cy, cz, GW_U0, bar);
    tma_load4(smem_u32(dst + 2 * GE::PAIR), map, it.y, cy, cz, GW_U0 + 2, bar);
    tma_load4(smem_u32(dst + 3 * GE::PAIR), map, it.y, cy, cz, GW_U0 + 4, bar);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < GWT_P && issued < nplanes; ++issued) issue(issued);

  const double eta = *A.eta_start + A.c_stage;
  const T c_fric = (T)(A.friction ? 2.0 / eta : 0.0);
  const T ha = (T)A.ha, hb = (T)A.hb, idx = (T)A.inv_dx, idx2 = (T)A.inv_dx2;
  const long long cs = B.cs, sz = (long long)B.pitch * B.pny;
  const T* __restrict__ in = A.in;
  const T* __restrict__ yn = A.yn;
  T* __restrict__ dd = A.d;
  T* __restrict__ out = A.out;
  T* __restrict__ cc = A.cc;
  const int stage = A.stage;
  const bool ssp = A.ssp != 0;
  const T sa = (T)A.sa, sb = (T)A.sb;
  const int cell = (ty + G) * SXL + 4 + tx;   // this thread's cell in a component plane
  long long e = B.off + ((long long)(z0 + A.gl) * B.pny + (y + A.gl)) * B.pitch + x + XPAD;

  int t = 0;
  bool aborted = false;
  for (; t < nplanes; ++t) {
    if (tid == 0 && issued < nplanes) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
    const bool ok = mbar_wait(smem_u32(&bars[t % RU]), (unsigned)((t / RU) & 1));
    const int z = z0 - 2 * G + t;
    if (ok && active && z >= z0) {
      // ring slots of planes z-G .. z+G
      int sb_[2 * G + 1];
#pragma unroll
      for (int k = 0; k <= 2 * G; ++k) sb_[k] = ((t - 2 * G + k) % RU) * GE::SLOT + cell;
      auto S = [&](int comp, int dx, int dy, int dz) -> T { return ring[sb_[dz + G] + comp * PLANE + dy * SXL + dx]; };
      // pointwise operands of the six components, all issued first
      T v[6], yu[6], yv[6], du[6], dv[6], cu[6], cv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const long long eu = e + (GW_U0 + k) * cs, ev = e + (GW_V0 + k) * cs;
        v[k] = __ldg(in + ev);
        yu[k] = yv[k] = du[k] = dv[k] = cu[k] = cv[k] = 0;
        if (stage >= 2) {
          yu[k] = __ldg(yn + eu);
          yv[k] = __ldg(yn + ev);
          if (!ssp) {
            du[k] = dd[eu];
            dv[k] = dd[ev];
          }
        }
        if (stage == 4 && cc != nullptr) {
          cu[k] = cc[eu];
          cv[k] = cc[ev];
        }
      }
      // gradients of psi1, psi2
      T g1[3], g2[3];
#pragma unroll
      for (int dir = 0; dir < 3; ++dir) {
        T a1 = 0, a2 = 0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)grad_w<G>(m);
          const int dx = dir == 0 ? m : 0, dy = dir == 1 ? m : 0, dz = dir == 2 ? m : 0;
          a1 += w * (S(0, dx, dy, dz) - S(0, -dx, -dy, -dz));
          a2 += w * (S(1, dx, dy, dz) - S(1, -dx, -dy, -dz));
        }
        g1[dir] = a1 * idx;
        g2[dir] = a2 * idx;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const long long eu = e + (GW_U0 + k) * cs, ev = e + (GW_V0 + k) * cs;
        const int c = 2 + k;
        const T u0 = S(c, 0, 0, 0);
        // difference form, as the scalar FP32 stage
        T a = 0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
          const T w = (T)lap_w<G>(m);
          a += w * ((((S(c, m, 0, 0) - u0) + (S(c, -m, 0, 0) - u0)) + ((S(c, 0, m, 0) - u0) + (S(c, 0, -m, 0) - u0))) +
                    ((S(c, 0, 0, m) - u0) + (S(c, 0, 0, -m) - u0)));
        }
        const T lap = a * idx2;
        const int i = pair_i(k), j = pair_j(k);
        const T g1i = i == 0 ? g1[0] : (i == 1 ? g1[1] : g1[2]), g1j = j == 0 ? g1[0] : (j == 1 ? g1[1] : g1[2]);
        const T g2i = i == 0 ? g2[0] : (i == 1 ? g2[1] : g2[2]), g2j = j == 0 ? g2[0] : (j == 1 ? g2[1] : g2[2]);
        const T src = (T)2 * (g1i * g1j + g2i * g2j);
        const T ku = v[k];
        const T kv = ((-c_fric) * v[k] + lap) + src;
        if (ssp) {
          const T fu = u0 + ha * ku, fv = v[k] + ha * kv;
          if (stage == 1) {
            out[eu] = fu;
            out[ev] = fv;
          } else {
            out[eu] = sa * yu[k] + sb * fu;
            out[ev] = sa * yv[k] + sb * fv;
          }
        } else if (A.rkn) {
          // RKN4 with positions u, velocities v (see the scalar stage kernel)
          const T hc = (T)A.hc, hd = (T)A.hd, he = (T)A.he;
          if (stage == 1) {
            out[eu] = u0 + ha * v[k] + hb * kv;
            out[ev] = v[k] + hc * kv;
            dd[eu] = hd * kv;
            dd[ev] = he * kv;
          } else if (stage <= 3) {
            if (stage == 3) out[eu] = yu[k] + ha * yv[k] + hb * kv;
            out[ev] = yv[k] + hc * kv;
            dd[eu] = du[k] + hd * kv;
            dd[ev] = dv[k] + he * kv;
          } else {
            const T iu = ha * yv[k] + du[k], iv = dv[k] + he * kv;
            if (cc != nullptr) {
              T w, sm;
              w = iu - cu[k]; sm = yu[k] + w; cc[eu] = (sm - yu[k]) - w; out[eu] = sm;
              w = iv - cv[k]; sm = yv[k] + w; cc[ev] = (sm - yv[k]) - w; out[ev] = sm;
            } else {
              out[eu] = yu[k] + iu;
              out[ev] = yv[k] + iv;
            }
          }
        } else if (stage == 1) {
          out[eu] = u0 + ha * ku;
          out[ev] = v[k] + ha * kv;
          dd[eu] = hb * ku;
          dd[ev] = hb * kv;
        } else if (stage == 2 || stage == 3) {
          out[eu] = yu[k] + ha * ku;
          out[ev] = yv[k] + ha * kv;
          dd[eu] = du[k] + hb * ku;
          dd[ev] = dv[k] + hb * kv;
        } else {
          const T iu = du[k] + hb * ku, iv = dv[k] + hb * kv;
          if (cc != nullptr) {
            // compensated sum y + inc, the rounding error carried in C
            T w, sm;
            w = iu - cu[k]; sm = yu[k] + w; cc[eu] = (sm - yu[k]) - w; out[eu] = sm;
            w = iv - cv[k]; sm = yv[k] + w; cc[ev] = (sm - yv[k]) - w; out[ev] = sm;
          } else {
            out[eu] = yu[k] + iu;
            out[ev] = yv[k] + iv;
          }
        }
      }
    }
    if (z >= z0) e += sz;
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
  }
  if (aborted) {
    // latch the error and drain every copy still in flight (bounded)
    if (tid == 0) {
      atomicCAS(A.err, 0, DERR_TIMEOUT);
      for (int u = t; u < issued; ++u) mbar_wait(smem_u32(&bars[u % RU]), (unsigned)((u / RU) & 1));
    }
    __syncthreads();
  }
}

template <int G>
static slh_status gw_tma_launch(slh_ctx* c, Level& L, const StageLaunch& s, GwArgs<float>& A) {
  CUtensorMap* maps = nullptr;
  slh_status st = build_gw_tmaps(c, L, G, COL_TX, COL_TY, &maps);
  if (st != SLH_OK) return st;
  static bool attr = false;
  if (!attr) {
    SLH_CUDA(cudaFuncSetAttribute(gw_tma_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, GwTmaGeo<G>::SMEM));
    attr = true;
  }
  if (s.dry) return SLH_OK;   // preparation only (before stream capture)
  A.tmaps = maps;
  A.in_buf = s.in_buf;
  gw_tma_kernel<G><<<L.ncol_items, dim3(COL_TX, COL_TY), GwTmaGeo<G>::SMEM, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

template <typename T>
static slh_status gw_stage_t(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s) {
  if (L.ncol_items == 0) return SLH_OK;
  GwArgs<T> A;
  A.boxes = L.d_boxes;
  A.items = L.d_col_items;
  A.gl = c->g;
  A.in = static_cast<const T*>(L.buf[s.in_buf]);
  A.yn = static_cast<const T*>(L.buf[s.yn_buf]);
  A.d = static_cast<T*>(L.buf[s.d_buf]);
  A.out = static_cast<T*>(L.buf[s.out_buf]);
  A.cc = s.c_buf >= 0 ? static_cast<T*>(L.buf[s.c_buf]) : nullptr;
  A.stage = s.stage;
  A.eta_start = c->d_time + 2 * s.lev + 1;
  A.c_stage = s.c_stage;
  A.friction = p.friction;
  A.inv_dx = 1.0 / L.dx;
  A.inv_dx2 = 1.0 / (L.dx * L.dx);
  A.ha = s.ha;
  A.hb = s.hb;
  A.ssp = s.ssp;
  A.sa = s.sa;
  A.sb = s.sb;
  A.rkn = s.rkn;
  A.hc = s.hc;
  A.hd = s.hd;
  A.he = s.he;
  A.tmaps = nullptr;
  A.in_buf = s.in_buf;
  A.err = c->d_err;
  if constexpr (sizeof(T) == 4) {
    if (c->prec == SLH_F32_BF16) {
      // BF16 tensor storage: SSPRK3 only (three level buffers)
      if (s.dry) return SLH_OK;
      if (!s.ssp) return fail(SLH_ERR_INVALID_ARG, "BF16 tensor storage runs SSPRK3 only");
      const dim3 block(COL_TX, COL_TY);
      switch (p.lap_order) {
        case 2: gw_bf16_kernel<1><<<L.ncol_items, block, 0, c->stream>>>(A); break;
        case 4: gw_bf16_kernel<2><<<L.ncol_items, block, 0, c->stream>>>(A); break;
        case 6: gw_bf16_kernel<3><<<L.ncol_items, block, 0, c->stream>>>(A); break;
        default: return fail(SLH_ERR_INVALID_ARG, "lap_order must be 2, 4 or 6 (got %d)", p.lap_order);
      }
      SLH_CUDA(cudaGetLastError());
      return SLH_OK;
    }
    // FP32, Laplacian radius <= 2: the TMA-fed form
    if (p.lap_order == 2) return gw_tma_launch<1>(c, L, s, A);
    if (p.lap_order == 4) return gw_tma_launch<2>(c, L, s, A);
  }
  if (s.dry) return SLH_OK;
  const dim3 block(COL_TX, COL_TY);
  switch (p.lap_order) {
    case 2: gw_stage_kernel<T, 1><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    case 4: gw_stage_kernel<T, 2><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    case 6: gw_stage_kernel<T, 3><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    default: return fail(SLH_ERR_INVALID_ARG, "lap_order must be 2, 4 or 6 (got %d)", p.lap_order);
  }
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_gw_stage(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s) {
  if (s.stage < 1 || s.stage > 4) return fail(SLH_ERR_INVALID_ARG, "gw stage %d outside 1..4", s.stage);
  return c->prec == SLH_F64 ? gw_stage_t<double>(c, L, p, s) : gw_stage_t<float>(c, L, p, s);
}

}  // namespace slh
