// Fused RK4 stage kernel: finite-difference Laplacian (App. A), right-hand
// side of the axion-string system (Sec. 3.1, Eqs. EOM1-EOM2), classic RK4
// stage combination (integrator type 4), and -- in stage 1 or the
// diagnostics-only pass -- the string-winding tags and energy partials of
// the stage input.
//
// Work decomposition: a persistent grid walks a list of (box, x0, y0, z0)
// tiles; each CTA marches along z through a TX x TY column tile, keeping a
// ring of 2G+2 halo'd psi1/psi2 planes in shared memory that cp.async
// streams from global memory one plane ahead.  Pointwise data (momenta, y_n,
// the increment accumulator, the Kahan compensation) is read straight from
// global memory into registers, coalesced along x.  Every value a cell needs
// is read once from HBM per stage (halo re-reads hit L2).
#include <stdio.h>

#include "slh_internal.cuh"

namespace slh {

template <typename T>
struct StageArgs {
  const BoxDev* boxes;
  const int4* items;
  int nitems;
  int zlen;
  int gl;                  // ghost layers of the level layout
  const T* yin;            // stage input Y_s
  const T* yn;             // y_n (stages 2..4)
  T* dacc;                 // increment accumulator
  T* yout;                 // Y_{s+1} or y_{n+1}
  T* comp;                 // Kahan compensation (stage 4, FP32) or null
  int stage;               // 0 = diagnostics only
  const double* eta_start; // device eta at the start of the step
  double c_stage;          // c_s * dt
  double lambda, a;
  int friction, eta_power;
  double inv_dx2;
  double ha, hb;
  uint8_t* tags;
  double* epart;
  unsigned long long* tagcount;
  const uint8_t* covered;
  int cov_shift, cov_nb;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Winding contribution of the edge a -> b: +1 when it leaves the upper half
// plane (Im >= 0) turning counter-clockwise, -1 when it enters it turning
// clockwise (the sign of X = Re a Im b - Im a Re b); products and the
// difference rounded separately in FP64 (exact sign for FP32 inputs).
__device__ __forceinline__ int edge_delta(double ar, double ai, double br, double bi) {
  const bool ua = ai >= 0.0, ub = bi >= 0.0;
  if (ua == ub) return 0;
  const double X = __dsub_rn(__dmul_rn(ar, bi), __dmul_rn(ai, br));
  if (ua) return X > 0.0 ? 1 : 0;
  return X < 0.0 ? -1 : 0;
}

// Central second-difference weights w_m, m = 1..G (the centre weight is
// -2 sum w_m and drops out of the difference form used below).
template <int G>
__device__ __forceinline__ double lap_w(int m);
template <>
__device__ __forceinline__ double lap_w<1>(int) { return 1.0; }
template <>
__device__ __forceinline__ double lap_w<2>(int m) { return m == 1 ? 4.0 / 3.0 : -1.0 / 12.0; }
template <>
__device__ __forceinline__ double lap_w<3>(int m) {
  return m == 1 ? 1.5 : (m == 2 ? -0.15 : 1.0 / 90.0);
}

template <typename T, int G, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) stage_kernel(const StageArgs<T> A) {
  constexpr int NT = TX * TY;
  constexpr int VEC = 16 / sizeof(T);
  constexpr int SXL = TX + 8;          // loaded row: valid x0-4 .. x0+TX+3
  constexpr int SY = TY + 2 * G;
  constexpr int R = 2 * G + 2;         // ring of planes
  constexpr int PLANE = SY * SXL;
  constexpr int CROW = SXL / VEC;
  constexpr int CHUNKS = 2 * SY * CROW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int gl = A.gl;

  const double eta = *A.eta_start + A.c_stage;
  const double cfd = A.friction ? 2.0 / eta : 0.0;
  const double cpd = A.eta_power == 2 ? A.lambda * (eta * eta) : A.lambda;
  const T c_fric = (T)cfd, c_pot = (T)cpd, a_c = (T)A.a;
  const T ha = (T)A.ha, hb = (T)A.hb, idx2 = (T)A.inv_dx2;
  const bool diag = (A.tags != nullptr) || (A.epart != nullptr);

  double s_kin = 0.0, s_grad = 0.0, s_pot = 0.0;
  unsigned long long n_pierced = 0, n_tagged = 0;

  for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    const int4 it = A.items[item];
    const BoxDev B = A.boxes[it.x];
    const int x0 = it.y, y0 = it.z, z0 = it.w;
    const int z1 = min(z0 + A.zlen, B.n[2]);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < B.n[0]) && (y < B.n[1]);
    const long long rowstride = B.pitch;
    const long long planestride = (long long)B.pny * B.pitch;
    T i_kin = 0, i_grad = 0, i_pot = 0;

    auto load_plane = [&](int zz) {
      const int slot = (zz - z0 + G) % R;
      T* dst = ring + slot * 2 * PLANE;
      const long long pz = zz + gl;
      for (int ch = tid; ch < CHUNKS; ch += NT) {
        const int comp = ch / (SY * CROW);
        const int rem = ch - comp * (SY * CROW);
        const int row = rem / CROW;
        const int cc = rem - row * CROW;
        const int py = y0 - G + row + gl;
        const int px = x0 + cc * VEC;
        if (py < B.pny && px < B.pitch) {
          const T* src = A.yin + B.off + comp * B.cs + pz * planestride + (long long)py * rowstride + px;
          cp_async16(dst + comp * PLANE + row * SXL + cc * VEC, src);
        }
      }
    };

    for (int j = 0; j < 2 * G + 1; ++j) {
      load_plane(z0 - G + j);
      cp_async_commit();
    }

    for (int z = z0; z < z1; ++z) {
      if (z + G + 1 <= z1 + G - 1) load_plane(z + G + 1);
      cp_async_commit();

      // pointwise operands of this cell (issued before the wait)
      const long long e0 = B.off + (long long)(z + gl) * planestride + (long long)(y + gl) * rowstride + x + XPAD;
      T P1 = 0, P2 = 0, yn0 = 0, yn1 = 0, yn2 = 0, yn3 = 0, d0 = 0, d1 = 0, d2 = 0, d3 = 0;
      T k0c = 0, k1c = 0, k2c = 0, k3c = 0;
      if (active) {
        P1 = A.yin[e0 + 2 * B.cs];
        P2 = A.yin[e0 + 3 * B.cs];
        if (A.stage >= 2) {
          yn0 = A.yn[e0];
          yn1 = A.yn[e0 + B.cs];
          yn2 = A.yn[e0 + 2 * B.cs];
          yn3 = A.yn[e0 + 3 * B.cs];
          d0 = A.dacc[e0];
          d1 = A.dacc[e0 + B.cs];
          d2 = A.dacc[e0 + 2 * B.cs];
          d3 = A.dacc[e0 + 3 * B.cs];
          if (A.stage == 4 && A.comp != nullptr) {
            k0c = A.comp[e0];
            k1c = A.comp[e0 + B.cs];
            k2c = A.comp[e0 + 2 * B.cs];
            k3c = A.comp[e0 + 3 * B.cs];
          }
        }
      }

      cp_async_wait<1>();
      __syncthreads();

      if (active) {
        auto S = [&](int c, int dx, int dy, int dz) -> T {
          const int slot = (z + dz - z0 + G) % R;
          return ring[(slot * 2 + c) * PLANE + (ty + G + dy) * SXL + 4 + tx + dx];
        };
        const T p1 = S(0, 0, 0, 0), p2 = S(1, 0, 0, 0);
        T l1 = 0, l2 = 0;
        {
          T sx1 = 0, sy1 = 0, sz1 = 0, sx2 = 0, sy2 = 0, sz2 = 0;
#pragma unroll
          for (int m = 1; m <= G; ++m) {
            const T w = (T)lap_w<G>(m);
            sx1 += w * ((S(0, m, 0, 0) - p1) + (S(0, -m, 0, 0) - p1));
            sy1 += w * ((S(0, 0, m, 0) - p1) + (S(0, 0, -m, 0) - p1));
            sz1 += w * ((S(0, 0, 0, m) - p1) + (S(0, 0, 0, -m) - p1));
            sx2 += w * ((S(1, m, 0, 0) - p2) + (S(1, -m, 0, 0) - p2));
            sy2 += w * ((S(1, 0, m, 0) - p2) + (S(1, 0, -m, 0) - p2));
            sz2 += w * ((S(1, 0, 0, m) - p2) + (S(1, 0, 0, -m) - p2));
          }
          l1 = ((sx1 + sy1) + sz1) * idx2;
          l2 = ((sx2 + sy2) + sz2) * idx2;
        }
        const T r2 = p1 * p1 + p2 * p2;
        const T pot = c_pot * (r2 - (T)1) + a_c;
        const T kP1 = (-c_fric) * P1 + l1 - p1 * pot;
        const T kP2 = (-c_fric) * P2 + l2 - p2 * pot;

        if (A.stage == 1) {
          A.yout[e0] = p1 + ha * P1;
          A.yout[e0 + B.cs] = p2 + ha * P2;
          A.yout[e0 + 2 * B.cs] = P1 + ha * kP1;
          A.yout[e0 + 3 * B.cs] = P2 + ha * kP2;
          A.dacc[e0] = hb * P1;
          A.dacc[e0 + B.cs] = hb * P2;
          A.dacc[e0 + 2 * B.cs] = hb * kP1;
          A.dacc[e0 + 3 * B.cs] = hb * kP2;
        } else if (A.stage == 2 || A.stage == 3) {
          A.yout[e0] = yn0 + ha * P1;
          A.yout[e0 + B.cs] = yn1 + ha * P2;
          A.yout[e0 + 2 * B.cs] = yn2 + ha * kP1;
          A.yout[e0 + 3 * B.cs] = yn3 + ha * kP2;
          A.dacc[e0] = d0 + hb * P1;
          A.dacc[e0 + B.cs] = d1 + hb * P2;
          A.dacc[e0 + 2 * B.cs] = d2 + hb * kP1;
          A.dacc[e0 + 3 * B.cs] = d3 + hb * kP2;
        } else if (A.stage == 4) {
          const T inc0 = d0 + hb * P1, inc1 = d1 + hb * P2;
          const T inc2 = d2 + hb * kP1, inc3 = d3 + hb * kP2;
          if (A.comp != nullptr) {
            // compensated sum y + inc carrying the rounding error in comp
            T v, t;
            v = inc0 - k0c; t = yn0 + v; A.comp[e0] = (t - yn0) - v; A.yout[e0] = t;
            v = inc1 - k1c; t = yn1 + v; A.comp[e0 + B.cs] = (t - yn1) - v; A.yout[e0 + B.cs] = t;
            v = inc2 - k2c; t = yn2 + v; A.comp[e0 + 2 * B.cs] = (t - yn2) - v; A.yout[e0 + 2 * B.cs] = t;
            v = inc3 - k3c; t = yn3 + v; A.comp[e0 + 3 * B.cs] = (t - yn3) - v; A.yout[e0 + 3 * B.cs] = t;
          } else {
            A.yout[e0] = yn0 + inc0;
            A.yout[e0 + B.cs] = yn1 + inc1;
            A.yout[e0 + 2 * B.cs] = yn2 + inc2;
            A.yout[e0 + 3 * B.cs] = yn3 + inc3;
          }
        }

        if (diag) {
          // plaquette windings around this cell (12 plaquettes, 3 owned)
          bool tagged = false;
          int owned = 0;
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            // (u, v) in-plane unit offsets: normal z: (x, y); x: (y, z); y: (z, x)
            const int ux = (w == 0) ? 1 : 0, uy = (w == 1) ? 1 : 0, uz = (w == 2) ? 1 : 0;
            const int vx = (w == 2) ? 1 : 0, vy = (w == 0) ? 1 : 0, vz = (w == 1) ? 1 : 0;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
#pragma unroll
              for (int b = 0; b < 2; ++b) {
                const int ox = -a * ux - b * vx, oy = -a * uy - b * vy, oz = -a * uz - b * vz;
                const double r0 = (double)S(0, ox, oy, oz), i0 = (double)S(1, ox, oy, oz);
                const double r1 = (double)S(0, ox + ux, oy + uy, oz + uz), i1 = (double)S(1, ox + ux, oy + uy, oz + uz);
                const double r2c = (double)S(0, ox + ux + vx, oy + uy + vy, oz + uz + vz),
                             i2c = (double)S(1, ox + ux + vx, oy + uy + vy, oz + uz + vz);
                const double r3 = (double)S(0, ox + vx, oy + vy, oz + vz), i3 = (double)S(1, ox + vx, oy + vy, oz + vz);
                const int Wn = edge_delta(r0, i0, r1, i1) + edge_delta(r1, i1, r2c, i2c) +
                               edge_delta(r2c, i2c, r3, i3) + edge_delta(r3, i3, r0, i0);
                if (Wn != 0) {
                  tagged = true;
                  if (a == 0 && b == 0) ++owned;
                }
              }
            }
          }
          if (A.tags != nullptr) {
            A.tags[B.voff + ((long long)z * B.n[1] + y) * B.n[0] + x] = tagged ? 1 : 0;
            n_tagged += tagged ? 1 : 0;
          }
          if (A.epart != nullptr) {
            bool cov = false;
            if (A.covered != nullptr) {
              const int gx = (B.lo[0] + x) >> A.cov_shift, gy = (B.lo[1] + y) >> A.cov_shift,
                        gz = (B.lo[2] + z) >> A.cov_shift;
              cov = A.covered[((long long)gz * A.cov_nb + gy) * A.cov_nb + gx] != 0;
            }
            if (!cov) {
              const T dd = r2 - (T)1;
              i_kin += (T)0.5 * (P1 * P1 + P2 * P2);
              i_grad += (T)(-0.5) * (p1 * l1 + p2 * l2);
              i_pot += ((T)0.25 * c_pot) * (dd * dd) + ((T)0.5 * a_c) * r2;
              n_pierced += owned;
            }
          }
        }
      }
      __syncthreads();
    }
    s_kin += (double)i_kin;
    s_grad += (double)i_grad;
    s_pot += (double)i_pot;
  }

  if (A.epart != nullptr || A.tagcount != nullptr) {
    // fixed-order block reduction: warp shuffles, then warp 0 over warps
    __shared__ double red[4][NT / 32];
    __shared__ unsigned long long redt[NT / 32];
    double v0 = s_kin, v1 = s_grad, v2 = s_pot, v3 = (double)n_pierced;
    unsigned long long vt = n_tagged;
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
      for (int w = 0; w < NT / 32; ++w) {
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

template <typename T, int G, int TX, int TY>
static size_t stage_smem() {
  return (size_t)(2 * G + 2) * 2 * (TY + 2 * G) * (TX + 8) * sizeof(T);
}

template <typename T, int G, int TX, int TY>
static int stage_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    const size_t smem = stage_smem<T, G, TX, TY>();
    cudaFuncSetAttribute(stage_kernel<T, G, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, stage_kernel<T, G, TX, TY>, TX * TY, smem);
    occ = o > 0 ? o : 1;
  }
  return occ;
}

template <typename T, int G, int TX, int TY>
static slh_status launch_t(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s,
                           int* ctas_used) {
  StageArgs<T> A;
  A.boxes = L.d_boxes;
  A.items = L.d_items;
  A.nitems = L.nitems;
  A.zlen = L.zlen;
  A.gl = c->g;
  A.yin = static_cast<const T*>(s.yin);
  A.yn = static_cast<const T*>(s.yn);
  A.dacc = static_cast<T*>(s.dacc);
  A.yout = static_cast<T*>(s.yout);
  A.comp = static_cast<T*>(s.comp);
  A.stage = s.stage;
  A.eta_start = c->d_time + 2 * s.lev + (s.cur_eta ? 0 : 1);
  A.c_stage = s.c_stage;
  A.lambda = p.lambda;
  A.a = p.a;
  A.friction = p.friction;
  A.eta_power = p.eta_power;
  A.inv_dx2 = 1.0 / (L.dx * L.dx);
  A.ha = s.ha;
  A.hb = s.hb;
  A.tags = s.tags;
  A.epart = s.epart;
  A.tagcount = s.tagcount;
  A.covered = s.covered;
  A.cov_shift = s.cov_shift;
  A.cov_nb = s.cov_nb;
  const int occ = stage_occupancy<T, G, TX, TY>();
  int grid = occ * c->num_sms;
  if (grid > L.nitems) grid = L.nitems;
  if (grid < 1) grid = 1;
  if (s.epart != nullptr && grid > L.epart_cap) grid = L.epart_cap;
  if (ctas_used) *ctas_used = grid;
  if (L.nitems == 0) return SLH_OK;
  stage_kernel<T, G, TX, TY><<<grid, TX * TY, stage_smem<T, G, TX, TY>(), c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

template <typename T, int TY>
static slh_status dispatch_g(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* u) {
  switch (p.lap_order) {
    case 2: return launch_t<T, 1, 32, TY>(c, L, p, s, u);
    case 4: return launch_t<T, 2, 32, TY>(c, L, p, s, u);
    case 6: return launch_t<T, 3, 32, TY>(c, L, p, s, u);
    default: return fail(SLH_ERR_INVALID_ARG, "lap_order must be 2, 4 or 6 (got %d)", p.lap_order);
  }
}

slh_status launch_stage(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s,
                        int* ctas_used) {
  if (c->prec == SLH_F64) {
    if (L.tile_y != 8) return fail(SLH_ERR_STATE, "tile mismatch");
    return dispatch_g<double, 8>(c, L, p, s, ctas_used);
  }
  if (L.tile_y != 16) return fail(SLH_ERR_STATE, "tile mismatch");
  return dispatch_g<float, 16>(c, L, p, s, ctas_used);
}

int stage_grid(slh_ctx* c, Level& L, int order) {
  int occ = 1;
  const int G = order / 2;
  if (c->prec == SLH_F64) {
    occ = G == 1 ? stage_occupancy<double, 1, 32, 8>() : G == 2 ? stage_occupancy<double, 2, 32, 8>()
                                                                 : stage_occupancy<double, 3, 32, 8>();
  } else {
    occ = G == 1 ? stage_occupancy<float, 1, 32, 16>() : G == 2 ? stage_occupancy<float, 2, 32, 16>()
                                                                 : stage_occupancy<float, 3, 32, 16>();
  }
  return occ * c->num_sms;
}

}  // namespace slh
