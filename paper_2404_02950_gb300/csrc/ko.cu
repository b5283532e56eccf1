// Kreiss-Oliger dissipation (Sec. 2.4) of the scalar fields psi1, psi2, Pi1,
// Pi2 of an RK stage input:
//   Q f = (-1)^((p+3)/2) eps / (2^(p+1) dx) sum_d delta_d^(p+1) f,
// delta^(p+1) the central (p+1)-st difference (binomial weights, radius
// R = (p+1)/2).  One launch per RK stage, next to the stage kernel, folds the
// stage's share of Q into the stage outputs: out += cout Q, D += cd Q (the
// coefficients are the stage's a dt and b dt of classic RK4, or b dt of
// SSPRK3).  The dissipation may reach farther than the Laplacian (App. C
// pairs a 5-point gradient with a 7-point dissipation), which is why it is a
// kernel of its own: one thread per cell column marching in z, operands from
// global memory through L1/L2, like the GW stage kernel.
#include "slh_internal.cuh"

namespace slh {

template <int R>
__device__ __forceinline__ double binom_w(int j);   // weight of offset j - R, j = 0..2R
template <>
__device__ __forceinline__ double binom_w<1>(int j) { return j == 1 ? -2.0 : 1.0; }
template <>
__device__ __forceinline__ double binom_w<2>(int j) { return j == 2 ? 6.0 : ((j == 1 || j == 3) ? -4.0 : 1.0); }
template <>
__device__ __forceinline__ double binom_w<3>(int j) {
  return j == 3 ? -20.0 : ((j == 2 || j == 4) ? 15.0 : ((j == 1 || j == 5) ? -6.0 : 1.0));
}

template <typename T>
struct KoArgs {
  const BoxDev* boxes;
  const int4* items;
  int gl;
  const T* in;
  T* out;
  T* d;          // null: no increment update
  double kappa;  // (-1)^((p+3)/2) eps / (2^(p+1) dx)
  double cout, cd;
};

template <typename T, int R>
__global__ void __launch_bounds__(COL_TX * COL_TY, 4) ko_kernel(const KoArgs<T> A) {
  const int4 it = A.items[blockIdx.x];
  const BoxDev B = A.boxes[it.x];
  const int x = it.y + threadIdx.x, y = it.z + threadIdx.y;
  if (x >= B.n[0] || y >= B.n[1]) return;
  const int z1 = min(it.w + COL_ZLEN, B.n[2]);
  const long long sy = B.pitch, sz = (long long)B.pitch * B.pny, cs = B.cs;
  const T* __restrict__ in = A.in;
  T* __restrict__ out = A.out;
  T* __restrict__ dd = A.d;
  const T ko = (T)A.kappa, co = (T)A.cout, cd = (T)A.cd;
  long long e = B.off + ((long long)(it.w + A.gl) * B.pny + (y + A.gl)) * B.pitch + x + XPAD;
#pragma unroll 1
  for (int z = it.w; z < z1; ++z, e += sz) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* f = in + e + c * cs;
      T sx = 0, syy = 0, szz = 0;
#pragma unroll
      for (int j = 0; j <= 2 * R; ++j) {
        const T w = (T)binom_w<R>(j);
        sx += w * __ldg(f + (j - R));
        syy += w * __ldg(f + (j - R) * sy);
        szz += w * __ldg(f + (j - R) * sz);
      }
      const T q = ko * ((sx + syy) + szz);
      const long long ec = e + c * cs;
      if (co != (T)0) out[ec] = out[ec] + co * q;
      if (dd != nullptr) dd[ec] = dd[ec] + cd * q;
    }
  }
}

template <typename T>
static slh_status ko_t(slh_ctx* c, Level& L, const slh_eom_params& p, int in_buf, int out_buf, int d_buf,
                       double cout, double cd) {
  if (L.ncol_items == 0) return SLH_OK;
  KoArgs<T> A;
  A.boxes = L.d_boxes;
  A.items = L.d_col_items;
  A.gl = c->g;
  A.in = static_cast<const T*>(L.buf[in_buf]);
  A.out = static_cast<T*>(L.buf[out_buf]);
  A.d = d_buf >= 0 ? static_cast<T*>(L.buf[d_buf]) : nullptr;
  const int P = p.ko_order;
  A.kappa = (((P + 3) / 2) % 2 ? -1.0 : 1.0) * p.ko_eps / (std::ldexp(1.0, P + 1) * L.dx);
  A.cout = cout;
  A.cd = cd;
  const dim3 block(COL_TX, COL_TY);
  switch (P) {
    case 1: ko_kernel<T, 1><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    case 3: ko_kernel<T, 2><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    case 5: ko_kernel<T, 3><<<L.ncol_items, block, 0, c->stream>>>(A); break;
    default: return fail(SLH_ERR_INVALID_ARG, "dissipation order must be 1, 3 or 5 (got %d)", P);
  }
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_ko(slh_ctx* c, Level& L, const slh_eom_params& p, int in_buf, int out_buf, int d_buf, double cout,
                     double cd) {
  return c->prec == SLH_F64 ? ko_t<double>(c, L, p, in_buf, out_buf, d_buf, cout, cd)
                            : ko_t<float>(c, L, p, in_buf, out_buf, d_buf, cout, cd);
}

}  // namespace slh
