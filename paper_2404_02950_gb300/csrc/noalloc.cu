// Energy and string length of a dense periodic lattice with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a host callback
// or another library's stream-ordered section where allocation would
// synchronise or is forbidden, embedders with a fixed memory budget that hand
// out every byte themselves, and processes whose allocator is owned by a
// framework that must not see foreign allocations.  For them this file keeps
// its reduction scratch in one fixed array in device global memory that is
// part of the library image: every GPU that loads the library holds it until
// the process exits, whether or not the entry point is used.
//
// The quantity is the one slh_reduce_energy computes for a single periodic
// box (kinetic, gradient and potential energy of Sec. 3.1's fields and the
// number of plaquettes with nonzero winding), here for a dense lattice the
// caller owns.
#include <mutex>

#include "slh_internal.cuh"

namespace {

// Largest lattice side: one partial-sum row (4 doubles) per z-plane.
constexpr int NOALLOC_MAX_PLANES = 4096;

// The scratch: per z-plane partial sums, 4096 x 4 doubles = 128 KiB.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_PLANES * 4];

std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
double* g_scratch[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (host code only
// sees a host-side stand-in for the symbol, never a device address).
slh_status scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return slh::cuda_fail(e, "energy_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return slh::fail(SLH_ERR_OUT_OF_RANGE, "energy_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return slh::cuda_fail(e, "energy_noalloc: cudaGetSymbolAddress of the scratch array");
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return SLH_OK;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// winding term of the edge a -> b (exact sign of the cross product in FP64;
// for FP32 inputs the products are exact)
__device__ __forceinline__ int edge_term(double ar, double ai, double br, double bi) {
  const bool ua = ai >= 0.0, ub = bi >= 0.0;
  if (ua == ub) return 0;
  const double X = __dsub_rn(__dmul_rn(ar, bi), __dmul_rn(ai, br));
  return (int)(ua && X > 0.0) - (int)(ub && X < 0.0);
}

__device__ __forceinline__ double lapw(int G, int m) {
  if (G == 1) return m == 0 ? -2.0 : 1.0;
  if (G == 2) return m == 0 ? -2.5 : (m == 1 ? 4.0 / 3.0 : -1.0 / 12.0);
  return m == 0 ? -49.0 / 18.0 : (m == 1 ? 1.5 : (m == 2 ? -0.15 : 1.0 / 90.0));
}

// One CTA per z-plane: per-thread FP64 sums over the plane's cells in a fixed
// order, then a fixed tree; partial row z of the scratch receives
// (kinetic, gradient, potential, pierced plaquettes).
template <typename T>
__global__ void plane_energy_kernel(const T* __restrict__ f, int n, int G, double inv_dx2, double c_pot, double a,
                                    double* __restrict__ partials) {
  const int z = blockIdx.x;
  const long long N3 = (long long)n * n * n;
  const T* p1f = f;
  const T* p2f = f + N3;
  const T* P1f = f + 2 * N3;
  const T* P2f = f + 3 * N3;
  auto at = [&](const T* c, int x, int y, int zz) -> double {
    return (double)c[((long long)wrap(zz, n) * n + wrap(y, n)) * n + wrap(x, n)];
  };
  double sk = 0.0, sg = 0.0, sp = 0.0, sn = 0.0;
  for (int xy = threadIdx.x; xy < n * n; xy += blockDim.x) {
    const int x = xy % n, y = xy / n;
    const double p1 = at(p1f, x, y, z), p2 = at(p2f, x, y, z);
    double l1 = 3.0 * lapw(G, 0) * p1, l2 = 3.0 * lapw(G, 0) * p2;
    for (int m = 1; m <= G; ++m) {
      const double w = lapw(G, m);
      l1 += w * ((at(p1f, x + m, y, z) + at(p1f, x - m, y, z)) + (at(p1f, x, y + m, z) + at(p1f, x, y - m, z)) +
                 (at(p1f, x, y, z + m) + at(p1f, x, y, z - m)));
      l2 += w * ((at(p2f, x + m, y, z) + at(p2f, x - m, y, z)) + (at(p2f, x, y + m, z) + at(p2f, x, y - m, z)) +
                 (at(p2f, x, y, z + m) + at(p2f, x, y, z - m)));
    }
    l1 *= inv_dx2;
    l2 *= inv_dx2;
    const double P1 = at(P1f, x, y, z), P2 = at(P2f, x, y, z);
    const double r2 = p1 * p1 + p2 * p2, d = r2 - 1.0;
    sk += 0.5 * (P1 * P1 + P2 * P2);
    sg += -0.5 * (p1 * l1 + p2 * l2);
    sp += (0.25 * c_pot) * (d * d) + (0.5 * a) * r2;
    // the three plaquettes owned by the cell: normals z (x,y), x (y,z), y (z,x)
    const int us[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int vs[3][3] = {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}};
    for (int w = 0; w < 3; ++w) {
      const int ux = us[w][0], uy = us[w][1], uz = us[w][2], vx = vs[w][0], vy = vs[w][1], vz = vs[w][2];
      const double r0 = at(p1f, x, y, z), i0 = at(p2f, x, y, z);
      const double r1 = at(p1f, x + ux, y + uy, z + uz), i1 = at(p2f, x + ux, y + uy, z + uz);
      const double rr = at(p1f, x + ux + vx, y + uy + vy, z + uz + vz), ii = at(p2f, x + ux + vx, y + uy + vy, z + uz + vz);
      const double r3 = at(p1f, x + vx, y + vy, z + vz), i3 = at(p2f, x + vx, y + vy, z + vz);
      const int W = edge_term(r0, i0, r1, i1) + edge_term(r1, i1, rr, ii) + edge_term(rr, ii, r3, i3) +
                    edge_term(r3, i3, r0, i0);
      sn += W != 0 ? 1.0 : 0.0;
    }
  }
  __shared__ double red[4][256];
  red[0][threadIdx.x] = sk;
  red[1][threadIdx.x] = sg;
  red[2][threadIdx.x] = sp;
  red[3][threadIdx.x] = sn;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[4 * z + threadIdx.x] = red[threadIdx.x][0];
}

// Sums the n partial rows in a fixed order and writes the five outputs.
__global__ void planes_sum_kernel(const double* __restrict__ partials, int n, double dx, double* __restrict__ out) {
  __shared__ double s[4][256];
  const int t = threadIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = t; r < n; r += 256)
    for (int q = 0; q < 4; ++q) a[q] += partials[4 * r + q];
  for (int q = 0; q < 4; ++q) s[q][t] = a[q];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h)
      for (int q = 0; q < 4; ++q) s[q][t] += s[q][t + h];
    __syncthreads();
  }
  if (t == 0) {
    const double vol = dx * dx * dx;
    out[0] = s[0][0] * vol;
    out[1] = s[1][0] * vol;
    out[2] = s[2][0] * vol;
    out[3] = out[0] + out[1] + out[2];
    out[4] = s[3][0] * dx;
  }
}

}  // namespace

extern "C" slh_status slh_energy_noalloc(const void* fields_dev, int32_t n, int32_t prec, double dx, double eta,
                                         const slh_eom_params* p, double* out_dev, void* stream) {
  if (!fields_dev || !out_dev || !p) return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: null argument");
  if (prec != SLH_F64 && prec != SLH_F32_KAHAN) return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: unknown precision %d", prec);
  if (p->lap_order != 2 && p->lap_order != 4 && p->lap_order != 6)
    return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: lap_order must be 2, 4 or 6");
  if (p->eta_power != 0 && p->eta_power != 2) return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: eta_power must be 0 or 2");
  const int G = p->lap_order / 2;
  if (n < 2 * G + 1)
    return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: lattice side %d is smaller than the stencil width %d", n, 2 * G + 1);
  if (n > NOALLOC_MAX_PLANES)
    return slh::fail(SLH_ERR_OUT_OF_RANGE,
                     "energy_noalloc: lattice side %d exceeds the fixed scratch limit of %d planes; use slh_reduce_energy",
                     n, NOALLOC_MAX_PLANES);
  if (!(dx > 0.0)) return slh::fail(SLH_ERR_INVALID_ARG, "energy_noalloc: dx must be positive");
  double* scratch = nullptr;
  slh_status st = scratch_on_current_device(&scratch);
  if (st != SLH_OK) return st;
  const double c_pot = p->eta_power == 2 ? p->lambda * (eta * eta) : p->lambda;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == SLH_F64)
    plane_energy_kernel<double><<<n, 256, 0, s>>>(static_cast<const double*>(fields_dev), n, G, 1.0 / (dx * dx), c_pot,
                                                  p->a, scratch);
  else
    plane_energy_kernel<float><<<n, 256, 0, s>>>(static_cast<const float*>(fields_dev), n, G, 1.0 / (dx * dx), c_pot,
                                                 p->a, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return slh::cuda_fail(e, "energy_noalloc: plane kernel");
  planes_sum_kernel<<<1, 256, 0, s>>>(scratch, n, dx, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return slh::cuda_fail(e, "energy_noalloc: sum kernel");
  return SLH_OK;
}
