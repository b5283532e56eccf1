// Floating-point issue rate of the device: the ALU roofline of the FP64 form.
//
// The FP64 stage kernel does ~56 FP64 operations per cell and stage against
// 17 values moved, and GB300 issues FP64 at a small fraction of its FP32
// rate, so the FP64 form is bound by its FP64 pipe, not by HBM.  Its roofline
// denominator is the device's sustained rate of independent FMAs, measured
// here: every thread runs CHAINS independent fma recurrences (enough to cover
// the pipe's latency), a grid of 8 CTAs of 256 threads per SM, timed with
// CUDA events around one launch, best of `reps`.  Nothing is allocated: the
// sink that keeps the chains alive is a static device variable.
#include "slh_internal.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 8;

static __device__ double g_sink_f64;
static __device__ float g_sink_f32;

template <typename T>
__global__ void alu_fma_kernel(T* out, int iters, T a, T b) {
  T x[CHAINS];
  for (int k = 0; k < CHAINS; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  // the recurrence tends to b / (1 - a) = 0.1: never equal to this value,
  // but the compiler cannot know that
  if (s == (T)123456.0) out[0] = s;
}

template <typename T>
slh_status measure(int iters, int reps, double* out) {
  int dev = 0, sms = 0;
  SLH_CUDA(cudaGetDevice(&dev));
  SLH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const dim3 grid(sms * CTAS_PER_SM), block(THREADS);
  const T a = (T)0.999999, b = (T)1e-7;
  T* sink = nullptr;
  SLH_CUDA(cudaGetSymbolAddress((void**)&sink, sizeof(T) == 8 ? (const void*)&g_sink_f64 : (const void*)&g_sink_f32));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SLH_CUDA(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return slh::cuda_fail(e, "alu_rate: cudaEventCreate");
  }
  double best = 0;
  alu_fma_kernel<T><<<grid, block>>>(sink, 100, a, b);  // warm-up
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0);
    alu_fma_kernel<T><<<grid, block>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0) {
      const double fmas = (double)CHAINS * iters * (double)grid.x * THREADS;
      best = fmax(best, fmas / (ms * 1e-3));
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return slh::cuda_fail(e, "alu_rate: timed FMA launch");
  *out = best;
  return SLH_OK;
}

}  // namespace

extern "C" slh_status slh_alu_rate(int32_t prec, int32_t reps, double* fma_per_s) {
  if (fma_per_s == nullptr) return slh::fail(SLH_ERR_INVALID_ARG, "alu_rate: null output");
  if (reps < 1 || reps > 100) return slh::fail(SLH_ERR_INVALID_ARG, "alu_rate: reps must be in [1, 100] (got %d)", reps);
  // iteration counts sized for ~15-80 ms per launch on a 152-SM part
  if (prec == SLH_F64) return measure<double>(20000, reps, fma_per_s);
  if (prec == SLH_F32_KAHAN) return measure<float>(200000, reps, fma_per_s);
  return slh::fail(SLH_ERR_INVALID_ARG, "alu_rate: prec must be SLH_F64 or SLH_F32_KAHAN (got %d)", prec);
}
