// Reductions and regrid support: fixed-order sum of the per-CTA energy
// partials, and the grown-tag block mask used by regridding (Sec. 2.2:
// tags grown by a buffer of n_error_buf cells, then coarsened to blocks).
#include "slh_internal.cuh"

namespace slh {

// One CTA sums n rows of 4 partials in a fixed order: thread t takes rows
// t, t+256, ...; then a fixed tree.  Bit-reproducible for a fixed n.
__global__ void energy_final_kernel(const double* part, int n, double* out4) {
  __shared__ double s[4][256];
  const int t = threadIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = t; r < n; r += 256) {
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] += part[4 * r + q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q][t] = a[q];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q][t] += s[q][t + h];
    }
    __syncthreads();
  }
  if (t < 4) out4[t] = s[t][0];
}

slh_status launch_energy_final(slh_ctx* c, const double* epart, int n, double* out4) {
  energy_final_kernel<<<1, 256, 0, c->stream>>>(epart, n, out4);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

struct TagBlockArgs {
  const BoxDev* boxes;
  int nboxes;
  const uint8_t* tags;    // either may be null: a cell is tagged if either tags it
  const uint8_t* tags2;
  long long nvalid;
  int nbuf, r, nb, ndom;
  uint8_t* mask;
};

// One thread per valid cell; a tagged cell marks every block its grown cube
// (side 2 n_error_buf + 1, periodic) intersects.
__global__ void tag_blocks_kernel(const TagBlockArgs A) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < A.nvalid; t += stride) {
    if (!((A.tags != nullptr && A.tags[t]) || (A.tags2 != nullptr && A.tags2[t]))) continue;
    int lo = 0, hi = A.nboxes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.boxes[mid].voff <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev B = A.boxes[lo];
    const long long loc = t - B.voff;
    const int x = B.lo[0] + (int)(loc % B.n[0]);
    const int y = B.lo[1] + (int)((loc / B.n[0]) % B.n[1]);
    const int z = B.lo[2] + (int)(loc / ((long long)B.n[0] * B.n[1]));
    // floor division of possibly negative cell indices
    auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int bx0 = fdiv(x - A.nbuf, A.r), bx1 = fdiv(x + A.nbuf, A.r);
    const int by0 = fdiv(y - A.nbuf, A.r), by1 = fdiv(y + A.nbuf, A.r);
    const int bz0 = fdiv(z - A.nbuf, A.r), bz1 = fdiv(z + A.nbuf, A.r);
    for (int bz = bz0; bz <= bz1; ++bz)
      for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx) {
          const int wx = ((bx % A.nb) + A.nb) % A.nb, wy = ((by % A.nb) + A.nb) % A.nb,
                    wz = ((bz % A.nb) + A.nb) % A.nb;
          A.mask[((long long)wz * A.nb + wy) * A.nb + wx] = 1;
        }
  }
}

slh_status launch_tag_blocks(slh_ctx* c, Level& L, const uint8_t* tags, const uint8_t* tags2, int nbuf, int r,
                             uint8_t* mask, int nb) {
  TagBlockArgs A;
  A.boxes = L.d_boxes;
  A.nboxes = (int)L.boxes.size();
  A.tags = tags;
  A.tags2 = tags2;
  A.nvalid = L.lay.nvalid;
  A.nbuf = nbuf;
  A.r = r;
  A.nb = nb;
  A.ndom = L.n_dom;
  A.mask = mask;
  const int threads = 256;
  long long blocks = (A.nvalid + threads - 1) / threads;
  const long long cap = (long long)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  tag_blocks_kernel<<<(int)blocks, threads, 0, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

// A wait nothing completes: one CTA initialises an mbarrier expecting two
// arrivals, arrives once and polls the phase with a bounded loop like the
// stage kernel's waits (here limited to `polls`); on expiry it latches
// DERR_TIMEOUT exactly as the stage kernel does, so the host sees
// SLH_ERR_TIMEOUT at its next synchronising call and the context stays usable.
__global__ void expired_wait_kernel(int* err, long long polls) {
  __shared__ unsigned long long bar;
  const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(&bar));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(2) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(addr) : "memory");
    bool done = false;
    for (long long i = 0; i < polls && !done; ++i) {
      unsigned ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(addr), "r"(0u)
          : "memory");
      done = ok != 0;
    }
    if (!done) atomicCAS(err, 0, DERR_TIMEOUT);
  }
  __syncthreads();
}

slh_status launch_expired_wait(slh_ctx* c, long long polls) {
  expired_wait_kernel<<<1, 32, 0, c->stream>>>(c->d_err, polls);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

}  // namespace slh
