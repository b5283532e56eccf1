// Shadow level of level 0 for the truncation-error estimate (Sec. 2.2):
// level 0 coarsened by 2^3 into a context of half the resolution, and, after
// the shadow has taken one step of 2 dt0 and level 0 two of dt0, the
// comparison |shadow - mean of children| that writes level 0's TEE tags.
// The means are FP64 sums of the 8 children in the order x, y, z (the same
// order as the restriction), so they are bit-identical to it.
#include "slh_internal.cuh"

namespace slh {

__device__ __forceinline__ long long cell_at(const BoxDev& B, int gl, int x, int y, int z) {
  return B.off + ((long long)(z + gl) * B.pny + (y + gl)) * B.pitch + (x + XPAD);
}

template <typename T>
struct ShadowArgs {
  const BoxDev* sboxes;   // shadow level 0
  int nsb;
  long long nvalid;
  T* sy;                  // shadow state
  int sgl;
  const BoxDev* fboxes;   // level 0 of the context
  const T* fy;
  const int* fbmap;
  int fbshift, fnbd;
  int fgl;
  int ncomp;
  int compare;            // 0: write the means into the shadow; 1: compare and tag
  uint8_t* tee;           // level 0's TEE tags (compare)
  double eps[4];
};

template <typename T>
__global__ void shadow_kernel(const ShadowArgs<T> A) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < A.nvalid; t += stride) {
    int lo = 0, hi = A.nsb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.sboxes[mid].voff <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev S = A.sboxes[lo];
    const long long loc = t - S.voff;
    const int rx = (int)(loc % S.n[0]);
    const int ry = (int)((loc / S.n[0]) % S.n[1]);
    const int rz = (int)(loc / ((long long)S.n[0] * S.n[1]));
    const int fx = 2 * (S.lo[0] + rx), fy = 2 * (S.lo[1] + ry), fz = 2 * (S.lo[2] + rz);   // first child
    // the 8 children lie in one block of the fine level, hence in one box
    const int own = A.fbmap[((long long)(fz >> A.fbshift) * A.fnbd + (fy >> A.fbshift)) * A.fnbd + (fx >> A.fbshift)];
    const BoxDev F = A.fboxes[own];
    const long long f000 = cell_at(F, A.fgl, fx - F.lo[0], fy - F.lo[1], fz - F.lo[2]);
    const long long sy = F.pitch, sz = (long long)F.pny * F.pitch;
    const long long dst = cell_at(S, A.sgl, rx, ry, rz);
    bool hit = false;
    const int nc = A.compare ? 4 : A.ncomp;
    for (int c = 0; c < nc; ++c) {
      const T* f = A.fy + f000 + c * F.cs;
      double s = (double)f[0];
      s += (double)f[1];
      s += (double)f[sy];
      s += (double)f[sy + 1];
      s += (double)f[sz];
      s += (double)f[sz + 1];
      s += (double)f[sz + sy];
      s += (double)f[sz + sy + 1];
      s *= 0.125;
      if (A.compare) {
        if (A.eps[c] > 0.0) hit |= fabs((double)A.sy[dst + c * S.cs] - s) > A.eps[c];
      } else {
        A.sy[dst + c * S.cs] = (T)s;
      }
    }
    if (A.compare) {
      const uint8_t tv = hit ? 1 : 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int cx = fx - F.lo[0] + (a & 1), cy = fy - F.lo[1] + ((a >> 1) & 1), cz = fz - F.lo[2] + (a >> 2);
        A.tee[F.voff + ((long long)cz * F.n[1] + cy) * F.n[0] + cx] = tv;
      }
    }
  }
}

template <typename T>
static slh_status shadow_t(slh_ctx* c, slh_ctx* s, bool compare) {
  Level& F = c->lev[0];
  Level& S = s->lev[0];
  ShadowArgs<T> A;
  A.sboxes = S.d_boxes;
  A.nsb = (int)S.boxes.size();
  A.nvalid = S.lay.nvalid;
  A.sy = static_cast<T*>(S.buf[S.role_y]);
  A.sgl = s->g;
  A.fboxes = F.d_boxes;
  A.fy = static_cast<const T*>(F.buf[F.role_y]);
  A.fbmap = F.d_bmap;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.fbshift = sh;
  A.fnbd = F.nb_dom;
  A.fgl = c->g;
  A.ncomp = c->ncomp;
  A.compare = compare ? 1 : 0;
  A.tee = F.d_tee;
  for (int q = 0; q < 4; ++q) A.eps[q] = c->te_crit[q];
  const int threads = 256;
  long long blocks = (A.nvalid + threads - 1) / threads;
  const long long cap = (long long)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  shadow_kernel<T><<<(int)blocks, threads, 0, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_shadow(slh_ctx* c, slh_ctx* shadow, bool compare) {
  return c->prec == SLH_F64 ? shadow_t<double>(c, shadow, compare) : shadow_t<float>(c, shadow, compare);
}

}  // namespace slh
