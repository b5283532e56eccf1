// Inter-level transfer (Sec. 2.1): ghost fill of a level's psi components
// (and, with the gravitational-wave tensor, the six u_ij) from its own boxes (periodic wrap) or, where no box of the level covers a
// ghost cell, by ratio-2 prolongation of the coarser level interpolated in
// time; restriction of a fine level onto the covered coarse cells; and the
// small kernel that advances the per-level conformal time.
#include "slh_internal.cuh"

namespace slh {

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// (i, j, k) of the flat index t in an e0 x e1 x ... box with quotients by
// float reciprocals: t = q d + r gives (t + 1/2)/d in [q + 1/(2d), q + 1 -
// 1/(2d)], and the rounding of the product stays below 1/(2d) while t d <
// 2^22, which region, piece and patch indexes (<= 32*32*4) satisfy.
struct Split3 {
  int e0, e01;
  float r0, r01;
  __device__ __forceinline__ Split3(int a, int b) : e0(a), e01(a * b), r0(1.0f / (float)a), r01(1.0f / (float)(a * b)) {}
  __device__ __forceinline__ void operator()(int t, int& i, int& j, int& k) const {
    k = (int)(((float)t + 0.5f) * r01);
    const int rem = t - k * e01;
    j = (int)(((float)rem + 0.5f) * r0);
    i = rem - j * e0;
  }
};

__device__ __forceinline__ long long cell_index(const BoxDev& B, int gl, int x, int y, int z) {
  // valid-relative (x, y, z), may lie in the ghost shell
  return B.off + ((long long)(z + gl) * B.pny + (y + gl)) * B.pitch + (x + XPAD);
}

// 1D prolongation weights for offsets -2..2 (type 4: fine-cell average of
// the quartic matching five coarse averages; type 2: quadratic through
// three coarse centres evaluated at the fine centre; type 0: parent value).
// child 0 is the lower half of the coarse cell, child 1 the upper half.
__device__ __forceinline__ double pw(int itype, int child, int off) {
  if (itype == 4) {
    const int j = child == 0 ? off : -off;  // child 1 is the mirror image
    switch (j) {
      case -2: return -3.0 / 128.0;
      case -1: return 11.0 / 64.0;
      case 0: return 1.0;
      case 1: return -11.0 / 64.0;
      default: return 3.0 / 128.0;
    }
  }
  if (itype == 2) {
    const int j = child == 0 ? off : -off;
    switch (j) {
      case -1: return 5.0 / 32.0;
      case 0: return 15.0 / 16.0;
      case 1: return -3.0 / 32.0;
      default: return 0.0;
    }
  }
  return off == 0 ? 1.0 : 0.0;
}

// Ghost fill by regions (see GhostRegion): copy regions are plain strided
// copies; prolongation regions first gather the coarser level's cells under
// the region's stencil footprint, time-interpolated, into shared memory (one
// box lookup per coarse cell instead of one per stencil point), then one
// thread per coarse cell under the region evaluates the (2r+1)^3
// tensor-product stencil of its 8 children at once, as separable partial
// sums along x, then y, then z (each patch value read once per coarse cell
// instead of once per child); mixed regions decide cell by cell.
constexpr int PATCH_MAX = 21 * 21 * 7;   // coarse cells under a 32 x 32 x g region (r <= 2, g <= 4)

template <typename T>
struct GhostArgs {
  const BoxDev* boxes;
  const GhostRegion* regions;
  int nregions;
  const PatchPiece* pieces;
  T* y;
  int gl;
  const int* bmap;
  int bshift, nbd, ndom;
  // coarser level
  const BoxDev* cboxes;
  const T* cold;
  const T* cnew;
  const int* cbmap;
  int cnbd, cndom;
  double alpha;
  int itype;
  int npairs;   // field pairs filled: (psi1, psi2) and with 16 fields (u_xx, u_yy), (u_zz, u_xy), (u_xz, u_yz)
  int* err;
};

// first component of field pair q
__device__ __forceinline__ int pair_comp(int q) { return q == 0 ? 0 : GW_U0 + 2 * (q - 1); }

template <typename T, int RAD>
__global__ void __launch_bounds__(256, 3) ghost_region_kernel(const GhostArgs<T> A) {
  // [2][pz][py][px]: time-interpolated psi1, psi2 in the field precision
  // (the stencil weights are dyadic rationals, exact in FP32 and FP64)
  extern __shared__ __align__(16) unsigned char patch_raw[];
  T* patch = reinterpret_cast<T*>(patch_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const T al = (T)A.alpha, bl = (T)1 - (T)A.alpha;
  for (int r = blockIdx.x; r < A.nregions; r += gridDim.x) {
    const GhostRegion R = A.regions[r];
    const BoxDev B = A.boxes[R.box];
    const int ncell = R.ext[0] * R.ext[1] * R.ext[2];
    if (R.kind == GHOST_COPY) {
      const BoxDev S = A.boxes[R.src];
      const Split3 sp(R.ext[0], R.ext[1]);
      for (int t = tid; t < ncell; t += nt) {
        int i, j, k;
        sp(t, i, j, k);
        const int rx = R.lo[0] + i, ry = R.lo[1] + j, rz = R.lo[2] + k;
        const long long dst = cell_index(B, A.gl, rx, ry, rz);
        const long long src = cell_index(S, A.gl, rx + R.d[0], ry + R.d[1], rz + R.d[2]);
        for (int q = 0; q < A.npairs; ++q) {
          const int c0 = pair_comp(q);
          A.y[dst + c0 * B.cs] = A.y[src + c0 * S.cs];
          A.y[dst + (c0 + 1) * B.cs] = A.y[src + (c0 + 1) * S.cs];
        }
      }
      continue;   // uniform over the CTA: no shared memory used
    }
    // coarse footprint of the widest stencil (unwrapped coarse coordinates);
    // narrower stencils use part of it
    int plo[3], pn[3];
    for (int d = 0; d < 3; ++d) {
      const int flo = B.lo[d] + R.lo[d], fhi = flo + R.ext[d] - 1;
      plo[d] = (flo >> 1) - PROLONG_RAD_MAX;
      pn[d] = (fhi >> 1) + PROLONG_RAD_MAX - plo[d] + 1;
    }
    const int np = pn[0] * pn[1] * pn[2];
    const bool have_coarse = A.cboxes != nullptr && np <= PATCH_MAX;
    for (int q = 0; q < A.npairs; ++q) {
      const int c0 = pair_comp(q);
      if (have_coarse && R.covered) {
        // planned gather: strided copies of the pieces, no lookups
        for (int pi = R.p0; pi < R.p0 + R.np; ++pi) {
          const PatchPiece P = A.pieces[pi];
          const BoxDev C = A.cboxes[P.cbox];
          const int ne = P.ext[0] * P.ext[1] * P.ext[2];
          const Split3 sp(P.ext[0], P.ext[1]);
          for (int t = tid; t < ne; t += nt) {
            int i, j, k;
            sp(t, i, j, k);
            const long long ci = cell_index(C, A.gl, P.src[0] + i, P.src[1] + j, P.src[2] + k) + c0 * C.cs;
            const int pt = ((P.dst[2] + k) * pn[1] + (P.dst[1] + j)) * pn[0] + (P.dst[0] + i);
            patch[pt] = bl * A.cold[ci] + al * A.cnew[ci];
            patch[np + pt] = bl * A.cold[ci + C.cs] + al * A.cnew[ci + C.cs];
          }
        }
      } else if (have_coarse) {
        // footprint not tiled by the coarse level (a nesting violation, or a
        // level built without a plan): per-cell lookup, NaN where uncovered
        const Split3 sp(pn[0], pn[1]);
#pragma unroll 4
        for (int t = tid; t < np; t += nt) {
          int i, j, k;
          sp(t, i, j, k);
          const int qx = wrapi(plo[0] + i, A.cndom), qy = wrapi(plo[1] + j, A.cndom), qz = wrapi(plo[2] + k, A.cndom);
          const int cown = A.cbmap[((long long)(qz >> A.bshift) * A.cnbd + (qy >> A.bshift)) * A.cnbd + (qx >> A.bshift)];
          T v0 = (T)__longlong_as_double(0x7ff8000000000000ll), v1 = v0;   // NaN: not covered
          if (cown >= 0) {
            const BoxDev C = A.cboxes[cown];
            const long long ci = cell_index(C, A.gl, qx - C.lo[0], qy - C.lo[1], qz - C.lo[2]) + c0 * C.cs;
            v0 = bl * A.cold[ci] + al * A.cnew[ci];
            v1 = bl * A.cold[ci + C.cs] + al * A.cnew[ci + C.cs];
          }
          patch[t] = v0;
          patch[np + t] = v1;
        }
      }
      __syncthreads();
      // one task per coarse cell under the region: its stencil is read from
      // the patch once and all 8 children follow by separable partial sums
      // (x, then y, then z); children outside the region are not stored
      int clo[3], cn[3], flo[3], fhi[3];
      for (int d = 0; d < 3; ++d) {
        flo[d] = B.lo[d] + R.lo[d];
        fhi[d] = flo[d] + R.ext[d] - 1;
        clo[d] = flo[d] >> 1;
        cn[d] = (fhi[d] >> 1) - clo[d] + 1;
      }
      const int ntask = cn[0] * cn[1] * cn[2];
      const Split3 sp(cn[0], cn[1]);
      T w[2][2 * RAD + 1];   // 1D weights of child 0 and child 1
#pragma unroll
      for (int o = -RAD; o <= RAD; ++o) {
        w[0][o + RAD] = (T)pw(A.itype, 0, o);
        w[1][o + RAD] = (T)pw(A.itype, 1, o);
      }
      for (int t = tid; t < ntask; t += nt) {
        int ti, tj, tk;
        sp(t, ti, tj, tk);
        const int Px = clo[0] + ti, Py = clo[1] + tj, Pz = clo[2] + tk;
        T out[2][2][2][2];   // [field][cz][cy][cx]
        if (have_coarse) {
#pragma unroll
          for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int a = 0; a < 8; ++a) out[f][a >> 2][(a >> 1) & 1][a & 1] = 0;
          const int base = ((Pz - RAD - plo[2]) * pn[1] + (Py - RAD - plo[1])) * pn[0] + (Px - RAD - plo[0]);
#pragma unroll
          for (int oz = 0; oz <= 2 * RAD; ++oz) {
            T ay[2][2][2] = {};   // [field][cy][cx]
#pragma unroll
            for (int oy = 0; oy <= 2 * RAD; ++oy) {
              const int rowb = base + (oz * pn[1] + oy) * pn[0];
              T sx[2][2] = {};    // [field][cx]
#pragma unroll
              for (int ox = 0; ox <= 2 * RAD; ++ox) {
                const T v0 = patch[rowb + ox], v1 = patch[np + rowb + ox];
                sx[0][0] += w[0][ox] * v0;
                sx[0][1] += w[1][ox] * v0;
                sx[1][0] += w[0][ox] * v1;
                sx[1][1] += w[1][ox] * v1;
              }
#pragma unroll
              for (int f = 0; f < 2; ++f)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy) {
                  ay[f][cy][0] += w[cy][oy] * sx[f][0];
                  ay[f][cy][1] += w[cy][oy] * sx[f][1];
                }
            }
#pragma unroll
            for (int f = 0; f < 2; ++f)
#pragma unroll
              for (int a = 0; a < 8; ++a)
                out[f][a >> 2][(a >> 1) & 1][a & 1] += w[a >> 2][oz] * ay[f][(a >> 1) & 1][a & 1];
          }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int cz = a >> 2, cy = (a >> 1) & 1, cx = a & 1;
          const int gx = 2 * Px + cx, gy = 2 * Py + cy, gz = 2 * Pz + cz;   // unwrapped fine coordinates
          if (gx < flo[0] || gx > fhi[0] || gy < flo[1] || gy > fhi[1] || gz < flo[2] || gz > fhi[2]) continue;
          const long long dst = cell_index(B, A.gl, gx - B.lo[0], gy - B.lo[1], gz - B.lo[2]) + c0 * B.cs;
          if (R.kind == GHOST_MIXED) {
            const int wx = wrapi(gx, A.ndom), wy = wrapi(gy, A.ndom), wz = wrapi(gz, A.ndom);
            const int own = A.bmap[((long long)(wz >> A.bshift) * A.nbd + (wy >> A.bshift)) * A.nbd + (wx >> A.bshift)];
            if (own >= 0) {
              const BoxDev Sb = A.boxes[own];
              const long long src = cell_index(Sb, A.gl, wx - Sb.lo[0], wy - Sb.lo[1], wz - Sb.lo[2]) + c0 * Sb.cs;
              A.y[dst] = A.y[src];
              A.y[dst + B.cs] = A.y[src + Sb.cs];
              continue;
            }
          }
          if (!have_coarse) {
            atomicCAS(A.err, 0, DERR_NESTING);
            continue;
          }
          const T v0 = out[0][cz][cy][cx], v1 = out[1][cz][cy][cx];
          if (v0 != v0) atomicCAS(A.err, 0, DERR_NESTING);   // the stencil met an uncovered (NaN) coarse cell
          A.y[dst] = v0;
          A.y[dst + B.cs] = v1;
        }
      }
      __syncthreads();   // the patch is reused by the next pair or region
    }
  }
}

template <typename T>
static slh_status ghosts_t(slh_ctx* c, int lev, int role, double alpha, int itype) {
  Level& L = c->lev[lev];
  if (L.ngregions == 0) return SLH_OK;
  GhostArgs<T> A;
  A.boxes = L.d_boxes;
  A.regions = L.d_gregions;
  A.nregions = L.ngregions;
  A.pieces = L.d_pieces;
  A.y = static_cast<T*>(L.buf[role]);
  A.gl = c->g;
  A.bmap = L.d_bmap;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.bshift = sh;
  A.nbd = L.nb_dom;
  A.ndom = L.n_dom;
  if (lev > 0) {
    Level& C = c->lev[lev - 1];
    A.cboxes = C.d_boxes;
    A.cold = static_cast<const T*>(C.buf[C.role_prev]);
    A.cnew = static_cast<const T*>(C.buf[C.role_y]);
    A.cbmap = C.d_bmap;
    A.cnbd = C.nb_dom;
    A.cndom = C.n_dom;
  } else {
    A.cboxes = nullptr;
    A.cold = A.cnew = nullptr;
    A.cbmap = nullptr;
    A.cnbd = A.cndom = 0;
  }
  A.alpha = alpha;
  A.itype = itype;
  A.npairs = c->ncomp == NCOMP_GW ? 4 : 1;
  A.err = c->d_err;
  const int smem = 2 * PATCH_MAX * (int)sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ghost_region_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(ghost_region_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(ghost_region_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  // many more CTAs than resident slots: prolongation and copy regions cost
  // very different amounts, and the block scheduler evens them out
  long long blocks = L.ngregions;
  const long long cap = (long long)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (itype == 4) ghost_region_kernel<T, 2><<<(int)blocks, 256, smem, c->stream>>>(A);
  else if (itype == 2) ghost_region_kernel<T, 1><<<(int)blocks, 256, smem, c->stream>>>(A);
  else ghost_region_kernel<T, 0><<<(int)blocks, 256, smem, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_ghosts(slh_ctx* c, int lev, int role, double alpha, int itype) {
  if (itype != 0 && itype != 2 && itype != 4)
    return fail(SLH_ERR_INVALID_ARG, "interp_type must be 0, 2 or 4 (got %d)", itype);
  return c->prec == SLH_F64 ? ghosts_t<double>(c, lev, role, alpha, itype)
                            : ghosts_t<float>(c, lev, role, alpha, itype);
}

// ---------------------------------------------------------------------------
// restriction: coarse cell = mean of its 8 children (FP64 sum, order x, y, z);
// with the truncation-error estimate enabled (Sec. 2.2, self-shadow), the
// coarse scalar values just before they are replaced are compared with the
// means and the 8 children's TEE tags written

template <typename T>
struct RestrictArgs {
  const BoxDev* fboxes;
  const RestrictItem* items;
  const long long* off;
  int nitems;
  long long total;
  const T* fy;
  const BoxDev* cboxes;
  T* cy;
  const int* cbmap;
  int cbshift, cnbd;
  int gl;
  int ncomp;
  uint8_t* tee;      // fine level's TEE tags (null: no estimate)
  double eps[4];     // thresholds of psi1, psi2, Pi1, Pi2 (<= 0: left out)
  int* err;
};

template <typename T>
__global__ void restrict_kernel(const RestrictArgs<T> A) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < A.total; t += stride) {
    int lo = 0, hi = A.nitems - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const RestrictItem I = A.items[lo];
    const long long loc = t - A.off[lo];
    const int i = (int)(loc % I.n[0]);
    const int j = (int)((loc / I.n[0]) % I.n[1]);
    const int k = (int)(loc / ((long long)I.n[0] * I.n[1]));
    const BoxDev F = A.fboxes[I.fbox];
    const int gx = (F.lo[0] >> 1) + i, gy = (F.lo[1] >> 1) + j, gz = (F.lo[2] >> 1) + k;
    const int own = A.cbmap[((long long)(gz >> A.cbshift) * A.cnbd + (gy >> A.cbshift)) * A.cnbd + (gx >> A.cbshift)];
    if (own < 0) {
      atomicCAS(A.err, 0, DERR_RESTRICT);
      continue;
    }
    const BoxDev C = A.cboxes[own];
    const long long dsti = cell_index(C, A.gl, gx - C.lo[0], gy - C.lo[1], gz - C.lo[2]);
    const long long f000 = cell_index(F, A.gl, 2 * i, 2 * j, 2 * k);
    const long long sy = F.pitch, sz = (long long)F.pny * F.pitch;
    bool hit = false;
    for (int c = 0; c < A.ncomp; ++c) {
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
      if (A.tee != nullptr && c < 4 && A.eps[c] > 0.0) hit |= fabs((double)A.cy[dsti + c * C.cs] - s) > A.eps[c];
      A.cy[dsti + c * C.cs] = (T)s;
    }
    if (A.tee != nullptr) {
      const uint8_t tv = hit ? 1 : 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int fx = 2 * i + (a & 1), fy = 2 * j + ((a >> 1) & 1), fz = 2 * k + (a >> 2);
        A.tee[F.voff + ((long long)fz * F.n[1] + fy) * F.n[0] + fx] = tv;
      }
    }
  }
}

template <typename T>
static slh_status restrict_t(slh_ctx* c, int fl) {
  Level& F = c->lev[fl];
  Level& C = c->lev[fl - 1];
  if (F.nrcells == 0) return SLH_OK;
  RestrictArgs<T> A;
  A.fboxes = F.d_boxes;
  A.items = F.d_ritems;
  A.off = F.d_roff;
  A.nitems = F.nritems;
  A.total = F.nrcells;
  A.fy = static_cast<const T*>(F.buf[F.role_y]);
  A.cboxes = C.d_boxes;
  A.cy = static_cast<T*>(C.buf[C.role_y]);
  A.cbmap = C.d_bmap;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.cbshift = sh;
  A.cnbd = C.nb_dom;
  A.gl = c->g;
  A.ncomp = c->ncomp;
  A.tee = (c->tag_criteria & SLH_TAG_TEE) ? F.d_tee : nullptr;
  for (int q = 0; q < 4; ++q) A.eps[q] = c->te_crit[q];
  A.err = c->d_err;
  const int threads = 256;
  long long blocks = (F.nrcells + threads - 1) / threads;
  const long long cap = (long long)c->num_sms * 8;
  if (blocks > cap) blocks = cap;
  restrict_kernel<T><<<(int)blocks, threads, 0, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_restrict(slh_ctx* c, int fine_lev) {
  return c->prec == SLH_F64 ? restrict_t<double>(c, fine_lev) : restrict_t<float>(c, fine_lev);
}

// ---------------------------------------------------------------------------
// conformal time bookkeeping (FP64 on the device):
//   level 0: eta_start = eta;  eta = eta_start + dt_0
//   level l: eta_start = eta_start[l-1] + sub * dt_l;  eta = eta_start + dt_l

__global__ void time_begin_kernel(double* t, int lev, int sub, double dt_l) {
  double es;
  if (lev == 0) es = t[0];
  else es = t[2 * (lev - 1) + 1] + (double)sub * dt_l;
  t[2 * lev + 1] = es;
  t[2 * lev] = es + dt_l;
}

slh_status launch_time_begin(slh_ctx* c, int lev, int sub, double dt_l) {
  time_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_time, lev, sub, dt_l);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

}  // namespace slh

namespace slh {

// ---------------------------------------------------------------------------
// regrid fill (Sec. 2.3): each valid cell of a level's new boxes takes the
// old level's value where an old box covers it, else the prolongation of the
// coarser level's current state (every field); the Kahan compensation is
// carried over where covered and zero elsewhere.

template <typename T>
struct RegridFillArgs {
  const BoxDev* nboxes;
  int nnb;
  long long nvalid;
  T* ny;
  T* nc;                 // new Kahan buffer or null
  const BoxDev* oboxes;  // old level (null: none)
  const T* oy;
  const T* oc;
  const int* obmap;
  int nbd;               // blocks per axis of the level domain (old and new)
  const BoxDev* cboxes;  // coarser level
  const T* cy;
  const int* cbmap;
  int cnbd, cndom;
  int bshift;
  int gl;
  int itype;
  int ncomp;
  int* err;
};

template <typename T>
__global__ void regrid_fill_kernel(const RegridFillArgs<T> A) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < A.nvalid; t += stride) {
    int lo = 0, hi = A.nnb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.nboxes[mid].voff <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev B = A.nboxes[lo];
    const long long loc = t - B.voff;
    const int rx = (int)(loc % B.n[0]);
    const int ry = (int)((loc / B.n[0]) % B.n[1]);
    const int rz = (int)(loc / ((long long)B.n[0] * B.n[1]));
    const int gx = B.lo[0] + rx, gy = B.lo[1] + ry, gz = B.lo[2] + rz;
    const long long dst = cell_index(B, A.gl, rx, ry, rz);
    if (A.oboxes != nullptr) {
      const int own = A.obmap[((long long)(gz >> A.bshift) * A.nbd + (gy >> A.bshift)) * A.nbd + (gx >> A.bshift)];
      if (own >= 0) {
        const BoxDev O = A.oboxes[own];
        const long long src = cell_index(O, A.gl, gx - O.lo[0], gy - O.lo[1], gz - O.lo[2]);
        for (int c = 0; c < A.ncomp; ++c) {
          A.ny[dst + c * B.cs] = A.oy[src + c * O.cs];
          if (A.nc) A.nc[dst + c * B.cs] = A.oc ? A.oc[src + c * O.cs] : (T)0;
        }
        continue;
      }
    }
    const int Px = gx >> 1, Py = gy >> 1, Pz = gz >> 1;
    const int cx = gx & 1, cy = gy & 1, cz = gz & 1;
    const int rad = A.itype == 4 ? 2 : (A.itype == 2 ? 1 : 0);
    bool bad = false;
    // fields in groups of four (one stencil walk per group)
    for (int c0 = 0; c0 < A.ncomp; c0 += NCOMP) {
      double acc[NCOMP] = {0.0, 0.0, 0.0, 0.0};
      for (int oz = -rad; oz <= rad; ++oz) {
        const double wzv = pw(A.itype, cz, oz);
        const int qz = wrapi(Pz + oz, A.cndom);
        for (int oy = -rad; oy <= rad; ++oy) {
          const double wyv = pw(A.itype, cy, oy);
          const int qy = wrapi(Py + oy, A.cndom);
          for (int ox = -rad; ox <= rad; ++ox) {
            const double wxv = pw(A.itype, cx, ox);
            const int qx = wrapi(Px + ox, A.cndom);
            const int cown = A.cbmap[((long long)(qz >> A.bshift) * A.cnbd + (qy >> A.bshift)) * A.cnbd + (qx >> A.bshift)];
            if (cown < 0) {
              bad = true;
              continue;
            }
            const BoxDev C = A.cboxes[cown];
            const long long ci = cell_index(C, A.gl, qx - C.lo[0], qy - C.lo[1], qz - C.lo[2]) + c0 * C.cs;
            const double wgt = wzv * wyv * wxv;
#pragma unroll
            for (int c = 0; c < NCOMP; ++c) acc[c] += wgt * (double)A.cy[ci + c * C.cs];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) {
        A.ny[dst + (c0 + c) * B.cs] = (T)acc[c];
        if (A.nc) A.nc[dst + (c0 + c) * B.cs] = (T)0;
      }
    }
    if (bad) atomicCAS(A.err, 0, DERR_NESTING);
  }
}

template <typename T>
static slh_status regrid_fill_t(slh_ctx* c, int lev, Level& N, Level* O) {
  Level& C = c->lev[lev - 1];
  RegridFillArgs<T> A;
  A.nboxes = N.d_boxes;
  A.nnb = (int)N.boxes.size();
  A.nvalid = N.lay.nvalid;
  A.ny = static_cast<T*>(N.buf[N.role_y]);
  A.nc = static_cast<T*>(N.buf[SLH_BUF_C]);
  if (O != nullptr && O->defined) {
    A.oboxes = O->d_boxes;
    A.oy = static_cast<const T*>(O->buf[O->role_y]);
    A.oc = static_cast<const T*>(O->buf[SLH_BUF_C]);
    A.obmap = O->d_bmap;
  } else {
    A.oboxes = nullptr;
    A.oy = nullptr;
    A.oc = nullptr;
    A.obmap = nullptr;
  }
  A.nbd = N.nb_dom;
  A.cboxes = C.d_boxes;
  A.cy = static_cast<const T*>(C.buf[C.role_y]);
  A.cbmap = C.d_bmap;
  A.cnbd = C.nb_dom;
  A.cndom = C.n_dom;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.bshift = sh;
  A.gl = c->g;
  A.itype = c->regrid_itype;
  A.ncomp = c->ncomp;
  A.err = c->d_err;
  const int threads = 256;
  long long blocks = (A.nvalid + threads - 1) / threads;
  const long long cap = (long long)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  regrid_fill_kernel<T><<<(int)blocks, threads, 0, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_regrid_fill(slh_ctx* c, int lev, Level& fresh, Level* old) {
  return c->prec == SLH_F64 ? regrid_fill_t<double>(c, lev, fresh, old) : regrid_fill_t<float>(c, lev, fresh, old);
}

}  // namespace slh
