// Inter-level transfer (Sec. 2.1): ghost fill of a level's psi components
// (and, with the gravitational-wave tensor, the six u_ij) from its own boxes (periodic wrap) or, where no box of the level covers a
// ghost cell, by ratio-2 prolongation of the coarser level interpolated in
// time; restriction of a fine level onto the covered coarse cells; and the
// small kernel that advances the per-level conformal time.
#include <cuda_bf16.h>

#include <cstring>

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

// SLH_F32_BF16 storage: two BF16 fields in one 4-byte slot (the first in
// the low half).  Widening is exact; narrowing rounds to nearest even.
__device__ __forceinline__ float bf16_half(float slot, int h) {
  const unsigned w = __float_as_uint(slot);
  return __uint_as_float(h ? (w & 0xFFFF0000u) : (w << 16));
}
__device__ __forceinline__ float bf16_pack(float lo, float hi) {
  const unsigned a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const unsigned b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return __uint_as_float(a | (b << 16));
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
// box lookup per coarse cell instead of one per stencil point), field by
// field, then apply the tensor-product stencil as three separable 1D passes
// (coarse -> fine along one axis per pass, thinnest region extent first, so
// the intermediate arrays stay small and no coarse cell's stencil is
// evaluated for children outside the region); mixed regions decide cell by
// cell in the last pass.
// Shared-memory buffers of a prolongation region of at most 32 x 32 x g fine
// cells (g <= 4): the coarse patch (radius-2 footprint: 21 coarse cells along
// a 32-cell axis, (g >> 1) + 5 along the thin one), the result of the pass
// along the thinnest axis (g fine x 21 x 21 coarse) and of the second pass
// (g x 32 x 21).  Sized by the level's g at launch, so that thin ghost
// shells leave room for more CTAs per SM.
__host__ __device__ constexpr int patch_max(int g) { return 21 * 21 * ((g >> 1) + 5); }
__host__ __device__ constexpr int pass1_max(int g) { return g * 21 * 21; }
__host__ __device__ constexpr int pass2_max(int g) { return g * 32 * 21; }

template <typename T>
struct GhostArgs {
  const BoxDev* boxes;
  const GhostRegion* regions;
  int r0, nregions;   // the region kernel takes regions [r0, nregions), the copy kernel [0, r0)
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
  int npairs;   // field pairs filled: (psi1, psi2), (Pi1, Pi2) under dissipation, and with 16
                // fields (u_xx, u_yy), (u_zz, u_xy), (u_xz, u_yz)
  int pc[5];    // first component of each pair (its slot, when packed)
  int packed;   // bit q: pair q is one slot of two BF16 fields (SLH_F32_BF16)
  int* err;
};


// geometry of a region's separable prolongation passes: the region's first
// fine cell (unwrapped), the coarse patch origin and the fine extents
struct PassGeo {
  int flo[3];
  int plo[3];
  int ext[3];
  int pn[3];
};

// Coverage of the coarse patch where the planned pieces do not tile it: one
// bit per patch cell, set where no coarse box holds the cell (its patch
// value is then 0).  The widest patch (g = 4) has 21 x 21 x 7 cells.
constexpr int UNC_WORDS = (21 * 21 * 7 + 31) / 32;

// Whether the radius-RAD stencil of the fine cell (unwrapped fine
// coordinates f) meets an uncovered patch cell.
template <int RAD>
__device__ __forceinline__ bool stencil_uncovered(const unsigned* unc, const PassGeo& geo, int fx, int fy, int fz) {
  const int px = (fx >> 1) - geo.plo[0], py = (fy >> 1) - geo.plo[1], pz = (fz >> 1) - geo.plo[2];
  for (int oz = -RAD; oz <= RAD; ++oz)
    for (int oy = -RAD; oy <= RAD; ++oy)
      for (int ox = -RAD; ox <= RAD; ++ox) {
        const int q = ((pz + oz) * geo.pn[1] + (py + oy)) * geo.pn[0] + (px + ox);
        if ((unc[q >> 5] >> (q & 31)) & 1u) return true;
      }
  return false;
}

template <int AX>
__device__ __forceinline__ int pick(int a, int b, int c) { return AX == 0 ? a : (AX == 1 ? b : c); }

// One coarse -> fine pass along axis AX over NF fields in shared memory
// (field f at src + f * sstr): input extents d (x, y, z), output extent
// geo.ext[AX] along AX; d is updated to the output extents.
template <typename T, int RAD, int AX, int NF>
__device__ __forceinline__ void smem_pass(const T* __restrict__ src, int sstr, T* __restrict__ dst, int dstr,
                                          int (&d)[3], const PassGeo& geo, const T (&w0)[2 * RAD + 1],
                                          const T (&w1)[2 * RAD + 1]) {
  const int o0 = AX == 0 ? geo.ext[0] : d[0], o1 = AX == 1 ? geo.ext[1] : d[1], o2 = AX == 2 ? geo.ext[2] : d[2];
  const int sa = AX == 0 ? 1 : (AX == 1 ? d[0] : d[0] * d[1]);
  const int fa = geo.flo[AX], pa = geo.plo[AX];
  const int nout = o0 * o1 * o2;
  const Split3 sp(o0, o1);
  for (int t = threadIdx.x; t < nout; t += blockDim.x) {
    int i0, i1, i2;
    sp(t, i0, i1, i2);
    const int g = fa + pick<AX>(i0, i1, i2);       // unwrapped fine coordinate along AX
    const int pc = (g >> 1) - pa - RAD;             // first stencil cell of the input along AX
    const bool ch = (g & 1) != 0;
    const int base = (pick<AX>(i2, i2, pc) * d[1] + pick<AX>(i1, pc, i1)) * d[0] + pick<AX>(pc, i0, i0);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T acc = 0;
#pragma unroll
      for (int o = 0; o <= 2 * RAD; ++o) acc += (ch ? w1[o] : w0[o]) * src[f * sstr + base + o * sa];
      dst[f * dstr + t] = acc;
    }
  }
  d[0] = o0;
  d[1] = o1;
  d[2] = o2;
}

template <typename T, int RAD, int NF>
__device__ __forceinline__ void smem_pass_any(int ax, const T* src, int sstr, T* dst, int dstr, int (&d)[3],
                                              const PassGeo& geo, const T (&w0)[2 * RAD + 1],
                                              const T (&w1)[2 * RAD + 1]) {
  if (ax == 0) smem_pass<T, RAD, 0, NF>(src, sstr, dst, dstr, d, geo, w0, w1);
  else if (ax == 1) smem_pass<T, RAD, 1, NF>(src, sstr, dst, dstr, d, geo, w0, w1);
  else smem_pass<T, RAD, 2, NF>(src, sstr, dst, dstr, d, geo, w0, w1);
}

// The last pass, along axis AX: writes the region's ghost cells of fields
// f0 .. f0+NF-1 (mixed regions copy the cells a same-level box covers).
template <typename T, int RAD, int AX, int NF>
__device__ __forceinline__ void final_pass(const T* __restrict__ src, int sstr, const int (&d)[3], const PassGeo& geo,
                                           const T (&w0)[2 * RAD + 1], const T (&w1)[2 * RAD + 1],
                                           const GhostArgs<T>& A, const GhostRegion& R, const BoxDev& B, int f0,
                                           bool have_coarse, const unsigned* unc) {
  const int o0 = AX == 0 ? geo.ext[0] : d[0], o1 = AX == 1 ? geo.ext[1] : d[1], o2 = AX == 2 ? geo.ext[2] : d[2];
  const int sa = AX == 0 ? 1 : (AX == 1 ? d[0] : d[0] * d[1]);
  const int fa = geo.flo[AX], pa = geo.plo[AX];
  const int nout = o0 * o1 * o2;
  const Split3 sp(o0, o1);
  for (int t = threadIdx.x; t < nout; t += blockDim.x) {
    int i0, i1, i2;
    sp(t, i0, i1, i2);
    const int rx = R.lo[0] + i0, ry = R.lo[1] + i1, rz = R.lo[2] + i2;
    const long long dg = cell_index(B, A.gl, rx, ry, rz);
    if (R.kind == GHOST_MIXED) {
      const int gx = B.lo[0] + rx, gy = B.lo[1] + ry, gz = B.lo[2] + rz;
      const int wx = wrapi(gx, A.ndom), wy = wrapi(gy, A.ndom), wz = wrapi(gz, A.ndom);
      const int own = A.bmap[((long long)(wz >> A.bshift) * A.nbd + (wy >> A.bshift)) * A.nbd + (wx >> A.bshift)];
      if (own >= 0) {
        const BoxDev Sb = A.boxes[own];
        const long long sg = cell_index(Sb, A.gl, wx - Sb.lo[0], wy - Sb.lo[1], wz - Sb.lo[2]);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int q = (f0 + f) >> 1;
          const bool pk = (A.packed >> q) & 1;
          if (pk && ((f0 + f) & 1)) continue;   // a packed pair is one slot
          const int comp = A.pc[q] + (pk ? 0 : ((f0 + f) & 1));
          A.y[dg + comp * B.cs] = A.y[sg + comp * Sb.cs];
        }
        continue;
      }
    }
    if (!have_coarse) {
      atomicCAS(A.err, 0, DERR_NESTING);
      continue;
    }
    // a stencil that reaches a coarse cell no coarse box holds (the patch
    // was not tiled by the plan) is a nesting violation; field values, NaN
    // or infinite ones included, are never inspected
    if (unc != nullptr &&
        stencil_uncovered<RAD>(unc, geo, geo.flo[0] + i0, geo.flo[1] + i1, geo.flo[2] + i2)) {
      atomicCAS(A.err, 0, DERR_NESTING);
      continue;
    }
    const int g = fa + pick<AX>(i0, i1, i2);
    const int pc = (g >> 1) - pa - RAD;
    const bool ch = (g & 1) != 0;
    const int base = (pick<AX>(i2, i2, pc) * d[1] + pick<AX>(i1, pc, i1)) * d[0] + pick<AX>(pc, i0, i0);
    T acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      acc[f] = 0;
#pragma unroll
      for (int o = 0; o <= 2 * RAD; ++o) acc[f] += (ch ? w1[o] : w0[o]) * src[f * sstr + base + o * sa];
    }
    if constexpr (NF == 2) {
      if ((A.packed >> (f0 >> 1)) & 1) {   // both fields of a packed pair: one slot
        A.y[dg + A.pc[f0 >> 1] * B.cs] = (T)bf16_pack((float)acc[0], (float)acc[1]);
        continue;
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int comp = A.pc[(f0 + f) >> 1] + ((f0 + f) & 1);
      A.y[dg + comp * B.cs] = acc[f];
    }
  }
}

template <typename T, int RAD, int NF>
__device__ __forceinline__ void final_pass_any(int ax, const T* src, int sstr, const int (&d)[3], const PassGeo& geo,
                                               const T (&w0)[2 * RAD + 1], const T (&w1)[2 * RAD + 1],
                                               const GhostArgs<T>& A, const GhostRegion& R, const BoxDev& B, int f0,
                                               bool have_coarse, const unsigned* unc) {
  if (ax == 0) final_pass<T, RAD, 0, NF>(src, sstr, d, geo, w0, w1, A, R, B, f0, have_coarse, unc);
  else if (ax == 1) final_pass<T, RAD, 1, NF>(src, sstr, d, geo, w0, w1, A, R, B, f0, have_coarse, unc);
  else final_pass<T, RAD, 2, NF>(src, sstr, d, geo, w0, w1, A, R, B, f0, have_coarse, unc);
}

// Same-level copy regions [0, r0): no shared memory, so many CTAs per SM
// keep loads in flight; each thread reads CU cells of every field pair
// before writing them (source and destination cells never overlap: the
// source is valid cells of a box, the destination ghost cells).
template <typename T>
__global__ void __launch_bounds__(256, 4) ghost_copy_kernel(const GhostArgs<T> A) {
  constexpr int CU = 4;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int r = blockIdx.x; r < A.r0; r += gridDim.x) {
    const GhostRegion R = A.regions[r];
    const BoxDev B = A.boxes[R.box];
    const BoxDev S = A.boxes[R.src];
    const int ncell = R.ext[0] * R.ext[1] * R.ext[2];
    const Split3 sp(R.ext[0], R.ext[1]);
    for (int t0 = tid; t0 < ncell; t0 += CU * nt) {
      long long dst[CU], src[CU];
      bool ok[CU];
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int t = t0 + u * nt;
        ok[u] = t < ncell;
        int i = 0, j = 0, k = 0;
        if (ok[u]) sp(t, i, j, k);
        const int rx = R.lo[0] + i, ry = R.lo[1] + j, rz = R.lo[2] + k;
        dst[u] = cell_index(B, A.gl, rx, ry, rz);
        src[u] = cell_index(S, A.gl, rx + R.d[0], ry + R.d[1], rz + R.d[2]);
      }
      for (int q = 0; q < A.npairs; ++q) {
        const int c0 = A.pc[q];
        const bool two = !((A.packed >> q) & 1);   // a packed pair is one slot
        T v0[CU], v1[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u)
          if (ok[u]) {
            v0[u] = A.y[src[u] + c0 * S.cs];
            if (two) v1[u] = A.y[src[u] + (c0 + 1) * S.cs];
          }
#pragma unroll
        for (int u = 0; u < CU; ++u)
          if (ok[u]) {
            A.y[dst[u] + c0 * B.cs] = v0[u];
            if (two) A.y[dst[u] + (c0 + 1) * B.cs] = v1[u];
          }
      }
    }
  }
}

template <typename T, int RAD>
__global__ void __launch_bounds__(256, 5) ghost_region_kernel(const GhostArgs<T> A) {
  // [2][pz][py][px]: time-interpolated psi1, psi2 in the field precision
  // (the stencil weights are dyadic rationals, exact in FP32 and FP64)
  extern __shared__ __align__(16) unsigned char patch_raw[];
  constexpr int NF = sizeof(T) == 4 ? 2 : 1;   // fields per pass (shared memory ~60 KB either way)
  T* patch = reinterpret_cast<T*>(patch_raw);
  const int PATCH_MAX = patch_max(A.gl), PASS1_MAX = pass1_max(A.gl), PASS2_MAX = pass2_max(A.gl);
  T* buf1 = patch + NF * PATCH_MAX;
  T* buf2 = buf1 + NF * PASS1_MAX;
  __shared__ unsigned s_unc[UNC_WORDS];
  const int tid = threadIdx.x, nt = blockDim.x;
  const T al = (T)A.alpha, bl = (T)1 - (T)A.alpha;
  T w0[2 * RAD + 1], w1[2 * RAD + 1];   // 1D weights of child 0 and child 1
#pragma unroll
  for (int o = -RAD; o <= RAD; ++o) {
    w0[o + RAD] = (T)pw(A.itype, 0, o);
    w1[o + RAD] = (T)pw(A.itype, 1, o);
  }
  for (int r = A.r0 + blockIdx.x; r < A.nregions; r += gridDim.x) {
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
          const int c0 = A.pc[q];
          A.y[dst + c0 * B.cs] = A.y[src + c0 * S.cs];
          if (!((A.packed >> q) & 1)) A.y[dst + (c0 + 1) * B.cs] = A.y[src + (c0 + 1) * S.cs];
        }
      }
      continue;   // uniform over the CTA: no shared memory used
    }
    // coarse footprint of the widest stencil (unwrapped coarse coordinates);
    // narrower stencils use part of it
    int flo[3], plo[3], pn[3];
    for (int d = 0; d < 3; ++d) {
      flo[d] = B.lo[d] + R.lo[d];
      const int fhi = flo[d] + R.ext[d] - 1;
      plo[d] = (flo[d] >> 1) - PROLONG_RAD_MAX;
      pn[d] = (fhi >> 1) + PROLONG_RAD_MAX - plo[d] + 1;
    }
    const int np = pn[0] * pn[1] * pn[2];
    const bool have_coarse = A.cboxes != nullptr && np <= PATCH_MAX;
    // the three separable passes go thinnest fine extent first, so that the
    // intermediate arrays stay small (a slab is at most g <= 4 cells thick)
    const int ex0 = R.ext[0], ex1 = R.ext[1], ex2 = R.ext[2];
    auto ext_of = [&](int a) { return a == 0 ? ex0 : (a == 1 ? ex1 : ex2); };
    int a0 = 0, a1 = 1, a2 = 2;
    if (ext_of(a1) < ext_of(a0)) { const int s_ = a0; a0 = a1; a1 = s_; }
    if (ext_of(a2) < ext_of(a1)) { const int s_ = a1; a1 = a2; a2 = s_; }
    if (ext_of(a1) < ext_of(a0)) { const int s_ = a0; a0 = a1; a1 = s_; }
    const PassGeo geo{{flo[0], flo[1], flo[2]}, {plo[0], plo[1], plo[2]}, {ex0, ex1, ex2}, {pn[0], pn[1], pn[2]}};
    // patch not tiled by the planned pieces (uniform over the CTA): the
    // gather looks every cell up and marks the uncovered ones
    const bool lookup = have_coarse && !R.covered;
    if (lookup) {
      for (int w = tid; w < UNC_WORDS; w += nt) s_unc[w] = 0u;
      __syncthreads();
    }
    for (int f0 = 0; f0 < 2 * A.npairs; f0 += NF) {
      // gather NF fields into the patch (field f of the region's pair list)
      for (int f = 0; f < NF; ++f) {
        const int q = (f0 + f) >> 1, half = (f0 + f) & 1;
        const bool pk = sizeof(T) == 4 && ((A.packed >> q) & 1);
        const int comp = A.pc[q] + (pk ? 0 : half);
        // a field value of the coarse level, time-interpolated
        auto cval = [&](long long ci) -> T {
          if constexpr (sizeof(T) == 4) {
            if (pk) return bl * (T)bf16_half((float)A.cold[ci], half) + al * (T)bf16_half((float)A.cnew[ci], half);
          }
          return bl * A.cold[ci] + al * A.cnew[ci];
        };
        T* pf = patch + f * PATCH_MAX;
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
              const long long ci = cell_index(C, A.gl, P.src[0] + i, P.src[1] + j, P.src[2] + k) + comp * C.cs;
              pf[((P.dst[2] + k) * pn[1] + (P.dst[1] + j)) * pn[0] + (P.dst[0] + i)] = cval(ci);
            }
          }
        } else if (have_coarse) {
          // footprint not tiled by the coarse level (a nesting violation, or a
          // level built without a plan): per-cell lookup; an uncovered cell
          // reads 0 and is marked in s_unc
          const Split3 sp(pn[0], pn[1]);
#pragma unroll 4
          for (int t = tid; t < np; t += nt) {
            int i, j, k;
            sp(t, i, j, k);
            const int qx = wrapi(plo[0] + i, A.cndom), qy = wrapi(plo[1] + j, A.cndom), qz = wrapi(plo[2] + k, A.cndom);
            const int cown = A.cbmap[((long long)(qz >> A.bshift) * A.cnbd + (qy >> A.bshift)) * A.cnbd + (qx >> A.bshift)];
            T v = 0;
            if (cown >= 0) {
              const BoxDev C = A.cboxes[cown];
              const long long ci = cell_index(C, A.gl, qx - C.lo[0], qy - C.lo[1], qz - C.lo[2]) + comp * C.cs;
              v = cval(ci);
            } else if (f == 0 && f0 == 0) {
              atomicOr(&s_unc[t >> 5], 1u << (t & 31));
            }
            pf[t] = v;
          }
        }
      }
      __syncthreads();
      // passes: coarse -> fine along a0 (patch -> buf1), a1 (buf1 -> buf2),
      // a2 (buf2 -> the ghost cells)
      int d[3] = {pn[0], pn[1], pn[2]};
      if (have_coarse) {
        smem_pass_any<T, RAD, NF>(a0, patch, PATCH_MAX, buf1, PASS1_MAX, d, geo, w0, w1);
        __syncthreads();
        smem_pass_any<T, RAD, NF>(a1, buf1, PASS1_MAX, buf2, PASS2_MAX, d, geo, w0, w1);
        __syncthreads();
      } else {
        d[0] = ex0;   // no coarse data: the last pass only copies or flags
        d[1] = ex1;
        d[2] = ex2;
      }
      final_pass_any<T, RAD, NF>(a2, buf2, PASS2_MAX, d, geo, w0, w1, A, R, B, f0, have_coarse,
                                 lookup ? s_unc : nullptr);
      __syncthreads();   // the buffers are reused by the next fields or region
    }
  }
}

// Prolongation regions [r0, nregions) of a fill whose prolonged values are
// already known: they are copied cell by cell from buffer ysrc of the same
// level, which a fill with the same coarse data and time fraction wrote
// (nothing to copy when ysrc is the buffer itself); cells of mixed regions
// that a box of the level covers are copied from that box, as the
// prolongation kernel does.
template <typename T>
__global__ void __launch_bounds__(256, 4) ghost_reuse_kernel(const GhostArgs<T> A, const T* __restrict__ ysrc) {
  constexpr int CU = 4;
  const bool same = ysrc == A.y;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int r = A.r0 + blockIdx.x; r < A.nregions; r += gridDim.x) {
    const GhostRegion R = A.regions[r];
    if (same && R.kind != GHOST_MIXED) continue;
    const BoxDev B = A.boxes[R.box];
    const int ncell = R.ext[0] * R.ext[1] * R.ext[2];
    const Split3 sp(R.ext[0], R.ext[1]);
    if (R.kind != GHOST_MIXED) {
      // a pure prolongation region: every cell from ysrc, CU cells per
      // thread in flight (source and destination buffers differ)
      for (int t0 = tid; t0 < ncell; t0 += CU * nt) {
        long long dg[CU];
        bool ok[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u) {
          const int t = t0 + u * nt;
          ok[u] = t < ncell;
          int i = 0, j = 0, k = 0;
          if (ok[u]) sp(t, i, j, k);
          dg[u] = cell_index(B, A.gl, R.lo[0] + i, R.lo[1] + j, R.lo[2] + k);
        }
        for (int q = 0; q < A.npairs; ++q) {
          const long long o0 = A.pc[q] * B.cs, o1 = o0 + B.cs;
          const bool two = !((A.packed >> q) & 1);   // a packed pair is one slot
          T v0[CU], v1[CU];
#pragma unroll
          for (int u = 0; u < CU; ++u)
            if (ok[u]) {
              v0[u] = ysrc[dg[u] + o0];
              if (two) v1[u] = ysrc[dg[u] + o1];
            }
#pragma unroll
          for (int u = 0; u < CU; ++u)
            if (ok[u]) {
              A.y[dg[u] + o0] = v0[u];
              if (two) A.y[dg[u] + o1] = v1[u];
            }
        }
      }
      continue;
    }
    for (int t = tid; t < ncell; t += nt) {
      int i, j, k;
      sp(t, i, j, k);
      const int rx = R.lo[0] + i, ry = R.lo[1] + j, rz = R.lo[2] + k;
      const long long dg = cell_index(B, A.gl, rx, ry, rz);
      const int gx = B.lo[0] + rx, gy = B.lo[1] + ry, gz = B.lo[2] + rz;
      const int wx = wrapi(gx, A.ndom), wy = wrapi(gy, A.ndom), wz = wrapi(gz, A.ndom);
      const int own = A.bmap[((long long)(wz >> A.bshift) * A.nbd + (wy >> A.bshift)) * A.nbd + (wx >> A.bshift)];
      const T* src;
      long long sg;
      if (own >= 0) {   // a box of the level covers the cell: its current value
        const BoxDev& Sb = A.boxes[own];
        src = A.y;
        sg = cell_index(Sb, A.gl, wx - Sb.lo[0], wy - Sb.lo[1], wz - Sb.lo[2]);
        for (int q = 0; q < A.npairs; ++q) {
          const int c0 = A.pc[q];
          A.y[dg + c0 * B.cs] = src[sg + c0 * Sb.cs];
          if (!((A.packed >> q) & 1)) A.y[dg + (c0 + 1) * B.cs] = src[sg + (c0 + 1) * Sb.cs];
        }
        continue;
      }
      if (same) continue;
      for (int q = 0; q < A.npairs; ++q) {
        const int c0 = A.pc[q];
        A.y[dg + c0 * B.cs] = ysrc[dg + c0 * B.cs];
        if (!((A.packed >> q) & 1)) A.y[dg + (c0 + 1) * B.cs] = ysrc[dg + (c0 + 1) * B.cs];
      }
    }
  }
}

template <typename T>
static slh_status ghosts_t(slh_ctx* c, int lev, int role, double alpha, int itype, bool with_pi) {
  Level& L = c->lev[lev];
  if (L.ngregions == 0) return SLH_OK;
  GhostArgs<T> A;
  A.boxes = L.d_boxes;
  A.regions = L.d_gregions;
  A.r0 = L.ncopyregions;
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
  A.npairs = 0;
  A.packed = 0;
  A.pc[A.npairs++] = 0;
  if (with_pi) A.pc[A.npairs++] = 2;
  if (c->ncomp == NCOMP_GW)
    for (int q = 0; q < 3; ++q) {
      if (c->prec == SLH_F32_BF16) A.packed |= 1 << A.npairs;
      A.pc[A.npairs] = c->prec == SLH_F32_BF16 ? SLOT_U0 + q : GW_U0 + 2 * q;
      ++A.npairs;
    }
  A.err = c->d_err;
  const int smem = (sizeof(T) == 4 ? 2 : 1) * (patch_max(c->g) + pass1_max(c->g) + pass2_max(c->g)) * (int)sizeof(T);
  const int smem_max = (sizeof(T) == 4 ? 2 : 1) * (patch_max(4) + pass1_max(4) + pass2_max(4)) * (int)sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ghost_region_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaFuncSetAttribute(ghost_region_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaFuncSetAttribute(ghost_region_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    attr = true;
  }
  // many more CTAs than resident slots: regions cost very different
  // amounts, and the block scheduler evens them out
  const long long cap = (long long)c->num_sms * 16;
  if (A.r0 > 0) {
    const long long blocks = std::min<long long>(A.r0, cap);
    ghost_copy_kernel<T><<<(int)blocks, 256, 0, c->stream>>>(A);
    SLH_CUDA(cudaGetLastError());
  }
  if (A.nregions > A.r0) {
    const long long blocks = std::min<long long>(A.nregions - A.r0, cap);
    if (itype == 4) ghost_region_kernel<T, 2><<<(int)blocks, 256, smem, c->stream>>>(A);
    else if (itype == 2) ghost_region_kernel<T, 1><<<(int)blocks, 256, smem, c->stream>>>(A);
    else ghost_region_kernel<T, 0><<<(int)blocks, 256, smem, c->stream>>>(A);
    SLH_CUDA(cudaGetLastError());
  }
  return SLH_OK;
}

slh_status launch_ghosts(slh_ctx* c, int lev, int role, double alpha, int itype, bool with_pi) {
  if (itype != 0 && itype != 2 && itype != 4)
    return fail(SLH_ERR_INVALID_ARG, "interp_type must be 0, 2 or 4 (got %d)", itype);
  return c->prec == SLH_F64 ? ghosts_t<double>(c, lev, role, alpha, itype, with_pi)
                            : ghosts_t<float>(c, lev, role, alpha, itype, with_pi);
}

template <typename T>
static slh_status ghosts_reuse_t(slh_ctx* c, int lev, int role, int src, bool with_pi) {
  Level& L = c->lev[lev];
  if (L.ngregions == 0) return SLH_OK;
  GhostArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.boxes = L.d_boxes;
  A.regions = L.d_gregions;
  A.r0 = L.ncopyregions;
  A.nregions = L.ngregions;
  A.y = static_cast<T*>(L.buf[role]);
  A.gl = c->g;
  A.bmap = L.d_bmap;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.bshift = sh;
  A.nbd = L.nb_dom;
  A.ndom = L.n_dom;
  A.pc[A.npairs++] = 0;
  if (with_pi) A.pc[A.npairs++] = 2;
  if (c->ncomp == NCOMP_GW)
    for (int q = 0; q < 3; ++q) {
      if (c->prec == SLH_F32_BF16) A.packed |= 1 << A.npairs;
      A.pc[A.npairs] = c->prec == SLH_F32_BF16 ? SLOT_U0 + q : GW_U0 + 2 * q;
      ++A.npairs;
    }
  A.err = c->d_err;
  const long long cap = (long long)c->num_sms * 16;
  if (A.r0 > 0) {
    ghost_copy_kernel<T><<<(int)std::min<long long>(A.r0, cap), 256, 0, c->stream>>>(A);
    SLH_CUDA(cudaGetLastError());
  }
  if (A.nregions > A.r0) {
    ghost_reuse_kernel<T><<<(int)std::min<long long>(A.nregions - A.r0, cap), 256, 0, c->stream>>>(
        A, static_cast<const T*>(L.buf[src]));
    SLH_CUDA(cudaGetLastError());
  }
  return SLH_OK;
}

slh_status launch_ghosts_reuse(slh_ctx* c, int lev, int role, int src, bool with_pi) {
  return c->prec == SLH_F64 ? ghosts_reuse_t<double>(c, lev, role, src, with_pi)
                            : ghosts_reuse_t<float>(c, lev, role, src, with_pi);
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
  const int2* chunks;    // (item, first coarse cell) of each chunk
  int nchunks;
  const T* fy;
  const BoxDev* cboxes;
  T* cy;
  const int* cbmap;
  int cbshift, cnbd;
  int gl;
  int ncomp;         // leading components of the field precision
  int npacked;       // then slots of two BF16 fields each (SLH_F32_BF16)
  uint8_t* tee;      // fine level's TEE tags (null: no estimate)
  double eps[4];     // thresholds of psi1, psi2, Pi1, Pi2 (<= 0: left out)
  int* err;
};

// FP32 -> FP64 widening (exact) in integer arithmetic for zeros and normal
// numbers, which GB300 would otherwise convert on its 1/62-rate FP64 pipe;
// subnormals, Inf and NaN take the conversion instruction.
__device__ __forceinline__ double widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u)   // normal: rebias the exponent, move the 23 fraction bits up by 29
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
  if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)v;
}
__device__ __forceinline__ double widen(double v) { return v; }

template <typename T>
__global__ void __launch_bounds__(RESTRICT_CHUNK) restrict_kernel(const RestrictArgs<T> A) {
  // a CTA takes chunks of RESTRICT_CHUNK consecutive coarse cells of one
  // fine box (x fastest), a thread one cell of the chunk
  for (int ck = blockIdx.x; ck < A.nchunks; ck += gridDim.x) {
    const int2 chunk = A.chunks[ck];
    const RestrictItem I = A.items[chunk.x];
    const int loc = chunk.y + (int)threadIdx.x;
    if (loc >= I.n[0] * I.n[1] * I.n[2]) continue;
    const int i = loc % I.n[0];
    const int j = (loc / I.n[0]) % I.n[1];
    const int k = loc / (I.n[0] * I.n[1]);
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
      double s = widen(f[0]);
      s += widen(f[1]);
      s += widen(f[sy]);
      s += widen(f[sy + 1]);
      s += widen(f[sz]);
      s += widen(f[sz + 1]);
      s += widen(f[sz + sy]);
      s += widen(f[sz + sy + 1]);
      s *= 0.125;
      if (A.tee != nullptr && c < 4 && A.eps[c] > 0.0) hit |= fabs((double)A.cy[dsti + c * C.cs] - s) > A.eps[c];
      A.cy[dsti + c * C.cs] = (T)s;
    }
    if constexpr (sizeof(T) == 4) {
      for (int c = A.ncomp; c < A.ncomp + A.npacked; ++c) {
        const T* f = A.fy + f000 + c * F.cs;
        const long long off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          s0 += widen(bf16_half(f[off[a]], 0));
          s1 += widen(bf16_half(f[off[a]], 1));
        }
        A.cy[dsti + c * C.cs] = bf16_pack((float)(s0 * 0.125), (float)(s1 * 0.125));
      }
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
  A.chunks = F.d_rchunks;
  A.nchunks = F.nrchunks;
  A.fy = static_cast<const T*>(F.buf[F.role_y]);
  A.cboxes = C.d_boxes;
  A.cy = static_cast<T*>(C.buf[C.role_y]);
  A.cbmap = C.d_bmap;
  int sh = 0;
  while ((1 << sh) < c->bf) ++sh;
  A.cbshift = sh;
  A.cnbd = C.nb_dom;
  A.gl = c->g;
  A.ncomp = c->prec == SLH_F32_BF16 ? NCOMP : c->ncomp;
  A.npacked = c->prec == SLH_F32_BF16 ? c->nslots - NCOMP : 0;
  A.tee = (c->tag_criteria & SLH_TAG_TEE) ? F.d_tee : nullptr;
  for (int q = 0; q < 4; ++q) A.eps[q] = c->te_crit[q];
  A.err = c->d_err;
  const int blocks = std::min(F.nrchunks, c->num_sms * 8);
  restrict_kernel<T><<<blocks, RESTRICT_CHUNK, 0, c->stream>>>(A);
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
  const int4* items;     // column items (box, x0, y0, z0) of the new level
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
  int ncomp;             // slots per cell (copied bit for bit)
  int nscalar;           // of which the leading ones hold one field of the precision;
                         // the rest (SLH_F32_BF16) two BF16 fields each
  int* err;
};

// One CTA of COL_TX x COL_TY threads per column item of the new level, a
// thread per cell column (no index division).  Prolonged cells sum the
// tensor-product stencil in the field precision (FP64 for FP64 levels, FP32
// otherwise, as the ghost prolongation does; the weights are dyadic and exact
// in both); where the stencil's coarse footprint lies inside one coarse box
// it is addressed linearly from one lookup, else cell by cell with the
// periodic wrap.
template <typename T>
__global__ void __launch_bounds__(COL_TX * COL_TY) regrid_fill_kernel(const RegridFillArgs<T> A) {
  using Acc = T;
  const int4 it = A.items[blockIdx.x];
  const BoxDev B = A.nboxes[it.x];
  const int rx = it.y + threadIdx.x, ry = it.z + threadIdx.y;
  if (rx >= B.n[0] || ry >= B.n[1]) return;
  const int z1 = min(it.w + COL_ZLEN, B.n[2]);
  const int gx = B.lo[0] + rx, gy = B.lo[1] + ry;
  const int rad = A.itype == 4 ? 2 : (A.itype == 2 ? 1 : 0);
  const int Px = gx >> 1, Py = gy >> 1, cx = gx & 1, cy = gy & 1;
  Acc wx[5], wy[5];
#pragma unroll
  for (int o = -2; o <= 2; ++o) {
    wx[o + 2] = (Acc)pw(A.itype, cx, o);
    wy[o + 2] = (Acc)pw(A.itype, cy, o);
  }
  bool bad = false;
#pragma unroll 1
  for (int rz = it.w; rz < z1; ++rz) {
    const int gz = B.lo[2] + rz;
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
    const int Pz = gz >> 1, cz = gz & 1;
    // the coarse box holding the whole footprint, if one does
    const int own0 = A.cbmap[((long long)(Pz >> A.bshift) * A.cnbd + (Py >> A.bshift)) * A.cnbd + (Px >> A.bshift)];
    BoxDev C0;
    bool inside = false;
    if (own0 >= 0) {
      C0 = A.cboxes[own0];
      inside = Px - rad >= C0.lo[0] && Px + rad < C0.lo[0] + C0.n[0] && Py - rad >= C0.lo[1] &&
               Py + rad < C0.lo[1] + C0.n[1] && Pz - rad >= C0.lo[2] && Pz + rad < C0.lo[2] + C0.n[2];
    }
    // one stencil walk per group of four values: four slots of one field
    // each, then (SLH_F32_BF16) two slots of two BF16 fields each; the same
    // summation order on both paths
    auto add = [&](const T* q, long long cs, Acc wgt, bool pk, Acc (&acc)[NCOMP]) {
      if (pk) {
        const float v0 = (float)q[0], v1 = (float)q[cs];
        acc[0] += wgt * (Acc)bf16_half(v0, 0);
        acc[1] += wgt * (Acc)bf16_half(v0, 1);
        acc[2] += wgt * (Acc)bf16_half(v1, 0);
        acc[3] += wgt * (Acc)bf16_half(v1, 1);
      } else {
#pragma unroll
        for (int c = 0; c < NCOMP; ++c) acc[c] += wgt * (Acc)q[c * cs];
      }
    };
    auto walk = [&](int c0, bool pk, Acc (&acc)[NCOMP]) {
      if (inside) {
        const long long sy = C0.pitch, sz = (long long)C0.pitch * C0.pny;
        const T* base = A.cy + cell_index(C0, A.gl, Px - C0.lo[0], Py - C0.lo[1], Pz - C0.lo[2]) + c0 * C0.cs;
#pragma unroll 1
        for (int oz = -rad; oz <= rad; ++oz) {
          const Acc wzv = (Acc)pw(A.itype, cz, oz);
#pragma unroll 1
          for (int oy = -rad; oy <= rad; ++oy) {
            const Acc wyz = wzv * wy[oy + 2];
            const T* rowp = base + oz * sz + oy * sy;
            for (int ox = -rad; ox <= rad; ++ox) add(rowp + ox, C0.cs, wyz * wx[ox + 2], pk, acc);
          }
        }
        return;
      }
#pragma unroll 1
      for (int oz = -rad; oz <= rad; ++oz) {
        const Acc wzv = (Acc)pw(A.itype, cz, oz);
        const int qz = wrapi(Pz + oz, A.cndom);
#pragma unroll 1
        for (int oy = -rad; oy <= rad; ++oy) {
          const Acc wyz = wzv * wy[oy + 2];
          const int qy = wrapi(Py + oy, A.cndom);
#pragma unroll 1
          for (int ox = -rad; ox <= rad; ++ox) {
            const int qx = wrapi(Px + ox, A.cndom);
            const int cown = A.cbmap[((long long)(qz >> A.bshift) * A.cnbd + (qy >> A.bshift)) * A.cnbd + (qx >> A.bshift)];
            if (cown < 0) {
              bad = true;
              continue;
            }
            const BoxDev& C = A.cboxes[cown];
            add(A.cy + cell_index(C, A.gl, qx - C.lo[0], qy - C.lo[1], qz - C.lo[2]) + c0 * C.cs, C.cs,
                wyz * wx[ox + 2], pk, acc);
          }
        }
      }
    };
#pragma unroll 1
    for (int c0 = 0; c0 < A.nscalar; c0 += NCOMP) {
      Acc acc[NCOMP] = {0, 0, 0, 0};
      walk(c0, false, acc);
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) {
        A.ny[dst + (c0 + c) * B.cs] = (T)acc[c];
        if (A.nc) A.nc[dst + (c0 + c) * B.cs] = (T)0;
      }
    }
    if constexpr (sizeof(T) == 4) {
      // packed slots come in pairs (SLH_SLOTS_BF16 - 4 = 6)
#pragma unroll 1
      for (int c0 = A.nscalar; c0 + 1 < A.ncomp; c0 += 2) {
        Acc acc[NCOMP] = {0, 0, 0, 0};
        walk(c0, true, acc);
        A.ny[dst + c0 * B.cs] = bf16_pack((float)acc[0], (float)acc[1]);
        A.ny[dst + (c0 + 1) * B.cs] = bf16_pack((float)acc[2], (float)acc[3]);
      }
    }
  }
  if (bad) atomicCAS(A.err, 0, DERR_NESTING);
}

template <typename T>
static slh_status regrid_fill_t(slh_ctx* c, int lev, Level& N, Level* O) {
  Level& C = c->lev[lev - 1];
  RegridFillArgs<T> A;
  A.nboxes = N.d_boxes;
  A.items = N.d_col_items;
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
  A.ncomp = c->nslots;
  A.nscalar = c->prec == SLH_F32_BF16 ? NCOMP : c->nslots;
  A.err = c->d_err;
  if (N.ncol_items < 1) return SLH_OK;
  regrid_fill_kernel<T><<<N.ncol_items, dim3(COL_TX, COL_TY), 0, c->stream>>>(A);
  SLH_CUDA(cudaGetLastError());
  return SLH_OK;
}

slh_status launch_regrid_fill(slh_ctx* c, int lev, Level& fresh, Level* old) {
  return c->prec == SLH_F64 ? regrid_fill_t<double>(c, lev, fresh, old) : regrid_fill_t<float>(c, lev, fresh, old);
}

}  // namespace slh
