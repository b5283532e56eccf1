// Gravitational-wave spectrum of level 0 (Sec. 7.4, Eq. gw_spectrum):
//   G(n^2) = N^-6 sum_{|n(k)|^2 = n^2} Lambda_ij,lm(k) v~_ij(k) v~*_lm(k)
// with Lambda_ij,lm = P_il P_jm - P_ij P_lm / 2 (Sec. 5, Eq. Lambda_ijlm),
// P = 1 - khat khat^T, khat the unit effective lattice momentum of
// projection type 1 (sin(theta)/dx) or 2 ((8 sin(theta) - sin(2 theta))/(6 dx)),
// khat = 0 where it vanishes.  The six v_ij of the level's boxes are gathered
// into dense N^3 arrays, transformed by a batched real-to-complex FFT
// (cuFFT, the library's plain FFT).  The contraction of each mode of the
// half spectrum (weight 2 for the modes whose conjugate partner is not
// stored) is summed into FP64 bins indexed by n^2 in a fixed order, so the
// spectrum is bit-reproducible run to run: the rows (ky, kz) of the half
// spectrum are grouped by q = sy^2 + sz^2 (signed frequencies); one thread
// per (q, kx) sums the modes of its rows in a fixed row order into
// S[q][kx], and one thread per bin adds S[n^2 - kx^2][kx] over kx in
// ascending order (within one row every kx has its own n^2, so each mode
// lands in exactly one S entry).  The contraction is evaluated as
// Re tr(P V P V*) - |tr(P V)|^2 / 2 for the symmetric complex 3x3 matrix V
// of the mode.
#include <cufft.h>
#include <dlfcn.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "slh_internal.cuh"

namespace slh {

// --- cuFFT, resolved on first use (the rest of the library does not need it)
struct CufftApi {
  cufftResult (*plan_many)(cufftHandle*, int, int*, int*, int, int, int*, int, int, cufftType, int) = nullptr;
  cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
  cufftResult (*exec_r2c)(cufftHandle, cufftReal*, cufftComplex*) = nullptr;
  cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal*, cufftDoubleComplex*) = nullptr;
  cufftResult (*destroy)(cufftHandle) = nullptr;
  bool ok = false;
};

static const CufftApi& cufft_api() {
  static CufftApi api;
  static std::once_flag once;
  std::call_once(once, [] {
    // by soname, through the dynamic loader's search path
    const char* names[] = {"libcufft.so.12", "libcufft.so"};
    void* h = nullptr;
    for (const char* n : names)
      if ((h = dlopen(n, RTLD_NOW | RTLD_GLOBAL)) != nullptr) break;
    if (!h) return;
    api.plan_many = reinterpret_cast<decltype(api.plan_many)>(dlsym(h, "cufftPlanMany"));
    api.set_stream = reinterpret_cast<decltype(api.set_stream)>(dlsym(h, "cufftSetStream"));
    api.exec_r2c = reinterpret_cast<decltype(api.exec_r2c)>(dlsym(h, "cufftExecR2C"));
    api.exec_d2z = reinterpret_cast<decltype(api.exec_d2z)>(dlsym(h, "cufftExecD2Z"));
    api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "cufftDestroy"));
    api.ok = api.plan_many && api.set_stream && api.exec_r2c && api.exec_d2z && api.destroy;
  });
  return api;
}

// --- gather v_ij of a level into dense [6][N][N][N] arrays
template <typename T>
__global__ void gather_v_kernel(const BoxDev* boxes, int nboxes, long long nvalid, const T* y, int gl, int n,
                                T* out, int packed) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long n3 = (long long)n * n * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nvalid; t += stride) {
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (boxes[mid].voff <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev B = boxes[lo];
    const long long loc = t - B.voff;
    const int rx = (int)(loc % B.n[0]);
    const int ry = (int)((loc / B.n[0]) % B.n[1]);
    const int rz = (int)(loc / ((long long)B.n[0] * B.n[1]));
    const long long src = B.off + ((long long)(rz + gl) * B.pny + (ry + gl)) * B.pitch + (rx + XPAD);
    const long long dst = ((long long)(B.lo[2] + rz) * n + (B.lo[1] + ry)) * n + (B.lo[0] + rx);
    if (packed) {
      // SLH_F32_BF16: v_ij as BF16 pairs in slots SLOT_V0 .. SLOT_V0 + 2
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const unsigned w = __float_as_uint((float)y[src + (SLOT_V0 + c / 2) * B.cs]);
        out[c * n3 + dst] = (T)__uint_as_float((c & 1) ? (w & 0xFFFF0000u) : (w << 16));
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) out[c * n3 + dst] = y[src + (GW_V0 + c) * B.cs];
    }
  }
}

template <typename C>
__device__ __forceinline__ double2 as_d2(const C& v) { return make_double2((double)v.x, (double)v.y); }

// --- the contraction of one mode (kx, ky, kz) of the half spectrum
template <typename C>
__device__ __forceinline__ double mode_contraction(const C* vt, long long cstride, long long t, int kx, int ky, int kz,
                                                   const double* keff) {
  double kh[3] = {keff[kx], keff[ky], keff[kz]};
  const double kk = kh[0] * kh[0] + kh[1] * kh[1] + kh[2] * kh[2];
  if (kk > 0.0) {
    const double inv = 1.0 / sqrt(kk);
    kh[0] *= inv;
    kh[1] *= inv;
    kh[2] *= inv;
  } else {
    kh[0] = kh[1] = kh[2] = 0.0;
  }
  double P[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[i][j] = (i == j ? 1.0 : 0.0) - kh[i] * kh[j];
  // V symmetric from (xx, yy, zz, xy, xz, yz)
  double2 V[3][3];
  const double2 vxx = as_d2(vt[0 * cstride + t]), vyy = as_d2(vt[1 * cstride + t]), vzz = as_d2(vt[2 * cstride + t]);
  const double2 vxy = as_d2(vt[3 * cstride + t]), vxz = as_d2(vt[4 * cstride + t]), vyz = as_d2(vt[5 * cstride + t]);
  V[0][0] = vxx; V[1][1] = vyy; V[2][2] = vzz;
  V[0][1] = V[1][0] = vxy;
  V[0][2] = V[2][0] = vxz;
  V[1][2] = V[2][1] = vyz;
  // W = P V P (complex), tr(P V)
  double2 PV[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        re += P[i][a] * V[a][j].x;
        im += P[i][a] * V[a][j].y;
      }
      PV[i][j] = make_double2(re, im);
    }
  const double tre = PV[0][0].x + PV[1][1].x + PV[2][2].x, tim = PV[0][0].y + PV[1][1].y + PV[2][2].y;
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      double wre = 0.0, wim = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        wre += PV[l][b].x * P[b][m];
        wim += PV[l][b].y * P[b][m];
      }
      acc += wre * V[l][m].x + wim * V[l][m].y;   // Re(W_lm conj(V_lm))
    }
  return acc - 0.5 * (tre * tre + tim * tim);
}

// weight of column kx of the half spectrum: 2 where the conjugate partner
// (-kx) is not stored
__device__ __forceinline__ int col_weight(int kx, int n) { return (kx == 0 || 2 * kx == n) ? 1 : 2; }

// --- S[iq][kx] = sum over the rows of group iq (fixed order) of the weighted
// contraction of mode (kx, row); one thread per (iq, kx)
template <typename C>
__global__ void spectrum_rows_kernel(const C* vt, int n, const double* keff, const int* row_start, const int* rows,
                                     int nq, double* S) {
  const int nh = n / 2 + 1;
  const long long cstride = (long long)n * n * nh;
  const long long total = (long long)nq * nh;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += stride) {
    const int iq = (int)(u / nh), kx = (int)(u % nh);
    double acc = 0.0;
    for (int r = row_start[iq]; r < row_start[iq + 1]; ++r) {
      const int row = rows[r];   // ky + n kz
      const int ky = row % n, kz = row / n;
      acc += mode_contraction<C>(vt, cstride, (long long)row * nh + kx, kx, ky, kz, keff);
    }
    S[u] = (double)col_weight(kx, n) * acc;
  }
}

// --- bins[b] = sum_{kx ascending, kx^2 <= b} S[qmap[b - kx^2]][kx]; counts
// likewise from the group sizes; one thread per bin
__global__ void spectrum_bins_kernel(const double* S, const int* qmap, const int* row_start, int qmax, int n,
                                     int nbins, double* bins, unsigned long long* counts) {
  const int nh = n / 2 + 1;
  const int stride = gridDim.x * blockDim.x;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += stride) {
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int kx = 0; kx < nh && kx * kx <= b; ++kx) {
      const int q = b - kx * kx;
      if (q > qmax) continue;
      const int iq = qmap[q];
      if (iq < 0) continue;
      acc += S[(long long)iq * nh + kx];
      cnt += (unsigned long long)(row_start[iq + 1] - row_start[iq]) * (unsigned long long)col_weight(kx, n);
    }
    bins[b] = acc;
    counts[b] = cnt;
  }
}

template <typename T>
static slh_status spectrum_t(slh_ctx* c, int ptype, std::vector<double>* bins_h, std::vector<unsigned long long>* cnt_h) {
  const CufftApi& api = cufft_api();
  if (!api.ok) return fail(SLH_ERR_CUDA, "gw_spectrum: cuFFT (libcufft.so.12) could not be loaded");
  Level& L = c->lev[0];
  const int n = L.n_dom;
  const long long n3 = (long long)n * n * n;
  const long long nm = (long long)n * n * (n / 2 + 1);
  const int nbins = 3 * (n / 2) * (n / 2) + 1;
  using Cx = typename std::conditional<sizeof(T) == 8, cufftDoubleComplex, cufftComplex>::type;
  T* dense = nullptr;
  Cx* vt = nullptr;
  double* bins = nullptr;
  double* keff = nullptr;
  unsigned long long* counts = nullptr;
  double* S = nullptr;
  int *d_qmap = nullptr, *d_rstart = nullptr, *d_rows = nullptr;
  cufftHandle plan = 0;
  bool have_plan = false;
  slh_status st = SLH_OK;
  auto cleanup = [&]() {
    if (have_plan) api.destroy(plan);
    cudaFree(dense);
    cudaFree(vt);
    cudaFree(bins);
    cudaFree(keff);
    cudaFree(counts);
    cudaFree(S);
    cudaFree(d_qmap);
    cudaFree(d_rstart);
    cudaFree(d_rows);
  };
  // rows (ky, kz) of the half spectrum grouped by q = sy^2 + sz^2, groups in
  // ascending q, rows of a group in ascending (kz, ky)
  const int qmax = 2 * (n / 2) * (n / 2);
  std::vector<int> qcount(qmax + 1, 0);
  auto sgn = [n](int k) { return k <= n / 2 ? k : k - n; };
  for (int kz = 0; kz < n; ++kz)
    for (int ky = 0; ky < n; ++ky) ++qcount[sgn(ky) * sgn(ky) + sgn(kz) * sgn(kz)];
  std::vector<int> qmap(qmax + 1, -1), rstart(1, 0);
  for (int q = 0; q <= qmax; ++q)
    if (qcount[q]) {
      qmap[q] = (int)rstart.size() - 1;
      rstart.push_back(rstart.back() + qcount[q]);
    }
  const int nq = (int)rstart.size() - 1;
  std::vector<int> fillp(rstart.begin(), rstart.end() - 1), rows((size_t)n * n);
  for (int kz = 0; kz < n; ++kz)
    for (int ky = 0; ky < n; ++ky) rows[fillp[qmap[sgn(ky) * sgn(ky) + sgn(kz) * sgn(kz)]]++] = ky + n * kz;
  cudaError_t e = cudaMalloc(&dense, sizeof(T) * 6 * n3);
  if (e == cudaSuccess) e = cudaMalloc(&vt, sizeof(Cx) * 6 * nm);
  if (e == cudaSuccess) e = cudaMalloc(&bins, sizeof(double) * nbins);
  if (e == cudaSuccess) e = cudaMalloc(&counts, sizeof(unsigned long long) * nbins);
  if (e == cudaSuccess) e = cudaMalloc(&keff, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(double) * (size_t)nq * (n / 2 + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_qmap, sizeof(int) * qmap.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_rstart, sizeof(int) * rstart.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_rows, sizeof(int) * rows.size());
  if (e != cudaSuccess) {
    cleanup();
    return fail(SLH_ERR_NOMEM, "gw_spectrum: %s", cudaGetErrorString(e));
  }
  std::vector<double> kh(n);
  for (int i = 0; i < n; ++i) {
    const double th = 6.283185307179586 * i / n;   // 2 pi i / n
    kh[i] = ptype == 1 ? sin(th) / L.dx : (8.0 * sin(th) - sin(2.0 * th)) / (6.0 * L.dx);
  }
  e = cudaMemcpyAsync(keff, kh.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_qmap, qmap.data(), sizeof(int) * qmap.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rstart, rstart.data(), sizeof(int) * rstart.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "gw_spectrum setup");
  }
  const int threads = 256;
  long long blocks = (L.lay.nvalid + threads - 1) / threads;
  if (blocks > (long long)c->num_sms * 16) blocks = (long long)c->num_sms * 16;
  gather_v_kernel<T><<<(int)std::max<long long>(1, blocks), threads, 0, c->stream>>>(
      L.d_boxes, (int)L.boxes.size(), L.lay.nvalid, static_cast<const T*>(L.buf[L.role_y]), c->g, n, dense,
      c->prec == SLH_F32_BF16 ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "gather_v_kernel");
  }
  int dims[3] = {n, n, n};
  cufftResult r = api.plan_many(&plan, 3, dims, nullptr, 1, (int)n3, nullptr, 1, (int)nm,
                                sizeof(T) == 8 ? CUFFT_D2Z : CUFFT_R2C, 6);
  if (r == CUFFT_SUCCESS) {
    have_plan = true;
    r = api.set_stream(plan, c->stream);
  }
  if (r == CUFFT_SUCCESS) {
    if (sizeof(T) == 8)
      r = api.exec_d2z(plan, reinterpret_cast<cufftDoubleReal*>(dense), reinterpret_cast<cufftDoubleComplex*>(vt));
    else
      r = api.exec_r2c(plan, reinterpret_cast<cufftReal*>(dense), reinterpret_cast<cufftComplex*>(vt));
  }
  if (r != CUFFT_SUCCESS) {
    cleanup();
    return fail(SLH_ERR_CUDA, "gw_spectrum: cuFFT failed (%d)", (int)r);
  }
  const long long nS = (long long)nq * (n / 2 + 1);
  blocks = (nS + threads - 1) / threads;
  if (blocks > (long long)c->num_sms * 32) blocks = (long long)c->num_sms * 32;
  spectrum_rows_kernel<Cx><<<(int)blocks, threads, 0, c->stream>>>(vt, n, keff, d_rstart, d_rows, nq, S);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "spectrum_rows_kernel");
  }
  blocks = std::min<long long>((nbins + threads - 1) / threads, (long long)c->num_sms * 32);
  spectrum_bins_kernel<<<(int)blocks, threads, 0, c->stream>>>(S, d_qmap, d_rstart, qmax, n, nbins, bins, counts);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "spectrum_bins_kernel");
  }
  bins_h->resize(nbins);
  cnt_h->resize(nbins);
  e = cudaMemcpyAsync(bins_h->data(), bins, sizeof(double) * nbins, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt_h->data(), counts, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "gw_spectrum readback");
  return st;
}

slh_status gw_spectrum_impl(slh_ctx* c, int ptype, std::vector<double>* bins, std::vector<unsigned long long>* counts) {
  return c->prec == SLH_F64 ? spectrum_t<double>(c, ptype, bins, counts) : spectrum_t<float>(c, ptype, bins, counts);
}

}  // namespace slh
