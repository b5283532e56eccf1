// Host side of the fused stage kernel (stage_kernel.cuh): tensor maps of the
// level buffers, the tile variants the autotuners choose among, and the
// dispatch of a stage launch to its kernel instantiation.  The plain classic
// RK4 and SSPRK3 instantiations are compiled here, the plain Nystrom ones in
// stage_rkn.cu and every diagnostics stage 1 in stage_diag.cu (translation
// units of their own, compiled in parallel).
#include <map>
#include <mutex>

#include "stage_kernel.cuh"

namespace slh {

// ---------------------------------------------------------------------------
// host side: tensor maps, variant table, launch

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor maps of every (box, buffer): kind 0 the halo'd psi box
// {TX+8, TY+2G, 1, 2}, kind 1 the pointwise box {TX, TY, 1, 2}, over the
// 4D view {pitch, pny, pnz, 4 components} of the box; out-of-range parts of
// a box read as zero.
slh_status build_tmaps(slh_ctx* c, Level& L, int G, int TX, int TY, CUtensorMap** out) {
  const unsigned long long key = ((unsigned long long)G << 32) | ((unsigned long long)TX << 16) | (unsigned)TY;
  auto it = L.tmaps.find(key);
  if (it != L.tmaps.end()) {
    *out = static_cast<CUtensorMap*>(it->second);
    return SLH_OK;
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(SLH_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const size_t es = c->prec == SLH_F64 ? 8 : 4;
  const int nb = (int)L.lay.boxes.size();
  std::vector<CUtensorMap> maps((size_t)nb * SLH_NBUF * 2);
  for (int b = 0; b < nb; ++b) {
    const BoxDev& B = L.lay.boxes[b];
    for (int k = 0; k < SLH_NBUF; ++k) {
      for (int kind = 0; kind < 2; ++kind) {
        CUtensorMap& m = maps[((size_t)b * SLH_NBUF + k) * 2 + kind];
        memset(&m, 0, sizeof(m));
        if (!L.buf[k]) continue;
        void* base = static_cast<char*>(L.buf[k]) + (size_t)B.off * es;
        cuuint64_t dims[4] = {(cuuint64_t)B.pitch, (cuuint64_t)B.pny, (cuuint64_t)B.pnz, 4};
        cuuint64_t strides[3] = {(cuuint64_t)B.pitch * es, (cuuint64_t)B.pitch * B.pny * es, (cuuint64_t)B.cs * es};
        cuuint32_t box[4] = {(cuuint32_t)(kind == 0 ? TX + 8 : TX), (cuuint32_t)(kind == 0 ? TY + 2 * G : TY), 1, 2};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        CUresult r = enc(&m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return fail(SLH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for box %d buffer %d", (int)r, b, k);
      }
    }
  }
  CUtensorMap* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(CUtensorMap) * maps.size());
  if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "tensor maps: %s", cudaGetErrorString(e));
  e = cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "tensor maps upload");
  }
  L.tmaps[key] = d;
  *out = d;
  return SLH_OK;
}

// Tensor maps of the TMA-fed gravitational-wave stage: per (box, buffer)
// one map of the 4D view {pitch, pny, pnz, 16 components} of the box with
// the halo'd 2-component box {TX+8, TY+2G, 1, 2}; psi and the three pairs of
// u_ij are four copies of it per plane.  FP32 levels only.
slh_status build_gw_tmaps(slh_ctx* c, Level& L, int G, int TX, int TY, CUtensorMap** out) {
  const unsigned long long key = (1ull << 63) | ((unsigned long long)G << 32) | ((unsigned long long)TX << 16) | (unsigned)TY;
  auto it = L.tmaps.find(key);
  if (it != L.tmaps.end()) {
    *out = static_cast<CUtensorMap*>(it->second);
    return SLH_OK;
  }
  if (c->prec != SLH_F32_KAHAN || c->ncomp != NCOMP_GW)
    return fail(SLH_ERR_STATE, "gw tensor maps: FP32 16-field levels only");
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(SLH_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const size_t es = 4;
  const int nb = (int)L.lay.boxes.size();
  std::vector<CUtensorMap> maps((size_t)nb * SLH_NBUF);
  for (int b = 0; b < nb; ++b) {
    const BoxDev& B = L.lay.boxes[b];
    for (int k = 0; k < SLH_NBUF; ++k) {
      CUtensorMap& m = maps[(size_t)b * SLH_NBUF + k];
      memset(&m, 0, sizeof(m));
      if (!L.buf[k]) continue;
      void* base = static_cast<char*>(L.buf[k]) + (size_t)B.off * es;
      cuuint64_t dims[4] = {(cuuint64_t)B.pitch, (cuuint64_t)B.pny, (cuuint64_t)B.pnz, (cuuint64_t)NCOMP_GW};
      cuuint64_t strides[3] = {(cuuint64_t)B.pitch * es, (cuuint64_t)B.pitch * B.pny * es, (cuuint64_t)B.cs * es};
      cuuint32_t box[4] = {(cuuint32_t)(TX + 8), (cuuint32_t)(TY + 2 * G), 1, 2};
      cuuint32_t estr[4] = {1, 1, 1, 1};
      CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(SLH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for gw box %d buffer %d", (int)r, b, k);
    }
  }
  CUtensorMap* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(CUtensorMap) * maps.size());
  if (e != cudaSuccess) return fail(SLH_ERR_NOMEM, "gw tensor maps: %s", cudaGetErrorString(e));
  e = cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "gw tensor maps upload");
  }
  L.tmaps[key] = d;
  *out = d;
  return SLH_OK;
}

// Tile variants (x extent, y extent, pipeline depth) the autotuner chooses
// among; variant 0 is the default.
const TileVariant* tile_variants(int prec, int* n) {
  static const TileVariant f32[] = {{32, 16, 2, 64}, {32, 8, 3, 64}, {32, 16, 3, 128}, {16, 16, 2, 64},
                                    {64, 8, 2, 64}, {32, 8, 3, 128}, {128, 4, 2, 64}};
  static const TileVariant f64[] = {{32, 8, 2, 64}, {32, 4, 3, 64}, {16, 8, 2, 64}};
  if (prec == SLH_F64) {
    *n = 3;
    return f64;
  }
  *n = 7;
  return f32;
}

// the diagnostics variant (tags and/or energy partials) runs on the level's
// diagnostics tile, every other stage on its plain tile; RKN4 stages run the
// kernels instantiated in stage_rkn.cu
slh_status launch_stage(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used) {
  const bool diag = s.tags != nullptr || s.epart != nullptr;
  if (s.rkn) return diag ? launch_stage_diag(c, L, p, s, ctas_used, true) : launch_stage_rkn(c, L, p, s, ctas_used);
  return diag ? launch_stage_diag(c, L, p, s, ctas_used, false) : launch_tile<false, false>(c, L, p, s, ctas_used);
}

void free_tmaps(Level& L) {
  for (auto& kv : L.tmaps) cudaFree(kv.second);
  L.tmaps.clear();
}

}  // namespace slh
