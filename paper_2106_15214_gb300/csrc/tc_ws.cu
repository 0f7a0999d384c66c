// tc_ws.cu -- host side of the warp-specialised tensor-core sweeps (padded
// rank kp <= 64): tensor maps and one launch per sweep. The kernel is in
// tc_ws.cuh.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "tc_ws.cuh"

namespace nmf {
using namespace tc;

namespace {

// ---- host: tensor maps --------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// 2-D float tensor map: `cols` x `rows` elements, row pitch `pitch` elements,
// box boxCols x boxRows; false when TMA cannot address it.
bool map2d(CUtensorMap* m, const float* ptr, int64_t cols, int64_t rows, int64_t pitch, uint32_t boxCols,
           uint32_t boxRows, CUtensorMapSwizzle sw) {
  if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15u) || ((pitch * 4) & 15)) return false;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(pitch * 4)};
  const cuuint32_t box[2] = {boxCols, boxRows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename Kern>
cudaError_t prep(Kern k, size_t sm) {
  return ensure_smem_attr(reinterpret_cast<const void*>(k), sm);
}

template <bool CHI, bool ROW>
cudaError_t launch_ws(const Prob<float>& P, const TcMaps& m, int flags, const BetaParams& bp, double* lossPart,
                      int* status, cudaStream_t st, const SideJob* sidep) {
  const SideJob side = sidep ? *sidep : SideJob();
  const int kp = P.kp;
  int nop = 0, nv = 0;
  if (!pick_rings(kp, CHI, &nop, &nv)) return cudaErrorInvalidValue;
  CUtensorMap tmV;
  memset(&tmV, 0, sizeof(tmV));
  const int useTma = ROW ? map2d(&tmV, P.V, P.N, P.F, P.ldv, TL, MT, CU_TENSOR_MAP_SWIZZLE_128B)
                         : map2d(&tmV, P.V, P.N, P.F, P.ldv, MT, TL, CU_TENSOR_MAP_SWIZZLE_NONE);
  const CUtensorMap& once = ROW ? m.wsA : m.htA;
  const CUtensorMap& fa = ROW ? m.htB : m.wsB;
  const CUtensorMap& d1 = ROW ? (CHI ? m.ch1 : m.hs) : (CHI ? m.cw1 : m.wt);
  const CUtensorMap& d2 = ROW ? (CHI ? m.ch2 : m.hs) : (CHI ? m.cw2 : m.wt);
  const WsLayout lay = ws_layout(kp, CHI, nop, nv);
  const size_t sm = 1024 + lay.total;
  const int csize = ROW ? P.tcClusterS : P.tcClusterR;
  // the cluster exchange buffers (A/B tiles, stage ring) each hold kp KB
  if (csize > 1 && lay.total - lay.fa0 < 2048u * kp) return cudaErrorInvalidValue;
  // the row sweep stages its [P | Q] tile (2 x 128 x (K | 1) floats) over the stage ring and the A/B tiles
  if (ROW && lay.total - lay.fa0 < 2u * MT * (uint32_t)(P.K | 1) * 4u) return cudaErrorInvalidValue;
  const bool sk = !ROW && P.tcSK;
  const unsigned grid = (unsigned)(ROW ? P.tcRowTiles * P.tcSplitS : (sk ? P.tcSKBlocks : P.tcColTiles * P.tcSplitR));
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(WS_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaSuccess;
#define NMF_WS_CASE(BKV)                                                                                   \
  case BKV:                                                                                                \
    if (sk) {                                                                                              \
      e = prep(tc_ws_sk_kernel<BKV, CHI>, sm);                                                              \
      if (e == cudaSuccess)                                                                                \
        e = cudaLaunchKernelEx(&cfg, tc_ws_sk_kernel<BKV, CHI>, tmV, once, fa, d1, d2, useTma, nop, nv, P, flags, \
                               bp, lossPart, status, side);                                                \
    } else {                                                                                               \
      e = prep(tc_ws_kernel<BKV, CHI, ROW>, sm);                                                            \
      if (e == cudaSuccess)                                                                                \
        e = cudaLaunchKernelEx(&cfg, tc_ws_kernel<BKV, CHI, ROW>, tmV, once, fa, d1, d2, useTma, nop, nv, P, flags, \
                               bp, lossPart, status, side);                                                \
    }                                                                                                      \
    break;
  switch (bp.kind) {
    NMF_WS_CASE(BK_IS)
    NMF_WS_CASE(BK_KL)
    NMF_WS_CASE(BK_EUC)
    NMF_WS_CASE(BK_B15)
    NMF_WS_CASE(BK_GENERAL)
  }
#undef NMF_WS_CASE
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool tc_map_v(const Prob<float>& P, bool row, CUtensorMap* m) {
  memset(m, 0, sizeof(*m));
  return row ? map2d(m, P.V, P.N, P.F, P.ldv, TL, MT, CU_TENSOR_MAP_SWIZZLE_128B)
             : map2d(m, P.V, P.N, P.F, P.ldv, MT, TL, CU_TENSOR_MAP_SWIZZLE_NONE);
}

bool tc_ws_rings(int kp, bool chi, int* nop, int* nv, size_t* smem) {
  if (!pick_rings(kp, chi, nop, nv)) return false;
  *smem = 1024 + ws_layout(kp, chi, *nop, *nv).total;
  return true;
}

bool tc_build_maps(const Prob<float>& P, TcMaps* m) {
  m->ok = false;
  if (!P.sWS || P.kp > 64) return false;
  const int64_t F = P.F, N = P.N;
  const int kp = P.kp, ks = P.ks;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  bool ok = true;
  ok = ok && map2d(&m->wsA, P.sWS, ks, F, ks, 32, MT, SW);
  ok = ok && map2d(&m->wsB, P.sWS, ks, F, ks, 32, BT * TL, SW);
  ok = ok && map2d(&m->htA, P.sHT, ks, N, ks, 32, MT, SW);
  ok = ok && map2d(&m->htB, P.sHT, ks, N, ks, 32, BT * TL, SW);
  ok = ok && map2d(&m->hs, P.sHS, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->ch1, P.sCH1, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->ch2, P.sCH2, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->wt, P.sWT, F, kp, P.Fp, 32, kp, SW);
  ok = ok && map2d(&m->cw1, P.sCW1, F, kp, P.Fp, 32, kp, SW);
  ok = ok && map2d(&m->cw2, P.sCW2, F, kp, P.Fp, 32, kp, SW);
  m->ok = ok;
  return ok;
}

bool tc_fused_maps(const Prob<float>& P, CUtensorMap out[3]) {
  if (!P.sWS || !P.sHT || P.kp > 32) return false;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  return tc_map_v(P, true, &out[0]) && map2d(&out[1], P.sWS, P.ks, P.F, P.ks, 32, MT, SW) &&
         map2d(&out[2], P.sHT, P.ks, P.N, P.ks, 32, BT * TL, SW);
}

int tc_ws_capacity(int kp, int csize) {
  if (kp > 64 || kp < 16) return 0;
  int nop = 0, nv = 0;
  if (!pick_rings(kp, true, &nop, &nv)) return 0;
  const size_t sm = 1024 + ws_layout(kp, true, nop, nv).total;
  auto kern = tc_ws_kernel<BK_GENERAL, true, true>;
  if (prep(kern, sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(csize * 64));
  cfg.blockDim = dim3(WS_THREADS);
  cfg.dynamicSmemBytes = sm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n * csize;
}

cudaError_t launch_tc_ws_row(const Prob<float>& P, const TcMaps& m, int dsel, int flags, const BetaParams& bp,
                             double* lossPart, int* status, cudaStream_t st, const SideJob* side) {
  return dsel == OP_CHI ? launch_ws<true, true>(P, m, flags, bp, lossPart, status, st, side)
                        : launch_ws<false, true>(P, m, flags, bp, lossPart, status, st, side);
}

cudaError_t launch_tc_ws_col(const Prob<float>& P, const TcMaps& m, int csel, int flags, const BetaParams& bp,
                             double* lossPart, int* status, cudaStream_t st, const SideJob* side) {
  return csel == OP_CHI ? launch_ws<true, false>(P, m, flags, bp, lossPart, status, st, side)
                        : launch_ws<false, false>(P, m, flags, bp, lossPart, status, st, side);
}

}  // namespace nmf
