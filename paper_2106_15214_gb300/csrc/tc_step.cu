// tc_step.cu -- one JMM outer iteration (Algorithm 2 with L = 1, eq.
// jnt_update, the Sec. 4.1.2 normalisation and the objective of eq. obj_fct
// at the iterate) of a single dense TF32 problem in ONE persistent
// cooperative launch. The phases are those of the per-kernel sequence,
// separated by grid barriers instead of kernel boundaries:
//
//   W first: copies | row sweep (objective) | W update, chi(W), norm partials |
//            column sweep (+ norms, objective finalised by idle warps) |
//            H update scaled by the norms, W divided by them
//   H first: copies | column sweep (objective) | H update, chi(H) |
//            row sweep (+ objective finalised) | W update, norm partials |
//            normalisation (every block reduces the norm partials itself)
//
// Every block stays resident (cooperative launch, one block per SM); the
// sweeps' units (128-wide tile x chunk) are spread over the blocks. Data a
// block reads that another block wrote in an earlier phase is read through L2
// (__ldcg: L1 is not coherent across SMs), and generic writes that TMA reads
// in a later phase are followed by a proxy fence. Every barrier wait is
// bounded (1 s, then NMF_ETIMEOUT).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "tc_ws.cuh"

namespace nmf {
using namespace tc;

namespace {

struct StepMaps {
  CUtensorMap rV, rOnce, rFa, rD1, rD2;   // row sweep
  CUtensorMap cV, cOnce, cFa, cD1, cD2;   // column sweep
};

struct StepParams {
  int G;                                  // resident blocks
  int wfirst, wantLoss;
  int useTmaR, useTmaC, nopR, nvR, nopC, nvC;
  int rowUnits, colUnits;
  double* lossPart;
  double* lossOut;
  float* normPart;                        // [K][G]
  unsigned* bar;                          // [0] arrivals, [1] generation
  int* status;
  unsigned extra;                         // arrivals expected beyond the G blocks (0; 1 in the timeout test)
  uint64_t limitNs;                       // bound of every barrier wait (1 s unless a test shortens it)
};

__device__ __forceinline__ bool status_set(const int* st) { return *reinterpret_cast<const volatile int*>(st) != 0; }

__device__ __forceinline__ void proxy_fence_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded grid barrier over the S.G resident blocks.
__device__ __forceinline__ void grid_sync(const StepParams& S) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = S.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(S.bar, 1u) == (unsigned)S.G + S.extra - 1) {
      atomicExch(S.bar, 0u);
      __threadfence();
      atomicAdd(S.bar + 1, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (*gen == g0) {
        if (globaltimer_ns() - t0 > S.limitNs) {
          atomicExch(S.status, ETIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// W~, H~ and their TF32 copies (as tc_copies_kernel; `tile` = 32 x (KMAX + 1) floats).
__device__ void phase_copies(const Prob<float>& P, const StepParams& S, float* tile) {
  const int T = WS_THREADS;
  const int64_t FK = P.F * P.K;
  for (int64_t idx = (int64_t)blockIdx.x * T + threadIdx.x; idx < FK; idx += (int64_t)S.G * T) {
    const float w = P.W[idx];
    P.Wt[idx] = w;
    const int64_t f = idx / P.K, k = idx - f * P.K;
    const float r = tf32_round(w);
    P.sWS[f * P.ks + k] = r;
    P.sWT[k * P.Fp + f] = r;
  }
  const int nT = (int)((P.N + 31) / 32);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < nT; t += S.G) {
    const int64_t n0 = (int64_t)t * 32, n = n0 + lane;
    for (int k = w; k < P.K; k += T / 32) {
      if (n < P.N) {
        const float h = P.H[(int64_t)k * P.N + n];
        P.Ht[(int64_t)k * P.N + n] = h;
        const float r = tf32_round(h);
        P.sHS[(int64_t)k * P.Np + n] = r;
        tile[lane * (KMAX + 1) + k] = r;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * P.K; i += T) {
      const int nl = i / P.K, k = i - nl * P.K;
      if (n0 + nl < P.N) P.sHT[(n0 + nl) * P.ks + k] = tile[nl * (KMAX + 1) + k];
    }
    __syncthreads();
  }
}

// Fixed-order sum of `slices` partial slices (stride 2 * len) of numerator and denominator.
__device__ __forceinline__ void slice_sums(const float* part, int64_t len, int slices, float& num, float& den) {
  num = 0.f;
  den = 0.f;
  for (int s0 = 0; s0 < slices; s0 += 8) {
    float vn[8], vd[8];
    #pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int sl = s0 + u;
      vn[u] = sl < slices ? __ldcg(part + (int64_t)sl * 2 * len) : 0.f;
      vd[u] = sl < slices ? __ldcg(part + (int64_t)sl * 2 * len + len) : 0.f;
    }
    #pragma unroll
    for (int u = 0; u < 8; ++u) {
      num += vn[u];
      den += vd[u];
    }
  }
}

// W-half update from the row sweep's slices (eq. jnt_update): W = W~ (P/Q)^gamma,
// optionally chi(W) as TF32 copies for the column sweep; column sums of
// squares of the new W per block into normPart[k][block] (fixed order).
// Each block takes a contiguous range of entries; when the range is short
// against the block, Gl lanes share an entry's slice sums (lane j sums slices
// j, j + Gl, ..., then a fixed butterfly).
template <int BK>
__device__ void phase_rows_epi(const Prob<float>& P, const BetaParams& bp, const StepParams& S, bool skip,
                               bool wantChi, float* s_sq) {
  const int T = WS_THREADS;
  const int64_t FK = P.F * P.K;
  const int64_t per = (FK + S.G - 1) / S.G;
  const int64_t e0 = (int64_t)blockIdx.x * per, e1 = e0 + per < FK ? e0 + per : FK;
  int Gl = 1;
  while (Gl < 8 && (int64_t)(2 * Gl) * per <= T && 2 * Gl <= P.tcS) Gl *= 2;
  const int epc = T / Gl;                            // entries per chunk
  const int sub = threadIdx.x % Gl, ent = threadIdx.x / Gl;
  const int slices = P.tcS;
  float acc = 0.f;                                   // thread k < K: column k's running sum
  for (int64_t c0 = e0; c0 < e1; c0 += epc) {
    const int64_t idx = c0 + ent;
    const bool inside = idx < e1 && !skip;
    float num = 0.f, den = 0.f;
    if (inside) {
      const float* part = P.rowPart + idx;
      for (int s0 = sub; s0 < slices; s0 += 8 * Gl) {
        float vn[8], vd[8];
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int sl = s0 + u * Gl;
          vn[u] = sl < slices ? __ldcg(part + (int64_t)sl * 2 * FK) : 0.f;
          vd[u] = sl < slices ? __ldcg(part + (int64_t)sl * 2 * FK + FK) : 0.f;
        }
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
          num += vn[u];
          den += vd[u];
        }
      }
    }
    for (int o = 1; o < Gl; o <<= 1) {               // the Gl lanes of an entry share a warp
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    float sq = 0.f;
    if (inside && sub == 0) {
      const float wt = __ldcg(P.Wt + idx);
      const float x = apply_floor(wt * mu_ratio<BK, float>(num, den, (float)bp.gamma), (float)bp.floor);
      if (!isfinite(x)) atomicExch(S.status, 4);
      P.W[idx] = x;
      sq = x * x;
      if (wantChi) {
        float c1, c2;
        chi_terms<BK, float>(x, wt, (float)bp.beta, c1, c2);
        const int64_t f = idx / P.K, k = idx - f * P.K;
        P.sCW1[k * P.Fp + f] = tf32_round(c1);
        P.sCW2[k * P.Fp + f] = tf32_round(c2);
      }
    }
    if (sub == 0) s_sq[ent] = sq;
    __syncthreads();
    if (threadIdx.x < P.K) {
      const int k = threadIdx.x;
      for (int i = (int)(((int64_t)k - c0 % P.K + P.K) % P.K); i < epc && c0 + i < e1; i += P.K) acc += s_sq[i];
    }
    __syncthreads();
  }
  if (threadIdx.x < P.K) S.normPart[(int64_t)threadIdx.x * S.G + blockIdx.x] = acc;
}

// H-half update from the column sweep's slices: H = H~ (Hn/Hd)^gamma, with
// chi(H) as TF32 copies (H first) or scaled by W's column norms (W first,
// the iteration's last phase, which also divides W's columns by them).
template <int BK>
__device__ void phase_cols_epi(const Prob<float>& P, const BetaParams& bp, const StepParams& S, bool skip,
                               bool wantChi, bool applyNorm) {
  if (skip) return;
  const int T = WS_THREADS;
  const int64_t KN = (int64_t)P.K * P.N;
  for (int64_t idx = (int64_t)blockIdx.x * T + threadIdx.x; idx < KN; idx += (int64_t)S.G * T) {
    float num, den;
    slice_sums(P.colPart + idx, KN, P.tcR, num, den);
    const float ht = __ldcg(P.Ht + idx);
    const float x = apply_floor(ht * mu_ratio<BK, float>(num, den, (float)bp.gamma), (float)bp.floor);
    if (!isfinite(x)) atomicExch(S.status, 4);
    const int64_t k = idx / P.N;
    if (wantChi) {
      float c1, c2;
      chi_terms<BK, float>(x, ht, (float)bp.beta, c1, c2);
      const int64_t n = idx - k * P.N;
      P.sCH1[k * P.Np + n] = tf32_round(c1);
      P.sCH2[k * P.Np + n] = tf32_round(c2);
    }
    float y = x;
    if (applyNorm) {
      const float nk = __ldcg(P.norms + k);
      if (nk > 0.f) y = x * nk;
    }
    P.H[idx] = y;
  }
  if (applyNorm) {
    const int64_t FK = P.F * P.K;
    for (int64_t idx = (int64_t)blockIdx.x * T + threadIdx.x; idx < FK; idx += (int64_t)S.G * T) {
      const float nk = __ldcg(P.norms + idx % P.K);
      if (nk > 0.f) P.W[idx] = __ldcg(P.W + idx) / nk;
    }
  }
}

// H first, last phase: every block reduces the norm partials itself (fixed
// order, identical in every block), then scales its share of W and H.
__device__ void phase_normalize(const Prob<float>& P, const StepParams& S, bool skip, float* s_red, float* s_norm) {
  if (skip) return;
  const int T = WS_THREADS, K = P.K, R = T / K;
  float v = 0.f;
  if ((int)threadIdx.x < R * K) {
    const int k = threadIdx.x / R, j = threadIdx.x - k * R;
    for (int b = j; b < S.G; b += R) v += __ldcg(S.normPart + (int64_t)k * S.G + b);
  }
  s_red[threadIdx.x] = v;
  __syncthreads();
  if ((int)threadIdx.x < K) {
    float sum = 0.f;
    for (int j = 0; j < R; ++j) sum += s_red[threadIdx.x * R + j];
    s_norm[threadIdx.x] = sqrtf(sum);
    if (blockIdx.x == 0) P.norms[threadIdx.x] = s_norm[threadIdx.x];
  }
  __syncthreads();
  const int64_t FK = P.F * P.K, KN = (int64_t)K * P.N;
  for (int64_t idx = (int64_t)blockIdx.x * T + threadIdx.x; idx < FK; idx += (int64_t)S.G * T) {
    const float nk = s_norm[idx % K];
    if (nk > 0.f) P.W[idx] = __ldcg(P.W + idx) / nk;
  }
  for (int64_t idx = (int64_t)blockIdx.x * T + threadIdx.x; idx < KN; idx += (int64_t)S.G * T) {
    const float nk = s_norm[idx / P.N];
    if (nk > 0.f) P.H[idx] = __ldcg(P.H + idx) * nk;
  }
}

template <int BK>
__global__ void __launch_bounds__(WS_THREADS, 1)
tc_step_kernel(const __grid_constant__ StepMaps M, Prob<float> P, BetaParams bp, StepParams S) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  __shared__ double red[32];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* scratch = reinterpret_cast<float*>(base);   // epilogue phases: the sweeps' rings are idle then
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 2) tmem_alloc(&tslot, TM_COLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const int lossFlag = S.wantLoss ? SWEEP_LOSS : 0;

  // ---- copies
  if (!status_set(S.status)) phase_copies(P, S, scratch);
  proxy_fence_global();
  grid_sync(S);

  // ---- first sweep (with the objective at the iterate)
  {
    const bool skip = status_set(S.status);
    if (S.wfirst) {
      for (int u = blockIdx.x; u < S.rowUnits; u += S.G) {
        const double l = ws_unit<BK, false, true>(M.rV, M.rOnce, M.rFa, M.rD1, M.rD2, S.useTmaR, S.nopR, S.nvR, P,
                                                  lossFlag, bp, S.status, uniform_geom<true>(P, u), skip, base, tbase,
                                                  bars, s_abort, red, nullptr, true);
        if (lossFlag && threadIdx.x == 0) S.lossPart[u] = l;
      }
    } else {
      for (int u = blockIdx.x; u < S.colUnits; u += S.G) {
        const double l = ws_unit<BK, false, false>(M.cV, M.cOnce, M.cFa, M.cD1, M.cD2, S.useTmaC, S.nopC, S.nvC, P,
                                                   lossFlag, bp, S.status, uniform_geom<false>(P, u), skip, base,
                                                   tbase, bars, s_abort, red, nullptr, true);
        if (lossFlag && threadIdx.x == 0) S.lossPart[u] = l;
      }
    }
  }
  grid_sync(S);

  // ---- first epilogue
  {
    const bool skip = status_set(S.status);
    if (S.wfirst) phase_rows_epi<BK>(P, bp, S, skip, true, scratch);
    else phase_cols_epi<BK>(P, bp, S, skip, true, false);
  }
  proxy_fence_global();
  grid_sync(S);

  // ---- second sweep; idle warps finalise the norms (W first) and the objective
  {
    const bool skip = status_set(S.status);
    SideJob side;
    side.normPart = S.normPart;
    side.nparts = S.G;
    side.normK = (S.wfirst && (int)blockIdx.x < P.K) ? (int)blockIdx.x : -1;
    side.normStride = P.K;                           // one column per block (S.G >= K)
    side.norms = P.norms;
    side.lossPart = S.lossPart;
    side.nloss = (S.wantLoss && blockIdx.x == 0) ? (S.wfirst ? S.rowUnits : S.colUnits) : 0;
    side.lossOut = S.lossOut;
    const SideJob* sp = (side.normK >= 0 || side.nloss > 0) ? &side : nullptr;
    const int units = S.wfirst ? S.colUnits : S.rowUnits;
    if ((int)blockIdx.x >= units) {
      if (warp == 3) side_run(sp, lane, P.K);
    }
    for (int u = blockIdx.x; u < units; u += S.G) {
      if (S.wfirst)
        ws_unit<BK, true, false>(M.cV, M.cOnce, M.cFa, M.cD1, M.cD2, S.useTmaC, S.nopC, S.nvC, P, 0, bp, S.status,
                                 uniform_geom<false>(P, u), skip, base, tbase, bars, s_abort, red, sp, true);
      else
        ws_unit<BK, true, true>(M.rV, M.rOnce, M.rFa, M.rD1, M.rD2, S.useTmaR, S.nopR, S.nvR, P, 0, bp, S.status,
                                uniform_geom<true>(P, u), skip, base, tbase, bars, s_abort, red, sp, true);
      sp = nullptr;                                  // the side job runs with the block's first unit only
    }
  }
  grid_sync(S);

  // ---- second epilogue (+ normalisation)
  {
    const bool skip = status_set(S.status);
    if (S.wfirst) {
      phase_cols_epi<BK>(P, bp, S, skip, false, true);
    } else {
      phase_rows_epi<BK>(P, bp, S, skip, false, scratch);
      grid_sync(S);
      phase_normalize(P, S, status_set(S.status), scratch, scratch + WS_THREADS);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tbase, TM_COLS);
}

size_t step_smem(int kp, int* nopR, int* nvR, int* nopC, int* nvC, bool wfirst) {
  size_t a = 0, b = 0;
  // W first: row sweep without chi, column sweep with; H first the reverse
  if (!tc_ws_rings(kp, !wfirst, nopR, nvR, &a) || !tc_ws_rings(kp, wfirst, nopC, nvC, &b)) return 0;
  size_t m = a > b ? a : b;
  const size_t scratch = 1024 + sizeof(float) * 32 * (KMAX + 1);
  return m > scratch ? m : scratch;
}

}  // namespace

bool tc_step_supported(const Prob<float>& P, const TcMaps& m, int sms) {
  if (!m.ok || !P.sWS || P.kp > 64 || P.tcClusterS != 1 || P.tcClusterR != 1 || P.tcSK) return false;
  if (P.K > WS_THREADS / 8 || P.K > sms) return false;   // norm reductions: >= 8 threads, one block per column
  (void)sms;
  return true;
}

cudaError_t launch_tc_step(const Prob<float>& P, const TcMaps& m, const BetaParams& bp, const TcStepArgs& a,
                           int sms, cudaStream_t st) {
  StepMaps M;
  memset(&M, 0, sizeof(M));
  StepParams S;
  memset(&S, 0, sizeof(S));
  const size_t sm = step_smem(P.kp, &S.nopR, &S.nvR, &S.nopC, &S.nvC, a.wfirst);
  if (sm == 0) return cudaErrorInvalidValue;
  S.useTmaR = tc_map_v(P, true, &M.rV) ? 1 : 0;
  S.useTmaC = tc_map_v(P, false, &M.cV) ? 1 : 0;
  M.rOnce = m.wsA;
  M.rFa = m.htB;
  M.cOnce = m.htA;
  M.cFa = m.wsB;
  if (a.wfirst) {            // row sweep on H~ itself, column sweep on chi(W)
    M.rD1 = m.hs;
    M.rD2 = m.hs;
    M.cD1 = m.cw1;
    M.cD2 = m.cw2;
  } else {                   // column sweep on W~ itself, row sweep on chi(H)
    M.cD1 = m.wt;
    M.cD2 = m.wt;
    M.rD1 = m.ch1;
    M.rD2 = m.ch2;
  }
  S.wfirst = a.wfirst ? 1 : 0;
  S.wantLoss = a.wantLoss ? 1 : 0;
  S.rowUnits = P.tcRowTiles * P.tcSplitS;
  S.colUnits = P.tcColTiles * P.tcSplitR;
  S.lossPart = a.lossPart;
  S.lossOut = a.lossOut;
  S.normPart = a.normPart;
  S.bar = a.gridBar;
  S.status = a.status;
  S.extra = a.extraArrivals;
  S.limitNs = a.waitLimitNs;

  void (*kern)(const StepMaps, Prob<float>, BetaParams, StepParams) = nullptr;
  switch (bp.kind) {
    case BK_IS: kern = tc_step_kernel<BK_IS>; break;
    case BK_KL: kern = tc_step_kernel<BK_KL>; break;
    case BK_EUC: kern = tc_step_kernel<BK_EUC>; break;
    case BK_B15: kern = tc_step_kernel<BK_B15>; break;
    default: kern = tc_step_kernel<BK_GENERAL>; break;
  }
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(kern), sm);
  if (e != cudaSuccess) return e;
  int perSm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSm, kern, WS_THREADS, sm);
  if (e != cudaSuccess) return e;
  if (perSm < 1) return cudaErrorInvalidConfiguration;
  S.G = sms;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)S.G);
  cfg.blockDim = dim3(WS_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, M, P, bp, S);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace nmf
