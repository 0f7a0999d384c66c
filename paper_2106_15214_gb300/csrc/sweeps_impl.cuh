// sweeps_impl.cuh -- SIMT kernels of the dense path, templated on the element
// type (double for NMF_FP64, float for NMF_FP32).
//
// Every update of Algorithm 1 (BMM, eq. alt_update) and Algorithm 2 (JMM,
// eq. jnt_update) is a product of the two elementwise terms
//     A = (V + kappa) . Vp^(beta-2),   B = Vp . Vp^(beta-2),   Vp = Wp Hp + kappa
// with a factor-shaped matrix, reduced either over columns n (the W half) or
// over rows f (the H half):
//   row sweep:    P = A D1^T,  Q = B D2^T     (F x K, reduced over n)
//   column sweep: Hn = C1^T A, Hd = C2^T B    (K x N, reduced over f)
// JMM takes Wp = Wt, Hp = Ht (the product is formed at the iterate only,
// Algorithm 2) and D/C = chi_1, chi_2 of the other factor; BMM takes the
// current factors and D = C = that factor. Vp is recomputed per tile in
// shared memory and never stored.
//
// Tiling: a block owns a BF x BN tile at a time; phase A forms Vp, A and B
// for the tile in shared memory (plus the objective when asked, eq.
// obj_fct), phase B accumulates the contraction in registers. Partial sums go
// to per-chunk slices that the epilogue adds in a fixed order, so every
// result is deterministic.
#pragma once

#include <algorithm>

#include <type_traits>

#include "internal.h"

namespace nmf {

constexpr int TP = BN + 1;  // padded shared-memory row of a BN-wide tile

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

// Phase A: Vp, A, B for rows [f0, f0+BF) x cols [n0, n0+BN) of one problem.
// Ws: [BF][KP] rows of Wp; Hs: [K][TP] columns of Hp. Out-of-range entries get
// A = B = 0 so they add nothing. Returns this thread's share of the objective.
template <typename T, int BK>
__device__ __forceinline__ T phase_a(const T* Ws, int KP, const T* Hs, int K,
                                     const T* __restrict__ V, int64_t ldv, int64_t f0,
                                     int64_t fLim, int64_t n0, int64_t nLim,
                                     const BetaParams& bp, T* As, T* Bs, bool wantLoss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T kappa = (T)bp.kappa, bm2 = (T)(bp.beta - 2.0);
  T tl = T(0);
  #pragma unroll
  for (int i = 0; i < BF / 8; ++i) {
    const int f = warp + 8 * i;
    const int64_t gf = f0 + f, gn = n0 + lane;
    T a = T(0), b = T(0);
    if (gf < fLim && gn < nLim) {
      T vt = T(0);
      const T* wrow = Ws + f * KP;
      for (int k = 0; k < K; ++k) vt = fma(wrow[k], Hs[k * TP + lane], vt);
      vt += kappa;
      const T v = V[gf * ldv + gn] + kappa;
      ab_terms_g<BK>(v, vt, bm2, a, b, bp.tiny);
      if (wantLoss) tl += (T)DB<T>::eval(v, vt, bp, BK);
    }
    As[f * TP + lane] = a;
    Bs[f * TP + lane] = b;
  }
  return tl;
}

// float: three blocks per SM (80 registers, no spills; 128 at two blocks)
template <typename T, int BK, int KJ>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1)
row_sweep_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefix,
                 int wsel, int hsel, int dsel, int flags, BetaParams bp,
                 double* __restrict__ lossPart, const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  const int b = blockIdx.x;
  const int pi = find_problem(prefix, count, b);
  const Prob<T> P = probs[pi];
  const int local = b - prefix[pi];
  const int ft = local % P.rowTilesF;
  const int s = local / P.rowTilesF;
  const int K = P.K, KP = K + 1;
  const bool contract = flags & SWEEP_CONTRACT, wantLoss = flags & SWEEP_LOSS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  T* Hs = Ws + BF * KP;
  T* D1s = Hs + K * TP;
  T* D2s = D1s + K * TP;
  T* As = dsel == OP_CHI ? D2s + K * TP : D1s;
  T* Bs = As + BF * TP;
  __shared__ double red[32];

  const T* __restrict__ Wp = wsel == SEL_TILDE ? P.Wt : P.W;
  const T* __restrict__ Hp = hsel == SEL_TILDE ? P.Ht : P.H;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t f0 = (int64_t)ft * BF;
  for (int i = tid; i < BF * K; i += NT) {
    const int f = i / K, k = i - f * K;
    Ws[f * KP + k] = (f0 + f < P.F) ? Wp[(f0 + f) * K + k] : T(0);
  }
  T accP[BF / 8][KJ], accQ[BF / 8][KJ];
  #pragma unroll
  for (int i = 0; i < BF / 8; ++i)
    #pragma unroll
    for (int j = 0; j < KJ; ++j) accP[i][j] = accQ[i][j] = T(0);
  double loss = 0.0;
  const int64_t nBeg = (int64_t)s * P.chunkN;
  const int64_t nEnd = lmin(P.N, nBeg + P.chunkN);
  for (int64_t n0 = nBeg; n0 < nEnd; n0 += BN) {
    __syncthreads();
    for (int i = tid; i < K * BN; i += NT) {
      const int k = i / BN, n = i - k * BN;
      const int64_t gn = n0 + n;
      const bool in = gn < nEnd;
      Hs[k * TP + n] = in ? Hp[k * P.N + gn] : T(0);
      if (dsel == OP_CHI) {
        D1s[k * TP + n] = in ? P.chiH1[k * P.N + gn] : T(0);
        D2s[k * TP + n] = in ? P.chiH2[k * P.N + gn] : T(0);
      }
    }
    __syncthreads();
    T tl = phase_a<T, BK>(Ws, KP, Hs, K, P.V, P.ldv, f0, P.F, n0, nEnd, bp, As, Bs, wantLoss);
    if (wantLoss) loss += (double)tl;
    if (!contract) continue;
    __syncthreads();
    const T* D1 = dsel == OP_CHI ? D1s : Hs;
    const T* D2 = dsel == OP_CHI ? D2s : Hs;
    #pragma unroll 4
    for (int n = 0; n < BN; ++n) {
      T av[BF / 8], bv[BF / 8];
      #pragma unroll
      for (int i = 0; i < BF / 8; ++i) {
        av[i] = As[(warp + 8 * i) * TP + n];
        bv[i] = Bs[(warp + 8 * i) * TP + n];
      }
      #pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        const T d1 = k < K ? D1[k * TP + n] : T(0);
        const T d2 = k < K ? D2[k * TP + n] : T(0);
        #pragma unroll
        for (int i = 0; i < BF / 8; ++i) {
          accP[i][j] = fma(av[i], d1, accP[i][j]);
          accQ[i][j] = fma(bv[i], d2, accQ[i][j]);
        }
      }
    }
  }
  if (contract) {
    T* part = P.rowPart + (int64_t)s * 2 * P.F * K;
    #pragma unroll
    for (int i = 0; i < BF / 8; ++i) {
      const int64_t gf = f0 + warp + 8 * i;
      #pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        if (gf < P.F && k < K) {
          part[gf * K + k] = accP[i][j];
          part[P.F * K + gf * K + k] = accQ[i][j];
        }
      }
    }
  }
  if (wantLoss) {
    const double t = block_sum(loss, red);
    if (tid == 0) lossPart[b] = t;
  }
}

template <typename T, int BK, int KJ8>
__global__ void __launch_bounds__(NT)
col_sweep_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefix,
                 int wsel, int hsel, int csel, int flags, BetaParams bp,
                 double* __restrict__ lossPart, const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  const int b = blockIdx.x;
  const int pi = find_problem(prefix, count, b);
  const Prob<T> P = probs[pi];
  const int local = b - prefix[pi];
  const int nt = local % P.colTilesN;
  const int r = local / P.colTilesN;
  const int K = P.K, KP = K + 1;
  const bool contract = flags & SWEEP_CONTRACT, wantLoss = flags & SWEEP_LOSS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Hs = reinterpret_cast<T*>(smem_raw);
  T* Ws = Hs + K * TP;
  T* C1s = Ws + BF * KP;
  T* C2s = C1s + BF * KP;
  T* As = csel == OP_CHI ? C2s + BF * KP : C1s;
  T* Bs = As + BF * TP;
  __shared__ double red[32];

  const T* __restrict__ Wp = wsel == SEL_TILDE ? P.Wt : P.W;
  const T* __restrict__ Hp = hsel == SEL_TILDE ? P.Ht : P.H;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n0 = (int64_t)nt * BN;
  for (int i = tid; i < K * BN; i += NT) {
    const int k = i / BN, n = i - k * BN;
    Hs[k * TP + n] = (n0 + n < P.N) ? Hp[k * P.N + n0 + n] : T(0);
  }
  T num[KJ8], den[KJ8];
  #pragma unroll
  for (int j = 0; j < KJ8; ++j) num[j] = den[j] = T(0);
  double loss = 0.0;
  const int64_t fBeg = (int64_t)r * P.chunkF;
  const int64_t fEnd = lmin(P.F, fBeg + P.chunkF);
  for (int64_t f0 = fBeg; f0 < fEnd; f0 += BF) {
    __syncthreads();
    for (int i = tid; i < BF * K; i += NT) {
      const int f = i / K, k = i - f * K;
      const int64_t gf = f0 + f;
      const bool in = gf < fEnd;
      Ws[f * KP + k] = in ? Wp[gf * K + k] : T(0);
      if (csel == OP_CHI) {
        C1s[f * KP + k] = in ? P.chiW1[gf * K + k] : T(0);
        C2s[f * KP + k] = in ? P.chiW2[gf * K + k] : T(0);
      }
    }
    __syncthreads();
    T tl = phase_a<T, BK>(Ws, KP, Hs, K, P.V, P.ldv, f0, fEnd, n0, P.N, bp, As, Bs, wantLoss);
    if (wantLoss) loss += (double)tl;
    if (!contract) continue;
    __syncthreads();
    const T* C1 = csel == OP_CHI ? C1s : Ws;
    const T* C2 = csel == OP_CHI ? C2s : Ws;
    #pragma unroll 4
    for (int f = 0; f < BF; ++f) {
      const T a = As[f * TP + lane], bb = Bs[f * TP + lane];
      #pragma unroll
      for (int j = 0; j < KJ8; ++j) {
        const int k = warp + 8 * j;
        if (k < K) {
          num[j] = fma(C1[f * KP + k], a, num[j]);
          den[j] = fma(C2[f * KP + k], bb, den[j]);
        }
      }
    }
  }
  if (contract) {
    T* part = P.colPart + (int64_t)r * 2 * K * P.N;
    const int64_t gn = n0 + lane;
    #pragma unroll
    for (int j = 0; j < KJ8; ++j) {
      const int k = warp + 8 * j;
      if (k < K && gn < P.N) {
        part[k * P.N + gn] = num[j];
        part[(int64_t)K * P.N + k * P.N + gn] = den[j];
      }
    }
  }
  if (wantLoss) {
    const double t = block_sum(loss, red);
    if (tid == 0) lossPart[b] = t;
  }
}

// Fixed-order sum of `slices` partial slices at stride `stride`, loads in
// flight together (8 at a time), additions in slice order.
template <typename T>
__device__ __forceinline__ void sum_slices(const T* __restrict__ part, int64_t stride, int64_t half, int slices,
                                           T& num, T& den) {
  num = T(0);
  den = T(0);
  int s = 0;
  for (; s + 8 <= slices; s += 8) {
    T a[8], b[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = part[(int64_t)(s + j) * stride];
      b[j] = part[(int64_t)(s + j) * stride + half];
    }
    #pragma unroll
    for (int j = 0; j < 8; ++j) { num += a[j]; den += b[j]; }
  }
  for (; s < slices; ++s) {
    num += part[(int64_t)s * stride];
    den += part[(int64_t)s * stride + half];
  }
}

// The last block to finish (after every block published its partials) does
// the fixed-order finalisations: column norms of W from the per-block partial
// sums of squares, and / or the objective from the sweep's loss partials.
template <typename T>
__device__ __forceinline__ void last_block_finalize(const EpiFuse& fz, const Prob<T>& P, int nblocks,
                                                    T* sbuf /* blockDim.x values, for FUSE_NORM_PART */) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(fz.counter, 1u) == (unsigned)nblocks - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (fz.flags & FUSE_NORM_PART) {
    // Partials are [k][block] in the context's precision (a column norm needs
    // no FP64; FP64 issues at a small fraction of the FP32 rate here). R
    // threads per column: thread (k, j) sums blocks j, j + R, ... (coalesced
    // over j, eight loads in flight), then thread k adds its R sums in order:
    // deterministic.
    const int t = threadIdx.x, R = blockDim.x / P.K;
    const T* part = static_cast<const T*>(fz.normPart);
    T sq = T(0);
    if (t < R * P.K) {
      const int k = t / R, j = t - k * R;
      const T* row = part + (int64_t)k * nblocks;
      for (int b0 = j; b0 < nblocks; b0 += 8 * R) {
        T v[8];
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int bb = b0 + u * R;
          v[u] = bb < nblocks ? __ldcg(&row[bb]) : T(0);
        }
        #pragma unroll
        for (int u = 0; u < 8; ++u) sq += v[u];
      }
    }
    sbuf[t] = sq;
    __syncthreads();
    if (t < P.K) {
      T sum = T(0);
      for (int j = 0; j < R; ++j) sum += sbuf[t * R + j];
      P.norms[t] = sqrt(sum);
    }
  }
  if ((fz.flags & FUSE_LOSS) && threadIdx.x < 32) {
    // the objective in FP64, by one warp: a few partials per lane (loads in
    // flight together, added in order), one butterfly
    double sl = 0.0;
    for (int b0 = threadIdx.x; b0 < fz.lossBlocks; b0 += 256) {
      double v[8];
      #pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = b0 + 32 * u < fz.lossBlocks ? __ldcg(&fz.lossPart[b0 + 32 * u]) : 0.0;
      #pragma unroll
      for (int u = 0; u < 8; ++u) sl += v[u];
    }
    sl = warp_sum(sl);
    if (threadIdx.x == 0) fz.lossOut[0] = sl;
  }
  if (threadIdx.x == 0) *fz.counter = 0u;
}

// W-half epilogue over F x K entries. With fusion flags (single problem):
// FUSE_NORM_PART also publishes this block's sums of squares of the new W per
// column (the last block turns them into the column norms), FUSE_LOSS
// finalises the objective of the preceding sweep.
// NTH threads per block: 256 for batched contexts (blocks follow the prefix
// table), 1024 for a single problem (fewer blocks, so fewer norm partials).
template <typename T, int BK, int NTH>
__global__ void __launch_bounds__(NTH)
rows_epilogue_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefix,
                     int mode, int basesel, int want_chi, BetaParams bp, T* __restrict__ gout,
                     int* __restrict__ status, int tc, EpiFuse fz, int G) {
  pdl_wait();
  pdl_trigger();                 // after the wait: see SWEEP_EARLY
  // With fusion every block must reach the completion counter, so a set status
  // word only skips the arithmetic.
  const bool skip = *status != 0;
  if (skip && !fz.flags) return;
  __shared__ T s_sq[NTH];
  // G lanes per entry (single problem): lane j sums slices j, j + G, ... and a
  // fixed butterfly combines them; G = 1 for batched contexts.
  const int epb = NTH / G;                                 // entries per block
  const int b = blockIdx.x;
  const int pi = count == 1 ? 0 : find_problem(prefix, count, b);
  const Prob<T> P = probs[pi];
  const int64_t FK = P.F * P.K;
  const int sub = threadIdx.x % G;
  const int64_t idx = (int64_t)(b - (count == 1 ? 0 : prefix[pi])) * epb + threadIdx.x / G;
  const bool inside = idx < FK && !skip;
  const int slices = tc == 3 ? P.fuS : (tc ? P.tcS : P.S);
  T num = T(0), den = T(0);
  if (inside) {
    const T* part = P.rowPart + idx;
    for (int s0 = sub; s0 < slices; s0 += 8 * G) {        // eight slices' loads in flight, added in slice order
      T vn[8], vd[8];
      #pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int sl = s0 + u * G;
        vn[u] = sl < slices ? part[(int64_t)sl * 2 * FK] : T(0);
        vd[u] = sl < slices ? part[(int64_t)sl * 2 * FK + FK] : T(0);
      }
      #pragma unroll
      for (int u = 0; u < 8; ++u) {
        num += vn[u];
        den += vd[u];
      }
    }
  }
  for (int o = 1; o < G; o <<= 1) {                        // G in {1, 2, 4, 8}: lanes of an entry share a warp
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  T sq = T(0);
  if (inside && sub == 0) {
    if (mode == EPI_GRAD) {
      gout[idx] = den - num;
    } else {
      const T base = basesel == SEL_TILDE ? P.Wt[idx] : P.W[idx];
      const T x = apply_floor(base * mu_ratio<BK, T>(num, den, (T)bp.gamma), (T)bp.floor);
      if (!isfinite(x)) atomicExch(status, 4);
      P.W[idx] = x;
      sq = x * x;
      if (want_chi) {
        T c1, c2;
        chi_terms<BK, T>(x, P.Wt[idx], (T)bp.beta, c1, c2);
        if (tc != 2) {                            // tc == 2: the sweeps read only the TF32 copies below
          P.chiW1[idx] = c1;
          P.chiW2[idx] = c2;
        }
        if (tc && P.sCW1) {                       // transposed TF32 copies for the tensor-core sweeps
          const int64_t f = idx / P.K, k = idx - f * P.K;
          P.sCW1[k * P.Fp + f] = tf32_round(c1);
          P.sCW2[k * P.Fp + f] = tf32_round(c2);
        }
      }
    }
  }
  if (!fz.flags) return;
  if (fz.flags & FUSE_NORM_PART) {
    s_sq[threadIdx.x] = sq;
    __syncthreads();
    const int64_t first = (int64_t)b * epb;
    for (int k = threadIdx.x; k < P.K; k += NTH) {
      // entries of column k inside this block, summed in index order
      int i = (int)(((int64_t)k - first % P.K + P.K) % P.K);
      T acc = T(0);
      for (; i < epb && first + i < FK; i += P.K) acc += s_sq[i * G];
      static_cast<T*>(fz.normPart)[(int64_t)k * gridDim.x + b] = acc;
    }
  }
  if (fz.flags & FUSE_NO_FINALIZE) return;
  last_block_finalize<T>(fz, P, gridDim.x, s_sq);
}

// H-half epilogue over K x N entries. FUSE_LOSS finalises the objective of
// the preceding sweep; FUSE_NORM_APPLY (the iteration's last kernel) scales
// the new H rows by the column norms of W and, in extra blocks
// [totH, totH + totW), divides W's columns by them (Sec. 4.1.2).
template <typename T, int BK>
__global__ void __launch_bounds__(EW)
cols_epilogue_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefix,
                     int mode, int basesel, int want_chi, BetaParams bp, T* __restrict__ gout,
                     int* __restrict__ status, int tc, EpiFuse fz, int totH) {
  pdl_wait();
  pdl_trigger();                 // after the wait: see SWEEP_EARLY
  const bool skip = *status != 0;
  if (skip && !(fz.flags & FUSE_LOSS)) return;
  const int b = blockIdx.x;
  if ((fz.flags & FUSE_NORM_APPLY) && b >= totH) {      // W /= norms (single problem)
    const Prob<T> P = probs[0];
    const int64_t idx = (int64_t)(b - totH) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const T nk = P.norms[idx % P.K];
      if (nk > T(0)) P.W[idx] = P.W[idx] / nk;
    }
    return;
  }
  const int pi = find_problem(prefix, count, b);
  const Prob<T> P = probs[pi];
  const int64_t KN = (int64_t)P.K * P.N;
  const int64_t idx = (int64_t)(b - prefix[pi]) * EW + threadIdx.x;
  if (idx < KN && !skip) {
    T num, den;
    int slices = tc ? P.tcR : P.R;
    if (tc && P.tcSK) {                                  // stream-K: this column tile's own count
      const int64_t ft = (P.F + 31) / 32, steps = (int64_t)P.tcColTiles * ft;
      slices = sk_slices((idx % P.N) / 128, ft, steps, P.tcSKBlocks);
    }
    sum_slices(P.colPart + idx, 2 * KN, KN, slices, num, den);
    if (mode == EPI_GRAD) {
      gout[idx] = den - num;
    } else {
      const T base = basesel == SEL_TILDE ? P.Ht[idx] : P.H[idx];
      const T x = apply_floor(base * mu_ratio<BK, T>(num, den, (T)bp.gamma), (T)bp.floor);
      if (!isfinite(x)) atomicExch(status, 4);
      if (want_chi) {
        T c1, c2;
        chi_terms<BK, T>(x, P.Ht[idx], (T)bp.beta, c1, c2);
        if (tc != 2) {
          P.chiH1[idx] = c1;
          P.chiH2[idx] = c2;
        }
        if (tc && P.sCH1) {
          const int64_t k = idx / P.N, n = idx - k * P.N;
          P.sCH1[k * P.Np + n] = tf32_round(c1);
          P.sCH2[k * P.Np + n] = tf32_round(c2);
        }
      }
      T y = x;
      if (fz.flags & FUSE_NORM_APPLY) {
        const T nk = P.norms[idx / P.N];
        if (nk > T(0)) y = x * nk;
      }
      P.H[idx] = y;
    }
  }
  if (fz.flags & FUSE_LOSS) last_block_finalize<T>(fz, P, totH, nullptr);
}

// The H epilogue above (MU update only) for one float problem with N % 4 == 0
// and H 16-byte aligned: each thread takes four consecutive columns of one
// row of H (same column tile, same norm), with 16-byte loads and stores; the
// arithmetic is the same per entry. Blocks [totQ, ...) divide W's columns by
// the norms as above.
template <int BK>
__global__ void __launch_bounds__(EW)
cols_epilogue_vec4_kernel(const Prob<float>* __restrict__ probs, int basesel, int want_chi, BetaParams bp,
                          int* __restrict__ status, int tc, EpiFuse fz, int totQ) {
  pdl_wait();
  pdl_trigger();                 // after the wait: see SWEEP_EARLY
  const bool skip = *status != 0;
  if (skip && !(fz.flags & FUSE_LOSS)) return;
  const int b = blockIdx.x;
  const Prob<float> P = probs[0];
  if ((fz.flags & FUSE_NORM_APPLY) && b >= totQ) {      // W /= norms
    const int64_t idx = (int64_t)(b - totQ) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const float nk = P.norms[idx % P.K];
      if (nk > 0.f) P.W[idx] = P.W[idx] / nk;
    }
    return;
  }
  const int64_t KN = (int64_t)P.K * P.N;
  const int64_t idx = 4 * ((int64_t)b * EW + threadIdx.x);
  if (idx < KN && !skip) {
    const int64_t k = idx / P.N, n = idx - k * P.N;
    int slices = tc ? P.tcR : P.R;
    if (tc && P.tcSK) {
      const int64_t ft = (P.F + 31) / 32, T = (int64_t)P.tcColTiles * ft;
      slices = sk_slices(n / 128, ft, T, P.tcSKBlocks);
    }
    float4 num = make_float4(0.f, 0.f, 0.f, 0.f), den = num;
    const float* part = P.colPart + idx;
    for (int s0 = 0; s0 < slices; s0 += 4) {           // four slices' loads in flight, added in slice order
      float4 vn[4], vd[4];
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sl = s0 + u;
        vn[u] = sl < slices ? *reinterpret_cast<const float4*>(part + (int64_t)sl * 2 * KN) : make_float4(0.f, 0.f, 0.f, 0.f);
        vd[u] = sl < slices ? *reinterpret_cast<const float4*>(part + (int64_t)sl * 2 * KN + KN)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        num.x += vn[u].x; num.y += vn[u].y; num.z += vn[u].z; num.w += vn[u].w;
        den.x += vd[u].x; den.y += vd[u].y; den.z += vd[u].z; den.w += vd[u].w;
      }
    }
    const float nv[4] = {num.x, num.y, num.z, num.w}, dv[4] = {den.x, den.y, den.z, den.w};
    {
      const float4 ht4 = *reinterpret_cast<const float4*>(P.Ht + idx);
      const float4 b4 = basesel == SEL_TILDE ? ht4 : *reinterpret_cast<const float4*>(P.H + idx);
      const float ht[4] = {ht4.x, ht4.y, ht4.z, ht4.w}, bs[4] = {b4.x, b4.y, b4.z, b4.w};
      const float nk = (fz.flags & FUSE_NORM_APPLY) ? P.norms[k] : 0.f;
      float y[4], c1[4], c2[4];
      bool finite = true;
      #pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float x = apply_floor(bs[j] * mu_ratio<BK, float>(nv[j], dv[j], (float)bp.gamma), (float)bp.floor);
        finite = finite && isfinite(x);
        if (want_chi) chi_terms<BK, float>(x, ht[j], (float)bp.beta, c1[j], c2[j]);
        y[j] = ((fz.flags & FUSE_NORM_APPLY) && nk > 0.f) ? x * nk : x;
      }
      if (!finite) atomicExch(status, 4);
      if (want_chi) {
        if (tc != 2) {
          *reinterpret_cast<float4*>(P.chiH1 + idx) = make_float4(c1[0], c1[1], c1[2], c1[3]);
          *reinterpret_cast<float4*>(P.chiH2 + idx) = make_float4(c2[0], c2[1], c2[2], c2[3]);
        }
        if (tc && P.sCH1) {
          *reinterpret_cast<float4*>(P.sCH1 + k * P.Np + n) =
              make_float4(tf32_round(c1[0]), tf32_round(c1[1]), tf32_round(c1[2]), tf32_round(c1[3]));
          *reinterpret_cast<float4*>(P.sCH2 + k * P.Np + n) =
              make_float4(tf32_round(c2[0]), tf32_round(c2[1]), tf32_round(c2[2]), tf32_round(c2[3]));
        }
      }
      *reinterpret_cast<float4*>(P.H + idx) = make_float4(y[0], y[1], y[2], y[3]);
    }
  }
  if (fz.flags & FUSE_LOSS) last_block_finalize<float>(fz, P, totQ, nullptr);
}

// The iteration's last H epilogue (W first, normalisation on, one
// tensor-core problem) fused with the next iteration's operand copies.
// Blocks [0, nt) take a tile of 8 rows k x 32 V columns n of H each (a warp
// per row, V consecutive entries per thread; V = 4 needs N % 4 == 0 and H
// 16-byte aligned): slice sums, the MU update, the floor, the norm scaling,
// then H, Ht, the TF32 copy sHS and, through a shared-memory transpose, the
// TF32 copy sHT (N x ks: 32 bytes of each of the tile's rows n). Blocks
// [nt, ...) divide W's columns by the norms and write W, Wt, sWS and sWT.
// Every value is the one the H epilogue followed by the copies kernel would
// produce (same operations, same order).
template <int BK, int V>
__global__ void __launch_bounds__(EW)
cols_next_kernel(const Prob<float>* __restrict__ probs, BetaParams bp, int* __restrict__ status, int nt) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  constexpr int TK = EW / 32;                          // rows k per tile
  constexpr int TN = 32 * V;                           // columns n per tile
  __shared__ float tile[TN][TK + 1];                   // odd row stride: few bank conflicts
  const Prob<float> P = probs[0];
  const int b = blockIdx.x;
  if (b >= nt) {                                       // W /= norms and W's copies
    const int64_t idx = (int64_t)(b - nt) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const int64_t f = idx / P.K, k = idx - f * P.K;
      const float nk = P.norms[k];
      const float w = nk > 0.f ? P.W[idx] / nk : P.W[idx];
      P.W[idx] = w;
      P.Wt[idx] = w;
      const float r = tf32_round(w);
      P.sWS[f * P.ks + k] = r;
      P.sWT[k * P.Fp + f] = r;
    }
    return;
  }
  const int ntN = (int)((P.N + TN - 1) / TN);
  const int64_t n0 = (int64_t)(b % ntN) * TN;
  const int k0 = (b / ntN) * TK;
  const int lane = threadIdx.x & 31, kk = threadIdx.x >> 5;
  const int64_t KN = (int64_t)P.K * P.N, n = n0 + (int64_t)V * lane;
  const int k = k0 + kk;
  if (n < P.N && k < P.K) {
    int slices = P.tcR;
    if (P.tcSK) {                                      // stream-K: this column tile's own count
      const int64_t ft = (P.F + 31) / 32, steps = (int64_t)P.tcColTiles * ft;
      slices = sk_slices(n / 128, ft, steps, P.tcSKBlocks);
    }
    const int64_t idx = (int64_t)k * P.N + n;
    const float nk = P.norms[k];
    float y[V];
    bool finite = true;
    if (V == 1) {
      float num, den;
      sum_slices(P.colPart + idx, 2 * KN, KN, slices, num, den);
      const float x = apply_floor(P.Ht[idx] * mu_ratio<BK, float>(num, den, (float)bp.gamma), (float)bp.floor);
      finite = isfinite(x);
      y[0] = nk > 0.f ? x * nk : x;
      P.H[idx] = y[0];
      P.Ht[idx] = y[0];
    } else {
      float4 num = make_float4(0.f, 0.f, 0.f, 0.f), den = num;
      const float* part = P.colPart + idx;
      for (int s0 = 0; s0 < slices; s0 += 4) {         // four slices' loads in flight, added in slice order
        float4 vn[4], vd[4];
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int sl = s0 + u;
          vn[u] = sl < slices ? *reinterpret_cast<const float4*>(part + (int64_t)sl * 2 * KN) : make_float4(0.f, 0.f, 0.f, 0.f);
          vd[u] = sl < slices ? *reinterpret_cast<const float4*>(part + (int64_t)sl * 2 * KN + KN)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
          num.x += vn[u].x; num.y += vn[u].y; num.z += vn[u].z; num.w += vn[u].w;
          den.x += vd[u].x; den.y += vd[u].y; den.z += vd[u].z; den.w += vd[u].w;
        }
      }
      const float nv[4] = {num.x, num.y, num.z, num.w}, dv[4] = {den.x, den.y, den.z, den.w};
      const float4 ht4 = *reinterpret_cast<const float4*>(P.Ht + idx);
      const float ht[4] = {ht4.x, ht4.y, ht4.z, ht4.w};
      #pragma unroll
      for (int j = 0; j < V; ++j) {
        const float x = apply_floor(ht[j] * mu_ratio<BK, float>(nv[j], dv[j], (float)bp.gamma), (float)bp.floor);
        finite = finite && isfinite(x);
        y[j] = nk > 0.f ? x * nk : x;
      }
      const float4 y4 = make_float4(y[0], y[1], y[2], y[3]);
      *reinterpret_cast<float4*>(P.H + idx) = y4;
      *reinterpret_cast<float4*>(P.Ht + idx) = y4;
    }
    if (!finite) atomicExch(status, 4);
    float r[V];
    #pragma unroll
    for (int j = 0; j < V; ++j) {
      r[j] = tf32_round(y[j]);
      tile[V * lane + j][kk] = r[j];
    }
    if (V == 1) P.sHS[(int64_t)k * P.Np + n] = r[0];
    else *reinterpret_cast<float4*>(P.sHS + (int64_t)k * P.Np + n) = make_float4(r[0], r[1], r[2], r[3]);
  }
  __syncthreads();
  if (V == 1) {
    const int nl = threadIdx.x / TK, kt = threadIdx.x % TK;   // 32 rows n x TK columns k
    if (n0 + nl < P.N && k0 + kt < P.K) P.sHT[(n0 + nl) * P.ks + k0 + kt] = tile[nl][kt];
  } else {
    // 128 rows n x 8 columns k: two 16-byte pieces per row (k0 and ks are
    // multiples of 8, so each piece is aligned); columns k >= K stay zero
    const int nl = threadIdx.x >> 1, h = threadIdx.x & 1;
    if (n0 + nl < P.N) {
      float4 v = make_float4(tile[nl][4 * h], tile[nl][4 * h + 1], tile[nl][4 * h + 2], tile[nl][4 * h + 3]);
      const int kb = k0 + 4 * h;
      if (kb + 0 >= P.K) v.x = 0.f;
      if (kb + 1 >= P.K) v.y = 0.f;
      if (kb + 2 >= P.K) v.z = 0.f;
      if (kb + 3 >= P.K) v.w = 0.f;
      if (kb < P.K) *reinterpret_cast<float4*>(P.sHT + (n0 + nl) * P.ks + kb) = v;
    }
  }
}

// Normalisation of one problem from the W epilogue's norm partials
// ([K][nparts]): every block reduces them itself (R threads per column, then
// a fixed-order sum: the same norms in every block), then blocks [0, totW)
// divide W's columns by them and blocks [totW, ...) scale H's rows.
template <typename T>
__global__ void __launch_bounds__(EW)
normalize_parts_kernel(const Prob<T>* __restrict__ probs, const T* __restrict__ normPart, int nparts, int totW,
                       const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  __shared__ T s_red[EW];
  __shared__ T s_norm[KMAX];
  const Prob<T> P = probs[0];
  const int K = P.K, R = EW / K;
  T v = T(0);
  if ((int)threadIdx.x < R * K) {
    const int k = threadIdx.x / R, j = threadIdx.x - k * R;
    const T* row = normPart + (int64_t)k * nparts;
    for (int b0 = j; b0 < nparts; b0 += 4 * R) {
      T u4[4];
      #pragma unroll
      for (int u = 0; u < 4; ++u) u4[u] = b0 + u * R < nparts ? row[b0 + u * R] : T(0);
      #pragma unroll
      for (int u = 0; u < 4; ++u) v += u4[u];
    }
  }
  s_red[threadIdx.x] = v;
  __syncthreads();
  if ((int)threadIdx.x < K) {
    T sum = T(0);
    for (int j = 0; j < R; ++j) sum += s_red[threadIdx.x * R + j];
    s_norm[threadIdx.x] = sqrt(sum);
    if (blockIdx.x == 0) P.norms[threadIdx.x] = s_norm[threadIdx.x];
  }
  __syncthreads();
  const int b = blockIdx.x;
  if (b < totW) {
    const int64_t idx = (int64_t)b * EW + threadIdx.x;
    if (idx < P.F * K) {
      const T nk = s_norm[idx % K];
      if (nk > T(0)) P.W[idx] = P.W[idx] / nk;
    }
  } else {
    const int64_t idx = (int64_t)(b - totW) * EW + threadIdx.x;
    if (idx < (int64_t)K * P.N) {
      const T nk = s_norm[idx / P.N];
      if (nk > T(0)) P.H[idx] = P.H[idx] * nk;
    }
  }
}

// Blocks [0, totW) copy W -> Wt, blocks [totW, totW + totH) copy H -> Ht.
template <typename T>
__global__ void __launch_bounds__(EW)
begin_iteration_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefW,
                       int totW, const int* __restrict__ prefH, const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  int b = blockIdx.x;
  if (b < totW) {
    const int pi = find_problem(prefW, count, b);
    const Prob<T> P = probs[pi];
    const int64_t idx = (int64_t)(b - prefW[pi]) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const T w = P.W[idx];
      P.Wt[idx] = w;
      if (P.sWS) {                         // TF32 shadows for the tensor-core sweeps
        const int64_t f = idx / P.K, k = idx - f * P.K;
        P.sWS[f * P.ks + k] = tf32_round(w);
        P.sWT[k * P.Fp + f] = tf32_round(w);
      }
    }
  } else {
    b -= totW;
    const int pi = find_problem(prefH, count, b);
    const Prob<T> P = probs[pi];
    const int64_t idx = (int64_t)(b - prefH[pi]) * EW + threadIdx.x;
    if (idx < (int64_t)P.K * P.N) {
      const T h = P.H[idx];
      P.Ht[idx] = h;
      if (P.sHT) {
        const int64_t k = idx / P.N, n = idx - k * P.N;
        P.sHT[n * P.ks + k] = tf32_round(h);
        P.sHS[k * P.Np + n] = tf32_round(h);
      }
    }
  }
}

// One block per column k of W: norms[k] = ||W[:, k]||_2 (fixed-order sum).
template <typename T>
__global__ void __launch_bounds__(EW)
colnorm_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefK,
               const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  __shared__ double red[32];
  const int b = blockIdx.x;
  const int pi = find_problem(prefK, count, b);
  const Prob<T> P = probs[pi];
  const int k = b - prefK[pi];
  double s = 0.0;
  for (int64_t f = threadIdx.x; f < P.F; f += EW) {
    const double w = (double)P.W[f * P.K + k];
    s += w * w;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) P.norms[k] = (T)sqrt(s);
}

template <typename T>
__global__ void __launch_bounds__(EW)
normalize_apply_kernel(const Prob<T>* __restrict__ probs, int count, const int* __restrict__ prefW,
                       int totW, const int* __restrict__ prefH, const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  int b = blockIdx.x;
  if (b < totW) {
    const int pi = find_problem(prefW, count, b);
    const Prob<T> P = probs[pi];
    const int64_t idx = (int64_t)(b - prefW[pi]) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const T nk = P.norms[idx % P.K];
      if (nk > T(0)) P.W[idx] = P.W[idx] / nk;
    }
  } else {
    b -= totW;
    const int pi = find_problem(prefH, count, b);
    const Prob<T> P = probs[pi];
    const int64_t idx = (int64_t)(b - prefH[pi]) * EW + threadIdx.x;
    if (idx < (int64_t)P.K * P.N) {
      const T nk = P.norms[idx / P.N];
      if (nk > T(0)) P.H[idx] = P.H[idx] * nk;
    }
  }
}

// Shadows of the current W (which & 1) and / or H (which & 2), TF32-rounded,
// in the layouts the tensor-core sweeps load by TMA (single problem).
template <typename T>
__global__ void __launch_bounds__(EW)
shadow_factors_kernel(Prob<T> P, int which, const int* __restrict__ status) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  const int64_t FK = P.F * P.K, KN = (int64_t)P.K * P.N;
  const int64_t lo = (which & 1) ? 0 : FK, hi = (which & 2) ? FK + KN : FK;
  for (int64_t i = lo + (int64_t)blockIdx.x * EW + threadIdx.x; i < hi; i += (int64_t)gridDim.x * EW) {
    if (i < FK) {
      const int64_t f = i / P.K, k = i - f * P.K;
      const T w = tf32_round(P.W[i]);
      P.sWS[f * P.ks + k] = w;
      P.sWT[k * P.Fp + f] = w;
    } else {
      const int64_t j = i - FK, k = j / P.N, n = j - k * P.N;
      const T h = tf32_round(P.H[j]);
      P.sHT[n * P.ks + k] = h;
      P.sHS[k * P.Np + n] = h;
    }
  }
}

// Tensor-core copies of the factors for one problem, written coalesced.
// Blocks [0, wBlocks) take EW entries of W each (W~ copy when `tilde`, then the
// TF32 copies sWS (F x ks) and sWT (K x Fp)); block wBlocks + b takes columns
// [32 b, 32 b + 32) of H, all K rows: read along n, H~ and sHS (K x Np) written
// along n, sHT (N x ks) written along k after a transpose in shared memory
// (a direct transposed store would put every element in its own sector).
// mode (the fused single-read path's last kernel, COPIES_*): APPLY scales W's
// columns down and H's rows up by P.norms (Sec. 4.1.2) and writes W and H
// back before copying; LEAN skips the copies that path does not read (sWT, sHS).
template <typename T>
__global__ void __launch_bounds__(EW)
tc_copies_kernel(Prob<T> P, int wBlocks, int doW, int doH, int tilde, const int* __restrict__ status, int mode) {
  pdl_trigger();
  pdl_wait();
  if (*status) return;
  __shared__ float tile[32][KMAX + 1];
  if ((int)blockIdx.x < wBlocks) {
    if (!doW) return;
    const int64_t idx = (int64_t)blockIdx.x * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      T w = P.W[idx];
      const int64_t f = idx / P.K, k = idx - f * P.K;
      if (mode & COPIES_APPLY) {
        const T nk = P.norms[k];
        if (nk > T(0)) w = w / nk;
        P.W[idx] = w;
      }
      if (tilde) P.Wt[idx] = w;
      const float r = tf32_round((float)w);
      P.sWS[f * P.ks + k] = (T)r;
      if (!(mode & COPIES_LEAN)) P.sWT[k * P.Fp + f] = (T)r;
    }
    return;
  }
  if (!doH) return;
  const int64_t n0 = (int64_t)(blockIdx.x - wBlocks) * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = n0 + lane;
  for (int k = w; k < P.K; k += EW / 32) {
    if (n < P.N) {
      T h = P.H[(int64_t)k * P.N + n];
      if (mode & COPIES_APPLY) {
        const T nk = P.norms[k];
        if (nk > T(0)) h = h * nk;
        P.H[(int64_t)k * P.N + n] = h;
      }
      if (tilde) P.Ht[(int64_t)k * P.N + n] = h;
      const float r = tf32_round((float)h);
      if (!(mode & COPIES_LEAN)) P.sHS[(int64_t)k * P.Np + n] = (T)r;
      tile[lane][k] = r;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * P.K; i += EW) {
    const int nl = i / P.K, k = i - nl * P.K;
    if (n0 + nl < P.N) P.sHT[(n0 + nl) * P.ks + k] = (T)tile[nl][k];
  }
}

template <typename T>
cudaError_t launch_tc_copies(const Prob<T>& P, bool doW, bool doH, bool tilde, const int* status, cudaStream_t st) {
  const int wBlocks = doW ? (int)((P.F * P.K + EW - 1) / EW) : 0;
  const int hBlocks = doH ? (int)((P.N + 31) / 32) : 0;
  if (wBlocks + hBlocks == 0) return cudaSuccess;
  return launch_pdl(tc_copies_kernel<T>, dim3(wBlocks + hBlocks), dim3(EW), 0, st, P, wBlocks, doW ? 1 : 0, doH ? 1 : 0,
                    tilde ? 1 : 0, status, 0);
}

template <typename T>
cudaError_t launch_fused_next(const Prob<T>& P, bool norm, const int* status, cudaStream_t st) {
  const int wBlocks = (int)((P.F * P.K + EW - 1) / EW);
  const int hBlocks = (int)((P.N + 31) / 32);
  return launch_pdl(tc_copies_kernel<T>, dim3(wBlocks + hBlocks), dim3(EW), 0, st, P, wBlocks, 1, 1, 1, status,
                    COPIES_LEAN | (norm ? COPIES_APPLY : 0));
}

template <typename T>
cudaError_t launch_shadow_factors(const Prob<T>& P, int which, const int* status, cudaStream_t st) {
  return launch_tc_copies<T>(P, (which & 1) != 0, (which & 2) != 0, false, status, st);
}

template <typename T>
__global__ void __launch_bounds__(EW)
kkt_kernel(const T* __restrict__ W, const T* __restrict__ gW, int64_t nW, const T* __restrict__ H,
           const T* __restrict__ gH, int64_t nH, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  __shared__ double red[32];
  double sw = 0.0, sh = 0.0;
  for (int64_t i = threadIdx.x; i < nW; i += EW) sw += fabs((double)min(W[i], gW[i]));
  for (int64_t i = threadIdx.x; i < nH; i += EW) sh += fabs((double)min(H[i], gH[i]));
  sw = block_sum(sw, red);
  __syncthreads();
  sh = block_sum(sh, red);
  if (threadIdx.x == 0) { out[0] = sw; out[1] = sh; }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

template <typename T>
inline size_t row_smem_bytes(int K, int dsel) {
  return sizeof(T) * ((size_t)BF * (K + 1) + (size_t)K * TP * (dsel == OP_CHI ? 3 : 1) + 2 * BF * TP);
}
template <typename T>
inline size_t col_smem_bytes(int K, int csel) {
  return sizeof(T) * ((size_t)K * TP + (size_t)BF * (K + 1) * (csel == OP_CHI ? 3 : 1) + 2 * BF * TP);
}

template <typename KernelT>
inline cudaError_t prep_smem(KernelT kernel, size_t bytes) {
  return ensure_smem_attr(reinterpret_cast<const void*>(kernel), bytes);
}

template <typename T, int BK, int KJ>
cudaError_t row_sweep_bk_kj(const Plan<T>& pl, int wsel, int hsel, int dsel, int flags,
                            const BetaParams& bp, double* lossPart, const int* status,
                            cudaStream_t st) {
  auto kern = row_sweep_kernel<T, BK, KJ>;
  const size_t sm = row_smem_bytes<T>(pl.maxK, dsel);
  cudaError_t e = prep_smem(kern, sm);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t le_ = launch_pdl(kern, dim3(pl.totRow), dim3(NT), sm, st, pl.d_probs, pl.count, pl.d_prefRow, wsel, hsel, dsel, flags, bp, lossPart, status);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T, int BK>
cudaError_t row_sweep_bk(const Plan<T>& pl, int wsel, int hsel, int dsel, int flags,
                         const BetaParams& bp, double* lossPart, const int* status, cudaStream_t st) {
  if (pl.maxK <= 32) return row_sweep_bk_kj<T, BK, 1>(pl, wsel, hsel, dsel, flags, bp, lossPart, status, st);
  if (pl.maxK <= 64) return row_sweep_bk_kj<T, BK, 2>(pl, wsel, hsel, dsel, flags, bp, lossPart, status, st);
  return row_sweep_bk_kj<T, BK, 4>(pl, wsel, hsel, dsel, flags, bp, lossPart, status, st);
}

template <typename T, int BK, int KJ8>
cudaError_t col_sweep_bk_kj(const Plan<T>& pl, int wsel, int hsel, int csel, int flags,
                            const BetaParams& bp, double* lossPart, const int* status,
                            cudaStream_t st) {
  auto kern = col_sweep_kernel<T, BK, KJ8>;
  const size_t sm = col_smem_bytes<T>(pl.maxK, csel);
  cudaError_t e = prep_smem(kern, sm);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t le_ = launch_pdl(kern, dim3(pl.totCol), dim3(NT), sm, st, pl.d_probs, pl.count, pl.d_prefCol, wsel, hsel, csel, flags, bp, lossPart, status);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T, int BK>
cudaError_t col_sweep_bk(const Plan<T>& pl, int wsel, int hsel, int csel, int flags,
                         const BetaParams& bp, double* lossPart, const int* status, cudaStream_t st) {
  if (pl.maxK <= 16) return col_sweep_bk_kj<T, BK, 2>(pl, wsel, hsel, csel, flags, bp, lossPart, status, st);
  if (pl.maxK <= 32) return col_sweep_bk_kj<T, BK, 4>(pl, wsel, hsel, csel, flags, bp, lossPart, status, st);
  if (pl.maxK <= 64) return col_sweep_bk_kj<T, BK, 8>(pl, wsel, hsel, csel, flags, bp, lossPart, status, st);
  return col_sweep_bk_kj<T, BK, 16>(pl, wsel, hsel, csel, flags, bp, lossPart, status, st);
}

#define NMF_BK_DISPATCH(FN, ...)                                   \
  switch (bp.kind) {                                               \
    case BK_IS: return FN<T, BK_IS>(__VA_ARGS__);                  \
    case BK_KL: return FN<T, BK_KL>(__VA_ARGS__);                  \
    case BK_EUC: return FN<T, BK_EUC>(__VA_ARGS__);                \
    case BK_B15: return FN<T, BK_B15>(__VA_ARGS__);                \
    default: return FN<T, BK_GENERAL>(__VA_ARGS__);                \
  }

template <typename T>
cudaError_t launch_row_sweep(const Plan<T>& pl, int wsel, int hsel, int dsel, int flags,
                             const BetaParams& bp, double* lossPart, const int* status,
                             cudaStream_t st) {
  NMF_BK_DISPATCH(row_sweep_bk, pl, wsel, hsel, dsel, flags, bp, lossPart, status, st)
}

template <typename T>
cudaError_t launch_col_sweep(const Plan<T>& pl, int wsel, int hsel, int csel, int flags,
                             const BetaParams& bp, double* lossPart, const int* status,
                             cudaStream_t st) {
  NMF_BK_DISPATCH(col_sweep_bk, pl, wsel, hsel, csel, flags, bp, lossPart, status, st)
}

template <typename T, int BK>
cudaError_t rows_epi_bk(const Plan<T>& pl, int mode, int basesel, int want_chi,
                        const BetaParams& bp, T* gout, int* status, cudaStream_t st, int tc, const EpiFuse& fz) {
  const int G = rows_epilogue_lanes(pl, tc);
  if (pl.count == 1)
    {
      const cudaError_t le_ = launch_pdl(rows_epilogue_kernel<T, BK, 1024>, dim3(rows_epilogue_grid(pl.totW, G)), dim3(1024), 0, st, pl.d_probs, pl.count, pl.d_prefW, mode, basesel, want_chi, bp, gout, status, tc, fz, G);
      if (le_ != cudaSuccess) return le_;
    }
  else
    {
      const cudaError_t le_ = launch_pdl(rows_epilogue_kernel<T, BK, EW>, dim3(pl.totW), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefW, mode, basesel, want_chi, bp, gout, status, tc, fz, 1);
      if (le_ != cudaSuccess) return le_;
    }
  return cudaGetLastError();
}
template <typename T, int BK>
cudaError_t cols_epi_bk(const Plan<T>& pl, int mode, int basesel, int want_chi,
                        const BetaParams& bp, T* gout, int* status, cudaStream_t st, int tc, const EpiFuse& fz) {
  if constexpr (std::is_same<T, float>::value) {
    if (pl.colVec4 && mode != EPI_GRAD) {                // (gradient buffers are the caller's: alignment unknown)
      const int totQ = (pl.totH + 3) / 4;               // totH blocks of EW entries -> quads
      const int grid = totQ + ((fz.flags & FUSE_NORM_APPLY) ? pl.totW : 0);
      const cudaError_t le_ = launch_pdl(cols_epilogue_vec4_kernel<BK>, dim3(grid), dim3(EW), 0, st,
                                         (const Prob<float>*)pl.d_probs, basesel, want_chi, bp, status, tc, fz, totQ);
      if (le_ != cudaSuccess) return le_;
      return cudaGetLastError();
    }
  }
  const int grid = pl.totH + ((fz.flags & FUSE_NORM_APPLY) ? pl.totW : 0);
  {
    const cudaError_t le_ = launch_pdl(cols_epilogue_kernel<T, BK>, dim3(grid), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefH, mode, basesel, want_chi, bp, gout, status, tc, fz, pl.totH);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_epilogue(const Plan<T>& pl, int mode, int basesel, int want_chi,
                                 const BetaParams& bp, T* gout, int* status, cudaStream_t st, int tc,
                                 const EpiFuse& fz) {
  NMF_BK_DISPATCH(rows_epi_bk, pl, mode, basesel, want_chi, bp, gout, status, st, tc, fz)
}
template <typename T>
cudaError_t launch_cols_epilogue(const Plan<T>& pl, int mode, int basesel, int want_chi,
                                 const BetaParams& bp, T* gout, int* status, cudaStream_t st, int tc,
                                 const EpiFuse& fz) {
  NMF_BK_DISPATCH(cols_epi_bk, pl, mode, basesel, want_chi, bp, gout, status, st, tc, fz)
}

// W /= norms, H *= norms from P.norms (the norms a fused W epilogue produced).
template <typename T>
cudaError_t launch_normalize_apply(const Plan<T>& pl, const int* status, cudaStream_t st) {
  {
    const cudaError_t le_ = launch_pdl(normalize_apply_kernel<T>, dim3(pl.totW + pl.totH), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefW, pl.totW, pl.d_prefH, status);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_normalize_parts(const Plan<T>& pl, const T* normPart, int nparts, const int* status,
                                   cudaStream_t st) {
  if (pl.count != 1 || pl.maxK > EW) return cudaErrorInvalidValue;
  const cudaError_t le = launch_pdl(normalize_parts_kernel<T>, dim3(pl.totW + pl.totH), dim3(EW), 0, st,
                                    (const Prob<T>*)pl.d_probs, normPart, nparts, pl.totW, status);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cols_next(const Plan<T>& pl, const Prob<T>& hp, const BetaParams& bp, int* status,
                             cudaStream_t st) {
  if constexpr (!std::is_same<T, float>::value) {
    return cudaErrorInvalidValue;
  } else {
    if (pl.count != 1 || hp.K > KMAX || !hp.sWS || !hp.sHT || hp.ks % 8 != 0) return cudaErrorInvalidValue;
    const bool v4 = pl.colVec4;
    const int64_t tn = v4 ? 128 : 32;
    const int nt = (int)(((hp.N + tn - 1) / tn) * ((hp.K + EW / 32 - 1) / (EW / 32)));
    const dim3 grid((unsigned)(nt + (hp.F * hp.K + EW - 1) / EW));
    const Prob<float>* probs = pl.d_probs;
    cudaError_t le = cudaErrorInvalidValue;
#define NMF_NEXT_CASE(BKV)                                                                                  \
  case BKV:                                                                                                 \
    le = v4 ? launch_pdl(cols_next_kernel<BKV, 4>, grid, dim3(EW), 0, st, probs, bp, status, nt)            \
            : launch_pdl(cols_next_kernel<BKV, 1>, grid, dim3(EW), 0, st, probs, bp, status, nt);           \
    break;
    switch (bp.kind) {
      NMF_NEXT_CASE(BK_IS)
      NMF_NEXT_CASE(BK_KL)
      NMF_NEXT_CASE(BK_EUC)
      NMF_NEXT_CASE(BK_B15)
      default:
        le = v4 ? launch_pdl(cols_next_kernel<BK_GENERAL, 4>, grid, dim3(EW), 0, st, probs, bp, status, nt)
                : launch_pdl(cols_next_kernel<BK_GENERAL, 1>, grid, dim3(EW), 0, st, probs, bp, status, nt);
    }
#undef NMF_NEXT_CASE
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
  }
}

template <typename T>
cudaError_t launch_begin_iteration(const Plan<T>& pl, const int* status, cudaStream_t st) {
  {
    const cudaError_t le_ = launch_pdl(begin_iteration_kernel<T>, dim3(pl.totW + pl.totH), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefW, pl.totW, pl.d_prefH, status);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_normalize(const Plan<T>& pl, const int* status, cudaStream_t st) {
  {
    const cudaError_t le_ = launch_pdl(colnorm_kernel<T>, dim3(pl.totK), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefK, status);
    if (le_ != cudaSuccess) return le_;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    const cudaError_t le_ = launch_pdl(normalize_apply_kernel<T>, dim3(pl.totW + pl.totH), dim3(EW), 0, st, pl.d_probs, pl.count, pl.d_prefW, pl.totW, pl.d_prefH, status);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kkt(const T* W, const T* gW, int64_t nW, const T* H, const T* gH, int64_t nH,
                       double* out, cudaStream_t st) {
  {
    const cudaError_t le_ = launch_pdl(kkt_kernel<T>, dim3(1), dim3(EW), 0, st, W, gW, nW, H, gH, nH, out);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

#define NMF_INSTANTIATE_SWEEPS(T)                                                                   \
  template cudaError_t launch_row_sweep<T>(const Plan<T>&, int, int, int, int, const BetaParams&,  \
                                           double*, const int*, cudaStream_t);                     \
  template cudaError_t launch_col_sweep<T>(const Plan<T>&, int, int, int, int, const BetaParams&,  \
                                           double*, const int*, cudaStream_t);                     \
  template cudaError_t launch_rows_epilogue<T>(const Plan<T>&, int, int, int, const BetaParams&,   \
                                               T*, int*, cudaStream_t, int, const EpiFuse&);       \
  template cudaError_t launch_cols_epilogue<T>(const Plan<T>&, int, int, int, const BetaParams&,   \
                                               T*, int*, cudaStream_t, int, const EpiFuse&);       \
  template cudaError_t launch_normalize_apply<T>(const Plan<T>&, const int*, cudaStream_t);        \
  template cudaError_t launch_begin_iteration<T>(const Plan<T>&, const int*, cudaStream_t);        \
  template cudaError_t launch_normalize_parts<T>(const Plan<T>&, const T*, int, const int*, cudaStream_t); \
  template cudaError_t launch_tc_copies<T>(const Prob<T>&, bool, bool, bool, const int*, cudaStream_t); \
  template cudaError_t launch_fused_next<T>(const Prob<T>&, bool, const int*, cudaStream_t);       \
  template cudaError_t launch_cols_next<T>(const Plan<T>&, const Prob<T>&, const BetaParams&, int*, cudaStream_t); \
  template cudaError_t launch_normalize<T>(const Plan<T>&, const int*, cudaStream_t);              \
  template cudaError_t launch_kkt<T>(const T*, const T*, int64_t, const T*, const T*, int64_t,     \
                                     double*, cudaStream_t);                                       \
  template cudaError_t launch_shadow_factors<T>(const Prob<T>&, int, const int*, cudaStream_t);

}  // namespace nmf
