// tc_sweeps.cu -- tensor-core (tcgen05, kind::tf32) versions of the two sweeps.
//
// Same contract as the SIMT sweeps (sweeps_impl.cuh): with Vp = Wp Hp + kappa,
// A = (V + kappa) . Vp^(beta-2), B = Vp . Vp^(beta-2) (eq. alt_update /
// eq. jnt_update),
//   row sweep    P = A D1^T, Q = B D2^T  (F x K, reduced over n)
//   column sweep Hn = C1^T A, Hd = C2^T B (K x N, reduced over f)
// written as fixed slices of partial sums that the epilogue kernels add.
//
// All three products per tile run on the tensor cores with FP32 accumulation
// in tensor memory; the operands are rounded to TF32 (round to nearest) when
// staged. The powers, the objective and the staging run on the CUDA cores.
//
// Row sweep (M = 128 rows f of the tile, loop over 32-column tiles n):
//   MMA1: Vp[f, n]  (TMEM, 32 columns)  = Wp[f, :] . Hp[:, n]       (K-dim = kp)
//   CUDA cores: Vp -> A[f, n], B[f, n] into 128B-swizzled shared tiles
//   MMA2: P[f, k]   (TMEM, kp columns) += A[f, n] . D1[k, n]^T      (K-dim = 32)
//   MMA3: Q[f, k]   (TMEM, kp columns) += B[f, n] . D2[k, n]^T
// Column sweep (M = 128 columns n, loop over 32-row tiles f): the transpose,
//   MMA1: Vp^T[n, f] = Hp^T[n, :] . Wp[f, :]^T; MMA2/3: Hn^T[n, k] += A^T[n, f] . C1[f, k].
//
// Every shared operand is K-major with the 128-byte swizzle (tc_ptx.cuh);
// K-atoms of 32 fp32 are stacked. Waits on MMA completion are bounded (1 s):
// a timeout sets the status word to NMF_ETIMEOUT and the block frees its
// tensor memory and returns.
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace nmf {
using namespace tc;

namespace {

constexpr int TC_THREADS = 256;   // 8 warps: warps w and w+4 share TMEM lanes 32(w%4)..+31
constexpr int TL = 32;            // n-tile of the row sweep, f-tile of the column sweep
constexpr int MT = 128;           // MMA M
constexpr uint32_t TILE_BYTES = 128u * 128u;   // one K-atom of a 128-row operand (16 KB)
constexpr int ETIMEOUT = 5;

__host__ __device__ inline int natoms_of(int kp) { return (kp + 31) / 32; }
// TMEM columns: Vp at [0, 32), the two accumulators at 128 and 128 + (64 | 128).
__host__ __device__ inline uint32_t tmem_cols_of(int kp) { return kp <= 64 ? 256u : 512u; }
__host__ __device__ inline uint32_t tmem_second_acc(int kp) { return 128u + (kp <= 64 ? 64u : 128u); }

inline size_t row_smem(int kp) {
  const int na = natoms_of(kp);
  return 1024 + (size_t)na * TILE_BYTES          // Ws   [128 f][kp]
         + (size_t)na * TL * 128                 // HsT  [32 n][kp]
         + 2 * (size_t)kp * 128                  // D1s, D2s [kp k][32 n]
         + 3 * (size_t)TILE_BYTES;               // Vs, As, Bs [128 f][32 n]
}
inline size_t col_smem(int kp) {
  const int na = natoms_of(kp);
  return 1024 + (size_t)na * TILE_BYTES          // HsT  [128 n][kp]
         + (size_t)na * TL * 128                 // Ws   [32 f][kp]
         + 2 * (size_t)kp * 128                  // C1s, C2s [kp k][32 f]
         + 3 * (size_t)TILE_BYTES;               // Vs [32 f][128 n], As, Bs [128 n][32 f]
}

__device__ __forceinline__ void st_f32(unsigned char* base, uint32_t off, float x) {
  *reinterpret_cast<float*>(base + off) = x;
}

// Bounded wait shared by the whole block: returns false (after recording a
// timeout) if any thread gave up, so every thread leaves the loop together.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, int* s_abort, int* status) {
  if (!mbar_wait(bar, parity)) {
    *s_abort = 1;
    atomicExch(status, ETIMEOUT);
  }
  __syncthreads();
  return *s_abort == 0;
}

template <int BK>
__global__ void __launch_bounds__(TC_THREADS)
tc_row_sweep_kernel(Prob<float> P, int wsel, int hsel, int dsel, int flags, BetaParams bp,
                    double* __restrict__ lossPart, int* __restrict__ status) {
  if (*status) return;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_v, bar_pq;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  __shared__ double red[32];
  const int K = P.K, kp = (K + 15) & ~15, na = natoms_of(kp);
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Ws = base;
  unsigned char* HsT = Ws + na * TILE_BYTES;
  unsigned char* D1s = HsT + na * TL * 128;
  unsigned char* D2s = D1s + kp * 128;
  unsigned char* Vs = D2s + kp * 128;
  unsigned char* As = Vs + TILE_BYTES;
  unsigned char* Bs = As + TILE_BYTES;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ft = blockIdx.x / P.tcSplitS, s = blockIdx.x % P.tcSplitS;
  const int64_t f0 = (int64_t)ft * MT;
  const int64_t nBeg = (int64_t)s * P.tcChunkN;
  const int64_t nEnd = nBeg + P.tcChunkN < P.N ? nBeg + P.tcChunkN : P.N;
  const float* __restrict__ Wp = wsel == SEL_TILDE ? P.Wt : P.W;
  const float* __restrict__ Hp = hsel == SEL_TILDE ? P.Ht : P.H;
  const bool wantLoss = flags & SWEEP_LOSS;
  const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
  const uint32_t ncols = tmem_cols_of(kp);

  if (tid == 0) {
    s_abort = 0;
    mbar_init(&bar_v, 1);
    mbar_init(&bar_pq, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  // Wp rows [f0, f0+128) -> Ws (K-major, one K-atom per 32 k)
  for (int i = tid; i < MT * kp; i += TC_THREADS) {
    const int f = i / kp, k = i - f * kp;
    const int64_t gf = f0 + f;
    const float w = (k < K && gf < P.F) ? Wp[gf * K + k] : 0.f;
    st_f32(Ws + (k >> 5) * TILE_BYTES, sw128_offset(f, 4 * (k & 31)), to_tf32(w));
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t t_v = tbase, t_p = tbase + 128, t_q = tbase + tmem_second_acc(kp);
  const uint32_t id_v = idesc(MT, TL, kFmtTF32), id_pq = idesc(MT, kp, kFmtTF32);
  const int q4 = warp & 3, half = warp >> 2;
  const int frow = 32 * q4 + lane;          // this thread's TMEM lane = tile row f
  const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
  double loss = 0.0;
  int tile = 0;
  for (int64_t n0 = nBeg; n0 < nEnd; n0 += TL, ++tile) {
    // stage Hp^T (B operand of MMA1), D1/D2 (B operands of MMA2/3) and V
    for (int i = tid; i < TL * kp; i += TC_THREADS) {
      const int k = i / TL, n = i - k * TL;
      const int64_t gn = n0 + n;
      const bool in = k < K && gn < nEnd;
      const float h = in ? Hp[(int64_t)k * P.N + gn] : 0.f;
      st_f32(HsT + (k >> 5) * (TL * 128), sw128_offset(n, 4 * (k & 31)), to_tf32(h));
      if (dsel == OP_CHI) {
        st_f32(D1s, sw128_offset(k, 4 * n), to_tf32(in ? P.chiH1[(int64_t)k * P.N + gn] : 0.f));
        st_f32(D2s, sw128_offset(k, 4 * n), to_tf32(in ? P.chiH2[(int64_t)k * P.N + gn] : 0.f));
      } else {
        st_f32(D1s, sw128_offset(k, 4 * n), to_tf32(h));
      }
    }
    for (int i = tid; i < MT * TL; i += TC_THREADS) {
      const int f = i / TL, n = i - f * TL;
      const int64_t gf = f0 + f, gn = n0 + n;
      st_f32(Vs, sw128_offset(f, 4 * n), (gf < P.F && gn < nEnd) ? P.V[gf * P.ldv + gn] : 0.f);
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      for (int ks = 0; ks < kp / 8; ++ks) {
        const int k0 = ks * 8;
        const uint32_t within = (uint32_t)(k0 & 31) * 4u;
        const uint64_t ad = desc_sw128(smem_u32(Ws + (k0 >> 5) * TILE_BYTES) + within);
        const uint64_t bd = desc_sw128(smem_u32(HsT + (k0 >> 5) * (TL * 128)) + within);
        mma_tf32(t_v, ad, bd, id_v, ks > 0);
      }
      mma_commit(&bar_v);
    }
    if (!block_wait(&bar_v, tile & 1, &s_abort, status)) break;
    fence_after_sync();
    // Vp row f, columns [16 half, 16 half + 16) -> A, B
    {
      float vt[16];
      tmem_ld16(t_v + lane_off + 16 * half, vt);
      tmem_ld_wait();
      const int64_t gf = f0 + frow;
      float tl = 0.f;
      #pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int nb = 16 * half + 4 * c;
        const uint32_t off = sw128_offset(frow, 4 * nb);
        const float4 v4 = *reinterpret_cast<const float4*>(Vs + off);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
        float a[4], b[4];
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool valid = gf < P.F && n0 + nb + j < nEnd;
          a[j] = 0.f;
          b[j] = 0.f;
          if (valid) {
            const float v = vv[j] + kappa, y = vt[4 * c + j] + kappa;
            ab_terms_g<BK>(v, y, bm2, a[j], b[j], bp.tiny);
            if (wantLoss) tl += (float)DB<float>::eval(v, y, bp, BK);
          }
        }
        *reinterpret_cast<float4*>(As + off) = make_float4(to_tf32(a[0]), to_tf32(a[1]), to_tf32(a[2]), to_tf32(a[3]));
        *reinterpret_cast<float4*>(Bs + off) = make_float4(to_tf32(b[0]), to_tf32(b[1]), to_tf32(b[2]), to_tf32(b[3]));
      }
      loss += (double)tl;
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const unsigned char* D2 = dsel == OP_CHI ? D2s : D1s;
      for (int ks = 0; ks < TL / 8; ++ks) {
        const uint32_t within = (uint32_t)ks * 32u;
        const uint32_t acc = (tile > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(t_p, desc_sw128(smem_u32(As) + within), desc_sw128(smem_u32(D1s) + within), id_pq, acc);
        mma_tf32(t_q, desc_sw128(smem_u32(Bs) + within), desc_sw128(smem_u32(D2) + within), id_pq, acc);
      }
      mma_commit(&bar_pq);
    }
    if (!block_wait(&bar_pq, tile & 1, &s_abort, status)) break;
    fence_after_sync();
  }
  if (!s_abort && tile > 0) {
    // P (warps 0-3) or Q (warps 4-7) row frow -> partial slice s
    const int64_t gf = f0 + frow;
    float* part = P.rowPart + (int64_t)s * 2 * P.F * K + (half ? P.F * K : 0);
    const uint32_t tcol = half ? t_q : t_p;
    for (int c = 0; c < kp; c += 16) {
      float r[16];
      tmem_ld16(tcol + lane_off + c, r);
      tmem_ld_wait();
      if (gf < P.F) {
        #pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < K) part[gf * K + c + j] = r[j];
      }
    }
  }
  if (wantLoss) {
    const double t = block_sum(loss, red);
    if (tid == 0) lossPart[blockIdx.x] = t;
  }
  fence_before_sync();
  __syncthreads();
  if (s_abort) {
    // give MMAs still in flight a bounded chance to drain before freeing TMEM
    mbar_wait(&bar_pq, tile & 1, 100000000ull);
  }
  if (warp == 0) tmem_dealloc(tbase, ncols);
}

template <int BK>
__global__ void __launch_bounds__(TC_THREADS)
tc_col_sweep_kernel(Prob<float> P, int wsel, int hsel, int csel, int flags, BetaParams bp,
                    double* __restrict__ lossPart, int* __restrict__ status) {
  if (*status) return;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_v, bar_hd;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  __shared__ double red[32];
  const int K = P.K, kp = (K + 15) & ~15, na = natoms_of(kp);
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* HsT = base;
  unsigned char* Ws = HsT + na * TILE_BYTES;
  unsigned char* C1s = Ws + na * TL * 128;
  unsigned char* C2s = C1s + kp * 128;
  unsigned char* Vs = C2s + kp * 128;
  unsigned char* As = Vs + TILE_BYTES;
  unsigned char* Bs = As + TILE_BYTES;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = blockIdx.x / P.tcSplitR, r = blockIdx.x % P.tcSplitR;
  const int64_t n0 = (int64_t)nt * MT;
  const int64_t fBeg = (int64_t)r * P.tcChunkF;
  const int64_t fEnd = fBeg + P.tcChunkF < P.F ? fBeg + P.tcChunkF : P.F;
  const float* __restrict__ Wp = wsel == SEL_TILDE ? P.Wt : P.W;
  const float* __restrict__ Hp = hsel == SEL_TILDE ? P.Ht : P.H;
  const bool wantLoss = flags & SWEEP_LOSS;
  const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
  const uint32_t ncols = tmem_cols_of(kp);

  if (tid == 0) {
    s_abort = 0;
    mbar_init(&bar_v, 1);
    mbar_init(&bar_hd, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  // Hp columns [n0, n0+128) transposed -> HsT (A operand of MMA1)
  for (int i = tid; i < MT * kp; i += TC_THREADS) {
    const int k = i / MT, n = i - k * MT;
    const int64_t gn = n0 + n;
    const float h = (k < K && gn < P.N) ? Hp[(int64_t)k * P.N + gn] : 0.f;
    st_f32(HsT + (k >> 5) * TILE_BYTES, sw128_offset(n, 4 * (k & 31)), to_tf32(h));
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t t_v = tbase, t_n = tbase + 128, t_d = tbase + tmem_second_acc(kp);
  const uint32_t id_v = idesc(MT, TL, kFmtTF32), id_hd = idesc(MT, kp, kFmtTF32);
  const int q4 = warp & 3, half = warp >> 2;
  const int ncol = 32 * q4 + lane;          // this thread's TMEM lane = tile column n
  const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
  double loss = 0.0;
  int tile = 0;
  for (int64_t f0 = fBeg; f0 < fEnd; f0 += TL, ++tile) {
    // stage Wp rows (B operand of MMA1), C1/C2 transposed (B operands of MMA2/3) and V
    for (int i = tid; i < TL * kp; i += TC_THREADS) {
      const int f = i / kp, k = i - f * kp;
      const int64_t gf = f0 + f;
      const bool in = k < K && gf < fEnd;
      const float w = in ? Wp[gf * K + k] : 0.f;
      st_f32(Ws + (k >> 5) * (TL * 128), sw128_offset(f, 4 * (k & 31)), to_tf32(w));
      if (csel == OP_CHI) {
        st_f32(C1s, sw128_offset(k, 4 * f), to_tf32(in ? P.chiW1[gf * K + k] : 0.f));
        st_f32(C2s, sw128_offset(k, 4 * f), to_tf32(in ? P.chiW2[gf * K + k] : 0.f));
      } else {
        st_f32(C1s, sw128_offset(k, 4 * f), to_tf32(w));
      }
    }
    for (int i = tid; i < TL * MT; i += TC_THREADS) {
      const int f = i / MT, n = i - f * MT;
      const int64_t gf = f0 + f, gn = n0 + n;
      reinterpret_cast<float*>(Vs)[f * MT + n] = (gf < fEnd && gn < P.N) ? P.V[gf * P.ldv + gn] : 0.f;
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      for (int ks = 0; ks < kp / 8; ++ks) {
        const int k0 = ks * 8;
        const uint32_t within = (uint32_t)(k0 & 31) * 4u;
        const uint64_t ad = desc_sw128(smem_u32(HsT + (k0 >> 5) * TILE_BYTES) + within);
        const uint64_t bd = desc_sw128(smem_u32(Ws + (k0 >> 5) * (TL * 128)) + within);
        mma_tf32(t_v, ad, bd, id_v, ks > 0);
      }
      mma_commit(&bar_v);
    }
    if (!block_wait(&bar_v, tile & 1, &s_abort, status)) break;
    fence_after_sync();
    // Vp^T row n, columns f in [16 half, 16 half + 16) -> A^T, B^T
    {
      float vt[16];
      tmem_ld16(t_v + lane_off + 16 * half, vt);
      tmem_ld_wait();
      const int64_t gn = n0 + ncol;
      float tl = 0.f;
      #pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int fb = 16 * half + 4 * c;
        float a[4], b[4];
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int f = fb + j;
          const bool valid = gn < P.N && f0 + f < fEnd;
          a[j] = 0.f;
          b[j] = 0.f;
          if (valid) {
            const float v = reinterpret_cast<const float*>(Vs)[f * MT + ncol] + kappa;
            const float y = vt[4 * c + j] + kappa;
            ab_terms_g<BK>(v, y, bm2, a[j], b[j], bp.tiny);
            if (wantLoss) tl += (float)DB<float>::eval(v, y, bp, BK);
          }
        }
        const uint32_t off = sw128_offset(ncol, 4 * fb);
        *reinterpret_cast<float4*>(As + off) = make_float4(to_tf32(a[0]), to_tf32(a[1]), to_tf32(a[2]), to_tf32(a[3]));
        *reinterpret_cast<float4*>(Bs + off) = make_float4(to_tf32(b[0]), to_tf32(b[1]), to_tf32(b[2]), to_tf32(b[3]));
      }
      loss += (double)tl;
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const unsigned char* C2 = csel == OP_CHI ? C2s : C1s;
      for (int ks = 0; ks < TL / 8; ++ks) {
        const uint32_t within = (uint32_t)ks * 32u;
        const uint32_t acc = (tile > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(t_n, desc_sw128(smem_u32(As) + within), desc_sw128(smem_u32(C1s) + within), id_hd, acc);
        mma_tf32(t_d, desc_sw128(smem_u32(Bs) + within), desc_sw128(smem_u32(C2) + within), id_hd, acc);
      }
      mma_commit(&bar_hd);
    }
    if (!block_wait(&bar_hd, tile & 1, &s_abort, status)) break;
    fence_after_sync();
  }
  if (!s_abort && tile > 0) {
    // Hn^T (warps 0-3) or Hd^T (warps 4-7) row ncol -> partial slice r (K x N layout)
    const int64_t gn = n0 + ncol;
    const int64_t KN = (int64_t)K * P.N;
    float* part = P.colPart + (int64_t)r * 2 * KN + (half ? KN : 0);
    const uint32_t tcol = half ? t_d : t_n;
    for (int c = 0; c < kp; c += 16) {
      float rr[16];
      tmem_ld16(tcol + lane_off + c, rr);
      tmem_ld_wait();
      if (gn < P.N) {
        #pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < K) part[(int64_t)(c + j) * P.N + gn] = rr[j];
      }
    }
  }
  if (wantLoss) {
    const double t = block_sum(loss, red);
    if (tid == 0) lossPart[blockIdx.x] = t;
  }
  fence_before_sync();
  __syncthreads();
  if (s_abort) mbar_wait(&bar_hd, tile & 1, 100000000ull);
  if (warp == 0) tmem_dealloc(tbase, ncols);
}

template <typename Kern>
cudaError_t prep(Kern k, size_t sm) {
  return ensure_smem_attr(reinterpret_cast<const void*>(k), sm);
}

}  // namespace

int tc_kp(int K) { return (K + 15) & ~15; }

#define NMF_TC_BK_DISPATCH(KERN, GRID, SM, ...)                                                   \
  do {                                                                                            \
    cudaError_t e_ = cudaSuccess;                                                                 \
    switch (bp.kind) {                                                                            \
      case BK_IS: e_ = prep(KERN<BK_IS>, SM); if (e_ == cudaSuccess) KERN<BK_IS><<<GRID, TC_THREADS, SM, st>>>(__VA_ARGS__); break;          \
      case BK_KL: e_ = prep(KERN<BK_KL>, SM); if (e_ == cudaSuccess) KERN<BK_KL><<<GRID, TC_THREADS, SM, st>>>(__VA_ARGS__); break;          \
      case BK_EUC: e_ = prep(KERN<BK_EUC>, SM); if (e_ == cudaSuccess) KERN<BK_EUC><<<GRID, TC_THREADS, SM, st>>>(__VA_ARGS__); break;       \
      case BK_B15: e_ = prep(KERN<BK_B15>, SM); if (e_ == cudaSuccess) KERN<BK_B15><<<GRID, TC_THREADS, SM, st>>>(__VA_ARGS__); break;       \
      default: e_ = prep(KERN<BK_GENERAL>, SM); if (e_ == cudaSuccess) KERN<BK_GENERAL><<<GRID, TC_THREADS, SM, st>>>(__VA_ARGS__); break; \
    }                                                                                             \
    if (e_ != cudaSuccess) return e_;                                                             \
    return cudaGetLastError();                                                                    \
  } while (0)

cudaError_t launch_tc_row_sweep(const Prob<float>& P, const TcMaps* maps, int wsel, int hsel, int dsel, int flags,
                                bool bf16, const BetaParams& bp, double* lossPart, int* status, cudaStream_t st,
                                const SideJob* side) {
  (void)bf16;
  const int kp = tc_kp(P.K);
  if (kp > TC_KPMAX) return cudaErrorInvalidValue;
  if (kp <= 64 && maps && maps->ok) return launch_tc_ws_row(P, *maps, dsel, flags, bp, lossPart, status, st, side);
  if (P.tcClusterS != 1 || side) return cudaErrorNotSupported;   // clustered tilings need the warp-specialised kernel
  const size_t sm = row_smem(kp);
  const unsigned grid = (unsigned)(P.tcRowTiles * P.tcSplitS);
  NMF_TC_BK_DISPATCH(tc_row_sweep_kernel, grid, sm, P, wsel, hsel, dsel, flags, bp, lossPart, status);
}

cudaError_t launch_tc_col_sweep(const Prob<float>& P, const TcMaps* maps, int wsel, int hsel, int csel, int flags,
                                bool bf16, const BetaParams& bp, double* lossPart, int* status, cudaStream_t st,
                                const SideJob* side) {
  (void)bf16;
  const int kp = tc_kp(P.K);
  if (kp > TC_KPMAX) return cudaErrorInvalidValue;
  if (kp <= 64 && maps && maps->ok) return launch_tc_ws_col(P, *maps, csel, flags, bp, lossPart, status, st, side);
  if (P.tcClusterR != 1 || P.tcSK || side) return cudaErrorNotSupported;   // clustered / stream-K splits need the warp-specialised kernel
  const size_t sm = col_smem(kp);
  const unsigned grid = (unsigned)(P.tcColTiles * P.tcSplitR);
  NMF_TC_BK_DISPATCH(tc_col_sweep_kernel, grid, sm, P, wsel, hsel, csel, flags, bp, lossPart, status);
}

}  // namespace nmf
