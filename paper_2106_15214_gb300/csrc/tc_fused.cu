// tc_fused.cu -- one read of V per JMM iteration: the H-first update of
// eq. jnt_update (L = 1; the inverted order of Sec. 4.1.1) with the product
// Vt = Wt Ht formed once (Algorithm 2, step "Vt <- Wt Ht"; Sec. 3.4.2,
// Table 3), A = V . Vt^(beta-2) and B = Vt^(beta-1) evaluated once, and BOTH
// contractions taken from on-chip copies of A and B:
//
//   H = Ht . ((Wt^T A) / (Wt^T B))^gamma            (reduction over f)
//   W = Wt . ((A chi_1(H, Ht)^T) / (B chi_2(H, Ht)^T))^gamma  (reduction over n)
//
// Work split. A cluster of c blocks owns a run of 128-column batches of V;
// block r of the cluster owns rows [128 r, 128 r + 128) (the TMEM lanes of its
// tiles). c = ceil(F / 128), except when F = 128 c + 1 (a spectrogram's
// F = 2^m + 1 frequency bins): then the last block's warp 0 also takes the row
// past its 128 in FP32, so that one block per cluster less is needed (36
// clusters of 4 instead of 28 of 5 at F = 513). Per batch each block
//   1. forms Vt (128 x 128, tcgen05 kind::tf32, W~ rows in TMEM, H~^T rows in
//      shared memory) and, tile by tile (32 columns), reads V, evaluates A, B
//      and the objective in registers (FP32; FP64 below the small-Vt guard),
//      writes A and B as bf16 back into the Vt columns of TMEM (the A operand
//      of the W contraction) and, transposed, into a shared-memory copy (the A
//      operand of the H contraction, M = 128 columns n);
//   2. contracts that copy with W~ (bf16): its partial H numerator and
//      denominator over its 128 rows (TMEM, lanes = columns n);
//   3. exchanges those partials inside the cluster through distributed shared
//      memory: every block reduces 1/c of the batch's entries of H over the
//      c partials in a fixed order, forms them (written to global memory) and
//      chi_1, chi_2, and pushes those chi entries (bf16) into every block's
//      operand buffer;
//   4. contracts its TMEM copy of A and B with chi_1, chi_2 (kind::f16) into
//      its W numerator and denominator (TMEM, accumulated over the batches).
// At the end every block writes its [P | Q] rows as one partial slice (one per
// cluster); fused_w_kernel sums the slices in fixed order. The next
// batch's product and epilogue overlap the exchange: three TMEM batch buffers,
// two H~^T slots and two chi slots alternate.
//
// Roles (24 warps): 0 operand loads (W~ rows once, H~^T rows per batch) and
// the tail rows, 1 V tiles, 2 MMA issue, 4-19 epilogue (two groups of 8 warps
// on alternate tiles, each thread one TMEM lane and 16 columns of a tile),
// 20-23 and 3 the exchange (20-23 read one TMEM lane quarter each; all five
// reduce). Every wait is bounded (1 s, then
// NMF_ETIMEOUT and every role leaves its loop); the blocks of a cluster meet
// only in bounded mbarrier waits, plus one cluster barrier at entry and one at
// exit that every block reaches.
//
// Precision: the product in TF32 (10-bit mantissas, FP32 accumulation), A, B,
// W~ and chi rounded to bf16 (8-bit mantissas) for the two contractions (FP32
// accumulation), the powers in FP32, the objective accumulated in float-float
// then FP64. Limits: K <= 32 (kp <= 32), F <= 1024 (c <= 8).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "tc_ptx.cuh"

namespace nmf {
using namespace tc;

namespace {

constexpr int FU_THREADS = 768;
constexpr int FU_EPI0 = 4;           // first epilogue warp
constexpr int FU_EX0 = 20;           // first exchange warp
// exchange warps: 20-23 read the H accumulator (one TMEM lane quarter each)
// and reduce; with tail rows (clusters of F / 128 blocks, 25 % more tasks a
// block) warp 3 reduces too
constexpr int FU_TAIL_MAX = 1;       // rows past the last block's 128 handled in FP32 by warp 0 (F = 128 c + tail)
constexpr size_t FU_STATIC_RESERVE = 1024;   // the kernel's static shared memory (barriers)
// tail-row buffers: W~ rows [FU_TAIL_MAX][32], then A, B per slot [2][FU_TAIL_MAX][2][128] (floats)
constexpr uint32_t FU_TAIL_BYTES = 4u * (FU_TAIL_MAX * 32 + 2 * FU_TAIL_MAX * 2 * 128);
constexpr int FU_MAXV = 6;
constexpr int FU_ETIMEOUT = 5;
constexpr uint32_t FU_TB = 16384;    // one V tile (128 x 32 floats) or one H~^T batch (128 x 32)
constexpr size_t FU_SMEM_LIMIT = 227 * 1024;
// TMEM columns: three batch buffers (Vt of 4 tiles, then [A | B] bf16 in
// place), the H accumulator (Hn at +0, Hd at +32), P, Q.
constexpr int FU_NBUF = 3;
constexpr uint32_t FT_BUF = 0, FT_HACC = 384, FT_P = 448, FT_Q = 480, FT_COLS = 512;

struct FuLayout {
  uint32_t fa0;      // 2 H~^T batch slots (128 rows x 32 floats, SW128)
  uint32_t wt;       // W~ rows (MMA1's A operand, 128 rows x 32 floats, SW128)
  uint32_t v0;       // nv V tiles
  uint32_t sa, sb;   // A^T, B^T copies: 2 K-atoms (64 rows f each) x 128 rows n x 128 B (bf16, SW128)
  uint32_t wb;       // W~^T bf16: 2 K-atoms x kp rows x 128 B
  uint32_t chi0;     // 2 chi slots: chi_1 then chi_2, each 2 K-atoms (64 columns n) x kp rows x 128 B
  uint32_t chiSlot;
  uint32_t mb;       // mailbox: 2K rows (Hn then Hd) x 128 floats
  uint32_t tail;     // tail-row buffers (FU_TAIL_BYTES)
  uint32_t total;
  int nv;
};

__host__ __device__ inline FuLayout fu_layout(int K, int kp, int nv) {
  FuLayout L;
  L.fa0 = 0;
  L.wt = 2 * FU_TB;
  L.v0 = 3 * FU_TB;
  L.sa = L.v0 + (uint32_t)nv * FU_TB;
  L.sb = L.sa + 32768u;
  L.wb = L.sb + 32768u;
  L.chi0 = L.wb + 2u * (uint32_t)kp * 128u;
  L.chiSlot = 4u * (uint32_t)kp * 128u;
  L.mb = L.chi0 + 2u * L.chiSlot;
  L.tail = L.mb + 2u * (uint32_t)K * 512u;
  L.total = L.tail + FU_TAIL_BYTES;
  L.nv = nv;
  return L;
}

// Deepest V ring that fits (at least 2 tiles).
inline int fu_pick_nv(int K, int kp) {
  for (int nv = FU_MAXV; nv >= 2; --nv)
    if (1024 + fu_layout(K, kp, nv).total + FU_STATIC_RESERVE <= FU_SMEM_LIMIT) return nv;
  return 0;
}

struct FuBars {
  uint64_t vfull[FU_MAXV], vempty[FU_MAXV];
  uint64_t fafull[2], fafree[2], tfull[FU_NBUF], buffree[FU_NBUF], chiready[2];
  uint64_t haccfull, haccfree, stashfull, stashfree, once, done;
  // arrived on by every block of the cluster, alternating by batch parity: a
  // block can arrive for batch j + 1 before another block's arrival for batch
  // j has landed (that one reaches the barrier only through a third block),
  // but its arrival for j + 2 is causally after this block's own wait for j.
  uint64_t mailfull[2], chifull[2];
  // tail rows (last block): their A, B of batch j are in slot j & 1; warp 0
  // has read batch j's chi
  uint64_t tailfull[2], tailfree[2];
};

struct FuParams {
  int c;             // blocks per cluster (row tiles of 128)
  int ncl;           // clusters
  int nbatch;        // 128-column batches of V
  int nv;
  int layK, laykp;   // the rank the shared-memory layout is sized for (many problems: the largest)
  double* lossPart;  // one partial per block
  int* status;
  uint64_t limitNs;  // bound of every wait
  unsigned extra;    // arrivals the cluster barriers expect beyond the c blocks (0; 1 in the timeout test)
  int early;         // launched without programmatic dependent launch: the operand copies are complete at
                     // entry, so their first loads go out with the first V tiles
  int tail;          // F = 128 c + tail, 0 <= tail <= FU_TAIL_MAX: the last block's warp 0 takes the
                     // rows past its 128 (one problem only)
  float* gH;         // not null: the adjoint instead of the update: the exchange writes
                     // grad_H = W~^T (B - A) here and pushes chi_1 = chi_2 = H~, so the W
                     // contraction gives P = A H~^T, Q = B H~^T (grad_W = Q - P); H is not written
  // many problems in one launch: cluster i runs work item items[i] = {problem,
  // first batch, end batch, partial slice}, reads the problem's descriptor
  // from probs and its V, W~-row and H~^T tensor maps from maps[3 p ..], and
  // writes its blocks' objective partials from lossPart[lossBase[i]] on
  const int4* items;
  const Prob<float>* probs;
  const CUtensorMap* maps;
  const int* lossBase;
};

// Bounded local wait shared by every role (gives up when another role did).
__device__ __forceinline__ bool fu_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status,
                                        uint64_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (globaltimer_ns() - t0 > limit) {
      *abort = 1;
      atomicExch(status, FU_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// Bounded wait for arrivals of the cluster's blocks (acquire at cluster
// scope: their writes before arriving are visible afterwards).
__device__ __forceinline__ bool fu_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort, int* status,
                                                uint64_t limit) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort) return false;
    if (globaltimer_ns() - t0 > limit) {
      *abort = 1;
      atomicExch(status, FU_ETIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Byte offset of bf16 element e (0..63) of row r in a 128B-swizzled K-atom.
__device__ __forceinline__ uint32_t sw_bf16(uint32_t r, uint32_t e) { return sw128_offset(r, 2u * e); }

__device__ __forceinline__ void fu_init_bars(FuBars& B, int nv, int c, int nex, unsigned extra) {
  for (int s = 0; s < nv; ++s) {
    mbar_init(&B.vfull[s], 1u);
    mbar_init(&B.vempty[s], 8u);           // the 8 warps of the group reading the tile
  }
  for (int s = 0; s < FU_NBUF; ++s) {
    mbar_init(&B.tfull[s], 1u);
    mbar_init(&B.buffree[s], 1u);
  }
  mbar_init(&B.haccfull, 1u);
  mbar_init(&B.haccfree, 4u);              // the 4 exchange warps
  for (int s = 0; s < 2; ++s) {
    mbar_init(&B.fafull[s], 1u);
    mbar_init(&B.fafree[s], 1u);
    mbar_init(&B.chiready[s], (uint32_t)nex);
    mbar_init(&B.mailfull[s], 4u * (uint32_t)c + extra);    // every reading exchange warp of every block
    mbar_init(&B.chifull[s], (uint32_t)nex * (uint32_t)c + extra);   // every exchange warp of every block
    mbar_init(&B.tailfull[s], 1u);
    mbar_init(&B.tailfree[s], 1u);
  }
  mbar_init(&B.stashfull, 32u);            // 4 tiles x 8 warps per batch
  mbar_init(&B.stashfree, 1u);
  mbar_init(&B.once, 1u);
  mbar_init(&B.done, 1u);
  fence_mbar_init();
}

// ---- tail rows (F = 128 c + t, t <= FU_TAIL_MAX = 1): warp 0 of the last block --
//
// The rows past the block's 128 TMEM lanes, in FP32 between the warp's H~^T
// loads. Per batch j, once its H~^T rows are in their slot: the rows' product
// with H~ (the TF32 values MMA1 reads), A, B and objective terms, four
// columns per lane, into tail slot j & 1, from which the cluster's owners add
// the rows' terms to the H numerator and denominator of their tasks. Once chi of batch j is in: the rows'
// W numerators and denominators, lane k summing over the batch's columns in
// order, accumulated over the batches and written into the cluster's slice at
// the end. A load goes out as soon as its slot is free (MMA1 and these
// rows done with it); every wait polls the loads and is bounded. Not inlined:
// its registers stay out of the kernel's hot roles. Returns the loads issued.
struct FuTail {
  const float* V;
  int64_t ldv, N, F;
  float* rowPart;                 // this cluster's slice [P | Q]
  int K, kp, row0, tailE, b0, nbr, issued;
  unsigned char* fa;              // H~^T slots
  unsigned char* chi;             // chi slots
  uint32_t chiSlot;
  const CUtensorMap* tmH;
  FuBars* bars;
  const float* wtail;             // [FU_TAIL_MAX][32] W~ rows (zero past the tail and K)
  float* tab;                     // [2][FU_TAIL_MAX][2][128] A, B per slot
  volatile int* abort;
  int* status;
  uint64_t lim;
};

template <int BK>
__device__ __noinline__ int fu_tail_warp(const FuTail& A, const BetaParams& bp, float& lossHi, float& lossLo) {
  const int lane = threadIdx.x & 31;
  // the descriptor's fields once, in registers
  const int K = A.K, kp = A.kp, tailE = A.tailE, nbr = A.nbr, b0 = A.b0, row0 = A.row0;
  const int64_t N = A.N, ldv = A.ldv, F = A.F;
  const float* V = A.V;
  unsigned char* const faB = A.fa;
  const unsigned char* const chiB = A.chi;
  const uint32_t chiSlot = A.chiSlot;
  const float* const wtail = A.wtail;
  float* const tabB = A.tab;
  FuBars* const bars = A.bars;
  const CUtensorMap* const tmH = A.tmH;
  volatile int* const abort = A.abort;
  int* const status = A.status;
  const uint64_t lim = A.lim;
  float* const rowPart = A.rowPart;
  auto tab = [&](int s, int e, int ab) -> float* { return tabB + ((s * FU_TAIL_MAX + e) * 2 + ab) * 128; };
  float pt[FU_TAIL_MAX], qt[FU_TAIL_MAX];
  #pragma unroll
  for (int e = 0; e < FU_TAIL_MAX; ++e) pt[e] = qt[e] = 0.f;
  const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
  int issued = A.issued, tb = 0;       // tb: batches whose tail terms are out (their slots' reads done)
  auto pump = [&]() {
    while (issued < nbr && issued - 2 < tb &&
           (issued < 2 ||
            __all_sync(0xffffffffu, mbar_test(&bars->fafree[issued & 1], (uint32_t)((issued - 2) >> 1) & 1u)))) {
      const int s = issued & 1;
      if (elect_one()) {
        mbar_arrive_expect_tx(&bars->fafull[s], FU_TB);
        tma_load_2d(faB + s * FU_TB, tmH, 0, (int)(128 * (int64_t)(b0 + issued)), &bars->fafull[s]);
      }
      __syncwarp();
      ++issued;
    }
  };
  auto wait_pump = [&](uint64_t* bar, uint32_t par) -> bool {
    const uint64_t t0 = globaltimer_ns();
    while (!__all_sync(0xffffffffu, mbar_test(bar, par))) {
      pump();
      if (*abort) return false;
      if (globaltimer_ns() - t0 > lim) {
        if (lane == 0) {
          *abort = 1;
          atomicExch(status, FU_ETIMEOUT);
        }
        __syncwarp();
        return false;
      }
    }
    return true;
  };
  auto tail_ab = [&](int j) {
    const int s = j & 1;
    const int64_t nb0 = 128 * (int64_t)(b0 + j);
    const unsigned char* fa = faB + s * FU_TB;
    float v[FU_TAIL_MAX][4];                         // V of the rows, issued first (in flight with the product)
    #pragma unroll
    for (int e = 0; e < FU_TAIL_MAX; ++e)
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t n = nb0 + lane + 32 * u;
        v[e][u] = 1.f;
        if (e < tailE && n < N) v[e][u] = __ldg(&V[(int64_t)(row0 + e) * ldv + n]);
      }
    float y[FU_TAIL_MAX][4];
    #pragma unroll
    for (int e = 0; e < FU_TAIL_MAX; ++e)
      #pragma unroll
      for (int u = 0; u < 4; ++u) y[e][u] = 0.f;
    for (int k4 = 0; k4 < K; k4 += 4) {                // H~^T rows n, elements k4 .. k4 + 3 (zeros past K)
      float4 w[FU_TAIL_MAX];
      #pragma unroll
      for (int e = 0; e < FU_TAIL_MAX; ++e) w[e] = *reinterpret_cast<const float4*>(wtail + 32 * e + k4);
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 h = *reinterpret_cast<const float4*>(fa + sw128_offset((uint32_t)(lane + 32 * u), 4u * k4));
        #pragma unroll
        for (int e = 0; e < FU_TAIL_MAX; ++e) {
          y[e][u] = fmaf(w[e].x, h.x, y[e][u]);
          y[e][u] = fmaf(w[e].y, h.y, y[e][u]);
          y[e][u] = fmaf(w[e].z, h.z, y[e][u]);
          y[e][u] = fmaf(w[e].w, h.w, y[e][u]);
        }
      }
    }
    fence_smem_to_async();                             // the slot's reads before its next TMA load
    __syncwarp();
    tb = j + 1;
    pump();
    float tl = 0.f;
    #pragma unroll
    for (int e = 0; e < FU_TAIL_MAX; ++e)
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nl = lane + 32 * u;
        float a = 0.f, b = 0.f;
        if (e < tailE && nb0 + nl < N) epi_terms<BK>(v[e][u] + kappa, y[e][u] + kappa, bm2, bp, true, tl, a, b);
        tab(s, e, 0)[nl] = a;
        tab(s, e, 1)[nl] = b;
      }
    ff_add(lossHi, lossLo, tl);
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->tailfull[s]);
  };
  // the rows' W numerators and denominators over batch j: lane k takes chi
  // row k, eight columns (one 16-byte chunk) at a time, in column order
  auto tail_chi = [&](int j) {
    const int s = j & 1;
    const unsigned char* chi = chiB + s * chiSlot;
    if (lane < K) {
      const uint32_t k = (uint32_t)lane;
      for (int n0 = 0; n0 < 128; n0 += 8) {
        const uint32_t off = ((uint32_t)n0 >> 6) * (uint32_t)(kp * 128) + k * 128u +
                             (((((uint32_t)n0 & 63u) >> 3) ^ (k & 7u)) << 4);
        const uint4 c1 = *reinterpret_cast<const uint4*>(chi + off);
        const uint4 c2 = *reinterpret_cast<const uint4*>(chi + off + 2u * (uint32_t)kp * 128u);
        const uint32_t w1[4] = {c1.x, c1.y, c1.z, c1.w}, w2[4] = {c2.x, c2.y, c2.z, c2.w};
        #pragma unroll
        for (int e = 0; e < FU_TAIL_MAX; ++e) {
          if (e < tailE) {
            const float4 a0 = *reinterpret_cast<const float4*>(tab(s, e, 0) + n0);
            const float4 a1 = *reinterpret_cast<const float4*>(tab(s, e, 0) + n0 + 4);
            const float4 g0 = *reinterpret_cast<const float4*>(tab(s, e, 1) + n0);
            const float4 g1 = *reinterpret_cast<const float4*>(tab(s, e, 1) + n0 + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
            #pragma unroll
            for (int i = 0; i < 4; ++i) {
              const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&w1[i]);
              const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&w2[i]);
              const float2 x1 = __bfloat1622float2(h1), x2 = __bfloat1622float2(h2);
              pt[e] = fmaf(av[2 * i], x1.x, pt[e]);
              pt[e] = fmaf(av[2 * i + 1], x1.y, pt[e]);
              qt[e] = fmaf(bv[2 * i], x2.x, qt[e]);
              qt[e] = fmaf(bv[2 * i + 1], x2.y, qt[e]);
            }
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->tailfree[s]);
  };
  bool full = nbr > 0;
  pump();
  for (int j = 0; full && j < nbr; ++j) {
    // H~^T of batch j in its slot: its tail terms (tail slot j & 1 last held
    // batch j - 2, read out before chi of j - 2 came in)
    full = wait_pump(&bars->fafull[j & 1], (uint32_t)(j >> 1) & 1u);
    if (!full) break;
    tail_ab(j);
    if (j >= 1) {
      full = wait_pump(&bars->chiready[(j - 1) & 1], (uint32_t)((j - 1) >> 1) & 1u);
      if (full) tail_chi(j - 1);
    }
  }
  if (full) full = wait_pump(&bars->chiready[(nbr - 1) & 1], (uint32_t)((nbr - 1) >> 1) & 1u);
  if (full) tail_chi(nbr - 1);
  if (full && !*abort && lane < K) {                   // the tail rows of this cluster's slice
    #pragma unroll
    for (int e = 0; e < FU_TAIL_MAX; ++e)
      if (e < tailE) {
        rowPart[(int64_t)(row0 + e) * K + lane] = pt[e];
        rowPart[F * K + (int64_t)(row0 + e) * K + lane] = qt[e];
      }
  }
  return issued;
}

// One launch per iteration; grid = ncl clusters x c blocks. BATCH: the
// clusters run work items of many problems (FuParams::items).
template <int BK, bool BATCH, bool TAIL>
__global__ void __launch_bounds__(FU_THREADS, 1)
tc_fused_kernel(const __grid_constant__ CUtensorMap tmV0, const __grid_constant__ CUtensorMap tmW0,
                const __grid_constant__ CUtensorMap tmH0, Prob<float> P0, BetaParams bp, FuParams S) {
  pdl_trigger();
  extern __shared__ unsigned char smem_raw[];
  __shared__ FuBars bars;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  __shared__ int s_skip;
  __shared__ double red[32];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = S.c;
  const int r = (int)cluster_rank();                 // row tile of this block
  const int cl = (int)(blockIdx.x / (unsigned)c);
  int pi = 0, b0, b1, slice, lossIdx;
  if constexpr (BATCH) {
    const int4 it = S.items[cl];
    pi = it.x; b0 = it.y; b1 = it.z; slice = it.w;
    lossIdx = S.lossBase[cl] + r;
  } else {
    b0 = (int)((int64_t)cl * S.nbatch / S.ncl);
    b1 = (int)((int64_t)(cl + 1) * S.nbatch / S.ncl);
    slice = cl;
    lossIdx = (int)blockIdx.x;
  }
  const Prob<float>& P = BATCH ? S.probs[pi] : P0;
  const CUtensorMap* tmV = BATCH ? S.maps + 3 * pi : &tmV0;
  const CUtensorMap* tmW = BATCH ? S.maps + 3 * pi + 1 : &tmW0;
  const CUtensorMap* tmH = BATCH ? S.maps + 3 * pi + 2 : &tmH0;
  const int K = P.K, kp = (K + 15) & ~15;
  const int nb = b1 - b0;
  const int nv = S.nv;
  const FuLayout L = fu_layout(S.layK, S.laykp, nv);
  // tail rows: their W~ rows, and per batch slot their A and B over the batch's columns
  float* s_wtail = reinterpret_cast<float*>(base + L.tail);           // [FU_TAIL_MAX][32]
  const float* s_tab = s_wtail + FU_TAIL_MAX * 32;                    // [2][FU_TAIL_MAX][2][128]
  const int64_t m0 = (int64_t)r * 128;
  // TAIL (one problem, S.tail > 0): the last block's warp 0 takes rows
  // 128 c .. 128 c + tailE - 1, and warp 3 joins the exchange
  const int tailE = (TAIL && r == c - 1) ? S.tail : 0;
  constexpr int nex = TAIL ? 5 : 4;                         // exchange warps
  const uint64_t lim = S.limitNs;
  const int ntiles = 4 * nb;
  const int vPre = nv < ntiles ? nv : ntiles;

  // ---- prologue: TMEM, barriers, tensor maps, the first V tiles (V is never
  // written by the step's kernels), then the dependency wait
  if (warp == 2) tmem_alloc(&tslot, FT_COLS);
  if (tid == 0) {
    s_abort = 0;
    prefetch_tmap(tmV);
    prefetch_tmap(tmW);
    prefetch_tmap(tmH);
    fu_init_bars(bars, nv, c, nex, S.extra);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1 && elect_one()) {
    for (int t = 0; t < vPre; ++t) {
      mbar_arrive_expect_tx(&bars.vfull[t], FU_TB);
      tma_load_2d(base + L.v0 + t * FU_TB, tmV, (int)(128 * (int64_t)b0 + 32 * t), (int)m0, &bars.vfull[t]);
    }
  }
  const int faPre = (S.early && nb > 0) ? (nb < 2 ? nb : 2) : 0;   // H~^T batches loaded before the wait
  if (warp == 0 && faPre > 0 && elect_one()) {
    mbar_arrive_expect_tx(&bars.once, FU_TB);
    tma_load_2d(base + L.wt, tmW, 0, (int)m0, &bars.once);           // W~ rows (TF32 copy)
    for (int j = 0; j < faPre; ++j) {
      mbar_arrive_expect_tx(&bars.fafull[j], FU_TB);
      tma_load_2d(base + L.fa0 + j * FU_TB, tmH, 0, (int)(128 * (int64_t)(b0 + j)), &bars.fafull[j]);
    }
  }
  __syncwarp();
  pdl_wait();
  // W~^T (bf16, the B operand of the H contraction) from the full-precision
  // W~ (= W at entry: every path leaves Wt equal to W before this launch, and
  // the W half after a single-problem sweep takes its base from W); chi slots
  // zeroed (their padded rows k >= K stay zero)
  for (int i = tid; i < 128 * kp; i += FU_THREADS) {
    const int k = i / 128, f = i - k * 128;
    const float w = (k < K && m0 + f < P.F) ? P.W[(m0 + f) * K + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    *reinterpret_cast<__nv_bfloat16*>(base + L.wb + (f >> 6) * (kp * 128) + sw_bf16(k, f & 63)) = h;
  }
  for (uint32_t o = tid * 16u; o < 2u * L.chiSlot; o += FU_THREADS * 16u)
    *reinterpret_cast<uint4*>(base + L.chi0 + o) = make_uint4(0u, 0u, 0u, 0u);
  if (TAIL && tid < FU_TAIL_MAX * 32) {              // (every block: the owners add the tail rows' terms)
    const int e = tid >> 5, k = tid & 31;
    s_wtail[tid] = (e < S.tail && k < K) ? P.W[(int64_t)(128 * c + e) * K + k] : 0.f;
  }
  fence_smem_to_async();
  // every block of the cluster has its barriers and buffers ready before any
  // block arrives on them or writes into them; block 0 of the cluster decides
  // for all whether the status word stops this launch
  cluster_sync();
  if (r == 0 && tid == 0) {
    const int sk = *S.status != 0;
    for (int q = 0; q < c; ++q) {
      const uint32_t a = dsmem_map((const void*)&s_skip, (uint32_t)q);
      asm volatile("st.shared::cluster.b32 [%0], %1;" :: "r"(a), "r"(sk) : "memory");
    }
  }
  cluster_sync();
  const bool skip = s_skip != 0;
  const int nbr = skip ? 0 : nb;                      // batches this launch runs
  const uint32_t tbase = tslot;
  float lossHi = 0.f, lossLo = 0.f;

  if (warp == 0) {
    // ---------------- operand loads ----------------
    if (faPre == 0 && nbr > 0 && elect_one()) {
      mbar_arrive_expect_tx(&bars.once, FU_TB);
      tma_load_2d(base + L.wt, tmW, 0, (int)m0, &bars.once);           // W~ rows (TF32 copy)
    }
    __syncwarp();
    if (nbr == 0 && faPre > 0) {                       // issued before the skip decision: wait for them
      mbar_wait(&bars.once, 0u, 100000000ull);
      for (int j = 0; j < faPre; ++j) mbar_wait(&bars.fafull[j], 0u, 100000000ull);
    }
    int issued = faPre < nbr ? faPre : nbr;
    auto issue = [&](int j) {
      const int s = j & 1;
      if (elect_one()) {
        mbar_arrive_expect_tx(&bars.fafull[s], FU_TB);
        tma_load_2d(base + L.fa0 + s * FU_TB, tmH, 0, (int)(128 * (int64_t)(b0 + j)), &bars.fafull[s]);
      }
      __syncwarp();
    };
    if (!TAIL || tailE == 0) {
      for (int j = issued; j < nbr; ++j, ++issued) {
        if (j >= 2 && !__all_sync(0xffffffffu, fu_wait(&bars.fafree[j & 1], (uint32_t)((j - 2) >> 1) & 1u, &s_abort,
                                                         S.status, lim)))
          break;
        issue(j);
      }
    } else {
      FuTail A;
      A.V = P.V;
      A.ldv = P.ldv;
      A.N = P.N;
      A.F = P.F;
      A.rowPart = P.rowPart + (int64_t)slice * 2 * P.F * K;
      A.K = K;
      A.kp = kp;
      A.row0 = 128 * c;
      A.tailE = tailE;
      A.b0 = b0;
      A.nbr = nbr;
      A.issued = issued;
      A.fa = base + L.fa0;
      A.chi = base + L.chi0;
      A.chiSlot = L.chiSlot;
      A.tmH = tmH;
      A.bars = &bars;
      A.wtail = s_wtail;
      A.tab = s_wtail + FU_TAIL_MAX * 32;
      A.abort = &s_abort;
      A.status = S.status;
      A.lim = lim;
      issued = fu_tail_warp<BK>(A, bp, lossHi, lossLo);
    }
    // after a timeout no copy may land once the block has ended: wait (bounded)
    // for the last loads of each slot (their consumers may have given up)
    if (s_abort && nbr > 0) {
      mbar_wait(&bars.once, 0u, 100000000ull);
      for (int j = issued > 2 ? issued - 2 : 0; j < issued; ++j)
        mbar_wait(&bars.fafull[j & 1], (uint32_t)(j >> 1) & 1u, 100000000ull);
    }
  } else if (warp == 1) {
    // ---------------- V tiles ----------------
    const int nt = 4 * nbr;
    for (int t = nt; t < vPre; ++t)                    // issued before the skip decision: wait for them
      if (!__all_sync(0xffffffffu, mbar_wait(&bars.vfull[t], 0u, 100000000ull))) break;
    int issued = nt < vPre ? nt : vPre;               // the first tiles went out before the dependency wait
    for (int t = vPre; t < nt; ++t, ++issued) {
      const int sv = t % nv;
      if (!__all_sync(0xffffffffu, fu_wait(&bars.vempty[sv], (uint32_t)((t / nv) - 1) & 1u, &s_abort, S.status, lim)))
        break;
      if (elect_one()) {
        mbar_arrive_expect_tx(&bars.vfull[sv], FU_TB);
        tma_load_2d(base + L.v0 + sv * FU_TB, tmV, (int)(128 * (int64_t)b0 + 32 * t), (int)m0, &bars.vfull[sv]);
      }
      __syncwarp();
    }
    if (s_abort)                                       // as above: the last tile of every slot
      for (int t = issued > nv ? issued - nv : 0; t < issued; ++t)
        mbar_wait(&bars.vfull[t % nv], (uint32_t)(t / nv) & 1u, 100000000ull);
  } else if (warp == 2) {
    // ---------------- MMA issue ----------------
    // MMA1(j): Vt of batch j (W~ rows and the H~^T slot j & 1, both in shared
    // memory) into buffer j % 3. H-MMA(j): the A^T, B^T copies times W~ into
    // the H accumulator. W-MMA(j): [A | B] of buffer j % 3 times chi slot
    // j & 1 into P, Q. Order: MMA1(0..2), then per j: H-MMA(j) (as soon as
    // the epilogue has finished batch j, so that the exchange of batch j
    // starts at once), W-MMA(j - 1), MMA1(j + 2) (its buffer is the one
    // W-MMA(j - 1) read); finally W-MMA(last). The exchange of batch j thus
    // has the epilogue of batches j + 1 and j + 2 to complete in: the three
    // buffers take it off the per-batch critical path.
    const uint32_t id1 = idesc(128, 128, kFmtTF32), idk = idesc(128, kp, kFmtBF16);
    const uint64_t dFa = desc_sw128(smem_u32(base + L.fa0)), dWt = desc_sw128(smem_u32(base + L.wt));
    const uint64_t dSA = desc_sw128(smem_u32(base + L.sa)), dSB = desc_sw128(smem_u32(base + L.sb));
    const uint64_t dWb = desc_sw128(smem_u32(base + L.wb)), dChi = desc_sw128(smem_u32(base + L.chi0));
    const uint32_t atomK16 = (uint32_t)(kp * 128) >> 4;   // one K-atom of kp rows, in 16-byte units
    bool ok = nbr > 0 && __all_sync(0xffffffffu, fu_wait(&bars.once, 0u, &s_abort, S.status, lim));
    auto mma1 = [&](int j) -> bool {
      const int s = j & 1, b = j % FU_NBUF;
      if (!__all_sync(0xffffffffu, fu_wait(&bars.fafull[s], (uint32_t)(j >> 1) & 1u, &s_abort, S.status, lim)))
        return false;
      if (j >= FU_NBUF && !__all_sync(0xffffffffu, fu_wait(&bars.buffree[b], (uint32_t)(j / FU_NBUF - 1) & 1u,
                                                             &s_abort, S.status, lim)))
        return false;
      fence_after_sync();
      if (elect_one()) {
        for (int ks = 0; ks < kp / 8; ++ks)
          mma_tf32(tbase + FT_BUF + 128u * b, dWt + 2u * ks, dFa + (uint64_t)(s * (FU_TB >> 4)) + 2u * ks, id1, ks > 0);
        mma_commit(&bars.tfull[b]);
        mma_commit(&bars.fafree[s]);
      }
      __syncwarp();
      return true;
    };
    auto hmma = [&](int j) -> bool {
      if (!__all_sync(0xffffffffu, fu_wait(&bars.stashfull, (uint32_t)j & 1u, &s_abort, S.status, lim))) return false;
      // the exchange has read batch j - 1 out of the accumulator
      if (j >= 1 && !__all_sync(0xffffffffu, fu_wait(&bars.haccfree, (uint32_t)(j - 1) & 1u, &s_abort, S.status, lim)))
        return false;
      fence_after_sync();
      if (elect_one()) {
        const uint32_t acc = tbase + FT_HACC;
        for (int st = 0; st < 8; ++st) {               // K = 128 rows f in steps of 16
          const uint64_t ka = 1024u * (st >> 2) + 2u * (st & 3);
          const uint64_t kb = (uint64_t)atomK16 * (st >> 2) + 2u * (st & 3);
          mma_bf16(acc, dSA + ka, dWb + kb, idk, st > 0);
          mma_bf16(acc + 32u, dSB + ka, dWb + kb, idk, st > 0);
        }
        mma_commit(&bars.stashfree);
        mma_commit(&bars.haccfull);
      }
      __syncwarp();
      return true;
    };
    auto wmma = [&](int j) -> bool {
      const int s = j & 1, b = j % FU_NBUF;
      if (!__all_sync(0xffffffffu, fu_wait(&bars.chiready[s], (uint32_t)(j >> 1) & 1u, &s_abort, S.status, lim)))
        return false;
      fence_after_sync();
      if (elect_one()) {
        const uint32_t buf = tbase + FT_BUF + 128u * b;
        const uint64_t c1 = dChi + (uint64_t)(s * (L.chiSlot >> 4)), c2 = c1 + 2u * atomK16;
        for (int st = 0; st < 8; ++st) {               // K = 128 columns n in steps of 16
          const uint32_t a = buf + 32u * (st >> 1) + 16u * (st & 1);
          const uint64_t kb = (uint64_t)atomK16 * (st >> 2) + 2u * (st & 3);
          const uint32_t acc = (j > 0 || st > 0) ? 1u : 0u;
          mma_bf16_ts(tbase + FT_P, a, c1 + kb, idk, acc);
          mma_bf16_ts(tbase + FT_Q, a + 8u, c2 + kb, idk, acc);
        }
        mma_commit(&bars.buffree[b]);
      }
      __syncwarp();
      return true;
    };
    for (int j = 0; ok && j < nbr && j < FU_NBUF; ++j) ok = mma1(j);
    for (int j = 0; ok && j < nbr; ++j) {
      ok = hmma(j);
      if (ok && j >= 1) ok = wmma(j - 1);
      if (ok && j >= 1 && j + FU_NBUF - 1 < nbr) ok = mma1(j + FU_NBUF - 1);
    }
    if (ok && nbr > 0) wmma(nbr - 1);
    if (elect_one()) mma_commit(&bars.done);
    __syncwarp();
  } else if (warp >= FU_EPI0 && warp < FU_EX0) {
    // ---------------- epilogue ----------------
    // Group g (0, 1) takes tiles g, g + 2 of every batch; warp (q4, half) owns
    // TMEM lanes 32 q4 .. + 31 (rows f) and columns 16 half .. + 15 of a tile.
    const int ew = warp - FU_EPI0, q4 = warp & 3, g = (ew >> 2) & 1, half = ew >> 3;
    const int mrow = 32 * q4 + lane;
    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
    const bool mvalid = m0 + mrow < P.F;
    const int jb0 = 16 * half;
    const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
    // this thread's place in the transposed copies: K-atom mrow / 64, element mrow % 64 (pairs: even element)
    const uint32_t atomOff = (uint32_t)(mrow >> 6) * 16384u, ePair = (uint32_t)(mrow & 62);
    const bool odd = lane & 1;
    for (int t = g; t < 4 * nbr; t += 2) {
      const int j = t >> 2, q = t & 3, b = j % FU_NBUF;
      const int sv = t % nv;
      const uint32_t col = FT_BUF + 128u * b + 32u * q + jb0;
      // A group starts a new batch only once the previous batch's H contraction
      // has completed. It then also may overwrite the transposed copies; and on
      // GB300 a first tile whose TMEM reads and writes overlapped that
      // contraction (and the other group's last tile of the previous batch)
      // came out wrong in some runs, which this ordering removes.
      if (q == g && j >= 1 &&
          !__all_sync(0xffffffffu, fu_wait(&bars.stashfree, (uint32_t)(j - 1) & 1u, &s_abort, S.status, lim)))
        break;
      if (!__all_sync(0xffffffffu, fu_wait(&bars.tfull[b], (uint32_t)(j / FU_NBUF) & 1u, &s_abort, S.status, lim)))
        break;
      if (!__all_sync(0xffffffffu, fu_wait(&bars.vfull[sv], (uint32_t)(t / nv) & 1u, &s_abort, S.status, lim))) break;
      fence_after_sync();
      float vt[16], vv[16];
      tmem_ld16(tbase + col + lane_off, vt);
      const unsigned char* vb = base + L.v0 + sv * FU_TB;
      #pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v4 = *reinterpret_cast<const float4*>(vb + sw128_offset(mrow, 4 * jb0 + 16 * i));
        vv[4 * i] = v4.x; vv[4 * i + 1] = v4.y; vv[4 * i + 2] = v4.z; vv[4 * i + 3] = v4.w;
      }
      tmem_ld_wait();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.vempty[sv]);
      const int64_t n1 = 128 * (int64_t)(b0 + j) + 32 * q + jb0;   // first column of this thread's 16
      const int nvalid = (int)(P.N - n1 < 16 ? (P.N - n1 > 0 ? P.N - n1 : 0) : 16);
      float tl = 0.f;
      if (mvalid && nvalid == 16) {
        #pragma unroll
        for (int i = 0; i < 16; ++i) epi_terms<BK>(vv[i] + kappa, vt[i] + kappa, bm2, bp, true, tl, vv[i], vt[i]);
      } else {
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float v = vv[i] + kappa, y = vt[i] + kappa;
          vv[i] = 0.f;
          vt[i] = 0.f;
          if (mvalid && i < nvalid) epi_terms<BK>(v, y, bm2, bp, true, tl, vv[i], vt[i]);
        }
      }
      // A (vv) and B (vt) as bf16 pairs over this thread's Vt columns: [A | B]
      float cells[16];
      #pragma unroll
      for (int p = 0; p < 8; ++p) {
        cells[p] = __uint_as_float(pack_bf16(vv[2 * p], vv[2 * p + 1]));
        cells[8 + p] = __uint_as_float(pack_bf16(vt[2 * p], vt[2 * p + 1]));
      }
      tmem_st16(tbase + col + lane_off, cells);
      // neighbouring lanes (rows f, f + 1) exchange values so that each writes
      // one 32-bit pair: even lanes row n = .. + i, odd lanes row n = .. + i + 1
      #pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const float ra = __shfl_xor_sync(0xffffffffu, odd ? vv[i] : vv[i + 1], 1);
        const float rb = __shfl_xor_sync(0xffffffffu, odd ? vt[i] : vt[i + 1], 1);
        const uint32_t n = (uint32_t)(32 * q + jb0 + i + (odd ? 1 : 0));
        const uint32_t off = atomOff + sw_bf16(n, ePair);       // (sw_bf16 includes the row offset n * 128)
        *reinterpret_cast<uint32_t*>(base + L.sa + off) = odd ? pack_bf16(ra, vv[i + 1]) : pack_bf16(vv[i], ra);
        *reinterpret_cast<uint32_t*>(base + L.sb + off) = odd ? pack_bf16(rb, vt[i + 1]) : pack_bf16(vt[i], rb);
      }
      ff_add(lossHi, lossLo, tl);
      tmem_st_wait();
      fence_before_sync();
      fence_smem_to_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.stashfull);
    }
  } else if (warp >= FU_EX0 || (TAIL && warp == 3)) {
    // ---------------- cluster exchange ----------------
    // Thread x < 128 (the first four warps) owns TMEM lane x = column x of
    // the batch for the mailbox write. The batch's K x 32 tasks (row k, four
    // columns 4u .. 4u + 3; task t = 32 k + u) are split evenly over the
    // cluster's blocks: block r reduces tasks [32 K r / c, 32 K (r + 1) / c),
    // over all five warps (one task per thread up to 160 a block). Each warp
    // publishes what it wrote itself (warp barrier, one fence at cluster
    // scope, relaxed arrivals; the mailbox barriers count the 4 c reading
    // warps, the chi barriers the 5 c warps), so the warps never wait for one
    // another.
    const int x = (TAIL && warp == 3) ? 128 + lane : tid - FU_EX0 * 32;   // 0 .. 32 nex - 1
    const bool rd = !TAIL || warp != 3;               // reads TMEM lanes 32 (warp & 3) .. + 31 into the mailbox
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int tLo = 32 * K * r / c, ntask = 32 * K * (r + 1) / c - tLo;
    const uint32_t mbS = smem_u32(base + L.mb);
    const float gam = (float)bp.gamma, flo = (float)bp.floor, beta = (float)bp.beta;
    float* mb = reinterpret_cast<float*>(base + L.mb);
    for (int j = 0; j < nbr; ++j) {
      const int s = j & 1;
      // The mailbox is rewritten only after this block has received every
      // owner's chi of the previous batch (which the owners sent after
      // reading it), and chi slot s of every block is free once the mailbox
      // handshake of batch j completes: each block writes its mailbox after
      // its H contraction of batch j, whose completion covers its W
      // contraction of batch j - 2. So two handshakes per batch suffice.
      bool go = true;
      if (rd) {
        go = __all_sync(0xffffffffu, fu_wait(&bars.haccfull, (uint32_t)j & 1u, &s_abort, S.status, lim));
        if (TAIL && go && tailE > 0)                  // the tail rows' A, B of this batch, read by the owners
          go = __all_sync(0xffffffffu, fu_wait(&bars.tailfull[s], (uint32_t)(j >> 1) & 1u, &s_abort, S.status, lim));
      }
      if (rd && go) {
        fence_after_sync();
        for (int k0 = 0; k0 < kp; k0 += 16) {
          float hn[16], hd[16];
          tmem_ld16(tbase + FT_HACC + lane_off + k0, hn);
          tmem_ld16(tbase + FT_HACC + 32u + lane_off + k0, hd);
          tmem_ld_wait();
          #pragma unroll
          for (int i = 0; i < 16; ++i)
            if (k0 + i < K) {
              mb[(k0 + i) * 128 + x] = hn[i];
              mb[(K + k0 + i) * 128 + x] = hd[i];
            }
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.haccfree);
        // chi slot s is rewritten once every block's mailbox of this batch is
        // out: warp 0 must have read chi of batch j - 2 from it first
        if (TAIL && tailE > 0 && j >= 2)
          go = __all_sync(0xffffffffu, fu_wait(&bars.tailfree[s], (uint32_t)((j - 2) >> 1) & 1u, &s_abort, S.status,
                                               lim));
        // each warp publishes its own columns: warp barrier (cumulative), one
        // fence at cluster scope, relaxed arrivals
        __syncwarp();
        if (go && lane == 0 && !s_abort) {
          fence_acq_rel_cluster();
          for (int q = 0; q < c; ++q) mbar_arrive_remote_relaxed(dsmem_map(&bars.mailfull[s], (uint32_t)q));
        }
      }
      const int64_t nb0 = 128 * (int64_t)(b0 + j);
      // this thread's H~ values (one task, four columns; they do not depend
      // on the exchange) load while the other blocks' partials arrive
      float htp[4];
      {
        const int task = x, k = (tLo + task) >> 5, n4 = 4 * ((tLo + task) & 31);
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t n = nb0 + n4 + i;
          htp[i] = (task < ntask && n < P.N) ? __ldg(&P.Ht[(int64_t)k * P.N + n]) : 1.f;
        }
      }
      float hkeep[4] = {0.f, 0.f, 0.f, 0.f};
      go = !s_abort && __all_sync(0xffffffffu, fu_wait_cluster(&bars.mailfull[s], (uint32_t)(j >> 1) & 1u, &s_abort,
                                                               S.status, lim));
      // tasks of (row k, 4 columns): the four columns' numerators and
      // denominators of up to four ranks in flight together, summed in rank order
      for (int task = x; go && task < ntask; task += 32 * nex) {
        const int k = (tLo + task) >> 5, n4 = 4 * ((tLo + task) & 31);
        const uint32_t on = mbS + (uint32_t)(k * 512 + 4 * n4), od = mbS + (uint32_t)((K + k) * 512 + 4 * n4);
        float ht[4];
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t n = nb0 + n4 + i;
          ht[i] = task == x ? htp[i] : (n < P.N ? __ldg(&P.Ht[(int64_t)k * P.N + n]) : 1.f);
        }
        float hn[4] = {0.f, 0.f, 0.f, 0.f}, hd[4] = {0.f, 0.f, 0.f, 0.f};
        float4 tA = make_float4(0.f, 0.f, 0.f, 0.f), tB = tA;
        if (TAIL) {                                   // the tail rows' A, B at these columns (last block's slot s)
          const uint32_t ta = smem_u32(s_tab + (s * FU_TAIL_MAX * 2 + 0) * 128 + n4);
          tA = dsmem_ld4(dsmem_map_addr(ta, (uint32_t)(c - 1)));
          tB = dsmem_ld4(dsmem_map_addr(ta + 512u, (uint32_t)(c - 1)));
        }
        for (int q0 = 0; q0 < c; q0 += 4) {
          float4 pn[4], pd[4];
          #pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u < c) {
              pn[u] = dsmem_ld4(dsmem_map_addr(on, (uint32_t)(q0 + u)));
              pd[u] = dsmem_ld4(dsmem_map_addr(od, (uint32_t)(q0 + u)));
            }
          #pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u < c) {
              hn[0] += pn[u].x; hn[1] += pn[u].y; hn[2] += pn[u].z; hn[3] += pn[u].w;
              hd[0] += pd[u].x; hd[1] += pd[u].y; hd[2] += pd[u].z; hd[3] += pd[u].w;
            }
        }
        if (TAIL) {                                   // + W~[f, k] A[f, n], W~[f, k] B[f, n] of the tail row
          const float w = s_wtail[k];
          hn[0] = fmaf(w, tA.x, hn[0]); hn[1] = fmaf(w, tA.y, hn[1]); hn[2] = fmaf(w, tA.z, hn[2]); hn[3] = fmaf(w, tA.w, hn[3]);
          hd[0] = fmaf(w, tB.x, hd[0]); hd[1] = fmaf(w, tB.y, hd[1]); hd[2] = fmaf(w, tB.z, hd[2]); hd[3] = fmaf(w, tB.w, hd[3]);
        }
        float c1[4], c2[4];
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t n = nb0 + n4 + i;
          c1[i] = c2[i] = 0.f;
          if (n < P.N && S.gH) {                    // the adjoint (Sec. 4.1.5's gradient)
            S.gH[(int64_t)k * P.N + n] = hd[i] - hn[i];
            c1[i] = c2[i] = ht[i];
          } else if (n < P.N) {
            const float h = apply_floor(ht[i] * mu_ratio<BK, float>(hn[i], hd[i], gam), flo);
            if (!isfinite(h)) atomicExch(S.status, 4);
            if (task == x) hkeep[i] = h;            // this thread's first task: stored after the handshake
            else P.H[(int64_t)k * P.N + n] = h;
            chi_terms<BK, float>(h, ht[i], beta, c1[i], c2[i]);
          }
        }
        // chi rows k, columns n4 .. n4 + 3: 8 bytes of a 16-byte chunk of K-atom n4 / 64
        const uint32_t off = L.chi0 + s * L.chiSlot + (uint32_t)(n4 >> 6) * (kp * 128u) + (uint32_t)k * 128u +
                             ((((uint32_t)(n4 & 63) >> 3) ^ ((uint32_t)k & 7u)) << 4) + (uint32_t)(n4 & 4) * 2u;
        const uint32_t dst = smem_u32(base + off);
        const uint32_t a1 = pack_bf16(c1[0], c1[1]), b1 = pack_bf16(c1[2], c1[3]);
        const uint32_t a2 = pack_bf16(c2[0], c2[1]), b2 = pack_bf16(c2[2], c2[3]);
        for (int q = 0; q < c; ++q) {
          dsmem_st2u(dsmem_map_addr(dst, (uint32_t)q), a1, b1);
          dsmem_st2u(dsmem_map_addr(dst + 2u * kp * 128u, (uint32_t)q), a2, b2);
        }
      }
      fence_smem_cluster_to_async();
      __syncwarp();
      if (lane == 0 && !s_abort) {
        fence_acq_rel_cluster();
        for (int q = 0; q < c; ++q) mbar_arrive_remote_relaxed(dsmem_map(&bars.chifull[s], (uint32_t)q));
      }
      {                                             // H of this thread's first task, now off the fence's path
        const int task = x, k = (tLo + task) >> 5, n4 = 4 * ((tLo + task) & 31);
        if (go && task < ntask && !S.gH)
          #pragma unroll
          for (int i = 0; i < 4; ++i)
            if (nb0 + n4 + i < P.N) P.H[(int64_t)k * P.N + nb0 + n4 + i] = hkeep[i];
      }
      go = !s_abort &&
           __all_sync(0xffffffffu, fu_wait_cluster(&bars.chifull[s], (uint32_t)(j >> 1) & 1u, &s_abort, S.status, lim));
      fence_smem_to_async();
      __syncwarp();
      if (lane == 0 && go && !s_abort) mbar_arrive(&bars.chiready[s]);   // one arrival per exchange warp
    }
    // (no block touches this block's shared memory after the last chi
    // handshake: the owners read its mailbox before pushing their chi)
  }

  // ---------------- P, Q: one partial slice per cluster ----------------
  // Epilogue thread (mrow, grp) owns kp / 2 columns of P (grp 0, 1) or Q
  // (grp 2, 3) in TMEM lane mrow; the rows go out through shared memory (the
  // A^T, B^T copies are idle once every MMA is done) as two contiguous runs.
  const bool epi = warp >= FU_EPI0 && warp < FU_EX0;
  const int grp = (warp - FU_EPI0) >> 2, mrow = 32 * (warp & 3) + lane;
  const int per = kp / 2;
  const bool isQ = grp >= 2;
  const int col0 = (grp & 1) * per;
  bool have = false;
  if (epi) {
    have = nbr > 0 && !s_abort && fu_wait(&bars.done, 0u, &s_abort, S.status, lim);
    have = __all_sync(0xffffffffu, have);
  }
  float acc[16];
  #pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  if (epi && have) {
    fence_after_sync();
    const uint32_t ta = tbase + (isQ ? FT_Q : FT_P) + ((uint32_t)(32 * (warp & 3)) << 16) + col0;
    tmem_ld8(ta, acc);
    if (per > 8) tmem_ld8(ta + 8, acc + 8);
    tmem_ld_wait();
  }
  const int Ks = K | 1;
  float* stg = reinterpret_cast<float*>(base + L.sa);
  __syncthreads();
  const bool write = __syncthreads_or(have ? 1 : 0) != 0;
  if (epi && have) {
    float* row = stg + (isQ ? 128 * Ks : 0) + mrow * Ks + col0;
    #pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < per && col0 + i < K) row[i] = acc[i];
  }
  __syncthreads();
  if (write) {
    const int nrows = (int)(P.F - m0 < 128 ? P.F - m0 : 128);
    float* outP = P.rowPart + (int64_t)slice * 2 * P.F * K + m0 * K;
    float* outQ = outP + P.F * K;
    for (int rr = warp; rr < nrows; rr += FU_THREADS / 32)
      for (int cc = lane; cc < K; cc += 32) {
        outP[rr * K + cc] = stg[rr * Ks + cc];
        outQ[rr * K + cc] = stg[128 * Ks + rr * Ks + cc];
      }
  }
  const double unitLoss = block_sum_ff(lossHi, lossLo, reinterpret_cast<float2*>(red));
  if (tid == 0) S.lossPart[lossIdx] = unitLoss;
  fence_before_sync();
  __syncthreads();
  if (s_abort) mbar_wait(&bars.done, 0u, 100000000ull);
  // no block leaves while another may still arrive on or read its barriers
  cluster_sync();
  if (warp == 2) tmem_dealloc(tbase, FT_COLS);
}

// W~ = W, H~ = H and their TF32 shadows (sWS: F x ks rows, sHT: N x ks rows)
// of every problem of a batched context: blocks [0, totW) take EW entries of
// some W (prefW), the others 32 columns of some H (prefHc), transposed through
// shared memory so that both the reads of H and the writes of sHT coalesce.
__global__ void __launch_bounds__(EW)
fused_batch_copies_kernel(const Prob<float>* __restrict__ probs, int count, const int* __restrict__ prefW, int totW,
                          const int* __restrict__ prefHc, const int* __restrict__ status) {
  if (*status) return;
  __shared__ float tile[32][33];
  int b = blockIdx.x;
  if (b < totW) {
    const int pi = find_problem(prefW, count, b);
    const Prob<float>& P = probs[pi];
    const int64_t idx = (int64_t)(b - prefW[pi]) * EW + threadIdx.x;
    if (idx < P.F * P.K) {
      const float w = P.W[idx];
      P.Wt[idx] = w;
      const int64_t f = idx / P.K, k = idx - f * P.K;
      P.sWS[f * P.ks + k] = tf32_round(w);
    }
    return;
  }
  b -= totW;
  const int pi = find_problem(prefHc, count, b);
  const Prob<float>& P = probs[pi];
  const int64_t n0 = (int64_t)(b - prefHc[pi]) * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < P.K; k += EW / 32)
    if (n0 + lane < P.N) {
      const float h = P.H[(int64_t)k * P.N + n0 + lane];
      P.Ht[(int64_t)k * P.N + n0 + lane] = h;
      tile[lane][k] = tf32_round(h);
    }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * P.K; i += EW) {
    const int nl = i / P.K, k = i - nl * P.K;
    if (n0 + nl < P.N) P.sHT[(n0 + nl) * P.ks + k] = tile[nl][k];
  }
}

// ---- the W half of the iteration and the normalisation ---------------------
//
// After the fused sweep the W update needs the sum of the clusters' partial
// slices of [P | Q] (2 x slices x F x K floats, resident in L2), and the
// normalisation of Sec. 4.1.2 needs the column norms of the whole new W before
// any entry of W or H can be scaled. Two launches, each spread over every SM:
//   fused_w_kernel     the slice sums and the W update of this block's share
//                      of the entries (the new W written in place: each entry
//                      is read as the base W~ and rewritten by one thread), and
//                      the block's per-column sums of squares;
//   fused_norm_kernel  launched early (programmatic dependent launch): it loads
//                      its columns of H (final since the fused sweep) before
//                      waiting for fused_w_kernel; then every block sums the
//                      column partials in the same fixed order (the same norms
//                      in every block), divides its share of W by them (with
//                      the TF32 row copy), scales its columns of H (H, Ht, the
//                      transposed TF32 copy), and block 0 sums the objective.
constexpr int POST_THREADS = 512;    // both kernels; two blocks per SM (one of each), <= 64 registers
constexpr int POST_CH = 256;         // columns of H per pass through shared memory
constexpr int POST_DEPTH = 4;        // slices per lane with loads in flight together
// fused_w_kernel: lane partials of P and Q (2 x POST_THREADS float4), the W~ quads, then the squares
constexpr size_t POSTW_SMEM = 3 * POST_THREADS * sizeof(float4);
// fused_norm_kernel: the H tile (POST_CH x (K + 1) floats, K <= 32), then its
// rows in the layout of the transposed TF32 copy (POST_CH x 32 floats)
constexpr size_t POSTN_SMEM = (size_t)POST_CH * 33 * sizeof(float) + (size_t)POST_CH * 32 * sizeof(float);

struct PostParams {
  int slices;               // partial slices of [P | Q] (the fused sweep's clusters)
  int norm;                 // normalise (Sec. 4.1.2)
  float* normPart;          // [K][gridDim of fused_w_kernel] sums of squares
  const double* lossPart;   // the fused sweep's objective partials
  int lossBlocks;
  double* lossOut;          // null: the objective is not wanted
  int* status;
};

// Four consecutive entries from e (the entries past FK read as zero).
__device__ __forceinline__ float4 post_ld4(const float* p, int e, int FK, bool vec) {
  if (vec) return *reinterpret_cast<const float4*>(p + e);
  float4 v;
  v.x = e < FK ? p[e] : 0.f;
  v.y = e + 1 < FK ? p[e + 1] : 0.f;
  v.z = e + 2 < FK ? p[e + 2] : 0.f;
  v.w = e + 3 < FK ? p[e + 3] : 0.f;
  return v;
}
__device__ __forceinline__ void add4(float4& a, const float4& b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}
__device__ __forceinline__ float get4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

template <int BK, bool VEC>
__global__ void __launch_bounds__(POST_THREADS, 2)
fused_w_kernel(Prob<float> P, BetaParams bp, PostParams Q) {
  extern __shared__ float4 post_sm[];
  float4* redN = post_sm;                                   // [G][nq] lane partials of P
  float4* redD = post_sm + POST_THREADS;                    // and of Q
  float4* base4 = post_sm + 2 * POST_THREADS;               // W~ of quad tid, then its squares
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = (int)blockIdx.x, nb = (int)gridDim.x;
  pdl_wait();
  pdl_trigger();         // after the wait: the next kernel reads H before its own wait
  const bool skip = *Q.status != 0;
  const int K = P.K;
  const int FK = (int)(P.F * K), NQ = (FK + 3) / 4;          // F K <= 32768: 32-bit entry indices
  const int qa = (int)((int64_t)NQ * b / nb), qb = (int)((int64_t)NQ * (b + 1) / nb);
  const int nq = qb - qa;                                    // this block's quads of entries (<= POST_THREADS)
  const int G = nq > 0 ? max(1, min(Q.slices, POST_THREADS / nq)) : 1;   // lanes per quad
  constexpr bool vec = VEC;            // F K a multiple of 4: 16-byte loads of whole quads
  if (tid < nq) {
    const int e0 = 4 * (qa + tid);
    if (vec) {
      cp_async16(&base4[tid], P.W + e0);
    } else {
      float* bs = reinterpret_cast<float*>(&base4[tid]);
      for (int i = 0; i < 4; ++i) cp_async4(bs + i, e0 + i < FK ? P.W + e0 + i : P.W, e0 + i < FK ? 4u : 0u);
    }
  }
  // P and Q of the block's entries: lane g of a quad sums slices g, g + G, ...
  // in order, then the G lanes in order
  if (tid < G * nq) {
    const int q = tid % nq, g = tid / nq;
    const int e0 = 4 * (qa + q);
    float4 n4 = make_float4(0.f, 0.f, 0.f, 0.f), d4 = n4;
    const int step = 2 * FK * G;                   // floats from one of this lane's slices to its next
    const float* part = P.rowPart + (int64_t)g * 2 * FK;
    for (int s0 = g; s0 < Q.slices; s0 += POST_DEPTH * G, part += POST_DEPTH * step) {
      float4 vn[POST_DEPTH], vd[POST_DEPTH];
      #pragma unroll
      for (int u = 0; u < POST_DEPTH; ++u) {
        const bool in = s0 + u * G < Q.slices;
        vn[u] = in ? post_ld4(part + u * step, e0, FK, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
        vd[u] = in ? post_ld4(part + u * step + FK, e0, FK, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      #pragma unroll
      for (int u = 0; u < POST_DEPTH; ++u) {
        add4(n4, vn[u]);
        add4(d4, vd[u]);
      }
    }
    redN[g * nq + q] = n4;
    redD[g * nq + q] = d4;
  }
  cp_async_wait_all();
  __syncthreads();
  // the W update of eq. jnt_update (W half, base W~), written in place
  float* sq = reinterpret_cast<float*>(base4);
  if (tid < nq) {
    const float4 base = base4[tid];
    float4 n4 = redN[tid], d4 = redD[tid];
    for (int g = 1; g < G; ++g) {
      add4(n4, redN[g * nq + tid]);
      add4(d4, redD[g * nq + tid]);
    }
    const int e0 = 4 * (qa + tid);
    float x[4];
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] = 0.f;
      if (e0 + i < FK) {
        x[i] = apply_floor(get4(base, i) * mu_ratio<BK, float>(get4(n4, i), get4(d4, i), (float)bp.gamma),
                           (float)bp.floor);
        if (!skip) {
          if (!isfinite(x[i])) atomicExch(Q.status, 4);
          P.W[e0 + i] = x[i];
        }
      }
    }
    #pragma unroll
    for (int i = 0; i < 4; ++i) sq[4 * tid + i] = x[i] * x[i];   // (the thread's own W~ quad, read above)
  }
  __syncthreads();
  // per-column sums of squares over the block's entries: warp w takes columns
  // w, w + 16, ...; its lanes every 32nd entry of the column in order, then a
  // fixed butterfly
  const int jn = min(4 * nq, FK - 4 * qa);
  for (int k = warp; k < K; k += POST_THREADS / 32) {
    const int j0 = ((k - (4 * qa) % K) % K + K) % K;
    float acc = 0.f;
    for (int j = j0 + K * lane; j < jn; j += 32 * K) acc += sq[j];
    acc = warp_sum(acc);
    if (lane == 0) Q.normPart[(int64_t)k * nb + b] = acc;
  }
}

__global__ void __launch_bounds__(POST_THREADS, 2)
fused_norm_kernel(Prob<float> P, PostParams Q, int nparts) {
  extern __shared__ float4 post_sm[];
  float* tile = reinterpret_cast<float*>(post_sm);
  float* rows = tile + POST_CH * 33;                 // 16-byte aligned (POST_CH * 33 * 4 bytes)
  __shared__ float s_norm[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = (int)blockIdx.x, nb = (int)gridDim.x;
  const int K = P.K, K1 = P.K + 1;
  // this block's columns of H; the first pass is loaded before the wait (H is
  // final since the fused sweep, which completed before fused_w_kernel let this
  // launch start). Units of 32 consecutive columns of one row k: warp w takes
  // units w, w + 16, ... (lane = column), no division per entry.
  const int64_t n_lo = P.N * b / nb, n_hi = P.N * (b + 1) / nb;
  auto load_h = [&](int64_t c0, int len) {
    const int ng = (len + 31) >> 5;
    for (int u = warp; u < K * ng; u += POST_THREADS / 32) {
      const int k = u / ng, nl = ((u - k * ng) << 5) + lane;
      if (nl < len) cp_async4(&tile[nl * K1 + k], P.H + (int64_t)k * P.N + c0 + nl, 4u);
    }
  };
  if (n_lo < n_hi) load_h(n_lo, (int)min((int64_t)POST_CH, n_hi - n_lo));
  pdl_wait();
  const bool skip = *Q.status != 0;
  if (Q.lossOut && b == 0 && warp == POST_THREADS / 32 - 1) {
    // the objective of the sweep: its block partials in a fixed order, FP64
    double sl = 0.0;
    for (int b0 = lane; b0 < Q.lossBlocks; b0 += 256) {
      double v[8];
      #pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = b0 + 32 * u < Q.lossBlocks ? Q.lossPart[b0 + 32 * u] : 0.0;
      #pragma unroll
      for (int u = 0; u < 8; ++u) sl += v[u];
    }
    sl = warp_sum(sl);
    if (lane == 0) Q.lossOut[0] = sl;
  }
  // column norms: 16 lanes per column (thread (k, j) sums the partials j,
  // j + 16, ... in order), one fixed butterfly over the 16: the same value in
  // every block
  {
    const int k = tid >> 4, j = tid & 15;
    float acc = 0.f;
    if (k < K)
      for (int i = j; i < nparts; i += 16) acc += Q.normPart[(int64_t)k * nparts + i];
    #pragma unroll
    for (int o = 8; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (k < K && j == 0) s_norm[k] = Q.norm ? sqrtf(acc) : 1.f;
  }
  __syncthreads();
  // this block's share of W: W /= norms, with the TF32 row copy
  const int FK = (int)(P.F * K);
  const int e_lo = (int)((int64_t)FK * b / nb), e_hi = (int)((int64_t)FK * (b + 1) / nb);
  if (!skip)
    for (int e = e_lo + tid; e < e_hi; e += POST_THREADS) {
      const int f = e / K, k = e - f * K;
      const float nk = s_norm[k];
      float w = P.W[e];
      if (nk > 0.f) w = w / nk;
      P.W[e] = w;
      P.sWS[f * P.ks + k] = tf32_round(w);
    }
  if (b == 0 && tid < K && !skip) P.norms[tid] = s_norm[tid];
  // H[k, :] *= norm_k over this block's columns, with Ht and the transposed
  // TF32 copy: its rows (ks = 32 floats; the padding k >= K written as the
  // zeros it holds) for columns [c0, c0 + len) are contiguous, built in shared
  // memory and written with one bulk copy
  for (int64_t c0 = n_lo; c0 < n_hi; c0 += POST_CH) {
    const int len = (int)min((int64_t)POST_CH, n_hi - c0);
    if (c0 != n_lo) {
      if (tid == 0) bulk_wait_read();          // the previous pass's rows were read out
      __syncthreads();
      load_h(c0, len);
    }
    cp_async_wait_all();
    __syncthreads();
    const int ng = (len + 31) >> 5;
    for (int u = warp; u < K * ng; u += POST_THREADS / 32) {
      const int k = u / ng, nl = ((u - k * ng) << 5) + lane;
      if (nl < len) {
        float h = tile[nl * K1 + k];
        const float nk = s_norm[k];
        if (nk > 0.f) h = h * nk;
        if (!skip) {
          P.H[(int64_t)k * P.N + c0 + nl] = h;
          P.Ht[(int64_t)k * P.N + c0 + nl] = h;
        }
        tile[nl * K1 + k] = tf32_round(h);
      }
    }
    __syncthreads();
    for (int nl = warp; nl < len; nl += POST_THREADS / 32) rows[nl * 32 + lane] = lane < K ? tile[nl * K1 + lane] : 0.f;
    fence_smem_to_async();
    __syncthreads();
    if (tid == 0 && !skip) {
      bulk_store(P.sHT + c0 * 32, rows, (uint32_t)len * 128u);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_read();
}

}  // namespace

// ---- host ------------------------------------------------------------------

// The W half and the normalisation after a fused single-problem sweep: two
// launches over every SM, the second with programmatic dependent launch (its
// blocks sit beside the first's: two blocks per SM).
namespace {
template <typename KernelT>
cudaError_t post_smem_once(KernelT kern, size_t bytes) {
  return ensure_smem_attr(reinterpret_cast<const void*>(kern), bytes);
}
}  // namespace

cudaError_t launch_fused_post(const Prob<float>& P, const BetaParams& bp, int slices, bool norm, float* normPart,
                              int nparts, const double* lossPart, int lossBlocks, double* lossOut, int* status,
                              cudaStream_t st) {
  const int64_t FK = P.F * P.K;
  // every block of the first launch takes at most POST_THREADS quads of entries
  // (the transposed copy's rows are 32 floats: ks = 32 for K <= 32)
  if (P.K > 32 || P.ks != 32 || slices < 1 || nparts < 1 || (FK + 3) / 4 > (int64_t)POST_THREADS * nparts ||
      FK > 32768)
    return cudaErrorInvalidValue;
  PostParams Q;
  Q.slices = slices;
  Q.norm = norm ? 1 : 0;
  Q.normPart = normPart;
  Q.lossPart = lossPart;
  Q.lossBlocks = lossBlocks;
  Q.lossOut = lossOut;
  Q.status = status;
  const bool vec = FK % 4 == 0;
  cudaError_t e = cudaSuccess;
#define NMF_POSTW_CASE(BKV)                                                                               \
  case BKV:                                                                                               \
    if (vec) {                                                                                            \
      e = post_smem_once(fused_w_kernel<BKV, true>, POSTW_SMEM);                                          \
      if (e == cudaSuccess)                                                                               \
        e = launch_pdl(fused_w_kernel<BKV, true>, dim3(nparts), dim3(POST_THREADS), POSTW_SMEM, st, P, bp, Q); \
    } else {                                                                                              \
      e = post_smem_once(fused_w_kernel<BKV, false>, POSTW_SMEM);                                         \
      if (e == cudaSuccess)                                                                               \
        e = launch_pdl(fused_w_kernel<BKV, false>, dim3(nparts), dim3(POST_THREADS), POSTW_SMEM, st, P, bp, Q); \
    }                                                                                                     \
    break;
  switch (bp.kind) {
    NMF_POSTW_CASE(BK_IS)
    NMF_POSTW_CASE(BK_KL)
    NMF_POSTW_CASE(BK_EUC)
    NMF_POSTW_CASE(BK_B15)
    NMF_POSTW_CASE(BK_GENERAL)
  }
#undef NMF_POSTW_CASE
  if (e != cudaSuccess) return e;
  e = post_smem_once(fused_norm_kernel, POSTN_SMEM);
  if (e == cudaSuccess)
    e = launch_pdl(fused_norm_kernel, dim3(nparts), dim3(POST_THREADS), POSTN_SMEM, st, P, Q, nparts);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_fused_batch_copies(const Plan<float>& pl, const int* prefHc, int totHc, const int* status,
                                      cudaStream_t st) {
  fused_batch_copies_kernel<<<(unsigned)(pl.totW + totHc), EW, 0, st>>>(pl.d_probs, pl.count, pl.d_prefW, pl.totW,
                                                                         prefHc, status);
  return cudaGetLastError();
}

// Blocks per cluster and tail rows of one problem: F = 128 c + tail with
// 1 <= tail <= FU_TAIL_MAX (= 1) takes c = F / 128 blocks (warp 0 of the last
// one has the tail row), else c = ceil(F / 128) and no tail (NMF_FU_TAIL=0:
// never a tail).
static void fu_geometry(int64_t F, int* c, int* tail) {
  const char* env = std::getenv("NMF_FU_TAIL");
  const bool allow = !(env && std::atoi(env) == 0);
  const int t = (int)(F % 128);
  if (allow && F > 128 && t >= 1 && t <= FU_TAIL_MAX) {
    *c = (int)(F / 128);
    *tail = t;
  } else {
    *c = (int)((F + 127) / 128);
    *tail = 0;
  }
}

int tc_fused_cluster_blocks(const Prob<float>& P) {
  int c = 0, t = 0;
  fu_geometry(P.F, &c, &t);
  return c;
}

bool tc_fused_supported(const Prob<float>& P) {
  return P.sWS && P.kp <= 32 && P.F <= 1024 && fu_pick_nv(P.K, P.kp) >= 2;
}

int tc_fused_clusters(const Prob<float>& P, int sms) {
  const int c = tc_fused_cluster_blocks(P);
  const int nbatch = (int)((P.N + 127) / 128);
  const int nv = fu_pick_nv(P.K, P.kp);
  const size_t sm = 1024 + fu_layout(P.K, P.kp, nv).total;
  auto kern = tc_fused_kernel<BK_GENERAL, false, false>;
  if (ensure_smem_attr(reinterpret_cast<const void*>(kern), sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(c * ((sms + c - 1) / c)));
  cfg.blockDim = dim3(FU_THREADS);
  cfg.dynamicSmemBytes = sm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // NMF_FU_CLUSTERS=<n>: at most n clusters (each then runs more batches; for tests and tuning)
  const char* env = std::getenv("NMF_FU_CLUSTERS");
  if (env && std::atoi(env) > 0 && std::atoi(env) < n) n = std::atoi(env);
  return n < nbatch ? n : nbatch;
}

cudaError_t launch_tc_fused(const Prob<float>& P, const TcMaps& m, const BetaParams& bp, int ncl, double* lossPart,
                            int* status, uint64_t limitNs, unsigned extra, cudaStream_t st, float* gH) {
  FuParams S;
  memset(&S, 0, sizeof(S));
  S.gH = gH;
  fu_geometry(P.F, &S.c, &S.tail);
  S.nbatch = (int)((P.N + 127) / 128);
  S.ncl = ncl;
  S.nv = fu_pick_nv(P.K, P.kp);
  S.layK = P.K;
  S.laykp = P.kp;
  S.lossPart = lossPart;
  S.status = status;
  S.limitNs = limitNs;
  S.extra = extra;
  if (S.nv < 2 || ncl < 1 || ncl > S.nbatch || S.c > 8) return cudaErrorInvalidValue;
  CUtensorMap tmV;
  if (!tc_map_v(P, true, &tmV)) return cudaErrorInvalidValue;   // V rows must be 16-byte aligned (the context pads them)
  const size_t sm = 1024 + fu_layout(P.K, P.kp, S.nv).total;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(S.c * ncl));
  cfg.blockDim = dim3(FU_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S.c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  // No programmatic dependent launch by default: launched early, the clusters
  // are placed around the previous kernel's blocks, and (measured on GB300) in
  // most steps one of the co-resident clusters the grid is sized for was left
  // for a second wave, nearly doubling the kernel's time. NMF_FU_PDL=1 turns
  // it on (A/B measurement).
  static const bool pdl = std::getenv("NMF_FU_PDL") && std::atoi(std::getenv("NMF_FU_PDL")) == 1;
  cfg.numAttrs = pdl ? 2 : 1;
  S.early = pdl ? 0 : 1;
  cudaError_t e = cudaSuccess;
#define NMF_FU_CASE(BKV)                                                                   \
  case BKV:                                                                                \
    if (S.tail > 0) {                                                                      \
      e = ensure_smem_attr(reinterpret_cast<const void*>(tc_fused_kernel<BKV, false, true>), sm);  \
      if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, tc_fused_kernel<BKV, false, true>, tmV, m.wsA, m.htB, P, bp, S); \
    } else {                                                                               \
      e = ensure_smem_attr(reinterpret_cast<const void*>(tc_fused_kernel<BKV, false, false>), sm);  \
      if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, tc_fused_kernel<BKV, false, false>, tmV, m.wsA, m.htB, P, bp, S); \
    }                                                                                      \
    break;
  switch (bp.kind) {
    NMF_FU_CASE(BK_IS)
    NMF_FU_CASE(BK_KL)
    NMF_FU_CASE(BK_EUC)
    NMF_FU_CASE(BK_B15)
    NMF_FU_CASE(BK_GENERAL)
  }
#undef NMF_FU_CASE
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int tc_fused_batch_nv(int layK) { return fu_pick_nv(layK, (layK + 15) & ~15); }

cudaError_t launch_tc_fused_batch(const FuBatch& fb, const BetaParams& bp, int* status, uint64_t limitNs,
                                  unsigned extra, cudaStream_t st) {
  FuParams S;
  memset(&S, 0, sizeof(S));
  S.c = fb.c;
  S.ncl = fb.nitems;
  S.nbatch = 0;
  S.layK = fb.layK;
  S.laykp = (fb.layK + 15) & ~15;
  S.nv = fu_pick_nv(S.layK, S.laykp);
  S.lossPart = fb.lossPart;
  S.status = status;
  S.limitNs = limitNs;
  S.extra = extra;
  S.items = fb.items;
  S.probs = fb.probs;
  S.maps = fb.maps;
  S.lossBase = fb.lossBase;
  S.early = 1;                                        // launched without programmatic dependent launch
  if (S.nv < 2 || fb.nitems < 1 || S.c < 1 || S.c > 8 || S.laykp > 32) return cudaErrorInvalidValue;
  const size_t sm = 1024 + fu_layout(S.layK, S.laykp, S.nv).total;
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  Prob<float> P0;
  memset(static_cast<void*>(&P0), 0, sizeof(P0));
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(S.c * fb.nitems));
  cfg.blockDim = dim3(FU_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S.c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
#define NMF_FU_CASE(BKV)                                                                  \
  case BKV:                                                                               \
    e = ensure_smem_attr(reinterpret_cast<const void*>(tc_fused_kernel<BKV, true, false>), sm);  \
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, tc_fused_kernel<BKV, true, false>, none, none, none, P0, bp, S); \
    break;
  switch (bp.kind) {
    NMF_FU_CASE(BK_IS)
    NMF_FU_CASE(BK_KL)
    NMF_FU_CASE(BK_EUC)
    NMF_FU_CASE(BK_B15)
    NMF_FU_CASE(BK_GENERAL)
  }
#undef NMF_FU_CASE
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace nmf
