// tc_ws.cu -- warp-specialised tensor-core sweeps (padded rank kp <= 64).
//
// Same contract as tc_sweeps.cu: with Vp = Wp Hp + kappa, A = (V + kappa) .
// Vp^(beta-2), B = Vp . Vp^(beta-2) (eq. alt_update / eq. jnt_update),
//   row sweep    P = A D1^T, Q = B D2^T   (F x K, over 32-column tiles n)
//   column sweep Hn = C1^T A, Hd = C2^T B  (K x N, over 32-row tiles f)
// with every product on the tensor cores (tcgen05 kind::tf32, FP32 in TMEM).
//
// Roles (20 warps):
//   warp 0 (+1)  producer: TMA loads of each tile's operands into a ring of
//                stages (V by TMA when its rows are 16-byte aligned, else by
//                cp.async from warps 0-1); the factor operands come from the
//                TF32 shadow copies, already in the 128B-swizzled K-major
//                layout the MMAs read.
//   warp 2       MMA issuer (one thread): MMA1 of tile t into a double-buffered
//                TMEM tile, then MMA2/MMA3 of tile t-1 from the A/B tiles the
//                epilogue produced, so the tensor core never waits on the
//                CUDA cores and vice versa.
//   warps 4-19   epilogue: TMEM -> registers, the powers (and the objective),
//                A and B into a double-buffered shared tile; each thread owns
//                one TMEM lane and 8 of the tile's 32 streamed indices.
// mbarriers connect the roles; every wait is bounded (1 s) and a timeout sets
// NMF_ETIMEOUT, makes every role leave its loop, and frees the TMEM.
//
// Blocks that stream consecutive chunks of the same 128-wide tile form a
// thread-block cluster of c = 1, 2, 4 or 8 blocks. Once its MMAs are done each
// block holds a partial [P | Q] (or [Hn | Hd]) tile; the cluster adds them in a
// fixed binary tree through distributed shared memory (rank r + s sends to rank
// r in round s = 1, 2, 4, ...) and rank 0 writes one partial slice, so the
// epilogue sums blocks / c slices. Blocks of a cluster never leave early:
// every one of them reaches every cluster barrier.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "internal.h"
#include "tc_ptx.cuh"

namespace nmf {
using namespace tc;

namespace {

constexpr int WS_THREADS = 640;
constexpr int TL = 32;
constexpr int MT = 128;
constexpr uint32_t TB = 16384;
constexpr int EPI_WARP0 = 4;
constexpr uint32_t EPI_THREADS = 512;
constexpr int MAX_STAGES = 4;
constexpr int ETIMEOUT = 5;
constexpr size_t SMEM_LIMIT = 227 * 1024;

struct WsLayout {
  uint32_t once;                 // A operand of MMA1, loaded once per block
  uint32_t stage0, stage_bytes;  // stage s at stage0 + s * stage_bytes: V, B of MMA1, B of MMA2, B of MMA3
  uint32_t off_fa, off_d1, off_d2;
  uint32_t ab;                   // A0, B0, A1, B1 tiles (16 KB each)
  uint32_t total;
  int nstages;
};

__host__ __device__ inline WsLayout ws_layout(int kp, bool chi, int nstages) {
  WsLayout L;
  const uint32_t na = (kp + 31) / 32;
  L.once = 0;
  L.stage0 = na * TB;
  L.off_fa = TB;
  L.off_d1 = TB + na * (TL * 128u);
  L.off_d2 = chi ? L.off_d1 + (uint32_t)kp * 128u : L.off_d1;
  L.stage_bytes = L.off_d1 + (uint32_t)kp * 128u * (chi ? 2u : 1u);
  L.stage_bytes = (L.stage_bytes + 1023u) & ~1023u;
  L.ab = L.stage0 + nstages * L.stage_bytes;
  L.total = L.ab + 4 * TB;
  L.nstages = nstages;
  return L;
}

inline int pick_stages(int kp, bool chi) {
  for (int s = MAX_STAGES; s >= 2; --s)
    if (1024 + ws_layout(kp, chi, s).total + 1024 <= SMEM_LIMIT) return s;
  return 0;
}

// Bounded wait shared by every role: gives up on timeout or when another role
// has already given up.
__device__ __forceinline__ bool role_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (globaltimer_ns() - t0 > 1000000000ull) {
      *abort = 1;
      atomicExch(status, ETIMEOUT);
      return false;
    }
  }
  return true;
}

struct Bars {
  uint64_t full[MAX_STAGES], empty[MAX_STAGES], vfull[2], vfree[2], abready[2], abfree[2], once, done;
};

// ROW = true: row sweep (M = 128 rows f, tiles of 32 columns n).
// ROW = false: column sweep (M = 128 columns n, tiles of 32 rows f).
template <int BK, bool CHI, bool ROW>
__global__ void __launch_bounds__(WS_THREADS, 1)
tc_ws_kernel(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmOnce,
             const __grid_constant__ CUtensorMap tmFa, const __grid_constant__ CUtensorMap tmD1,
             const __grid_constant__ CUtensorMap tmD2, int useTma, int nstages, Prob<float> P, int flags,
             BetaParams bp, double* __restrict__ lossPart, int* __restrict__ status) {
  const bool skip = *status != 0;   // read once; the block still runs to the end (cluster barriers)
  extern __shared__ unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  __shared__ double red[32];
  const int K = P.K, kp = (K + 15) & ~15, na = (kp + 31) / 32;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const WsLayout L = ws_layout(kp, CHI, nstages);
  const int NS = nstages;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // block coordinates: the fixed 128-wide dimension (m0) and the streamed chunk [s0, s1)
  // (blocks of one tile are consecutive, so a cluster shares m0)
  const int split = ROW ? P.tcSplitS : P.tcSplitR;
  const int csize = ROW ? P.tcClusterS : P.tcClusterR;
  const int mt = blockIdx.x / split, sl = blockIdx.x % split;
  const int64_t m0 = (int64_t)mt * MT;
  const int64_t mLim = ROW ? P.F : P.N;
  const int64_t chunk = ROW ? P.tcChunkN : P.tcChunkF;
  const int64_t sLim = ROW ? P.N : P.F;
  const int64_t s0 = (int64_t)sl * chunk;
  const int64_t s1 = s0 + chunk < sLim ? s0 + chunk : sLim;
  // padding blocks of the last cluster (s0 >= sLim) stream nothing and add zeros
  const int ntiles = (!skip && s0 < sLim) ? (int)((s1 - s0 + TL - 1) / TL) : 0;
  const bool wantLoss = flags & SWEEP_LOSS;
  const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
  const uint32_t ncols = 256;
  const uint32_t faBytes = (uint32_t)na * TL * 128u, dBytes = (uint32_t)kp * 128u;
  const uint32_t stageTx = (useTma ? TB : 0u) + faBytes + dBytes * (CHI ? 2u : 1u);

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bars.full[s], useTma ? 1u : 65u);
      mbar_init(&bars.empty[s], 1u);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.vfull[b], 1u);
      mbar_init(&bars.vfree[b], EPI_THREADS);
      mbar_init(&bars.abready[b], EPI_THREADS);
      mbar_init(&bars.abfree[b], 1u);
    }
    mbar_init(&bars.once, 1u);
    mbar_init(&bars.done, 1u);
    fence_mbar_init();
  }
  if (warp == 2) tmem_alloc(&tslot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t t_acc1 = tbase + 128, t_acc2 = tbase + 192;   // P | Hn, Q | Hd
  double loss = 0.0;

  if (warp < 2) {
    // ---------------- producer ----------------
    const bool leader = warp == 0 && lane == 0;
    if (leader && ntiles > 0) {
      mbar_arrive_expect_tx(&bars.once, (uint32_t)na * TB);
      for (int a = 0; a < na; ++a) tma_load_2d(base + L.once + a * TB, &tmOnce, 32 * a, (int)m0, &bars.once);
    }
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % NS;
      const int64_t c0 = s0 + (int64_t)t * TL;     // first streamed index of the tile
      if (t >= NS && !role_wait(&bars.empty[st], (uint32_t)(t / NS - 1) & 1u, &s_abort, status)) break;
      unsigned char* sb = base + L.stage0 + st * L.stage_bytes;
      if (leader) {
        mbar_arrive_expect_tx(&bars.full[st], stageTx);
        if (useTma) {
          if (ROW) tma_load_2d(sb, &tmV, (int)c0, (int)m0, &bars.full[st]);
          else tma_load_2d(sb, &tmV, (int)m0, (int)c0, &bars.full[st]);
        }
        for (int a = 0; a < na; ++a) tma_load_2d(sb + L.off_fa + a * (TL * 128), &tmFa, 32 * a, (int)c0, &bars.full[st]);
        tma_load_2d(sb + L.off_d1, &tmD1, (int)c0, 0, &bars.full[st]);
        if (CHI) tma_load_2d(sb + L.off_d2, &tmD2, (int)c0, 0, &bars.full[st]);
      }
      if (!useTma) {
        const int pl = tid;                          // 0..63
        for (int j = 0; j < (MT * TL) / 64; ++j) {
          const int i = pl + 64 * j;
          int64_t gf, gn;
          uint32_t off;
          bool ok;
          if (ROW) {
            const int f = i >> 5, n = i & 31;
            gf = m0 + f; gn = c0 + n;
            ok = gf < P.F && gn < s1;
            off = sw128_offset(f, 4 * n);
          } else {
            const int f = i >> 7, n = i & 127;
            gf = c0 + f; gn = m0 + n;
            ok = gf < s1 && gn < P.N;
            off = 4u * i;
          }
          cp_async4(sb + off, ok ? (const void*)(P.V + gf * P.ldv + gn) : (const void*)P.V, ok ? 4u : 0u);
        }
        cp_async_mbar_arrive(&bars.full[st]);
      }
    }
  } else if (warp == 2) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id_v = idesc(MT, TL, kFmtTF32), id_acc = idesc(MT, kp, kFmtTF32);
      bool ok = ntiles > 0 && role_wait(&bars.once, 0u, &s_abort, status);
      for (int t = 0; ok && t <= ntiles; ++t) {
        if (t < ntiles) {
          const int st = t % NS, b = t & 1;
          if (!role_wait(&bars.full[st], (uint32_t)(t / NS) & 1u, &s_abort, status)) break;
          if (t >= 2 && !role_wait(&bars.vfree[b], (uint32_t)((t - 2) >> 1) & 1u, &s_abort, status)) break;
          fence_after_sync();
          const unsigned char* sb = base + L.stage0 + st * L.stage_bytes;
          for (int ks = 0; ks < kp / 8; ++ks) {
            const int k0 = ks * 8;
            const uint32_t within = (uint32_t)(k0 & 31) * 4u;
            mma_tf32(tbase + 32 * b, desc_sw128(smem_u32(base + L.once + (k0 >> 5) * TB) + within),
                     desc_sw128(smem_u32(sb + L.off_fa + (k0 >> 5) * (TL * 128)) + within), id_v, ks > 0);
          }
          mma_commit(&bars.vfull[b]);
        }
        if (t >= 1) {
          const int u = t - 1, bu = u & 1, su = u % NS;
          if (!role_wait(&bars.abready[bu], (uint32_t)(u >> 1) & 1u, &s_abort, status)) break;
          fence_after_sync();
          const unsigned char* sb = base + L.stage0 + su * L.stage_bytes;
          const unsigned char* As = base + L.ab + bu * 2 * TB;
          const unsigned char* Bs = As + TB;
          for (int ks = 0; ks < TL / 8; ++ks) {
            const uint32_t within = (uint32_t)ks * 32u;
            const uint32_t acc = (u > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(t_acc1, desc_sw128(smem_u32(As) + within), desc_sw128(smem_u32(sb + L.off_d1) + within), id_acc, acc);
            mma_tf32(t_acc2, desc_sw128(smem_u32(Bs) + within), desc_sw128(smem_u32(sb + L.off_d2) + within), id_acc, acc);
          }
          mma_commit(&bars.abfree[bu]);
          mma_commit(&bars.empty[su]);
        }
      }
      mma_commit(&bars.done);
    }
  } else if (warp >= EPI_WARP0) {
    // ---------------- epilogue ----------------
    const int q4 = warp & 3, grp = (warp - EPI_WARP0) >> 2;   // TMEM lane quarter, group of 8 streamed indices
    const int mrow = 32 * q4 + lane;                          // this thread's TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
    const int64_t gm = m0 + mrow;
    const bool mvalid = gm < mLim;
    const int jb0 = 8 * grp;
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % NS, b = t & 1;
      const int64_t c0 = s0 + (int64_t)t * TL;
      const int nvalid = (int)((s1 - c0) < TL ? (s1 - c0) : TL);   // streamed indices of this tile inside the chunk
      if (!role_wait(&bars.vfull[b], (uint32_t)(t >> 1) & 1u, &s_abort, status)) break;
      if (!role_wait(&bars.full[st], (uint32_t)(t / NS) & 1u, &s_abort, status)) break;
      fence_after_sync();
      float vt[8];
      tmem_ld8(tbase + 32 * b + lane_off + jb0, vt);
      tmem_ld_wait();
      fence_before_sync();
      mbar_arrive(&bars.vfree[b]);
      if (t >= 2 && !role_wait(&bars.abfree[b], (uint32_t)((t - 2) >> 1) & 1u, &s_abort, status)) break;
      const unsigned char* sb = base + L.stage0 + st * L.stage_bytes;
      unsigned char* As = base + L.ab + b * 2 * TB;
      unsigned char* Bs = As + TB;
      float vv[8];
      if (ROW) {
        const float4 v0 = *reinterpret_cast<const float4*>(sb + sw128_offset(mrow, 4 * jb0));
        const float4 v1 = *reinterpret_cast<const float4*>(sb + sw128_offset(mrow, 4 * jb0 + 16));
        vv[0] = v0.x; vv[1] = v0.y; vv[2] = v0.z; vv[3] = v0.w;
        vv[4] = v1.x; vv[5] = v1.y; vv[6] = v1.z; vv[7] = v1.w;
      } else {
        const float* Vs = reinterpret_cast<const float*>(sb) + mrow;
        #pragma unroll
        for (int j = 0; j < 8; ++j) vv[j] = Vs[(jb0 + j) * MT];
      }
      float a[8], bb[8];
      float tl = 0.f;
      if (mvalid && jb0 + 8 <= nvalid) {             // every entry of this thread's group is inside
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float v = vv[j] + kappa, y = vt[j] + kappa;
          ab_terms_fast<BK>(v, y, bm2, a[j], bb[j]);
          if (wantLoss) tl += dbeta_fast<BK>(v, y, (float)bp.beta, bp.series);
        }
      } else {
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          a[j] = 0.f;
          bb[j] = 0.f;
          if (mvalid && jb0 + j < nvalid) {
            const float v = vv[j] + kappa, y = vt[j] + kappa;
            ab_terms_fast<BK>(v, y, bm2, a[j], bb[j]);
            if (wantLoss) tl += dbeta_fast<BK>(v, y, (float)bp.beta, bp.series);
          }
        }
      }
      const uint32_t off0 = sw128_offset(mrow, 4 * jb0), off1 = sw128_offset(mrow, 4 * jb0 + 16);
      *reinterpret_cast<float4*>(As + off0) = make_float4(to_tf32(a[0]), to_tf32(a[1]), to_tf32(a[2]), to_tf32(a[3]));
      *reinterpret_cast<float4*>(As + off1) = make_float4(to_tf32(a[4]), to_tf32(a[5]), to_tf32(a[6]), to_tf32(a[7]));
      *reinterpret_cast<float4*>(Bs + off0) = make_float4(to_tf32(bb[0]), to_tf32(bb[1]), to_tf32(bb[2]), to_tf32(bb[3]));
      *reinterpret_cast<float4*>(Bs + off1) = make_float4(to_tf32(bb[4]), to_tf32(bb[5]), to_tf32(bb[6]), to_tf32(bb[7]));
      loss += (double)tl;
      fence_smem_to_async();
      mbar_arrive(&bars.abready[b]);
    }
  }

  // ---------------- accumulators: cluster tree, then one partial slice ----------------
  // Epilogue thread (mrow, grp) owns kp / 2 consecutive columns of [P | Q] in
  // TMEM lane mrow: groups 0-1 the first accumulator, 2-3 the second.
  const bool epi = warp >= EPI_WARP0;
  const int q4 = warp & 3, grp = (warp - EPI_WARP0) >> 2;
  const int mrow = 32 * q4 + lane;
  const int per = kp / 2;                             // 8, 16, 24 or 32
  const bool isQ = grp >= 2;
  const int col0 = (grp & 1) * per;                   // first column inside P or Q
  float acc[32];
  #pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
  if (epi) {
    bool have = !s_abort && ntiles > 0 && role_wait(&bars.done, 0u, &s_abort, status);
    have = __all_sync(0xffffffffu, have);             // tcgen05.ld is warp-wide
    if (have) {
      fence_after_sync();
      const uint32_t ta = (isQ ? t_acc2 : t_acc1) + ((uint32_t)(32 * q4) << 16) + col0;
      #pragma unroll
      for (int i = 0; i < 4; ++i)
        if (8 * i < per) tmem_ld8(ta + 8 * i, &acc[8 * i]);
      tmem_ld_wait();
    }
  }
  if (csize > 1) {
    const uint32_t rank = cluster_rank();
    // Two exchange buffers of kp KB, alternating by round: the A/B tiles and
    // the stage ring, both idle once the block's MMAs have completed (the
    // first barrier below). Layout [float4 q][lane m] keeps the stores
    // conflict-free.
    cluster_sync();
    int round = 0;
    for (int stp = 1; stp < csize; stp <<= 1, ++round) {
      unsigned char* buf = base + ((round & 1) ? L.stage0 : L.ab);
      const uint32_t qbase = (uint32_t)((isQ ? per * 2 : 0) + col0) / 4;   // this thread's first float4
      if (epi && (rank & (2 * stp - 1)) == (uint32_t)stp) {
        const uint32_t remote = dsmem_map(buf, rank - stp);
        #pragma unroll
        for (int i = 0; i < 8; ++i)
          if (4 * i < per)
            dsmem_st4(remote + ((qbase + i) * MT + mrow) * 16u, acc[4 * i], acc[4 * i + 1], acc[4 * i + 2],
                      acc[4 * i + 3]);
      }
      cluster_sync();
      if (epi && (rank & (2 * stp - 1)) == 0u) {
        #pragma unroll
        for (int i = 0; i < 8; ++i)
          if (4 * i < per) {
            const float4 v = *reinterpret_cast<const float4*>(buf + ((qbase + i) * MT + mrow) * 16u);
            acc[4 * i] += v.x; acc[4 * i + 1] += v.y; acc[4 * i + 2] += v.z; acc[4 * i + 3] += v.w;
          }
      }
    }
  }
  if (ROW) {
    // P and Q of rows [m0, m0 + 128) are two contiguous runs of rowPart
    // (row-major F x K): stage them in shared memory (odd row stride, no bank
    // conflicts) and let the whole block write them out coalesced.
    const int Ks = K | 1;
    float* stg = reinterpret_cast<float*>(base + L.stage0);   // idle: MMAs done, exchange rounds over
    __syncthreads();
    if (epi && sl % csize == 0) {
      float* row = stg + (isQ ? MT * Ks : 0) + mrow * Ks + col0;
      #pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < per && col0 + j < K) row[j] = acc[j];
    }
    __syncthreads();
    if (sl % csize == 0) {
      const int nrows = (int)(mLim - m0 < MT ? mLim - m0 : MT);
      const int cnt = nrows * K;
      float* outP = P.rowPart + (int64_t)(sl / csize) * 2 * P.F * K + m0 * K;
      float* outQ = outP + P.F * K;
      for (int i = tid; i < cnt; i += WS_THREADS) {
        const int r = i / K, c = i - r * K;
        outP[i] = stg[r * Ks + c];
        outQ[i] = stg[MT * Ks + r * Ks + c];
      }
    }
  } else if (epi && sl % csize == 0) {
    const int64_t gm = m0 + mrow;
    if (gm < mLim) {
      const int64_t KN = (int64_t)K * P.N;
      float* part = P.colPart + (int64_t)(sl / csize) * 2 * KN + (isQ ? KN : 0) + (int64_t)col0 * P.N + gm;
      #pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < per && col0 + j < K) part[(int64_t)j * P.N] = acc[j];
    }
  }
  if (wantLoss) {
    const double tt = block_sum(loss, red);
    if (tid == 0) lossPart[blockIdx.x] = tt;
  }
  fence_before_sync();
  __syncthreads();
  if (s_abort) mbar_wait(&bars.done, 0u, 100000000ull);
  if (warp == 2) tmem_dealloc(tbase, ncols);
}

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
                      int* status, cudaStream_t st) {
  const int kp = P.kp;
  const int ns = pick_stages(kp, CHI);
  if (ns == 0) return cudaErrorInvalidValue;
  CUtensorMap tmV;
  memset(&tmV, 0, sizeof(tmV));
  const int useTma = ROW ? map2d(&tmV, P.V, P.N, P.F, P.ldv, TL, MT, CU_TENSOR_MAP_SWIZZLE_128B)
                         : map2d(&tmV, P.V, P.N, P.F, P.ldv, MT, TL, CU_TENSOR_MAP_SWIZZLE_NONE);
  const CUtensorMap& once = ROW ? m.wsA : m.htA;
  const CUtensorMap& fa = ROW ? m.htB : m.wsB;
  const CUtensorMap& d1 = ROW ? (CHI ? m.ch1 : m.hs) : (CHI ? m.cw1 : m.wt);
  const CUtensorMap& d2 = ROW ? (CHI ? m.ch2 : m.hs) : (CHI ? m.cw2 : m.wt);
  const WsLayout lay = ws_layout(kp, CHI, ns);
  const size_t sm = 1024 + lay.total;
  const int csize = ROW ? P.tcClusterS : P.tcClusterR;
  // the cluster exchange buffers (A/B tiles, stage ring) each hold kp KB
  if (csize > 1 && ((uint32_t)ns * lay.stage_bytes < 1024u * kp || 4 * TB < 1024u * kp)) return cudaErrorInvalidValue;
  // the row sweep stages its [P | Q] tile (2 x 128 x (K | 1) floats) over the stage ring and the A/B tiles
  if (ROW && lay.total - lay.stage0 < 2u * MT * (uint32_t)(P.K | 1) * 4u) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(ROW ? P.tcRowTiles * P.tcSplitS : P.tcColTiles * P.tcSplitR);
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(WS_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
#define NMF_WS_CASE(BKV)                                                                                   \
  case BKV:                                                                                                \
    e = prep(tc_ws_kernel<BKV, CHI, ROW>, sm);                                                              \
    if (e == cudaSuccess)                                                                                  \
      e = cudaLaunchKernelEx(&cfg, tc_ws_kernel<BKV, CHI, ROW>, tmV, once, fa, d1, d2, useTma, ns, P, flags, bp, \
                             lossPart, status);                                                            \
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

bool tc_build_maps(const Prob<float>& P, TcMaps* m) {
  m->ok = false;
  if (!P.sWS || P.kp > 64) return false;
  const int64_t F = P.F, N = P.N;
  const int kp = P.kp, ks = P.ks;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  bool ok = true;
  ok = ok && map2d(&m->wsA, P.sWS, ks, F, ks, 32, MT, SW);
  ok = ok && map2d(&m->wsB, P.sWS, ks, F, ks, 32, TL, SW);
  ok = ok && map2d(&m->htA, P.sHT, ks, N, ks, 32, MT, SW);
  ok = ok && map2d(&m->htB, P.sHT, ks, N, ks, 32, TL, SW);
  ok = ok && map2d(&m->hs, P.sHS, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->ch1, P.sCH1, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->ch2, P.sCH2, N, kp, P.Np, 32, kp, SW);
  ok = ok && map2d(&m->wt, P.sWT, F, kp, P.Fp, 32, kp, SW);
  ok = ok && map2d(&m->cw1, P.sCW1, F, kp, P.Fp, 32, kp, SW);
  ok = ok && map2d(&m->cw2, P.sCW2, F, kp, P.Fp, 32, kp, SW);
  m->ok = ok;
  return ok;
}

int tc_ws_capacity(int kp, int csize) {
  if (kp > 64 || kp < 16) return 0;
  const int ns = pick_stages(kp, true);
  if (ns == 0) return 0;
  const size_t sm = 1024 + ws_layout(kp, true, ns).total;
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
                             double* lossPart, int* status, cudaStream_t st) {
  return dsel == OP_CHI ? launch_ws<true, true>(P, m, flags, bp, lossPart, status, st)
                        : launch_ws<false, true>(P, m, flags, bp, lossPart, status, st);
}

cudaError_t launch_tc_ws_col(const Prob<float>& P, const TcMaps& m, int csel, int flags, const BetaParams& bp,
                             double* lossPart, int* status, cudaStream_t st) {
  return csel == OP_CHI ? launch_ws<true, false>(P, m, flags, bp, lossPart, status, st)
                        : launch_ws<false, false>(P, m, flags, bp, lossPart, status, st);
}

}  // namespace nmf
