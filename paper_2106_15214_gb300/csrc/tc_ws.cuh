// tc_ws.cuh -- warp-specialised tensor-core sweeps (padded rank kp <= 64):
// the sweep as a device function over one unit (one 128-wide tile, one chunk
// of the streamed dimension), used by the one-launch-per-sweep kernel below
// (host side in tc_ws.cu) and by the persistent step kernel (tc_step.cu).
//
// Same contract as tc_sweeps.cu: with Vp = Wp Hp + kappa, A = (V + kappa) .
// Vp^(beta-2), B = Vp . Vp^(beta-2) (eq. alt_update / eq. jnt_update),
//   row sweep    P = A D1^T, Q = B D2^T   (F x K, over 32-column tiles n)
//   column sweep Hn = C1^T A, Hd = C2^T B  (K x N, over 32-row tiles f)
// with every product on the tensor cores (tcgen05 kind::tf32, FP32 in TMEM).
//
// Roles (20 warps):
//   warp 0       operand producer: TMA loads of the MMA1 A tile (once per
//                block) and, per tile, of the B operands of MMA1/2/3 into a
//                ring of operand slots; they come from the TF32 shadow copies,
//                already in the 128B-swizzled K-major layout the MMAs read.
//   warp 1       V producer: the V tile of each tile step into its own ring
//                (TMA when V's rows are 16-byte aligned, else cp.async).
//   warp 2       MMA issuer (converged warp, an elected lane issues, the
//                warp sleeping in each wait): MMA1 of a batch of 4 tiles
//                into one of 2 TMEM Vt buffers, MMA2/MMA3 of a tile as soon
//                as its A/B tiles are written, so the tensor core and the
//                CUDA cores overlap. Every A operand is read from TMEM (the
//                MMA1 tile, moved there once, and the epilogue's A/B tiles):
//                about 2.5x the issue rate of shared-memory A operands, and
//                no shared-memory traffic for them.
//   warp 3       side jobs: column norms and the objective's final sum from
//                the previous kernel's partials.
//   warps 4-19   epilogue: Vt from TMEM and V from shared memory to
//                registers, the powers (and the objective), A and B back to
//                TMEM. Two groups of 8 warps take alternate tiles; each
//                thread owns one TMEM lane and 16 of the tile's 32 streamed
//                indices.
// Before the dependency wait on the previous kernel: TMEM allocation, barrier
// initialisation, the tensor maps' prefetch and the first V tiles.
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
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

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
constexpr int MAX_OP = 8;          // per-tile operand ring slots (B of MMA2, B of MMA3)
constexpr int MAX_V = 6;           // V ring slots
constexpr int NFA = 2;             // batch slots for the B operand of MMA1
constexpr int BT = 4;              // tiles per MMA1 batch (N = 128)
constexpr int ETIMEOUT = 5;
constexpr size_t SMEM_LIMIT = 227 * 1024;
// TMEM columns (512 allocated): two Vt buffers of a batch of 4 tiles (tile t of
// batch j at 128 (j & 1) + 32 (t & 3)); the epilogue overwrites each tile's
// Vt with its A tile. The B tiles of epilogue group g at 256 + 32 g, the
// accumulators at 320 and 384, the A operand of MMA1 at 448 (kp <= 64).
constexpr uint32_t TM_B = 256, TM_ACC1 = 320, TM_ACC2 = 384, TM_ONCE = 448, TM_COLS = 512;

// Shared memory: the A operand of MMA1 as loaded (it moves on to TMEM), a
// double buffer of MMA1 B operands (128 streamed rows each), a ring of
// per-tile MMA2/3 B operands and a ring of V tiles.
struct WsLayout {
  uint32_t once;
  uint32_t fa0, fa_bytes;        // MMA1 B slot s at fa0 + s * fa_bytes
  uint32_t op0, op_bytes;        // MMA2/3 slot s at op0 + s * op_bytes
  uint32_t off_d2;               // second operand inside a slot
  uint32_t v0;                   // V slot s at v0 + s * TB
  uint32_t total;
};

__host__ __device__ inline WsLayout ws_layout(int kp, bool chi, int nop, int nv) {
  WsLayout L;
  const uint32_t na = (kp + 31) / 32;
  L.once = 0;
  L.fa0 = na * TB;
  L.fa_bytes = na * TB;                                   // na sub-tiles of 128 rows x 32 floats
  L.op0 = L.fa0 + NFA * L.fa_bytes;
  L.off_d2 = chi ? (uint32_t)kp * 128u : 0u;
  L.op_bytes = (uint32_t)kp * 128u * (chi ? 2u : 1u);
  L.op_bytes = (L.op_bytes + 1023u) & ~1023u;
  L.v0 = L.op0 + nop * L.op_bytes;
  L.total = L.v0 + nv * TB;
  return L;
}

// Deepest rings that fit: V slots first (down to 4), then operand slots.
inline bool pick_rings(int kp, bool chi, int* nop, int* nv) {
  for (int v = MAX_V; v >= 3; --v)
    for (int o = MAX_OP; o >= (v >= 5 ? 6 : 3); --o)
      if (1024 + ws_layout(kp, chi, o, v).total + 1024 <= SMEM_LIMIT) {
        *nop = o;
        *nv = v;
        return true;
      }
  return false;
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
  uint64_t opfull[MAX_OP], opempty[MAX_OP], vfull[MAX_V], vempty[MAX_V];
  uint64_t fafull[NFA], fafree[NFA], tfull[2], vafree[2], abready[2], abfree[2], once, onceT, done;
};

// ROW = true: row sweep (M = 128 rows f, tiles of 32 columns n).
// ROW = false: column sweep (M = 128 columns n, tiles of 32 rows f).

// Run by one warp: the side job's column norm and objective (fixed-order
// lane sums and butterfly: deterministic).
__device__ __forceinline__ void side_run(const SideJob* side, int lane, int K) {
  if (side && side->normPart && side->normK >= 0) {
    for (int k = side->normK; k < K; k += side->normStride) {
      float sq = 0.f;
      const float* row = side->normPart + (int64_t)k * side->nparts;
      for (int b0 = lane; b0 < side->nparts; b0 += 256) {   // loads in flight together, added in order
        float v[8];
        #pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = b0 + 32 * u < side->nparts ? __ldcg(&row[b0 + 32 * u]) : 0.f;
        #pragma unroll
        for (int u = 0; u < 8; ++u) sq += v[u];
      }
      sq = warp_sum(sq);
      if (lane == 0) side->norms[k] = sqrtf(sq);
    }
  }
  if (side && side->nloss > 0) {
    double sl = 0.0;
    for (int b0 = lane; b0 < side->nloss; b0 += 256) {
      double v[8];
      #pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = b0 + 32 * u < side->nloss ? __ldcg(&side->lossPart[b0 + 32 * u]) : 0.0;
      #pragma unroll
      for (int u = 0; u < 8; ++u) sl += v[u];
    }
    sl = warp_sum(sl);
    if (lane == 0) side->lossOut[0] = sl;
  }
}

// What one unit covers: the 128-wide tile mt of the fixed dimension, the
// streamed range [s0, s1), the partial slice it writes (outSlice; with a
// cluster, the blocks of slices sl .. sl + c - 1 write slice sl / c).
struct UnitGeom {
  int mt, sl, outSlice;
  int64_t s0, s1;
};

// The uniform split: unit = mt * split + sl, chunks of tcChunkN / tcChunkF.
template <bool ROW>
__device__ __forceinline__ UnitGeom uniform_geom(const Prob<float>& P, int unit) {
  UnitGeom g;
  const int split = ROW ? P.tcSplitS : P.tcSplitR;
  const int csize = ROW ? P.tcClusterS : P.tcClusterR;
  g.mt = unit / split;
  g.sl = unit % split;
  g.outSlice = g.sl / csize;
  const int64_t chunk = ROW ? P.tcChunkN : P.tcChunkF;
  const int64_t sLim = ROW ? P.N : P.F;
  g.s0 = (int64_t)g.sl * chunk;
  g.s1 = g.s0 + chunk < sLim ? g.s0 + chunk : sLim;
  return g;
}

// Initialises the unit's barriers (one thread; a __syncthreads must follow).
__device__ __forceinline__ void ws_init_bars(Bars& bars, int nop, int nv, int useTma) {
  for (int s = 0; s < nop; ++s) {
    mbar_init(&bars.opfull[s], 1u);
    mbar_init(&bars.opempty[s], 1u);
  }
  for (int s = 0; s < nv; ++s) {
    mbar_init(&bars.vfull[s], useTma ? 1u : 32u);
    mbar_init(&bars.vempty[s], EPI_THREADS / 64);   // the 8 warps of the group that reads the tile
  }
  for (int b = 0; b < NFA; ++b) {
    mbar_init(&bars.fafull[b], 1u);
    mbar_init(&bars.fafree[b], 1u);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_init(&bars.tfull[b], 1u);
    mbar_init(&bars.vafree[b], 1u);
    mbar_init(&bars.abready[b], EPI_THREADS / 64);
    mbar_init(&bars.abfree[b], 1u);
  }
  mbar_init(&bars.once, 1u);
  mbar_init(&bars.onceT, 4u);                      // epilogue warps 4-7 after moving it to TMEM
  mbar_init(&bars.done, 1u);
  fence_mbar_init();
}

// Streamed tiles of a unit and the V tiles that may be loaded before the
// previous kernel has finished (V is never written by the step's kernels):
// the first min(nv, tiles) through TMA.
__device__ __forceinline__ int ws_tiles(const Prob<float>& P, bool row, const UnitGeom& g) {
  const int64_t sLim = row ? P.N : P.F;
  return g.s0 < sLim ? (int)((g.s1 - g.s0 + TL - 1) / TL) : 0;
}

// Run by the V producer warp before the dependency wait: issues V tiles
// 0 .. n - 1 of the unit into ring slots 0 .. n - 1 (one elected lane).
template <bool ROW>
__device__ __forceinline__ void ws_v_issue(const CUtensorMap& tmV, const Prob<float>& P, const UnitGeom& g, int n,
                                           unsigned char* vring, Bars& bars) {
  if (elect_one()) {
    const int m0 = g.mt * MT;
    for (int t = 0; t < n; ++t) {
      const int c0 = (int)(g.s0 + (int64_t)t * TL);
      mbar_arrive_expect_tx(&bars.vfull[t], TB);
      if (ROW) tma_load_2d(vring + t * TB, &tmV, c0, m0, &bars.vfull[t]);
      else tma_load_2d(vring + t * TB, &tmV, m0, c0, &bars.vfull[t]);
    }
  }
  __syncwarp();
}

// Returns the unit's objective partial (valid in thread 0; 0 without SWEEP_LOSS).
// barsReady: the caller initialised the barriers; vPre: V tiles the caller
// already issued (ws_v_issue), which are waited for even when the unit skips.
template <int BK, bool CHI, bool ROW>
__device__ __forceinline__ double ws_unit(const CUtensorMap& tmV, const CUtensorMap& tmOnce, const CUtensorMap& tmFa,
                                          const CUtensorMap& tmD1, const CUtensorMap& tmD2, int useTma, int nop,
                                          int nv, const Prob<float>& P, int flags, const BetaParams& bp,
                                          int* __restrict__ status, const UnitGeom& geo, bool skip,
                                          unsigned char* base, uint32_t tbase, Bars& bars, volatile int& s_abort,
                                          double* red, const SideJob* side, bool reuse, bool barsReady = false,
                                          int vPre = 0) {
  const int K = P.K, kp = (K + 15) & ~15, na = (kp + 31) / 32;
  const WsLayout L = ws_layout(kp, CHI, nop, nv);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the fixed 128-wide dimension (m0) and the streamed range [s0, s1)
  // (blocks of one tile are consecutive, so a cluster shares m0)
  const int csize = ROW ? P.tcClusterS : P.tcClusterR;
  const int mt = geo.mt, sl = geo.sl;
  const int64_t m0 = (int64_t)mt * MT;
  const int64_t mLim = ROW ? P.F : P.N;
  const int64_t s0 = geo.s0;
  const int64_t s1 = geo.s1;
  // padding blocks of the last cluster (s0 >= sLim) stream nothing and add zeros
  const int ntilesGeom = ws_tiles(P, ROW, geo);
  const bool wantLoss = flags & SWEEP_LOSS;
  const bool early = flags & SWEEP_EARLY;
  const float kappa = (float)bp.kappa, bm2 = (float)(bp.beta - 2.0);
  const uint32_t dBytes = (uint32_t)kp * 128u;
  const uint32_t opTx = dBytes * (CHI ? 2u : 1u);

  if (tid == 0) {
    s_abort = 0;
    if (!barsReady) ws_init_bars(bars, nop, nv, useTma);
  }
  __syncthreads();
  const int ntiles = skip ? 0 : ntilesGeom;
  const int nbatch = (ntiles + BT - 1) / BT;
  const uint32_t t_acc1 = tbase + TM_ACC1, t_acc2 = tbase + TM_ACC2;   // P | Hn, Q | Hd
  // the unit's objective partial per thread, in float-float (FP64 arithmetic
  // in the tile loop would occupy the SM's FP64 pipe for ~500 cycles a tile)
  float lossHi = 0.f, lossLo = 0.f;

  if (warp == 0) {
    // ---------------- operand producer ----------------
    // The MMA1 A tile once; per batch of 4 tiles the MMA1 B operand (128
    // streamed rows); per tile the MMA2/3 B operands. The warp runs the loop
    // converged; one elected lane issues each copy.
    if (ntiles > 0) {
      if (elect_one()) {
        mbar_arrive_expect_tx(&bars.once, (uint32_t)na * TB);
        for (int a = 0; a < na; ++a) tma_load_2d(base + L.once + a * TB, &tmOnce, 32 * a, (int)m0, &bars.once);
      }
      int st = 0;
      uint32_t ph = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int c0 = (int)(s0 + (int64_t)t * TL);   // first streamed index of the tile
        if ((t & (BT - 1)) == 0) {
          const int j = t / BT, fs = j & (NFA - 1);
          if (j >= NFA && !__all_sync(0xffffffffu, role_wait(&bars.fafree[fs], (uint32_t)((j - NFA) / NFA) & 1u, &s_abort, status)))
            break;
          if (elect_one()) {
            mbar_arrive_expect_tx(&bars.fafull[fs], (uint32_t)na * TB);
            for (int a = 0; a < na; ++a)
              tma_load_2d(base + L.fa0 + fs * L.fa_bytes + a * TB, &tmFa, 32 * a, c0, &bars.fafull[fs]);
          }
          __syncwarp();
        }
        if (t >= nop && !__all_sync(0xffffffffu, role_wait(&bars.opempty[st], ph ^ 1u, &s_abort, status))) break;
        if (early && t == 0) pdl_wait();              // the MMA2/3 operands come from the previous kernel
        unsigned char* sb = base + L.op0 + st * L.op_bytes;
        if (elect_one()) {
          mbar_arrive_expect_tx(&bars.opfull[st], opTx);
          tma_load_2d(sb, &tmD1, c0, 0, &bars.opfull[st]);
          if (CHI) tma_load_2d(sb + L.off_d2, &tmD2, c0, 0, &bars.opfull[st]);
        }
        __syncwarp();
        if (++st == nop) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- V producer: TMA from an elected lane, else cp.async from the warp ----------------
    // tiles 0 .. vPre - 1 were issued before the dependency wait; a unit
    // that skips still waits for them (no copy may land after the block ends)
    for (int t = ntiles; t < vPre; ++t)
      if (!__all_sync(0xffffffffu, mbar_wait(&bars.vfull[t], 0u, 100000000ull))) break;
    int st = vPre < nv ? vPre : 0;
    uint32_t ph = vPre < nv ? 0u : 1u;
    for (int t = vPre; t < ntiles; ++t) {
      const int64_t c0 = s0 + (int64_t)t * TL;
      if (t >= nv && !__all_sync(0xffffffffu, role_wait(&bars.vempty[st], ph ^ 1u, &s_abort, status))) break;
      unsigned char* vb = base + L.v0 + st * TB;
      if (useTma) {
        if (elect_one()) {
          mbar_arrive_expect_tx(&bars.vfull[st], TB);
          if (ROW) tma_load_2d(vb, &tmV, (int)c0, (int)m0, &bars.vfull[st]);
          else tma_load_2d(vb, &tmV, (int)m0, (int)c0, &bars.vfull[st]);
        }
        __syncwarp();
      } else {
        for (int j = 0; j < (MT * TL) / 32; ++j) {
          const int i = lane + 32 * j;
          int64_t gf, gn;
          uint32_t off;
          bool in;
          if (ROW) {
            const int f = i >> 5, n = i & 31;
            gf = m0 + f; gn = c0 + n;
            in = gf < P.F && gn < s1;
            off = sw128_offset(f, 4 * n);
          } else {
            const int f = i >> 7, n = i & 127;
            gf = c0 + f; gn = m0 + n;
            in = gf < s1 && gn < P.N;
            off = 4u * i;
          }
          cp_async4(vb + off, in ? (const void*)(P.V + gf * P.ldv + gn) : (const void*)P.V, in ? 4u : 0u);
        }
        cp_async_mbar_arrive(&bars.vfull[st]);
      }
      if (++st == nv) {
        st = 0;
        ph ^= 1u;
      }
    }
  } else if (warp == 2) {
    // ---------------- MMA issuer ----------------
    // A fixed schedule; the warp sleeps in each wait (mbarrier try_wait with a
    // suspend hint) and one elected lane issues:
    //   MMA1 of batches 0 and 1 (Vt of 4 tiles each, N = 128, into TMEM
    //   buffer j & 1);
    //   per tile t2: MMA2/3 once the epilogue has written its A/B tiles and
    //   the tile's B operands are loaded; after the first tile of batch
    //   j - 1, MMA1 of batch j (its buffer's previous batch, j - 2, has been
    //   issued completely one tile earlier, so its completion is near).
    // A sleeping warp takes no issue slots from the epilogue warps that share
    // its scheduler and wakes when the barrier completes (a loop polling the
    // queues in turn measured the same step time; the fixed order is simpler).
    // Every A operand is read from TMEM, every B operand from shared memory.
    // Descriptors are built once; an operand at byte offset o is the base
    // descriptor plus o / 16 (the start-address field, bits 0-13, cannot carry
    // below 256 KB).
    const uint32_t id_v = idesc(MT, BT * TL, kFmtTF32), id_acc = idesc(MT, kp, kFmtTF32);
    const uint64_t dFa = desc_sw128(smem_u32(base + L.fa0));
    const uint64_t dOp = desc_sw128(smem_u32(base + L.op0));
    const uint32_t fa16 = L.fa_bytes >> 4, op16 = L.op_bytes >> 4, d2_16 = L.off_d2 >> 4;
    int j1 = 0, so2 = 0;
    uint32_t po2 = 0;
    bool ok = ntiles > 0 && role_wait(&bars.onceT, 0u, &s_abort, status);
    ok = __all_sync(0xffffffffu, ok);
    // MMA1 of batch j: Fa tile loaded, TMEM buffer j & 1 free (batch j - 2's MMA2/3 complete)
    auto mma1 = [&](int j) -> bool {
      const int fs = j & (NFA - 1);
      if (!__all_sync(0xffffffffu, role_wait(&bars.fafull[fs], (uint32_t)(j / NFA) & 1u, &s_abort, status)))
        return false;
      if (j >= 2 &&
          !__all_sync(0xffffffffu, role_wait(&bars.vafree[j & 1], (uint32_t)((j - 2) >> 1) & 1u, &s_abort, status)))
        return false;
      fence_after_sync();
      const uint64_t db0 = dFa + (uint64_t)(fs * fa16);
      const uint32_t dv = tbase + 128u * (j & 1);
      if (elect_one()) {
        #pragma unroll
        for (int ks = 0; ks < 8; ++ks)
          if (ks < kp / 8) {
            const uint32_t k0 = (uint32_t)ks * 8u;
            mma_tf32_ts(dv, tbase + TM_ONCE + k0, db0 + (((k0 >> 5) * TB + (k0 & 31u) * 4u) >> 4), id_v, ks > 0);
          }
        mma_commit(&bars.tfull[j & 1]);
        mma_commit(&bars.fafree[fs]);
      }
      __syncwarp();
      return true;
    };
    if (ok) ok = mma1(j1++);
    if (ok && j1 < nbatch) ok = mma1(j1++);
    for (int t2 = 0; ok && t2 < ntiles; ++t2) {
      if (!__all_sync(0xffffffffu, role_wait(&bars.abready[t2 & 1], (uint32_t)(t2 >> 1) & 1u, &s_abort, status)))
        break;
      if (!__all_sync(0xffffffffu, role_wait(&bars.opfull[so2], po2, &s_abort, status))) break;
      fence_after_sync();
      const int b = t2 & 1;
      const uint32_t tA = tbase + 128u * ((t2 >> 2) & 1) + 32u * (t2 & 3), tB = tbase + TM_B + 32u * b;
      const uint64_t dD1 = dOp + (uint64_t)(so2 * op16), dD2 = dD1 + d2_16;
      const bool lastOfBatch = (t2 & (BT - 1)) == BT - 1 || t2 == ntiles - 1;
      if (elect_one()) {
        #pragma unroll
        for (int ks = 0; ks < TL / 8; ++ks) {
          const uint32_t acc = (t2 > 0 || ks > 0) ? 1u : 0u;
          mma_tf32_ts(t_acc1, tA + 8u * ks, dD1 + 2u * ks, id_acc, acc);   // 32 bytes along K
          mma_tf32_ts(t_acc2, tB + 8u * ks, dD2 + 2u * ks, id_acc, acc);
        }
        mma_commit(&bars.abfree[b]);
        mma_commit(&bars.opempty[so2]);
        if (lastOfBatch) mma_commit(&bars.vafree[(t2 >> 2) & 1]);
      }
      __syncwarp();
      if (++so2 == nop) {
        so2 = 0;
        po2 ^= 1u;
      }
      if (j1 < nbatch && t2 == BT * (j1 - 1)) ok = mma1(j1++);
    }
    if (elect_one()) mma_commit(&bars.done);
    __syncwarp();
  } else if (warp == 3) {
    // ---------------- side job ----------------
    if (early && side) pdl_wait();                  // it reads the previous kernels' partials
    side_run(side, lane, K);
  } else if (warp >= EPI_WARP0) {
    // ---------------- epilogue ----------------
    // Two groups of 8 warps take alternate tiles (group g: tiles g, g + 2, ...;
    // TMEM B buffer g), so one group's waits overlap the other's work. Within
    // a group, warp (q4, half) owns TMEM lanes 32 q4 .. 32 q4 + 31 and
    // streamed indices 16 half .. 16 half + 15 of the tile. A replaces the
    // tile's Vt in TMEM (each thread rewrites the columns it read).
    const int ew = warp - EPI_WARP0;
    const int q4 = warp & 3;
    const int g = (ew >> 2) & 1, half = ew >> 3;
    const int mrow = 32 * q4 + lane;                          // this thread's TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
    const int64_t gm = m0 + mrow;
    const bool mvalid = gm < mLim;
    const int jb0 = 16 * half;
    const uint32_t tBg = tbase + TM_B + 32u * g + lane_off + jb0;
    if (ew < 4 && ntiles > 0) {
      // warps 4-7 move the A operand of MMA1 (row mrow, kp columns) from shared memory to TMEM
      if (__all_sync(0xffffffffu, role_wait(&bars.once, 0u, &s_abort, status))) {
        for (int k0 = 0; k0 < kp; k0 += 16) {
          const unsigned char* src = base + L.once + (k0 >> 5) * TB;
          float o[16];
          #pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 v4 = *reinterpret_cast<const float4*>(src + sw128_offset(mrow, 4 * (k0 & 31) + 16 * i));
            o[4 * i] = v4.x; o[4 * i + 1] = v4.y; o[4 * i + 2] = v4.z; o[4 * i + 3] = v4.w;
          }
          tmem_st16(tbase + TM_ONCE + lane_off + k0, o);
        }
        tmem_st_wait();
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.onceT);
      }
    }
    int sv = g;                                               // nv >= 2: tile g sits in V slot g, phase 0
    uint32_t pv = 0;
    for (int t = g; t < ntiles; t += 2) {
      const int64_t c0 = s0 + (int64_t)t * TL;
      const int nvalid = (int)((s1 - c0) < TL ? (s1 - c0) : TL);   // streamed indices of this tile inside the chunk
      const uint32_t tV = tbase + 128u * ((t >> 2) & 1) + 32u * (t & 3) + lane_off + jb0;
      // waits decided warp-wide (the warp arrives once and tcgen05.ld/st are warp-wide)
      if (!__all_sync(0xffffffffu, role_wait(&bars.tfull[(t >> 2) & 1], (uint32_t)(t >> 3) & 1u, &s_abort, status))) break;
      if (!__all_sync(0xffffffffu, role_wait(&bars.vfull[sv], pv, &s_abort, status))) break;
      fence_after_sync();
      float vt[16];
      tmem_ld16(tV, vt);
      const unsigned char* vb = base + L.v0 + sv * TB;
      float vv[16];
      if (ROW) {
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 v4 = *reinterpret_cast<const float4*>(vb + sw128_offset(mrow, 4 * jb0 + 16 * i));
          vv[4 * i] = v4.x; vv[4 * i + 1] = v4.y; vv[4 * i + 2] = v4.z; vv[4 * i + 3] = v4.w;
        }
      } else {
        const float* Vs = reinterpret_cast<const float*>(vb) + mrow;
        #pragma unroll
        for (int j = 0; j < 16; ++j) vv[j] = Vs[(jb0 + j) * MT];
      }
      tmem_ld_wait();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.vempty[sv]);
      if (t >= 2 && !__all_sync(0xffffffffu, role_wait(&bars.abfree[g], (uint32_t)((t - 2) >> 1) & 1u, &s_abort, status)))
        break;
      float tl = 0.f;
      if (mvalid && jb0 + 16 <= nvalid) {            // every entry of this thread is inside
        #pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float v = vv[j] + kappa, y = vt[j] + kappa;
          epi_terms<BK>(v, y, bm2, bp, wantLoss, tl, vv[j], vt[j]);   // A into vv, B into vt
        }
      } else {
        #pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float v = vv[j] + kappa, y = vt[j] + kappa;
          vv[j] = 0.f;
          vt[j] = 0.f;
          if (mvalid && jb0 + j < nvalid) {
            epi_terms<BK>(v, y, bm2, bp, wantLoss, tl, vv[j], vt[j]);
          }
        }
      }
      // A and B go to the tensor core unrounded: kind::tf32 ignores the 13 low
      // mantissa bits (measured: bit-identical to truncated inputs). The
      // truncation lowers numerator and denominator terms alike (by < 2^-10
      // relative, ~2^-11 on average), so their ratio keeps far less; the
      // factor copies, made once per iteration, are rounded to nearest.
      tmem_st16(tV, vv);                               // A over this tile's Vt
      tmem_st16(tBg, vt);
      if (wantLoss) ff_add(lossHi, lossLo, tl);
      tmem_st_wait();
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.abready[g]);
      sv += 2;
      if (sv >= nv) {
        sv -= nv;
        pv ^= 1u;
      }
    }
  }

  // ---------------- accumulators: cluster tree, then one partial slice ----------------
  if (early) pdl_wait();                              // (long since satisfied: the producer waited)
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
    // Two exchange buffers of kp KB, alternating by round, over the rings
    // (idle once the block's MMAs have completed: the first barrier below).
    // Layout [float4 q][lane m] keeps the stores conflict-free.
    cluster_sync();
    int round = 0;
    for (int stp = 1; stp < csize; stp <<= 1, ++round) {
      unsigned char* buf = base + L.fa0 + ((round & 1) ? 1024u * kp : 0u);
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
    float* stg = reinterpret_cast<float*>(base + L.fa0);   // rings idle: MMAs done, exchange over
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
      float* outP = P.rowPart + (int64_t)geo.outSlice * 2 * P.F * K + m0 * K;
      float* outQ = outP + P.F * K;
      for (int r = warp; r < nrows; r += WS_THREADS / 32)     // a warp per row, lanes along the row
        for (int c = lane; c < K; c += 32) {
          outP[r * K + c] = stg[r * Ks + c];
          outQ[r * K + c] = stg[MT * Ks + r * Ks + c];
        }
    }
  } else if (epi && sl % csize == 0) {
    const int64_t gm = m0 + mrow;
    if (gm < mLim) {
      const int64_t KN = (int64_t)K * P.N;
      float* part = P.colPart + (int64_t)geo.outSlice * 2 * KN + (isQ ? KN : 0) + (int64_t)col0 * P.N + gm;
      #pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < per && col0 + j < K) part[(int64_t)j * P.N] = acc[j];
    }
  }
  double unitLoss = 0.0;
  if (wantLoss) unitLoss = block_sum_ff(lossHi, lossLo, reinterpret_cast<float2*>(red));
  fence_before_sync();
  __syncthreads();
  if (s_abort) mbar_wait(&bars.done, 0u, 100000000ull);
  // reuse: invalidate the barriers so that the next unit of a persistent
  // block may initialise them again (mbarrier.init over a valid barrier is
  // not allowed). Every MMA has completed (done) and every copy was consumed,
  // so nothing is pending on them (a unit that gave up is the exception; it
  // has already set the status word).
  if (reuse && tid == 0) {
    for (int s = 0; s < nop; ++s) {
      mbar_inval(&bars.opfull[s]);
      mbar_inval(&bars.opempty[s]);
    }
    for (int s = 0; s < nv; ++s) {
      mbar_inval(&bars.vfull[s]);
      mbar_inval(&bars.vempty[s]);
    }
    for (int b = 0; b < NFA; ++b) {
      mbar_inval(&bars.fafull[b]);
      mbar_inval(&bars.fafree[b]);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_inval(&bars.tfull[b]);
      mbar_inval(&bars.vafree[b]);
      mbar_inval(&bars.abready[b]);
      mbar_inval(&bars.abfree[b]);
    }
    mbar_inval(&bars.once);
    mbar_inval(&bars.onceT);
    mbar_inval(&bars.done);
  }
  if (reuse) __syncthreads();
  return unitLoss;
}

// One launch, one unit per block.
template <int BK, bool CHI, bool ROW>
__global__ void __launch_bounds__(WS_THREADS, 1)
tc_ws_kernel(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmOnce,
             const __grid_constant__ CUtensorMap tmFa, const __grid_constant__ CUtensorMap tmD1,
             const __grid_constant__ CUtensorMap tmD2, int useTma, int nop, int nv, Prob<float> P, int flags,
             BetaParams bp, double* __restrict__ lossPart, int* __restrict__ status, SideJob side) {
  pdl_trigger();
  extern __shared__ unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  __shared__ double red[32];
  __shared__ int s_skip;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5;
  const UnitGeom geo = uniform_geom<ROW>(P, blockIdx.x);
  const int vPre = useTma ? min(nv, ws_tiles(P, ROW, geo)) : 0;
  // Everything up to the dependency wait overlaps the previous kernel's
  // tail: TMEM allocation, barrier initialisation, the tensor maps' fetch
  // and the first V tiles (V is read-only for the whole step).
  if (warp == 2) tmem_alloc(&tslot, TM_COLS);
  if (threadIdx.x == 0) {
    prefetch_tmap(&tmV);
    prefetch_tmap(&tmOnce);
    prefetch_tmap(&tmFa);
    prefetch_tmap(&tmD1);
    prefetch_tmap(&tmD2);
    ws_init_bars(bars, nop, nv, useTma);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1 && vPre > 0)
    ws_v_issue<ROW>(tmV, P, geo, vPre, base + ws_layout((P.K + 15) & ~15, CHI, nop, nv).v0, bars);
  // from here on the previous kernel's writes (the factor copies, the status
  // word) are visible; the status is read once for the whole block. Early
  // sweeps read it without waiting (a status the previous kernel sets stops
  // the kernels after this one) and wait where they need its data.
  if (!(flags & SWEEP_EARLY)) pdl_wait();
  if (threadIdx.x == 0) s_skip = *status != 0;
  __syncthreads();
  const bool skip = s_skip != 0;    // the block still runs to the end (cluster barriers)
  SideJob sj = side;
  sj.normK = side.normPart ? (int)blockIdx.x : -1;
  sj.normStride = gridDim.x;
  sj.nloss = blockIdx.x == 0 ? side.nloss : 0;
  const bool hasSide = sj.normK >= 0 || sj.nloss > 0;
  const double l = ws_unit<BK, CHI, ROW>(tmV, tmOnce, tmFa, tmD1, tmD2, useTma, nop, nv, P, flags, bp, status, geo,
                                         skip, base, tslot, bars, s_abort, red, hasSide ? &sj : nullptr, false, true,
                                         vPre);
  if ((flags & SWEEP_LOSS) && threadIdx.x == 0) lossPart[blockIdx.x] = l;
  if ((threadIdx.x >> 5) == 2) tmem_dealloc(tslot, TM_COLS);
}

// Stream-K column sweep: block g runs its range of tile steps as one unit per
// column tile it touches (see sk_block_of); the objective partial of the
// block is the sum of its units'.
template <int BK, bool CHI>
__global__ void __launch_bounds__(WS_THREADS, 1)
tc_ws_sk_kernel(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmOnce,
                const __grid_constant__ CUtensorMap tmFa, const __grid_constant__ CUtensorMap tmD1,
                const __grid_constant__ CUtensorMap tmD2, int useTma, int nop, int nv, Prob<float> P, int flags,
                BetaParams bp, double* __restrict__ lossPart, int* __restrict__ status, SideJob side) {
  pdl_trigger();
  extern __shared__ unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  __shared__ double red[32];
  __shared__ int s_skip;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5;
  const int64_t ft = (P.F + 31) / 32, T = (int64_t)P.tcColTiles * ft, G = gridDim.x;
  const int64_t a = (int64_t)blockIdx.x * T / G, b = ((int64_t)blockIdx.x + 1) * T / G;
  // unit of tile steps [st, e): the steps of column tile st / ft inside [a, b)
  auto unit_of = [&](int64_t st, int64_t* e) {
    const int64_t nt = st / ft;
    *e = (nt + 1) * ft < b ? (nt + 1) * ft : b;
    UnitGeom geo;
    geo.mt = (int)nt;
    geo.sl = 0;
    geo.outSlice = (int)(blockIdx.x - sk_block_of(nt * ft, T, G));
    geo.s0 = (st - nt * ft) * TL;
    geo.s1 = (*e - nt * ft) * TL < P.F ? (*e - nt * ft) * TL : P.F;
    return geo;
  };
  int64_t e0 = a;
  const UnitGeom geo0 = a < b ? unit_of(a, &e0) : UnitGeom();
  const int vPre = useTma && a < b ? min(nv, ws_tiles(P, false, geo0)) : 0;
  // as in tc_ws_kernel: the first unit's set-up and V tiles before the wait
  if (warp == 2) tmem_alloc(&tslot, TM_COLS);
  if (threadIdx.x == 0) {
    prefetch_tmap(&tmV);
    prefetch_tmap(&tmOnce);
    prefetch_tmap(&tmFa);
    prefetch_tmap(&tmD1);
    prefetch_tmap(&tmD2);
    ws_init_bars(bars, nop, nv, useTma);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1 && vPre > 0)
    ws_v_issue<false>(tmV, P, geo0, vPre, base + ws_layout((P.K + 15) & ~15, CHI, nop, nv).v0, bars);
  if (!(flags & SWEEP_EARLY)) pdl_wait();               // as in tc_ws_kernel
  if (threadIdx.x == 0) s_skip = *status != 0;
  __syncthreads();
  const bool skip = s_skip != 0;
  SideJob sj = side;
  sj.normK = side.normPart ? (int)blockIdx.x : -1;
  sj.normStride = gridDim.x;
  sj.nloss = blockIdx.x == 0 ? side.nloss : 0;
  const SideJob* sp = (sj.normK >= 0 || sj.nloss > 0) ? &sj : nullptr;
  if (a >= b && warp == 3) {                       // no unit: run the side job directly
    if (flags & SWEEP_EARLY) pdl_wait();
    side_run(sp, threadIdx.x & 31, P.K);
  }
  double l = 0.0;
  bool first = true;
  for (int64_t st = a; st < b;) {
    int64_t e = e0;
    const UnitGeom geo = first ? geo0 : unit_of(st, &e);
    l += ws_unit<BK, CHI, false>(tmV, tmOnce, tmFa, tmD1, tmD2, useTma, nop, nv, P, flags, bp, status, geo, skip, base,
                                 tslot, bars, s_abort, red, sp, e < b, first, first ? vPre : 0);
    sp = nullptr;                                    // with the block's first unit only
    first = false;
    st = e;
  }
  if ((flags & SWEEP_LOSS) && threadIdx.x == 0) lossPart[blockIdx.x] = l;
  if ((threadIdx.x >> 5) == 2) tmem_dealloc(tslot, TM_COLS);
}

}  // namespace
}  // namespace nmf
