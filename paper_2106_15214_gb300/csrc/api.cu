// api.cu -- the C ABI declared in include/nmf.h: contexts, scratch planning,
// and the drivers that compose the sweep kernels into Algorithm 1 (BMM) and
// Algorithm 2 (JMM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "nmf.h"

using namespace nmf;

struct nmf_ctx {
  bool batched = false;
  int count = 1;
  std::vector<int64_t> F, N;
  std::vector<int> K;
  double beta = 1.0;
  nmf_precision prec = NMF_FP32;
  nmf_order order = NMF_W_FIRST;
  int normalize = 1;
  double kappa = 0.0;
  double floorEps = -1.0;          // < 0: the precision's default (floor_of)
  // The operand copies (tilde and TF32 copies) of the current W, H were made
  // by the last kernel of the previous step (W first, tensor cores): the next
  // step skips its copies kernel. Cleared by every call that may change W, H.
  bool copiesValid = false;
  int deterministic = 1;
  cudaStream_t stream = nullptr;
  int L = 1;
  // single-problem data
  const void* V = nullptr;
  int64_t ldv = 0;
  void* W = nullptr;
  void* H = nullptr;
  // batched packed data
  const void* Vp = nullptr;
  void* Wp = nullptr;
  void* Hp = nullptr;
  // sparse data
  bool sparse = false;
  int64_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const float* val = nullptr;
  bool cscBuilt = false;
  // device state
  bool prepared = false;
  bool tableDirty = true;
  std::vector<void*> allocs;
  Plan<float> pf;
  Plan<double> pd;
  std::vector<Prob<float>> hpf;
  std::vector<Prob<double>> hpd;
  int* d_status = nullptr;
  double* d_lossPart = nullptr;
  double* d_lossOut = nullptr;
  double* h_pinned = nullptr;  // count losses + status + kkt
  int lossPrefix = 0;          // 0: row-sweep blocks, 1: column-sweep blocks
  bool lossValid = false;
  std::vector<double> lastLosses;
  void* tildeW = nullptr;      // packed W at the start of the iteration
  void* tildeH = nullptr;
  size_t elemsW = 0, elemsH = 0, elemsV = 0;
  void* d_gW = nullptr;
  void* d_gH = nullptr;
  double* d_kkt = nullptr;
  void* stageV = nullptr;
  void* stageW = nullptr;
  void* stageH = nullptr;
  SparseKL sp;
  Timer timer;
  TcMaps tcmaps;
  double* d_normPart = nullptr;   // fused normalisation: [W epilogue blocks][K]
  unsigned* d_counter = nullptr;  // completion counter of the fused epilogues
  bool lossFused = false;
  void* Vpad = nullptr;           // row-padded copy of V (tensor-core contexts, unaligned rows)
  // batched NMF_BF16: the fused sweep's work items, tables and tensor maps
  struct FuBatchState {
    bool ok = false;
    int c = 1, nitems = 0, layK = 32, totHc = 0;
    int4* d_items = nullptr;       // launch order (longest first)
    int* d_lossBase = nullptr;     // per launched item: its first objective partial
    int* d_prefLoss = nullptr;     // per problem: first objective partial (count + 1 entries)
    int* d_prefHc = nullptr;       // per problem: first 32-column block of the copies kernel
    CUtensorMap* d_maps = nullptr; // 3 per problem
    std::vector<int64_t> padOff;   // per problem: offset of its V in the padded copy (empty: no copy)
  } fb;
  const void* vpadSrc = nullptr;
  bool vDirty = true;
  // CUDA graphs of step calls (see capture_step)
  struct GraphEntry {
    uint64_t key = 0;
    cudaGraphExec_t exec = nullptr;
    Timer::Sink sink;
    const void* ptrs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // data captured with
    bool copiesAfter = false;      // copiesValid after the captured step
  };
  std::vector<GraphEntry> graphs;
  std::vector<uint64_t> seenKeys;
  bool useGraphs = true;
  cudaStream_t gs = nullptr;
  cudaEvent_t evIn = nullptr, evOut = nullptr;
  int sms = 148;
  int chunkCap = 64;               // SIMT sweeps: most 64- or 32-wide tiles per chunk (nmf_autotune)
  // nmf_set_barrier_test: bound of the persistent kernels' barrier waits and
  // arrivals they expect beyond the launched blocks
  uint64_t waitLimitNs = 1000000000ull;
  unsigned extraArrivals = 0;
};

namespace {

size_t esize(const nmf_ctx* c) { return c->prec == NMF_FP64 ? 8 : 4; }

nmf_status cu(cudaError_t e) { return e == cudaSuccess ? NMF_OK : NMF_ECUDA; }

#define NMF_TRY(x)                     \
  do {                                 \
    nmf_status _s = (x);               \
    if (_s != NMF_OK) return _s;       \
  } while (0)
#define NMF_CU(x) NMF_TRY(cu(x))

void invalidate_graphs(nmf_ctx* c);

void free_all(nmf_ctx* c) {
  invalidate_graphs(c);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  c->h_pinned = nullptr;
  c->prepared = false;
  c->tableDirty = true;
  c->cscBuilt = false;
  c->d_gW = c->d_gH = nullptr;
  c->d_kkt = nullptr;
  c->stageV = c->stageW = c->stageH = nullptr;
  // every device pointer of the context went with the allocations: calls
  // before the next prepare() (nmf_set_factors clears the status word when
  // there is one) must not reach freed memory
  c->d_status = nullptr;
  c->d_lossPart = c->d_lossOut = nullptr;
  c->tildeW = c->tildeH = nullptr;
  c->d_normPart = nullptr;
  c->d_counter = nullptr;
  c->sp = SparseKL();
  // the padded copy of V went with the other allocations: the next upload
  // allocates and fills it again
  c->Vpad = nullptr;
  c->vpadSrc = nullptr;
  c->vDirty = true;
  c->fb = nmf_ctx::FuBatchState();
}

nmf_status dalloc(nmf_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NMF_ENOMEM;
  }
  c->allocs.push_back(*p);
  return NMF_OK;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Batched fused sweep: 128-column batches per work item for a chunk cap (the
// autotuned parameter of batched contexts, 8 ... 128): 2 ... 32.
int fu_batches(int cap) { return std::max(1, cap / 4); }

struct Tiling {
  int rowTilesF, S, colTilesN, R;
  int64_t chunkN, chunkF;
};

// Splits of the two sweeps: enough blocks to fill the GPU twice over for a
// single problem; for batches, chunks capped (at `cap` tiles, 64 unless
// nmf_autotune chose another) so no block walks a whole long row or column of
// a big member while small members finish early.
Tiling tiling(int64_t F, int64_t N, int sms, bool batched, int cap) {
  Tiling t;
  t.rowTilesF = (int)cdiv(F, BF);
  t.colTilesN = (int)cdiv(N, BN);
  const int64_t nTiles = cdiv(N, BN), fTiles = cdiv(F, BF);
  const int64_t target = 2LL * sms;
  int64_t S = batched ? 1 : std::max<int64_t>(1, cdiv(target, t.rowTilesF));
  S = std::max<int64_t>(S, cdiv(nTiles, cap));
  S = std::min<int64_t>(S, nTiles);
  t.chunkN = cdiv(nTiles, S) * BN;
  t.S = (int)cdiv(N, t.chunkN);
  int64_t R = batched ? 1 : std::max<int64_t>(1, cdiv(target, t.colTilesN));
  R = std::max<int64_t>(R, cdiv(fTiles, cap));
  R = std::min<int64_t>(R, fTiles);
  t.chunkF = cdiv(fTiles, R) * BF;
  t.R = (int)cdiv(F, t.chunkF);
  return t;
}

bool data_ready(const nmf_ctx* c) {
  if (c->batched) return c->Vp && c->Wp && c->Hp;
  if (c->sparse) return c->rowptr && c->W && c->H;
  return c->V && c->W && c->H;
}

// Tensor-core sweeps: 128-row (row sweep) or 128-column (column sweep) MMA
// tiles, split along the streamed dimension into chunks of 32-wide tiles.
// The split minimises an estimate of the sweep's time in tile units: waves of
// one block per SM times (tiles per block + a fixed per-block cost of two
// tiles for set-up and the partial-sum write). NMF_TC_TARGET=<blocks> forces
// about that many blocks instead (for tuning).
int64_t best_split(int64_t fixedTiles, int64_t streamTiles, int sms) {
  const char* env = std::getenv("NMF_TC_TARGET");
  if (env && std::atoi(env) > 0) {
    const int64_t target = std::atoi(env);
    return std::min<int64_t>(std::max<int64_t>(1, cdiv(target, fixedTiles)), streamTiles);
  }
  int64_t best = 1;
  double bestCost = 1e300;
  for (int64_t S = 1; S <= std::min<int64_t>(streamTiles, 64); ++S) {
    const double waves = (double)cdiv(fixedTiles * S, sms);
    const double cost = waves * ((double)cdiv(streamTiles, S) + 2.0);
    if (cost < bestCost - 1e-9) { bestCost = cost; best = S; }
  }
  return best;
}

// Tiling of one tensor-core sweep: `fixedTiles` 128-wide tiles, `streamLen`
// streamed indices (32 per tile step). NMF_TC_CLUSTER=<c> (2, 4 or 8) makes
// the blocks of one tile form clusters of c whose partial sums are added
// through distributed shared memory, so the sweep writes split / c slices
// (the split sized for the blocks resident in clusters of c). Off by default:
// on the 361 x 2429 and 513 x 20000 workloads the tree and the cluster
// scheduling cost the sweep more than the shorter slice sums save.
void tc_split(int64_t fixedTiles, int64_t streamLen, int kp, int sms, int64_t& chunk, int& split, int& cluster,
              int& slices) {
  const int64_t streamTiles = cdiv(streamLen, 32);
  const char* env = std::getenv("NMF_TC_CLUSTER");
  const int forced = env ? std::atoi(env) : 0;
  cluster = 1;
  int64_t S = best_split(fixedTiles, streamTiles, sms);
  if (kp <= 64 && (forced == 2 || forced == 4 || forced == 8)) {
    const int cap = tc_ws_capacity(kp, forced);
    if (cap >= forced) {
      cluster = forced;
      S = best_split(fixedTiles, streamTiles, cap);
    }
  }
  chunk = cdiv(streamTiles, S) * 32;
  const int64_t sp = cdiv(streamLen, chunk);
  split = (int)(cdiv(sp, cluster) * cluster);
  slices = split / cluster;
}

void tc_tiling(Prob<float>& P, int sms) {
  const int kp = (P.K + 15) & ~15;
  P.tcRowTiles = (int)cdiv(P.F, 128);
  tc_split(P.tcRowTiles, P.N, kp, sms, P.tcChunkN, P.tcSplitS, P.tcClusterS, P.tcS);
  P.tcColTiles = (int)cdiv(P.N, 128);
  tc_split(P.tcColTiles, P.F, kp, sms, P.tcChunkF, P.tcSplitR, P.tcClusterR, P.tcR);
  // Column sweep over more than one wave of blocks (e.g. 157 column tiles on
  // 152 SMs): split its tile steps stream-K over one wave instead
  // (warp-specialised kernel only; NMF_TC_SK=0 keeps the uniform split).
  P.tcSK = 0;
  P.tcSKBlocks = 0;
  const char* skEnv = std::getenv("NMF_TC_SK");
  const bool skOn = !(skEnv && skEnv[0] == '0');
  const int64_t units = (int64_t)P.tcColTiles * P.tcSplitR;
  if (skOn && kp <= 64 && P.tcClusterR == 1 && units > sms) {
    const int64_t ft = cdiv(P.F, 32), T = (int64_t)P.tcColTiles * ft;
    const int64_t G = std::min<int64_t>(sms, T);
    int most = 1;
    for (int64_t nt = 0; nt < P.tcColTiles; ++nt) most = std::max(most, sk_slices(nt, ft, T, G));
    P.tcSK = 1;
    P.tcSKBlocks = (int)G;
    P.tcR = most;
  }
  if (std::getenv("NMF_TC_DEBUG"))
    std::fprintf(stderr, "nmf tc capacity (blocks resident) cluster 1/2/4/8: %d %d %d %d (sms %d)\n",
                 tc_ws_capacity(kp, 1), tc_ws_capacity(kp, 2), tc_ws_capacity(kp, 4), tc_ws_capacity(kp, 8), sms);
  if (std::getenv("NMF_TC_DEBUG"))
    std::fprintf(stderr, "nmf tc tiling F=%lld N=%lld K=%d: row %d tiles x %d blocks (cluster %d, %d slices, chunk %lld); "
                 "col %d tiles x %d blocks (cluster %d, %d slices, chunk %lld, stream-K %d blocks)\n",
                 (long long)P.F, (long long)P.N, P.K, P.tcRowTiles, P.tcSplitS, P.tcClusterS, P.tcS,
                 (long long)P.tcChunkN, P.tcColTiles, P.tcSplitR, P.tcClusterR, P.tcR, (long long)P.tcChunkF,
                 P.tcSK ? P.tcSKBlocks : 0);
}
template <typename T> void tc_tiling(Prob<T>&, int) {}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T>
nmf_status build_plan(nmf_ctx* c, Plan<T>& pl, std::vector<Prob<T>>& probs) {
  const int cnt = c->count;
  probs.assign(cnt, Prob<T>());
  std::vector<int> pr(cnt + 1), pc(cnt + 1), pw(cnt + 1), ph(cnt + 1), pk(cnt + 1);
  pr[0] = pc[0] = pw[0] = ph[0] = pk[0] = 0;
  // scratch bytes per problem (excluding the packed tilde buffers)
  std::vector<size_t> off(cnt + 1, 0);
  std::vector<Tiling> tl(cnt);
  int maxK = 0;
  for (int i = 0; i < cnt; ++i) {
    const int64_t F = c->F[i], N = c->N[i];
    const int K = c->K[i];
    maxK = std::max(maxK, K);
    tl[i] = tiling(F, N, c->sms, c->batched, c->chunkCap);
    probs[i].F = F; probs[i].N = N; probs[i].K = K;
    probs[i].tcS = probs[i].tcR = 1;
    probs[i].tcSplitS = probs[i].tcSplitR = 1;
    probs[i].tcClusterS = probs[i].tcClusterR = 1;
    probs[i].tcSK = probs[i].tcSKBlocks = 0;
    if (!c->batched) tc_tiling(probs[i], c->sms);
    probs[i].fuS = 1;
    if constexpr (std::is_same<T, float>::value) {
      if (!c->batched && c->prec == NMF_BF16 && K <= 32 && F <= 1024) {
        probs[i].kp = (K + 15) & ~15;
        probs[i].fuS = std::max(1, tc_fused_clusters(probs[i], c->sms));
      }
      // batched: items of fu_batches(chunkCap) 128-column batches, one slice each
      if (c->batched && c->prec == NMF_BF16)
        probs[i].fuS = (int)cdiv(cdiv(N, 128), (int64_t)fu_batches(c->chunkCap));
    }
    const int Smax = std::max({tl[i].S, probs[i].tcS, probs[i].fuS}), Rmax = std::max(tl[i].R, probs[i].tcR);
    const size_t FK = (size_t)F * K, KN = (size_t)K * N;
    size_t bytes = 0;
    bytes += align256(sizeof(T) * FK) * 2;                         // chiW1, chiW2
    bytes += align256(sizeof(T) * KN) * 2;                         // chiH1, chiH2
    bytes += align256(sizeof(T) * FK * 2 * Smax);                  // rowPart
    bytes += align256(sizeof(T) * KN * 2 * Rmax);                  // colPart
    bytes += align256(sizeof(T) * K);                              // norms
    off[i + 1] = off[i] + bytes;
    pr[i + 1] = pr[i] + tl[i].rowTilesF * tl[i].S;
    pc[i + 1] = pc[i] + tl[i].colTilesN * tl[i].R;
    pw[i + 1] = pw[i] + (int)cdiv((int64_t)FK, EW);
    ph[i + 1] = ph[i] + (int)cdiv((int64_t)KN, EW);
    pk[i + 1] = pk[i] + K;
  }
  void* scratch = nullptr;
  NMF_TRY(dalloc(c, &scratch, off[cnt]));
  NMF_TRY(dalloc(c, &c->tildeW, sizeof(T) * c->elemsW));
  NMF_TRY(dalloc(c, &c->tildeH, sizeof(T) * c->elemsH));
  size_t oW = 0, oH = 0, oV = 0;
  for (int i = 0; i < cnt; ++i) {
    Prob<T>& P = probs[i];
    const int64_t F = c->F[i], N = c->N[i];
    const int K = c->K[i];
    const size_t FK = (size_t)F * K, KN = (size_t)K * N;
    char* base = static_cast<char*>(scratch) + off[i];
    auto take = [&](size_t bytes) { T* p = reinterpret_cast<T*>(base); base += align256(bytes); return p; };
    P.chiW1 = take(sizeof(T) * FK);
    P.chiW2 = take(sizeof(T) * FK);
    P.chiH1 = take(sizeof(T) * KN);
    P.chiH2 = take(sizeof(T) * KN);
    P.rowPart = take(sizeof(T) * FK * 2 * std::max({tl[i].S, P.tcS, P.fuS}));
    P.colPart = take(sizeof(T) * KN * 2 * std::max(tl[i].R, P.tcR));
    P.norms = take(sizeof(T) * K);
    P.Wt = static_cast<T*>(c->tildeW) + oW;
    P.Ht = static_cast<T*>(c->tildeH) + oH;
    P.S = tl[i].S; P.R = tl[i].R;
    P.rowTilesF = tl[i].rowTilesF; P.colTilesN = tl[i].colTilesN;
    P.chunkN = tl[i].chunkN; P.chunkF = tl[i].chunkF;
    P.V = nullptr; P.W = nullptr; P.H = nullptr;
    P.ldv = c->batched ? N : c->ldv;
    oW += FK; oH += KN; oV += (size_t)F * N;
  }
  // TF32 operand shadows for the tensor-core sweeps (single float problems)
  if (!c->batched && sizeof(T) == 4 && (c->prec == NMF_TF32 || c->prec == NMF_BF16)) {
    Prob<T>& P = probs[0];
    P.kp = (P.K + 15) & ~15;
    P.ks = (P.kp + 31) & ~31;
    P.Fp = (P.F + 3) & ~int64_t(3);
    P.Np = (P.N + 3) & ~int64_t(3);
    const size_t nWS = (size_t)P.F * P.ks, nT = (size_t)P.kp * P.Fp, nHT = (size_t)P.N * P.ks, nH = (size_t)P.kp * P.Np;
    const size_t parts[8] = {nWS, nT, nHT, nH, nT, nT, nH, nH};
    size_t total = 0;
    for (size_t q : parts) total += align256(sizeof(T) * q);
    void* sh = nullptr;
    NMF_TRY(dalloc(c, &sh, total));
    NMF_CU(cudaMemset(sh, 0, total));
    T* ptrs[8];
    char* cur = static_cast<char*>(sh);
    for (int q = 0; q < 8; ++q) { ptrs[q] = reinterpret_cast<T*>(cur); cur += align256(sizeof(T) * parts[q]); }
    P.sWS = ptrs[0]; P.sWT = ptrs[1]; P.sHT = ptrs[2]; P.sHS = ptrs[3];
    P.sCW1 = ptrs[4]; P.sCW2 = ptrs[5]; P.sCH1 = ptrs[6]; P.sCH2 = ptrs[7];
  }
  // batched NMF_BF16: per-problem TF32 shadows (sWS, sHT) and the fused
  // sweep's work items (problem order for slices and objective partials,
  // launched longest first)
  if constexpr (std::is_same<T, float>::value) {
    c->fb = nmf_ctx::FuBatchState();
    if (c->batched && c->prec == NMF_BF16) {
      int maxF = 0;
      bool fits = true;
      for (int i = 0; i < cnt; ++i) {
        maxF = (int)std::max<int64_t>(maxF, c->F[i]);
        fits = fits && c->K[i] <= 32;
      }
      fits = fits && maxF <= 1024 && tc_fused_batch_nv(32) >= 2;
      if (fits) {
        size_t total = 0;
        std::vector<size_t> so(cnt);
        for (int i = 0; i < cnt; ++i) {
          Prob<T>& P = probs[i];
          P.kp = (P.K + 15) & ~15;
          P.ks = 32;
          P.Fp = (P.F + 3) & ~int64_t(3);
          P.Np = (P.N + 3) & ~int64_t(3);
          so[i] = total;
          total += align256(sizeof(T) * (size_t)P.F * P.ks) + align256(sizeof(T) * (size_t)P.N * P.ks);
        }
        void* sh = nullptr;
        NMF_TRY(dalloc(c, &sh, total));
        NMF_CU(cudaMemset(sh, 0, total));
        for (int i = 0; i < cnt; ++i) {
          Prob<T>& P = probs[i];
          char* b = static_cast<char*>(sh) + so[i];
          P.sWS = reinterpret_cast<T*>(b);
          P.sHT = reinterpret_cast<T*>(b + align256(sizeof(T) * (size_t)P.F * P.ks));
        }
        const int cc = (int)cdiv(maxF, 128), B = fu_batches(c->chunkCap);
        std::vector<int4> items;
        std::vector<int> lossBase, prefLoss(cnt + 1), prefHc(cnt + 1);
        prefLoss[0] = prefHc[0] = 0;
        for (int i = 0; i < cnt; ++i) {
          const int nb = (int)cdiv(c->N[i], 128), n = probs[i].fuS;
          for (int q = 0; q < n; ++q) {
            items.push_back(make_int4(i, (int)((int64_t)nb * q / n), (int)((int64_t)nb * (q + 1) / n), q));
            lossBase.push_back(cc * (int)(items.size() - 1));
          }
          prefLoss[i + 1] = cc * (int)items.size();
          prefHc[i + 1] = prefHc[i] + (int)cdiv(c->N[i], 32);
        }
        std::vector<int> order(items.size());
        for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
          return items[a].z - items[a].y > items[b].z - items[b].y;
        });
        std::vector<int4> itemsL(items.size());
        std::vector<int> baseL(items.size());
        for (size_t q = 0; q < order.size(); ++q) { itemsL[q] = items[order[q]]; baseL[q] = lossBase[order[q]]; }
        auto& fb = c->fb;
        fb.c = cc;
        fb.nitems = (int)items.size();
        fb.layK = 32;
        fb.totHc = prefHc[cnt];
        NMF_TRY(dalloc(c, reinterpret_cast<void**>(&fb.d_items), sizeof(int4) * itemsL.size()));
        NMF_TRY(dalloc(c, reinterpret_cast<void**>(&fb.d_lossBase), sizeof(int) * baseL.size()));
        NMF_TRY(dalloc(c, reinterpret_cast<void**>(&fb.d_prefLoss), sizeof(int) * prefLoss.size()));
        NMF_TRY(dalloc(c, reinterpret_cast<void**>(&fb.d_prefHc), sizeof(int) * prefHc.size()));
        NMF_TRY(dalloc(c, reinterpret_cast<void**>(&fb.d_maps), sizeof(CUtensorMap) * 3 * (size_t)cnt));
        NMF_CU(cudaMemcpy(fb.d_items, itemsL.data(), sizeof(int4) * itemsL.size(), cudaMemcpyHostToDevice));
        NMF_CU(cudaMemcpy(fb.d_lossBase, baseL.data(), sizeof(int) * baseL.size(), cudaMemcpyHostToDevice));
        NMF_CU(cudaMemcpy(fb.d_prefLoss, prefLoss.data(), sizeof(int) * prefLoss.size(), cudaMemcpyHostToDevice));
        NMF_CU(cudaMemcpy(fb.d_prefHc, prefHc.data(), sizeof(int) * prefHc.size(), cudaMemcpyHostToDevice));
        fb.ok = true;          // until the tensor maps fail to build (upload_table)
      }
    }
  }
  void* d = nullptr;
  NMF_TRY(dalloc(c, &d, sizeof(Prob<T>) * cnt));
  pl.d_probs = static_cast<Prob<T>*>(d);
  pl.count = cnt;
  pl.maxK = maxK;
  int* tabs = nullptr;
  NMF_TRY(dalloc(c, reinterpret_cast<void**>(&tabs), sizeof(int) * (5 * (cnt + 1) + 4)));
  std::vector<int> all;
  all.insert(all.end(), pr.begin(), pr.end());
  all.insert(all.end(), pc.begin(), pc.end());
  all.insert(all.end(), pw.begin(), pw.end());
  all.insert(all.end(), ph.begin(), ph.end());
  all.insert(all.end(), pk.begin(), pk.end());
  const int tcRowGrid = probs[0].tcRowTiles * probs[0].tcSplitS;
  const int tcColGrid = probs[0].tcSK ? probs[0].tcSKBlocks : probs[0].tcColTiles * probs[0].tcSplitR;
  all.insert(all.end(), {0, c->batched ? 0 : tcRowGrid, 0, c->batched ? 0 : tcColGrid});
  NMF_CU(cudaMemcpy(tabs, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
  pl.d_prefTc = tabs + 5 * (cnt + 1);
  pl.rowSlices[0] = probs[0].S;
  pl.rowSlices[1] = probs[0].tcS;
  pl.rowSlices[2] = probs[0].fuS;
  pl.d_prefRow = tabs; pl.totRow = pr[cnt];
  pl.d_prefCol = tabs + (cnt + 1); pl.totCol = pc[cnt];
  pl.d_prefW = tabs + 2 * (cnt + 1); pl.totW = pw[cnt];
  pl.d_prefH = tabs + 3 * (cnt + 1); pl.totH = ph[cnt];
  pl.d_prefK = tabs + 4 * (cnt + 1); pl.totK = pk[cnt];
  size_t lossLen = (size_t)std::max(pl.totRow, pl.totCol);
  if constexpr (std::is_same<T, float>::value) lossLen = std::max<size_t>(lossLen, (size_t)c->fb.c * c->fb.nitems);
  if (!c->batched) lossLen = std::max<size_t>(lossLen, (size_t)std::max({tcRowGrid, tcColGrid, c->sms + 8}));
  NMF_TRY(dalloc(c, reinterpret_cast<void**>(&c->d_lossPart), sizeof(double) * lossLen));
  if (!c->batched) {
    // W-epilogue norm partials ([K][blocks]), or [K][SMs] for the persistent step kernel
    const size_t normParts = std::max<size_t>((size_t)rows_epilogue_grid(pl.totW, ROWS_EPI_MAX_LANES), (size_t)c->sms);
    NMF_TRY(dalloc(c, reinterpret_cast<void**>(&c->d_normPart), sizeof(double) * normParts * c->K[0]));
    NMF_TRY(dalloc(c, reinterpret_cast<void**>(&c->d_counter), 256));
    NMF_CU(cudaMemset(c->d_counter, 0, 256));
  }
  return NMF_OK;
}

template <typename T>
nmf_status upload_table(nmf_ctx* c, Plan<T>& pl, std::vector<Prob<T>>& probs) {
  if constexpr (std::is_same<T, float>::value) {
    auto& fb = c->fb;
    if (c->batched && fb.ok) {
      // row-padded packed copy of V when some problem's rows or base are not 16-byte aligned
      bool aligned = (reinterpret_cast<uintptr_t>(c->Vp) & 15u) == 0;
      for (int i = 0; i < c->count; ++i) aligned = aligned && (c->N[i] % 4 == 0) && ((c->F[i] * c->N[i]) % 4 == 0);
      fb.padOff.clear();
      if (!aligned) {
        int64_t tot = 0;
        for (int i = 0; i < c->count; ++i) {
          fb.padOff.push_back(tot);
          tot += c->F[i] * ((c->N[i] + 3) & ~int64_t(3));
        }
        if (!c->Vpad) NMF_TRY(dalloc(c, &c->Vpad, sizeof(float) * (size_t)tot));
        if (c->vDirty || c->vpadSrc != c->Vp) {
          int64_t oSrc = 0;
          for (int i = 0; i < c->count; ++i) {
            const int64_t Np = (c->N[i] + 3) & ~int64_t(3);
            NMF_CU(cudaMemcpy2DAsync(static_cast<float*>(c->Vpad) + fb.padOff[i], sizeof(float) * Np,
                                     static_cast<const float*>(c->Vp) + oSrc, sizeof(float) * c->N[i],
                                     sizeof(float) * c->N[i], c->F[i], cudaMemcpyDeviceToDevice, c->stream));
            oSrc += c->F[i] * c->N[i];
          }
          c->vpadSrc = c->Vp;
          c->vDirty = false;
        }
      }
    }
  }
  size_t oW = 0, oH = 0, oV = 0;
  for (int i = 0; i < c->count; ++i) {
    Prob<T>& P = probs[i];
    if (c->batched) {
      P.V = static_cast<const T*>(c->Vp) + oV;
      P.W = static_cast<T*>(c->Wp) + oW;
      P.H = static_cast<T*>(c->Hp) + oH;
      P.ldv = P.N;
      if constexpr (std::is_same<T, float>::value) {
        // the fused sweep streams V by TMA: rows and bases 16-byte aligned,
        // else a row-padded packed copy (taken when V is set)
        auto& fb = c->fb;
        if (fb.ok && !fb.padOff.empty()) {
          P.V = static_cast<const T*>(c->Vpad) + fb.padOff[i];
          P.ldv = (P.N + 3) & ~int64_t(3);
        }
      }
    } else {
      P.V = static_cast<const T*>(c->V);
      P.W = static_cast<T*>(c->W);
      P.H = static_cast<T*>(c->H);
      P.ldv = c->ldv;
      // Tensor-core sweeps stream V by TMA, which needs 16-byte aligned rows:
      // otherwise keep a row-padded copy, taken when V is set.
      const bool tcPrec = c->prec == NMF_TF32 || c->prec == NMF_BF16;
      if (tcPrec && sizeof(T) == 4 &&
          (((c->ldv * 4) & 15) != 0 || (reinterpret_cast<uintptr_t>(c->V) & 15u) != 0)) {
        const int64_t Np = (P.N + 3) & ~int64_t(3);
        if (!c->Vpad) NMF_TRY(dalloc(c, &c->Vpad, sizeof(T) * (size_t)P.F * Np));
        if (c->vDirty || c->vpadSrc != c->V) {
          NMF_CU(cudaMemcpy2DAsync(c->Vpad, sizeof(T) * Np, c->V, sizeof(T) * c->ldv, sizeof(T) * P.N, P.F,
                                   cudaMemcpyDeviceToDevice, c->stream));
          c->vpadSrc = c->V;
          c->vDirty = false;
        }
        P.V = static_cast<const T*>(c->Vpad);
        P.ldv = Np;
      }
    }
    oW += (size_t)P.F * P.K; oH += (size_t)P.K * P.N; oV += (size_t)P.F * P.N;
  }
  if constexpr (std::is_same<T, float>::value) {
    auto& fb = c->fb;
    if (c->batched && fb.ok) {
      std::vector<CUtensorMap> maps(3 * (size_t)c->count);
      for (int i = 0; i < c->count && fb.ok; ++i) fb.ok = tc_fused_maps(probs[i], &maps[3 * (size_t)i]);
      if (fb.ok)
        NMF_CU(cudaMemcpyAsync(fb.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                               c->stream));
      // a host-memory source: the copy must finish before `maps` goes away
      NMF_CU(cudaStreamSynchronize(c->stream));
    }
  }
  // 16-byte H epilogue: one float problem, N % 4 == 0 and the caller's H aligned
  pl.colVec4 = (!c->batched && c->count == 1 && sizeof(T) == 4 && c->N[0] % 4 == 0 &&
                (reinterpret_cast<uintptr_t>(c->H) & 15u) == 0) ? 1 : 0;
  NMF_CU(cudaMemcpyAsync(pl.d_probs, probs.data(), sizeof(Prob<T>) * c->count,
                         cudaMemcpyHostToDevice, c->stream));
  c->tableDirty = false;
  return NMF_OK;
}

// Allocates the context's scratch on first use (or after a precision change),
// then uploads the problem table if data pointers changed. Anything allocated
// after the first prepare() (staging, gradient scratch) survives later calls.
nmf_status prepare(nmf_ctx* c) {
  if (!c->prepared) {
    free_all(c);
    NMF_TRY(dalloc(c, reinterpret_cast<void**>(&c->d_status), sizeof(int)));
    NMF_CU(cudaMemset(c->d_status, 0, sizeof(int)));
    NMF_TRY(dalloc(c, reinterpret_cast<void**>(&c->d_lossOut), sizeof(double) * (c->count + 4)));
    if (cudaMallocHost(&c->h_pinned, sizeof(double) * (c->count + 8)) != cudaSuccess) {
      cudaGetLastError();
      c->h_pinned = nullptr;
      return NMF_ENOMEM;
    }
    if (c->sparse) {
      // sparse KL path has its own scratch (sparse_kl.cu)
      SparseKL& s = c->sp;
      s.F = c->F[0]; s.N = c->N[0]; s.K = c->K[0]; s.nnz = c->nnz;
      const int K = s.K;
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.rowidx), sizeof(int32_t) * std::max<int64_t>(1, s.nnz)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.colptr), sizeof(int32_t) * (s.N + 1)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.cscRow), sizeof(int32_t) * std::max<int64_t>(1, s.nnz)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.cscPos), sizeof(int64_t) * std::max<int64_t>(1, s.nnz)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.a), sizeof(float) * std::max<int64_t>(1, s.nnz)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.Wt), sizeof(float) * s.F * K));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.Ht), sizeof(float) * s.N * K * 2));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.colsumW), sizeof(float) * K * 4));
      s.rowsumH = s.colsumW + K;
      s.chi = s.colsumW + 2 * K;
      s.lossBlocks = (int)std::max<int64_t>(cdiv(s.F, 8), cdiv(s.N, 32));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.lossPart), sizeof(double) * (s.lossBlocks + 64)));
      NMF_TRY(dalloc(c, reinterpret_cast<void**>(&s.sums), sizeof(double) * 64));
      c->tildeW = s.Wt;
      c->tildeH = s.Ht;  // H tilde, row-major K x N (first half of the Ht buffer)
      c->prepared = true;
      return NMF_OK;
    }
    // TF32/BF16 contexts also get the float plan: their loss, gradient and
    // alternating baseline run on the FP32 SIMT kernels.
    if (c->prec == NMF_FP64) NMF_TRY(build_plan<double>(c, c->pd, c->hpd));
    else NMF_TRY(build_plan<float>(c, c->pf, c->hpf));
    c->tcmaps.ok = false;
    if (c->prec != NMF_FP64 && !c->batched && c->hpf[0].sWS) tc_build_maps(c->hpf[0], &c->tcmaps);
    c->prepared = true;
    c->tableDirty = true;
  }
  if (c->tableDirty && !c->sparse && data_ready(c)) {
    if (c->prec == NMF_FP64) NMF_TRY(upload_table<double>(c, c->pd, c->hpd));
    else NMF_TRY(upload_table<float>(c, c->pf, c->hpf));
  }
  return NMF_OK;
}


// Floor on W and H (every update is clamped to it): the one set by
// nmf_set_floor, else 0 in FP64 and 1e-30 in single precision, where
// entries that MU drives toward zero would otherwise underflow after some
// hundreds of iterations (beta < 1) and make chi's ratio X / Xt = 0 / 0.
double floor_of(const nmf_ctx* c) {
  if (c->floorEps >= 0.0) return c->floorEps;
  return c->prec == NMF_FP64 ? 0.0 : 1e-30;
}

BetaParams beta_params(const nmf_ctx* c) {
  BetaParams bp;
  bp.beta = c->beta;
  bp.gamma = gamma_of(c->beta);
  bp.kappa = c->kappa;
  bp.floor = floor_of(c);
  bp.kind = beta_kind(c->beta);
  fill_series(bp);
  return bp;
}

// One or more outer iterations of Algorithm 2 (joint) or Algorithm 1 (alternating).
// tc: the two sweeps run on the tensor-core kernels (single float problems).
template <typename T>
nmf_status run_dense(nmf_ctx* c, Plan<T>& pl, bool joint, int iters, bool wantLoss, bool tc) {
  const BetaParams bp = beta_params(c);
  cudaStream_t st = c->stream;
  int* status = c->d_status;
  double* lp = c->d_lossPart;
  const bool wfirst = c->order == NMF_W_FIRST ||
                      (c->order == NMF_ORDER_AUTO && c->F[0] >= c->N[0]);
  const int L = c->L;
  const int C = SWEEP_CONTRACT;
  // 2: tensor-core path whose sweeps read only the TF32 copies of chi
  // (warp-specialised kernels), so the epilogues skip the full-precision chi
  int tci = tc ? 1 : 0;
  if (tc && c->tcmaps.ok && c->count == 1 && c->hpf[0].kp <= 64) tci = 2;
  // single problems fold the objective's finalisation and the normalisation
  // into the epilogues (EpiFuse); batched contexts use the separate kernels
  const bool fuse = !c->batched;
  const bool norm = c->normalize != 0;
  // W first on the warp-specialised path: the iteration's last kernel also
  // makes the next iteration's copies, so that iteration (in this call or,
  // while nothing changes W and H in between, the next call) skips the copies
  // kernel. NMF_TC_FUSE_COPIES=0 keeps the separate copies kernel.
  const char* fcEnv = std::getenv("NMF_TC_FUSE_COPIES");
  const bool fuseCopies = !(fcEnv && fcEnv[0] == '0') && tci == 2 && joint && L == 1 && fuse && norm && wfirst &&
                          c->hpf[0].sWS;
  const bool copiesIn = c->copiesValid;    // the copies of the current W, H exist (see the BF16 path too)
  bool haveCopies = fuseCopies && copiesIn;
  c->copiesValid = false;
  auto row_sweep = [&](int wsel, int hsel, int dsel, int flags, const SideJob* side = nullptr) -> nmf_status {
    if constexpr (std::is_same<T, float>::value) {
      if (tc)
        return cu(timed(&c->timer, st, "tc_row_sweep", 1, [&] {
          return launch_tc_row_sweep(c->hpf[0], &c->tcmaps, wsel, hsel, dsel, flags, c->prec == NMF_BF16, bp, lp,
                                     status, st, side);
        }));
    }
    return cu(timed(&c->timer, st, "row_sweep", 1, [&] {
      return launch_row_sweep<T>(pl, wsel, hsel, dsel, flags, bp, lp, status, st);
    }));
  };
  auto col_sweep = [&](int wsel, int hsel, int csel, int flags, const SideJob* side = nullptr) -> nmf_status {
    if constexpr (std::is_same<T, float>::value) {
      if (tc)
        return cu(timed(&c->timer, st, "tc_col_sweep", 1, [&] {
          return launch_tc_col_sweep(c->hpf[0], &c->tcmaps, wsel, hsel, csel, flags, c->prec == NMF_BF16, bp, lp,
                                     status, st, side);
        }));
    }
    return cu(timed(&c->timer, st, "col_sweep", 1, [&] {
      return launch_col_sweep<T>(pl, wsel, hsel, csel, flags, bp, lp, status, st);
    }));
  };
  // tensor-core mode: TF32 shadows of the factors the next sweep reads
  auto shadows = [&](int which) -> nmf_status {
    if constexpr (std::is_same<T, float>::value) {
      if (tc && c->hpf[0].sWS)
        return cu(timed(&c->timer, st, "shadow_factors", 1, [&] {
          return launch_shadow_factors<float>(c->hpf[0], which, status, st);
        }));
    }
    return NMF_OK;
  };
  const int rowGrid = tc ? c->hpf[0].tcRowTiles * c->hpf[0].tcSplitS : pl.totRow;
  const int colGrid = tc ? (c->hpf[0].tcSK ? c->hpf[0].tcSKBlocks : c->hpf[0].tcColTiles * c->hpf[0].tcSplitR)
                       : pl.totCol;
  auto fz_for = [&](int flags, bool lossFromRow) {
    EpiFuse f;
    if (!fuse) return f;
    f.flags = flags;
    f.lossPart = lp;
    f.lossBlocks = lossFromRow ? rowGrid : colGrid;
    f.lossOut = c->d_lossOut;
    f.normPart = static_cast<void*>(c->d_normPart);
    f.counter = c->d_counter;
    return f;
  };
  auto rows_epi = [&](int basesel, int chi, int flags) -> nmf_status {
    const EpiFuse f = fz_for(flags, true);
    NMF_TRY(cu(timed(&c->timer, st, "rows_epilogue", 1, [&] {
      return launch_rows_epilogue<T>(pl, EPI_UPDATE, basesel, chi, bp, nullptr, status, st, tci, f);
    })));
    return basesel == SEL_CUR ? shadows(1) : NMF_OK;   // alternating: the new W feeds the next sweep
  };
  auto cols_epi = [&](int basesel, int chi, int flags) -> nmf_status {
    const EpiFuse f = fz_for(flags, false);
    NMF_TRY(cu(timed(&c->timer, st, "cols_epilogue", 1, [&] {
      return launch_cols_epilogue<T>(pl, EPI_UPDATE, basesel, chi, bp, nullptr, status, st, tci, f);
    })));
    return basesel == SEL_CUR ? shadows(2) : NMF_OK;
  };
  // NMF_TC_STEP=1: one persistent cooperative launch per iteration
  // (tc_step.cu) where it applies. Off by default: on the 361 x 2429 and
  // 513 x 20000 workloads it measured slower than the per-kernel sequence
  // below with programmatic dependent launch (the sweeps' pipeline fill no
  // longer overlaps the previous phase, and the cooperative launch costs more).
  if constexpr (std::is_same<T, float>::value) {
    const char* stepEnv = std::getenv("NMF_TC_STEP");
    const bool stepOn = stepEnv && stepEnv[0] == '1';
    if (tc && c->prec == NMF_TF32 && stepOn && joint && L == 1 && norm && fuse && c->count == 1 &&
        tc_step_supported(c->hpf[0], c->tcmaps, c->sms)) {
      for (int it = 0; it < iters; ++it) {
        TcStepArgs a;
        a.wfirst = wfirst;
        a.wantLoss = wantLoss && it == iters - 1;
        a.lossPart = lp;
        a.lossOut = c->d_lossOut;
        a.normPart = reinterpret_cast<float*>(c->d_normPart);
        a.gridBar = c->d_counter + 16;
        a.status = status;
        a.extraArrivals = c->extraArrivals;
        a.waitLimitNs = c->waitLimitNs;
        // both barrier words start at zero: a launch whose barrier wait timed
        // out leaves its arrivals count behind
        NMF_CU(cudaMemsetAsync(a.gridBar, 0, 2 * sizeof(unsigned), st));
        NMF_CU(timed(&c->timer, st, "tc_step", 1,
                     [&] { return launch_tc_step(c->hpf[0], c->tcmaps, bp, a, c->sms, st); }));
      }
      c->lossFused = true;
      return NMF_OK;
    }
  }
  // NMF_BF16: the fused single-read H-first iteration (tc_fused.cu): the
  // fused sweep (product, A, B, objective, H update, both contractions; H
  // written) | the W update from its partial slices with the column-norm
  // partials | the norms, the normalisation, the next iteration's copies of
  // W~, H~ and the objective. The copies of the first iteration come from
  // the previous call's last kernel while nothing changed W and H in between
  // (copiesValid), else from the copies kernel.
  if constexpr (std::is_same<T, float>::value) {
    if (c->prec == NMF_BF16 && c->batched) {
      // many problems: every iteration's copies of all W~, H~ | the fused
      // sweep over every problem's work items (one launch) | the W updates
      // from each problem's slices | normalisation; the objectives per problem
      // from the fused sweep's partials
      auto& fb = c->fb;
      FuBatch b;
      b.c = fb.c;
      b.nitems = fb.nitems;
      b.layK = fb.layK;
      b.items = fb.d_items;
      b.probs = pl.d_probs;
      b.maps = fb.d_maps;
      b.lossBase = fb.d_lossBase;
      b.lossPart = lp;
      for (int it = 0; it < iters; ++it) {
        NMF_CU(timed(&c->timer, st, "begin_iteration", 1,
                     [&] { return launch_fused_batch_copies(pl, fb.d_prefHc, fb.totHc, status, st); }));
        NMF_CU(timed(&c->timer, st, "tc_fused", 1,
                     [&] { return launch_tc_fused_batch(b, bp, status, c->waitLimitNs, c->extraArrivals, st); }));
        NMF_CU(timed(&c->timer, st, "rows_epilogue", 1, [&] {
          return launch_rows_epilogue<T>(pl, EPI_UPDATE, SEL_TILDE, 0, bp, nullptr, status, st, 3, EpiFuse());
        }));
        if (norm) NMF_CU(timed(&c->timer, st, "normalize", 2, [&] { return launch_normalize<T>(pl, status, st); }));
      }
      if (wantLoss)
        NMF_CU(timed(&c->timer, st, "loss_finalize", 1,
                     [&] { return launch_loss_finalize(fb.d_prefLoss, c->count, lp, c->d_lossOut, st); }));
      c->lossFused = true;
      c->copiesValid = false;
      return NMF_OK;
    }
    if (c->prec == NMF_BF16) {
      const Prob<float>& P0 = c->hpf[0];
      const int ncl = P0.fuS, cgrid = tc_fused_cluster_blocks(P0) * ncl;
      const bool haveCopies = copiesIn;
      // the W half and the normalisation over every SM, the second launch
      // started early (NMF_FU_POST=0: the W epilogue kernel with its
      // last-block finalisation, then the normalisation with the next copies)
      const char* postEnvS = std::getenv("NMF_FU_POST");
      const bool postOne = !(postEnvS && std::atoi(postEnvS) == 0);
      for (int it = 0; it < iters; ++it) {
        const bool lossHere = wantLoss && it == iters - 1;
        if (it == 0 && !haveCopies)
          NMF_CU(timed(&c->timer, st, "begin_iteration", 1,
                       [&] { return launch_tc_copies<float>(P0, true, true, true, status, st); }));
        NMF_CU(timed(&c->timer, st, "tc_fused", 1, [&] {
          return launch_tc_fused(P0, c->tcmaps, bp, ncl, lp, status, c->waitLimitNs, c->extraArrivals, st);
        }));
        if (postOne) {
          NMF_CU(timed(&c->timer, st, "fused_post", 2, [&] {
            return launch_fused_post(P0, bp, ncl, norm, reinterpret_cast<float*>(c->d_normPart), c->sms, lp, cgrid,
                                     lossHere ? c->d_lossOut : nullptr, status, st);
          }));
          continue;
        }
        EpiFuse f;
        f.flags = (lossHere ? FUSE_LOSS : 0) | (norm ? FUSE_NORM_PART : 0);
        f.lossPart = lp;
        f.lossBlocks = cgrid;
        f.lossOut = c->d_lossOut;
        f.normPart = static_cast<void*>(c->d_normPart);
        f.counter = c->d_counter;
        NMF_CU(timed(&c->timer, st, "rows_epilogue", 1, [&] {
          return launch_rows_epilogue<T>(pl, EPI_UPDATE, SEL_TILDE, 0, bp, nullptr, status, st, 3, f);
        }));
        NMF_CU(timed(&c->timer, st, "normalize_next", 1, [&] { return launch_fused_next<float>(P0, norm, status, st); }));
      }
      c->lossFused = true;
      c->copiesValid = true;
      return NMF_OK;
    }
  }
  for (int it = 0; it < iters; ++it) {
    const bool lossHere = wantLoss && it == iters - 1;
    const int CL = C | (lossHere ? SWEEP_LOSS : 0);
    const int lossFlag = (fuse && lossHere) ? FUSE_LOSS : 0;
    if (tci && c->count == 1 && c->hpf[0].sWS) {
      if constexpr (std::is_same<T, float>::value)
        if (!haveCopies)
          NMF_CU(timed(&c->timer, st, "begin_iteration", 1,
                       [&] { return launch_tc_copies<float>(c->hpf[0], true, true, true, status, st); }));
      haveCopies = false;            // this iteration's updates change W and H
    } else {
      NMF_CU(timed(&c->timer, st, "begin_iteration", 1, [&] { return launch_begin_iteration<T>(pl, status, st); }));
    }
    bool normDone = false;
    // Warp-specialised path, L = 1: the W epilogue only writes the norm
    // partials; the next sweep's idle warps reduce them (and the objective of
    // the first sweep), or (H first) the normalisation kernel does.
    const bool sideScheme = tci == 2 && joint && L == 1 && fuse && norm;
    // the second sweep reads W~, H~ and V before the epilogue ahead of it
    // has finished (NMF_TC_EARLY=0: it waits for it at entry)
    const char* earlyEnv = std::getenv("NMF_TC_EARLY");
    const int early = (earlyEnv && earlyEnv[0] == '0') ? 0 : SWEEP_EARLY;
    if (sideScheme) {
      SideJob sj;
      const int nparts = rows_epilogue_grid(pl.totW, rows_epilogue_lanes(pl, tci));
      if (lossHere) {
        sj.lossPart = lp;
        sj.nloss = wfirst ? rowGrid : colGrid;
        sj.lossOut = c->d_lossOut;
      }
      if (wfirst) {
        sj.normPart = reinterpret_cast<const float*>(c->d_normPart);
        sj.nparts = nparts;
        if constexpr (std::is_same<T, float>::value) sj.norms = c->hpf[0].norms;
        NMF_TRY(row_sweep(SEL_TILDE, SEL_TILDE, OP_SELF, CL));
        NMF_TRY(rows_epi(SEL_TILDE, 1, FUSE_NORM_PART | FUSE_NO_FINALIZE));
        NMF_TRY(col_sweep(SEL_TILDE, SEL_TILDE, OP_CHI, C | early, &sj));
        if (fuseCopies) {
          if constexpr (std::is_same<T, float>::value)
            NMF_CU(timed(&c->timer, st, "cols_epilogue", 1,
                         [&] { return launch_cols_next<float>(pl, c->hpf[0], bp, status, st); }));
          haveCopies = true;
        } else {
          NMF_TRY(cols_epi(SEL_TILDE, 0, FUSE_NORM_APPLY));
        }
      } else {
        NMF_TRY(col_sweep(SEL_TILDE, SEL_TILDE, OP_SELF, CL));
        NMF_TRY(cols_epi(SEL_TILDE, 1, 0));
        NMF_TRY(row_sweep(SEL_TILDE, SEL_TILDE, OP_CHI, C | early, lossHere ? &sj : nullptr));
        NMF_TRY(rows_epi(SEL_TILDE, 0, FUSE_NORM_PART | FUSE_NO_FINALIZE));
        NMF_CU(timed(&c->timer, st, "normalize", 1, [&] {
          return launch_normalize_parts<T>(pl, reinterpret_cast<const T*>(c->d_normPart), nparts, status, st);
        }));
      }
      continue;
    }
    if (joint) {
      for (int l = 1; l <= L; ++l) {
        const int f1 = l == 1 ? CL : C;
        const int lf = l == 1 ? lossFlag : 0;
        const bool lastL = l == L;
        if (wfirst) {
          NMF_TRY(row_sweep(SEL_TILDE, SEL_TILDE, l == 1 ? OP_SELF : OP_CHI, f1));
          NMF_TRY(rows_epi(SEL_TILDE, 1, lf | ((fuse && norm && lastL) ? FUSE_NORM_PART : 0)));
          NMF_TRY(col_sweep(SEL_TILDE, SEL_TILDE, OP_CHI, C));
          NMF_TRY(cols_epi(SEL_TILDE, l < L, (fuse && norm && lastL) ? FUSE_NORM_APPLY : 0));
          normDone = normDone || (fuse && norm && lastL);
        } else {
          NMF_TRY(col_sweep(SEL_TILDE, SEL_TILDE, l == 1 ? OP_SELF : OP_CHI, f1));
          NMF_TRY(cols_epi(SEL_TILDE, 1, lf));
          NMF_TRY(row_sweep(SEL_TILDE, SEL_TILDE, OP_CHI, C));
          NMF_TRY(rows_epi(SEL_TILDE, l < L, (fuse && norm && lastL) ? FUSE_NORM_PART : 0));
          if (fuse && norm && lastL) {
            NMF_CU(timed(&c->timer, st, "normalize", 1, [&] { return launch_normalize_apply<T>(pl, status, st); }));
            normDone = true;
          }
        }
      }
    } else {
      for (int half = 0; half < 2; ++half) {
        const bool doW = (half == 0) == wfirst;
        for (int l = 1; l <= L; ++l) {
          const int fl = (half == 0 && l == 1) ? CL : C;
          const int lf = (half == 0 && l == 1) ? lossFlag : 0;
          const bool lastUpdate = half == 1 && l == L;    // the iteration's last update
          if (doW) {
            NMF_TRY(row_sweep(SEL_CUR, SEL_CUR, OP_SELF, fl));
            // norms of the final W: W's last update (W first: end of half 0; H first: the last update)
            const bool finalW = l == L;
            NMF_TRY(rows_epi(SEL_CUR, 0, lf | ((fuse && norm && finalW) ? FUSE_NORM_PART : 0)));
            if (lastUpdate && fuse && norm) {
              NMF_CU(timed(&c->timer, st, "normalize", 1, [&] { return launch_normalize_apply<T>(pl, status, st); }));
              normDone = true;
            }
          } else {
            NMF_TRY(col_sweep(SEL_CUR, SEL_CUR, OP_SELF, fl));
            NMF_TRY(cols_epi(SEL_CUR, 0, lf | ((fuse && norm && lastUpdate) ? FUSE_NORM_APPLY : 0)));
            normDone = normDone || (fuse && norm && lastUpdate);
          }
        }
      }
    }
    if (norm && !normDone) NMF_CU(timed(&c->timer, st, "normalize", 2, [&] { return launch_normalize<T>(pl, status, st); }));
  }
  c->lossFused = fuse;
  c->copiesValid = haveCopies;
  if (wantLoss) c->lossPrefix = (wfirst ? 0 : 1) + (tc ? 2 : 0);
  return NMF_OK;
}

nmf_status finalize_loss_dense(nmf_ctx* c) {
  const int* pref = nullptr;
  if (c->prec == NMF_FP64) pref = c->lossPrefix == 0 ? c->pd.d_prefRow : c->pd.d_prefCol;
  else if (c->lossPrefix >= 2) pref = c->pf.d_prefTc + (c->lossPrefix == 2 ? 0 : 2);
  else pref = c->lossPrefix == 0 ? c->pf.d_prefRow : c->pf.d_prefCol;
  return cu(timed(&c->timer, c->stream, "loss_finalize", 1, [&] {
    return launch_loss_finalize(pref, c->count, c->d_lossPart, c->d_lossOut, c->stream);
  }));
}

// Copies the loss (when asked) and the status word into pinned host memory.
nmf_status enqueue_readback(nmf_ctx* c, bool readLoss) {
  const int cnt = c->count;
  if (readLoss)
    NMF_CU(cudaMemcpyAsync(c->h_pinned, c->d_lossOut, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  NMF_CU(cudaMemcpyAsync(reinterpret_cast<int*>(c->h_pinned + cnt + 1), c->d_status, sizeof(int),
                         cudaMemcpyDeviceToHost, c->stream));
  return NMF_OK;
}

// After the stream `sync` has completed the readback: on a device-side
// non-finite flag restores W, H from the tilde copies; else publishes the loss.
nmf_status complete_readback(nmf_ctx* c, bool readLoss, double* loss_out) {
  const int cnt = c->count;
  const int hs = *reinterpret_cast<int*>(c->h_pinned + cnt + 1);
  if (hs != 0) {
    c->copiesValid = false;
    const size_t es = c->sparse ? 4 : esize(c);
    void* W = c->batched ? c->Wp : c->W;
    void* H = c->batched ? c->Hp : c->H;
    NMF_CU(cudaMemcpyAsync(W, c->tildeW, es * c->elemsW, cudaMemcpyDeviceToDevice, c->stream));
    NMF_CU(cudaMemcpyAsync(H, c->tildeH, es * c->elemsH, cudaMemcpyDeviceToDevice, c->stream));
    NMF_CU(cudaStreamSynchronize(c->stream));
    return (nmf_status)hs;
  }
  if (readLoss) {
    c->lastLosses.assign(c->h_pinned, c->h_pinned + cnt);
    c->lossValid = true;
    if (loss_out) {
      double s = 0.0;
      for (int i = 0; i < cnt; ++i) s += c->h_pinned[i];
      *loss_out = s;
    }
  }
  return NMF_OK;
}

// Synchronises; on a device-side non-finite flag restores W, H from the tilde copies.
nmf_status sync_and_check(nmf_ctx* c, bool readLoss, double* loss_out) {
  NMF_TRY(enqueue_readback(c, readLoss));
  NMF_CU(cudaStreamSynchronize(c->stream));
  return complete_readback(c, readLoss, loss_out);
}

// Sparse contexts: binds the caller's CSR arrays and builds the CSC copy once
// (every sparse entry point calls this after prepare()).
nmf_status ensure_sparse(nmf_ctx* c) {
  if (c->cscBuilt) return NMF_OK;
  c->sp.rowptr = c->rowptr;
  c->sp.col = c->col;
  c->sp.val = c->val;
  void* tmp = nullptr;
  const size_t tb = sparse_csc_tmp_bytes(c->sp.F, c->sp.N, c->nnz);
  NMF_TRY(dalloc(c, &tmp, tb));
  const cudaError_t be = sparse_build_csc(c->sp, tmp, tb, c->stream);
  if (be == cudaErrorInvalidValue) return NMF_EINVAL;  // malformed CSR arrays, nothing was indexed
  NMF_CU(be);
  c->cscBuilt = true;
  return NMF_OK;
}

// Every kernel and copy of one step call, enqueued on c->stream (no host
// synchronisation, no allocation: the sequence can be captured into a graph).
// readback = false: the loss (when wanted) stays in d_lossOut and nothing is
// copied to the host (asynchronous steps).
nmf_status enqueue_step(nmf_ctx* c, bool joint, int32_t iters, bool wantLoss, bool readback = true) {
  if (c->sparse) {
    const bool hfirst = c->order == NMF_H_FIRST || (c->order == NMF_ORDER_AUTO && c->F[0] < c->N[0]);
    for (int it = 0; it < iters; ++it) {
      const bool lossHere = wantLoss && it == iters - 1;
      NMF_CU(sparse_step(c->sp, static_cast<float*>(c->W), static_cast<float*>(c->H), joint, hfirst,
                         lossHere, c->normalize != 0, c->d_status, &c->timer, c->stream));
    }
    if (wantLoss) NMF_CU(cudaMemcpyAsync(c->d_lossOut, c->sp.sums, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    const bool tc = c->prec == NMF_TF32 || c->prec == NMF_BF16;
    if (c->prec == NMF_FP64) NMF_TRY(run_dense<double>(c, c->pd, joint, iters, wantLoss, false));
    else NMF_TRY(run_dense<float>(c, c->pf, joint, iters, wantLoss, tc));
    if (wantLoss && !c->lossFused) NMF_TRY(finalize_loss_dense(c));
  }
  return readback ? enqueue_readback(c, wantLoss) : NMF_OK;
}

// ---- CUDA graphs --------------------------------------------------------------
// A step configuration seen once runs eagerly; from its second call on it is
// captured once (on the context's own stream) and replayed with one launch.
// The caller's stream and the context stream are ordered with events, so the
// call stays stream-ordered on the caller's stream.

uint64_t step_key(const nmf_ctx* c, bool joint, int iters, bool wantLoss, bool readback) {
  uint64_t k = (uint64_t)(uint32_t)iters;
  k = k * 4 + (joint ? 1 : 0) + (wantLoss ? 2 : 0);
  k = k * 2 + (c->timer.on ? 1 : 0);
  k = k * 2 + (readback ? 1 : 0);
  k = k * 2 + (c->copiesValid ? 1 : 0);
  return k;
}

void invalidate_graphs(nmf_ctx* c) {
  c->copiesValid = false;
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& p : g.sink.pairs) { c->timer.pool.push_back(p.a); c->timer.pool.push_back(p.b); }
  }
  c->graphs.clear();
  c->seenKeys.clear();
}

nmf_status ensure_graph_stream(nmf_ctx* c) {
  if (c->gs) return NMF_OK;
  if (cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return NMF_ECUDA; }
  if (cudaEventCreateWithFlags(&c->evIn, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->evOut, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return NMF_ECUDA;
  }
  return NMF_OK;
}

// Captures enqueue_step into a graph; returns nullptr (graphs then stay off
// for this context) if capture is not possible.
nmf_ctx::GraphEntry* capture_step(nmf_ctx* c, uint64_t key, bool joint, int32_t iters, bool wantLoss, bool readback) {
  if (ensure_graph_stream(c) != NMF_OK) return nullptr;
  cudaStream_t user = c->stream;
  nmf_ctx::GraphEntry e;
  e.key = key;
  const void* ptrs[6] = {c->V, c->W, c->H, c->Vp, c->Wp, c->Hp};
  std::copy(ptrs, ptrs + 6, e.ptrs);
  c->stream = c->gs;
  c->timer.sink = &e.sink;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  nmf_status st = ok ? enqueue_step(c, joint, iters, wantLoss, readback) : NMF_ECUDA;
  e.copiesAfter = c->copiesValid;
  if (ok) ok = cudaStreamEndCapture(c->gs, &graph) == cudaSuccess && st == NMF_OK && graph;
  if (ok) ok = cudaGraphInstantiate(&e.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  c->timer.sink = nullptr;
  c->stream = user;
  if (!ok) {
    cudaGetLastError();
    for (auto& p : e.sink.pairs) { c->timer.pool.push_back(p.a); c->timer.pool.push_back(p.b); }
    c->useGraphs = false;
    c->copiesValid = false;       // the captured step never ran
    return nullptr;
  }
  c->graphs.push_back(std::move(e));
  return &c->graphs.back();
}

// loss_dev != nullptr: asynchronous step; the loss goes to that device buffer
// (loss_dev == d_lossOut: it stays where the step leaves it).
nmf_status replay(nmf_ctx* c, nmf_ctx::GraphEntry& g, bool wantLoss, double* loss_out, double* loss_dev) {
  c->copiesValid = g.copiesAfter;
  NMF_CU(cudaEventRecord(c->evIn, c->stream));
  NMF_CU(cudaStreamWaitEvent(c->gs, c->evIn, 0));
  NMF_CU(cudaGraphLaunch(g.exec, c->gs));
  NMF_CU(cudaEventRecord(c->evOut, c->gs));
  NMF_CU(cudaStreamWaitEvent(c->stream, c->evOut, 0));
  if (loss_dev) {
    if (loss_dev != c->d_lossOut)
      NMF_CU(cudaMemcpyAsync(loss_dev, c->d_lossOut, sizeof(double) * c->count, cudaMemcpyDeviceToDevice, c->stream));
    if (c->timer.on) NMF_CU(cudaStreamSynchronize(c->gs));
    c->timer.credit(g.sink, c->timer.on);
    return NMF_OK;
  }
  if (c->timer.on || wantLoss) NMF_CU(cudaStreamSynchronize(c->gs));
  c->timer.credit(g.sink, c->timer.on);
  if (!wantLoss) return NMF_OK;
  return complete_readback(c, true, loss_out);
}

nmf_status step(nmf_ctx* c, bool joint, int32_t iters, double* loss_out, double* loss_dev = nullptr) {
  if (!c || iters < 1) return NMF_EINVAL;
  if (!data_ready(c)) return NMF_ENOTREADY;
  NMF_TRY(prepare(c));
  if (c->sparse) NMF_TRY(ensure_sparse(c));
  const bool tc = c->prec == NMF_TF32 || c->prec == NMF_BF16;
  if (!c->sparse && tc && ((c->batched && c->prec != NMF_BF16) || (!c->batched && tc_kp(c->K[0]) > TC_KPMAX)))
    return NMF_EUNSUPPORTED;
  // NMF_BF16 is the fused single-read joint iteration: H first, L = 1, K <= 32, F <= 1024
  if (!c->sparse && c->prec == NMF_BF16 &&
      (!joint || c->L != 1 || c->order == NMF_W_FIRST ||
       (c->batched ? !c->fb.ok : (!c->tcmaps.ok || !tc_fused_supported(c->hpf[0])))))
    return NMF_EUNSUPPORTED;
  const bool wantLoss = loss_out != nullptr || loss_dev != nullptr;
  const bool readback = loss_dev == nullptr;
  if (c->useGraphs && c->stream != c->gs) {
    const uint64_t key = step_key(c, joint, iters, wantLoss, readback);
    const void* ptrs[6] = {c->V, c->W, c->H, c->Vp, c->Wp, c->Hp};
    for (auto& g : c->graphs)
      if (!std::equal(ptrs, ptrs + 6, g.ptrs)) { invalidate_graphs(c); break; }
    for (auto& g : c->graphs)
      if (g.key == key) return replay(c, g, wantLoss, loss_out, loss_dev);
    bool seen = false;
    for (uint64_t k : c->seenKeys) seen = seen || k == key;
    if (seen) {
      nmf_ctx::GraphEntry* g = capture_step(c, key, joint, iters, wantLoss, readback);
      if (g) return replay(c, *g, wantLoss, loss_out, loss_dev);
    } else {
      c->seenKeys.push_back(key);
    }
  }
  NMF_TRY(enqueue_step(c, joint, iters, wantLoss, readback));
  if (loss_dev) {
    if (loss_dev != c->d_lossOut)
      NMF_CU(cudaMemcpyAsync(loss_dev, c->d_lossOut, sizeof(double) * c->count, cudaMemcpyDeviceToDevice, c->stream));
    return NMF_OK;
  }
  if (!wantLoss) return NMF_OK;
  NMF_CU(cudaStreamSynchronize(c->stream));
  return complete_readback(c, true, loss_out);
}

bool valid_beta(double b) { return std::isfinite(b); }

}  // namespace

// ---------------------------------------------------------------------------
// Loss finalisation kernel: per problem, fixed-order sum of its block partials.
// ---------------------------------------------------------------------------
namespace nmf {
int rows_epilogue_lanes_host(int count, int slices) {
  if (count != 1) return 1;
  return slices >= 16 ? 8 : slices >= 8 ? 4 : slices >= 4 ? 2 : 1;
}

__global__ void loss_finalize_kernel(const int* __restrict__ prefix, const double* __restrict__ part,
                                     double* __restrict__ out) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = prefix[i] + threadIdx.x; b < prefix[i + 1]; b += blockDim.x) s += part[b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[i] = s;
}
cudaError_t launch_loss_finalize(const int* d_prefix, int count, const double* lossPart, double* out,
                                 cudaStream_t st) {
  loss_finalize_kernel<<<count, 256, 0, st>>>(d_prefix, lossPart, out);
  return cudaGetLastError();
}
}  // namespace nmf

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

nmf_status nmf_create(int64_t F, int64_t N, int32_t K, double beta, nmf_ctx** out) {
  if (!out) return NMF_EINVAL;
  *out = nullptr;
  if (F < 1 || N < 1 || K < 1 || !valid_beta(beta)) return NMF_EINVAL;
  if (K > KMAX) return NMF_EUNSUPPORTED;
  if (F > (int64_t)1 << 31 || N > (int64_t)1 << 31) return NMF_EINVAL;
  nmf_ctx* c = new (std::nothrow) nmf_ctx();
  if (!c) return NMF_ENOMEM;
  c->F = {F}; c->N = {N}; c->K = {K};
  c->beta = beta;
  c->elemsW = (size_t)F * K; c->elemsH = (size_t)K * N; c->elemsV = (size_t)F * N;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  *out = c;
  return NMF_OK;
}

nmf_status nmf_batch_create(int32_t count, const int64_t* F, const int64_t* N, const int32_t* K,
                            double beta, nmf_ctx** out) {
  if (!out) return NMF_EINVAL;
  *out = nullptr;
  if (count < 1 || !F || !N || !K || !valid_beta(beta)) return NMF_EINVAL;
  nmf_ctx* c = new (std::nothrow) nmf_ctx();
  if (!c) return NMF_ENOMEM;
  c->batched = true;
  c->count = count;
  c->beta = beta;
  for (int i = 0; i < count; ++i) {
    if (F[i] < 1 || N[i] < 1 || K[i] < 1 || K[i] > KMAX) { delete c; return K[i] > KMAX ? NMF_EUNSUPPORTED : NMF_EINVAL; }
    c->F.push_back(F[i]); c->N.push_back(N[i]); c->K.push_back(K[i]);
    c->elemsW += (size_t)F[i] * K[i]; c->elemsH += (size_t)K[i] * N[i]; c->elemsV += (size_t)F[i] * N[i];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  *out = c;
  return NMF_OK;
}

nmf_status nmf_set_options(nmf_ctx* c, nmf_precision precision, nmf_order order, int normalize,
                           double kappa, int deterministic, void* cuda_stream) {
  if (!c) return NMF_EINVAL;
  if (precision < NMF_FP64 || precision > NMF_BF16) return NMF_EINVAL;
  if (order < NMF_W_FIRST || order > NMF_ORDER_AUTO) return NMF_EINVAL;
  if (!(kappa >= 0.0) || !std::isfinite(kappa)) return NMF_EINVAL;
  if (c->sparse && (precision != NMF_FP32 || kappa != 0.0)) return NMF_EINVAL;
  if (precision != c->prec && c->prepared) { cudaStreamSynchronize(c->stream); free_all(c); }
  invalidate_graphs(c);
  c->prec = precision;
  c->order = order;
  c->normalize = normalize ? 1 : 0;
  c->kappa = kappa;
  c->deterministic = deterministic ? 1 : 0;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return NMF_OK;
}

nmf_status nmf_set_floor(nmf_ctx* c, double eps) {
  if (!c || std::isnan(eps) || std::isinf(eps)) return NMF_EINVAL;
  invalidate_graphs(c);
  c->floorEps = eps < 0.0 ? -1.0 : eps;
  return NMF_OK;
}

nmf_status nmf_set_barrier_test(nmf_ctx* c, int64_t limit_ns, int32_t extra_arrivals) {
  if (!c || limit_ns < 1000000 || limit_ns > 10000000000LL || extra_arrivals < 0 || extra_arrivals > 1)
    return NMF_EINVAL;
  invalidate_graphs(c);
  c->waitLimitNs = (uint64_t)limit_ns;
  c->extraArrivals = (unsigned)extra_arrivals;
  return NMF_OK;
}

nmf_status nmf_set_subiterations(nmf_ctx* c, int32_t L) {
  if (!c || L < 1) return NMF_EINVAL;
  if (c->sparse && L != 1) return NMF_EUNSUPPORTED;
  invalidate_graphs(c);
  c->L = L;
  return NMF_OK;
}

nmf_status nmf_set_dense(nmf_ctx* c, const void* V_dev, int64_t ldv) {
  if (!c || !V_dev || c->batched || c->sparse || ldv < c->N[0]) return NMF_EINVAL;
  invalidate_graphs(c);
  c->V = V_dev;
  c->ldv = ldv;
  c->tableDirty = true;
  c->vDirty = true;
  return NMF_OK;
}

nmf_status nmf_set_csr(nmf_ctx* c, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                       const float* val) {
  if (!c || c->batched || nnz < 0 || (nnz > 0 && (!col || !val)) || !rowptr) return NMF_EINVAL;
  if (c->beta != 1.0 || c->kappa != 0.0 || c->prec != NMF_FP32 || c->L != 1) return NMF_EINVAL;
  if (nnz >= ((int64_t)1 << 31)) return NMF_EUNSUPPORTED;
  if (c->V) return NMF_EINVAL;
  if (c->prepared) { cudaStreamSynchronize(c->stream); free_all(c); }
  invalidate_graphs(c);
  c->sparse = true;
  c->nnz = nnz;
  c->rowptr = rowptr; c->col = col; c->val = val;
  c->cscBuilt = false;
  return NMF_OK;
}

nmf_status nmf_set_factors(nmf_ctx* c, void* W_dev, void* H_dev) {
  if (!c || !W_dev || !H_dev || c->batched) return NMF_EINVAL;
  invalidate_graphs(c);
  c->W = W_dev;
  c->H = H_dev;
  c->tableDirty = true;
  if (c->d_status) {
    if (cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) != cudaSuccess) return NMF_ECUDA;
  }
  return NMF_OK;
}

nmf_status nmf_batch_set_packed(nmf_ctx* c, const void* V_packed, void* W_packed, void* H_packed) {
  if (!c || !c->batched || !V_packed || !W_packed || !H_packed) return NMF_EINVAL;
  invalidate_graphs(c);
  c->Vp = V_packed; c->Wp = W_packed; c->Hp = H_packed;
  c->tableDirty = true;
  c->vDirty = true;
  if (c->d_status) {
    if (cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) != cudaSuccess) return NMF_ECUDA;
  }
  return NMF_OK;
}

nmf_status nmf_step_joint(nmf_ctx* c, int32_t iters, double* loss_out) {
  return step(c, true, iters, loss_out);
}

nmf_status nmf_step_alternating(nmf_ctx* c, int32_t iters, double* loss_out) {
  return step(c, false, iters, loss_out);
}

nmf_status nmf_step_joint_async(nmf_ctx* c, int32_t iters, double* loss_dev) {
  if (!loss_dev) return NMF_EINVAL;
  return step(c, true, iters, nullptr, loss_dev);
}

nmf_status nmf_step_alternating_async(nmf_ctx* c, int32_t iters, double* loss_dev) {
  if (!loss_dev) return NMF_EINVAL;
  return step(c, false, iters, nullptr, loss_dev);
}

nmf_status nmf_loss(nmf_ctx* c, double* out_host) {
  if (!c || !out_host) return NMF_EINVAL;
  if (!data_ready(c)) return NMF_ENOTREADY;
  c->copiesValid = false;          // the evaluation runs in FP32 and may rebuild scratch
  nmf_precision keep = c->prec;
  if (keep == NMF_TF32 || keep == NMF_BF16) c->prec = NMF_FP32;
  nmf_status s = prepare(c);
  if (s == NMF_OK && c->sparse) s = ensure_sparse(c);
  if (s == NMF_OK) {
    if (c->sparse) {
      s = cu(sparse_loss(c->sp, static_cast<const float*>(c->W), static_cast<const float*>(c->H),
                         c->d_lossOut, c->stream));
    } else {
      const BetaParams bp = beta_params(c);
      if (c->prec == NMF_FP64)
        s = cu(launch_row_sweep<double>(c->pd, SEL_CUR, SEL_CUR, OP_SELF, SWEEP_LOSS, bp, c->d_lossPart, c->d_status, c->stream));
      else
        s = cu(launch_row_sweep<float>(c->pf, SEL_CUR, SEL_CUR, OP_SELF, SWEEP_LOSS, bp, c->d_lossPart, c->d_status, c->stream));
      c->lossPrefix = 0;
      if (s == NMF_OK) s = finalize_loss_dense(c);
    }
    if (s == NMF_OK) s = sync_and_check(c, true, out_host);
  }
  c->prec = keep;
  return s;
}

nmf_status nmf_grad(nmf_ctx* c, void* gW_dev, void* gH_dev, double* loss_out) {
  if (!c || !gW_dev || !gH_dev) return NMF_EINVAL;
  if (c->batched) return NMF_EUNSUPPORTED;
  if (!data_ready(c)) return NMF_ENOTREADY;
  // NMF_BF16 dense contexts: the fused single-read sweep in its adjoint mode
  // (one read of V: both gradients and the objective, bf16 contractions)
  if (c->prec == NMF_BF16 && !c->sparse) {
    nmf_status s = prepare(c);
    if (s == NMF_OK && c->tcmaps.ok && tc_fused_supported(c->hpf[0])) {
      const Prob<float>& P0 = c->hpf[0];
      const BetaParams bp = beta_params(c);
      const int ncl = P0.fuS, cgrid = tc_fused_cluster_blocks(P0) * ncl;
      const bool wantLoss = loss_out != nullptr;
      int* status = c->d_status;
      double* lp = c->d_lossPart;
      cudaStream_t st = c->stream;
      invalidate_graphs(c);
      s = cu(launch_tc_copies<float>(P0, true, true, true, status, st));
      if (s == NMF_OK)
        s = cu(launch_tc_fused(P0, c->tcmaps, bp, ncl, lp, status, c->waitLimitNs, c->extraArrivals, st,
                               static_cast<float*>(gH_dev)));
      EpiFuse f;
      f.flags = wantLoss ? FUSE_LOSS : 0;
      f.lossPart = lp;
      f.lossBlocks = cgrid;
      f.lossOut = c->d_lossOut;
      f.counter = c->d_counter;
      if (s == NMF_OK)
        s = cu(launch_rows_epilogue<float>(c->pf, EPI_GRAD, SEL_TILDE, 0, bp, static_cast<float*>(gW_dev), status, st,
                                           3, f));
      c->copiesValid = s == NMF_OK;      // the copies are of the current W, H
      if (s == NMF_OK && wantLoss) s = sync_and_check(c, true, loss_out);
      return s;
    }
    if (s != NMF_OK) return s;
  }
  c->copiesValid = false;
  nmf_precision keep = c->prec;
  if (keep == NMF_TF32 || keep == NMF_BF16) c->prec = NMF_FP32;
  nmf_status s = prepare(c);
  if (s == NMF_OK && c->sparse) s = ensure_sparse(c);
  const bool wantLoss = loss_out != nullptr;
  if (s == NMF_OK) {
    if (c->sparse) {
      s = cu(sparse_grad(c->sp, static_cast<const float*>(c->W), static_cast<const float*>(c->H),
                         static_cast<float*>(gW_dev), static_cast<float*>(gH_dev), c->stream));
      if (s == NMF_OK && wantLoss)
        s = cu(sparse_loss_finalize(c->sp, static_cast<const float*>(c->W), static_cast<const float*>(c->H),
                                    c->d_lossOut, c->stream));
    } else {
      const BetaParams bp = beta_params(c);
      const int fl = SWEEP_CONTRACT | (wantLoss ? SWEEP_LOSS : 0);
      if (c->prec == NMF_FP64) {
        s = cu(launch_row_sweep<double>(c->pd, SEL_CUR, SEL_CUR, OP_SELF, fl, bp, c->d_lossPart, c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_rows_epilogue<double>(c->pd, EPI_GRAD, SEL_CUR, 0, bp, static_cast<double*>(gW_dev), c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_col_sweep<double>(c->pd, SEL_CUR, SEL_CUR, OP_SELF, SWEEP_CONTRACT, bp, c->d_lossPart, c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_cols_epilogue<double>(c->pd, EPI_GRAD, SEL_CUR, 0, bp, static_cast<double*>(gH_dev), c->d_status, c->stream));
      } else {
        s = cu(launch_row_sweep<float>(c->pf, SEL_CUR, SEL_CUR, OP_SELF, fl, bp, c->d_lossPart, c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_rows_epilogue<float>(c->pf, EPI_GRAD, SEL_CUR, 0, bp, static_cast<float*>(gW_dev), c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_col_sweep<float>(c->pf, SEL_CUR, SEL_CUR, OP_SELF, SWEEP_CONTRACT, bp, c->d_lossPart, c->d_status, c->stream));
        if (s == NMF_OK) s = cu(launch_cols_epilogue<float>(c->pf, EPI_GRAD, SEL_CUR, 0, bp, static_cast<float*>(gH_dev), c->d_status, c->stream));
      }
      c->lossPrefix = 0;
      if (s == NMF_OK && wantLoss) s = finalize_loss_dense(c);
    }
    if (s == NMF_OK && wantLoss) s = sync_and_check(c, true, loss_out);
  }
  c->prec = keep;
  return s;
}

nmf_status nmf_kkt(nmf_ctx* c, double* resW, double* resH) {
  if (!c || !resW || !resH) return NMF_EINVAL;
  if (c->batched) return NMF_EUNSUPPORTED;
  if (!data_ready(c)) return NMF_ENOTREADY;
  c->copiesValid = false;
  nmf_precision keep = c->prec;
  if (keep == NMF_TF32 || keep == NMF_BF16) c->prec = NMF_FP32;
  nmf_status s = prepare(c);
  const size_t es = c->sparse ? 4 : esize(c);
  if (s == NMF_OK && !c->d_gW) {
    s = dalloc(c, &c->d_gW, es * c->elemsW);
    if (s == NMF_OK) s = dalloc(c, &c->d_gH, es * c->elemsH);
    if (s == NMF_OK) s = dalloc(c, reinterpret_cast<void**>(&c->d_kkt), sizeof(double) * 2);
  }
  if (s == NMF_OK) {
    c->prec = keep;
    s = nmf_grad(c, c->d_gW, c->d_gH, nullptr);
    if (keep == NMF_TF32 || keep == NMF_BF16) c->prec = NMF_FP32;
  }
  if (s == NMF_OK) {
    if (c->prec == NMF_FP64)
      s = cu(launch_kkt<double>(static_cast<double*>(c->W), static_cast<double*>(c->d_gW), c->elemsW,
                                static_cast<double*>(c->H), static_cast<double*>(c->d_gH), c->elemsH, c->d_kkt, c->stream));
    else
      s = cu(launch_kkt<float>(static_cast<float*>(c->W), static_cast<float*>(c->d_gW), c->elemsW,
                               static_cast<float*>(c->H), static_cast<float*>(c->d_gH), c->elemsH, c->d_kkt, c->stream));
  }
  if (s == NMF_OK) {
    s = cu(cudaMemcpyAsync(c->h_pinned + c->count + 2, c->d_kkt, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    if (s == NMF_OK) s = sync_and_check(c, false, nullptr);
    if (s == NMF_OK) {
      *resW = c->h_pinned[c->count + 2] / (double)c->elemsW;
      *resH = c->h_pinned[c->count + 3] / (double)c->elemsH;
    }
  }
  c->prec = keep;
  return s;
}

nmf_status nmf_batch_get_losses(nmf_ctx* c, double* out_host) {
  if (!c || !out_host) return NMF_EINVAL;
  if (!c->lossValid) return NMF_ENOTREADY;
  std::copy(c->lastLosses.begin(), c->lastLosses.end(), out_host);
  return NMF_OK;
}

// Tile-shape autotuner for the SIMT sweeps (FP64, FP32 and batched contexts):
// every candidate chunk cap is timed over `trials` joint steps from the same
// W, H (restored after each), and the fastest is kept. Choices are cached per
// process under a shape signature, so a second context of the same shape
// skips the timing.
namespace {
std::mutex g_tuneMu;
std::map<std::vector<int64_t>, int> g_tuneCache;
}  // namespace

nmf_status nmf_autotune(nmf_ctx* c, int32_t trials, int32_t* chunk_cap) {
  if (!c || trials < 1) return NMF_EINVAL;
  if (c->sparse || (!c->batched && (c->prec == NMF_TF32 || c->prec == NMF_BF16))) return NMF_EUNSUPPORTED;
  if (!data_ready(c)) return NMF_ENOTREADY;
  std::vector<int64_t> sig = {c->count, (int64_t)c->prec, (int64_t)std::llround(c->beta * 1e6), c->batched ? 1 : 0};
  int64_t sf = 0, sn = 0, mk = 0;
  for (int i = 0; i < c->count; ++i) { sf += c->F[i]; sn += c->N[i]; mk = std::max<int64_t>(mk, c->K[i]); }
  sig.push_back(sf); sig.push_back(sn); sig.push_back(mk); sig.push_back(c->sms);
  {
    std::lock_guard<std::mutex> lk(g_tuneMu);
    auto it = g_tuneCache.find(sig);
    if (it != g_tuneCache.end()) {
      if (c->chunkCap != it->second) { c->chunkCap = it->second; c->prepared = false; }
      if (chunk_cap) *chunk_cap = it->second;
      return NMF_OK;
    }
  }
  const size_t es = esize(c);
  void* W = c->batched ? c->Wp : c->W;
  void* H = c->batched ? c->Hp : c->H;
  void *bW = nullptr, *bH = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  nmf_status s = NMF_OK;
  if (cudaMalloc(&bW, es * c->elemsW) != cudaSuccess || cudaMalloc(&bH, es * c->elemsH) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    s = NMF_ENOMEM;
  }
  if (s == NMF_OK) s = cu(cudaMemcpyAsync(bW, W, es * c->elemsW, cudaMemcpyDeviceToDevice, c->stream));
  if (s == NMF_OK) s = cu(cudaMemcpyAsync(bH, H, es * c->elemsH, cudaMemcpyDeviceToDevice, c->stream));
  const int caps[] = {8, 16, 32, 64, 128};
  const int keep = c->chunkCap;
  int best = keep;
  float bestMs = 3.4e38f;
  auto restore = [&]() -> nmf_status {
    NMF_CU(cudaMemcpyAsync(W, bW, es * c->elemsW, cudaMemcpyDeviceToDevice, c->stream));
    NMF_CU(cudaMemcpyAsync(H, bH, es * c->elemsH, cudaMemcpyDeviceToDevice, c->stream));
    if (c->d_status) NMF_CU(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    return NMF_OK;
  };
  for (int cap : caps) {
    if (s != NMF_OK) break;
    c->chunkCap = cap;
    c->prepared = false;                          // the next step rebuilds the plan with this cap
    s = step(c, true, 1, nullptr);                // warm-up (and the plan)
    if (s == NMF_OK) s = restore();
    if (s == NMF_OK) s = cu(cudaEventRecord(e0, c->stream));
    if (s == NMF_OK) s = step(c, true, trials, nullptr);
    if (s == NMF_OK) s = cu(cudaEventRecord(e1, c->stream));
    if (s == NMF_OK) s = cu(cudaEventSynchronize(e1));
    float ms = 0.f;
    if (s == NMF_OK) s = cu(cudaEventElapsedTime(&ms, e0, e1));
    if (s == NMF_OK && ms < bestMs) { bestMs = ms; best = cap; }
    if (s == NMF_OK) s = restore();
  }
  if (s == NMF_OK) s = cu(cudaStreamSynchronize(c->stream));
  c->chunkCap = s == NMF_OK ? best : keep;
  c->prepared = false;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (bW) cudaFree(bW);
  if (bH) cudaFree(bH);
  if (s != NMF_OK) return s;
  {
    std::lock_guard<std::mutex> lk(g_tuneMu);
    g_tuneCache[sig] = best;
  }
  if (chunk_cap) *chunk_cap = best;
  return NMF_OK;
}

nmf_status nmf_get_status(nmf_ctx* c) {
  if (!c) return NMF_EINVAL;
  if (!c->prepared) return NMF_OK;
  return sync_and_check(c, false, nullptr);
}

nmf_status nmf_step_joint_host(nmf_ctx* c, const void* V_host, void* W_host, void* H_host,
                               int32_t iters, double* loss_out) {
  if (!c || !V_host || !W_host || !H_host || iters < 1) return NMF_EINVAL;
  if (c->batched || c->sparse) return NMF_EUNSUPPORTED;
  const size_t es = esize(c);
  NMF_TRY(prepare(c));  // scratch first: a first-time prepare() must not free the staging buffers
  if (!c->stageV) {
    nmf_status s = dalloc(c, &c->stageV, es * c->elemsV);
    if (s == NMF_OK) s = dalloc(c, &c->stageW, es * c->elemsW);
    if (s == NMF_OK) s = dalloc(c, &c->stageH, es * c->elemsH);
    if (s != NMF_OK) return s;
  }
  const void* keepV = c->V; void* keepW = c->W; void* keepH = c->H; int64_t keepLd = c->ldv;
  const int64_t F = c->F[0], N = c->N[0];
  const bool tcPrec = c->prec == NMF_TF32 || c->prec == NMF_BF16;
  if (tcPrec && ((N * 4) & 15) != 0) {
    // rows of V are not 16-byte aligned: copy straight into the padded layout the tensor-core sweeps read
    const int64_t Np = (N + 3) & ~int64_t(3);
    if (!c->Vpad) NMF_TRY(dalloc(c, &c->Vpad, es * (size_t)F * Np));
    NMF_CU(cudaMemcpy2DAsync(c->Vpad, es * Np, V_host, es * N, es * N, F, cudaMemcpyHostToDevice, c->stream));
    c->V = c->Vpad; c->ldv = Np;
  } else {
    NMF_CU(cudaMemcpyAsync(c->stageV, V_host, es * c->elemsV, cudaMemcpyHostToDevice, c->stream));
    c->V = c->stageV; c->ldv = N;
  }
  NMF_CU(cudaMemcpyAsync(c->stageW, W_host, es * c->elemsW, cudaMemcpyHostToDevice, c->stream));
  NMF_CU(cudaMemcpyAsync(c->stageH, H_host, es * c->elemsH, cudaMemcpyHostToDevice, c->stream));
  c->W = c->stageW; c->H = c->stageH;
  c->tableDirty = true;
  c->copiesValid = false;          // W, H come from the host
  // the step, then the loss and status readback and the W, H copies back,
  // all enqueued before one synchronisation
  nmf_status s = step(c, true, iters, nullptr, loss_out ? c->d_lossOut : nullptr);
  if (s == NMF_OK) s = enqueue_readback(c, loss_out != nullptr);
  if (s == NMF_OK) s = cu(cudaMemcpyAsync(W_host, c->stageW, es * c->elemsW, cudaMemcpyDeviceToHost, c->stream));
  if (s == NMF_OK) s = cu(cudaMemcpyAsync(H_host, c->stageH, es * c->elemsH, cudaMemcpyDeviceToHost, c->stream));
  if (s == NMF_OK) s = cu(cudaStreamSynchronize(c->stream));
  if (s == NMF_OK) {
    s = complete_readback(c, loss_out != nullptr, loss_out);
    if (s == NMF_ENONFINITE) {   // W, H were restored on the device: copy those back instead
      nmf_status s2 = cu(cudaMemcpyAsync(W_host, c->stageW, es * c->elemsW, cudaMemcpyDeviceToHost, c->stream));
      if (s2 == NMF_OK) s2 = cu(cudaMemcpyAsync(H_host, c->stageH, es * c->elemsH, cudaMemcpyDeviceToHost, c->stream));
      if (s2 == NMF_OK) s2 = cu(cudaStreamSynchronize(c->stream));
      if (s2 != NMF_OK) s = s2;
    }
  }
  c->V = keepV; c->W = keepW; c->H = keepH; c->ldv = keepLd;
  c->tableDirty = true;
  c->vDirty = true;
  c->copiesValid = false;          // the copies are of the staged W, H
  return s;
}

nmf_status nmf_set_timing(nmf_ctx* c, int enable) {
  if (!c) return NMF_EINVAL;
  invalidate_graphs(c);
  c->timer.on = enable != 0;
  return NMF_OK;
}

nmf_status nmf_get_timing(nmf_ctx* c, int32_t i, const char** name, int64_t* launches, double* total_ms) {
  if (!c || !name || !launches || !total_ms) return NMF_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NMF_ECUDA;
  c->timer.resolve();
  if (i == -1) {
    *name = "all";
    *launches = c->timer.total;
    double s = 0.0;
    for (auto& r : c->timer.recs) s += r.ms;
    *total_ms = s;
    return NMF_OK;
  }
  if (i < 0 || i >= (int32_t)c->timer.recs.size()) return NMF_EINVAL;
  *name = c->timer.recs[i].name;
  *launches = c->timer.recs[i].launches;
  *total_ms = c->timer.recs[i].ms;
  return NMF_OK;
}

nmf_status nmf_reset_timing(nmf_ctx* c) {
  if (!c) return NMF_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NMF_ECUDA;
  c->timer.reset();
  return NMF_OK;
}

void nmf_destroy(nmf_ctx* c) {
  if (!c) return;
  if (c->prepared) cudaStreamSynchronize(c->stream);
  if (c->gs) cudaStreamSynchronize(c->gs);
  free_all(c);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->evIn) cudaEventDestroy(c->evIn);
  if (c->evOut) cudaEventDestroy(c->evOut);
  delete c;
}

const char* nmf_status_string(nmf_status s) {
  switch (s) {
    case NMF_OK: return "NMF_OK";
    case NMF_EINVAL: return "NMF_EINVAL: invalid argument";
    case NMF_ENOMEM: return "NMF_ENOMEM: allocation failed";
    case NMF_ECUDA: return "NMF_ECUDA: CUDA runtime error";
    case NMF_ENONFINITE: return "NMF_ENONFINITE: non-finite value in an update";
    case NMF_ETIMEOUT: return "NMF_ETIMEOUT: device wait timed out";
    case NMF_EUNSUPPORTED: return "NMF_EUNSUPPORTED: not supported by this library";
    case NMF_ENOTREADY: return "NMF_ENOTREADY: data or factors not set";
  }
  return "unknown nmf_status";
}

}  // extern "C"
