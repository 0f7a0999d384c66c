// internal.h -- host-side declarations shared by the translation units of libnmf.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <stdint.h>

#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace nmf {

constexpr int BF = 32;     // rows per SIMT tile
constexpr int BN = 32;     // columns per SIMT tile
constexpr int NT = 256;    // threads per SIMT block
constexpr int EW = 256;    // entries per elementwise block
constexpr int KMAX = 128;  // largest rank the SIMT kernels accept

// Per-context launch counting and optional CUDA-event timing of each kernel
// (nmf_set_timing / nmf_get_timing). Event pairs are resolved lazily. While a
// step is being captured into a CUDA graph, launch counts and event pairs go
// to the graph's own lists (`sink`) and are credited on every replay.
struct Timer {
  struct Rec { const char* name; int64_t launches; double ms; };
  struct Pending { cudaEvent_t a, b; int rec; };
  struct Sink { std::vector<std::pair<int, int>> counts; std::vector<Pending> pairs; };
  bool on = false;
  int64_t total = 0;
  std::vector<Rec> recs;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  Sink* sink = nullptr;

  int rec_index(const char* name) {
    for (size_t i = 0; i < recs.size(); ++i)
      if (recs[i].name == name) return (int)i;
    recs.push_back({name, 0, 0.0});
    return (int)recs.size() - 1;
  }
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
  }
  // Adds the elapsed time of every recorded eager pair (the stream must be synchronised).
  void resolve() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) recs[p.rec].ms += ms;
      else cudaGetLastError();
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  // Credits one replay of a captured graph (its events must have completed).
  void credit(const Sink& g, bool withTimes) {
    for (auto& c : g.counts) { recs[c.first].launches += c.second; total += c.second; }
    if (!withTimes) return;
    for (auto& p : g.pairs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) recs[p.rec].ms += ms;
      else cudaGetLastError();
    }
  }
  void reset() { resolve(); for (auto& r : recs) { r.launches = 0; r.ms = 0.0; } total = 0; }
  ~Timer() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Runs a launcher (which issues `nkern` kernels) under the timer.
template <typename Fn>
inline cudaError_t timed(Timer* t, cudaStream_t st, const char* name, int nkern, Fn&& fn) {
  if (!t) return fn();
  const int r = t->rec_index(name);
  if (t->sink) t->sink->counts.push_back({r, nkern});
  else { t->recs[r].launches += nkern; t->total += nkern; }
  cudaEvent_t a = nullptr, b = nullptr;
  if (t->on) {
    a = t->get();
    b = t->get();
    if (a && b) cudaEventRecord(a, st);
  }
  cudaError_t e = fn();
  if (t->on && a && b) {
    cudaEventRecord(b, st);
    if (t->sink) t->sink->pairs.push_back({a, b, r});
    else t->pending.push_back({a, b, r});
  }
  return e;
}

// Raises a kernel's dynamic shared-memory limit once per device (kept out of
// CUDA-graph capture, which replays launches only).
inline cudaError_t ensure_smem_attr(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mtx;
  static std::vector<std::tuple<const void*, int, size_t>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  std::lock_guard<std::mutex> lock(mtx);
  for (auto& t : done)
    if (std::get<0>(t) == func && std::get<1>(t) == dev && std::get<2>(t) >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.emplace_back(func, dev, bytes);
  return e;
}

// Operand selectors of the sweeps (see sweeps_impl.cuh).
enum { SEL_CUR = 0, SEL_TILDE = 1 };      // W or Wt, H or Ht
enum { OP_SELF = 0, OP_CHI = 1 };         // D1 = D2 = Hp (C1 = C2 = Wp) or the chi buffers
// SWEEP_EARLY (warp-specialised sweeps, the second sweep of a joint
// iteration): the MMA1 operands (W~, H~ copies) and V do not depend on the
// previous kernel, so only the MMA2/3 operand loads, the side jobs and the
// write-out wait for it. Safe because the kernel before such a sweep (an
// epilogue) signals its dependents only after its own dependency wait: when
// the sweep starts, everything two kernels back has completed.
enum { SWEEP_CONTRACT = 1, SWEEP_LOSS = 2, SWEEP_EARLY = 4 };
enum { EPI_UPDATE = 0, EPI_GRAD = 1 };

// Device tables of a context for element type T.
template <typename T>
struct Plan {
  Prob<T>* d_probs = nullptr;
  int count = 0;
  int maxK = 0;
  int* d_prefRow = nullptr; int totRow = 0;   // row-sweep blocks per problem
  int* d_prefCol = nullptr; int totCol = 0;   // column-sweep blocks
  int* d_prefW = nullptr; int totW = 0;       // EW-entry blocks over F x K
  int* d_prefH = nullptr; int totH = 0;       // EW-entry blocks over K x N
  int* d_prefK = nullptr; int totK = 0;       // one block per column of W
  int* d_prefTc = nullptr;                    // {0, tc row grid, 0, tc column grid} (single problem)
  int rowSlices[3] = {1, 1, 1};               // row-sweep partial slices: SIMT, tensor core, fused sweep (single problem)
  int colVec4 = 0;                            // single problem with N % 4 == 0: 16-byte H epilogue
};

template <typename T>
cudaError_t launch_row_sweep(const Plan<T>& pl, int wsel, int hsel, int dsel, int flags,
                             const BetaParams& bp, double* lossPart, const int* status,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_col_sweep(const Plan<T>& pl, int wsel, int hsel, int csel, int flags,
                             const BetaParams& bp, double* lossPart, const int* status,
                             cudaStream_t st);
// W epilogue: W = base . (sum num / sum den)^gamma (mode EPI_UPDATE, base = W or Wt,
// chi computed from (W_new, Wt) when want_chi) or gout = sum den - sum num (EPI_GRAD).
// Optional work fused into the epilogues (single problems only; flags 0 = none):
// FUSE_LOSS: the last block sums the preceding sweep's loss partials into lossOut;
// FUSE_NORM_PART (W epilogue): per-block sums of squares of the new W, turned into
// the column norms (Prob::norms) by the last block; FUSE_NORM_APPLY (H epilogue):
// H rows *= norms and W columns /= norms (normalisation, Sec. 4.1.2).
// FUSE_NO_FINALIZE (with FUSE_NORM_PART): write the partials only; the next
// tensor-core sweep's idle warps (SideJob) or the normalisation kernel reduce them.
enum { FUSE_LOSS = 1, FUSE_NORM_PART = 2, FUSE_NORM_APPLY = 4, FUSE_NO_FINALIZE = 8 };
struct EpiFuse {
  int flags = 0;
  const double* lossPart = nullptr;
  int lossBlocks = 0;
  double* lossOut = nullptr;
  void* normPart = nullptr;     // [K][W epilogue blocks], element type T
  unsigned* counter = nullptr;  // zero between launches
};

// tc != 0: the partials come from the tensor-core sweeps (tcS / tcR slices);
// tc == 3 (W epilogue only): from the fused single-read sweep (fuS slices).
template <typename T>
cudaError_t launch_rows_epilogue(const Plan<T>& pl, int mode, int basesel, int want_chi,
                                 const BetaParams& bp, T* gout, int* status, cudaStream_t st,
                                 int tc = 0, const EpiFuse& fz = EpiFuse());
template <typename T>
cudaError_t launch_cols_epilogue(const Plan<T>& pl, int mode, int basesel, int want_chi,
                                 const BetaParams& bp, T* gout, int* status, cudaStream_t st,
                                 int tc = 0, const EpiFuse& fz = EpiFuse());
template <typename T>
cudaError_t launch_normalize_apply(const Plan<T>& pl, const int* status, cudaStream_t st);
// Single problem: every block reduces the norm partials ([K][nparts], T)
// itself (fixed order), then W /= norms, H *= norms.
template <typename T>
cudaError_t launch_normalize_parts(const Plan<T>& pl, const T* normPart, int nparts, const int* status,
                                   cudaStream_t st);
// Lanes per entry of the W epilogue: for a single problem 8, 4 or 2 with
// >= 16, >= 8 or >= 4 partial slices, else 1. A single problem runs blocks of
// 1024 threads (1024 / G entries each), a batched context blocks of EW.
constexpr int ROWS_EPI_MAX_LANES = 8;
int rows_epilogue_lanes_host(int count, int slices);
// blocks of the single-problem W epilogue; totW blocks of EW entries cover F x K
inline int rows_epilogue_grid(int totW, int G) { return (int)(((int64_t)totW * EW * G + 1023) / 1024); }
template <typename T>
inline int rows_epilogue_lanes(const Plan<T>& pl, int tc) {
  return pl.count == 1 ? rows_epilogue_lanes_host(1, pl.rowSlices[tc == 3 ? 2 : (tc ? 1 : 0)]) : 1;
}
// Tensor-core copies (TF32 shadows) of W and/or H of one problem, and with
// `tilde` the W~, H~ copies too (the begin of a tensor-core iteration).
template <typename T>
cudaError_t launch_tc_copies(const Prob<T>& P, bool doW, bool doH, bool tilde, const int* status, cudaStream_t st);
// The last kernel of a fused single-read iteration: W /= norms, H *= norms
// (norm; Sec. 4.1.2) written back, and the copies the next iteration's fused
// sweep reads (W~, H~ and their TF32 shadows sWS, sHT) made from the result.
constexpr int COPIES_APPLY = 1, COPIES_LEAN = 2;
template <typename T>
cudaError_t launch_fused_next(const Prob<T>& P, bool norm, const int* status, cudaStream_t st);
// The last H epilogue of a W-first tensor-core iteration (normalisation on)
// fused with the next iteration's copies (what launch_tc_copies with tilde
// would make from the final W, H); single problem.
template <typename T>
cudaError_t launch_cols_next(const Plan<T>& pl, const Prob<T>& hp, const BetaParams& bp, int* status,
                             cudaStream_t st);
// Launch with programmatic stream serialization (the kernel calls pdl_wait()
// before reading anything its predecessor wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}
// Copies W -> Wt and H -> Ht for every problem (skipped once status is set).
template <typename T>
cudaError_t launch_begin_iteration(const Plan<T>& pl, const int* status, cudaStream_t st);
// Column l2 norms of W, then W[:,k] /= n_k, H[k,:] *= n_k (zero norms untouched).
template <typename T>
cudaError_t launch_normalize(const Plan<T>& pl, const int* status, cudaStream_t st);
// out[i] = fixed-order sum of lossPart over problem i's blocks of the given prefix table.
cudaError_t launch_loss_finalize(const int* d_prefix, int count, const double* lossPart,
                                 double* out, cudaStream_t st);
// TF32 shadows of the current W (which & 1) / H (which & 2) for the tensor-core sweeps.
template <typename T>
cudaError_t launch_shadow_factors(const Prob<T>& P, int which, const int* status, cudaStream_t st);
// KKT residual sums: out[0] = sum |min(W, gW)|, out[1] = sum |min(H, gH)| (single problem).
template <typename T>
cudaError_t launch_kkt(const T* W, const T* gW, int64_t nW, const T* H, const T* gH,
                       int64_t nH, double* out, cudaStream_t st);

// Tensor-core sweeps, single float problems: same operands and partial-sum
// layout as the SIMT sweeps, with tcS / tcR slices. kp <= 64 runs the
// warp-specialised kernels (tc_ws.cu) on TMA loads of the TF32 shadows;
// 64 < kp <= 128 the simpler kernels of tc_sweeps.cu.
constexpr int TC_KPMAX = 128;  // largest padded rank (multiple of 16) of the tensor-core sweeps
int tc_kp(int K);              // K padded to a multiple of 16

// Tensor maps over the shadow operand copies (built once per plan).
struct TcMaps {
  CUtensorMap wsA, wsB;      // sWS, boxes 32 x 128 and 32 x 32
  CUtensorMap htA, htB;      // sHT, boxes 32 x 128 and 32 x 32
  CUtensorMap hs, ch1, ch2;  // [kp][Np], box 32 x kp
  CUtensorMap wt, cw1, cw2;  // [kp][Fp], box 32 x kp
  bool ok = false;
};
bool tc_build_maps(const Prob<float>& P, TcMaps* m);

// Work for the otherwise idle warp 3 of a warp-specialised sweep's blocks:
// the column norms of W (column k = normK, normK + normStride, ...) from the
// W epilogue's partials ([k][part], float), and the FP64 objective from the
// previous sweep's partials (nloss of them). A kernel launch passes the job
// with normK < 0: block b then takes columns b, b + grid, ..., block 0 the
// objective.
struct SideJob {
  const float* normPart = nullptr;
  int nparts = 0;
  int normK = -1;
  int normStride = 1;
  float* norms = nullptr;
  const double* lossPart = nullptr;
  int nloss = 0;
  double* lossOut = nullptr;
};
// Tensor map of V for the row (row = true) or column sweep; false when V
// cannot be addressed by TMA (the kernels then load V with cp.async).
bool tc_map_v(const Prob<float>& P, bool row, CUtensorMap* m);
// Ring depths and dynamic shared memory of the warp-specialised sweep.
bool tc_ws_rings(int kp, bool chi, int* nop, int* nv, size_t* smem);

// One JMM outer iteration (L = 1, normalisation on) of a single dense TF32
// problem in one persistent cooperative launch (tc_step.cu): the factor
// copies, both sweeps, both epilogues and the normalisation as phases
// separated by grid barriers. False when the context does not qualify
// (the caller then runs the per-kernel sequence).
struct TcStepArgs {
  bool wfirst;
  bool wantLoss;
  double* lossPart;
  double* lossOut;
  float* normPart;      // [K][blocks]
  unsigned* gridBar;    // two words, cleared by the host before every launch
  int* status;
  unsigned extraArrivals = 0;            // nmf_set_barrier_test
  uint64_t waitLimitNs = 1000000000ull;
};
bool tc_step_supported(const Prob<float>& P, const TcMaps& m, int sms);
cudaError_t launch_tc_step(const Prob<float>& P, const TcMaps& m, const BetaParams& bp, const TcStepArgs& a,
                           int sms, cudaStream_t st);

cudaError_t launch_tc_row_sweep(const Prob<float>& P, const TcMaps* maps, int wsel, int hsel, int dsel, int flags,
                                bool bf16, const BetaParams& bp, double* lossPart, int* status, cudaStream_t st,
                                const SideJob* side = nullptr);
cudaError_t launch_tc_col_sweep(const Prob<float>& P, const TcMaps* maps, int wsel, int hsel, int csel, int flags,
                                bool bf16, const BetaParams& bp, double* lossPart, int* status, cudaStream_t st,
                                const SideJob* side = nullptr);
// Blocks of the warp-specialised sweep (padded rank kp) that can be resident
// at once when launched in clusters of `csize`; 0 when it cannot launch.
int tc_ws_capacity(int kp, int csize);
cudaError_t launch_tc_ws_row(const Prob<float>& P, const TcMaps& m, int dsel, int flags, const BetaParams& bp,
                             double* lossPart, int* status, cudaStream_t st, const SideJob* side);
cudaError_t launch_tc_ws_col(const Prob<float>& P, const TcMaps& m, int csel, int flags, const BetaParams& bp,
                             double* lossPart, int* status, cudaStream_t st, const SideJob* side);

// Fused single-read H-first JMM iteration sweep (tc_fused.cu; bf16
// contractions, TF32 product): K <= 32, F <= 1024. It writes H (before the
// normalisation), one [P | Q] partial slice per cluster into rowPart (ncl
// slices) and one objective partial per block (grid = ceil(F / 128) x ncl).
// Blocks per cluster of the single-problem fused sweep (ceil(F / 128), or
// F / 128 when the last block also takes the tail row of F = 128 c + 1).
int tc_fused_cluster_blocks(const Prob<float>& P);
bool tc_fused_supported(const Prob<float>& P);
// Clusters of ceil(F / 128) blocks that can be resident at once (at most the
// number of 128-column batches); 0 when the kernel cannot launch.
int tc_fused_clusters(const Prob<float>& P, int sms);
// gH not null: the adjoint instead of the update (H untouched): grad_H = W~^T (B - A)
// into gH, and slices of P = A H~^T, Q = B H~^T (grad_W = Q - P by the W epilogue's
// EPI_GRAD mode).
// The W half of a fused single-problem iteration and the normalisation
// (tc_fused.cu), two launches of nparts blocks: the slices' sum and the W update
// (in place, base W), per-block column sums of squares into normPart (K x
// nparts floats); then the column norms, W /= norms with its TF32 row copy,
// H *= norms with Ht and its transposed TF32 copy, and the objective from the
// sweep's partials (lossOut not null).
cudaError_t launch_fused_post(const Prob<float>& P, const BetaParams& bp, int slices, bool norm, float* normPart,
                              int nparts, const double* lossPart, int lossBlocks, double* lossOut, int* status,
                              cudaStream_t st);
cudaError_t launch_tc_fused(const Prob<float>& P, const TcMaps& m, const BetaParams& bp, int ncl, double* lossPart,
                            int* status, uint64_t limitNs, unsigned extra, cudaStream_t st, float* gH = nullptr);
// The same sweep over many problems in one launch (batched contexts): work
// item i = {problem, first 128-column batch, end batch, partial slice of that
// problem} runs on cluster i of c = ceil(max F / 128) blocks; the problems'
// descriptors (device Prob array), tensor maps (maps[3 p + 0..2]: V, W~ rows
// sWS, H~^T rows sHT, built by tc_fused_maps) and the index of each item's
// first objective partial (lossBase) live in device memory.
struct FuBatch {
  int c = 1, nitems = 0, layK = 32;
  const int4* items = nullptr;
  const Prob<float>* probs = nullptr;
  const CUtensorMap* maps = nullptr;
  const int* lossBase = nullptr;
  double* lossPart = nullptr;
};
cudaError_t launch_tc_fused_batch(const FuBatch& fb, const BetaParams& bp, int* status, uint64_t limitNs,
                                  unsigned extra, cudaStream_t st);
// V tile depth of the batched sweep's layout (0: does not fit).
int tc_fused_batch_nv(int layK);
// The three tensor maps of one problem for the fused sweep (false if V's rows
// or the shadows are not 16-byte aligned).
bool tc_fused_maps(const Prob<float>& P, CUtensorMap out[3]);
// W~, H~ and their TF32 shadows sWS, sHT of every problem of a batched
// context (the copies the batched fused sweep reads); blocks: the W blocks of
// pl (prefW) then cdiv(N, 32) per problem (prefHc, totHc of them).
cudaError_t launch_fused_batch_copies(const Plan<float>& pl, const int* prefHc, int totHc, const int* status,
                                      cudaStream_t st);

// Sparse beta = 1 path (sparse_kl.cu).
struct SparseKL {
  int64_t F = 0, N = 0, nnz = 0;
  int K = 0;
  const int32_t* rowptr = nullptr;  // CSR (borrowed)
  const int32_t* col = nullptr;
  const float* val = nullptr;
  int32_t* rowidx = nullptr;        // row of each CSR entry (owned)
  int32_t* colptr = nullptr;        // CSC (owned)
  int32_t* cscRow = nullptr;
  int64_t* cscPos = nullptr;        // CSC entry -> CSR position
  float* a = nullptr;               // A = V / Vt at the nonzeros, CSR order
  float* Wt = nullptr;
  float* Ht = nullptr;
  float* colsumW = nullptr;         // K
  float* rowsumH = nullptr;         // K
  float* chi = nullptr;             // scratch K-vector
  double* lossPart = nullptr;
  int lossBlocks = 0;
  double* sums = nullptr;           // scratch doubles
};
cudaError_t sparse_build_csc(SparseKL& s, void* tmp, size_t tmpBytes, cudaStream_t st);
size_t sparse_csc_tmp_bytes(int64_t F, int64_t N, int64_t nnz);
cudaError_t sparse_step(SparseKL& s, float* W, float* H, bool joint, bool hfirst,
                        bool wantLoss, bool normalize, int* status, Timer* tm, cudaStream_t st);
cudaError_t sparse_loss_finalize(SparseKL& s, const float* W, const float* H, double* out,
                                 cudaStream_t st);
cudaError_t sparse_loss(SparseKL& s, const float* W, const float* H, double* out,
                        cudaStream_t st);
cudaError_t sparse_grad(SparseKL& s, const float* W, const float* H, float* gW, float* gH,
                        cudaStream_t st);

}  // namespace nmf
