// sparse_kl.cu -- KL (beta = 1) NMF on sparse count data (Sec. 4.4 workload).
//
// At beta = 1, eq. jnt_update reduces to Table 2's JMM form:
//   W = Wt . (A Ht^T) / (1 chi_2(H, Ht)^T),  H = Ht . (chi_1(W, Wt)^T A) / (chi_2(W, Wt)^T 1)
// with chi_1(X, Xt) = Xt, chi_2(X, Xt) = X, gamma = 1, B = 1, and
// A = V / (Wt Ht) nonzero only where V is. So every numerator is a sampled
// product (SDDMM: Vt at the nonzeros, 2K flops each) followed by a sparse-
// dense product (SpMM), and every denominator is a row or column sum of a
// factor broadcast over the other index. One pass over the CSR rows gives
// the W numerators (and the W update row by row); one pass over the CSC
// columns gives the H numerators. The objective needs Vt only at the
// nonzeros: D = sum_nz [v log(v/vt) - v] + sum_k colsum(W)_k rowsum(H)_k.
//
// Layout: H is K x N row-major (the ABI); a transposed copy (N x K) serves
// the row gathers of the CSR pass, and the CSC pass stages 32 columns of H
// in shared memory so its reads and writes of H stay coalesced.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace nmf {
namespace {

constexpr int WPB = 8;   // warps per block
constexpr int CB = 32;   // columns per CSC block

__global__ void fill_rowidx_kernel(const int32_t* __restrict__ rowptr, int64_t F, int32_t* __restrict__ rowidx,
                                   const int* __restrict__ bad) {
  if (*bad) return;
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  for (int32_t e = rowptr[f]; e < rowptr[f + 1]; ++e) rowidx[e] = (int32_t)f;
}

// Checks the caller's CSR arrays before any index is used: rowptr[0] = 0,
// rowptr[F] = nnz, nondecreasing, 0 <= col < N. Sets *bad on violation.
__global__ void validate_csr_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    int64_t F, int64_t N, int64_t nnz, int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= F) {
    const int32_t r = rowptr[i];
    if (r < 0 || r > nnz) atomicExch(bad, 1);
    if (i == 0 && r != 0) atomicExch(bad, 1);
    if (i == F && r != nnz) atomicExch(bad, 1);
    if (i < F && rowptr[i + 1] < r) atomicExch(bad, 1);
  }
  if (i < nnz) {
    const int32_t c = col[i];
    if (c < 0 || c >= N) atomicExch(bad, 1);
  }
}

__global__ void count_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt,
                                  const int* __restrict__ bad) {
  if (*bad) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) atomicAdd(&cnt[col[e]], 1);
}

// Exclusive scan of cnt[0..N) into out[0..N] with one block (chunked).
__global__ void scan_kernel(const int32_t* __restrict__ cnt, int64_t N, int32_t* __restrict__ out) {
  __shared__ int32_t buf[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < N; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < N ? cnt[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int32_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < N) out[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[N] = carry;
}

__global__ void scatter_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ rowidx, int64_t nnz,
                               const int32_t* __restrict__ colptr, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ cscRow, int64_t* __restrict__ cscPos,
                               const int* __restrict__ bad) {
  if (*bad) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int32_t c = col[e];
  const int32_t p = colptr[c] + atomicAdd(&cursor[c], 1);
  cscRow[p] = rowidx[e];
  cscPos[p] = e;
}

// Orders each column's entries by CSR position so CSC sums are deterministic.
__global__ void sort_cols_kernel(const int32_t* __restrict__ colptr, int64_t N, int32_t* __restrict__ cscRow,
                                 int64_t* __restrict__ cscPos) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int32_t b = colptr[c], e = colptr[c + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    const int64_t p = cscPos[i];
    const int32_t r = cscRow[i];
    int32_t j = i - 1;
    while (j >= b && cscPos[j] > p) {
      cscPos[j + 1] = cscPos[j];
      cscRow[j + 1] = cscRow[j];
      --j;
    }
    cscPos[j + 1] = p;
    cscRow[j + 1] = r;
  }
}

// out[k] = sum_f X[f, k] (or of squares, then sqrt), one block per k, FP64 accumulation.
__global__ void colsum_kernel(const float* __restrict__ X, int64_t rows, int K, float* __restrict__ out,
                              int squares, const int* __restrict__ status) {
  if (status && *status) return;
  __shared__ double red[32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int64_t f = threadIdx.x; f < rows; f += blockDim.x) {
    const double x = X[f * K + k];
    s += squares ? x * x : x;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[k] = (float)(squares ? sqrt(s) : s);
}

// out[k] = sum_n H[k, n], one block per k.
__global__ void rowsum_kernel(const float* __restrict__ H, int K, int64_t N, float* __restrict__ out,
                              const int* __restrict__ status) {
  if (status && *status) return;
  __shared__ double red[32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s += H[(int64_t)k * N + n];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[k] = (float)s;
}

// HT (N x K) = H^T with 32 x 32 shared-memory tiles.
__global__ void transpose_kernel(const float* __restrict__ H, int K, int64_t N, float* __restrict__ HT,
                                 const int* __restrict__ status) {
  if (status && *status) return;
  __shared__ float t[32][33];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r;
    const int64_t n = n0 + threadIdx.x;
    t[r][threadIdx.x] = (k < K && n < N) ? H[(int64_t)k * N + n] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t n = n0 + r;
    const int k = k0 + threadIdx.x;
    if (n < N && k < K) HT[n * K + k] = t[threadIdx.x][r];
  }
}

__global__ void copy_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n,
                            const int* __restrict__ status) {
  if (*status) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void scale_kernel(float* __restrict__ W, int64_t F, int K, float* __restrict__ H, int64_t N,
                             const float* __restrict__ norms, const int* __restrict__ status) {
  if (*status) return;
  const int64_t FK = F * K, KN = (int64_t)K * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < FK + KN;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < FK) {
      const float nk = norms[i % K];
      if (nk > 0.f) W[i] = W[i] / nk;
    } else {
      const int64_t j = i - FK;
      const float nk = norms[j / N];
      if (nk > 0.f) H[j] = H[j] * nk;
    }
  }
}

enum { OUT_NONE = 0, OUT_UPDATE = 1, OUT_GRAD = 2 };

// Warp per CSR row f. COMPUTE: vt = <Wd[f,:], HxT[n,:]> and a = v / vt at each
// nonzero (stored at its CSR position), with the objective's nonzero terms;
// otherwise a is read back. The numerator P[f,:] = sum_n a HxT[n,:] then gives
// Wout[f,:] = Wbase[f,:] . P / den (update) or den - P (gradient).
template <int KJ, bool COMPUTE, int OUT>
__global__ void __launch_bounds__(WPB * 32)
csr_pass_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                const float* __restrict__ val, float* __restrict__ a, const float* __restrict__ Wd,
                const float* __restrict__ HxT, const float* __restrict__ Wbase, const float* __restrict__ den,
                float* __restrict__ Wout, int64_t F, int K, double* __restrict__ lossPart, int* __restrict__ status) {
  if (*status) return;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t f = (int64_t)blockIdx.x * WPB + warp;
  double loss = 0.0;
  if (f < F) {
    float w[KJ], p[KJ];
    #pragma unroll
    for (int j = 0; j < KJ; ++j) {
      const int k = lane + 32 * j;
      w[j] = (COMPUTE && k < K) ? Wd[f * K + k] : 0.f;
      p[j] = 0.f;
    }
    const int32_t eb = rowptr[f], ee = rowptr[f + 1];
    for (int32_t e = eb; e < ee; ++e) {
      const int64_t n = col[e];
      float h[KJ];
      #pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        h[j] = k < K ? HxT[n * K + k] : 0.f;
      }
      float av;
      if (COMPUTE) {
        float d = 0.f;
        #pragma unroll
        for (int j = 0; j < KJ; ++j) d = fmaf(w[j], h[j], d);
        d = warp_sum(d);
        const float v = val[e];
        av = v / d;
        if (lane == 0) {
          a[e] = av;
          if (v > 0.f) loss += (double)(v * logf(v / d) - v);
        }
      } else {
        av = a[e];
      }
      #pragma unroll
      for (int j = 0; j < KJ; ++j) p[j] = fmaf(av, h[j], p[j]);
    }
    if (OUT != OUT_NONE) {
      #pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        if (k < K) {
          float x;
          if (OUT == OUT_UPDATE) x = Wbase[f * K + k] * (p[j] / den[k]);
          else x = den[k] - p[j];
          if (!isfinite(x)) atomicExch(status, 4);
          Wout[f * K + k] = x;
        }
      }
    }
  }
  if (lossPart) {
    loss = block_sum(loss, red);
    if (threadIdx.x == 0) lossPart[blockIdx.x] = loss;
  }
}

// Block per 32 columns [n0, n0+32), warp per column. COMPUTE: vt = <Wd[f,:], Hd[:,n]>
// and a = v / vt at each nonzero of the column (written to its CSR position);
// otherwise a is read. The numerator N[:,n] = sum_f a Wd[f,:] gives
// Hout[:,n] = Hbase[:,n] . N / den (update) or den - N (gradient).
template <int KJ, bool COMPUTE, int OUT>
__global__ void __launch_bounds__(WPB * 32)
csc_pass_kernel(const int32_t* __restrict__ colptr, const int32_t* __restrict__ cscRow,
                const int64_t* __restrict__ cscPos, const float* __restrict__ val, float* __restrict__ a,
                const float* __restrict__ Wd, const float* __restrict__ Hd, const float* Hbase,
                const float* __restrict__ den, float* Hout, int64_t N, int K,
                double* __restrict__ lossPart, int* __restrict__ status) {
  if (*status) return;
  extern __shared__ float sh[];
  float* Hs = sh;                       // [K][CB + 1] columns of Hd
  float* Bs = Hs + K * (CB + 1);        // [K][CB + 1] columns of Hbase
  float* Os = Bs + K * (CB + 1);        // [K][CB + 1] results
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n0 = (int64_t)blockIdx.x * CB;
  for (int i = threadIdx.x; i < K * CB; i += blockDim.x) {
    const int k = i / CB, c = i - k * CB;
    const int64_t n = n0 + c;
    const bool in = n < N;
    if (COMPUTE) Hs[k * (CB + 1) + c] = in ? Hd[(int64_t)k * N + n] : 0.f;
    if (OUT == OUT_UPDATE) Bs[k * (CB + 1) + c] = in ? Hbase[(int64_t)k * N + n] : 0.f;
  }
  __syncthreads();
  double loss = 0.0;
  for (int c = warp; c < CB; c += WPB) {
    const int64_t n = n0 + c;
    if (n >= N) break;
    float hcol[KJ], acc[KJ];
    #pragma unroll
    for (int j = 0; j < KJ; ++j) {
      const int k = lane + 32 * j;
      hcol[j] = (COMPUTE && k < K) ? Hs[k * (CB + 1) + c] : 0.f;
      acc[j] = 0.f;
    }
    const int32_t eb = colptr[n], ee = colptr[n + 1];
    for (int32_t e = eb; e < ee; ++e) {
      const int64_t f = cscRow[e];
      const int64_t pos = cscPos[e];
      float w[KJ];
      #pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        w[j] = k < K ? Wd[f * K + k] : 0.f;
      }
      float av;
      if (COMPUTE) {
        float d = 0.f;
        #pragma unroll
        for (int j = 0; j < KJ; ++j) d = fmaf(w[j], hcol[j], d);
        d = warp_sum(d);
        const float v = val[pos];
        av = v / d;
        if (lane == 0) {
          a[pos] = av;
          if (v > 0.f) loss += (double)(v * logf(v / d) - v);
        }
      } else {
        av = a[pos];
      }
      #pragma unroll
      for (int j = 0; j < KJ; ++j) acc[j] = fmaf(av, w[j], acc[j]);
    }
    #pragma unroll
    for (int j = 0; j < KJ; ++j) {
      const int k = lane + 32 * j;
      if (k < K) {
        float x;
        if (OUT == OUT_UPDATE) x = Bs[k * (CB + 1) + c] * (acc[j] / den[k]);
        else x = den[k] - acc[j];
        if (!isfinite(x)) atomicExch(status, 4);
        Os[k * (CB + 1) + c] = x;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K * CB; i += blockDim.x) {
    const int k = i / CB, c = i - k * CB;
    const int64_t n = n0 + c;
    if (n < N) Hout[(int64_t)k * N + n] = Os[k * (CB + 1) + c];
  }
  if (lossPart) {
    loss = block_sum(loss, red);
    if (threadIdx.x == 0) lossPart[blockIdx.x] = loss;
  }
}

// sums[0] = fixed-order sum of the partials + sum_k cs[k] rs[k] (the objective).
__global__ void sparse_loss_final_kernel(const double* __restrict__ part, int nb, const float* __restrict__ cs,
                                         const float* __restrict__ rs, int K, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  __syncthreads();
  double t = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) t += (double)cs[k] * (double)rs[k];
  t = block_sum(t, red);
  if (threadIdx.x == 0) out[0] = s + t;
}

template <bool COMPUTE, int OUT>
cudaError_t csr_pass(const SparseKL& s, const float* Wd, const float* HxT, const float* Wbase,
                     const float* den, float* Wout, double* lossPart, int* status, cudaStream_t st) {
  const int grid = (int)((s.F + WPB - 1) / WPB);
  if (s.K <= 32)
    csr_pass_kernel<1, COMPUTE, OUT><<<grid, WPB * 32, 0, st>>>(s.rowptr, s.col, s.val, s.a, Wd, HxT, Wbase, den, Wout, s.F, s.K, lossPart, status);
  else if (s.K <= 64)
    csr_pass_kernel<2, COMPUTE, OUT><<<grid, WPB * 32, 0, st>>>(s.rowptr, s.col, s.val, s.a, Wd, HxT, Wbase, den, Wout, s.F, s.K, lossPart, status);
  else
    csr_pass_kernel<4, COMPUTE, OUT><<<grid, WPB * 32, 0, st>>>(s.rowptr, s.col, s.val, s.a, Wd, HxT, Wbase, den, Wout, s.F, s.K, lossPart, status);
  return cudaGetLastError();
}

template <int KJ, bool COMPUTE, int OUT>
cudaError_t csc_pass_kj(const SparseKL& s, const float* Wd, const float* Hd, const float* Hbase,
                        const float* den, float* Hout, double* lossPart, int* status, cudaStream_t st) {
  auto kern = csc_pass_kernel<KJ, COMPUTE, OUT>;
  const size_t sm = sizeof(float) * 3 * s.K * (CB + 1);
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(kern), sm);
  if (e != cudaSuccess) return e;
  const int grid = (int)((s.N + CB - 1) / CB);
  kern<<<grid, WPB * 32, sm, st>>>(s.colptr, s.cscRow, s.cscPos, s.val, s.a, Wd, Hd, Hbase, den, Hout, s.N, s.K,
                                   lossPart, status);
  return cudaGetLastError();
}

template <bool COMPUTE, int OUT>
cudaError_t csc_pass(const SparseKL& s, const float* Wd, const float* Hd, const float* Hbase,
                     const float* den, float* Hout, double* lossPart, int* status, cudaStream_t st) {
  if (s.K <= 32) return csc_pass_kj<1, COMPUTE, OUT>(s, Wd, Hd, Hbase, den, Hout, lossPart, status, st);
  if (s.K <= 64) return csc_pass_kj<2, COMPUTE, OUT>(s, Wd, Hd, Hbase, den, Hout, lossPart, status, st);
  return csc_pass_kj<4, COMPUTE, OUT>(s, Wd, Hd, Hbase, den, Hout, lossPart, status, st);
}

cudaError_t transpose(const float* H, int K, int64_t N, float* HT, const int* status, cudaStream_t st) {
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(H, K, N, HT, status);
  return cudaGetLastError();
}

#define SP_TRY(x)                                 \
  do {                                            \
    cudaError_t _e = (x);                         \
    if (_e != cudaSuccess) return _e;             \
  } while (0)

}  // namespace

size_t sparse_csc_tmp_bytes(int64_t, int64_t N, int64_t) { return sizeof(int32_t) * (2 * (N + 1) + 4); }

// Builds row indices and the CSC copy. Returns cudaErrorInvalidValue (no
// kernel past validation touches an index) when the CSR arrays are malformed.
cudaError_t sparse_build_csc(SparseKL& s, void* tmp, size_t, cudaStream_t st) {
  int32_t* cnt = static_cast<int32_t*>(tmp);
  int32_t* cursor = cnt + (s.N + 1);
  int* bad = reinterpret_cast<int*>(cursor + (s.N + 1));
  SP_TRY(cudaMemsetAsync(tmp, 0, sizeof(int32_t) * (2 * (s.N + 1) + 4), st));
  const int64_t nv = std::max<int64_t>(s.F + 1, s.nnz);
  validate_csr_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(s.rowptr, s.col, s.F, s.N, s.nnz, bad);
  SP_TRY(cudaGetLastError());
  int hbad = 0;
  SP_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  SP_TRY(cudaStreamSynchronize(st));
  if (hbad) return cudaErrorInvalidValue;
  fill_rowidx_kernel<<<(unsigned)((s.F + 255) / 256), 256, 0, st>>>(s.rowptr, s.F, s.rowidx, bad);
  SP_TRY(cudaGetLastError());
  if (s.nnz > 0) {
    count_cols_kernel<<<(unsigned)((s.nnz + 255) / 256), 256, 0, st>>>(s.col, s.nnz, cnt, bad);
    SP_TRY(cudaGetLastError());
  }
  scan_kernel<<<1, 1024, 0, st>>>(cnt, s.N, s.colptr);
  SP_TRY(cudaGetLastError());
  if (s.nnz > 0) {
    scatter_kernel<<<(unsigned)((s.nnz + 255) / 256), 256, 0, st>>>(s.col, s.rowidx, s.nnz, s.colptr, cursor,
                                                                     s.cscRow, s.cscPos, bad);
    SP_TRY(cudaGetLastError());
  }
  sort_cols_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, st>>>(s.colptr, s.N, s.cscRow, s.cscPos);
  return cudaGetLastError();
}

// One outer iteration. Ht buffer: [0, KN) = tilde H row-major, [KN, 2KN) = a transposed
// copy (N x K) of whichever H the CSR pass gathers from.
cudaError_t sparse_step(SparseKL& s, float* W, float* H, bool joint, bool hfirst, bool wantLoss,
                        bool normalize, int* status, Timer* tm, cudaStream_t st) {
  const int K = s.K;
  const int64_t F = s.F, N = s.N, FK = F * K, KN = (int64_t)K * N;
  float* HtRM = s.Ht;
  float* HxT = s.Ht + KN;
  float* colsumW = s.colsumW;
  float* rowsumH = s.rowsumH;
  float* chi = s.chi;
  float* norms = s.chi + K;
  const unsigned cgrid = (unsigned)std::min<int64_t>(4096, (FK + KN + 255) / 256);
  auto launch = [](auto&& body) { body(); return cudaGetLastError(); };
#define SP_T(name, n, ...) SP_TRY(timed(tm, st, name, n, [&] { return launch([&] { __VA_ARGS__; }); }))
  // begin: tilde copies, transposed H, sums at the iterate
  SP_T("sp_begin", 5,
       copy_kernel<<<(unsigned)std::min<int64_t>(4096, (FK + 255) / 256), 256, 0, st>>>(W, s.Wt, FK, status);
       copy_kernel<<<(unsigned)std::min<int64_t>(4096, (KN + 255) / 256), 256, 0, st>>>(H, HtRM, KN, status);
       transpose(H, K, N, HxT, status, st);
       colsum_kernel<<<K, 256, 0, st>>>(W, F, K, colsumW, 0, status);
       rowsum_kernel<<<K, 256, 0, st>>>(H, K, N, rowsumH, status));
  double* lp = wantLoss ? s.lossPart : nullptr;
  int nbLoss = 0;
  if (joint) {
    if (!hfirst) {
      // W half: W = Wt . (A Ht^T) / rowsum(Ht)   (chi_2(Ht, Ht) = Ht)
      SP_TRY(timed(tm, st, "sp_csr_pass", 1, [&] { return csr_pass<true, OUT_UPDATE>(s, s.Wt, HxT, s.Wt, rowsumH, W, lp, status, st); }));
      nbLoss = (int)((F + WPB - 1) / WPB);
      // H half: H = Ht . (Wt^T A) / colsum(W)    (chi_1(W, Wt) = Wt, chi_2(W, Wt) = W)
      SP_T("sp_sums", 1, colsum_kernel<<<K, 256, 0, st>>>(W, F, K, chi, 0, status));
      SP_TRY(timed(tm, st, "sp_csc_pass", 1, [&] { return csc_pass<false, OUT_UPDATE>(s, s.Wt, nullptr, HtRM, chi, H, nullptr, status, st); }));
    } else {
      // H half: H = Ht . (Wt^T A) / colsum(Wt)
      SP_TRY(timed(tm, st, "sp_csc_pass", 1, [&] { return csc_pass<true, OUT_UPDATE>(s, s.Wt, HtRM, HtRM, colsumW, H, lp, status, st); }));
      nbLoss = (int)((N + CB - 1) / CB);
      // W half: W = Wt . (A Ht^T) / rowsum(H)    (chi_1(H, Ht) = Ht, chi_2(H, Ht) = H)
      SP_T("sp_sums", 1, rowsum_kernel<<<K, 256, 0, st>>>(H, K, N, chi, status));
      SP_TRY(timed(tm, st, "sp_csr_pass", 1, [&] { return csr_pass<false, OUT_UPDATE>(s, nullptr, HxT, s.Wt, chi, W, nullptr, status, st); }));
    }
  } else {
    if (!hfirst) {
      SP_TRY(timed(tm, st, "sp_csr_pass", 1, [&] { return csr_pass<true, OUT_UPDATE>(s, s.Wt, HxT, s.Wt, rowsumH, W, lp, status, st); }));
      nbLoss = (int)((F + WPB - 1) / WPB);
      SP_T("sp_sums", 1, colsum_kernel<<<K, 256, 0, st>>>(W, F, K, chi, 0, status));
      // product recomputed with the new W (Algorithm 1)
      SP_TRY(timed(tm, st, "sp_csc_pass", 1, [&] { return csc_pass<true, OUT_UPDATE>(s, W, HtRM, HtRM, chi, H, nullptr, status, st); }));
    } else {
      SP_TRY(timed(tm, st, "sp_csc_pass", 1, [&] { return csc_pass<true, OUT_UPDATE>(s, s.Wt, HtRM, HtRM, colsumW, H, lp, status, st); }));
      nbLoss = (int)((N + CB - 1) / CB);
      SP_T("sp_sums", 2, rowsum_kernel<<<K, 256, 0, st>>>(H, K, N, chi, status); transpose(H, K, N, HxT, status, st));
      SP_TRY(timed(tm, st, "sp_csr_pass", 1, [&] { return csr_pass<true, OUT_UPDATE>(s, s.Wt, HxT, s.Wt, chi, W, nullptr, status, st); }));
    }
  }
  if (wantLoss) {
    SP_T("sp_loss_final", 1, sparse_loss_final_kernel<<<1, 256, 0, st>>>(s.lossPart, nbLoss, colsumW, rowsumH, K, s.sums));
  }
  if (normalize) {
    SP_T("sp_normalize", 2,
         colsum_kernel<<<K, 256, 0, st>>>(W, F, K, norms, 1, status);
         scale_kernel<<<cgrid, 256, 0, st>>>(W, F, K, H, N, norms, status));
  }
#undef SP_T
  return cudaSuccess;
}

// Objective at (W, H): the CSR pass evaluates the nonzero terms, the row/column sums the rest.
cudaError_t sparse_loss(SparseKL& s, const float* W, const float* H, double* out, cudaStream_t st) {
  const int K = s.K;
  const int64_t KN = (int64_t)K * s.N;
  float* HxT = s.Ht + KN;
  SP_TRY(transpose(H, K, s.N, HxT, nullptr, st));
  colsum_kernel<<<K, 256, 0, st>>>(W, s.F, K, s.colsumW, 0, nullptr);
  SP_TRY(cudaGetLastError());
  rowsum_kernel<<<K, 256, 0, st>>>(H, K, s.N, s.rowsumH, nullptr);
  SP_TRY(cudaGetLastError());
  // reuse the CSR pass in its loss-only form; it needs a writable status word
  int* zero = reinterpret_cast<int*>(s.sums + 8);
  SP_TRY(cudaMemsetAsync(zero, 0, sizeof(int), st));
  SP_TRY((csr_pass<true, OUT_NONE>(s, W, HxT, nullptr, nullptr, nullptr, s.lossPart, zero, st)));
  sparse_loss_final_kernel<<<1, 256, 0, st>>>(s.lossPart, (int)((s.F + WPB - 1) / WPB), s.colsumW, s.rowsumH,
                                              K, out);
  return cudaGetLastError();
}

// Gradient of D_1(V | WH): gW = 1 H^T - A H^T, gH = W^T 1 - W^T A, A = V / WH (nonzeros).
// Leaves the nonzero loss partials in lossPart for sparse_loss_finalize.
cudaError_t sparse_grad(SparseKL& s, const float* W, const float* H, float* gW, float* gH, cudaStream_t st) {
  const int K = s.K;
  const int64_t KN = (int64_t)K * s.N;
  float* HxT = s.Ht + KN;
  SP_TRY(transpose(H, K, s.N, HxT, nullptr, st));
  colsum_kernel<<<K, 256, 0, st>>>(W, s.F, K, s.colsumW, 0, nullptr);
  SP_TRY(cudaGetLastError());
  rowsum_kernel<<<K, 256, 0, st>>>(H, K, s.N, s.rowsumH, nullptr);
  SP_TRY(cudaGetLastError());
  int* zero = reinterpret_cast<int*>(s.sums + 8);
  SP_TRY(cudaMemsetAsync(zero, 0, sizeof(int), st));
  SP_TRY((csr_pass<true, OUT_GRAD>(s, W, HxT, nullptr, s.rowsumH, gW, s.lossPart, zero, st)));
  SP_TRY((csc_pass<false, OUT_GRAD>(s, W, nullptr, nullptr, s.colsumW, gH, nullptr, zero, st)));
  return cudaSuccess;
}

cudaError_t sparse_loss_finalize(SparseKL& s, const float*, const float*, double* out, cudaStream_t st) {
  sparse_loss_final_kernel<<<1, 256, 0, st>>>(s.lossPart, (int)((s.F + WPB - 1) / WPB), s.colsumW, s.rowsumH,
                                              s.K, out);
  return cudaGetLastError();
}

}  // namespace nmf
