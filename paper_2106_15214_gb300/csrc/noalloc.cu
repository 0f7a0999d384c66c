// noalloc.cu -- nmf_loss_noalloc: the objective D_beta(V + kappa | WH + kappa)
// without any device allocation.
//
// Why it exists: some callers cannot call cudaMalloc -- code that runs while
// a CUDA stream capture is active (allocation is not permitted there), hosts
// that hand the library a fixed memory budget or their own pool and forbid
// driver allocations, and latency-critical loops where cudaMalloc's implicit
// synchronisation is not acceptable. For them this entry point takes its
// scratch from one file-scope device array instead of a context.
//
// Scratch: kPartials per-tile partial sums (double) and one completion
// counter, in g_loss_scratch (about 512 KB). Every GPU that loads the library
// holds the array until the process exits. All calls share it and it keeps
// the last call's contents; the counter is cleared at the start of every call.
// Calls whose kernels overlap on the GPU (different streams, or the same
// array on one device from several threads) race on it.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "nmf.h"

namespace nmf {
namespace {

constexpr int kTile = 32;                   // tile edge (rows and columns)
constexpr int kThreads = 256;
constexpr int64_t kPartials = 1 << 16;      // largest number of 32 x 32 tiles
constexpr size_t kScratchBytes = sizeof(double) * kPartials + 256;

// Partial sums at offset 0, the completion counter right after them.
static __device__ __align__(256) unsigned char g_loss_scratch[kScratchBytes];

// The device address of the array in the current device's context. Host
// code must not pass the symbol itself to a kernel (it names a host-side
// stand-in), so the address is looked up, with the device current, on every
// call: after a device reset or in a new context the array may sit elsewhere,
// and the lookup allocates nothing. The first lookup on a device loads the
// library's device code there, which is why the first call should come before
// any stream capture.
nmf_status scratch_for_current_device(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return NMF_ECUDA;
  }
  *out = p;
  return NMF_OK;
}

// One block per 32 x 32 tile: the product at each entry (K terms), d_beta,
// a fixed-order block sum into partial[tile]; the last block to finish sums
// all partials in a fixed order into *out and clears the counter.
template <typename T>
__global__ void __launch_bounds__(kThreads)
loss_noalloc_kernel(int64_t F, int64_t N, int K, const T* __restrict__ V, int64_t ldv,
                    const T* __restrict__ W, const T* __restrict__ H, BetaParams bp,
                    double* __restrict__ partial, unsigned int* __restrict__ counter,
                    double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ bool last;
  const int64_t tilesN = (N + kTile - 1) / kTile;
  const int64_t tf = blockIdx.x / tilesN, tn = blockIdx.x % tilesN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T kappa = (T)bp.kappa;
  double acc = 0.0;
  for (int i = 0; i < kTile / 8; ++i) {
    const int64_t f = tf * kTile + warp + 8 * i;
    const int64_t n = tn * kTile + lane;
    if (f < F && n < N) {
      T vt = T(0);
      for (int k = 0; k < K; ++k) vt = fma(W[f * K + k], H[(int64_t)k * N + n], vt);
      acc += (double)DB<T>::eval(V[f * ldv + n] + kappa, vt + kappa, bp, bp.kind);
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = acc;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(&partial[b]);  // other blocks' stores, not L1
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    *out = s;
    *counter = 0u;
  }
}

}  // namespace
}  // namespace nmf

using namespace nmf;

extern "C" nmf_status nmf_loss_noalloc(int64_t F, int64_t N, int32_t K, double beta, double kappa,
                                       nmf_precision precision, const void* V_dev, int64_t ldv,
                                       const void* W_dev, const void* H_dev, double* loss_dev,
                                       void* cuda_stream) {
  if (F < 1 || N < 1 || K < 1 || !std::isfinite(beta) || !(kappa >= 0.0) || !std::isfinite(kappa))
    return NMF_EINVAL;
  if (!V_dev || !W_dev || !H_dev || !loss_dev || ldv < N) return NMF_EINVAL;
  if (precision < NMF_FP64 || precision > NMF_BF16) return NMF_EINVAL;
  const int64_t tiles = ((F + kTile - 1) / kTile) * ((N + kTile - 1) / kTile);
  if (tiles > kPartials) return NMF_EINVAL;  // ceil(F/32) * ceil(N/32) above 65536: beyond the static scratch
  void* base = nullptr;
  nmf_status s = scratch_for_current_device(&base);
  if (s != NMF_OK) return s;
  double* partial = static_cast<double*>(base);
  unsigned int* counter = reinterpret_cast<unsigned int*>(static_cast<char*>(base) + sizeof(double) * kPartials);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) { cudaGetLastError(); return NMF_ECUDA; }
  BetaParams bp;
  bp.beta = beta;
  bp.gamma = gamma_of(beta);
  bp.kappa = kappa;
  bp.floor = 0.0;
  bp.kind = beta_kind(beta);
  fill_series(bp);
  if (precision == NMF_FP64)
    loss_noalloc_kernel<double><<<(unsigned)tiles, kThreads, 0, st>>>(
        F, N, K, static_cast<const double*>(V_dev), ldv, static_cast<const double*>(W_dev),
        static_cast<const double*>(H_dev), bp, partial, counter, loss_dev);
  else
    loss_noalloc_kernel<float><<<(unsigned)tiles, kThreads, 0, st>>>(
        F, N, K, static_cast<const float*>(V_dev), ldv, static_cast<const float*>(W_dev),
        static_cast<const float*>(H_dev), bp, partial, counter, loss_dev);
  if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
  return NMF_OK;
}
