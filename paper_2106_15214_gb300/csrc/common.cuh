// common.cuh -- device-side building blocks shared by the CUDA kernels of libnmf.
//
// Notation follows the paper (arXiv 2106.15214): V (F x N), W (F x K),
// H (K x N), Vt = Wt Ht the product at the current iterate, and the two
// elementwise terms of eq. alt_update / eq. jnt_update:
//     A = V . Vt^(beta-2)          B = Vt^(beta-1) = Vt . Vt^(beta-2)
// B is formed as Vt times the same power so that V == Vt gives A == B.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace nmf {

// Compile-time specialisation of beta. The paper singles out beta = 0, 1, 2
// (Table 2); beta = 1.5 is the hyperspectral case of Sec. 4.5.
enum BetaKind : int { BK_GENERAL = 0, BK_IS = 1, BK_KL = 2, BK_EUC = 3, BK_B15 = 4 };

inline int beta_kind(double beta) {
  if (beta == 0.0) return BK_IS;
  if (beta == 1.0) return BK_KL;
  if (beta == 2.0) return BK_EUC;
  if (beta == 1.5) return BK_B15;
  return BK_GENERAL;
}

// gamma(beta), eq. def_gamma.
inline double gamma_of(double beta) {
  if (beta < 1.0) return 1.0 / (2.0 - beta);
  if (beta <= 2.0) return 1.0;
  return 1.0 / (beta - 1.0);
}

struct BetaParams {
  double beta;
  double gamma;
  double kappa;
  double floor = 0.0;  // every update is clamped to >= floor (0: off)
  int kind;
  float series[7];  // Taylor coefficients of phi_beta(u) for u^2 .. u^8 (fill_series)
  float tiny = 0.f; // small-Vt guard threshold of the single-precision kernels (fill_series)
};

// phi_b(u) = ((1+u)^b - 1 - b u) / (b (b-1)) = sum_{j>=2} c_j u^j with
// c_2 = 1/2 and c_{j+1} = c_j (b - j) / (j + 1); computed once on the host.
//
// Also the small-Vt guard threshold (not in the paper; the precision pattern
// asks for it): in single precision the power Vt^(beta-2) overflows once
// Vt < FLT_MAX^(-1/(2-beta)) (beta < 2), and the hardware reciprocal,
// logarithm and reciprocal square root flush subnormal Vt to zero, although
// A = V Vt^(beta-2) and B = Vt^(beta-1) may still be representable. Entries
// with Vt below 2^max(-125, -120/(2-beta)) (beta < 2; 2^-125 for beta > 2;
// no guard at beta = 2, where A = V and B = Vt) take their powers and their
// objective term in FP64 instead. At beta = 0 this is Vt < 2^-60.
inline void fill_series(BetaParams& bp) {
  double c = 0.5;
  for (int j = 2; j <= 8; ++j) {
    bp.series[j - 2] = (float)c;
    c *= (bp.beta - (double)j) / (double)(j + 1);
  }
  double e = -125.0;
  if (bp.beta < 2.0) e = -120.0 / (2.0 - bp.beta) > e ? -120.0 / (2.0 - bp.beta) : e;
  bp.tiny = bp.beta == 2.0 ? 0.f : (float)std::ldexp(1.0, (int)std::floor(e));
}

// One problem of a (possibly batched) context. Every pointer is device memory.
template <typename T>
struct Prob {
  const T* V;
  int64_t ldv;
  T* W;       // current W (in/out)
  T* H;       // current H (in/out)
  T* Wt;      // W at the start of the outer iteration (tilde point)
  T* Ht;      // H at the start of the outer iteration
  T* chiW1;   // chi_1(W, Wt), F x K
  T* chiW2;   // chi_2(W, Wt), F x K
  T* chiH1;   // chi_1(H, Ht), K x N
  T* chiH2;   // chi_2(H, Ht), K x N
  T* rowPart; // [S][2][F][K] partial numerators/denominators of the W half
  T* colPart; // [R][2][K][N] partial numerators/denominators of the H half
  T* norms;   // K column norms of W
  int64_t F, N;
  int K;
  int S;             // column chunks of a row sweep
  int R;             // row chunks of a column sweep
  int rowTilesF;     // ceil(F / BF)
  int colTilesN;     // ceil(N / BN)
  int64_t chunkN;    // columns per row-sweep chunk (multiple of BN)
  int64_t chunkF;    // rows per column-sweep chunk (multiple of BF)
  // tensor-core sweeps (single problems): 128-row / 128-column MMA tiles
  int tcRowTiles;    // ceil(F / 128)
  int tcS;           // partial slices the tensor-core row sweep writes (blocks / cluster size)
  int tcColTiles;    // ceil(N / 128)
  int tcR;           // partial slices the tensor-core column sweep writes
  int tcSplitS;      // blocks along N per row tile (padded to a multiple of tcClusterS)
  int tcClusterS;    // blocks of one cluster, combined through distributed shared memory
  int tcSplitR;      // blocks along F per column tile (padded to a multiple of tcClusterR)
  int tcClusterR;
  int tcSK;          // 1: the column sweep is split stream-K (below), tcR = most slices of any column tile
  int tcSKBlocks;    // blocks of the stream-K column sweep
  int fuS = 1;       // partial slices of the fused single-read sweep (its clusters)
  int64_t tcChunkN;  // multiple of 32
  int64_t tcChunkF;  // multiple of 32
  // TF32-rounded, zero-padded operand copies read by TMA in the tensor-core
  // sweeps (null outside tensor-core contexts). kp = K rounded up to 16,
  // ks = kp rounded up to 32, Fp / Np = F / N rounded up to 4 (16-byte rows).
  T* sWS;    // [F][ks]  W
  T* sWT;    // [kp][Fp] W transposed
  T* sHT;    // [N][ks]  H transposed
  T* sHS;    // [kp][Np] H
  T* sCW1;   // [kp][Fp] chi_1(W, Wt) transposed
  T* sCW2;   // [kp][Fp] chi_2(W, Wt) transposed
  T* sCH1;   // [kp][Np] chi_1(H, Ht)
  T* sCH2;   // [kp][Np] chi_2(H, Ht)
  int kp, ks;
  int64_t Fp, Np;
};

// Stream-K split of the tensor-core column sweep: its T = tiles x ft tile
// steps (ft = ceil(F / 32) per column tile, tile-major) are cut into G equal
// contiguous ranges, block g taking [floor(g T / G), floor((g + 1) T / G)).
// A column tile is then covered by a few consecutive blocks; block g writes
// its part of tile nt into slice g - first block of nt.
__host__ __device__ inline int64_t sk_block_of(int64_t step, int64_t T, int64_t G) { return ((step + 1) * G - 1) / T; }
__host__ __device__ inline int sk_slices(int64_t nt, int64_t ft, int64_t T, int64_t G) {
  return (int)(sk_block_of((nt + 1) * ft - 1, T, G) - sk_block_of(nt * ft, T, G) + 1);
}


// Finds the problem owning linear block index `b` given an exclusive prefix
// table of block counts (prefix[count] = total).
__device__ __forceinline__ int find_problem(const int* prefix, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Elementwise terms
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float pow_t(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double pow_t(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

// A = v . vt^(beta-2), B = vt . vt^(beta-2) (v and vt already include kappa).
template <int BK, typename T>
__device__ __forceinline__ void ab_terms(T v, T vt, T bm2, T& A, T& B) {
  if (BK == BK_KL) {
    A = v / vt;
    B = T(1);
  } else if (BK == BK_EUC) {
    A = v;
    B = vt;
  } else if (BK == BK_IS) {
    T r = T(1) / vt;
    B = r;
    A = v * r * r;
  } else if (BK == BK_B15) {
    T r = rsqrt_t(vt);
    A = v * r;
    B = vt * r;
  } else {
    T p = pow_t(vt, bm2);
    A = v * p;
    B = vt * p;
  }
}

// ab_terms with the small-Vt guard (fill_series): float entries whose
// product lies below bp.tiny take their powers in FP64 (rare; a warp-uniform
// branch in the common case). Double is unguarded.
template <int BK>
__device__ __forceinline__ void ab_terms_g(double v, double vt, double bm2, double& A, double& B, float) {
  ab_terms<BK, double>(v, vt, bm2, A, B);
}
template <int BK>
__device__ __forceinline__ void ab_terms_g(float v, float vt, float bm2, float& A, float& B, float tiny) {
  if (vt < tiny) {
    double a, b;
    ab_terms<BK, double>((double)v, (double)vt, (double)bm2, a, b);
    A = (float)a;
    B = (float)b;
  } else {
    ab_terms<BK, float>(v, vt, bm2, A, B);
  }
}

// An update clamped to eps: over x >= eps the minimiser of the per-entry
// convex auxiliary function is the unconstrained one clamped to eps (the
// positivity constraint W, H >= eps of eqs. Wll, Hll). NaN stays NaN, so the
// non-finite check still sees it; eps = 0 leaves x unchanged.
template <typename T>
__device__ __forceinline__ T apply_floor(T x, T eps) { return x < eps ? eps : x; }

// (num / den)^gamma
template <int BK, typename T>
__device__ __forceinline__ T mu_ratio(T num, T den, T gamma) {
  T r = num / den;
  if (BK == BK_KL || BK == BK_EUC || BK == BK_B15) return r;  // gamma = 1 on [1, 2]
  if (BK == BK_IS) return sqrt_t(r);                           // gamma = 1/2
  return pow_t(r, gamma);
}

// chi_1(x, xt) and chi_2(x, xt) of eq. jnt_update, written with rho = x / xt:
//   chi_1 = xt^(2-b) / x^(1-b) = xt rho^(b-1)   (b <= 2),   x   (b > 2)
//   chi_2 = x                                    (b < 1),    x^b / xt^(b-1) = xt rho^b (b >= 1)
template <int BK, typename T>
__device__ __forceinline__ void chi_terms(T x, T xt, T beta, T& c1, T& c2) {
  if (BK == BK_KL) { c1 = xt; c2 = x; return; }
  if (BK == BK_EUC) { c1 = x; c2 = x * (x / xt); return; }
  if (BK == BK_IS) { c1 = xt * (xt / x); c2 = x; return; }
  T rho = x / xt;
  if (BK == BK_B15) { c1 = xt * sqrt_t(rho); c2 = x * sqrt_t(rho); return; }
  c1 = (beta <= T(2)) ? xt * pow_t(rho, beta - T(1)) : x;
  c2 = (beta < T(1)) ? x : xt * pow_t(rho, beta);
}

// d_beta(x | y), eq. beta-div. Double: the formula as printed (0 log 0 = 0).
__device__ __forceinline__ double dbeta_direct(double x, double y, double beta, int bk) {
  if (bk == BK_KL) return (x > 0.0 ? x * log(x / y) : 0.0) - x + y;
  if (bk == BK_IS) { double r = x / y; return r - log(r) - 1.0; }
  if (bk == BK_EUC) { double d = x - y; return 0.5 * d * d; }
  return pow(x, beta) / (beta * (beta - 1.0)) + pow(y, beta) / beta
         - x * pow(y, beta - 1.0) / (beta - 1.0);
}

// Float: d = y^b phi_b(u) with u = x/y - 1 and
// phi_b(u) = ((1+u)^b - 1 - b u) / (b (b-1)); near u = 0 the Taylor series
// u^2/2 + (b-2)u^3/6 + (b-2)(b-3)u^4/24 + ... (coefficients in bp.series)
// avoids the cancellation that the printed formula suffers in single
// precision. beta = 1 and 0 are the limits (1+u) log1p(u) - u and u - log1p(u).
__device__ __forceinline__ float series_phi(float u, const float* c) {
  float s = c[6];
  #pragma unroll
  for (int j = 5; j >= 0; --j) s = fmaf(s, u, c[j]);
  return s * u * u;
}
__device__ __forceinline__ float dbeta_stable(float x, float y, float beta, int bk, const float* c) {
  if (bk == BK_EUC) { float d = x - y; return 0.5f * d * d; }
  if (bk == BK_KL && x <= 0.0f) return y;
  float u = (x - y) / y;
  float phi;
  if (fabsf(u) < 0.1f) {
    phi = series_phi(u, c);
  } else {
    // log(x / y): log1p of u where x - y is exact (y / 2 <= x <= 2 y), else the
    // log of the ratio itself; u = x / y - 1 rounds to -1 once x / y < 2^-24
    // and log1p(u) would turn into -inf
    const float r = x / y;
    const float lr = (r >= 0.5f && r <= 2.0f) ? log1pf(u) : logf(r);
    if (bk == BK_KL) phi = r * lr - u;
    else if (bk == BK_IS) phi = u - lr;
    else phi = (expm1f(beta * lr) - beta * u) / (beta * (beta - 1.0f));
  }
  float yb = (bk == BK_KL) ? y : (bk == BK_IS ? 1.0f : powf(y, beta));
  return yb * phi;
}

// Round to the nearest TF32 value (10-bit mantissa), kept in the container type.
// Nearest value with a 10-bit mantissa, ties away from zero (the rounding of
// cvt.rna.tf32.f32, done with integer operations; Inf and NaN unchanged).
__device__ __forceinline__ float tf32_round(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t r = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float((u & 0x7F800000u) == 0x7F800000u ? u : r);
}
__device__ __forceinline__ double tf32_round(double x) { return (double)tf32_round((float)x); }

// ---- hardware approximations for the TF32 tensor-core path -------------------
// (the operands there are rounded to 10-bit mantissas, far coarser than these)
__device__ __forceinline__ float rcp_fast(float x) { float r; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float lg2_fast(float x) { float r; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float ex2_fast(float x) { float r; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float rsqrt_fast(float x) { float r; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }

template <int BK>
__device__ __forceinline__ void ab_terms_fast(float v, float vt, float bm2, float& A, float& B) {
  if (BK == BK_KL) { A = v * rcp_fast(vt); B = 1.f; }
  else if (BK == BK_EUC) { A = v; B = vt; }
  else if (BK == BK_IS) { const float r = rcp_fast(vt); B = r; A = v * r * r; }
  else if (BK == BK_B15) { const float r = rsqrt_fast(vt); A = v * r; B = vt * r; }
  else { const float p = ex2_fast(bm2 * lg2_fast(vt)); A = v * p; B = vt * p; }
}

// The objective's terms for the tensor-core path, branch-free, with the
// approximations above (natural log = lg2 * ln 2). There Vt carries TF32
// rounding (relative ~1e-3), so each term is already uncertain by about
// |u| 1e-3 with u = x / y - 1; the direct forms' cancellation error near
// u = 0 (about 2e-7 absolute) is far below that, and the small-|u| series of
// dbeta_stable would only make warps diverge.
template <int BK>
__device__ __forceinline__ float dbeta_fast(float x, float y, float beta, const float* c) {
  (void)c;
  constexpr float LN2 = 0.69314718056f;
  if (BK == BK_EUC) { const float d = x - y; return 0.5f * d * d; }
  if (BK == BK_KL && x <= 0.0f) return y;
  // the logarithm of the ratio itself: 1 + (x - y) / y rounds to 0 once x / y
  // < 2^-24, which would make the term infinite
  const float r = x * rcp_fast(y), u = r - 1.0f, lr = LN2 * lg2_fast(r);
  float phi;
  if (BK == BK_KL) phi = r * lr - u;
  else if (BK == BK_IS) phi = u - lr;
  else phi = (ex2_fast(beta * lg2_fast(r)) - 1.0f - beta * u) * rcp_fast(beta * (beta - 1.0f));
  const float yb = (BK == BK_KL) ? y : (BK == BK_IS ? 1.0f : ex2_fast(beta * lg2_fast(y)));
  return yb * phi;
}

// The tensor-core epilogue's terms of one entry (v, y = Vt, both with kappa):
// A, B and, with the objective, d_beta(v | y) added to tl; the small-Vt guard
// takes entries below bp.tiny to FP64 (powers and objective term).
template <int BK>
__device__ __forceinline__ void epi_terms(float v, float y, float bm2, const BetaParams& bp, bool wantLoss,
                                          float& tl, float& A, float& B) {
  if (y < bp.tiny) {
    double a, b;
    ab_terms<BK, double>((double)v, (double)y, bp.beta - 2.0, a, b);
    A = (float)a;
    B = (float)b;
    if (wantLoss) tl += (float)dbeta_direct((double)v, (double)y, bp.beta, BK);
    return;
  }
  if (wantLoss) tl += dbeta_fast<BK>(v, y, (float)bp.beta, bp.series);
  ab_terms_fast<BK>(v, y, bm2, A, B);
}

template <typename T> struct DB;
template <> struct DB<double> {
  __device__ static double eval(double x, double y, const BetaParams& bp, int bk) { return dbeta_direct(x, y, bp.beta, bk); }
};
template <> struct DB<float> {
  __device__ static double eval(float x, float y, const BetaParams& bp, int bk) {
    if (y < bp.tiny) return dbeta_direct((double)x, (double)y, bp.beta, bk);   // small-Vt guard
    return (double)dbeta_stable(x, y, (float)bp.beta, bk, bp.series);
  }
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch. The step's kernels are launched with the
// programmatic-serialization attribute, so a kernel's blocks may be scheduled
// while its predecessor in the stream is still finishing. pdl_wait() returns
// once that predecessor has completed and its writes are visible (a no-op for
// a normal launch); every such kernel calls it before it touches anything a
// predecessor wrote (the status word included). pdl_trigger() lets the next
// kernel be scheduled as soon as every block of this one has started.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum (any blockDim multiple of 32, <= 1024); result valid in thread 0.
// Float-float (double-single) accumulation: a value carried as hi + lo,
// about 44 significant bits, with single-precision operations only (FP64
// runs at a small fraction of the FP32 rate on GB300). two_sum is Knuth's
// error-free transformation: s + e equals a + b exactly (round-to-nearest
// adds, no reassociation).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (bhi, blo), renormalised so that |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bhi, float blo = 0.f) {
  float s, e;
  two_sum(hi, bhi, s, e);
  e += lo + blo;
  hi = s + e;
  lo = e - (hi - s);
}

// Block sum of float-float values: lane and warp butterflies and the
// cross-warp sum in float-float, converted to double once (thread 0 returns
// it; the butterflies run in a fixed order, so the result is deterministic).
__device__ __forceinline__ double block_sum_ff(float hi, float lo, float2* sh /* >= 32 */) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, oh, ol);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (int)((blockDim.x + 31) >> 5);
  __syncthreads();
  if (l == 0) sh[w] = make_float2(hi, lo);
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const float2 v = l < nw ? sh[l] : make_float2(0.f, 0.f);
    hi = v.x;
    lo = v.y;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
      ff_add(hi, lo, oh, ol);
    }
    if (l == 0) r = (double)hi + (double)lo;
  }
  return r;
}

__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 */) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = (l < nw) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

}  // namespace nmf
