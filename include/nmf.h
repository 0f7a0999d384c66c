/*
 * nmf.h -- C ABI of the GB300 (sm_103a) joint-MM beta-NMF library (libnmf.so).
 *
 * Problem (Sec. 2.1, eq. nmf / obj_fct / beta-div): given a nonnegative
 * F x N matrix V, find nonnegative W (F x K) and H (K x N) minimising
 * D_beta(V | WH) = sum_fn d_beta(v_fn | [WH]_fn).
 *
 * Two iterations are offered on the same data:
 *   - nmf_step_joint:       joint majorisation-minimisation, Algorithm 2 with
 *                           the updates of eq. jnt_update (chi_1, chi_2, gamma
 *                           of eq. def_gamma); Vt = Wt Ht is formed once per
 *                           outer iteration and both factors are rescaled
 *                           from the iterate (Wt, Ht).
 *   - nmf_step_alternating: classic block MM, Algorithm 1 with eq. alt_update;
 *                           WH is recomputed before each factor's update.
 *
 * Layouts: every matrix is row-major. V is F x N with leading dimension ldv
 * (elements, ldv >= N). W is F x K (leading dimension K). H is K x N
 * (leading dimension N). Element type: double for NMF_FP64, float for every
 * other precision.
 *
 * Ownership: V, W, H, gradient outputs and CSR arrays are caller-owned DEVICE
 * buffers that must stay valid while a context uses them; the library only
 * borrows them. W and H are updated in place. The context owns its scratch
 * (tilde copies, partial sums, loss buffers, status word) and frees it in
 * nmf_destroy.
 *
 * Streams: every call is ordered on the stream given to nmf_set_options
 * (default: the legacy default stream). Calls that return a host value
 * (a non-NULL loss_out, nmf_loss, nmf_get_status, nmf_kkt) synchronise that
 * stream; the rest are asynchronous.
 *
 * Errors: every call returns an nmf_status; nothing aborts and no exception
 * crosses the ABI. Invalid sizes, non-finite beta, wrong precision/buffer
 * combinations -> NMF_EINVAL; allocation failure -> NMF_ENOMEM; a CUDA error
 * -> NMF_ECUDA. A non-finite value produced by an update sets a device status
 * word; the kernels of later iterations then do nothing, and the next
 * synchronising call returns NMF_ENONFINITE after restoring W and H to the
 * last finite iterate.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NMF_OK = 0,
  NMF_EINVAL = 1,        /* invalid argument */
  NMF_ENOMEM = 2,        /* device or host allocation failed */
  NMF_ECUDA = 3,         /* a CUDA runtime call failed */
  NMF_ENONFINITE = 4,    /* an update produced Inf/NaN; W, H restored */
  NMF_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  NMF_EUNSUPPORTED = 6,  /* valid request the library does not implement */
  NMF_ENOTREADY = 7      /* data or factors not set yet */
} nmf_status;

typedef enum {
  NMF_FP64 = 0,  /* double storage and arithmetic (SIMT DFMA) */
  NMF_FP32 = 1,  /* float storage and arithmetic (SIMT FFMA) */
  NMF_TF32 = 2,  /* float storage; products on tensor cores (tcgen05 kind::tf32),
                    FP32 accumulation, powers in FP32, loss accumulated in FP64 */
  NMF_BF16 = 3   /* float storage; the fused single-read JMM iteration: the
                    product Vt on tensor cores in TF32 (kind::tf32), A, B,
                    W~ and chi rounded to bf16 for both contractions
                    (kind::f16), FP32 accumulation, powers in FP32, loss in
                    FP64. Dense single problems and batched contexts,
                    nmf_step_joint only, L = 1, NMF_H_FIRST, K <= 32,
                    F <= 1024; anything else returns NMF_EUNSUPPORTED. */
} nmf_precision;

typedef enum {
  NMF_W_FIRST = 0,    /* W then H: the order of Algorithm 2 as printed */
  NMF_H_FIRST = 1,    /* H then W: the inverted order of Sec. 4.1.1 */
  NMF_ORDER_AUTO = 2  /* library picks (W_FIRST when F >= N, else H_FIRST) */
} nmf_order;

typedef struct nmf_ctx nmf_ctx; /* opaque */

/* Creates a context for one F x N problem of rank K with divergence beta
 * (eq. beta-div; any finite beta). F, N, K >= 1, else NMF_EINVAL. Allocates
 * scratch lazily on the first step. Default options: NMF_FP32, NMF_W_FIRST,
 * normalisation on (Sec. 4.1.2), kappa = 0, deterministic reductions, legacy
 * default stream, one sub-iteration (L = 1), the precision's default floor
 * (nmf_set_floor). */
nmf_status nmf_create(int64_t F, int64_t N, int32_t K, double beta, nmf_ctx** out);

/* Creates a context holding `count` independent problems of sizes F[i] x N[i]
 * with ranks K[i] (Sec. 4.5 workload shape); all share beta. Data are given
 * packed by nmf_batch_set_packed. Each problem is iterated exactly as a
 * single-problem context would iterate it. */
nmf_status nmf_batch_create(int32_t count, const int64_t* F, const int64_t* N,
                            const int32_t* K, double beta, nmf_ctx** out);

/* precision: see nmf_precision. order: see nmf_order. normalize != 0 divides
 * each column of W by its l2 norm and scales H's row by it after every outer
 * iteration (Sec. 4.1.2). kappa >= 0 minimises D_beta(V + kappa | WH + kappa)
 * (Sec. 4.1.3). deterministic != 0 requests fixed-order reductions (every
 * path here is deterministic; the flag is accepted for ABI stability).
 * cuda_stream is a cudaStream_t or NULL. Resets scratch if precision changes. */
nmf_status nmf_set_options(nmf_ctx* ctx, nmf_precision precision, nmf_order order,
                           int normalize, double kappa, int deterministic,
                           void* cuda_stream);

/* Floor eps on W and H: every update is clamped to max(update, eps), the
 * minimiser of the auxiliary function under the positivity constraint
 * W, H >= eps of eqs. Wll / Hll (Sec. 3.3.4). eps < 0 restores the default:
 * 0 for NMF_FP64, 1e-30 for single precision (there, entries that the updates
 * drive toward zero would underflow after some hundreds of iterations at
 * beta < 1 and turn chi's ratio into 0 / 0). eps = 0 is the unconstrained
 * method. NaN or Inf: NMF_EINVAL. */
nmf_status nmf_set_floor(nmf_ctx* ctx, double eps);

/* Tile-shape autotuner for the SIMT sweeps (NMF_FP64, NMF_FP32 and batched
 * contexts, whose work items are (problem, chunk of 32-wide tiles)): times
 * `trials` >= 1 joint steps for each cap in {8, 16, 32, 64, 128} on the number
 * of tiles one block sums (more chunks: more, shorter blocks and more partial
 * slices) and keeps the fastest; for a batched NMF_BF16 context the cap sets
 * the length of the fused sweep's work items instead (cap / 4 batches of 128
 * columns per item). W, H and the status word are restored after
 * every trial, so the call leaves the factors as it found them. Choices are
 * cached per process under a shape signature (count, sums of F and N, largest
 * K, beta, precision, SM count); a cached signature returns at once. The cap
 * changes the order of the partial sums, so iterates differ from the default
 * tiling by rounding only. *chunk_cap (nullable) receives the choice; sparse
 * and single-problem tensor-core contexts: NMF_EUNSUPPORTED. Synchronises. */
nmf_status nmf_autotune(nmf_ctx* ctx, int32_t trials, int32_t* chunk_cap);

/* Number L >= 1 of inner passes of Algorithm 2 (and L_W = L_H = L of
 * Algorithm 1) per outer iteration. */
nmf_status nmf_set_subiterations(nmf_ctx* ctx, int32_t L);

/* Borrows dense V (device, F x N row-major, leading dimension ldv >= N).
 * NMF_TF32 / NMF_BF16 contexts whose rows of V are not 16-byte aligned
 * (ldv * 4 not a multiple of 16, or V not 16-byte aligned) read V through a
 * row-padded device copy taken at the first step after this call: call
 * nmf_set_dense again after changing the contents of V. */
nmf_status nmf_set_dense(nmf_ctx* ctx, const void* V_dev, int64_t ldv);

/* Borrows sparse V in CSR form (device arrays): rowptr has F + 1 entries,
 * col and val have nnz entries; columns need not be sorted. Only beta = 1
 * (KL) is supported on sparse data (count data, Sec. 4.4); zeros of V then
 * contribute d_1(0 | [WH]_fn) = [WH]_fn to the objective. Precision must be
 * NMF_FP32. kappa must be 0. The context builds a CSC copy in its scratch. */
nmf_status nmf_set_csr(nmf_ctx* ctx, int64_t nnz, const int32_t* rowptr,
                       const int32_t* col, const float* val);

/* Borrows the factors (device): W F x K, H K x N, updated in place. A step
 * may leave in the context the operand copies of the W and H it returns
 * (NMF_TF32 W first, and NMF_BF16), which the next step then uses instead of
 * copying them again: after writing W or H in place between steps, call nmf_set_factors
 * again (same pointers are fine), which drops those copies and clears the
 * status word. */
nmf_status nmf_set_factors(nmf_ctx* ctx, void* W_dev, void* H_dev);

/* Batched contexts: V, W, H of every problem packed back to back, problem i
 * starting at offset sum_{j<i} F_j N_j (V), sum_{j<i} F_j K_j (W),
 * sum_{j<i} K_j N_j (H); each block row-major as above (ldv = N_i). */
nmf_status nmf_batch_set_packed(nmf_ctx* ctx, const void* V_packed, void* W_packed,
                                void* H_packed);

/* Runs `iters` >= 1 outer iterations of JMM (Algorithm 2). If loss_out is not
 * NULL it receives D_beta(V + kappa | Wt Ht + kappa) at the iterate entering
 * the LAST iteration (computed inside that iteration's first sweep), and the
 * call synchronises. For batched contexts loss_out is the sum over problems. */
nmf_status nmf_step_joint(nmf_ctx* ctx, int32_t iters, double* loss_out);

/* Same as nmf_step_joint for BMM (Algorithm 1). */
nmf_status nmf_step_alternating(nmf_ctx* ctx, int32_t iters, double* loss_out);

/* Asynchronous forms of nmf_step_joint / nmf_step_alternating: the same
 * iterations and the same objective (eq. obj_fct at the iterate entering the
 * last iteration), written to loss_dev, caller-owned DEVICE memory holding one
 * double per problem (a batched context writes its problems' losses in
 * order). Stream-ordered; nothing is copied to the host and nothing
 * synchronises, so a device-side error (non-finite update, timeout) is not
 * returned here: the next synchronising call (nmf_get_status, nmf_loss, a
 * step with a host loss_out) reports it and restores W and H. loss_dev ==
 * NULL -> NMF_EINVAL. */
nmf_status nmf_step_joint_async(nmf_ctx* ctx, int32_t iters, double* loss_dev);
nmf_status nmf_step_alternating_async(nmf_ctx* ctx, int32_t iters, double* loss_dev);

/* D_beta(V + kappa | WH + kappa) at the current factors (eq. obj_fct),
 * accumulated in FP64; synchronises. */
nmf_status nmf_loss(nmf_ctx* ctx, double* out_host);

/* Gradient of D_beta(V + kappa | WH + kappa): gW = [(WH)^(b-2).(WH - V)] H^T
 * (F x K) and gH = W^T [(WH)^(b-2).(WH - V)] (K x N), the terms of the KKT
 * residuals (Sec. 4.1.5); equivalently the MU denominator minus numerator.
 * gW_dev, gH_dev are caller-owned device buffers of the context's element
 * type. If loss_out is not NULL it receives the loss at (W, H) and the call
 * synchronises. NMF_FP64 / NMF_FP32 / NMF_TF32 contexts run the SIMT sweeps
 * (TF32: in FP32); a dense NMF_BF16 context runs the fused single-read sweep
 * in its adjoint mode (one read of V, bf16 contractions: relative error of
 * each of the two terms ~1e-2). */
nmf_status nmf_grad(nmf_ctx* ctx, void* gW_dev, void* gH_dev, double* loss_out);

/* KKT residuals res(W) = ||min{W, gW}||_1 / (FK), res(H) = ||min{H, gH}||_1 / (KN)
 * (Sec. 4.1.5) at the current factors; synchronises. */
nmf_status nmf_kkt(nmf_ctx* ctx, double* resW_host, double* resH_host);

/* Batched contexts: per-problem losses of the last step that requested a
 * loss (count doubles, host). */
nmf_status nmf_batch_get_losses(nmf_ctx* ctx, double* out_host);

/* Synchronises the stream and returns the sticky device status (NMF_OK or
 * NMF_ENONFINITE / NMF_ETIMEOUT), restoring W and H on NMF_ENONFINITE. */
nmf_status nmf_get_status(nmf_ctx* ctx);

/* Host-buffer convenience for end-to-end use: copies V (F x N, packed), W and
 * H from HOST memory (pinned memory is fastest) into context-owned device
 * buffers, runs `iters` JMM iterations, copies W and H back and returns the
 * loss as nmf_step_joint does. Single dense contexts only; the device
 * buffers are allocated on first use and reused. */
nmf_status nmf_step_joint_host(nmf_ctx* ctx, const void* V_host, void* W_host,
                               void* H_host, int32_t iters, double* loss_out);

/* Benchmark support. With enable != 0 the library records a CUDA event pair
 * on the context's stream around every kernel it launches for this context
 * and accumulates the durations per kernel name (adds two event records per
 * launch; off by default). Launch counts are kept either way. */
nmf_status nmf_set_timing(nmf_ctx* ctx, int enable);

/* Timing record i (0-based, in order of first launch): kernel name (static
 * string), number of launches and total device milliseconds since the last
 * nmf_reset_timing. i = -1 returns the total launch count over all kernels in
 * *launches (name "all", total_ms summed). Synchronises the stream.
 * Returns NMF_EINVAL when i is past the last record. */
nmf_status nmf_get_timing(nmf_ctx* ctx, int32_t i, const char** name, int64_t* launches,
                          double* total_ms);

/* Clears the timing records and launch counts. */
nmf_status nmf_reset_timing(nmf_ctx* ctx);

/* Test support for failure detection (the paper has no counterpart). Every
 * device-side wait of the library's persistent kernels gives up after a
 * bounded time, sets the status word to NMF_ETIMEOUT and lets the kernel run
 * to its end without further work; the next synchronising call then returns
 * NMF_ETIMEOUT. This call sets that bound for the grid barriers of the
 * persistent kernels to limit_ns (1e6 .. 1e10 ns; default 1e9) and makes
 * those barriers expect extra_arrivals (0 or 1) arrivals beyond the launched
 * blocks, so that with 1 every such wait runs out (a flag nothing sets): a
 * test can exercise the timeout path without a fault or a hang. Other values
 * -> NMF_EINVAL. Call with (1000000000, 0) to restore the defaults. A status
 * word left at NMF_ETIMEOUT is cleared by nmf_set_factors. */
nmf_status nmf_set_barrier_test(nmf_ctx* ctx, int64_t limit_ns, int32_t extra_arrivals);

/* Objective without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * running while a CUDA stream capture is active, hosts that give the library a
 * fixed memory budget or forbid driver allocations, and latency-critical
 * loops that cannot take cudaMalloc's implicit synchronisation. It computes
 * the same value as nmf_loss, D_beta(V + kappa | WH + kappa) accumulated in
 * FP64, without a context.
 *
 * Arguments: sizes, beta, kappa and precision as for nmf_create and
 * nmf_set_options; precision only selects the element type: NMF_FP64 means
 * double buffers and FP64 arithmetic, every other precision float buffers
 * and the FP32 evaluation that nmf_loss also uses for NMF_TF32 and NMF_BF16
 * contexts. V_dev (F x N, leading dimension ldv >= N), W_dev (F x K) and H_dev
 * (K x N) are caller-owned device inputs, row-major; loss_dev is a
 * caller-owned device double that receives the result. The call is
 * asynchronous on cuda_stream (NULL: legacy default stream): read *loss_dev
 * after synchronising that stream. It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Scratch: a static device array of 512 KB (65536 per-tile partial sums and a
 * counter) that every GPU loading the library holds until the process exits.
 * Limit: ceil(F/32) * ceil(N/32) <= 65536 (for example 8192 x 8192), else
 * NMF_EINVAL and nothing is launched. All calls share the array; calls whose
 * kernels overlap on the GPU (other streams, other host threads) race on it,
 * so serialise them. Every call looks up the array's device address in the
 * current device's context (an allocation-free query, so a device reset is
 * harmless); the first call on a device also loads the library's device code
 * there, so make that first call before any stream capture begins. */
nmf_status nmf_loss_noalloc(int64_t F, int64_t N, int32_t K, double beta, double kappa,
                            nmf_precision precision, const void* V_dev, int64_t ldv,
                            const void* W_dev, const void* H_dev, double* loss_dev,
                            void* cuda_stream);

/* Frees the context and its scratch (not the borrowed buffers). NULL is a no-op. */
void nmf_destroy(nmf_ctx* ctx);

/* Static string naming a status code. */
const char* nmf_status_string(nmf_status s);

#ifdef __cplusplus
}
#endif

#endif /* NMF_GB300_H */
