// tc_dense.h -- tensor-core (tcgen05) dense JMM path for float storage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "nmf.h"

namespace nmf {

struct TcState;

// Returns NMF_EUNSUPPORTED for shapes/beta the tensor-core kernels do not cover.
nmf_status tc_create(TcState** out, int64_t F, int64_t N, int K, double beta, double kappa,
                     bool bf16, int sms);
// `iters` outer JMM iterations (L = 1) on V (F x N, leading dim ldv), W, H in place.
// With want_loss, d_loss[0] receives D_beta at the iterate entering the last iteration.
nmf_status tc_step(TcState* s, const float* V, int64_t ldv, float* W, float* H, int iters,
                   bool want_loss, bool normalize, bool hfirst, int* d_status, double* d_loss,
                   Timer* tm, cudaStream_t st);
void tc_destroy(TcState* s);

}  // namespace nmf
