// tc_dense.cu -- tensor-core dense JMM path (placeholder until the tcgen05 kernels land).
#include "tc_dense.h"

namespace nmf {

struct TcState { int unused; };

nmf_status tc_create(TcState** out, int64_t, int64_t, int, double, double, bool, int) {
  *out = nullptr;
  return NMF_EUNSUPPORTED;
}
nmf_status tc_step(TcState*, const float*, int64_t, float*, float*, int, bool, bool, bool, int*,
                   double*, Timer*, cudaStream_t) {
  return NMF_EUNSUPPORTED;
}
void tc_destroy(TcState*) {}

}  // namespace nmf
