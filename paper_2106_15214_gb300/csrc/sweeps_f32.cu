// SIMT dense kernels instantiated for float (NMF_FP32).
#include "sweeps_impl.cuh"
namespace nmf {
NMF_INSTANTIATE_SWEEPS(float)
}  // namespace nmf
