// SIMT dense kernels instantiated for double (NMF_FP64).
#include "sweeps_impl.cuh"
namespace nmf {
NMF_INSTANTIATE_SWEEPS(double)
}  // namespace nmf
