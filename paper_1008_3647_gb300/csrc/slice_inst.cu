// Explicit instantiation of the slice kernels for one lattice extent N = UFG_N (compiled once per
// supported N so the heavy unrolled kernels build in parallel).
#include "slice_kernel.cuh"

#ifndef UFG_N
#error "UFG_N must be defined"
#endif

namespace ufg {
template cudaError_t slice_launch<UFG_N>(const SliceCall& c, cudaStream_t st);
}  // namespace ufg
