// Explicit instantiation of the slice kernels for one lattice extent N = UFG_N (compiled once per
// supported N so the heavy unrolled kernels build in parallel).
#include <cstdlib>

#include "slice_df.cuh"
#include "slice_kernel.cuh"
#include "slice_pair.cuh"
#include "slice_lowd.cuh"
#include "slice_q.cuh"
#include "slice_tma.cuh"

#ifndef UFG_N
#error "UFG_N must be defined"
#endif

namespace ufg {

static bool tma_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("UFG_NO_TMA");
    v = (e && e[0] == '1') ? 0 : 1;
  }
  return v == 1;
}

// The TMA-pipelined kernel where it applies, the shared-memory-staged kernel otherwise.
template <>
cudaError_t slice_launch<UFG_N>(const SliceCall& c, cudaStream_t st) {
  if (c.dim != 3) return slice_lowd_try<UFG_N>(c, st);       // 1-D and 2-D lattices
  if (c.fam == FAM_M1W) return slice_m1w_try<UFG_N>(c, st);  // callers check support first
  if (c.fam == FAM_Q) return slice_q_try<UFG_N>(c, st);      // callers check support first
  if (c.allow_tma && tma_enabled()) {
    const cudaError_t e = slice_tma_try<UFG_N>(c, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (c.prep_out != nullptr) return cudaErrorInvalidValue;  // the fused update is TMA-only
  return slice_launch_plain<UFG_N>(c, st);
}

template <>
bool slice_tma_prep_ok<UFG_N>(int prec, int allow_tma) {
  if (!allow_tma || !tma_enabled()) return false;
  return prec == 1 ? (UFG_N == 16 || UFG_N == 32) : (UFG_N == 8 || UFG_N == 16);
}

}  // namespace ufg
