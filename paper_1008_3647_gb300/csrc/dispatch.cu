// Runtime dispatch from the lattice extent N_x to the compiled slice-kernel instantiation.
#include "slice_call.h"

namespace ufg {

bool slice_supported_n(int N) {
  switch (N) {
    case 4: case 6: case 8: case 10: case 12: case 16: case 32: return true;
  }
  return false;
}

bool slice_m1w_supported(int N, int prec) {
  return prec == 1 ? N == 16 : (N == 8 || N == 16);
}

bool slice_tma_prep_supported(int N, int prec, int allow_tma) {
  switch (N) {
    case 4: return slice_tma_prep_ok<4>(prec, allow_tma);
    case 6: return slice_tma_prep_ok<6>(prec, allow_tma);
    case 8: return slice_tma_prep_ok<8>(prec, allow_tma);
    case 10: return slice_tma_prep_ok<10>(prec, allow_tma);
    case 12: return slice_tma_prep_ok<12>(prec, allow_tma);
    case 16: return slice_tma_prep_ok<16>(prec, allow_tma);
    case 32: return slice_tma_prep_ok<32>(prec, allow_tma);
  }
  return false;
}

cudaError_t slice_dispatch(int N, const SliceCall& c, cudaStream_t st) {
  switch (N) {
    case 4: return slice_launch<4>(c, st);
    case 6: return slice_launch<6>(c, st);
    case 8: return slice_launch<8>(c, st);
    case 10: return slice_launch<10>(c, st);
    case 12: return slice_launch<12>(c, st);
    case 16: return slice_launch<16>(c, st);
    case 32: return slice_launch<32>(c, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ufg
