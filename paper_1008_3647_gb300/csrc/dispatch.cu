// Runtime dispatch from the lattice extent N_x to the compiled slice-kernel instantiation.
#include <cstdlib>

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

bool slice_q_supported(int N, int prec, int ntau, int dim) {
  static int env = -1;
  if (env < 0) {
    const char* e = std::getenv("UFG_NO_FUSED_Q");
    const char* t = std::getenv("UFG_NO_TMA");
    env = ((e && e[0] == '1') || (t && t[0] == '1')) ? 0 : 1;
  }
  if (!env || dim != 3 || N != 16 || ntau < 3) return false;
  // one CTA per output slice with three kinetic stages: ahead of the two launches of M and M^T
  // while their slices fill at most about two CTAs per SM (16^3 x 256: 10.6 against 13.4 us in
  // FP32, 183 against 191 us in FP64); behind them on longer lattices (16^3 x 1024 FP32: 23.0
  // against 19.1 us) and on 8^3 slices (FP64 8^3 x 64: 17.3 against 14.7 us)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    sms = v;
  }
  (void)prec;
  return ntau <= 2 * sms;
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
