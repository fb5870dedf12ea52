// Type-erased description of one fused slice-kernel launch (see slice_kernel.cuh).
#pragma once
#include <cuda_runtime.h>

namespace ufg {

enum SliceFamily { FAM_KIN = 0, FAM_FWD = 1, FAM_INV = 2 };

// Runtime description of one slice launch (host side, type-erased pointers).
struct SliceCall {
  int fam = FAM_KIN;
  int prec = 0;               // 0 = FP64, 1 = FP32
  const void* coef = nullptr; // host LineCoef<N, R> for (fam, prec)
  const void* in = nullptr;
  const void* pre = nullptr;     // per-site load multiplier [S]
  const void* bkpre = nullptr;   // per-mode load multiplier [V]
  const void* bkpost = nullptr;  // per-mode output multiplier [V]
  void* out = nullptr;
  const void* id = nullptr;
  const void* post = nullptr;
  const void* post2 = nullptr;
  const void* U = nullptr;
  const void* V = nullptr;
  const void* dotP = nullptr;
  double a = 1.0, bU = 0.0, cV = 0.0;
  double* partials = nullptr;  // [grid][2] when want_dotP || want_self
  int want_dotP = 0, want_self = 0;
  const int* done = nullptr;   // optional early-exit flag (solver loops)
  int ntau = 0;
  int shift = 0;               // -1: t_in = t_out - 1, +1: t_in = t_out + 1, 0: t_in = t_out
  int spc = 1;                 // time slices per CTA (cluster)
  int C = 1;                   // cluster size (1, 2 or 4; N = 32 only uses 2 or 4)
  int nt = 256;                // threads per CTA (fixed at 256 in this build)
};

// Launches the slice kernel for lattice extent N (explicitly instantiated per N).
template <int N>
cudaError_t slice_launch(const SliceCall& c, cudaStream_t st);

// Runtime dispatch over the supported N (4, 6, 8, 10, 12, 16, 32).
cudaError_t slice_dispatch(int N, const SliceCall& c, cudaStream_t st);
bool slice_supported_n(int N);

}  // namespace ufg
