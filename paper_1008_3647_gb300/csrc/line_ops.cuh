// Register-resident 1-D line operators used by every slice kernel.
//
// The kinetic factor exp(-tau K) of the unitary-Fermi-gas fermion matrix (Sec. 1: K diagonal in
// momentum space, k_i = 2 pi n_i / N_x) is separable on the cubic lattice: exp(-tau K) = T (x) T (x) T
// where T is a real symmetric circulant N_x x N_x matrix.  Every operator applied along a line here
// (T itself, the real orthonormal Fourier basis F and its transpose) commutes with the reflection
// x -> -x (mod N), so a line v splits into an even part e (N/2+1 values) and an odd part o (N/2-1
// values) that the operator maps independently: (N/2+1)^2 + (N/2-1)^2 multiply-adds per line instead
// of N^2.
//
//   REAL input : e_0 = v_0, e_H = v_H, e_j = v_j + v_{N-j}, o_j = v_j - v_{N-j}   (H = N/2, 1<=j<H)
//   SPEC input : e_j = v_j (j = 0..H), o_j = v_{H+j}  (cosine slots, then sine slots)
//   REAL output: y_0 = E_0, y_H = E_H, y_i = E_i + O_i, y_{N-i} = E_i - O_i
//   SPEC output: y_i = E_i (i = 0..H), y_{H+i} = O_i
//
// The reduced matrices ce ((H+1)^2) and co ((H-1)^2) are built on the host in FP64 for each operator
// and live in the kernel's parameter space, so the compiler feeds them to FMA straight from the
// constant bank.
#pragma once
#include <cuda_runtime.h>

namespace ufg {

template <int N, typename R>
struct LineCoef {
  static_assert(N >= 4 && N % 2 == 0, "line operators need an even N >= 4");
  static constexpr int H = N / 2;
  R ce[(H + 1) * (H + 1)];
  R co[(H - 1) * (H - 1)];
};

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Applies the reduced operator to the line v[0..N) and hands every output (index, value) to st.
template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, class Store>
__device__ __forceinline__ void line_op(const R (&v)[N], const LineCoef<N, R>& c, Store&& st) {
  constexpr int H = N / 2;
  R e[H + 1];
  R o[H - 1];
  if constexpr (IN_SPEC) {
#pragma unroll
    for (int j = 0; j <= H; ++j) e[j] = v[j];
#pragma unroll
    for (int j = 1; j < H; ++j) o[j - 1] = v[H + j];
  } else {
    e[0] = v[0];
    e[H] = v[H];
#pragma unroll
    for (int j = 1; j < H; ++j) {
      e[j] = v[j] + v[N - j];
      o[j - 1] = v[j] - v[N - j];
    }
  }
#pragma unroll
  for (int i = 0; i <= H; ++i) {
    R E = c.ce[i * (H + 1)] * e[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) E = fmadd(c.ce[i * (H + 1) + j], e[j], E);
    if (i == 0 || i == H) {
      st(i, E);
    } else {
      R O = c.co[(i - 1) * (H - 1)] * o[0];
#pragma unroll
      for (int j = 2; j < H; ++j) O = fmadd(c.co[(i - 1) * (H - 1) + j - 1], o[j - 1], O);
      if constexpr (OUT_SPEC) {
        st(i, E);
        st(H + i, O);
      } else {
        st(i, E + O);
        st(N - i, E - O);
      }
    }
  }
}

}  // namespace ufg
