// The normal-equation operator Q = M^T M (Eq. 1) in one kernel per output slice.
//
// With B_t = e^{-tau K} w_t (Sec. 1; T = e^{-tau K} applied by the line operators, w the
// potential) and the antiperiodic signs of Eq. MatrixM,
//   y_s = (M x)_s = x_s + sm(s) T(w_{s-1} x_{s-1}),      sm(s) = -1 except sm(0) = +1,
//   q_t = (M^T y)_t = y_t + st(t) w_t T(y_{t+1}),        st(t) = -1 except st(N_tau - 1) = +1,
// so q_t needs x at t-1, t and t+1 (cyclically).  One CTA per output slice holds those three
// slices as TMA boxes and runs three kinetic stages in place:
//   A: X0 <- x_t + sm(t) T(w_{t-1} X0)          (= y_t)
//   B: X2 <- X2 + sm(t+1) T(w_t X1)             (= y_{t+1})
//   C: q_t = a (X0 + st(t) w_t T(X2)) + bU U + cV V, with the dot partials of the slice kernels.
// Three kinetic stages per slice instead of the two of M followed by M^T, in exchange for one
// launch instead of two and no intermediate vector in memory: at 16^3 the two launches are
// bound by latency (one CTA per slice, few CTAs per SM), not by their bytes.  The multiplier
// rows of the x-passes come from global memory (16-byte loads), the epilogue's w_t per site.
// Built for 16^3 slices (FP32 and FP64); slice_q_supported says where it runs.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "slice_tma.cuh"

namespace ufg {

template <int N, typename R>
struct QArgs {
  CUtensorMap tm_in;  // [rows][N] view of x, box = one slice
  // the kinetic line operator once per pass direction (constant-bank operands, see TmaArgs)
  LineCoef<N, R> cx, cy, cz;
  const R* w;  // the potential w = 1 + A sin(sigma) [S]
  R* out;
  const R* U;
  const R* V;
  const R* dotP;
  double a, bU, cV;
  double* partials;
  int want_dotP, want_self;
  const int* done;
  int exec_if;
  int ntau;
  int* err;
  int expire;  // test hook, see TmaArgs
};

template <int N, typename R>
constexpr int q_min_blocks() {
  // three boxes of one slice: FP32 16^3 48 KB (four CTAs per SM), FP64 16^3 96 KB (two)
  return (3 * N * N * N * (int)sizeof(R) + 1024) <= 56 * 1024 ? 4 : 2;
}

// x-pass in place: rows of X (times the multiplier rows of wg when given)
template <int N, typename R, class CF>
__device__ __forceinline__ void q_xpass(R* X, const R* __restrict__ wg, const CF& cf) {
  using G = SwzGeom<N, R>;
  constexpr int CPR = G::RB / 16, EPC = 16 / (int)sizeof(R);
  for (int r = threadIdx.x; r < N * N; r += TMA_NT) {
    R v[N];
#pragma unroll
    for (int c = 0; c < CPR; ++c) {
      const int o = G::chunk(r, c);
      R vc[EPC];
#pragma unroll
      for (int e = 0; e < EPC; ++e) vc[e] = X[o + e];
      if (wg != nullptr) {
        R wc[EPC];
        ld16(wg + r * N + c * EPC, wc);
        mul_chunk(vc, wc);
      }
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[c * EPC + e] = vc[e];
    }
    swz_store_row<N, R>(X, r, v, cf, false, false);
  }
}

template <int N, typename R, bool UV, bool DOT>
__global__ void __launch_bounds__(TMA_NT, (q_min_blocks<N, R>()))
slice_q_kernel(const __grid_constant__ QArgs<N, R> A) {
  pdl_begin();
  using G = SwzGeom<N, R>;
  constexpr int NN = N * N;
  constexpr int VOL = N * NN;
  static_assert(NN <= TMA_NT, "one row, line and column per thread and pass");
  extern __shared__ __align__(1024) unsigned char tma_smem[];
  __shared__ double red[TMA_NT / 32][2];
  __shared__ alignas(8) uint64_t bar, bar2;
  const int tid = threadIdx.x;
  const int t = blockIdx.x;
  const int ntau = A.ntau;
  if (A.done != nullptr && A.exec_if >= 0 && *A.done != A.exec_if) return;
  const int tm = t == 0 ? ntau - 1 : t - 1;
  const int tp = t == ntau - 1 ? 0 : t + 1;
  const R sA = t != 0 ? R(-1) : R(1);          // sm(t)
  const R sB = tp != 0 ? R(-1) : R(1);         // sm(t+1)
  const R sC = t != ntau - 1 ? R(-1) : R(1);   // st(t)
  unsigned char* const base = tma_smem + ((1024u - (smem_addr(tma_smem) & 1023u)) & 1023u);
  R* const X0 = reinterpret_cast<R*>(base);
  R* const X1 = X0 + VOL;
  R* const X2 = X1 + VOL;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, (uint32_t)(3 * VOL * sizeof(R)));
    tma_load_rows(X0, &A.tm_in, tm * NN, &bar);
    tma_load_rows(X1, &A.tm_in, t * NN, &bar);
    tma_load_rows(X2, &A.tm_in, tp * NN, &bar);
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0u, TMA_WAIT_LIMIT, A.err);
  if (A.expire && tid == 0) mbar_expire_one_wait(&bar2, EXPIRE_LIMIT, A.err);
  const R* const w_tm = A.w + (size_t)tm * VOL;
  const R* const w_t = A.w + (size_t)t * VOL;
  // ---- A: X0 <- x_t + sm(t) T(w_{t-1} x_{t-1}) ----
  q_xpass<N, R>(X0, w_tm, A.cx);
  __syncthreads();
  swz_ypass<N, R, false, false>(X0, A.cy);
  __syncthreads();
  for (int q = tid; q < NN; q += TMA_NT) {
    const int y = q / N, x = q - (q / N) * N;
    R v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = X0[G::off(z * N + y, x)];
    line_op<N, R, false, false>(v, A.cz, [&](int zp, R val) {
      const int o = G::off(zp * N + y, x);
      X0[o] = fmadd(sA, val, X1[o]);
    });
  }
  __syncthreads();
  // ---- B: X2 <- x_{t+1} + sm(t+1) T(w_t x_t) ----
  q_xpass<N, R>(X1, w_t, A.cx);
  __syncthreads();
  swz_ypass<N, R, false, false>(X1, A.cy);
  __syncthreads();
  for (int q = tid; q < NN; q += TMA_NT) {
    const int y = q / N, x = q - (q / N) * N;
    R v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = X1[G::off(z * N + y, x)];
    line_op<N, R, false, false>(v, A.cz, [&](int zp, R val) {
      const int o = G::off(zp * N + y, x);
      X2[o] = fmadd(sB, val, X2[o]);
    });
  }
  __syncthreads();
  // ---- C: q_t = a (y_t + st(t) w_t T(y_{t+1})) + bU U + cV V ----
  q_xpass<N, R>(X2, static_cast<const R*>(nullptr), A.cx);
  __syncthreads();
  swz_ypass<N, R, false, false>(X2, A.cy);
  __syncthreads();
  const size_t obase0 = (size_t)t * VOL;
  const R ra = R(A.a), rbU = R(A.bU), rcV = R(A.cV);
  R acc_dot = R(0), acc_self = R(0);
  for (int q = tid; q < NN; q += TMA_NT) {
    const int y = q / N, x = q - (q / N) * N;
    R v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = X2[G::off(z * N + y, x)];
    const size_t obase = obase0 + q;
    line_op<N, R, false, false>(v, A.cz, [&](int zp, R val) {
      const size_t g = obase + (size_t)zp * NN;
      const int o = G::off(zp * N + y, x);
      R r = ra * fmadd(sC * __ldg(w_t + zp * NN + q), val, X0[o]);
      if constexpr (UV) {
        if (A.U != nullptr) r = fmadd(rbU, __ldg(A.U + g), r);
        if (A.V != nullptr) r = fmadd(rcV, __ldg(A.V + g), r);
      }
      A.out[g] = r;
      if constexpr (DOT) {
        if (A.want_dotP) acc_dot = fmadd(r, __ldg(A.dotP + g), acc_dot);
        if (A.want_self) acc_self = fmadd(r, r, acc_self);
      }
    });
  }
  if constexpr (DOT) {  // one partial pair per CTA, as the slice kernels
    double pd = (double)acc_dot, ps = (double)acc_self;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      pd += __shfl_xor_sync(0xffffffffu, pd, o2);
      ps += __shfl_xor_sync(0xffffffffu, ps, o2);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = pd;
      red[tid >> 5][1] = ps;
    }
    __syncthreads();
    if (tid == 0) {
      double d = 0.0, q2 = 0.0;
      for (int wi = 0; wi < TMA_NT / 32; ++wi) {
        d += red[wi][0];
        q2 += red[wi][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
  }
}

template <int N, typename R, bool UV, bool DOT>
inline cudaError_t q_launch(const SliceCall& c, cudaStream_t st) {
  constexpr int VOL = N * N * N;
  QArgs<N, R> a;
  std::memset(&a, 0, sizeof(a));
  if (c.in == nullptr || c.pre == nullptr || c.out == nullptr || c.coef == nullptr ||
      c.ntau < 3 || c.tiles != nullptr || (c.want_dotP && c.dotP == nullptr) ||
      ((c.want_dotP || c.want_self) && c.partials == nullptr))
    return cudaErrorInvalidValue;
  if (encode_rows<R>(&a.tm_in, c.in, (long long)c.ntau * VOL, N, N * N) != cudaSuccess)
    return cudaErrorNotSupported;
  a.cx = *reinterpret_cast<const LineCoef<N, R>*>(c.coef);
  a.cy = a.cx;
  a.cz = a.cx;
  a.w = static_cast<const R*>(c.pre);
  a.out = static_cast<R*>(c.out);
  a.U = static_cast<const R*>(c.U);
  a.V = static_cast<const R*>(c.V);
  a.dotP = static_cast<const R*>(c.dotP);
  a.a = c.a;
  a.bU = c.bU;
  a.cV = c.cV;
  a.partials = c.partials;
  a.want_dotP = c.want_dotP;
  a.want_self = c.want_self;
  a.done = c.done;
  a.exec_if = c.exec_if;
  a.ntau = c.ntau;
  a.err = c.err;
  a.expire = take_expired_wait(st);
  const size_t smem = 3 * (size_t)VOL * sizeof(R) + 1024;
  auto kern = slice_q_kernel<N, R, UV, DOT>;
  static int configured = 0;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  if (c.grid_out) *c.grid_out = c.ntau;
  return launch_k(kern, dim3(c.ntau), dim3(TMA_NT), smem, st, 1, a);
}

template <int N, typename R>
inline cudaError_t q_launch_epi(const SliceCall& c, cudaStream_t st) {
  const bool uv = c.U != nullptr || c.V != nullptr;
  const bool dot = c.want_dotP || c.want_self;
  if (uv) return dot ? q_launch<N, R, true, true>(c, st) : q_launch<N, R, true, false>(c, st);
  return dot ? q_launch<N, R, false, true>(c, st) : q_launch<N, R, false, false>(c, st);
}

// The fused Q for 16^3 slices (FP32 and FP64), where the one-CTA TMA boxes hold one slice.
template <int N>
cudaError_t slice_q_try(const SliceCall& c, cudaStream_t st) {
  if constexpr (N == 16) {
    return c.prec == 1 ? q_launch_epi<16, float>(c, st) : q_launch_epi<16, double>(c, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ufg
