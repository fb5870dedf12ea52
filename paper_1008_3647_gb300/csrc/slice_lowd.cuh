// Slice kernels of lower-dimensional lattices (N_x^D x N_tau, D = 1 or 2), to which the method
// carries over with only the kinetic factor's dimension changed (Sec. 6): exp(-tau K) = T on a
// 1-D slice and T (x) T on a 2-D slice, with the same line operators, families (kinetic,
// forward / inverse real Fourier transform) and epilogue as the 3-D slice kernels
// (slice_kernel.cuh, run-time epilogue operands).  Layout: slice t holds [y][x] (D = 2) or [x]
// (D = 1), x fastest.  A CTA of 256 threads takes `spc` slices: D = 2 stages them in padded
// shared memory for the x-pass and the y-pass (whose outputs go straight to the epilogue); D = 1
// gives each thread one slice's line.  Single lattices only (no batch tiles, no fused scalar
// step); a slice has at most 32^2 sites, so these kernels are latency-bound by design.
#pragma once
#include <cuda_runtime.h>

#include "slice_kernel.cuh"

namespace ufg {

template <int N, typename R, int D, int FAM>
__global__ void __launch_bounds__(SLICE_NT) slice_lowd_kernel(const __grid_constant__ SliceArgs<N, R> A) {
  pdl_begin();
  static_assert(D == 1 || D == 2, "lower-dimensional slices only");
  constexpr bool IN_SPEC = (FAM == FAM_INV);
  constexpr bool OUT_SPEC = (FAM == FAM_FWD);
  constexpr int VOL = D == 1 ? N : N * N;  // sites per slice
  constexpr int PITCH = N + 1;             // padded row (D = 2)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* const sm = reinterpret_cast<R*>(smem_raw);
  __shared__ double red[SLICE_NT / 32][2];
  const int ntau = A.ntau;
  const int t0 = blockIdx.x * A.spc;
  if (A.done != nullptr && A.exec_if >= 0 && *A.done != A.exec_if) return;
  const int nsl = min(A.spc, ntau - t0);
  const int tid = threadIdx.x;
  auto t_in_of = [&](int t_out) {
    if (A.shift < 0) return t_out == 0 ? ntau - 1 : t_out - 1;
    if (A.shift > 0) return t_out == ntau - 1 ? 0 : t_out + 1;
    return t_out;
  };
  // load-side value: input times the per-site and per-mode multipliers
  auto load = [&](int t_in, int m) {
    const size_t g = (size_t)t_in * VOL + m;
    R v = A.in[g];
    if (A.pre != nullptr) v *= A.pre[g];
    if (A.bkpre != nullptr) v *= A.bkpre[m];
    return v;
  };
  R acc_dot = R(0), acc_self = R(0);
  // the epilogue of every output value (as the 3-D kernels' run-time epilogue)
  auto epi = [&](int t_out, int m, R val) {
    R sgn = R(1);
    if (A.shift < 0 && t_out != 0) sgn = R(-1);
    if (A.shift > 0 && t_out != ntau - 1) sgn = R(-1);
    const size_t g = (size_t)t_out * VOL + m;
    R b = sgn * val;
    if (A.bkpost != nullptr) b *= A.bkpost[m];
    if (A.post != nullptr) b *= A.post[g];
    if (A.post2 != nullptr) b *= A.post2[g];
    if (A.id != nullptr) b += A.id[g];
    R o = R(A.a) * b;
    if (A.U != nullptr) o += R(A.bU) * A.U[g];
    if (A.V != nullptr) o += R(A.cV) * A.V[g];
    A.out[g] = o;
    if (A.want_dotP) acc_dot += o * A.dotP[g];
    if (A.want_self) acc_self += o * o;
  };
  if constexpr (D == 1) {
    for (int s = tid; s < nsl; s += SLICE_NT) {
      const int t_out = t0 + s, t_in = t_in_of(t_out);
      R v[N];
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = load(t_in, i);
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_x, [&](int i, R val) { epi(t_out, i, val); });
    }
  } else {
    for (int e = tid; e < nsl * VOL; e += SLICE_NT) {
      const int s = e / VOL, m = e - (e / VOL) * VOL;
      const int y = m / N, x = m - (m / N) * N;
      sm[(s * N + y) * PITCH + x] = load(t_in_of(t0 + s), m);
    }
    __syncthreads();
    for (int l = tid; l < nsl * N; l += SLICE_NT) {  // x-pass: line (s, y), in place
      R* const row = sm + l * PITCH;
      R v[N];
#pragma unroll
      for (int x = 0; x < N; ++x) v[x] = row[x];
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_x, [&](int i, R val) { row[i] = val; });
    }
    __syncthreads();
    for (int l = tid; l < nsl * N; l += SLICE_NT) {  // y-pass: line (s, x), to the epilogue
      const int s = l / N, x = l - (l / N) * N;
      const R* const col = sm + s * N * PITCH + x;
      R v[N];
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = col[y * PITCH];
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_y,
                                       [&](int i, R val) { epi(t0 + s, i * N + x, val); });
    }
  }
  if (A.want_dotP || A.want_self) {  // one partial pair per CTA, as the other slice kernels
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
      for (int wi = 0; wi < SLICE_NT / 32; ++wi) {
        d += red[wi][0];
        q2 += red[wi][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
  }
}

template <int N, typename R, int D, int FAM>
inline cudaError_t lowd_launch(const SliceCall& c, cudaStream_t st) {
  if (c.tiles != nullptr || c.prep_out != nullptr || c.fop >= 0 || c.in == nullptr ||
      c.out == nullptr || c.coef == nullptr || c.ntau < 1 || (c.want_dotP && c.dotP == nullptr) ||
      ((c.want_dotP || c.want_self) && c.partials == nullptr))
    return cudaErrorInvalidValue;
  SliceArgs<N, R> a;
  fill_args<N, R>(a, c);
  // slices per CTA: one per thread in 1-D (a warp's worth per CTA); in 2-D as many padded
  // slices as fit 48 KB, at most 8
  constexpr size_t slice_bytes = (size_t)N * (N + 1) * sizeof(R);
  int spc = D == 1 ? 32 : (int)(48 * 1024 / slice_bytes);
  if (spc > 8 && D == 2) spc = 8;
  if (spc < 1) spc = 1;
  a.spc = spc;
  const size_t smem = D == 2 ? (size_t)spc * slice_bytes : 0;
  auto kern = slice_lowd_kernel<N, R, D, FAM>;
  static int configured = 0;
  if (!configured && smem > 0) {
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  const int grid = (c.ntau + spc - 1) / spc;
  if (c.grid_out) *c.grid_out = grid;
  return launch_k(kern, dim3(grid), dim3(SLICE_NT), smem, st, 1, a);
}

template <int N, typename R, int D>
inline cudaError_t lowd_fam(const SliceCall& c, cudaStream_t st) {
  switch (c.fam) {
    case FAM_KIN: return lowd_launch<N, R, D, FAM_KIN>(c, st);
    case FAM_FWD: return lowd_launch<N, R, D, FAM_FWD>(c, st);
    case FAM_INV: return lowd_launch<N, R, D, FAM_INV>(c, st);
  }
  return cudaErrorNotSupported;  // the fused families are 3-D only
}

// Slice launch of a lattice of dimension c.dim in {1, 2}.
template <int N>
cudaError_t slice_lowd_try(const SliceCall& c, cudaStream_t st) {
  if (c.dim == 1) return c.prec ? lowd_fam<N, float, 1>(c, st) : lowd_fam<N, double, 1>(c, st);
  if (c.dim == 2) return c.prec ? lowd_fam<N, float, 2>(c, st) : lowd_fam<N, double, 2>(c, st);
  return cudaErrorInvalidValue;
}

}  // namespace ufg
