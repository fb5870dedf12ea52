// The fused momentum-space operator (slice_m1w_kernel, FULL) on FP64 vectors with double-float
// arithmetic on the FP32 pipe (precision UFG_FP64_EMULATED of ufg_apply_M_momentum).
//
// On GB300 the FP64 pipe issues about 1/76 of the FP32 multiply-add rate and the FP64 operator is
// bound by it.  Here the slice arrives as FP64 TMA boxes as before, every value is turned into a
// double-float pair (hi, lo) on its first read, all six line passes, the multipliers and the
// epilogue run in double-float arithmetic (line_ops.cuh, about 46 significant bits), the
// intermediate slices stay in the same 8-byte shared-memory slots (as float pairs), and the
// result is written back as FP64.  Same operator, same layout and launch shape as the FP64
// kernel: (M x^)_t = x^_t + sgn b .* F(w_{t-1} .* F^T x^_{t-1}) (DIR 0) and its transpose (DIR 1).
// Measured at 16^3 x 256: 70 us against 105 us for the FP64 kernel.  Its error is about
// 2^-46 ||M|| ||x||: too large for a full residual b - M x of a nearly converged system (which
// cancels to 1e-10 of ||b||; the batched solve needed more iterations that way), small enough
// for the incremental reliable updates r -= M d of the batched mixed solve, whose error scales
// with the increment d.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "slice_tma.cuh"

namespace ufg {

template <int N>
struct M1wDfArgs {
  CUtensorMap tm_in, tm_s, tm_k, tm_dot;
  LineCoef<N, dfloat> ci_x, ci_y, ci_z;  // inverse transform, one copy per pass
  LineCoef<N, dfloat> cf_x, cf_y, cf_z;  // forward transform
  const double* bk;
  double* out;
  double a;
  const int* done;
  int exec_if;
  const BatchTile* tiles;
  const BatchProb* probs;
  int scale_by_A;
  int ntau;
  int* err;
  int expire;
  const double* U;
  double full_scale, bU;
  int want_dotP, want_self;
  double* partials;
  int fop;
  DevScalars* scs;
  unsigned* counters;
  int part_base;
};

// a shared-memory slot read as the FP64 value TMA put there, or as the double-float pair a pass
// stored in it
__device__ __forceinline__ dfloat df_ld64(const double* p) { return df_from(*p); }
__device__ __forceinline__ dfloat df_ld(const double* p) {
  return *reinterpret_cast<const dfloat*>(p);
}
__device__ __forceinline__ void df_st(double* p, dfloat v) { *reinterpret_cast<dfloat*>(p) = v; }

template <int N, bool IN_SPEC, bool OUT_SPEC, bool FROM64, bool MUL>
__device__ __forceinline__ void df_xpass(double* xs, const double* mul,
                                         const LineCoef<N, dfloat>& cf) {
  using G = SwzGeom<N, double>;
  for (int r = threadIdx.x; r < N * N; r += TMA_NT) {
    dfloat v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int o = G::off(r, i);
      v[i] = FROM64 ? df_ld64(xs + o) : df_ld(xs + o);
      if constexpr (MUL) v[i] = v[i] * df_ld64(mul + o);
    }
    line_op<N, dfloat, IN_SPEC, OUT_SPEC>(v, cf,
                                          [&](int i, dfloat val) { df_st(xs + G::off(r, i), val); });
  }
}

template <int N, bool IN_SPEC, bool OUT_SPEC>
__device__ __forceinline__ void df_ypass(double* xs, const LineCoef<N, dfloat>& cf) {
  using G = SwzGeom<N, double>;
  for (int l = threadIdx.x; l < N * N; l += TMA_NT) {
    const int p = l / N, x = l - (l / N) * N;
    dfloat v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = df_ld(xs + G::off(p * N + y, x));
    line_op<N, dfloat, IN_SPEC, OUT_SPEC>(
        v, cf, [&](int i, dfloat val) { df_st(xs + G::off(p * N + i, x), val); });
  }
}

// Resident CTAs per SM the register allocation allows: shared memory holds three 32 KB FP64
// boxes for DIR 1 (two CTAs per SM) and two for DIR 0 without a dot operand (three CTAs: 375
// against 417 us per batched update at 16^3 x 256 x 8 than at two)
template <int N, int DIR>
__global__ void __launch_bounds__(TMA_NT, DIR == 0 ? 3 : 2)
slice_m1w_df_kernel(const __grid_constant__ M1wDfArgs<N> A) {
  pdl_begin();
  using G = SwzGeom<N, double>;
  constexpr int NN = N * N;
  constexpr int VOL = N * NN;
  extern __shared__ __align__(1024) unsigned char tma_smem[];
  __shared__ alignas(8) uint64_t bar, bar2;
  __shared__ double red[TMA_NT / 32][2];
  const int tid = threadIdx.x;
  int t_out, ntau;
  size_t off = 0;
  const int* done = A.done;
  double acoef = A.a;
  if (A.tiles != nullptr) {
    const BatchTile tl = A.tiles[blockIdx.x];
    const BatchProb& pr = A.probs[tl.prob];
    t_out = tl.t0;
    ntau = pr.ntau;
    off = (size_t)pr.off;
    done = pr.done;
    if (A.scale_by_A) acoef *= pr.A;
  } else {
    t_out = blockIdx.x;
    ntau = A.ntau;
  }
  if (done != nullptr && A.exec_if >= 0 && *done != A.exec_if) return;
  const int t_in = DIR == 0 ? (t_out == 0 ? ntau - 1 : t_out - 1)
                            : (t_out == ntau - 1 ? 0 : t_out + 1);
  const double sgn = (DIR == 0 ? t_out != 0 : t_out != ntau - 1) ? -1.0 : 1.0;
  const int t_s = DIR == 0 ? t_in : t_out;  // slice of the site multiplier
  unsigned char* const base = tma_smem + ((1024u - (smem_addr(tma_smem) & 1023u)) & 1023u);
  double* const xs = reinterpret_cast<double*>(base);
  double* const ss = xs + VOL;
  double* const ks = ss + VOL;
  double* const ds = ks;  // the dot operand's slice (third box)
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, (uint32_t)(VOL * sizeof(double)) * (DIR == 1 ? 3u : 2u));
    tma_load_rows(xs, &A.tm_in, (int)((off + (size_t)t_in * VOL) / N), &bar);
    tma_load_rows(ss, &A.tm_s, (int)((off + (size_t)t_s * VOL) / N), &bar);
    if (DIR == 1) tma_load_rows(ks, &A.tm_k, 0, &bar);
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0u, TMA_WAIT_LIMIT, A.err);
  if (A.expire && tid == 0) mbar_expire_one_wait(&bar2, EXPIRE_LIMIT, A.err);
  // inverse transform (spectral input, FP64 box); DIR 1 weights the modes by b on the way in
  df_xpass<N, true, false, true, DIR == 1>(xs, ks, A.ci_x);
  __syncthreads();
  df_ypass<N, true, false>(xs, A.ci_y);
  __syncthreads();
  const dfloat f1 = df_from(DIR == 1 ? sgn * acoef : 1.0);
  for (int q = tid; q < NN; q += TMA_NT) {  // z pass, times the site multiplier, in place
    const int y = q / N, x = q - (q / N) * N;
    dfloat v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = df_ld(xs + G::off(z * N + y, x));
    line_op<N, dfloat, true, false>(v, A.ci_z, [&](int zp, dfloat val) {
      const int o = G::off(zp * N + y, x);
      df_st(xs + o, (f1 * df_ld64(ss + o)) * val);
    });
  }
  __syncthreads();
  if (tid == 0) {  // the multiplier and b boxes are free: prefetch the epilogue operands
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int row_out = (int)((off + (size_t)t_out * VOL) / N);
    mbar_expect_tx(&bar, (uint32_t)(VOL * sizeof(double)) * (A.want_dotP ? 2u : 1u));
    tma_load_rows(ss, &A.tm_in, row_out, &bar);
    if (A.want_dotP) tma_load_rows(ds, &A.tm_dot, row_out, &bar);
  }
  // forward transform (spectral output)
  df_xpass<N, false, true, false, false>(xs, nullptr, A.cf_x);
  __syncthreads();
  df_ypass<N, false, true>(xs, A.cf_y);
  __syncthreads();
  const dfloat f2 = df_from(DIR == 0 ? sgn * acoef : 1.0);
  double* const gout = A.out + off + (size_t)t_out * VOL;
  mbar_wait_bounded(&bar, 1u, TMA_WAIT_LIMIT, A.err);
  const size_t so = off + (size_t)t_out * VOL;
  const double* __restrict__ gU = A.U ? A.U + so : nullptr;
  const dfloat fs = df_from(A.full_scale), bU = df_from(A.bU);
  double acc_dot = 0.0, acc_self = 0.0;
  for (int q = tid; q < NN; q += TMA_NT) {
    const int y = q / N, x = q - (q / N) * N;
    dfloat v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = df_ld(xs + G::off(z * N + y, x));
    line_op<N, dfloat, false, true>(v, A.cf_z, [&](int zp, dfloat val) {
      const int g = zp * NN + q;
      const int os = G::off(zp * N + y, x);
      dfloat m = f2 * val;
      if constexpr (DIR == 0) m = m * df_from(__ldg(A.bk + g));
      dfloat o = fs * (m + df_ld64(ss + os));
      if (gU != nullptr) o = fmadd(bU, df_from(__ldg(gU + g)), o);
      const double od = df_to(o);
      gout[g] = od;
      if (A.want_dotP) acc_dot = fma(od, ds[os], acc_dot);
      if (A.want_self) acc_self = fma(od, od, acc_self);
    });
  }
  if (A.want_dotP || A.want_self) {  // one partial pair per CTA, as the other slice kernels
    double pd = acc_dot, ps = acc_self;
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
      for (int w = 0; w < TMA_NT / 32; ++w) {
        d += red[w][0];
        q2 += red[w][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
    if (A.fop >= 0 && A.tiles != nullptr) {
      const int prob = A.tiles[blockIdx.x].prob;
      last_block_update(A.fop, A.scs + prob, A.partials, A.probs[prob].st0 - A.part_base,
                        A.probs[prob].st1 - A.part_base, A.counters + prob);
    }
  }
}

template <int N>
inline void df_coef(LineCoef<N, dfloat>& out, const void* in) {
  const LineCoef<N, double>& cf = *reinterpret_cast<const LineCoef<N, double>*>(in);
  for (int i = 0; i < LineShape<N>::NC; ++i) out.c[i] = df_from(cf.c[i]);
}

template <int N, int DIR>
inline cudaError_t m1w_df_launch(const SliceCall& c, cudaStream_t st) {
  constexpr int VOL = N * N * N;
  M1wDfArgs<N> a;
  std::memset(&a, 0, sizeof(a));
  const long long nelem = c.nelem > 0 ? c.nelem : (long long)c.ntau * VOL;
  if (c.in == nullptr || c.pre == nullptr || c.out == nullptr || c.coef == nullptr ||
      c.coef2 == nullptr || (DIR == 1 ? c.bkpre : c.bkpost) == nullptr ||
      (c.want_dotP && c.dotP == nullptr) || ((c.want_dotP || c.want_self) && !c.partials) ||
      (c.fop >= 0 && (c.tiles == nullptr || c.scs == nullptr || c.counters == nullptr)))
    return cudaErrorInvalidValue;
  if (encode_rows<double>(&a.tm_in, c.in, nelem, N, N * N) != cudaSuccess ||
      encode_rows<double>(&a.tm_s, c.pre, nelem, N, N * N) != cudaSuccess ||
      (DIR == 1 && encode_rows<double>(&a.tm_k, c.bkpre, VOL, N, N * N) != cudaSuccess) ||
      (c.want_dotP && encode_rows<double>(&a.tm_dot, c.dotP, nelem, N, N * N) != cudaSuccess))
    return cudaErrorNotSupported;
  df_coef<N>(a.ci_x, c.coef);
  a.ci_y = a.ci_x;
  a.ci_z = a.ci_x;
  df_coef<N>(a.cf_x, c.coef2);
  a.cf_y = a.cf_x;
  a.cf_z = a.cf_x;
  a.bk = static_cast<const double*>(c.bkpost);
  a.out = static_cast<double*>(c.out);
  a.a = c.a;
  a.done = c.done;
  a.exec_if = c.exec_if;
  a.tiles = c.tiles;
  a.probs = c.probs;
  a.scale_by_A = c.scale_by_A;
  a.ntau = c.ntau;
  a.err = c.err;
  a.expire = take_expired_wait(st);
  a.U = static_cast<const double*>(c.U);
  a.full_scale = c.full_scale;
  a.bU = c.bU;
  a.want_dotP = c.want_dotP;
  a.want_self = c.want_self;
  a.partials = c.partials;
  a.fop = c.fop;
  a.scs = c.scs;
  a.counters = c.counters;
  a.part_base = c.part_base;
  const size_t smem = (size_t)((DIR == 1 || c.want_dotP) ? 3 : 2) * VOL * sizeof(double) + 1024;
  auto kern = slice_m1w_df_kernel<N, DIR>;
  static int configured = 0;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(3 * VOL * sizeof(double) + 1024));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  const int units = c.tiles != nullptr ? c.ntiles : c.ntau;
  if (c.grid_out) *c.grid_out = units;
  return launch_k(kern, dim3(units), dim3(TMA_NT), smem, st, 1, a);
}

// The double-float operator for FP64 N = 8 and 16 (the lattices with the fused FP64 kernel).
template <int N>
cudaError_t m1w_df_try(const SliceCall& c, cudaStream_t st) {
  if constexpr (N == 8 || N == 16) {
    if (c.prec != 0 || !c.m1w_full) return cudaErrorNotSupported;
    return c.shift < 0 ? m1w_df_launch<N, 0>(c, st) : m1w_df_launch<N, 1>(c, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ufg
