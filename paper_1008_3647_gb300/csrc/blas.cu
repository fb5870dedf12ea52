// BLAS-1 vector kernels and single-CTA scalar kernels of the Krylov solvers (see blas.cuh).
#include <cmath>
#include <cstdint>

#include "blas.cuh"
#include "scalar_ops.cuh"
#include "ufg_internal.h"
#include "launch.cuh"

namespace ufg {

constexpr int VEC_NT = 256;
static_assert(VEC_NT == SCAL_NT, "fused scalar updates reduce over SCAL_NT threads");

std::string vec_op_name(int op, int prec) {
  static const char* n[] = {"cg_update", "cg_p", "bi_p", "bi_s", "bi_x", "dot", "copy", "zero", "add"};
  return std::string("vec ") + ((op >= 0 && op <= V_ADD) ? n[op] : "?") + (prec ? " f32" : " f64");
}

int vec_op_arrays(int op, bool a_present, bool c_present) {
  switch (op) {
    case V_CG_UPDATE: return 6;  // x, p, r, q read; x, r written
    case V_CG_P: return 3;
    case V_BI_P: return 4;
    case V_BI_S: return 6;       // r, v, x, y read; s, x written
    case V_BI_X: return 7;       // x, z, s, t, rhat read; x, r written
    case V_DOT: return 2 * ((a_present ? 1 : 0) + (c_present ? 1 : 0));
    case V_COPY: return 2;
    case V_ZERO: return 1;
    case V_ADD: return 3;
  }
  return 0;
}

int vec_grid(long long n) {
  long long g = (n + VEC_NT * 4 - 1) / (VEC_NT * 4);
  if (g < 1) g = 1;
  if (g > 152 * 8) g = 152 * 8;
  return (int)g;
}

__device__ __forceinline__ void block_pair_store(double d1, double d2, double* part) {
  __shared__ double red[VEC_NT / 32][2];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    d1 += __shfl_xor_sync(0xffffffffu, d1, off);
    d2 += __shfl_xor_sync(0xffffffffu, d2, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w][0] = d1;
    red[w][1] = d2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < VEC_NT / 32; ++i) {
      a += red[i][0];
      b += red[i][1];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// W consecutive elements (W = 1, or 16 bytes of R) through registers.
template <typename R, int W> struct Pack;
template <typename R> struct Pack<R, 1> {
  __device__ __forceinline__ static void ld(const R* p, R (&o)[1]) { o[0] = *p; }
  __device__ __forceinline__ static void st(R* p, const R (&v)[1]) { *p = v[0]; }
};
template <> struct Pack<float, 4> {
  __device__ __forceinline__ static void ld(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Pack<double, 2> {
  __device__ __forceinline__ static void ld(const double* p, double (&o)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
  __device__ __forceinline__ static void st(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// One BLAS-1 step on elements [i, i + W).  Per-thread partial sums d1, d2 stay in the working
// precision (FP64 arithmetic is slow on this part and a thread sums a few dozen terms); the
// block reduction is FP64.
template <typename R, int OP, int W>
__device__ __forceinline__ void vec_step(long long i, R al, R be, R om, R* a, R* b, R* c, R* d,
                                         R* e, R* f, R& d1, R& d2) {
  using P = Pack<R, W>;
  R A[W], B[W], Cv[W], D[W], E[W], F[W];
  if constexpr (OP == V_CG_UPDATE) {
    P::ld(a + i, A); P::ld(b + i, B); P::ld(c + i, Cv); P::ld(d + i, D);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      A[k] += al * B[k];
      Cv[k] -= al * D[k];
      d2 += Cv[k] * Cv[k];
    }
    P::st(a + i, A); P::st(c + i, Cv);
  } else if constexpr (OP == V_CG_P) {
    P::ld(a + i, A); P::ld(b + i, B);
#pragma unroll
    for (int k = 0; k < W; ++k) A[k] = B[k] + be * A[k];
    P::st(a + i, A);
  } else if constexpr (OP == V_BI_P) {
    P::ld(a + i, A); P::ld(b + i, B); P::ld(c + i, Cv);
#pragma unroll
    for (int k = 0; k < W; ++k) A[k] = B[k] + be * (A[k] - om * Cv[k]);
    P::st(a + i, A);
  } else if constexpr (OP == V_BI_S) {
    P::ld(b + i, B); P::ld(c + i, Cv); P::ld(d + i, D); P::ld(e + i, E);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      A[k] = B[k] - al * Cv[k];
      D[k] += al * E[k];
      d2 += A[k] * A[k];
    }
    P::st(a + i, A); P::st(d + i, D);
  } else if constexpr (OP == V_BI_X) {
    P::ld(a + i, A); P::ld(b + i, B); P::ld(d + i, D); P::ld(e + i, E); P::ld(f + i, F);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      A[k] += om * B[k];
      Cv[k] = D[k] - om * E[k];
      d1 += F[k] * Cv[k];
      d2 += Cv[k] * Cv[k];
    }
    P::st(a + i, A); P::st(c + i, Cv);
  } else if constexpr (OP == V_DOT) {
    if (a != nullptr) {
      P::ld(a + i, A); P::ld(b + i, B);
#pragma unroll
      for (int k = 0; k < W; ++k) d1 += A[k] * B[k];
    }
    if (c != nullptr) {
      P::ld(c + i, Cv); P::ld(d + i, D);
#pragma unroll
      for (int k = 0; k < W; ++k) d2 += Cv[k] * D[k];
    }
  } else if constexpr (OP == V_COPY) {
    P::ld(b + i, B);
    P::st(a + i, B);
  } else if constexpr (OP == V_ZERO) {
#pragma unroll
    for (int k = 0; k < W; ++k) A[k] = R(0);
    P::st(a + i, A);
  } else if constexpr (OP == V_ADD) {
    P::ld(a + i, A); P::ld(b + i, B);
#pragma unroll
    for (int k = 0; k < W; ++k) A[k] += B[k];
    P::st(a + i, A);
  }
}

// VECW: every operand is 16-byte aligned and each CTA's range is a whole number of 16-byte
// vectors (the batched tiles always are); otherwise element by element.
// Batched launches may also apply a scalar op (fop >= 0) to each problem from the partials
// (last CTA of the problem's tiles, see last_block_update).
template <typename R, int OP, bool VECW>
__global__ void __launch_bounds__(VEC_NT)
vec_kernel(long long n, DevScalars* sc, R* a, R* b, R* c, R* d, R* e, R* f, double* part,
           const int4* tiles, int exec_if, int fop, const BatchProb* probs, unsigned* counters) {
  pdl_begin();
  constexpr int W = VECW ? 16 / (int)sizeof(R) : 1;
  long long lo = 0, hi = n, step = (long long)gridDim.x * VEC_NT * W;
  long long i0 = ((long long)blockIdx.x * VEC_NT + threadIdx.x) * W;
  if (tiles != nullptr) {  // batched: one contiguous range of one problem per CTA
    const int4 tl = tiles[blockIdx.x];
    sc = sc + tl.x;
    lo = tl.y;
    hi = (long long)tl.y + tl.z;
    i0 = lo + (long long)threadIdx.x * W;
    step = (long long)VEC_NT * W;
  }
  if (sc != nullptr && exec_if >= 0 && sc->done != exec_if) return;
  R al = R(0), be = R(0), om = R(0);
  if constexpr (OP == V_CG_UPDATE || OP == V_BI_S) al = (R)sc->alpha;
  if constexpr (OP == V_CG_P || OP == V_BI_P) be = (R)sc->beta;
  if constexpr (OP == V_BI_P || OP == V_BI_X) om = (R)sc->omega;
  R d1 = R(0), d2 = R(0);
#pragma unroll 2
  for (long long i = i0; i < hi; i += step)
    vec_step<R, OP, W>(i, al, be, om, a, b, c, d, e, f, d1, d2);
  if (part != nullptr) {
    block_pair_store((double)d1, (double)d2, part);
    if (fop >= 0 && tiles != nullptr) {
      const int prob = tiles[blockIdx.x].x;
      last_block_update(fop, sc, part, probs[prob].vt0, probs[prob].vt1, counters + prob);
    } else if (fop >= 0) {  // one vector: the last of the grid's CTAs takes the scalar step
      last_block_update(fop, sc, part, 0, (int)gridDim.x, counters);
    }
  }
}

template <typename R>
static cudaError_t vec_dispatch(int op, long long n, DevScalars* sc, R* a, R* b, R* c, R* d,
                                R* e, R* f, double* part, int grid, cudaStream_t st,
                                const int4* tiles = nullptr, int exec_if = 0, int fop = -1,
                                const BatchProb* probs = nullptr, unsigned* counters = nullptr) {
  // 16-byte vectors when every operand is aligned and the ranges split into whole vectors
  // (batched tiles start on 256-element boundaries and have lengths divisible by 8)
  const uintptr_t al = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                       reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d) |
                       reinterpret_cast<uintptr_t>(e) | reinterpret_cast<uintptr_t>(f);
  const long long wv = 16 / (long long)sizeof(R);
  const bool vecw = (al & 15u) == 0 && (tiles != nullptr || n % wv == 0);
  switch (op) {
#define CASE(OPC)                                                                          \
  case OPC:                                                                                \
    return vecw ? launch_k(vec_kernel<R, OPC, true>, dim3(grid), dim3(VEC_NT), 0, st, 1, n, sc, \
                           a, b, c, d, e, f, part, tiles, exec_if, fop, probs, counters)   \
                : launch_k(vec_kernel<R, OPC, false>, dim3(grid), dim3(VEC_NT), 0, st, 1, n,  \
                           sc, a, b, c, d, e, f, part, tiles, exec_if, fop, probs,         \
                           counters);
    CASE(V_CG_UPDATE)
    CASE(V_CG_P)
    CASE(V_BI_P)
    CASE(V_BI_S)
    CASE(V_BI_X)
    CASE(V_DOT)
    CASE(V_COPY)
    CASE(V_ZERO)
    CASE(V_ADD)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_vec(int prec, int op, long long n, const DevScalars* sc, void* a, void* b,
                       void* c, void* d, void* e, void* f, double* part, int* nparts,
                       cudaStream_t st) {
  const int grid = vec_grid(n);
  if (nparts) *nparts = grid;
  DevScalars* s = const_cast<DevScalars*>(sc);  // read only (no fused scalar op here)
  if (prec == 0)
    return vec_dispatch<double>(op, n, s, (double*)a, (double*)b, (double*)c, (double*)d,
                                (double*)e, (double*)f, part, grid, st);
  return vec_dispatch<float>(op, n, s, (float*)a, (float*)b, (float*)c, (float*)d, (float*)e,
                             (float*)f, part, grid, st);
}

cudaError_t launch_vec_fused(int prec, int op, long long n, DevScalars* sc, void* a, void* b,
                             void* c, void* d, void* e, void* f, double* part, int* nparts,
                             int fop, unsigned* counter, cudaStream_t st) {
  if (sc == nullptr || part == nullptr || counter == nullptr || fop < 0)
    return cudaErrorInvalidValue;
  const int grid = vec_grid(n);
  if (nparts) *nparts = grid;
  if (prec == 0)
    return vec_dispatch<double>(op, n, sc, (double*)a, (double*)b, (double*)c, (double*)d,
                                (double*)e, (double*)f, part, grid, st, nullptr, 0, fop, nullptr,
                                counter);
  return vec_dispatch<float>(op, n, sc, (float*)a, (float*)b, (float*)c, (float*)d, (float*)e,
                             (float*)f, part, grid, st, nullptr, 0, fop, nullptr, counter);
}

cudaError_t launch_vec_batch(int prec, int op, const int4* tiles, int ntiles, DevScalars* scs,
                             int exec_if, void* a, void* b, void* c, void* d, void* e, void* f,
                             double* part, cudaStream_t st, int fop, const BatchProb* probs,
                             unsigned* counters) {
  if (ntiles <= 0) return cudaSuccess;
  if (fop >= 0 && (part == nullptr || probs == nullptr || counters == nullptr))
    return cudaErrorInvalidValue;
  if (prec == 0)
    return vec_dispatch<double>(op, 0, scs, (double*)a, (double*)b, (double*)c, (double*)d,
                                (double*)e, (double*)f, part, ntiles, st, tiles, exec_if, fop,
                                probs, counters);
  return vec_dispatch<float>(op, 0, scs, (float*)a, (float*)b, (float*)c, (float*)d, (float*)e,
                             (float*)f, part, ntiles, st, tiles, exec_if, fop, probs, counters);
}

// ---- scalar kernels ------------------------------------------------------------------------


__global__ void __launch_bounds__(VEC_NT)
scalar_kernel(int op, DevScalars* sc, const double* part, int nparts, const double* part2,
              int nparts2) {
  pdl_begin();
  if (op != OP_CG_INIT && op != OP_BI_INIT_RHO && sc->done) return;
  // every thread takes part in the block sums; thread 0 then updates the scalars
  double r[4];
  block_sums4(part, 0, nparts, part2, 0, nparts2, r);
  if (threadIdx.x != 0) return;
  scalar_update(op, sc, part, r[0], r[1], part2, r[2], r[3]);
}

__global__ void __launch_bounds__(VEC_NT)
scalar_batch_kernel(int op, DevScalars* scs, const BatchProb* probs, const double* part, int kind,
                    const double* part2, int kind2, int exec_if) {
  pdl_begin();
  DevScalars* sc = scs + blockIdx.x;
  const BatchProb& pr = probs[blockIdx.x];
  if (exec_if >= 0 && sc->done != exec_if) return;
  const int i0 = kind == 0 ? pr.st0 : pr.vt0, i1 = kind == 0 ? pr.st1 : pr.vt1;
  const int j0 = kind2 == 0 ? pr.st0 : pr.vt0, j1 = kind2 == 0 ? pr.st1 : pr.vt1;
  double r[4];
  block_sums4(part, i0, i1, part2, j0, j1, r);
  if (threadIdx.x != 0) return;
  scalar_update(op, sc, part, r[0], r[1], part2, r[2], r[3]);
}

cudaError_t launch_scalar(int op, DevScalars* sc, const double* part, int nparts,
                          const double* part2, int nparts2, cudaStream_t st) {
  return launch_k(scalar_kernel, dim3(1), dim3(VEC_NT), 0, st, 1, op, sc, part, nparts, part2,
                  nparts2);
}

cudaError_t launch_scalar_batch(int op, DevScalars* scs, const BatchProb* probs, int nprob,
                                const double* part, int kind, const double* part2, int kind2,
                                int exec_if, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  return launch_k(scalar_batch_kernel, dim3(nprob), dim3(VEC_NT), 0, st, 1, op, scs, probs, part,
                  kind, part2, kind2, exec_if);
}

// ---- mixed precision glue ------------------------------------------------------------------
__global__ void to_f32_kernel(const double* x, double scale, float* y, long long n) {
  pdl_begin();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)(scale * x[i]);
}

__global__ void axpy_mixed_kernel(double* x, const float* e, double scale, long long n) {
  pdl_begin();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += scale * (double)e[i];
}

cudaError_t launch_to_f32(const double* x, double scale, float* y, long long n, cudaStream_t st) {
  return launch_k(to_f32_kernel, dim3(vec_grid(n)), dim3(VEC_NT), 0, st, 1, x, scale, y, n);
}

cudaError_t launch_axpy_f32_to_f64(double* x, const float* e, double scale, long long n,
                                   cudaStream_t st) {
  return launch_k(axpy_mixed_kernel, dim3(vec_grid(n)), dim3(VEC_NT), 0, st, 1, x, e, scale, n);
}

__global__ void reduce_to_kernel(const double* part, int nparts, int k, double* out) {
  pdl_begin();
  double r[4];
  block_sums4(part, 0, nparts, nullptr, 0, 0, r);
  if (threadIdx.x == 0) *out = r[k];
}

cudaError_t launch_reduce_to(const double* part, int nparts, int k, double* out, cudaStream_t st) {
  return launch_k(reduce_to_kernel, dim3(1), dim3(VEC_NT), 0, st, 1, part, nparts, k, out);
}

}  // namespace ufg
