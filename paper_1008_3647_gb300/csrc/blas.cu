// BLAS-1 vector kernels and single-CTA scalar kernels of the Krylov solvers (see blas.cuh).
#include <cmath>

#include "blas.cuh"
#include "ufg_internal.h"

namespace ufg {

constexpr int VEC_NT = 256;

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

template <typename R, int OP>
__global__ void __launch_bounds__(VEC_NT)
vec_kernel(long long n, const DevScalars* __restrict__ sc, R* a, R* b, R* c, R* d, R* e, R* f,
           double* part, const int4* tiles, int exec_if) {
  long long stride = (long long)gridDim.x * VEC_NT;
  long long i0 = (long long)blockIdx.x * VEC_NT + threadIdx.x;
  if (tiles != nullptr) {  // batched: one contiguous range of one problem per CTA
    const int4 tl = tiles[blockIdx.x];
    sc = sc + tl.x;
    i0 = (long long)tl.y + threadIdx.x;
    n = (long long)tl.y + tl.z;
    stride = VEC_NT;
  }
  if (sc != nullptr && exec_if >= 0 && sc->done != exec_if) return;
  double d1 = 0.0, d2 = 0.0;
  if constexpr (OP == V_CG_UPDATE) {
    const R al = (R)sc->alpha;
    for (long long i = i0; i < n; i += stride) {
      a[i] += al * b[i];
      const R r = c[i] - al * d[i];
      c[i] = r;
      d2 += (double)r * (double)r;
    }
  } else if constexpr (OP == V_CG_P) {
    const R be = (R)sc->beta;
    for (long long i = i0; i < n; i += stride) a[i] = b[i] + be * a[i];
  } else if constexpr (OP == V_BI_P) {
    const R be = (R)sc->beta, om = (R)sc->omega;
    for (long long i = i0; i < n; i += stride) a[i] = b[i] + be * (a[i] - om * c[i]);
  } else if constexpr (OP == V_BI_S) {
    const R al = (R)sc->alpha;
    for (long long i = i0; i < n; i += stride) {
      const R s = b[i] - al * c[i];
      a[i] = s;
      d[i] += al * e[i];
      d2 += (double)s * (double)s;
    }
  } else if constexpr (OP == V_BI_X) {
    const R om = (R)sc->omega;
    for (long long i = i0; i < n; i += stride) {
      a[i] += om * b[i];
      const R r = d[i] - om * e[i];
      c[i] = r;
      d1 += (double)f[i] * (double)r;
      d2 += (double)r * (double)r;
    }
  } else if constexpr (OP == V_DOT) {
    for (long long i = i0; i < n; i += stride) {
      if (a != nullptr) d1 += (double)a[i] * (double)b[i];
      if (c != nullptr) d2 += (double)c[i] * (double)d[i];
    }
  } else if constexpr (OP == V_COPY) {
    for (long long i = i0; i < n; i += stride) a[i] = b[i];
  } else if constexpr (OP == V_ZERO) {
    for (long long i = i0; i < n; i += stride) a[i] = R(0);
  } else if constexpr (OP == V_ADD) {
    for (long long i = i0; i < n; i += stride) a[i] += b[i];
  }
  if (part != nullptr) block_pair_store(d1, d2, part);
}

template <typename R>
static cudaError_t vec_dispatch(int op, long long n, const DevScalars* sc, R* a, R* b, R* c, R* d,
                                R* e, R* f, double* part, int grid, cudaStream_t st,
                                const int4* tiles = nullptr, int exec_if = 0) {
  switch (op) {
#define CASE(OPC)                                                                         \
  case OPC:                                                                               \
    vec_kernel<R, OPC><<<grid, VEC_NT, 0, st>>>(n, sc, a, b, c, d, e, f, part, tiles,     \
                                                exec_if);                                 \
    break;
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
  if (prec == 0)
    return vec_dispatch<double>(op, n, sc, (double*)a, (double*)b, (double*)c, (double*)d,
                                (double*)e, (double*)f, part, grid, st);
  return vec_dispatch<float>(op, n, sc, (float*)a, (float*)b, (float*)c, (float*)d, (float*)e,
                             (float*)f, part, grid, st);
}

cudaError_t launch_vec_batch(int prec, int op, const int4* tiles, int ntiles, const DevScalars* scs,
                             int exec_if, void* a, void* b, void* c, void* d, void* e, void* f,
                             double* part, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (prec == 0)
    return vec_dispatch<double>(op, 0, scs, (double*)a, (double*)b, (double*)c, (double*)d,
                                (double*)e, (double*)f, part, ntiles, st, tiles, exec_if);
  return vec_dispatch<float>(op, 0, scs, (float*)a, (float*)b, (float*)c, (float*)d, (float*)e,
                             (float*)f, part, ntiles, st, tiles, exec_if);
}

// ---- scalar kernels ------------------------------------------------------------------------
__device__ double block_sum(const double* part, int nparts, int k, int i0 = 0) {
  __shared__ double red[VEC_NT];
  double s = 0.0;
  if (part != nullptr)
    for (int i = i0 + threadIdx.x; i < nparts; i += VEC_NT) s += part[2 * i + k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = VEC_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

__device__ void scalar_update(int op, DevScalars* sc, const double* part, double a0, double a1,
                              const double* part2, double b0, double b1);

__global__ void __launch_bounds__(VEC_NT)
scalar_kernel(int op, DevScalars* sc, const double* part, int nparts, const double* part2,
              int nparts2) {
  if (op != OP_CG_INIT && op != OP_BI_INIT && sc->done) return;
  // every thread takes part in the block sums; thread 0 then updates the scalars
  const double a0 = block_sum(part, nparts, 0);
  const double a1 = block_sum(part, nparts, 1);
  const double b0 = block_sum(part2, nparts2, 0);
  const double b1 = block_sum(part2, nparts2, 1);
  if (threadIdx.x != 0) return;
  scalar_update(op, sc, part, a0, a1, part2, b0, b1);
}

__global__ void __launch_bounds__(VEC_NT)
scalar_batch_kernel(int op, DevScalars* scs, const BatchProb* probs, const double* part, int kind,
                    const double* part2, int kind2, int exec_if) {
  DevScalars* sc = scs + blockIdx.x;
  const BatchProb& pr = probs[blockIdx.x];
  if (exec_if >= 0 && sc->done != exec_if) return;
  const int i0 = kind == 0 ? pr.st0 : pr.vt0, i1 = kind == 0 ? pr.st1 : pr.vt1;
  const int j0 = kind2 == 0 ? pr.st0 : pr.vt0, j1 = kind2 == 0 ? pr.st1 : pr.vt1;
  const double a0 = block_sum(part, i1, 0, i0);
  const double a1 = block_sum(part, i1, 1, i0);
  const double b0 = block_sum(part2, j1, 0, j0);
  const double b1 = block_sum(part2, j1, 1, j0);
  if (threadIdx.x != 0) return;
  scalar_update(op, sc, part, a0, a1, part2, b0, b1);
}

__device__ void scalar_update(int op, DevScalars* sc, const double* part, double a0, double a1,
                              const double* part2, double b0, double b1) {
  if ((op == OP_CG_INIT || op == OP_BI_INIT) && part2 != nullptr) sc->bn = sqrt(b1);  // rhs.rhs
  const double tb = sc->tol * sc->bn;
  switch (op) {
    case OP_CG_INIT:  // part = (r.z, r.r), part2 = (-, rhs.rhs)
      sc->rz = a0;
      sc->rr = a1;
      sc->done = 0;
      if (bad(a0) || bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      break;
    case OP_CG_ALPHA:  // part = slice partials (p.q, -)
      sc->pq = a0;
      sc->alpha = sc->rz / a0;
      if (bad(sc->alpha)) sc->done = 4;
      break;
    case OP_CG_CHECK:  // part = (-, r.r)
      sc->iters += 1;
      sc->rr = a1;
      if (bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      else if (sc->div_limit > 0 && sqrt(a1) > sc->div_limit * sc->bn) sc->done = 6;
      else if (sc->iters >= sc->maxit) sc->done = 5;
      break;
    case OP_CG_BETA: {  // part = (r.z, -) or, without preconditioner, part2 = (-, r.r)
      const double rz_new = part != nullptr ? a0 : b1;
      sc->beta = rz_new / sc->rz;
      sc->rz = rz_new;
      if (bad(sc->beta)) sc->done = 4;
      break;
    }
    case OP_BI_INIT:  // part = (rhat.r, r.r), part2 = (rhat.rhat, rhs.rhs)
      sc->rho = a0;
      sc->rr = a1;
      sc->rhatn2 = b0;
      sc->rho_old = 1.0;
      sc->alpha = 1.0;
      sc->omega = 1.0;
      sc->done = 0;
      if (bad(a0) || bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      break;
    case OP_BI_RHO: {  // part = (rhat.r, r.r) of the last residual update (or of the init)
      const double rho = a0;
      if (fabs(rho) <= sc->restart_cos * sqrt(sc->rhatn2 * a1)) {
        sc->done = 2;  // near-breakdown: the host restarts from the true residual
        break;
      }
      sc->iters += 1;
      sc->rho = rho;
      sc->beta = (rho / sc->rho_old) * (sc->alpha / sc->omega);
      if (bad(sc->beta)) sc->done = 4;
      break;
    }
    case OP_BI_ALPHA:  // part = slice partials (v.rhat, -)
      sc->alpha = sc->rho / a0;
      if (bad(sc->alpha)) sc->done = 4;
      break;
    case OP_BI_SCHECK:  // part = (-, s.s)
      sc->ss = a1;
      if (bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      else if (sc->div_limit > 0 && sqrt(a1) > sc->div_limit * sc->bn) sc->done = 6;
      break;
    case OP_BI_OMEGA:  // part = slice partials (t.s, t.t)
      sc->omega = a1 > 0.0 ? a0 / a1 : 0.0;
      if (bad(sc->omega)) sc->done = 4;
      break;
    case OP_NORM2:  // part = (-, v.v)
      sc->rr = a1;
      break;
    case OP_BI_RCHECK:  // part = (rhat.r, r.r)
      sc->rr = a1;
      sc->rho_old = sc->rho;
      if (bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      else if (sc->div_limit > 0 && sqrt(a1) > sc->div_limit * sc->bn) sc->done = 6;
      else if (sc->omega == 0.0) sc->done = 2;
      else if (sc->iters >= sc->maxit) sc->done = 5;
      break;
  }
}

cudaError_t launch_scalar(int op, DevScalars* sc, const double* part, int nparts,
                          const double* part2, int nparts2, cudaStream_t st) {
  scalar_kernel<<<1, VEC_NT, 0, st>>>(op, sc, part, nparts, part2, nparts2);
  return cudaGetLastError();
}

cudaError_t launch_scalar_batch(int op, DevScalars* scs, const BatchProb* probs, int nprob,
                                const double* part, int kind, const double* part2, int kind2,
                                int exec_if, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  scalar_batch_kernel<<<nprob, VEC_NT, 0, st>>>(op, scs, probs, part, kind, part2, kind2,
                                                exec_if);
  return cudaGetLastError();
}

// ---- mixed precision glue ------------------------------------------------------------------
__global__ void to_f32_kernel(const double* x, double scale, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)(scale * x[i]);
}

__global__ void axpy_mixed_kernel(double* x, const float* e, double scale, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += scale * (double)e[i];
}

cudaError_t launch_to_f32(const double* x, double scale, float* y, long long n, cudaStream_t st) {
  to_f32_kernel<<<vec_grid(n), VEC_NT, 0, st>>>(x, scale, y, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy_f32_to_f64(double* x, const float* e, double scale, long long n,
                                   cudaStream_t st) {
  axpy_mixed_kernel<<<vec_grid(n), VEC_NT, 0, st>>>(x, e, scale, n);
  return cudaGetLastError();
}

__global__ void reduce_to_kernel(const double* part, int nparts, int k, double* out) {
  const double s = block_sum(part, nparts, k);
  if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_reduce_to(const double* part, int nparts, int k, double* out, cudaStream_t st) {
  reduce_to_kernel<<<1, VEC_NT, 0, st>>>(part, nparts, k, out);
  return cudaGetLastError();
}

}  // namespace ufg
