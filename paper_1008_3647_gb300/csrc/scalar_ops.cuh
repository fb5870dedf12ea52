// Krylov scalar updates on the device (one thread) and the block reductions that feed them; used
// by the single-CTA scalar kernels and, in batched solves, by the last CTA of a producing kernel
// (last_block_update), which then needs no separate launch.
#pragma once
#include <cuda_runtime.h>

#include "blas.cuh"

namespace ufg {

constexpr int SCAL_NT = 256;  // threads of every CTA that runs these reductions

static __device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

// The four sums (pairs [i0, i1) of part, pairs [j0, j1) of part2) in one sweep: each thread adds
// its strided share, the warps fold with shuffles and thread 0 adds the warp results in order
// (a fixed, launch-independent order: the result is deterministic).  Valid in thread 0.
// NT: threads of the calling CTA (SCAL_NT unless a kernel says otherwise).
template <int NT = SCAL_NT>
static __device__ void block_sums4(const double* part, int i0, int i1, const double* part2, int j0,
                            int j1, double (&out)[4]) {
  __shared__ double red[NT / 32][4];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (part != nullptr)
    for (int i = i0 + (int)threadIdx.x; i < i1; i += NT) {
      s[0] += part[2 * i];
      s[1] += part[2 * i + 1];
    }
  if (part2 != nullptr)
    for (int i = j0 + (int)threadIdx.x; i < j1; i += NT) {
      s[2] += part2[2 * i];
      s[3] += part2[2 * i + 1];
    }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], off);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[threadIdx.x >> 5][k] = s[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w][k];
      out[k] = t;
    }
  }
}

static __device__ __forceinline__ void bi_rho(DevScalars* sc, double rho, double rr) {
  if (fabs(rho) <= sc->restart_cos * sqrt(sc->rhatn2 * rr)) {
    sc->done = 2;  // near-breakdown: the host restarts from the true residual
    return;
  }
  sc->iters += 1;
  sc->rho = rho;
  sc->beta = (rho / sc->rho_old) * (sc->alpha / sc->omega);
  if (bad(sc->beta)) sc->done = 4;
}

static __device__ __forceinline__ void bi_rcheck(DevScalars* sc, double rr, double tb) {
  sc->rr = rr;
  sc->rho_old = sc->rho;
  if (bad(rr)) sc->done = 4;
  else if (sqrt(rr) <= tb) sc->done = 1;
  else if (sc->div_limit > 0 && sqrt(rr) > sc->div_limit * sc->bn) sc->done = 6;
  else if (sc->omega == 0.0) sc->done = 2;
  else if (sc->iters >= sc->maxit) sc->done = 5;
}

static __device__ __noinline__ void scalar_update(int op, DevScalars* sc, const double* part, double a0, double a1,
                              const double* part2, double b0, double b1) {
  if ((op == OP_CG_INIT || op == OP_BI_INIT_RHO) && part2 != nullptr)
    sc->bn = sqrt(b1);  // rhs.rhs
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
    case OP_BI_INIT_RHO:  // part = (rhat.r, r.r), part2 = (rhat.rhat, rhs.rhs); the first
                          // iteration's rho from the same partials
      sc->rho = a0;
      sc->rr = a1;
      sc->rhatn2 = b0;
      sc->rho_old = 1.0;
      sc->alpha = 1.0;
      sc->omega = 1.0;
      sc->done = 0;
      if (bad(a0) || bad(a1)) sc->done = 4;
      else if (sqrt(a1) <= tb) sc->done = 1;
      else bi_rho(sc, a0, a1);
      break;
    case OP_BI_RHO_REDO:  // part = (rhat.r, r.r) of the replaced residual
      sc->rr = a1;
      if (fabs(a0) <= sc->restart_cos * sqrt(sc->rhatn2 * a1)) {
        sc->done = 2;
        break;
      }
      sc->rho = a0;
      sc->beta = (a0 / sc->rho_old) * (sc->alpha / sc->omega);
      sc->done = bad(sc->beta) ? 4 : 0;
      break;
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
    case OP_BI_RCHECK_RHO:  // part = (rhat.r, r.r): the iteration's check, then (still
                            // running) the next one's rho
      bi_rcheck(sc, a1, tb);
      if (sc->done == 0) bi_rho(sc, a0, a1);
      break;
  }
}

// Called by every thread of a CTA of a producer whose thread 0 has just written the CTA's
// partial pair into `part`: the CTA that completes a problem's set [i0, i1) (counted on
// `counter`, left at 0 for the next producer) sums the set in fixed order and applies `op` to
// that problem's scalars.  Partials reach the summing CTA through thread 0's fence before its
// count (only thread 0 wrote them, so only it fences).
template <int NT = SCAL_NT>
static __device__ __forceinline__ void last_block_update(int op, DevScalars* sc, const double* part,
                                                        int i0, int i1, unsigned* counter) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(counter, 1u) == (unsigned)(i1 - i0 - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double r[4];
  block_sums4<NT>(part, i0, i1, nullptr, 0, 0, r);
  if (threadIdx.x == 0) {
    scalar_update(op, sc, part, r[0], r[1], nullptr, 0.0, 0.0);
    *counter = 0u;
  }
}

}  // namespace ufg
