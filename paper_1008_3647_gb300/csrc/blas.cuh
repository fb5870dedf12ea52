// BLAS-1 and scalar kernels of the Krylov solvers (declarations shared with solvers.cu).
//
// Every reduction is two-level and deterministic: the producing kernel (a vector update or the
// epilogue of a slice kernel) writes one FP64 partial pair per CTA, and a single-CTA "scalar" kernel
// sums the partials in a fixed order and updates the solver's scalars in device memory.  Vector
// kernels read alpha/beta/omega from there, so a whole iteration runs without the host and can be
// captured in a CUDA graph.  All kernels return immediately once `done` is set.
#pragma once
#include <string>
#include <cuda_runtime.h>

#include "slice_call.h"

namespace ufg {

// Solver scalars in device memory.
struct DevScalars {
  double bn;       // ||rhs||
  double tol;      // relative target on the recursive residual
  double rz, alpha, beta, pq;               // CG
  double rho, rho_old, omega, rhatn2;       // BiCGStab
  double rr, ss;
  double restart_cos;                       // near-breakdown threshold on |rho|
  double div_limit;                         // > 0: stop with done = 6 once ||r|| > div_limit ||rhs||
  int done;        // 0 running, 1 converged, 2 restart requested, 4 non-finite, 5 maxit,
                   // 6 diverged
  int iters;
  int maxit;
  int pad;
};

enum ScalarOp {
  OP_CG_INIT = 0,   // rr, rz from partials (a: r.z, b: r.r); convergence test at start
  OP_CG_ALPHA,      // alpha = rz / (p.q)
  OP_CG_CHECK,      // iters++, rr = r.r, converged?
  OP_CG_BETA,       // rz_new = r.z, beta = rz_new / rz
  OP_BI_ALPHA,      // alpha = rho / (rhat.v)
  OP_BI_SCHECK,     // ss = s.s, converged?
  OP_BI_OMEGA,      // omega = (t.s) / (t.t)
  OP_NORM2,         // rr = v.v only (no other state touched)
  OP_BI_RCHECK_RHO, // rr = r.r, converged?, rho_old = rho; then, if still running, the next
                    // iteration's rho = rhat.r (near-breakdown -> restart, else iters++, beta)
  OP_BI_INIT_RHO,   // rhatn2 = rhat.rhat, rr = r.r, rho_old = alpha = omega = 1; then, if still
                    // running, the first iteration's rho as above
  OP_BI_RHO_REDO,   // after a residual replacement: rho = rhat.r, beta again (no iteration
                    // counted); done = 0, or 2 on near-breakdown
};

// Partial pairs per producing CTA: up to this many CTAs per producer.
constexpr int MAX_PARTIAL_CTAS = 8192;

cudaError_t launch_scalar(int op, DevScalars* sc, const double* part, int nparts,
                          const double* part2, int nparts2, cudaStream_t st);

// Vector kernels (R = double or float); partials (nullable) receive [grid][2] FP64 pairs and the
// grid size is returned in *nparts.
enum VecOp {
  V_CG_UPDATE = 0,  // x += alpha p; r -= alpha q; part = (-, r.r)
  V_CG_P,           // p = z + beta p
  V_BI_P,           // p = r + beta (p - omega v)
  V_BI_S,           // s = r - alpha v; x += alpha y; part = (-, s.s)
  V_BI_X,           // x += omega z; r = s - omega t; part = (rhat.r, r.r)
  V_DOT,            // part = (a.b, c.d)
  V_COPY,           // a <- b
  V_ZERO,           // a <- 0
  V_ADD,            // a += b
};
cudaError_t launch_vec(int prec, int op, long long n, const DevScalars* sc, void* a, void* b,
                       void* c, void* d, void* e, void* f, double* part, int* nparts,
                       cudaStream_t st);
int vec_grid(long long n);
// launch_vec that also applies scalar op fop to *sc from the partials it writes: the last of its
// CTAs sums them in the scalar kernel's order and updates *sc (counter: zero between launches,
// left at zero), so no separate scalar launch follows.  Runs while sc->done == 0.
cudaError_t launch_vec_fused(int prec, int op, long long n, DevScalars* sc, void* a, void* b,
                             void* c, void* d, void* e, void* f, double* part, int* nparts,
                             int fop, unsigned* counter, cudaStream_t st);
// Instrumentation: "vec <op> f32|f64" and the vectors one element of the op reads plus writes
// (V_DOT: each present pair; a: first pair present, c: second pair present).
std::string vec_op_name(int op, int prec);
int vec_op_arrays(int op, bool a_present, bool c_present);

// Batched form: CTA i works on tiles[i] = (problem, start, length) of the packed arenas with
// the scalars scs[problem]; it runs while scs[problem].done == exec_if (exec_if < 0: always).
// fop >= 0 also applies scalar op fop to each problem once all of its tiles have written their
// partials (the last of them does it; counters: one per problem, zero between launches).
cudaError_t launch_vec_batch(int prec, int op, const int4* tiles, int ntiles, DevScalars* scs,
                             int exec_if, void* a, void* b, void* c, void* d, void* e, void* f,
                             double* part, cudaStream_t st, int fop = -1,
                             const BatchProb* probs = nullptr, unsigned* counters = nullptr);
// Batched scalar kernel: CTA p reduces problem p's partials (kind 0: slice CTAs [st0, st1),
// kind 1: vector CTAs [vt0, vt1)) and updates scs[p], while scs[p].done == exec_if.
cudaError_t launch_scalar_batch(int op, DevScalars* scs, const BatchProb* probs, int nprob,
                                const double* part, int kind, const double* part2, int kind2,
                                int exec_if, cudaStream_t st);

// Mixed-precision glue: y32 = scale * x64 and x64 += scale * e32.
cudaError_t launch_to_f32(const double* x, double scale, float* y, long long n, cudaStream_t st);
cudaError_t launch_axpy_f32_to_f64(double* x, const float* e, double scale, long long n,
                                   cudaStream_t st);
// Deterministic host-visible sum of partial pairs (column k) into *out (device double).
cudaError_t launch_reduce_to(const double* part, int nparts, int k, double* out, cudaStream_t st);

}  // namespace ufg
