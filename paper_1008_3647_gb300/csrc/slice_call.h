// Type-erased description of one fused slice-kernel launch (see slice_kernel.cuh).
#pragma once
#include <cuda_runtime.h>

namespace ufg {

// FAM_M1W: the weak-coupling term -A M1 (Sec. 3) in momentum space, -A S^{+-1} F^T (s * F x), for
// one slice in one kernel
// (inverse transform, site multiplier, forward transform); coef = inverse, coef2 = forward family.
// FAM_Q: the normal operator Q = M^T M (Eq. 1) in one kernel per output slice (slice_q.cuh):
// in = x, pre = the potential w, coef = the kinetic family, out = a Q x + bU U + cV V with the
// partials of the other families; whole slices of one lattice with N_tau >= 3.
enum SliceFamily { FAM_KIN = 0, FAM_FWD = 1, FAM_INV = 2, FAM_M1W = 3, FAM_Q = 4 };

// Batched mode: one problem of a batch as the kernels see it (device table).
struct BatchProb {
  long long off;     // element offset of the problem's vectors inside every arena
  int ntau;          // time slices of the problem
  int V;             // sites per slice
  int st0, st1;      // slice-kernel CTAs [st0, st1) of this problem (partials index range)
  int vt0, vt1;      // vector-kernel CTAs [vt0, vt1)
  int rt0, rt1;      // recurrence CTAs [rt0, rt1)
  double A;          // coupling of the problem
  int* done;         // the problem's solver state flag
};
// One slice-kernel work unit: `spc` time slices of one problem.
struct BatchTile {
  int prob;
  int t0;
};
// Run policy on the done flag: run while the flag equals exec_if (0: running, 2: restart
// requested); exec_if = -1 runs unconditionally.

struct DevScalars;

// Runtime description of one slice launch (host side, type-erased pointers).
struct SliceCall {
  int fam = FAM_KIN;
  int prec = 0;               // 0 = FP64, 1 = FP32
  const void* coef = nullptr; // host LineCoef<N, R> for (fam, prec)
  const void* coef2 = nullptr; // FAM_M1W: forward-transform coefficients
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
  int exec_if = 0;             // run while *done == exec_if (-1: always)
  const BatchTile* tiles = nullptr;  // batched mode: tile table (device), one tile per unit
  const BatchProb* probs = nullptr;  // batched mode: problem table (device)
  int ntiles = 0;
  int scale_by_A = 0;          // batched mode: multiply a by the problem's coupling A
  long long nelem = 0;         // elements of the arenas (0: ntau * N^3, a single problem)
  int* err = nullptr;          // device flag raised if a bounded wait ran out
  int allow_tma = 1;           // 0 forces the non-TMA kernel
  int* grid_out = nullptr;     // receives the number of CTAs launched (= partial pairs written)
  int ntau = 0;
  int dim = 3;                 // lattice dimension: 3, or 1 / 2 (slice_lowd.cuh)
  int shift = 0;               // -1: t_in = t_out - 1, +1: t_in = t_out + 1, 0: t_in = t_out
  int spc = 1;                 // time slices per CTA (cluster)
  int C = 1;                   // cluster size (1, 2 or 4; N = 32 only uses 2 or 4)
  int nt = 256;                // threads per CTA (the kernels are written for 256)
  // batched mode: scalar op applied to each problem from the partials by its last CTA
  int fop = -1;                // ScalarOp, -1: none
  DevScalars* scs = nullptr;   // per-problem solver scalars
  unsigned* counters = nullptr;  // per-problem CTA counters (zero between launches)
  int part_base = 0;           // CTA index of this launch's first CTA in the problems' ranges
  // batched forward transform fused with the BiCGStab direction update (TMA kernel only):
  // in = p, p' = prep_r + beta (p - omega prep_v) written to prep_out, scalars from scs
  const void* prep_r = nullptr;
  const void* prep_v = nullptr;
  void* prep_out = nullptr;
  // FAM_M1W with m1w_full = 1: the whole matrix M (shift -1) or M^T (shift +1) in the momentum
  // basis, out = full_scale * M x + bU * U with the partials as the KIN family; pre is then the
  // potential w = 1 + A sin(sigma) and a = 1
  int m1w_full = 0;
  double full_scale = 1.0;
  // FAM_M1W FULL on FP64 vectors: double-float arithmetic on the FP32 pipe (slice_df.cuh) instead
  // of FP64 arithmetic (ufg_apply_M_momentum with UFG_FP64_EMULATED; the batched incremental
  // reliable updates)
  int emulate64 = 0;
};

// Test hook of ufg_test_expire_waits: 1 if this TMA launch on st runs one bounded wait that is
// made to run out (consumes one of the requested launches), else 0; always 0 while st is being
// captured into a graph.
int take_expired_wait(cudaStream_t st);

// Launches the slice kernel for lattice extent N (explicitly instantiated per N).
template <int N>
cudaError_t slice_launch(const SliceCall& c, cudaStream_t st);

// Whether the TMA forward transform with the fused direction update (SliceCall::prep_out) runs
// for N, precision and the lattice's TMA setting (per N, and by runtime dispatch).
template <int N>
bool slice_tma_prep_ok(int prec, int allow_tma);
bool slice_tma_prep_supported(int N, int prec, int allow_tma);

// Runtime dispatch over the supported N (4, 6, 8, 10, 12, 16, 32).
cudaError_t slice_dispatch(int N, const SliceCall& c, cudaStream_t st);
bool slice_supported_n(int N);
// Whether the fused FAM_M1W kernel exists for (N, precision): one CTA per slice with the slice
// in 64- or 128-byte TMA rows (FP32 N = 16, FP64 N = 8 and 16).
bool slice_m1w_supported(int N, int prec);
// Whether the fused FAM_Q kernel runs for (N, precision, N_tau): N = 16 (FP32 and FP64),
// 3 <= N_tau <= twice the SM count, TMA enabled and UFG_NO_FUSED_Q unset.
bool slice_q_supported(int N, int prec, int ntau, int dim = 3);

}  // namespace ufg
