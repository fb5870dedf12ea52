/* ufg.h - C ABI of the GB300 (sm_103a) library for the unitary-Fermi-gas fermion matrix.
 *
 * The library applies the fermion matrix M[sigma] of Ten, Drut & Laehde, "Preconditioning the
 * non-relativistic many-fermion problem" (arXiv:1008.3647), Sec. 1, Eq. (MatrixM):
 *
 *     (M x)_0     = x_0     + B_{N_tau-1} x_{N_tau-1}
 *     (M x)_{t+1} = x_{t+1} - B_t x_t                       (t = 0 .. N_tau-2)
 *     B_t = exp(-tau K) (1 + A sin sigma_t),   A = sqrt(2) sqrt(exp(tau g) - 1),
 *     K diagonal in momentum space with E(k) = k^2/2 (hbar = m = 1), k_i = 2 pi n_i / N_x,
 *
 * matrix-free on the GPU, its transpose M^T (= M^dagger, M is real), the normal operator
 * Q = M^T M (Eq. 1), and the paper's Krylov solvers and preconditioners: CG on Q x = b (Eq. 1),
 * two-step BiCGStab M^T y = b, M x = y (Eq. 2), Chebyshev (Sec. 2), weak-coupling expansion with
 * exact Fourier-accelerated M0^{-1} (Sec. 3) and strong coupling (Sec. 4), plus the HMC fermion
 * force (Sec. 1).
 *
 * Conventions.
 *   - Vectors are contiguous arrays in the order [t][z][y][x] (time slice slowest), t = 0-based
 *     (the paper's 1-based slice j is t + 1).  S = N_x^3 N_tau sites.
 *   - Vector pointers are DEVICE pointers unless a function says otherwise, 16-byte aligned, not
 *     aliased with each other, owned by the caller.  FP64 entries are double, FP32 entries float.
 *   - Handles (lattice, field, solver) and their workspace are owned by the library; all device
 *     memory is allocated at creation, none inside applies or solve loops.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Applies are
 *     asynchronous on it; solves and the force return after the result is complete.
 *   - No function throws or aborts; every failure returns a status and leaves a thread-local
 *     message for ufg_last_error().
 *
 * Environment switches (read once per process; for comparisons and diagnosis):
 *   UFG_NO_TMA=1       the position-space slice kernels (applies, transforms) take the
 *                      shared-memory-staged path instead of TMA (the fused momentum-space
 *                      kernels are TMA-only);
 *   UFG_NO_GRAPH=1     solver loops are launched directly instead of replayed CUDA graphs;
 *   UFG_PDL=1          every kernel is launched with programmatic dependent launch (by
 *                      default only the launches of the standalone operator calls below);
 *   UFG_NO_FUSED_Q=1   Q = M^T M as two launches (M, then M^T) everywhere (by default one
 *                      kernel per output slice on 16^3 lattices with N_tau <= twice the SMs);
 *   UFG_NO_MOMENTUM=1  WCE-preconditioned BiCGStab stays in the position basis (by default it
 *                      iterates on F x where the lattice has the fused momentum-space operator);
 *   UFG_NO_PAIR=1      FP32 16^3 slices run one line per thread instead of two (packed FP32x2);
 *   UFG_TMA_C32=4      FP32 32^3 slices run in 4-CTA clusters instead of 8;
 *   UFG_TUNE_CACHE=f   ufg_lattice_autotune results are also kept in file f (see there).
 */
#ifndef UFG_H
#define UFG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UFG_OK = 0,
  UFG_INVALID_ARG = 1,   /* bad size, pointer, alignment or parameter */
  UFG_NOT_CONVERGED = 2, /* maxit reached before the residual target */
  UFG_BREAKDOWN = 3,     /* BiCGStab breakdown persisted through all restarts */
  UFG_NONFINITE = 4,     /* NaN or Inf in a residual or input */
  UFG_TIMEOUT = 5,       /* a bounded device wait ran out */
  UFG_CUDA_ERROR = 6,    /* a CUDA runtime call failed */
  UFG_OOM = 7,           /* device allocation failed at handle creation */
  UFG_INTERNAL = 8,      /* internal consistency check failed */
  UFG_UNSUPPORTED = 9    /* valid input outside what the library implements (e.g. N_x) */
} ufg_status;

/* UFG_FP64_EMULATED: FP64 vectors, arithmetic in double-float pairs on the FP32 pipe (about 46
 * significant bits; GB300's FP64 pipe is ~1/76 of its FP32 rate).  Accepted by
 * ufg_apply_M_momentum.  Its absolute error is about 2^-46 ||M|| ||x||, so a residual b - M x of
 * a nearly converged, ill-conditioned system (||x|| >> ||b||) is not resolved to 1e-10 of
 * ||b|| this way.  The batched mixed-precision solve uses it only for incremental residual
 * updates r -= M d after a first FP64 residual, where the error scales with the increment d;
 * every final residual is FP64. */
typedef enum { UFG_FP64 = 0, UFG_FP32 = 1, UFG_MIXED = 2, UFG_FP64_EMULATED = 3 } ufg_precision;

/* UFG_PC_SCA_CHEB: the strong-coupling factorisation with the Chebyshev polynomial as a secondary
 * filter (end of Sec. 4): P = P(G/s)/s (L^T D L)^{-1} with G = (L^T D L)^{-1} Q, for CG. */
typedef enum {
  UFG_PC_NONE = 0,
  UFG_PC_CHEB = 1,
  UFG_PC_SCA = 2,
  UFG_PC_WCE = 3,
  UFG_PC_SCA_CHEB = 4
} ufg_pc_kind;

typedef struct ufg_lattice ufg_lattice;
typedef struct ufg_field ufg_field;
typedef struct ufg_solver ufg_solver;

/* Preconditioner parameters (fields unused by a kind are ignored).
 *   degree : Chebyshev degree d = 2n of P(z) ~ 1/z (Sec. 2, Eq. ChebInv); even, 2..64.
 *   eps    : lower edge of [eps, 1] after normalisation; <= 0 selects (2 - 2 cos(pi/N_tau)) / scale
 *            (UFG_PC_CHEB) or 1e-3 (UFG_PC_SCA_CHEB).
 *   scale  : spectrum normalisation s of the operator the polynomial acts on (z = Q / s, or G / s
 *            for UFG_PC_SCA_CHEB); <= 0 selects (2 + A)^2 for Q, a rigorous bound on ||M||^2 since
 *            ||exp(-tau K)|| = 1 and |1 + A sin sigma| <= 1 + A, and for G 1.1 times the estimate
 *            of 30 power steps from w = 1 + A sin sigma (made once per field and alpha).
 *   alpha  : strong-coupling parameter alpha of D_t (Sec. 4); must be > 0.
 *   order  : weak-coupling expansion order d (Sec. 3, Eq. WCE); 0..16.
 *   euler  : acceleration of the order-d series over its partial sums S_{0,k} (Sec. 3.1), a
 *            ufg_accel value: UFG_ACCEL_NONE the plain sum S_{0,d}; UFG_ACCEL_EULER the Euler
 *            recursion S_{j+1,k} = p S_{j,k} + (1-p) S_{j,k+1} (Eq. Euler) down to S_{d,0};
 *            UFG_ACCEL_EULER23 its entry S_{j,d-j} with j the integer nearest 2d/3 (the paper's
 *            S_{2kmax/3,kmax/3}); UFG_ACCEL_VANW the special van Wijngaarden transformation
 *            (lambda_k = s^k/k!, phi(t) = s exp(-s t)) truncated at order d.  Every mode only
 *            changes the weights of the d + 1 series terms: the cost per application is that of
 *            the plain series.
 *   euler_p: p of the Euler recursion, in (0, 1); 0 selects 1/2, the paper's choice.
 *   vw_s   : the free parameter s > 0 of the special van Wijngaarden transformation; 0 selects 1.
 * All fields zero except those a kind uses is a valid set of defaults for euler_p and vw_s. */
typedef enum {
  UFG_ACCEL_NONE = 0,
  UFG_ACCEL_EULER = 1,
  UFG_ACCEL_EULER23 = 2,
  UFG_ACCEL_VANW = 3
} ufg_accel;

typedef struct {
  int degree;
  double eps;
  double scale;
  double alpha;
  int order;
  int euler;
  double euler_p;
  double vw_s;
} ufg_pc_params;

/* The weights c_0..c_order (host FP64, order + 1 entries written to `weights`, caller-owned) with
 * which the weak-coupling preconditioner of that order sums its terms, P_d r = sum_n c_n t_n,
 * t_n = (-A M0^{-1} M1)^n M0^{-1} r (Sec. 3, Eq. WCE), under acceleration `accel` (a ufg_accel)
 * with parameters euler_p and vw_s as in ufg_pc_params (0 selects 1/2 and 1); Sec. 3.1.  Host
 * only: runs without a GPU.  UFG_INVALID_ARG for an order outside 0..16, an unknown accel, or
 * parameters out of range (with a message). */
ufg_status ufg_wce_series_weights(int order, int accel, double euler_p, double vw_s,
                                  double* weights);

/* Solve parameters.
 *   tol       : target of the true relative residual ||b - M^T M x|| / ||b|| (Sec. 5 "reduction in
 *               the norm of the residual"), recomputed in FP64 at exit.
 *   maxit     : iteration cap of each Krylov solve.
 *   precision : UFG_FP64, or UFG_MIXED (FP32 inner solves inside an FP64 defect-correction loop).
 *   x0_given  : nonzero uses the content of x as the initial guess (else x0 = 0).
 *   inner_tol : MIXED only, relative reduction asked of each FP32 inner solve (0: 1e-5).  A
 *               negative value autotunes it: the first such call of a solver and method times
 *               the whole solve for 1e-3, 1e-4, 1e-5 and 1e-6 (four extra solves, from x0 = 0,
 *               the caller's x0 restored; with x0_given that call allocates one FP64 vector of
 *               the solver to keep x0) and keeps the fastest that converges.  Batched solves
 *               use reliable updates instead and ignore it.
 *   check_every : Krylov iterations between host convergence checks (CUDA-graph replay length). */
typedef struct {
  double tol;
  int maxit;
  int precision;
  int x0_given;
  double inner_tol;
  int check_every;
} ufg_params;

/* Solve statistics.  Apply counters count kernel applications of each operator (FP64 + FP32).
 * mv_paper is the paper's MV-operation count for the iterations done (Sec. 5: CG + Chebyshev
 * 2(d+1) per iteration, BiCGStab + WCE 2(d+1)(1+2 beta) with beta = 1, CG + SCA 3, none 2). */
typedef struct {
  int status;
  int iterations;          /* Krylov iterations, summed over both steps and all inner solves */
  int iterations_step[2];  /* two-step BiCGStab: step 1 (M^T y = b), step 2 (M x = y) */
  int outer_iterations;    /* MIXED: defect-correction rounds */
  int restarts;            /* BiCGStab restarts after near-breakdown */
  long long n_M, n_Mdag, n_M1, n_M1T, n_M0inv, n_M0invT, n_sca;
  double mv_paper;
  double true_residual;    /* ||b - M^T M x|| / ||b|| in FP64 at exit */
  double seconds;          /* wall time of the call */
  double inner_tol;        /* MIXED single-problem solves: the inner tolerance used (else 0) */
  int tile_slices;         /* batched solves: time slices per slice-kernel tile of the problem's
                              (N_x, tau) group, chosen by timing at the batch's set-up (else 0) */
} ufg_stats;

/* One independent problem of a batched solve.  sigma, b, x: FP64 arrays of its own lattice size
 * (device or host pointers). */
typedef struct {
  int nx, ntau;
  double tau, g;
  const double* sigma;
  const double* b;
  double* x;
} ufg_problem;

/* Last error message of the calling thread ("" if none). */
const char* ufg_last_error(void);

/* Build version / supported lattice extents (comma-separated N_x list). */
const char* ufg_version(void);
const char* ufg_supported_nx(void);
/* Number of this library's kernels launched so far in the process (graph replays count their
 * captured kernels); for benchmarks and launch-overhead accounting. */
long long ufg_kernel_launches(void);

/* Per-kernel device timing of instrumented runs.  The paper has no counterpart: this is
 * measurement support (roofline accounting of the kernels inside a real solve).  While enabled
 * (process-wide), every kernel launch is bracketed by a pair of CUDA events on its own stream;
 * solver loops capture and replay separate CUDA graphs that contain these event nodes, so the
 * kernels are timed as they run in an ordinary solve, and each replay is read back once it has
 * finished (one extra host synchronisation per replay).  Each record carries the launch's
 * algorithmic bytes: the operand elements read and written by the work items that run (a
 * stream-ordered copy of the solver flags taken just before the launch tells which problems
 * still run), times the element size; per-mode tables of one slice are included, scalars are
 * not.  ufg_profile_enable(1) clears earlier results; (0) stops recording and keeps them.
 * Captures made while enabled must not overlap between host threads. */
typedef struct {
  char name[64];       /* kernel class, e.g. "slice fwd N16 f32" */
  long long launches;
  double total_ms;     /* sum of the CUDA-event durations */
  double bytes;        /* sum of the algorithmic bytes */
} ufg_kernel_stat;
ufg_status ufg_profile_enable(int on);
/* Measured multiply-add throughput of the current GPU in precision UFG_FP64 or UFG_FP32, in
 * TFLOP/s (2 flops per FMA): a register-resident kernel of independent FMA chains filling every
 * SM, timed with CUDA events on stream over five launches after one warm-up.  The roofline
 * denominator of the applies that the arithmetic pipe rather than HBM bounds (FP64 on this part).
 * Allocates and frees a small output buffer; synchronises stream. */
ufg_status ufg_measure_fma_rate(int precision, void* stream, double* tflops);
/* Synchronises the device and aggregates the records by name into out[0 .. min(max, n) - 1],
 * sorted by total time (largest first); *n receives the number of distinct names.  out may be
 * NULL with max = 0 to query n. */
ufg_status ufg_profile_read(ufg_kernel_stat* out, int max, int* n);

/* Lattice N_x^3 x N_tau with time step tau and coupling g (Sec. 1; the paper uses tau = 0.05,
 * g in {2.5, 5, 7.5}).  dispersion 0: E(k) = k^2/2 (the paper's choice, hbar = m = 1);
 * dispersion 1: E(k) = sum_i (1 - cos k_i), a Hubbard-type lattice dispersion (Sec. 6).
 * N_x must be even and one of ufg_supported_nx(); N_tau >= 3 (<= 1024); tau > 0; g >= 0.
 * Builds the FP64 line-operator tables on the host and the per-mode table exp(-tau E(k)) on the
 * current device. */
ufg_status ufg_lattice_create(int nx, int ntau, double tau, double g, int dispersion,
                              ufg_lattice** out);
/* The same on a lattice of `dim` spatial dimensions, N_x^dim x N_tau with dim in {1, 2, 3}: the
 * method carries over to lower dimensions with only the kinetic factor changed (Sec. 6; there
 * exp(-tau K) = T on a 1-D slice and T (x) T on a 2-D slice).  Vectors are [N_tau][N_x]^dim,
 * x fastest.  dim = 3 is ufg_lattice_create.  On dim 1 and 2 every apply, the solvers, the
 * preconditioners, the force and the trajectories run on generic shared-memory slice kernels;
 * the 3-D-only paths (TMA-staged and fused momentum-space kernels, the one-kernel Q, the
 * momentum basis, ufg_apply_M_momentum, ufg_lattice_autotune and batched solves) are not used
 * or return UFG_UNSUPPORTED. */
ufg_status ufg_lattice_create_dim(int dim, int nx, int ntau, double tau, double g,
                                  int dispersion, ufg_lattice** out);
void ufg_lattice_destroy(ufg_lattice* lat);
/* Coupling A of the lattice (Sec. 1). */
double ufg_lattice_coupling(const ufg_lattice* lat);
/* Device-side failure check for asynchronous applies.  The TMA-staged kernels wait for their
 * shared-memory copies with a bounded number of polling rounds (under a second); a wait that runs
 * out raises a flag of the lattice and the kernel finishes on incomplete data.  Solves, the force
 * and batched solves read the flags themselves and return UFG_TIMEOUT; after applies, call this:
 * it synchronises stream, reads and clears the flag of lat, and returns UFG_TIMEOUT (with a
 * message) if any kernel launched on the lattice since the last check ran out of its wait, else
 * UFG_OK.  The paper has no counterpart (failure reporting of this library). */
ufg_status ufg_lattice_check(const ufg_lattice* lat, void* stream);
/* Test hook for the failure path above: the next `launches` TMA-staged slice-kernel launches (in
 * any lattice of the process) each run one extra bounded wait on a barrier whose expected bytes
 * never arrive, so that wait runs out after a few hundred polling rounds and raises the flag
 * exactly as a real timeout would.  The kernel's own copies complete as usual, nothing faults or
 * hangs, and the results stay correct; only the reported status changes.  0 cancels. */
void ufg_test_expire_waits(int launches);
/* Autotuner: times the fused M apply for every compiled launch shape (CTAs per cluster C, time
 * slices per CTA) on this lattice, in FP64 and FP32, and keeps the fastest for all later applies
 * and solves built on the lattice.  Results are cached per (GPU name, N_x, N_tau, precision) in
 * the process and, if the environment variable UFG_TUNE_CACHE names a file, appended to it and
 * read back by later processes.  Allocates and frees three temporary vectors; call it before any
 * stream capture.  Synchronises stream. */
ufg_status ufg_lattice_autotune(ufg_lattice* lat, void* stream);
/* The launch shape in use for a precision (UFG_FP64 / UFG_FP32): C = 0 means the TMA-staged
 * kernel (one time slice per CTA or cluster); otherwise C CTAs per cluster and spc slices per
 * CTA of the shared-memory-staged kernel. */
ufg_status ufg_lattice_launch_shape(const ufg_lattice* lat, int precision, int* C, int* spc);

/* Auxiliary field: copies sigma (device FP64, [N_tau][N_x]^3) and derives per site, in FP64 and
 * FP32, w = 1 + A sin sigma (B_t), s = sin sigma (C_t of Eq. MatrixM_1), c = A cos sigma (force),
 * calling CUDA's sin/cos.  Asynchronous on stream; sigma may be freed after the call returns
 * only once the stream has passed it. */
ufg_status ufg_field_create(const ufg_lattice* lat, const double* sigma, void* stream,
                            ufg_field** out);
/* Replaces sigma of an existing field (HMC step); same rules as ufg_field_create. */
ufg_status ufg_field_update(ufg_field* f, const double* sigma, void* stream);
void ufg_field_destroy(ufg_field* f);

/* y = M x (Eq. MatrixM), y = M^T x, y = M^T M x (Eq. 1), y = M1 x and y = M1^T x (Eq. MatrixM_1),
 * y = exp(-tau K) x on every slice, y = M0^{-1} x and y = M0^{-T} x (Sec. 3, exact: diagonal
 * [1 - exp(-i omega - tau E(k))]^{-1} in frequency-momentum space, omega = (2n+1) pi / N_tau).
 * precision UFG_FP64: x, y are double*; UFG_FP32: float*.  x and y must not overlap.  Q and
 * M0^{-1}/M0^{-T} use library workspace of the field, so calls on one field must not overlap in
 * time on different streams.  Q on a 16^3 lattice with 3 <= N_tau <= twice the GPU's SM count
 * runs as one kernel per output slice (x at t-1, t, t+1 in shared memory, three kinetic
 * stages, no intermediate vector); elsewhere as M followed by M^T. */
ufg_status ufg_apply_M(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_Mdag(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_Q(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_M1(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_M1T(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_kinetic(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_M0inv(ufg_field* f, const void* x, void* y, int precision, void* stream);
ufg_status ufg_apply_M0invT(ufg_field* f, const void* x, void* y, int precision, void* stream);

/* The momentum basis of Sec. 3 (Fourier acceleration).  ufg_fourier: y = F x (inverse = 0) or
 * y = F^T x (inverse = 1) on every slice, with F the orthogonal real Fourier basis in which
 * exp(-tau K) is diagonal (F^T F = 1, so norms and inner products are those of position space).
 * A momentum-space vector has the position-space shape [N_tau][N_x^3]; its modes are stored in
 * the library's per-axis slot order (cos and sin slots of each 1-D momentum), not FFT order.
 * ufg_apply_M_momentum: y^ = F M F^T x^ (transpose = 0) or F M^T F^T x^ (transpose = 1), one
 * fused kernel per slice (inverse transform, site multiplier, forward transform, the M0 part of
 * Sec. 3 and the identity).  Built for FP32 N_x = 16 and FP64 N_x = 8, 16; UFG_INVALID_ARG
 * elsewhere.  Same precision, alignment and overlap rules as the applies above; precision
 * UFG_FP64_EMULATED also takes FP64 vectors (double-float arithmetic). */
ufg_status ufg_fourier(ufg_field* f, const void* x, void* y, int precision, int inverse,
                       void* stream);
ufg_status ufg_apply_M_momentum(ufg_field* f, const void* x, void* y, int precision,
                                int transpose, void* stream);

/* Solver workspace for one lattice (all vectors the solvers and preconditioners need, FP64 and
 * FP32). */
ufg_status ufg_solver_create(const ufg_lattice* lat, ufg_solver** out);
void ufg_solver_destroy(ufg_solver* s);

/* Selects the preconditioner of the following solves.  UFG_PC_CHEB and UFG_PC_SCA precondition
 * Q = M^T M (CG); UFG_PC_WCE preconditions M and M^T separately (two-step BiCGStab) or, for CG,
 * Q from both sides. */
ufg_status ufg_set_preconditioner(ufg_solver* s, int kind, const ufg_pc_params* p);

/* z = P r with the current preconditioner: Chebyshev P(Q/s)/s ~ Q^{-1}; SCA (L^T D L)^{-1};
 * WCE P_d ~ M^{-1} (transpose = 1: P_d^T ~ M^{-T}; transpose = 2: P_d P_d^T ~ Q^{-1}, the SPD form
 * CG on the normal equations uses: M0^{-T} on the left and M0^{-1} on the right, end of Sec. 5).
 * For tests and for callers composing their own solvers. */
ufg_status ufg_apply_preconditioner(ufg_solver* s, ufg_field* f, const void* r, void* z,
                                    int transpose, int precision, void* stream);

/* Solves M^T M x = b by preconditioned CG (Eq. 1 with the left/SPD preconditioning of Eq. 3):
 * Chebyshev, SCA, or the weak-coupling series applied from both sides (P_d P_d^T).
 * b, x: FP64, device or host pointers (host buffers are staged through the workspace). */
ufg_status ufg_solve_cg_normal(ufg_solver* s, ufg_field* f, const double* b, double* x,
                               const ufg_params* p, ufg_stats* stats, void* stream);

/* Solves M^T y = b, then M x = y (Eq. 2) by right-preconditioned BiCGStab (van der Vorst 1992),
 * with P_d^T for the first and P_d for the second step when the WCE preconditioner is set.
 * Step 1 runs to tol/2, step 2 to tol ||b|| / (2 (2 + A) ||y||); the composite residual
 * ||b - M^T M x|| / ||b|| is checked at exit and one more correction round runs if needed. */
ufg_status ufg_solve_bicgstab_two_step(ufg_solver* s, ufg_field* f, const double* b, double* x,
                                       const ufg_params* p, ufg_stats* stats, void* stream);

/* HMC force of the pseudofermion action S = phi^T (M^T M)^{-1} phi (Sec. 1): solves
 * X = Q^{-1} phi with the two-step BiCGStab (WCE preconditioner if set; should its near-breakdown
 * persist, CG on M^T M with the Chebyshev preconditioner of degree 16 finishes the solve from the
 * BiCGStab iterate, and stats then describe that CG solve with the BiCGStab iterations added;
 * the solver's own preconditioner setting is kept) and returns
 * dS/dsigma_t(r) = 2 A cos sigma_t(r) X_t(r) [exp(-tau K) Y~_{t+1}](r), Y = M X, Y~_{N_tau} = -Y_0
 * (the paper's F with the opposite sign).  phi: device FP64.  dS (nullable: solve and action
 * only), X_out (nullable): device FP64; S_out (nullable, host) receives S. */
ufg_status ufg_hmc_force(ufg_solver* s, ufg_field* f, const double* phi, double* dS,
                         double* X_out, double* S_out, const ufg_params* p, ufg_stats* stats,
                         void* stream);
/* dS = scale * dS/dsigma from a given solution X = Q^{-1} phi (device FP64): Y = M X is recomputed
 * into solver workspace, then one fused slice kernel forms the force.  Asynchronous on stream. */
ufg_status ufg_force_from_solution(ufg_solver* s, ufg_field* f, const double* X, double* dS,
                                   double scale, void* stream);

/* Statistics of one HMC trajectory. */
typedef struct {
  int status;          /* UFG_OK, or the status of the force solve that failed */
  int accepted;        /* 1: the proposal was accepted (the field holds it), 0: rejected */
  int md_steps;        /* leapfrog steps done */
  int force_solves;    /* solves of M^T M X = phi (n_steps + 1) */
  long long iterations;  /* Krylov iterations summed over those solves */
  double H_old, H_new, dH;         /* MD Hamiltonian sum pi^2/2 + S_p before and after */
  double action_old, action_new;   /* S_p = phi^T (M^T M)^{-1} phi before and after */
  double seconds;
} ufg_hmc_stats;

/* One trajectory of the phi-algorithm of Sec. 1: pseudofermion heat bath phi = M^T[sigma] eta,
 * molecular dynamics of d sigma/dt = pi, d pi/dt = -dS_p/dsigma under H = sum pi^2/2 + S_p with
 * n_steps leapfrog steps of size dt (a half step in pi, then full steps, a final half step:
 * reversible and area-preserving), and a Metropolis accept/reject of exp(-dH) against u.  The
 * random numbers are the caller's: eta and pi0 (device FP64 [N_tau][N_x]^3, each N(0,1)) and
 * u in [0, 1).  Every force is ufg_hmc_force with the solver's preconditioner and p.  The field
 * holds the new sigma on acceptance and the old one otherwise; sigma_out and pi_out (nullable,
 * device or host FP64) receive the field's sigma and the final momenta.  The first call allocates
 * five FP64 vectors of the solver (kept until ufg_solver_destroy).  Synchronises stream. */
ufg_status ufg_hmc_trajectory(ufg_solver* s, ufg_field* f, const double* eta, const double* pi0,
                              double u, int n_steps, double dt, const ufg_params* p,
                              double* sigma_out, double* pi_out, ufg_hmc_stats* stats,
                              void* stream);

/* n independent problems of mixed lattice sizes, each solved by two-step BiCGStab with the
 * preconditioner settings pc_kind (UFG_PC_NONE or UFG_PC_WCE)/pc, all problems advanced together
 * by batched kernels (one launch per phase per lattice extent for the whole batch) with the
 * iteration body captured in a CUDA graph; a composite-residual correction round runs for the
 * problems that need it.  Batched N_x: 4..16 (even, built), 3 <= N_tau <= 512.  sigma, b, x of
 * each problem may be device or host pointers.  The workspace of a batch (arenas sized to the sum
 * of the problems, tile tables, graphs) is allocated on the first call with a given list of
 * shapes and kept for later calls with the same shapes (two such workspaces at most); release it
 * with ufg_batch_cache_clear.  Calls are serialised by a library lock.  stats: n entries
 * (nullable).  Returns the first non-OK problem status, UFG_OK if all converged. */
ufg_status ufg_solve_batch(int n, const ufg_problem* probs, int pc_kind, const ufg_pc_params* pc,
                           const ufg_params* p, ufg_stats* stats, void* stream);
/* Frees the cached batch workspaces. */
void ufg_batch_cache_clear(void);

/* y = M^T M x in FP64 without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc where they need the operator (code
 * under a memory pool or arena that forbids extra allocations, or a plugin that must not grow the
 * process's device footprint after start-up).  sigma, x, y: device FP64 [N_tau][N_x]^3, 16-byte
 * aligned, x and y not overlapping; the lattice (N_x, N_tau, tau, g, dispersion) is as in
 * ufg_lattice_create.  The two intermediates (1 + A sin sigma and M x) live in a file-scope static
 * device array of 2 x 2^20 doubles (16 MiB) that every GPU loading the library holds until exit,
 * so N_x^3 N_tau must be <= 2^20 sites (UFG_INVALID_ARG otherwise, with a message).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current.  Every call overwrites the whole used
 * part of the array before reading it, so nothing needs clearing, but calls share the array:
 * calls that overlap on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  It runs the shared-memory-staged slice kernels, which have no
 * bounded device wait, so it has no failure flag to read.  Asynchronous on stream. */
ufg_status ufg_apply_Q_noalloc(int nx, int ntau, double tau, double g, int dispersion,
                               const double* sigma, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UFG_H */
