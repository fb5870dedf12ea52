// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <string>
#include <vector>

#include "slice_call.h"
#include "ufg.h"

namespace ufg {

// ---- errors -------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
ufg_status cuda_fail(cudaError_t e, const char* what);

#define UFG_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::ufg::cuda_fail(e_, #call);      \
  } while (0)

#define UFG_TRY(call)                                               \
  do {                                                              \
    ufg_status s_ = (call);                                         \
    if (s_ != UFG_OK) return s_;                                    \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Kernel-launch accounting (every launch of this library's kernels, graph replays included).
void note_launches(long long n);
long long launches_so_far();

// ---- per-kernel timing of instrumented runs (ufg_profile_enable) ---------------------------
bool profiling();
// CUDA-graph replay of solver loops (off with UFG_NO_GRAPH=1)
bool graphs_enabled();
// Which work a launch does, for its algorithmic bytes: site_bytes[i] bytes for each problem i
// whose solver flag lets it run (exec_if < 0: always), plus fixed_bytes.  The flags are copied on
// the launch's stream just before it (flag i at flag_dev + i * stride bytes), so the stream is
// never drained and the events time the kernel alone; the bytes are resolved when read.
struct LaunchWork {
  const int* flag_dev = nullptr;  // nullptr: every problem runs
  size_t stride = sizeof(int);
  int exec_if = -1;
  std::vector<double> site_bytes;
  double fixed_bytes = 0.0;
};
// Brackets the launches issued during its lifetime with CUDA events on `st` (no-op unless
// profiling).
class KTimer {
 public:
  KTimer(const std::string& name, cudaStream_t st, LaunchWork work);
  ~KTimer();
  KTimer(const KTimer&) = delete;
  KTimer& operator=(const KTimer&) = delete;

 private:
  long long idx_ = -1;
  cudaStream_t st_ = nullptr;
  bool cap_ = false;
};
// Graph hooks: records made between capture_begin and capture_end belong to that graph and are
// timed again after each replay (after_replay synchronises the stream while profiling).
void profile_capture_begin();
void profile_capture_end(cudaGraphExec_t ex);
void profile_after_replay(cudaGraphExec_t ex, cudaStream_t st);
void profile_graph_destroyed(cudaGraphExec_t ex);
// "slice <family>[+epilogue operands] N<n> f32|f64" and the algorithmic bytes of one slice launch
// per site and per problem (its per-mode tables).
std::string slice_kernel_name(const SliceCall& c, int N);
double slice_bytes_per_site(const SliceCall& c);
double slice_bytes_per_problem(const SliceCall& c, int N);

// Flat line-operator coefficients (LineCoef layout, line_ops.cuh) from the first-level blocks ce,
// co of an operator; false if the second-level split does not hold.
bool line_coef_flat(int N, const std::vector<double>& ce, const std::vector<double>& co,
                    bool in_spec, bool out_spec, std::vector<double>& flat);

// Weights c_0..c_d of the weak-coupling series under the acceleration `accel` (ufg_accel) with
// Euler parameter p and van Wijngaarden parameter s (Sec. 3.1); false on invalid arguments.
bool wce_series_weights(int d, int accel, double p, double s, std::vector<double>& c);
// Validated copy of preconditioner parameters with the defaults applied (euler_p 0 -> 1/2,
// vw_s 0 -> 1); UFG_INVALID_ARG with a message otherwise.
ufg_status normalize_pc(int kind, const ufg_pc_params* in, ufg_pc_params* out);

// ---- small device buffers -----------------------------------------------------------------
template <typename T>
ufg_status dev_alloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return UFG_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
    return UFG_OOM;
  }
  return UFG_OK;
}
template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// ---- kernels living in other translation units --------------------------------------------
// Per-site potentials from sigma (FP64 in, FP64 + FP32 out).
cudaError_t launch_potentials(const double* sigma, double A, long long S, double* w64, double* s64,
                              double* c64, float* w32, float* s32, float* c32, cudaStream_t st);
// Exact M0^{-1} (transpose = 0) or M0^{-T} time recurrence per momentum mode, in place allowed.
// out (nullable) = out_scale * x; acc_mode 0: none, 1: acc = acc_coef * x, 2: acc += acc_coef * x.
// acc_mode 3: acc = acc_coef * x + c0 * e0 + c1 * e1 (the earlier terms of a series).
cudaError_t launch_recurrence(int prec, const void* in, void* out, const void* bk, long long V,
                              int ntau, int transpose, double out_scale, void* acc,
                              double acc_coef, int acc_mode, const int* done, cudaStream_t st,
                              const void* e0 = nullptr, const void* e1 = nullptr,
                              double c0 = 0.0, double c1 = 0.0);
// Batched form: one CTA per (problem, 32-mode block) tile; max_ntau bounds every problem's N_tau.
// acc_mode 3 as above.
cudaError_t launch_recurrence_batch(int prec, const void* in, void* out, const void* bk,
                                    int max_ntau, int transpose, double out_scale, void* acc,
                                    double acc_coef, int acc_mode, int exec_if, const int2* tiles,
                                    int ntiles, const BatchProb* probs, cudaStream_t st,
                                    const void* e0 = nullptr, const void* e1 = nullptr,
                                    double c0 = 0.0, double c1 = 0.0);
// Strong-coupling factors (per site, sequential in t) and apply.
cudaError_t launch_sca_setup(const double* w64, long long V, int ntau, double alpha, double* L64,
                             double* Di64, float* L32, float* Di32, cudaStream_t st);
// z = a (L^T D L)^{-1} y + bU U + cV W (U, W nullable and not aliasing z).
cudaError_t launch_sca_apply(int prec, const void* L, const void* Di, const void* y, void* z,
                             long long V, int ntau, const int* done, cudaStream_t st,
                             double a = 1.0, const void* U = nullptr, double bU = 0.0,
                             const void* W = nullptr, double cV = 0.0);

}  // namespace ufg

// ---- handles ------------------------------------------------------------------------------
struct ufg_lattice;
namespace ufg {
// Reads (synchronising st) and clears the lattice's device flag of bounded waits; UFG_TIMEOUT with
// a message if a wait of a kernel launched since the last check ran out.
ufg_status check_device_flag(const ufg_lattice* lat, cudaStream_t st);
}  // namespace ufg

struct ufg_lattice {
  int nx = 0, ntau = 0, dispersion = 0;
  int dim = 3;  // spatial dimension (1 and 2: slice_lowd.cuh; the fused 3-D kernels are off)
  double tau = 0, g = 0, A = 0;
  long long V = 0, S = 0;
  std::vector<double> lam;                 // exp(-tau E1) per 1-D spectral slot
  std::vector<unsigned char> coef[3][2];   // reduced line matrices [family][0 FP64 / 1 FP32]
  double* bk64 = nullptr;                  // per-mode exp(-tau E(k)), spectral layout [V]
  float* bk32 = nullptr;
  int* dev_err = nullptr;                  // device flag of bounded waits that ran out
  int spc[2] = {1, 1};                     // slices per CTA (KIN family) per precision
  int C[2] = {1, 1};                       // cluster size per precision
  int use_tma[2] = {1, 1};                 // TMA-staged slice kernel where it applies
  int device = 0;
};

struct ufg_field {
  const ufg_lattice* lat = nullptr;
  // process-unique identity: captured solver graphs are cached per field, and a field created
  // after another was destroyed may get the same host address but different device buffers
  unsigned long long id = 0;
  double* sigma = nullptr;
  double* w64 = nullptr;
  double* s64 = nullptr;
  double* c64 = nullptr;
  float* w32 = nullptr;
  float* s32 = nullptr;
  float* c32 = nullptr;
  double* tmp64 = nullptr;  // apply workspace (Q intermediate, momentum-space temp)
  float* tmp32 = nullptr;
  double sca_alpha = -1.0;  // alpha the SCA tables were built for (< 0: none)
  double gcheb_alpha = -1.0;  // alpha of the spectral estimate of (L^T D L)^{-1} Q (< 0: none)
  double gcheb_scale = 0.0;
  double* L64 = nullptr;
  double* Di64 = nullptr;
  float* L32 = nullptr;
  float* Di32 = nullptr;
};

namespace ufg {

// Generic slice-kernel call prefilled for a field/lattice and precision.
SliceCall base_call(const ufg_lattice* lat, int fam, int prec);
// Operator applications used by the C ABI and by the solvers (vectors in precision prec).
ufg_status op_M(const ufg_field* f, int prec, const void* x, void* y, cudaStream_t st);
ufg_status op_Mdag(const ufg_field* f, int prec, const void* x, void* y, cudaStream_t st);
ufg_status op_M0inv(const ufg_field* f, int prec, const void* x, void* y, void* tmp, int transpose,
                    cudaStream_t st);
ufg_status ensure_sca(ufg_field* f, double alpha, cudaStream_t st);
const void* fld(const ufg_field* f, char which, int prec);  // 'w', 's', 'c'

}  // namespace ufg
