// Q = M^T M applied without any device allocation, for callers that cannot call cudaMalloc.
//
// Some host programs cannot allocate device memory at the point where they need the operator:
// code running inside a pool or arena whose owner forbids extra allocations, or a plugin that must
// not grow the process's device footprint after start-up.
// This entry point serves them: the caller passes sigma, x and y; the library keeps its two
// intermediates (w = 1 + A sin sigma and the half-product M x) in a file-scope device array of fixed
// size that every GPU loading the library holds until the process exits.  No cudaMalloc, cudaFree
// or allocating library routine is called.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "line_ops.cuh"
#include "ufg_internal.h"
#include "launch.cuh"

namespace ufg {

// Largest lattice the static scratch serves: N_x^3 N_tau <= 2^20 sites (e.g. 16^3 x 256); two
// FP64 intermediates of that size = 16 MiB of device memory per GPU.
constexpr long long NOALLOC_MAX_SITES = 1LL << 20;

static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_SITES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_ptr[MAX_DEVICES] = {nullptr};

// The host-side name of g_noalloc_scratch is only a stand-in; kernels need the device address,
// resolved once per device with that device current.
ufg_status scratch_for_current_device(double** out) {
  int dev = 0;
  UFG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device index %d out of range", dev);
    return UFG_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return UFG_OK;
}

__global__ void noalloc_w_kernel(const double* __restrict__ sigma, double A, long long S,
                                 double* w) {
  pdl_begin();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;
       i += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincos(sigma[i], &sn, &cs);
    w[i] = 1.0 + A * sn;
  }
}

// exp(-tau K) along one axis as the even/odd reduced matrices: the circulant
// T[d] = (1/N) sum_n exp(-tau E1(k_n)) cos(k_n d), then
//   ce[i][0] = T[i], ce[i][H] = T[i-H], ce[i][j] = (T[i-j] + T[i+j]) / 2,
//   co[i][j] = (T[i-j] - T[i+j]) / 2   (indices mod N),
// split further into the kernel's coefficient layout (host memory only).
template <int N>
bool kinetic_coef(double tau, int dispersion, LineCoef<N, double>* c) {
  constexpr int H = N / 2;
  const double pi = 3.14159265358979323846;
  double T[N];
  for (int d = 0; d < N; ++d) {
    double acc = 0.0;
    for (int m = 0; m < N; ++m) {
      const int n = m < H ? m : m - N;
      const double k = 2.0 * pi * n / N;
      const double e1 = dispersion == 0 ? 0.5 * k * k : 1.0 - std::cos(k);
      acc += std::exp(-tau * e1) * std::cos(k * d);
    }
    T[d] = acc / N;
  }
  auto t = [&](int d) { return T[((d % N) + N) % N]; };
  std::vector<double> ce((H + 1) * (H + 1)), co((H - 1) * (H - 1)), flat;
  for (int i = 0; i <= H; ++i)
    for (int j = 0; j <= H; ++j)
      ce[i * (H + 1) + j] = (j == 0 || j == H) ? t(i - j) : 0.5 * (t(i - j) + t(i + j));
  for (int i = 1; i < H; ++i)
    for (int j = 1; j < H; ++j) co[(i - 1) * (H - 1) + (j - 1)] = 0.5 * (t(i - j) - t(i + j));
  if (!line_coef_flat(N, ce, co, false, false, flat) || (int)flat.size() != LineShape<N>::NC)
    return false;
  for (int i = 0; i < LineShape<N>::NC; ++i) c->c[i] = flat[i];
  return true;
}

template <int N>
ufg_status run_q(int ntau, double tau, int dispersion, double A, const double* x, double* y,
                 double* w, double* t, cudaStream_t st) {
  LineCoef<N, double> coef;
  if (!kinetic_coef<N>(tau, dispersion, &coef)) {
    set_error("apply_Q_noalloc: kinetic line operator does not split");
    return UFG_INTERNAL;
  }
  SliceCall c;
  c.fam = FAM_KIN;
  c.prec = 0;
  c.coef = &coef;
  c.ntau = ntau;
  // the shared-memory-staged kernels: they contain no bounded device wait, so nothing can run
  // out and there is no failure flag that would need a device allocation or a read-back here
  c.allow_tma = 0;
  // launch shape as for a lattice of this size (4-CTA clusters for 32^3 FP64 slices)
  if (N >= 32) {
    c.C = 4;
    c.spc = 1;
  } else {
    const size_t slice = (size_t)N * N * (N + 1) * sizeof(double);
    int spc = 1;
    while (spc < 8 && slice * (spc * 2) <= 48 * 1024 && ntau / (spc * 2) >= 152) spc *= 2;
    c.C = 1;
    c.spc = spc;
  }
  (void)A;
  SliceCall m = c;  // t = M x
  m.in = x;
  m.pre = w;
  m.id = x;
  m.shift = -1;
  m.out = t;
  cudaError_t e = slice_dispatch(N, m, st);
  if (e != cudaSuccess) return cuda_fail(e, "slice kernel (M)");
  note_launches(1);
  SliceCall md = c;  // y = M^T t
  md.in = t;
  md.post = w;
  md.id = t;
  md.shift = +1;
  md.out = y;
  e = slice_dispatch(N, md, st);
  if (e != cudaSuccess) return cuda_fail(e, "slice kernel (M^T)");
  note_launches(1);
  return UFG_OK;
}

}  // namespace
}  // namespace ufg

using namespace ufg;

extern "C" ufg_status ufg_apply_Q_noalloc(int nx, int ntau, double tau, double g, int dispersion,
                                          const double* sigma, const double* x, double* y,
                                          void* stream) {
  clear_error();
  if (nx < 4 || nx % 2 || !slice_supported_n(nx) || ntau < 3 || !(tau > 0) || !(g >= 0) ||
      !std::isfinite(tau) || !std::isfinite(g) || (dispersion != 0 && dispersion != 1)) {
    set_error("apply_Q_noalloc: invalid lattice (N_x=%d N_tau=%d tau=%g g=%g dispersion=%d; "
              "N_x one of %s)", nx, ntau, tau, g, dispersion, ufg_supported_nx());
    return UFG_INVALID_ARG;
  }
  const long long S = (long long)nx * nx * nx * ntau;
  if (S > NOALLOC_MAX_SITES) {
    set_error("apply_Q_noalloc: lattice of %lld sites exceeds the static scratch limit of %lld "
              "sites (N_x^3 N_tau); use ufg_apply_Q with a field", S, NOALLOC_MAX_SITES);
    return UFG_INVALID_ARG;
  }
  if (!sigma || !x || !y || ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) |
                              reinterpret_cast<uintptr_t>(sigma)) & 15u)) {
    set_error("apply_Q_noalloc: null or non-16-byte-aligned pointer");
    return UFG_INVALID_ARG;
  }
  const char* xa = reinterpret_cast<const char*>(x);
  const char* ya = reinterpret_cast<const char*>(y);
  const size_t bytes = (size_t)S * sizeof(double);
  if (xa < ya + bytes && ya < xa + bytes) {
    set_error("apply_Q_noalloc: x and y overlap");
    return UFG_INVALID_ARG;
  }
  double* scratch = nullptr;
  UFG_TRY(scratch_for_current_device(&scratch));
  double* w = scratch;                      // [0, S): 1 + A sin sigma
  double* t = scratch + NOALLOC_MAX_SITES;  // [MAX, MAX + S): M x
  const double A = std::sqrt(2.0) * std::sqrt(std::expm1(tau * g));
  cudaStream_t st = as_stream(stream);
  long long blocks = (S + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  noalloc_w_kernel<<<(unsigned)blocks, 256, 0, st>>>(sigma, A, S, w);
  UFG_CUDA(cudaGetLastError());
  note_launches(1);
  switch (nx) {
    case 4: return run_q<4>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 6: return run_q<6>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 8: return run_q<8>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 10: return run_q<10>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 12: return run_q<12>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 16: return run_q<16>(ntau, tau, dispersion, A, x, y, w, t, st);
    case 32: return run_q<32>(ntau, tau, dispersion, A, x, y, w, t, st);
  }
  set_error("apply_Q_noalloc: N_x=%d not built", nx);
  return UFG_UNSUPPORTED;
}
