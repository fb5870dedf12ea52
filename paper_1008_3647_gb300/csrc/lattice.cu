// Lattice and field handles, the host-side construction of the line-operator tables, and the
// C-ABI operator applications (M, M^T, Q, M1, M1^T, kinetic, M0^{-1}, M0^{-T}).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "launch.cuh"
#include "line_ops.cuh"
#include "ufg_internal.h"

namespace ufg {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Off for the solvers: on the batched 16^3 solve it measured slower (107.3 vs 102.1 ms per
// solve), the early-launched dependent CTAs only waiting on the previous grid.  On for
// standalone operator calls (back-to-back 32^3 x 512 applies: about 1.5 us less per call).
// UFG_PDL=1 turns it on everywhere.
static thread_local int g_pdl_scope = 0;
PdlScope::PdlScope() { ++g_pdl_scope; }
PdlScope::~PdlScope() { --g_pdl_scope; }
bool pdl_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("UFG_PDL");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1 || g_pdl_scope > 0;
}
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

// Test hook: the number of coming TMA slice launches that run one wait made to run out.
static std::atomic<int> g_expire{0};

int take_expired_wait(cudaStream_t st) {
  // never baked into a captured graph: its replays would all run the expiring wait
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 0;
  }
  int n = g_expire.load(std::memory_order_relaxed);
  while (n > 0 && !g_expire.compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) {
  }
  return n > 0 ? 1 : 0;
}

ufg_status check_device_flag(const ufg_lattice* lat, cudaStream_t st) {
  if (lat == nullptr || lat->dev_err == nullptr) return UFG_OK;
  int h = 0;
  UFG_CUDA(cudaMemcpyAsync(&h, lat->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  UFG_CUDA(cudaStreamSynchronize(st));
  if (h == 0) return UFG_OK;
  UFG_CUDA(cudaMemsetAsync(lat->dev_err, 0, sizeof(int), st));
  UFG_CUDA(cudaStreamSynchronize(st));
  set_error("a bounded device wait ran out (a TMA copy into shared memory did not complete); "
            "the results of the kernels launched since the last check are invalid");
  return UFG_TIMEOUT;
}

ufg_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return UFG_CUDA_ERROR;
}

// ---------------------------------------------------------------------------------------------
// Line-operator tables (FP64 on the host).
//
// 1-D spectrum: frequency n (numpy-style order, k = 2 pi n'/N with n' = n for n < N/2 and n - N
// otherwise, i.e. n' in -N/2..N/2-1, Sec. 1) has eigenvalue lam(n) = exp(-tau E1(k)),
// E1 = k^2/2 (dispersion 0) or 1 - cos k (dispersion 1); exp(-tau E(k)) = prod_i lam(n_i).
//
// Real orthonormal basis F (columns = spectral slots): slot 0 constant, slots 1..H-1 cosines,
// slot H the alternating vector, slots H+1..N-1 sines.  T = F diag(lam_slot) F^T is exp(-tau K)
// along one axis, a real symmetric circulant.
// ---------------------------------------------------------------------------------------------
static double e1(double k, int dispersion) {
  return dispersion == 0 ? 0.5 * k * k : 1.0 - std::cos(k);
}

static void basis(int N, std::vector<double>& F /*N x N, F[x*N+slot]*/, std::vector<int>& freq) {
  const int H = N / 2;
  F.assign((size_t)N * N, 0.0);
  freq.assign(N, 0);
  const double pi = 3.14159265358979323846;
  for (int x = 0; x < N; ++x) {
    F[x * N + 0] = 1.0 / std::sqrt((double)N);
    F[x * N + H] = ((x & 1) ? -1.0 : 1.0) / std::sqrt((double)N);
    for (int i = 1; i < H; ++i) {
      F[x * N + i] = std::sqrt(2.0 / N) * std::cos(2.0 * pi * i * x / N);
      F[x * N + H + i] = std::sqrt(2.0 / N) * std::sin(2.0 * pi * i * x / N);
    }
  }
  freq[0] = 0;
  freq[H] = H;
  for (int i = 1; i < H; ++i) {
    freq[i] = i;
    freq[H + i] = i;
  }
}

// Reduces a full N x N operator (y = A v) to its even/odd blocks for the given input/output
// representations; returns false if the operator mixes even and odd parts.
static bool reduce(int N, const std::vector<double>& A, bool in_spec, bool out_spec,
                   std::vector<double>& ce, std::vector<double>& co) {
  const int H = N / 2;
  ce.assign((H + 1) * (H + 1), 0.0);
  co.assign((H - 1) * (H - 1), 0.0);
  double cross = 0.0, scale = 0.0;
  auto to_out = [&](const std::vector<double>& y, std::vector<double>& E, std::vector<double>& O) {
    E.assign(H + 1, 0.0);
    O.assign(H + 1, 0.0);
    if (out_spec) {
      for (int i = 0; i <= H; ++i) E[i] = y[i];
      for (int i = 1; i < H; ++i) O[i] = y[H + i];
    } else {
      E[0] = y[0];
      E[H] = y[H];
      for (int i = 1; i < H; ++i) {
        E[i] = 0.5 * (y[i] + y[N - i]);
        O[i] = 0.5 * (y[i] - y[N - i]);
      }
    }
  };
  for (int odd = 0; odd < 2; ++odd) {
    const int jlo = odd ? 1 : 0, jhi = odd ? H - 1 : H;
    for (int j = jlo; j <= jhi; ++j) {
      std::vector<double> v(N, 0.0), y(N, 0.0), E, O;
      if (in_spec) {
        v[odd ? H + j : j] = 1.0;
      } else if (!odd && (j == 0 || j == H)) {
        v[j] = 1.0;
      } else {
        v[j] = 0.5;
        v[N - j] = odd ? -0.5 : 0.5;
      }
      for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc += A[(size_t)i * N + k] * v[k];
        y[i] = acc;
      }
      to_out(y, E, O);
      for (int i = 0; i <= H; ++i) scale = std::fmax(scale, std::fabs(E[i]) + std::fabs(O[i]));
      if (!odd) {
        for (int i = 0; i <= H; ++i) ce[i * (H + 1) + j] = E[i];
        for (int i = 1; i < H; ++i) cross = std::fmax(cross, std::fabs(O[i]));
      } else {
        for (int i = 1; i < H; ++i) co[(i - 1) * (H - 1) + (j - 1)] = O[i];
        for (int i = 0; i <= H; ++i) cross = std::fmax(cross, std::fabs(E[i]));
      }
    }
  }
  return cross <= 1e-13 * std::fmax(scale, 1.0);
}

// Second-level split of one first-level block (see line_ops.cuh): M (n x n, row = output) maps
// the block's inputs to its outputs; P_in rebuilds the block's inputs from (s, a), R_out takes the
// block's outputs to (U, W).  Returns the U<-s and W<-a blocks of R_out M P_in, or false if its
// cross blocks do not vanish.
static bool split_block(int H, const std::vector<double>& M, bool sine, bool in_spec,
                        bool out_spec, std::vector<double>& Bs, std::vector<double>& Ba) {
  const int Q = H / 2;
  const int n = sine ? H - 1 : H + 1;  // block indices: j0 .. j0 + n - 1
  const int j0 = sine ? 1 : 0;
  const int ns = sine ? Q : Q + 1, na = sine ? Q - 1 : Q;
  // columns of P_in (n x (ns + na)) and rows of R_out ((ns + na) x n), in block-local indices
  std::vector<double> P((size_t)n * (ns + na), 0.0), Rm((size_t)(ns + na) * n, 0.0);
  auto at = [&](std::vector<double>& X, int rows_or_cols, int r, int c) -> double& {
    return X[(size_t)r * rows_or_cols + c];
  };
  const int ncol = ns + na;
  if (in_spec) {  // spectral side: parity selection
    for (int m = 0; m < ns; ++m) at(P, ncol, (sine ? 2 * m + 1 : 2 * m) - j0, m) = 1.0;
    for (int m = 0; m < na; ++m) at(P, ncol, (sine ? 2 * m + 2 : 2 * m + 1) - j0, ns + m) = 1.0;
  } else {  // real side: pairs (j, H - j) and the centre Q
    for (int m = 0; m < na; ++m) {
      const int j = j0 + m;
      at(P, ncol, j - j0, m) += 0.5;
      at(P, ncol, H - j - j0, m) += 0.5;
      at(P, ncol, j - j0, ns + m) += 0.5;
      at(P, ncol, H - j - j0, ns + m) -= 0.5;
    }
    at(P, ncol, Q - j0, ns - 1) = 1.0;
  }
  if (out_spec) {
    for (int m = 0; m < ns; ++m) at(Rm, n, m, (sine ? 2 * m + 1 : 2 * m) - j0) = 1.0;
    for (int m = 0; m < na; ++m) at(Rm, n, ns + m, (sine ? 2 * m + 2 : 2 * m + 1) - j0) = 1.0;
  } else {
    for (int m = 0; m < na; ++m) {
      const int j = j0 + m;
      at(Rm, n, m, j - j0) += 0.5;
      at(Rm, n, m, H - j - j0) += 0.5;
      at(Rm, n, ns + m, j - j0) += 0.5;
      at(Rm, n, ns + m, H - j - j0) -= 0.5;
    }
    at(Rm, n, ns - 1, Q - j0) = 1.0;
  }
  // B = R_out M P_in
  std::vector<double> MP((size_t)n * ncol, 0.0), B((size_t)ncol * ncol, 0.0);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < ncol; ++c) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += M[(size_t)i * n + k] * P[(size_t)k * ncol + c];
      MP[(size_t)i * ncol + c] = acc;
    }
  double scale = 0.0, cross = 0.0;
  for (int r = 0; r < ncol; ++r)
    for (int c = 0; c < ncol; ++c) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += Rm[(size_t)r * n + k] * MP[(size_t)k * ncol + c];
      B[(size_t)r * ncol + c] = acc;
      scale = std::fmax(scale, std::fabs(acc));
      if ((r < ns) != (c < ns)) cross = std::fmax(cross, std::fabs(acc));
    }
  Bs.assign((size_t)ns * ns, 0.0);
  Ba.assign((size_t)na * na, 0.0);
  for (int r = 0; r < ns; ++r)
    for (int c = 0; c < ns; ++c) Bs[(size_t)r * ns + c] = B[(size_t)r * ncol + c];
  for (int r = 0; r < na; ++r)
    for (int c = 0; c < na; ++c) Ba[(size_t)r * na + c] = B[(size_t)(ns + r) * ncol + ns + c];
  return cross <= 1e-13 * std::fmax(scale, 1.0);
}

bool line_coef_flat(int N, const std::vector<double>& ce, const std::vector<double>& co,
                    bool in_spec, bool out_spec, std::vector<double>& flat) {
  const int H = N / 2;
  flat.clear();
  const bool two = (H % 2 == 0) && N >= 8;
  if (!two) {
    flat.insert(flat.end(), ce.begin(), ce.end());
    flat.insert(flat.end(), co.begin(), co.end());
    return true;
  }
  std::vector<double> cs, ca, ss, sa;
  if (!split_block(H, ce, false, in_spec, out_spec, cs, ca) ||
      !split_block(H, co, true, in_spec, out_spec, ss, sa))
    return false;
  for (auto* b : {&cs, &ca, &ss, &sa}) flat.insert(flat.end(), b->begin(), b->end());
  return true;
}

template <typename R>
static void pack(const std::vector<double>& flat, std::vector<unsigned char>& out) {
  std::vector<R> v(flat.begin(), flat.end());
  out.resize(v.size() * sizeof(R));
  std::memcpy(out.data(), v.data(), out.size());
}

static ufg_status build_tables(ufg_lattice* L) {
  const int N = L->nx, H = N / 2;
  const double pi = 3.14159265358979323846;
  std::vector<double> F;
  std::vector<int> freq;
  basis(N, F, freq);
  L->lam.assign(N, 0.0);
  for (int s = 0; s < N; ++s) L->lam[s] = std::exp(-L->tau * e1(2.0 * pi * freq[s] / N, L->dispersion));
  (void)H;
  // T = F diag(lam) F^T; Ft = F^T; Finv = F.
  std::vector<double> T((size_t)N * N, 0.0), Ft((size_t)N * N), Fi((size_t)N * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double acc = 0.0;
      for (int s = 0; s < N; ++s) acc += F[i * N + s] * L->lam[s] * F[j * N + s];
      T[(size_t)i * N + j] = acc;
      Ft[(size_t)i * N + j] = F[(size_t)j * N + i];
      Fi[(size_t)i * N + j] = F[(size_t)i * N + j];
    }
  std::vector<double> ce, co;
  struct Spec { const std::vector<double>* A; bool in_spec, out_spec; int fam; } specs[3] = {
      {&T, false, false, FAM_KIN}, {&Ft, false, true, FAM_FWD}, {&Fi, true, false, FAM_INV}};
  for (auto& sp : specs) {
    if (!reduce(N, *sp.A, sp.in_spec, sp.out_spec, ce, co)) {
      set_error("line operator of family %d does not split into even and odd parts", sp.fam);
      return UFG_INTERNAL;
    }
    std::vector<double> flat;
    if (!line_coef_flat(N, ce, co, sp.in_spec, sp.out_spec, flat)) {
      set_error("line operator of family %d does not split at the second level", sp.fam);
      return UFG_INTERNAL;
    }
    pack<double>(flat, L->coef[sp.fam][0]);
    pack<float>(flat, L->coef[sp.fam][1]);
  }
  // per-mode table in spectral layout [sz][sy][sx] (dim 3; [sy][sx], [sx] below): the product
  // of the 1-D eigenvalues of the mode's slots
  std::vector<double> bk((size_t)L->V);
  std::vector<float> bkf((size_t)L->V);
  for (long long i = 0; i < L->V; ++i) {
    double b = 1.0;
    long long r = i;
    for (int d = 0; d < L->dim; ++d, r /= N) b *= L->lam[(size_t)(r % N)];
    bk[(size_t)i] = b;
    bkf[(size_t)i] = (float)b;
  }
  UFG_TRY(dev_alloc(&L->bk64, (size_t)L->V));
  UFG_TRY(dev_alloc(&L->bk32, (size_t)L->V));
  UFG_TRY(dev_alloc(&L->dev_err, 1));
  UFG_CUDA(cudaMemset(L->dev_err, 0, sizeof(int)));
  UFG_CUDA(cudaMemcpy(L->bk64, bk.data(), bk.size() * sizeof(double), cudaMemcpyHostToDevice));
  UFG_CUDA(cudaMemcpy(L->bk32, bkf.data(), bkf.size() * sizeof(float), cudaMemcpyHostToDevice));
  return UFG_OK;
}

// Default launch shape: ~32-70 KB of shared memory per CTA so that several CTAs share an SM.
static void default_tuning(ufg_lattice* L) {
  const int N = L->nx;
  for (int prec = 0; prec < 2; ++prec) {
    const size_t es = prec == 0 ? 8 : 4;
    if (N >= 32) {
      L->C[prec] = prec == 0 ? 4 : 2;
      L->spc[prec] = 1;
    } else {
      L->C[prec] = 1;
      const size_t slice = (size_t)N * N * (N + 1) * es;
      int spc = 1;
      while (spc < 8 && slice * (spc * 2) <= 48 * 1024 && L->ntau / (spc * 2) >= 152) spc *= 2;
      L->spc[prec] = spc;
    }
  }
}

SliceCall base_call(const ufg_lattice* lat, int fam, int prec) {
  SliceCall c;
  c.fam = fam;
  c.prec = prec;
  c.coef = lat->coef[fam][prec].data();
  c.ntau = lat->ntau;
  c.dim = lat->dim;
  c.spc = lat->spc[prec];
  c.C = lat->C[prec];
  c.err = lat->dev_err;
  c.allow_tma = lat->use_tma[prec];
  return c;
}

const void* fld(const ufg_field* f, char which, int prec) {
  switch (which) {
    case 'w': return prec ? (const void*)f->w32 : (const void*)f->w64;
    case 's': return prec ? (const void*)f->s32 : (const void*)f->s64;
    case 'c': return prec ? (const void*)f->c32 : (const void*)f->c64;
  }
  return nullptr;
}

static ufg_status run(const ufg_lattice* lat, const SliceCall& c, cudaStream_t st) {
  cudaError_t e = slice_dispatch(lat->nx, c, st);
  note_launches(1);
  if (e != cudaSuccess) return cuda_fail(e, "slice kernel launch");
  return UFG_OK;
}

ufg_status op_M(const ufg_field* f, int prec, const void* x, void* y, cudaStream_t st) {
  SliceCall c = base_call(f->lat, FAM_KIN, prec);
  c.in = x;
  c.pre = fld(f, 'w', prec);
  c.id = x;
  c.shift = -1;
  c.out = y;
  return run(f->lat, c, st);
}

ufg_status op_Mdag(const ufg_field* f, int prec, const void* x, void* y, cudaStream_t st) {
  SliceCall c = base_call(f->lat, FAM_KIN, prec);
  c.in = x;
  c.post = fld(f, 'w', prec);
  c.id = x;
  c.shift = +1;
  c.out = y;
  return run(f->lat, c, st);
}

ufg_status op_M0inv(const ufg_field* f, int prec, const void* x, void* y, void* tmp, int transpose,
                    cudaStream_t st) {
  const ufg_lattice* lat = f->lat;
  SliceCall fw = base_call(lat, FAM_FWD, prec);
  fw.in = x;
  fw.out = tmp;
  UFG_TRY(run(lat, fw, st));
  const void* bk = prec ? (const void*)lat->bk32 : (const void*)lat->bk64;
  cudaError_t e = launch_recurrence(prec, tmp, tmp, bk, lat->V, lat->ntau, transpose, 1.0, nullptr,
                                    0.0, 0, nullptr, st);
  note_launches(1);
  if (e != cudaSuccess) return cuda_fail(e, "recurrence kernel launch");
  SliceCall iv = base_call(lat, FAM_INV, prec);
  iv.in = tmp;
  iv.out = y;
  return run(lat, iv, st);
}

ufg_status ensure_sca(ufg_field* f, double alpha, cudaStream_t st) {
  if (f->sca_alpha == alpha && f->L64 != nullptr) return UFG_OK;
  const ufg_lattice* lat = f->lat;
  if (f->L64 == nullptr) {
    UFG_TRY(dev_alloc(&f->L64, (size_t)lat->S));
    UFG_TRY(dev_alloc(&f->Di64, (size_t)lat->S));
    UFG_TRY(dev_alloc(&f->L32, (size_t)lat->S));
    UFG_TRY(dev_alloc(&f->Di32, (size_t)lat->S));
  }
  cudaError_t e = launch_sca_setup(f->w64, lat->V, lat->ntau, alpha, f->L64, f->Di64, f->L32,
                                   f->Di32, st);
  note_launches(1);
  if (e != cudaSuccess) return cuda_fail(e, "SCA setup launch");
  f->sca_alpha = alpha;
  return UFG_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static ufg_status check_vec(const ufg_field* f, const void* x, const void* y, int prec) {
  if (f == nullptr || f->lat == nullptr) {
    set_error("null field");
    return UFG_INVALID_ARG;
  }
  if (x == nullptr || y == nullptr) {
    set_error("null vector pointer");
    return UFG_INVALID_ARG;
  }
  if (prec != UFG_FP64 && prec != UFG_FP32) {
    set_error("apply precision must be UFG_FP64 or UFG_FP32");
    return UFG_INVALID_ARG;
  }
  if (!aligned16(x) || !aligned16(y)) {
    set_error("vector pointers must be 16-byte aligned");
    return UFG_INVALID_ARG;
  }
  const size_t bytes = (size_t)f->lat->S * (prec ? 4 : 8);
  const char* a = static_cast<const char*>(x);
  const char* b = static_cast<const char*>(y);
  if (a < b + bytes && b < a + bytes) {
    set_error("x and y overlap");
    return UFG_INVALID_ARG;
  }
  return UFG_OK;
}

}  // namespace ufg

using namespace ufg;

extern "C" {

const char* ufg_last_error(void) { return g_err.c_str(); }
const char* ufg_version(void) { return "ufg-gb300 0.1 (sm_103a)"; }
const char* ufg_supported_nx(void) { return "4,6,8,10,12,16,32"; }
long long ufg_kernel_launches(void) { return launches_so_far(); }

ufg_status ufg_lattice_create(int nx, int ntau, double tau, double g, int dispersion,
                              ufg_lattice** out) {
  return ufg_lattice_create_dim(3, nx, ntau, tau, g, dispersion, out);
}

ufg_status ufg_lattice_create_dim(int dim, int nx, int ntau, double tau, double g,
                                  int dispersion, ufg_lattice** out) {
  clear_error();
  if (out == nullptr) {
    set_error("out is null");
    return UFG_INVALID_ARG;
  }
  *out = nullptr;
  if (dim < 1 || dim > 3) {
    set_error("invalid lattice: dim must be 1, 2 or 3 (got %d)", dim);
    return UFG_INVALID_ARG;
  }
  if (nx < 2 || nx % 2 != 0 || ntau < 3 || ntau > 1024 || !(tau > 0) || !(g >= 0) ||
      (dispersion != 0 && dispersion != 1) || !std::isfinite(tau) || !std::isfinite(g)) {
    set_error("invalid lattice: need even N_x >= 2, 3 <= N_tau <= 1024, tau > 0, g >= 0, "
              "dispersion 0 or 1 (got N_x=%d N_tau=%d tau=%g g=%g dispersion=%d)",
              nx, ntau, tau, g, dispersion);
    return UFG_INVALID_ARG;
  }
  if (!slice_supported_n(nx)) {
    set_error("N_x=%d is not built; supported: %s", nx, ufg_supported_nx());
    return UFG_UNSUPPORTED;
  }
  ufg_lattice* L = new ufg_lattice();
  L->nx = nx;
  L->ntau = ntau;
  L->tau = tau;
  L->g = g;
  L->dispersion = dispersion;
  L->A = std::sqrt(2.0) * std::sqrt(std::expm1(tau * g));
  L->dim = dim;
  L->V = (long long)nx * (dim >= 2 ? nx : 1) * (dim >= 3 ? nx : 1);
  L->S = L->V * ntau;
  if (dim < 3) L->use_tma[0] = L->use_tma[1] = 0;
  cudaGetDevice(&L->device);
  ufg_status s = build_tables(L);
  if (s != UFG_OK) {
    ufg_lattice_destroy(L);
    return s;
  }
  default_tuning(L);
  *out = L;
  return UFG_OK;
}

void ufg_lattice_destroy(ufg_lattice* L) {
  if (!L) return;
  dev_free(L->bk64);
  dev_free(L->bk32);
  dev_free(L->dev_err);
  delete L;
}

double ufg_lattice_coupling(const ufg_lattice* L) { return L ? L->A : 0.0; }

ufg_status ufg_lattice_check(const ufg_lattice* L, void* stream) {
  clear_error();
  if (L == nullptr) {
    set_error("null lattice");
    return UFG_INVALID_ARG;
  }
  return check_device_flag(L, as_stream(stream));
}

void ufg_test_expire_waits(int launches) { g_expire.store(launches > 0 ? launches : 0); }

ufg_status ufg_field_update(ufg_field* f, const double* sigma, void* stream) {
  clear_error();
  if (f == nullptr || sigma == nullptr || !aligned16(sigma)) {
    set_error("field_update: null field or null/misaligned sigma");
    return UFG_INVALID_ARG;
  }
  const ufg_lattice* L = f->lat;
  cudaStream_t st = as_stream(stream);
  UFG_CUDA(cudaMemcpyAsync(f->sigma, sigma, (size_t)L->S * sizeof(double), cudaMemcpyDefault, st));
  UFG_CUDA(launch_potentials(f->sigma, L->A, L->S, f->w64, f->s64, f->c64, f->w32, f->s32, f->c32,
                             st));
  note_launches(1);
  f->sca_alpha = -1.0;
  f->gcheb_alpha = -1.0;
  return UFG_OK;
}

ufg_status ufg_field_create(const ufg_lattice* L, const double* sigma, void* stream,
                            ufg_field** out) {
  clear_error();
  if (L == nullptr || out == nullptr) {
    set_error("null lattice or out");
    return UFG_INVALID_ARG;
  }
  *out = nullptr;
  static std::atomic<unsigned long long> next_id{1};
  ufg_field* f = new ufg_field();
  f->lat = L;
  f->id = next_id.fetch_add(1, std::memory_order_relaxed);
  const size_t S = (size_t)L->S;
  ufg_status s = UFG_OK;
  if ((s = dev_alloc(&f->sigma, S)) || (s = dev_alloc(&f->w64, S)) || (s = dev_alloc(&f->s64, S)) ||
      (s = dev_alloc(&f->c64, S)) || (s = dev_alloc(&f->w32, S)) || (s = dev_alloc(&f->s32, S)) ||
      (s = dev_alloc(&f->c32, S)) || (s = dev_alloc(&f->tmp64, S)) || (s = dev_alloc(&f->tmp32, S))) {
    ufg_field_destroy(f);
    return s;
  }
  s = ufg_field_update(f, sigma, stream);
  if (s != UFG_OK) {
    ufg_field_destroy(f);
    return s;
  }
  *out = f;
  return UFG_OK;
}

void ufg_field_destroy(ufg_field* f) {
  if (!f) return;
  dev_free(f->sigma);
  dev_free(f->w64);
  dev_free(f->s64);
  dev_free(f->c64);
  dev_free(f->w32);
  dev_free(f->s32);
  dev_free(f->c32);
  dev_free(f->tmp64);
  dev_free(f->tmp32);
  dev_free(f->L64);
  dev_free(f->Di64);
  dev_free(f->L32);
  dev_free(f->Di32);
  delete f;
}

ufg_status ufg_apply_M(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  return op_M(f, prec, x, y, as_stream(stream));
}

ufg_status ufg_apply_Mdag(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  return op_Mdag(f, prec, x, y, as_stream(stream));
}

ufg_status ufg_apply_Q(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  if (slice_q_supported(f->lat->nx, prec, f->lat->ntau, f->lat->dim)) {  // Q in one kernel
    SliceCall c = base_call(f->lat, FAM_KIN, prec);
    c.fam = FAM_Q;
    c.in = x;
    c.pre = fld(f, 'w', prec);
    c.out = y;
    return run(f->lat, c, as_stream(stream));
  }
  void* tmp = prec ? (void*)f->tmp32 : (void*)f->tmp64;
  UFG_TRY(op_M(f, prec, x, tmp, as_stream(stream)));
  return op_Mdag(f, prec, tmp, y, as_stream(stream));
}

ufg_status ufg_apply_M1(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  SliceCall c = base_call(f->lat, FAM_KIN, prec);
  c.in = x;
  c.pre = fld(f, 's', prec);
  c.shift = -1;
  c.out = y;
  return run(f->lat, c, as_stream(stream));
}

ufg_status ufg_apply_M1T(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  SliceCall c = base_call(f->lat, FAM_KIN, prec);
  c.in = x;
  c.post = fld(f, 's', prec);
  c.shift = +1;
  c.out = y;
  return run(f->lat, c, as_stream(stream));
}

ufg_status ufg_apply_kinetic(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  SliceCall c = base_call(f->lat, FAM_KIN, prec);
  c.in = x;
  c.out = y;
  return run(f->lat, c, as_stream(stream));
}

ufg_status ufg_apply_M0inv(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  void* tmp = prec ? (void*)f->tmp32 : (void*)f->tmp64;
  return op_M0inv(f, prec, x, y, tmp, 0, as_stream(stream));
}

ufg_status ufg_apply_M0invT(ufg_field* f, const void* x, void* y, int prec, void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  void* tmp = prec ? (void*)f->tmp32 : (void*)f->tmp64;
  return op_M0inv(f, prec, x, y, tmp, 1, as_stream(stream));
}

ufg_status ufg_fourier(ufg_field* f, const void* x, void* y, int prec, int inverse,
                       void* stream) {
  clear_error();
  PdlScope pdl;
  UFG_TRY(check_vec(f, x, y, prec));
  SliceCall c = base_call(f->lat, inverse ? FAM_INV : FAM_FWD, prec);
  c.in = x;
  c.out = y;
  return run(f->lat, c, as_stream(stream));
}

ufg_status ufg_apply_M_momentum(ufg_field* f, const void* x, void* y, int prec, int transpose,
                                void* stream) {
  clear_error();
  PdlScope pdl;
  const bool emulated = (prec == UFG_FP64_EMULATED);
  if (emulated) prec = UFG_FP64;
  UFG_TRY(check_vec(f, x, y, prec));
  const ufg_lattice* lat = f->lat;
  if (lat->dim != 3 || !slice_m1w_supported(lat->nx, prec)) {
    set_error("momentum-space apply built for FP32 N_x = 16 and FP64 N_x = 8, 16 (got N_x = %d)",
              lat->nx);
    return UFG_INVALID_ARG;
  }
  SliceCall c = base_call(lat, FAM_INV, prec);
  c.fam = FAM_M1W;
  c.coef2 = base_call(lat, FAM_FWD, prec).coef;
  c.m1w_full = 1;
  c.in = x;
  c.pre = fld(f, 'w', prec);
  const void* bk = prec ? (const void*)lat->bk32 : (const void*)lat->bk64;
  if (transpose) c.bkpre = bk;
  else c.bkpost = bk;
  c.shift = transpose ? +1 : -1;
  c.a = 1.0;
  c.out = y;
  c.emulate64 = emulated ? 1 : 0;
  return run(lat, c, as_stream(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Launch-shape autotuner: times the fused M apply (the slice kernel every operator shares) for
// each compiled (cluster size, slices per CTA) candidate on this lattice and keeps the fastest per
// precision.  Results are cached per (device name, N_x, N_tau, precision) in the process and, when
// UFG_TUNE_CACHE names a file, in that file (one "name nx ntau prec C spc" line per entry).
// ---------------------------------------------------------------------------------------------
namespace ufg {
namespace {

std::mutex g_tune_mu;
std::vector<std::string> g_tune_lines;  // "name nx ntau prec C spc"
bool g_tune_loaded = false;

std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

void load_tune_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("UFG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char buf[256];
  while (std::fgets(buf, sizeof(buf), f)) {
    std::string l(buf);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    if (!l.empty()) g_tune_lines.push_back(l);
  }
  std::fclose(f);
}

bool lookup(const std::string& key, int* C, int* spc) {
  for (const auto& l : g_tune_lines) {
    if (l.compare(0, key.size(), key) == 0 && l.size() > key.size() && l[key.size()] == ' ') {
      return std::sscanf(l.c_str() + key.size(), "%d %d", C, spc) == 2;
    }
  }
  return false;
}

void store(const std::string& key, int C, int spc) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s %d %d", key.c_str(), C, spc);
  g_tune_lines.push_back(buf);
  const char* path = std::getenv("UFG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s\n", buf);
  std::fclose(f);
}

}  // namespace
}  // namespace ufg

extern "C" ufg_status ufg_lattice_autotune(ufg_lattice* L, void* stream) {
  clear_error();
  if (!L) {
    set_error("null lattice");
    return UFG_INVALID_ARG;
  }
  if (L->dim != 3) {
    set_error("autotune: the launch shapes it chooses exist for 3-D lattices only");
    return UFG_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_tune_file();
  cudaStream_t st = as_stream(stream);
  const int N = L->nx;
  for (int prec = 0; prec < 2; ++prec) {
    char key[160];
    std::snprintf(key, sizeof(key), "%s %d %d %d", device_name().c_str(), N, L->ntau, prec);
    int C = 0, spc = 0;
    if (lookup(key, &C, &spc)) {
      L->use_tma[prec] = C == 0;
      if (C > 0) {
        L->C[prec] = C;
        L->spc[prec] = spc;
      }
      continue;
    }
    std::vector<std::pair<int, int>> cand;
    cand.emplace_back(0, 1);  // (0, 1): the TMA-staged kernel (where it applies)
    const size_t es = prec ? 4 : 8;
    const int cs[] = {1, 2, 4};
    for (int c : cs) {
      if (c > 1 && N < 16) continue;
      if (N % c) continue;
      for (int s = 1; s <= 8; s *= 2) {
        const size_t smem = (size_t)s * (N / c) * N * (N + 1) * es;
        if (smem > 200 * 1024) continue;
        if (s > 1 && (L->ntau + s - 1) / s * c < 152) continue;  // keep at least one wave
        cand.emplace_back(c, s);
      }
    }
    if (cand.empty()) continue;
    const size_t n = (size_t)L->S;
    void *x = nullptr, *y = nullptr, *w = nullptr;
    if (cudaMalloc(&x, n * es) != cudaSuccess || cudaMalloc(&y, n * es) != cudaSuccess ||
        cudaMalloc(&w, n * es) != cudaSuccess) {
      cudaFree(x);
      cudaFree(y);
      cudaFree(w);
      cudaGetLastError();
      set_error("autotune: temporary allocation failed");
      return UFG_OOM;
    }
    cudaMemsetAsync(x, 0, n * es, st);
    cudaMemsetAsync(w, 0, n * es, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> bestc = {L->C[prec], L->spc[prec]};
    for (auto& cd : cand) {
      SliceCall c = base_call(L, FAM_KIN, prec);
      c.allow_tma = cd.first == 0;
      c.C = cd.first == 0 ? L->C[prec] : cd.first;
      c.spc = cd.first == 0 ? L->spc[prec] : cd.second;
      c.in = x;
      c.pre = w;
      c.id = x;
      c.shift = -1;
      c.out = y;
      if (slice_dispatch(N, c, st) != cudaSuccess) {  // shape not available: skip it
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, st);
      const int reps = 5;
      for (int r = 0; r < reps; ++r) slice_dispatch(N, c, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bestc = cd;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    cudaFree(w);
    if (bestc.first == 0) {
      L->use_tma[prec] = 1;
    } else {
      L->use_tma[prec] = 0;
      L->C[prec] = bestc.first;
      L->spc[prec] = bestc.second;
    }
    store(key, bestc.first, bestc.second);
  }
  return UFG_OK;
}

extern "C" ufg_status ufg_lattice_launch_shape(const ufg_lattice* L, int precision, int* C,
                                               int* spc) {
  if (!L || !C || !spc || (precision != UFG_FP64 && precision != UFG_FP32)) {
    set_error("launch_shape: bad arguments");
    return UFG_INVALID_ARG;
  }
  *C = L->use_tma[precision] ? 0 : L->C[precision];
  *spc = L->spc[precision];
  return UFG_OK;
}
