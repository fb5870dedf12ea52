// Time-direction kernels: the per-site potentials of a field, the exact M0^{-1} recurrence per
// momentum mode (Sec. 3) and the strong-coupling factorisation and apply (Sec. 4).
#include <cuda_runtime.h>

#include "ufg_internal.h"
#include "launch.cuh"

namespace ufg {

// ---- potentials: w = 1 + A sin sigma, s = sin sigma, c = A cos sigma (B_t, C_t, dB/dsigma) ----
__global__ void potentials_kernel(const double* __restrict__ sigma, double A, long long S,
                                  double* w64, double* s64, double* c64, float* w32, float* s32,
                                  float* c32) {
  pdl_begin();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;
       i += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincos(sigma[i], &sn, &cs);
    const double w = 1.0 + A * sn;
    w64[i] = w;
    s64[i] = sn;
    c64[i] = A * cs;
    w32[i] = (float)w;
    s32[i] = (float)sn;
    c32[i] = (float)(A * cs);
  }
}

cudaError_t launch_potentials(const double* sigma, double A, long long S, double* w64, double* s64,
                              double* c64, float* w32, float* s32, float* c32, cudaStream_t st) {
  const int nt = 256;
  long long blocks = (S + nt - 1) / nt;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return launch_k(potentials_kernel, dim3((unsigned)blocks), dim3(nt), 0, st, 1, sigma, A, S, w64,
                  s64, c64, w32, s32, c32);
}

// ---- exact M0^{-1} per momentum mode ------------------------------------------------------
// In the spatial eigenbasis of exp(-tau K) (eigenvalue b per mode) M0 acts on one mode as
//   (M0 x)_t = x_t - b x_{t-1},  x_{-1} = -x_{N_tau-1}  (antiperiodic, Eq. MatrixM at sigma = 0),
// so M0^{-1} is the first-order recurrence x_t = y_t + b x_{t-1} closed by
//   x_{N_tau-1} = sum_t b^{N_tau-1-t} y_t / (1 + b^{N_tau}),
// which is the frequency-space diagonal [1 - exp(-i omega - tau E(k))]^{-1} of Sec. 3 written in
// imaginary time.  M0^{-T} runs the same recurrence backwards in t.
//
// Layout: block = 32 modes (lanes, coalesced 128/256-byte rows) x REC_NCH time chunks (warps).
// Pass 1 streams the thread's chunk and forms its zero-start end value e and the propagator
// p = b^len; one warp folds the REC_NCH chunk pairs into the closed boundary value and each chunk's
// incoming state; pass 2 streams the chunk again (a re-read served from L2: a block's 32 modes x
// N_tau elements were read microseconds earlier), continues the recurrence and writes.  Nothing
// is held in registers across the passes, so eight 256-thread blocks fit on an SM and a batch of
// 8 x 16^3 x 256 sites (1024 blocks) runs as a single wave; N_tau is unbounded.
constexpr int REC_NCH = 8;
// Loads each thread keeps in flight (unroll depth of the streaming loops): with 4 the kernel was
// latency-bound (long-scoreboard stalls, ~1/3 of HBM); 16 measured best of 4/8/16/32 (8 and 32
// again with the grouped pass 2: 18.2 and 18.0 against 17.8 us per term-only batched launch).
constexpr int REC_UNROLL = 16;
constexpr int REC_MINB = 7;  // 7 x 152 CTA slots still hold a batch of 1024 CTAs in one wave
// Pass 2 stores each value it loads, and its input may alias its output, so a plain loop waits
// one load round trip per element.  Loading G elements (and the accumulator or a combining
// recurrence's earlier terms) ahead of their stores cuts that to one per group.  Per launch on an
// 8 x 16^3 x 256 FP32 batch: term-only 18.6 -> 17.4 us at G = 8 (18.4 at 16), combining
// 32.2 -> 27.8 us at G = 4 (8: 27.9 us, more spills).  FP64 keeps the plain loop (no change
// on the FP64 96-problem batch).
constexpr int REC_G_ONE = 8;
constexpr int REC_G_TWO = 4;

template <typename R>
struct RecArgs {
  const R* in;
  R* out;
  const R* bk;
  long long V;
  int ntau, transpose;
  double out_scale;
  R* acc;
  double acc_coef;
  int acc_mode;             // 0: none, 1: acc = coef x, 2: acc += coef x
  const int* done;
  int exec_if;
  const int2* tiles;        // batched mode: (problem, 32-mode block) per CTA
  const BatchProb* probs;
  const R* e0;              // acc_mode 3: acc = acc_coef x + c0 e0 + c1 e1
  const R* e1;
  double c0, c1;
};

template <typename R, int ACC, bool OUT, int G = 1>  // ACC = acc_mode; OUT: write out
__global__ void __launch_bounds__(32 * REC_NCH, sizeof(R) == 4 ? REC_MINB : 5) recurrence_kernel(const RecArgs<R> a) {
  pdl_begin();
  __shared__ R Es[REC_NCH][32];
  __shared__ R Ps[REC_NCH][32];
  __shared__ R Is[REC_NCH][32];
  const int lane = threadIdx.x;
  const int ch = threadIdx.y;
  long long V = a.V, mode;
  int ntau = a.ntau;
  size_t off = 0;
  const int* done = a.done;
  if (a.tiles != nullptr) {
    const int2 tl = a.tiles[blockIdx.x];
    const BatchProb& pr = a.probs[tl.x];
    V = pr.V;
    ntau = pr.ntau;
    off = (size_t)pr.off;
    done = pr.done;
    mode = (long long)tl.y * 32 + lane;
  } else {
    mode = (long long)blockIdx.x * 32 + lane;
  }
  if (done != nullptr && a.exec_if >= 0 && *done != a.exec_if) return;
  const bool active = mode < V;
  const R b = active ? a.bk[mode] : R(0);
  const int len = (ntau + REC_NCH - 1) / REC_NCH;
  const int l0 = ch * len;
  const int n = active ? max(0, min(len, ntau - l0)) : 0;  // elements of this thread's chunk
  // element l of the chunk sits at time t = l0 + l (forward) or N_tau - 1 - (l0 + l) (transpose)
  const long long step = a.transpose ? -V : V;
  const long long first =
      n > 0 ? (a.transpose ? (long long)(ntau - 1 - l0) : (long long)l0) * V + mode : 0;
  const R* in = a.in + off + first;  // may alias out (in-place): each element is read, then written
  R e = R(0), p = R(1);
  {
    const R* q = in;
#pragma unroll(REC_UNROLL)
    for (int l = 0; l < n; ++l, q += step) {
      e = *q + b * e;
      p = p * b;
    }
  }
  Es[ch][lane] = e;
  Ps[ch][lane] = p;
  __syncthreads();
  if (ch == 0) {
    R Z = R(0), bN = R(1);
#pragma unroll
    for (int c = 0; c < REC_NCH; ++c) {
      Z = Es[c][lane] + Ps[c][lane] * Z;
      bN = bN * Ps[c][lane];
    }
    R state = -(Z / (R(1) + bN));  // x_{-1} = -x_{N_tau-1}
#pragma unroll
    for (int c = 0; c < REC_NCH; ++c) {
      Is[c][lane] = state;
      state = Es[c][lane] + Ps[c][lane] * state;
    }
  }
  __syncthreads();
  R x = Is[ch][lane];
  R* out = OUT ? a.out + off + first : nullptr;
  R* acc = ACC ? a.acc + off + first : nullptr;
  const R* e0 = ACC == 3 ? a.e0 + off + first : nullptr;
  const R* e1 = ACC == 3 ? a.e1 + off + first : nullptr;
  const R oscale = R(a.out_scale), acoef = R(a.acc_coef), c0 = R(a.c0), c1 = R(a.c1);
  const R* q = in;
  int l = 0;
  if constexpr (G > 1) {  // groups of G: all loads, then the dependent updates and stores
    for (; l + G <= n; l += G) {
      R v[G], f0[ACC == 3 ? G : 1], f1[ACC == 3 ? G : 1];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        v[j] = q[j * step];
        if constexpr (ACC == 3) {
          f0[j] = e0[j * step];
          f1[j] = e1[j * step];
        }
      }
#pragma unroll
      for (int j = 0; j < G; ++j) {
        x = v[j] + b * x;
        if constexpr (ACC == 1) acc[j * step] = acoef * x;
        if constexpr (ACC == 2) acc[j * step] += acoef * x;
        if constexpr (ACC == 3) acc[j * step] = acoef * x + c0 * f0[j] + c1 * f1[j];
        if constexpr (OUT) out[j * step] = oscale * x;
      }
      q += G * step;
      if constexpr (ACC == 3) {
        e0 += G * step;
        e1 += G * step;
      }
      if constexpr (ACC != 0) acc += G * step;
      if constexpr (OUT) out += G * step;
    }
  }
#pragma unroll(REC_UNROLL)
  for (; l < n; ++l, q += step) {
    x = *q + b * x;
    if constexpr (ACC == 1) *acc = acoef * x;
    if constexpr (ACC == 2) *acc += acoef * x;
    if constexpr (ACC == 3) {
      *acc = acoef * x + c0 * *e0 + c1 * *e1;
      e0 += step;
      e1 += step;
    }
    if constexpr (OUT) *out = oscale * x;
    if constexpr (ACC != 0) acc += step;
    if constexpr (OUT) out += step;
  }
}

template <typename R>
static cudaError_t rec_launch(const RecArgs<R>& a, unsigned grid, cudaStream_t st) {
  const dim3 blk(32, REC_NCH);
  const bool out = a.out != nullptr;
  if (a.acc_mode != 0 && a.acc == nullptr) return cudaErrorInvalidValue;
  // FP32: pass 2 in groups, of REC_G_ONE elements where it reads only the input, of REC_G_TWO
  // where it also reads the accumulator or the earlier terms
  if constexpr (sizeof(R) == 4) {
    auto go = [&](auto kern) { return launch_k(kern, dim3(grid), blk, 0, st, 1, a); };
    switch (a.acc_mode * 2 + (out ? 1 : 0)) {
      case 1: return go(recurrence_kernel<R, 0, true, REC_G_ONE>);
      case 2: return go(recurrence_kernel<R, 1, false, REC_G_ONE>);
      case 3: return go(recurrence_kernel<R, 1, true, REC_G_ONE>);
      case 4: return go(recurrence_kernel<R, 2, false, REC_G_TWO>);
      case 5: return go(recurrence_kernel<R, 2, true, REC_G_TWO>);
      case 6:
        if (a.e0 == nullptr || a.e1 == nullptr) return cudaErrorInvalidValue;
        return go(recurrence_kernel<R, 3, false, REC_G_TWO>);
    }
    return cudaErrorInvalidValue;
  }
  switch (a.acc_mode * 2 + (out ? 1 : 0)) {
    case 1: return launch_k(recurrence_kernel<R, 0, true>, dim3(grid), blk, 0, st, 1, a);
    case 2: return launch_k(recurrence_kernel<R, 1, false>, dim3(grid), blk, 0, st, 1, a);
    case 3: return launch_k(recurrence_kernel<R, 1, true>, dim3(grid), blk, 0, st, 1, a);
    case 4: return launch_k(recurrence_kernel<R, 2, false>, dim3(grid), blk, 0, st, 1, a);
    case 5: return launch_k(recurrence_kernel<R, 2, true>, dim3(grid), blk, 0, st, 1, a);
    case 6:
      if (a.e0 == nullptr || a.e1 == nullptr) return cudaErrorInvalidValue;
      return launch_k(recurrence_kernel<R, 3, false>, dim3(grid), blk, 0, st, 1, a);
  }
  return cudaErrorInvalidValue;  // nothing to write
}

cudaError_t launch_recurrence(int prec, const void* in, void* out, const void* bk, long long V,
                              int ntau, int transpose, double out_scale, void* acc,
                              double acc_coef, int acc_mode, const int* done, cudaStream_t st,
                              const void* e0, const void* e1, double c0, double c1) {
  if (V <= 0 || ntau <= 0) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((V + 31) / 32);
  if (prec == 0) {
    RecArgs<double> a{(const double*)in, (double*)out, (const double*)bk, V, ntau, transpose,
                      out_scale, (double*)acc, acc_coef, acc_mode, done, 0, nullptr, nullptr,
                      (const double*)e0, (const double*)e1, c0, c1};
    return rec_launch(a, grid, st);
  }
  RecArgs<float> a{(const float*)in, (float*)out, (const float*)bk, V, ntau, transpose, out_scale,
                   (float*)acc, acc_coef, acc_mode, done, 0, nullptr, nullptr,
                   (const float*)e0, (const float*)e1, c0, c1};
  return rec_launch(a, grid, st);
}

cudaError_t launch_recurrence_batch(int prec, const void* in, void* out, const void* bk,
                                    int max_ntau, int transpose, double out_scale, void* acc,
                                    double acc_coef, int acc_mode, int exec_if, const int2* tiles,
                                    int ntiles, const BatchProb* probs, cudaStream_t st,
                                    const void* e0, const void* e1, double c0, double c1) {
  (void)max_ntau;  // any N_tau: the chunk length follows each problem's own N_tau
  if (ntiles <= 0) return cudaSuccess;
  if (prec == 0) {
    RecArgs<double> a{(const double*)in, (double*)out, (const double*)bk, 0, 0, transpose,
                      out_scale, (double*)acc, acc_coef, acc_mode, nullptr, exec_if, tiles, probs,
                      (const double*)e0, (const double*)e1, c0, c1};
    return rec_launch(a, (unsigned)ntiles, st);
  }
  RecArgs<float> a{(const float*)in, (float*)out, (const float*)bk, 0, 0, transpose, out_scale,
                   (float*)acc, acc_coef, acc_mode, nullptr, exec_if, tiles, probs,
                   (const float*)e0, (const float*)e1, c0, c1};
  return rec_launch(a, (unsigned)ntiles, st);
}

// ---- strong-coupling approximation (Sec. 4) -----------------------------------------------
// Per site r, with w_t = 1 + A sin sigma_t (B_{0,t}) and 0-based t (paper's j = t + 1):
//   D_0 = alpha + w_0^2,  D_t = alpha + w_t^2 - w_{t-1}^2 / D_{t-1}  (1 <= t <= N-2),
//   D_{N-1} = alpha + w_{N-1}^2 - w_{N-2}^2 / D_{N-2} - w_{N-1}^2 / D_0,
//   L_t = w_t / D_t (t < N-1),  L_{N-1} = w_{N-1} / D_0.
// Stored: L and 1/D, FP64 and FP32.
__global__ void sca_setup_kernel(const double* __restrict__ w, long long V, int ntau, double alpha,
                                 double* L64, double* Di64, float* L32, float* Di32) {
  pdl_begin();
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= V) return;
  const double w0 = w[r];
  const double D0 = alpha + w0 * w0;
  double Dprev = D0, wprev = w0;
  auto put = [&](int t, double L, double D) {
    const size_t g = (size_t)t * V + r;
    L64[g] = L;
    Di64[g] = 1.0 / D;
    L32[g] = (float)L;
    Di32[g] = (float)(1.0 / D);
  };
  put(0, w0 / D0, D0);
  for (int t = 1; t < ntau - 1; ++t) {
    const double wt = w[(size_t)t * V + r];
    const double Dt = alpha + wt * wt - wprev * wprev / Dprev;
    put(t, wt / Dt, Dt);
    Dprev = Dt;
    wprev = wt;
  }
  const double wl = w[(size_t)(ntau - 1) * V + r];
  const double Dl = alpha + wl * wl - wprev * wprev / Dprev - wl * wl / D0;
  put(ntau - 1, wl / D0, Dl);
}

cudaError_t launch_sca_setup(const double* w64, long long V, int ntau, double alpha, double* L64,
                             double* Di64, float* L32, float* Di32, cudaStream_t st) {
  sca_setup_kernel<<<(unsigned)((V + 127) / 128), 128, 0, st>>>(w64, V, ntau, alpha, L64, Di64, L32,
                                                                 Di32);
  return cudaGetLastError();
}

// Epilogue of the SCA sweep: every finished z_t is stored as a z_t + bU U_t + cV W_t (U, W
// nullable; neither may alias z, which holds the intermediate u = x / D until the backward sweep).
template <typename R>
struct ScaEpi {
  R a, bU, cV;
  const R* U;
  const R* W;
  __device__ __forceinline__ R operator()(R zt, size_t g) const {
    R o = a * zt;
    if (U != nullptr) o += bU * U[g];
    if (W != nullptr) o += cV * W[g];
    return o;
  }
};

// z = (L^T D L)^{-1} y: forward solve with the lower factor (the recursion printed in Sec. 4),
// pointwise 1/D, backward solve with the upper factor.  One thread per site, coalesced in r.
template <typename R>
__global__ void sca_apply_kernel(const R* __restrict__ L, const R* __restrict__ Di, const R* y,
                                 R* z, long long V, int ntau, const int* done, ScaEpi<R> ep) {
  pdl_begin();
  if (done != nullptr && *done) return;
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= V) return;
  const int N = ntau;
  const R x0 = y[r];
  R xp = x0;
  // forward: x_t = y_t + L_{t-1} x_{t-1}; x_{N-1} -= L_{N-1} x_0; store u = x / D into z
  z[r] = x0 * Di[r];
  for (int t = 1; t < N; ++t) {
    const size_t g = (size_t)t * V + r;
    R xt = y[g] + L[g - V] * xp;
    if (t == N - 1) xt -= L[g] * x0;
    z[g] = xt * Di[g];
    xp = xt;
  }
  // backward: z_{N-1} = u_{N-1}; z_t = u_t + L_t z_{t+1} (t = N-2..1);
  // z_0 = u_0 + L_0 z_1 - L_{N-1} z_{N-1}
  const size_t gl = (size_t)(N - 1) * V + r;
  const R zl = z[gl];
  z[gl] = ep(zl, gl);
  R zn = zl;
  for (int t = N - 2; t >= 1; --t) {
    const size_t g = (size_t)t * V + r;
    const R zt = z[g] + L[g] * zn;
    z[g] = ep(zt, g);
    zn = zt;
  }
  z[r] = ep(z[r] + L[r] * zn - L[gl] * zl, (size_t)r);
}

cudaError_t launch_sca_apply(int prec, const void* L, const void* Di, const void* y, void* z,
                             long long V, int ntau, const int* done, cudaStream_t st, double a,
                             const void* U, double bU, const void* W, double cV) {
  const unsigned grid = (unsigned)((V + 127) / 128);
  if (prec == 0) {
    const ScaEpi<double> ep{a, bU, cV, (const double*)U, (const double*)W};
    sca_apply_kernel<double><<<grid, 128, 0, st>>>((const double*)L, (const double*)Di,
                                                   (const double*)y, (double*)z, V, ntau, done,
                                                   ep);
  } else {
    const ScaEpi<float> ep{(float)a, (float)bU, (float)cV, (const float*)U, (const float*)W};
    sca_apply_kernel<float><<<grid, 128, 0, st>>>((const float*)L, (const float*)Di,
                                                  (const float*)y, (float*)z, V, ntau, done, ep);
  }
  return cudaGetLastError();
}

}  // namespace ufg
