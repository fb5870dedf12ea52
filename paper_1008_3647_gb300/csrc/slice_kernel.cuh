// The fused per-time-slice kernel behind every apply of the fermion matrix family.
//
// One CTA (or one thread-block cluster of C CTAs for the largest slices) owns `spc` consecutive
// output time slices.  For each it
//   1. streams the input slice t_in (t_out-1 for M-type, t_out+1 for M^T-type, t_out otherwise)
//      from HBM into shared memory, multiplied on the fly by a per-site field (w = 1 + A sin sigma,
//      s = sin sigma) and/or a per-mode table,
//   2. applies the separable line operator along x and along y in shared memory (in place,
//      padded rows of N+1 elements keep the three access patterns free of bank conflicts),
//   3. applies it along z column by column (a cluster reads the other CTAs' planes through
//      distributed shared memory) and finishes every output site in registers: antiperiodic
//      time-shift sign, post-multiplication, identity term, linear-combination epilogue and
//      FP64 dot-product partials, one coalesced HBM write.
//
// Operator families (line operator along all three axes):
//   KIN: T = exp(-tau K) restricted to one axis (REAL -> REAL)      -> M, M^T, M1, M1^T, force
//   FWD: F^T, the real orthonormal Fourier basis (REAL -> SPEC)     -> momentum space
//   INV: F (SPEC -> REAL)                                           -> back to real space
//
// Epilogue for an output site g of slice t_out (sgn = +1 for the antiperiodic wrap, -1 for the
// other shifted slices, +1 without shift):
//   base = sgn * op(...)[g] * bkpost[mode] * post[g] * post2[g] + id[g]      (absent factors = 1/0)
//   out[g] = a * base + bU * U[g] + cV * V[g];  partials += (out*dotP, out*out) in FP64.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "line_ops.cuh"
#include "scalar_ops.cuh"
#include "slice_call.h"
#include "launch.cuh"

namespace ufg {

namespace cg = cooperative_groups;

template <int N, typename R>
struct SliceArgs {
  // one copy of the line operator per pass, so that the compiler does not keep all of its
  // coefficients live in registers from the first pass to the last
  LineCoef<N, R> coef_x;
  LineCoef<N, R> coef_y;
  LineCoef<N, R> coef_z;
  const R* in;
  const R* pre;
  const R* bkpre;
  const R* bkpost;
  R* out;
  const R* id;
  const R* post;
  const R* post2;
  const R* U;
  const R* V;
  const R* dotP;
  double a, bU, cV;
  double* partials;
  int want_dotP, want_self;
  const int* done;
  int exec_if;
  const BatchTile* tiles;
  const BatchProb* probs;
  int scale_by_A;
  int ntau, shift, spc;
  int fop;       // batched: scalar op of the problem's last CTA (-1: none), see SliceCall
  DevScalars* scs;
  unsigned* counters;
  int part_base;
};

template <typename R> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int W = 2; };

template <typename R>
__device__ __forceinline__ void ld16(const R* p, R (&o)[Vec16<R>::W]) {
  typename Vec16<R>::T v = __ldg(reinterpret_cast<const typename Vec16<R>::T*>(p));
  if constexpr (Vec16<R>::W == 4) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  else { o[0] = v.x; o[1] = v.y; }
}

template <typename R>
__device__ __forceinline__ void st16(R* p, const R (&v)[Vec16<R>::W]) {
  typename Vec16<R>::T w;
  if constexpr (Vec16<R>::W == 4) { w.x = v[0]; w.y = v[1]; w.z = v[2]; w.w = v[3]; }
  else { w.x = v[0]; w.y = v[1]; }
  *reinterpret_cast<typename Vec16<R>::T*>(p) = w;
}

constexpr int SLICE_NT = 256;
static_assert(SLICE_NT == SCAL_NT, "fused scalar updates reduce over SCAL_NT threads");

// Epilogue operand mask: the specialised variants know at compile time which operands exist;
// EPI_ANY tests every optional pointer at run time.
enum EpiBits { E_ID = 1, E_POST = 2, E_POST2 = 4, E_UV = 8, E_DOT = 16, E_BK = 32, EPI_ANY = 63 };
// Load-side fusion of the TMA kernel (forward transform of batched BiCGStab): the input is p and
// the kernel first forms p' = r + beta (p - omega v) (per-problem scalars), writes p' back and
// transforms it.
constexpr int E_PREP = 64;
// TMA 8-CTA clusters on whole slices only (set by the launcher for the KIN family): the load
// multiplier arrives as a box in the receive buffer (E_PRE), the identity operand as a box in
// the x buffer once the y-pass has read it (E_IDB)
constexpr int E_PRE = 128;
constexpr int E_IDB = 256;

// Resident CTAs per SM the register allocation must allow (256 threads each).
template <int N, typename R>
constexpr int slice_min_blocks() {
  return N >= 32 ? (sizeof(R) == 4 ? 3 : 1) : (N >= 16 ? (sizeof(R) == 4 ? 3 : 2) : 3);
}

template <int N, typename R, int C, int FAM, int EPI>
__global__ void __launch_bounds__(SLICE_NT, (slice_min_blocks<N, R>()))
slice_kernel(const __grid_constant__ SliceArgs<N, R> A) {
  pdl_begin();
  constexpr int NP = N / C;          // z-planes of one slice held by this CTA
  constexpr int PITCH = N + 1;       // padded row
  constexpr int PLANE = N * PITCH;   // shared-memory elements per plane
  constexpr int NN = N * N;
  constexpr int VOL = N * N * N;
  constexpr int CHUNK = NP * NN;     // HBM elements per slice per CTA
  constexpr int VW = Vec16<R>::W;
  constexpr bool IN_SPEC = (FAM == FAM_INV);
  constexpr bool OUT_SPEC = (FAM == FAM_FWD);
  static_assert(CHUNK % VW == 0, "chunk must be a whole number of 16-byte vectors");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  __shared__ double red[SLICE_NT / 32][2];

  // single problem: unit -> slices [unit*spc, ...); batched: unit -> tile (problem, t0)
  const int unit = blockIdx.x / C;
  int t0, ntau;
  size_t off = 0;
  const int* done = A.done;
  double acoef = A.a;
  if (A.tiles != nullptr) {
    const BatchTile tl = A.tiles[unit];
    const BatchProb& pr = A.probs[tl.prob];
    t0 = tl.t0;
    ntau = pr.ntau;
    off = (size_t)pr.off;
    done = pr.done;
    if (A.scale_by_A) acoef *= pr.A;
  } else {
    t0 = unit * A.spc;
    ntau = A.ntau;
  }
  if (done != nullptr && A.exec_if >= 0 && *done != A.exec_if) return;  // uniform per problem

  int rank = 0;
  if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
  const int nsl = min(A.spc, ntau - t0);
  const int tid = threadIdx.x;
  const R* gin = A.in + off;
  const R* gpre = A.pre ? A.pre + off : nullptr;
  R* gout = A.out + off;
  const R* gid = A.id ? A.id + off : nullptr;
  const R* gpost = A.post ? A.post + off : nullptr;
  const R* gpost2 = A.post2 ? A.post2 + off : nullptr;
  const R* gU = A.U ? A.U + off : nullptr;
  const R* gV = A.V ? A.V + off : nullptr;
  const R* gdot = A.dotP ? A.dotP + off : nullptr;

  // ---- 1. load (with per-site / per-mode multipliers) ----
  for (int s = 0; s < nsl; ++s) {
    const int t_out = t0 + s;
    int t_in = t_out;
    if (A.shift < 0) t_in = (t_out == 0) ? ntau - 1 : t_out - 1;
    if (A.shift > 0) t_in = (t_out == ntau - 1) ? 0 : t_out + 1;
    const size_t gbase = (size_t)t_in * VOL + (size_t)rank * CHUNK;
    R* dst = sm + s * NP * PLANE;
#pragma unroll 4
    for (int e = tid * VW; e < CHUNK; e += SLICE_NT * VW) {
      R v[VW];
      ld16(gin + gbase + e, v);
      if (gpre != nullptr) {
        R w[VW];
        ld16(gpre + gbase + e, w);
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] *= w[k];
      }
      if (A.bkpre != nullptr) {
        R w[VW];
        ld16(A.bkpre + (size_t)rank * CHUNK + e, w);
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] *= w[k];
      }
      if constexpr (N % VW == 0) {  // a vector never crosses a row: one address per vector
        const int row = e / N;      // row index over all planes of this slice
        R* d = dst + row * PITCH + (e - row * N);
#pragma unroll
        for (int k = 0; k < VW; ++k) d[k] = v[k];
      } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          const int idx = e + k;
          const int row = idx / N;
          dst[row * PITCH + (idx - row * N)] = v[k];
        }
      }
    }
  }
  __syncthreads();

  // ---- 2. x-pass and y-pass, in place ----
  const int nlines = nsl * NP * N;
  for (int l = tid; l < nlines; l += SLICE_NT) {
    const int pl = l / N, r = l - (l / N) * N;
    R* base = sm + pl * PLANE + r * PITCH;
    R v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = base[j];
    line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_x, [&](int i, R val) { base[i] = val; });
  }
  __syncthreads();
  for (int l = tid; l < nlines; l += SLICE_NT) {
    const int pl = l / N, x = l - (l / N) * N;
    R* base = sm + pl * PLANE + x;
    R v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = base[j * PITCH];
    line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_y, [&](int i, R val) { base[i * PITCH] = val; });
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }

  // ---- 3. z-pass + epilogue ----
  const R* owner[C];
#pragma unroll
  for (int o = 0; o < C; ++o) {
    if constexpr (C > 1) {
      owner[o] = (o == rank) ? sm : cg::this_cluster().map_shared_rank(sm, o);
    } else {
      owner[o] = sm;
    }
  }
  constexpr int COLS = NN / C;
  // per-thread partial sums in the working precision (FP64 arithmetic is slow on this part and
  // a thread sums at most N terms); converted to FP64 for the block reduction
  R acc_dot = R(0), acc_self = R(0);
  const int ncols = nsl * COLS;
  for (int l = tid; l < ncols; l += SLICE_NT) {
    const int s = l / COLS;
    const int q = rank * COLS + (l - s * COLS);
    const int y = q / N, x = q - (q / N) * N;
    const int t_out = t0 + s;
    R sgn = R(1);
    if (A.shift < 0 && t_out != 0) sgn = R(-1);
    if (A.shift > 0 && t_out != ntau - 1) sgn = R(-1);
    R v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) {
      v[z] = owner[z / NP][(s * NP + (z % NP)) * PLANE + y * PITCH + x];
    }
    const size_t obase = (size_t)t_out * VOL + q;
    line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_z, [&](int zp, R val) {
      const size_t g = obase + (size_t)zp * NN;
      R b = sgn * val;
      if constexpr (EPI == EPI_ANY) {
        if (A.bkpost != nullptr) b *= A.bkpost[zp * NN + q];
        if (gpost != nullptr) b *= gpost[g];
        if (gpost2 != nullptr) b *= gpost2[g];
        if (gid != nullptr) b += gid[g];
        R o = R(acoef) * b;
        if (gU != nullptr) o += R(A.bU) * gU[g];
        if (gV != nullptr) o += R(A.cV) * gV[g];
        gout[g] = o;
        if (A.want_dotP) acc_dot += o * gdot[g];
        if (A.want_self) acc_self += o * o;
      } else if constexpr (EPI & E_UV) {  // U or V may alias out (in-place updates)
        if constexpr (EPI & E_BK) b *= A.bkpost[zp * NN + q];
        if constexpr (EPI & E_POST) b *= gpost[g];
        if constexpr (EPI & E_POST2) b *= gpost2[g];
        if constexpr (EPI & E_ID) b += gid[g];
        R o = R(acoef) * b;
        if (gU != nullptr) o += R(A.bU) * gU[g];
        if (gV != nullptr) o += R(A.cV) * gV[g];
        gout[g] = o;
        if constexpr (EPI & E_DOT) {
          if (A.want_dotP) acc_dot += o * gdot[g];
          if (A.want_self) acc_self += o * o;
        }
      } else {  // operands never alias the output: loads may move ahead of earlier stores
        const R* __restrict__ rid = gid;
        const R* __restrict__ rpost = gpost;
        const R* __restrict__ rpost2 = gpost2;
        const R* __restrict__ rdot = gdot;
        R* __restrict__ rout = gout;
        if constexpr (EPI & E_BK) b *= __ldg(A.bkpost + zp * NN + q);
        if constexpr (EPI & E_POST) b *= __ldg(rpost + g);
        if constexpr (EPI & E_POST2) b *= __ldg(rpost2 + g);
        if constexpr (EPI & E_ID) b += __ldg(rid + g);
        const R o = R(acoef) * b;
        rout[g] = o;
        if constexpr (EPI & E_DOT) {
          if (A.want_dotP) acc_dot += o * __ldg(rdot + g);
          if (A.want_self) acc_self += o * o;
        }
      }
    });
  }

  if (A.want_dotP || A.want_self) {
    double pd = (double)acc_dot, ps = (double)acc_self;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      pd += __shfl_xor_sync(0xffffffffu, pd, off);
      ps += __shfl_xor_sync(0xffffffffu, ps, off);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = pd;
      red[tid >> 5][1] = ps;
    }
    __syncthreads();
    if (tid == 0) {
      double d = 0.0, q2 = 0.0;
      for (int w = 0; w < SLICE_NT / 32; ++w) {
        d += red[w][0];
        q2 += red[w][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
    if (A.fop >= 0 && A.tiles != nullptr) {
      const int prob = A.tiles[unit].prob;
      last_block_update(A.fop, A.scs + prob, A.partials, A.probs[prob].st0 - A.part_base,
                        A.probs[prob].st1 - A.part_base, A.counters + prob);
    }
  }
  if constexpr (C > 1) cg::this_cluster().sync();  // peers may still read this CTA's planes
}

template <int N, typename R>
inline void fill_args(SliceArgs<N, R>& a, const SliceCall& c) {
  a.coef_x = *reinterpret_cast<const LineCoef<N, R>*>(c.coef);
  a.coef_y = a.coef_x;
  a.coef_z = a.coef_x;
  a.in = static_cast<const R*>(c.in);
  a.pre = static_cast<const R*>(c.pre);
  a.bkpre = static_cast<const R*>(c.bkpre);
  a.bkpost = static_cast<const R*>(c.bkpost);
  a.out = static_cast<R*>(c.out);
  a.id = static_cast<const R*>(c.id);
  a.post = static_cast<const R*>(c.post);
  a.post2 = static_cast<const R*>(c.post2);
  a.U = static_cast<const R*>(c.U);
  a.V = static_cast<const R*>(c.V);
  a.dotP = static_cast<const R*>(c.dotP);
  a.a = c.a;
  a.bU = c.bU;
  a.cV = c.cV;
  a.partials = c.partials;
  a.want_dotP = c.want_dotP;
  a.want_self = c.want_self;
  a.done = c.done;
  a.exec_if = c.exec_if;
  a.tiles = c.tiles;
  a.probs = c.probs;
  a.scale_by_A = c.scale_by_A;
  a.fop = c.fop;
  a.scs = c.scs;
  a.counters = c.counters;
  a.part_base = c.part_base;
  a.ntau = c.ntau;
  a.shift = c.shift;
  a.spc = c.spc;
}

template <int N, typename R, int C, int FAM, int EPI>
inline cudaError_t launch_epi(const SliceCall& c, cudaStream_t st) {
  SliceArgs<N, R> a;
  fill_args<N, R>(a, c);
  constexpr int PLANE = N * (N + 1);
  const size_t smem = (size_t)c.spc * (N / C) * PLANE * sizeof(R);
  auto kern = slice_kernel<N, R, C, FAM, EPI>;
  // attributes are set once per instantiation (outside any stream capture that follows)
  static int configured_smem = 0;
  if ((int)smem > configured_smem) {
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured_smem = (int)smem;
  }
  const int units = c.tiles != nullptr ? c.ntiles : (c.ntau + c.spc - 1) / c.spc;
  if (c.grid_out) *c.grid_out = units * C;
  return launch_k(kern, dim3(units * C), dim3(SLICE_NT), smem, st, C, a);
}

template <int N, typename R, int C, int FAM>
inline cudaError_t launch_one(const SliceCall& c, cudaStream_t st) {
  const int mask = (c.id ? E_ID : 0) | (c.post ? E_POST : 0) | (c.post2 ? E_POST2 : 0) |
                   ((c.U || c.V) ? E_UV : 0) | ((c.want_dotP || c.want_self) ? E_DOT : 0) |
                   (c.bkpost ? E_BK : 0);
  if constexpr (FAM == FAM_KIN) {
    switch (mask) {
      case E_ID: return launch_epi<N, R, C, FAM, E_ID>(c, st);                       // M
      case E_ID | E_POST: return launch_epi<N, R, C, FAM, E_ID | E_POST>(c, st);     // M^T
      case E_ID | E_DOT: return launch_epi<N, R, C, FAM, E_ID | E_DOT>(c, st);
      case E_ID | E_POST | E_DOT: return launch_epi<N, R, C, FAM, E_ID | E_POST | E_DOT>(c, st);
    }
  } else if constexpr (FAM == FAM_FWD) {
    switch (mask) {
      case 0: return launch_epi<N, R, C, FAM, 0>(c, st);
      case E_BK: return launch_epi<N, R, C, FAM, E_BK>(c, st);
    }
  } else {
    switch (mask) {
      case 0: return launch_epi<N, R, C, FAM, 0>(c, st);
      case E_POST: return launch_epi<N, R, C, FAM, E_POST>(c, st);
    }
  }
  return launch_epi<N, R, C, FAM, EPI_ANY>(c, st);
}

template <int N, typename R, int FAM>
inline cudaError_t launch_C(const SliceCall& c, cudaStream_t st) {
  if constexpr (N >= 16) {
    if (c.C == 4) return launch_one<N, R, 4, FAM>(c, st);
    if (c.C == 2) return launch_one<N, R, 2, FAM>(c, st);
  }
  if (c.C == 1) {
    // an FP64 32^3 slice (270 KB padded) exceeds one CTA's shared memory
    if constexpr (N < 32 || sizeof(R) == 4) return launch_one<N, R, 1, FAM>(c, st);
  }
  return cudaErrorInvalidValue;
}

template <int N>
cudaError_t slice_launch_plain(const SliceCall& c, cudaStream_t st) {
  if (c.prec == 0) {
    switch (c.fam) {
      case FAM_KIN: return launch_C<N, double, FAM_KIN>(c, st);
      case FAM_FWD: return launch_C<N, double, FAM_FWD>(c, st);
      case FAM_INV: return launch_C<N, double, FAM_INV>(c, st);
    }
  } else {
    switch (c.fam) {
      case FAM_KIN: return launch_C<N, float, FAM_KIN>(c, st);
      case FAM_FWD: return launch_C<N, float, FAM_FWD>(c, st);
      case FAM_INV: return launch_C<N, float, FAM_INV>(c, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ufg
