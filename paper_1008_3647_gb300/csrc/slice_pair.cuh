// Paired-line form of the TMA-staged slice kernel for FP32 16^3 slices.
//
// The kinetic factor exp(-tau K) = T (x) T (x) T (Sec. 1) is applied by three line passes over a
// slice held in shared memory.  Here every thread carries two lines of each pass at once, as the
// x and y halves of float2 values: each multiply-add and fold of the two-level even/odd line
// operator (line_ops.cuh) is then one packed FP32x2 instruction (sm_100 and later), and in the
// y- and z-passes and the epilogue the two lines are neighbouring x columns, so every
// shared-memory and global access moves 8 bytes instead of 4.  The staging is that of
// slice_tma_kernel: one 64-byte-swizzled TMA box per operand completing on an mbarrier with a
// bounded wait, one CTA of 128 threads per slice, six CTAs per SM.
//
//   x-pass: thread i owns rows i and i + 128 of the box, read and written as 16-byte chunks;
//   y-pass: thread i owns the column pair (x, x+1) of one plane;
//   z-pass: thread i owns the column pair (x, x+1) of one (y) row, finishing each output pair in
//           registers (time-shift sign, per-mode / per-site multipliers, identity term, scale,
//           dot partials).
#pragma once
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "slice_tma.cuh"

namespace ufg {

// Threads per CTA: one row pair of the slice box each.
template <int N>
constexpr int pair_nt() {
  return N * N / 2;
}

template <int N>
struct TmaPairArgs {
  CUtensorMap tm_in;   // [rows][N] view of the input, box N x ROWS
  CUtensorMap tm_pre;  // same view of the per-site load multiplier (or the per-mode table)
  // one copy of the line operator per pass (see TmaArgs), each entry twice (float2)
  LineCoef<N, float2> coef_x;
  LineCoef<N, float2> coef_y;
  LineCoef<N, float2> coef_z;
  const float* bkpost;
  float* out;
  const float* id;
  const float* post;
  const float* dotP;
  double a;
  double* partials;
  int want_dotP, want_self;
  const int* done;
  int exec_if;
  const BatchTile* tiles;
  const BatchProb* probs;
  int scale_by_A;
  int ntau, shift, units, has_pre, pre_mode;
  int* err;      // raised by a bounded wait that ran out
  int expire;    // test hook (ufg_test_expire_waits)
};

__device__ __forceinline__ float2 ldg2(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}

template <int N, int FAM, int EPI>
__global__ void __launch_bounds__((pair_nt<N>()), 6)
slice_tma_pair_kernel(const __grid_constant__ TmaPairArgs<N> A) {
  pdl_begin();
  using G = SwzGeom<N, float>;
  constexpr int PAIR_NT = pair_nt<N>();
  constexpr int NN = N * N;
  constexpr int VOL = N * NN;
  constexpr int BUF = VOL;         // elements of one box (the whole slice)
  constexpr int HR = NN / 2;
  constexpr int CPR = G::RB / 16;  // 16-byte chunks per row
  constexpr bool IN_SPEC = (FAM == FAM_INV);
  constexpr bool OUT_SPEC = (FAM == FAM_FWD);
  extern __shared__ __align__(1024) unsigned char tma_smem[];
  __shared__ double red[PAIR_NT / 32][2];
  __shared__ alignas(8) uint64_t bar, bar2;

  const int tid = threadIdx.x;
  const int unit = blockIdx.x;
  int t_out, ntau;
  size_t off = 0;
  const int* done = A.done;
  double acoef = A.a;
  if (A.tiles != nullptr) {
    const BatchTile tl = A.tiles[unit];
    const BatchProb& pr = A.probs[tl.prob];
    t_out = tl.t0;
    ntau = pr.ntau;
    off = (size_t)pr.off;
    done = pr.done;
    if (A.scale_by_A) acoef *= pr.A;
  } else {
    t_out = unit;
    ntau = A.ntau;
  }
  if (done != nullptr && A.exec_if >= 0 && *done != A.exec_if) return;
  int t_in = t_out;
  if (A.shift < 0) t_in = t_out == 0 ? ntau - 1 : t_out - 1;
  if (A.shift > 0) t_in = t_out == ntau - 1 ? 0 : t_out + 1;
  unsigned char* const base = tma_smem + ((1024u - (smem_addr(tma_smem) & 1023u)) & 1023u);
  float* const xs = reinterpret_cast<float*>(base);
  const float* const ws = xs + BUF;

  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const int row = (int)((off + (size_t)t_in * VOL) / N);
    mbar_expect_tx(&bar, (uint32_t)(BUF * sizeof(float)) * (A.has_pre ? 2u : 1u));
    tma_load_rows(xs, &A.tm_in, row, &bar);
    if (A.has_pre) tma_load_rows(const_cast<float*>(ws), &A.tm_pre, A.pre_mode ? 0 : row, &bar);
  }
  __syncthreads();  // the mbarrier is initialised before anyone waits on it
  mbar_wait_bounded(&bar, 0u, TMA_WAIT_LIMIT, A.err);
  if (A.expire && tid == 0) mbar_expire_one_wait(&bar2, EXPIRE_LIMIT, A.err);

  // ---- x-pass: rows tid and tid + HR, 16-byte chunks ----
  {
    const int r0 = tid, r1 = tid + HR;
    float2 v[N];
#pragma unroll
    for (int c = 0; c < CPR; ++c) {
      const float4 a = *reinterpret_cast<const float4*>(xs + G::chunk(r0, c));
      const float4 b = *reinterpret_cast<const float4*>(xs + G::chunk(r1, c));
      v[4 * c + 0] = make_float2(a.x, b.x);
      v[4 * c + 1] = make_float2(a.y, b.y);
      v[4 * c + 2] = make_float2(a.z, b.z);
      v[4 * c + 3] = make_float2(a.w, b.w);
      if (A.has_pre) {
        const float4 wa = *reinterpret_cast<const float4*>(ws + G::chunk(r0, c));
        const float4 wb = *reinterpret_cast<const float4*>(ws + G::chunk(r1, c));
        v[4 * c + 0] = v[4 * c + 0] * make_float2(wa.x, wb.x);
        v[4 * c + 1] = v[4 * c + 1] * make_float2(wa.y, wb.y);
        v[4 * c + 2] = v[4 * c + 2] * make_float2(wa.z, wb.z);
        v[4 * c + 3] = v[4 * c + 3] * make_float2(wa.w, wb.w);
      }
    }
    float2 o[N];
    line_op<N, float2, IN_SPEC, OUT_SPEC>(v, A.coef_x, [&](int i, float2 val) { o[i] = val; });
#pragma unroll
    for (int c = 0; c < CPR; ++c) {
      *reinterpret_cast<float4*>(xs + G::chunk(r0, c)) =
          make_float4(o[4 * c].x, o[4 * c + 1].x, o[4 * c + 2].x, o[4 * c + 3].x);
      *reinterpret_cast<float4*>(xs + G::chunk(r1, c)) =
          make_float4(o[4 * c].y, o[4 * c + 1].y, o[4 * c + 2].y, o[4 * c + 3].y);
    }
  }
  __syncthreads();
  // ---- y-pass: the column pair (x, x+1) of plane p, in place ----
  {
    const int p = tid / (N / 2), x = 2 * (tid % (N / 2));
    float2 v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = *reinterpret_cast<const float2*>(xs + G::off(p * N + y, x));
    line_op<N, float2, IN_SPEC, OUT_SPEC>(v, A.coef_y, [&](int i, float2 val) {
      *reinterpret_cast<float2*>(xs + G::off(p * N + i, x)) = val;
    });
  }
  __syncthreads();
  // ---- z-pass + epilogue: the column pair (x, x+1) of row y ----
  float2 sgn = make_float2(1.f, 1.f);
  if ((A.shift < 0 && t_out != 0) || (A.shift > 0 && t_out != ntau - 1)) sgn = make_float2(-1.f, -1.f);
  const float2 a2 = make_float2((float)acoef, (float)acoef);
  const float2 sa = sgn * a2;
  const float* __restrict__ gid = A.id ? A.id + off : nullptr;
  const float* __restrict__ gpost = A.post ? A.post + off : nullptr;
  const float* __restrict__ gdot = A.dotP ? A.dotP + off : nullptr;
  float* __restrict__ gout = A.out + off;
  float2 acc_dot = make_float2(0.f, 0.f), acc_self = make_float2(0.f, 0.f);
  {
    const int q = 2 * tid;
    const int y = q / N, x = q - (q / N) * N;
    float2 v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = *reinterpret_cast<const float2*>(xs + G::off(z * N + y, x));
    const size_t obase = (size_t)t_out * VOL + q;
    line_op<N, float2, IN_SPEC, OUT_SPEC>(v, A.coef_z, [&](int zp, float2 val) {
      const size_t g = obase + (size_t)zp * NN;
      float2 b = val;
      if constexpr (EPI & E_BK) b = b * ldg2(A.bkpost + zp * NN + q);
      if constexpr (EPI & E_POST) b = b * ldg2(gpost + g);
      float2 o;
      if constexpr (EPI & E_ID) {
        o = a2 * fmadd(sgn, b, ldg2(gid + g));
      } else {
        o = sa * b;
      }
      *reinterpret_cast<float2*>(gout + g) = o;
      if constexpr (EPI & E_DOT) {
        if (A.want_dotP) acc_dot = fmadd(o, ldg2(gdot + g), acc_dot);
        if (A.want_self) acc_self = fmadd(o, o, acc_self);
      }
    });
  }
  if constexpr (EPI & E_DOT) {  // one partial pair per CTA, indexed like the other slice kernels
    double pd = (double)acc_dot.x + (double)acc_dot.y;
    double ps = (double)acc_self.x + (double)acc_self.y;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      pd += __shfl_xor_sync(0xffffffffu, pd, o2);
      ps += __shfl_xor_sync(0xffffffffu, ps, o2);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = pd;
      red[tid >> 5][1] = ps;
    }
    __syncthreads();
    if (tid == 0) {
      double d = 0.0, q2 = 0.0;
      for (int w = 0; w < PAIR_NT / 32; ++w) {
        d += red[w][0];
        q2 += red[w][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
  }
}

// Paired kernels on by default; UFG_NO_PAIR=1 keeps FP32 on the one-line-per-thread kernel.
inline bool pair_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("UFG_NO_PAIR");
    v = (e && e[0] == '1') ? 0 : 1;
  }
  return v == 1;
}

template <int N, int FAM, int EPI>
inline cudaError_t pair_launch_epi(const SliceCall& c, cudaStream_t st) {
  constexpr int ROWS = N * N;
  constexpr int BUF = ROWS * N;
  TmaPairArgs<N> a;
  std::memset(&a, 0, sizeof(a));
  const long long nelem = c.nelem > 0 ? c.nelem : (long long)c.ntau * N * N * N;
  if (encode_rows<float>(&a.tm_in, c.in, nelem, N, ROWS) != cudaSuccess)
    return cudaErrorNotSupported;
  a.has_pre = (c.pre != nullptr || c.bkpre != nullptr) ? 1 : 0;
  a.pre_mode = c.bkpre != nullptr ? 1 : 0;
  if (a.has_pre) {
    const cudaError_t e = a.pre_mode
                              ? encode_rows<float>(&a.tm_pre, c.bkpre, (long long)N * N * N, N, ROWS)
                              : encode_rows<float>(&a.tm_pre, c.pre, nelem, N, ROWS);
    if (e != cudaSuccess) return cudaErrorNotSupported;
  }
  const LineCoef<N, float>& cf = *reinterpret_cast<const LineCoef<N, float>*>(c.coef);
  for (int i = 0; i < LineShape<N>::NC; ++i) a.coef_x.c[i] = make_float2(cf.c[i], cf.c[i]);
  a.coef_y = a.coef_x;
  a.coef_z = a.coef_x;
  a.bkpost = static_cast<const float*>(c.bkpost);
  a.out = static_cast<float*>(c.out);
  a.id = static_cast<const float*>(c.id);
  a.post = static_cast<const float*>(c.post);
  a.dotP = static_cast<const float*>(c.dotP);
  a.a = c.a;
  a.partials = c.partials;
  a.want_dotP = c.want_dotP;
  a.want_self = c.want_self;
  a.done = c.done;
  a.exec_if = c.exec_if;
  a.tiles = c.tiles;
  a.probs = c.probs;
  a.scale_by_A = c.scale_by_A;
  a.ntau = c.ntau;
  a.shift = c.shift;
  a.units = c.tiles != nullptr ? c.ntiles : c.ntau;
  a.err = c.err;
  a.expire = take_expired_wait(st);
  const size_t smem = (size_t)(a.has_pre ? 2 : 1) * BUF * sizeof(float) + 1024;
  auto kern = slice_tma_pair_kernel<N, FAM, EPI>;
  static int configured = 0;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(2 * BUF * sizeof(float) + 1024));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  if (c.grid_out) *c.grid_out = a.units;
  return launch_k(kern, dim3(a.units), dim3(pair_nt<N>()), smem, st, 1, a);
}

// The paired kernel for the epilogues it covers.
template <int N>
cudaError_t tma_pair_fam(const SliceCall& c, cudaStream_t st) {
  {
    if (!pair_enabled() || c.prec != 1 || c.fop >= 0 || c.prep_out != nullptr || c.post2 ||
        c.U || c.V || (c.bkpre != nullptr && c.pre != nullptr))
      return cudaErrorNotSupported;
    const int mask = (c.id ? E_ID : 0) | (c.post ? E_POST : 0) |
                     ((c.want_dotP || c.want_self) ? E_DOT : 0) | (c.bkpost ? E_BK : 0);
    switch (c.fam) {
      case FAM_KIN:
        switch (mask) {
          case E_ID: return pair_launch_epi<N, FAM_KIN, E_ID>(c, st);
          case E_ID | E_POST: return pair_launch_epi<N, FAM_KIN, E_ID | E_POST>(c, st);
          case E_ID | E_DOT: return pair_launch_epi<N, FAM_KIN, E_ID | E_DOT>(c, st);
          case E_ID | E_POST | E_DOT:
            return pair_launch_epi<N, FAM_KIN, E_ID | E_POST | E_DOT>(c, st);
        }
        break;
      case FAM_FWD:
        switch (mask) {
          case 0: return pair_launch_epi<N, FAM_FWD, 0>(c, st);
          case E_BK: return pair_launch_epi<N, FAM_FWD, E_BK>(c, st);
        }
        break;
      case FAM_INV:
        switch (mask) {
          case 0: return pair_launch_epi<N, FAM_INV, 0>(c, st);
          case E_POST: return pair_launch_epi<N, FAM_INV, E_POST>(c, st);
        }
        break;
    }
  }
  return cudaErrorNotSupported;
}

// The paired kernel for the epilogues it covers; cudaErrorNotSupported otherwise (the caller then
// takes the one-line-per-thread kernel).  Taken for 16^3 slices: 11.3 against 12.9 us for the M
// apply on 16^3 x 1024.  A paired form of the 32^3 cluster kernel measured slower (64-70 against
// 63 us for M on 32^3 x 512): at 168 registers its CTAs leave too few warps per SM to hide the
// cluster waits.
template <int N>
cudaError_t tma_pair_try(const SliceCall& c, cudaStream_t st) {
  if constexpr (N == 16) {
    return tma_pair_fam<N>(c, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace ufg
