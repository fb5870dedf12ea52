// TMA-staged form of the slice kernel for the shapes whose rows are one 64- or 128-byte swizzle
// span (FP32 N = 16, 32; FP64 N = 8, 16).
//
// Each CTA (or cluster of C CTAs splitting a slice's z-planes) handles one work unit (a time
// slice, or a (problem, slice) tile of a batch).  Its planes -- and those of the per-site load
// multiplier w / s -- arrive in shared memory through the tensor-memory accelerator
// (cp.async.bulk.tensor, one box per operand, 128B/64B swizzle) completing on an mbarrier, with no
// thread instructions spent on the copy.  The three line passes and the epilogue are those of
// slice_kernel.cuh; shared memory is addressed through the swizzle instead of padding, which
// keeps every pass free of bank conflicts:
//   x-pass: a thread owns a row and reads it as 16-byte chunks, chunk c of row r stored at
//           c ^ f(r) (f(r) = r & 7 for 128-byte rows, (r >> 1) & 3 for 64-byte rows);
//   y-, z-pass: lanes own consecutive x of one row, a permutation of the row's words.
// Clusters of four CTAs for 32^3 FP32 slices; two or three CTAs per SM.
#pragma once
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "line_ops.cuh"
#include "slice_call.h"
#include "scalar_ops.cuh"
#include "slice_kernel.cuh"
#include "launch.cuh"
#include "mbarrier.cuh"

namespace ufg {

// Coefficient table of the TMA slice kernels: column-paired (line_op_k) for FP32 N = 32, where
// the packed multiply-adds measured fastest, the plain row-major blocks otherwise.
template <int N, typename R>
struct TmaCoefSel {
  using type = LineCoef<N, R>;
};
template <>
struct TmaCoefSel<32, float> {
  using type = LineCoefK<32>;
};
template <int N, typename R>
using TmaCoef = typename TmaCoefSel<N, R>::type;

template <int N, typename R>
inline void tma_set_coef(LineCoef<N, R>& out, const void* in) {
  out = *reinterpret_cast<const LineCoef<N, R>*>(in);
}
template <int N>
inline void tma_set_coef(LineCoefK<N>& out, const void* in) {
  line_coef_pairs<N>(out, *reinterpret_cast<const LineCoef<N, float>*>(in));
}

template <int N, typename R>
struct TmaArgs {
  CUtensorMap tm_in;   // [rows][N] view of the input arena, box N x (N/C * N)
  CUtensorMap tm_pre;  // same view of the per-site multiplier (when has_pre)
  CUtensorMap tm_r;    // E_PREP: r and v (boxes 1 and 2)
  CUtensorMap tm_v;
  CUtensorMap tm_id;   // E_PRE with E_ID: 3-D view [t z][y][x] of the identity operand
  // The line operator once per pass: with a single copy the compiler keeps all of its
  // coefficients in registers from the first pass to the last (118 instead of 56 registers for
  // N = 16); separate copies stay constant-bank operands of the multiply-adds.
  TmaCoef<N, R> coef_x;
  TmaCoef<N, R> coef_y;
  TmaCoef<N, R> coef_z;
  const R* bkpost;
  const R* pre_g;  // the load multiplier in global memory (8-CTA clusters read it directly)
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
  int ntau, shift, units, has_pre;
  int pre_mode;  // the multiplier box is a per-mode table (one slice, the same for every t)
  R* prep_out;   // E_PREP: p' (written at the input slice)
  int fop;       // batched: scalar op of the problem's last CTA (-1: none), see SliceCall
  DevScalars* scs;
  unsigned* counters;
  int part_base;
  int* err;  // set on an mbarrier wait that ran out (never expected)
  int expire;  // test hook: run one wait that is made to run out (ufg_test_expire_waits)
};

template <int N, typename R>
struct SwzGeom {
  static constexpr int RB = N * (int)sizeof(R);
  static_assert(RB == 64 || RB == 128, "TMA path covers 64- and 128-byte rows");
  static constexpr unsigned EPC = 16 / sizeof(R);  // elements per 16-byte chunk
  // swizzle phase of row r: chunk c of the row is stored at chunk c ^ f(r)
  __device__ __forceinline__ static unsigned f(unsigned r) {
    return RB == 128 ? (r & 7u) : ((r >> 1) & 3u);
  }
  // element offset of (row r, column col) in a swizzled box (unsigned: shifts and masks only)
  __device__ __forceinline__ static int off(unsigned r, unsigned col) {
    return (int)(r * N + (((col / EPC) ^ f(r)) * EPC) + (col % EPC));
  }
  // element offset of chunk c (16 bytes) of row r
  __device__ __forceinline__ static int chunk(unsigned r, unsigned c) {
    return (int)(r * N + (c ^ f(r)) * EPC);
  }
};

__device__ __forceinline__ void tma_load_rows(void* dst, const CUtensorMap* tm, int row,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(row), "r"(smem_addr(bar))
      : "memory");
}
// box of a 3-D view starting at (x = 0, y, plane)
__device__ __forceinline__ void tma_load_planes(void* dst, const CUtensorMap* tm, int y, int plane,
                                                uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(plane), "r"(smem_addr(bar))
      : "memory");
}

// v[i] *= w[i] for one 16-byte chunk: packed FP32x2 multiplies for FP32
__device__ __forceinline__ void mul_chunk(float (&v)[4], const float (&w)[4]) {
  const float2 a = __fmul2_rn(make_float2(v[0], v[1]), make_float2(w[0], w[1]));
  const float2 b = __fmul2_rn(make_float2(v[2], v[3]), make_float2(w[2], w[3]));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void mul_chunk(double (&v)[2], const double (&w)[2]) {
  v[0] *= w[0];
  v[1] *= w[1];
}

// A store into another CTA's shared memory through its 32-bit shared::cluster address (mapa).
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  uint32_t d;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(smem_addr(p)), "r"(rank));
  return d;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v));
}

// x-pass output: the row's N results are collected in registers and written back as 16-byte
// chunks (chunk c at c ^ f(r)), which keeps the stores of a warp's 32 rows free of bank conflicts
// (element-wise stores of one column index would hit 8 banks only).
template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, class CF>
__device__ __forceinline__ void swz_store_row_impl(R* xs, int r, const R (&v)[N], const CF& cf) {
  using G = SwzGeom<N, R>;
  constexpr int CPR = G::RB / 16, EPC = 16 / (int)sizeof(R);
  R o[N];
  line_op<N, R, IN_SPEC, OUT_SPEC>(v, cf, [&](int i, R val) { o[i] = val; });
#pragma unroll
  for (int c = 0; c < CPR; ++c) {
    R* dst = xs + G::chunk(r, c);
    if constexpr (EPC == 4) {
      *reinterpret_cast<float4*>(dst) =
          make_float4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
    } else {
      *reinterpret_cast<double2*>(dst) = make_double2(o[2 * c], o[2 * c + 1]);
    }
  }
}
template <int N, typename R, class CF>
__device__ __forceinline__ void swz_store_row(R* xs, int r, const R (&v)[N], const CF& cf,
                                              bool in_spec, bool out_spec) {
  if (in_spec) {
    if (out_spec) swz_store_row_impl<N, R, true, true>(xs, r, v, cf);
    else swz_store_row_impl<N, R, true, false>(xs, r, v, cf);
  } else {
    if (out_spec) swz_store_row_impl<N, R, false, true>(xs, r, v, cf);
    else swz_store_row_impl<N, R, false, false>(xs, r, v, cf);
  }
}

constexpr int TMA_NT = 256;
static_assert(TMA_NT == SCAL_NT, "fused scalar updates reduce over SCAL_NT threads");
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 22;  // try_wait rounds before giving up (< 1 s)
constexpr uint32_t EXPIRE_LIMIT = 1u << 8;     // rounds of the wait ufg_test_expire_waits expires

// Resident CTAs per SM the register allocation must allow.
template <int N, typename R>
constexpr int tma_min_blocks() {
  return sizeof(R) == 4 ? (N == 16 ? 5 : 3) : (N <= 8 ? 4 : 3);
}

// Threads per CTA: 256, except for 8-CTA clusters of 32^3 slices (four z-planes per CTA, one
// line per thread and pass), which run 128 threads and twice as many CTAs per SM.
template <int C>
constexpr int tma_nt() {
  return C == 8 ? 128 : TMA_NT;
}
// Resident CTAs per SM of the 8-CTA-cluster kernel (registers: 65536 / (128 x blocks)); a
// compile-time tuning knob (-DUFG_C8_BLOCKS=n).
#ifndef UFG_C8_BLOCKS
#define UFG_C8_BLOCKS 6
#endif
// 8-CTA clusters: the load multiplier as a TMA box in the receive buffer (1) or as per-thread
// global loads (0); a compile-time tuning knob
#ifndef UFG_C8_WBOX
#define UFG_C8_WBOX 1
#endif
template <int N, typename R, int C>
constexpr int tma_blocks() {
  return C == 8 ? UFG_C8_BLOCKS : tma_min_blocks<N, R>();
}

// One work unit per CTA (a persistent loop would make the compiler hoist the ~500 line-operator
// coefficients out of it into registers); several CTAs per SM overlap one another's TMA loads,
// line passes and stores.
template <int N, typename R, int C, int FAM, int EPI>
__global__ void __launch_bounds__(tma_nt<C>(), (tma_blocks<N, R, C>()))
slice_tma_kernel(const __grid_constant__ TmaArgs<N, R> A) {
  pdl_begin();
  namespace cg = cooperative_groups;
  using G = SwzGeom<N, R>;
  constexpr int NP = N / C;
  constexpr int NT = tma_nt<C>();
  constexpr int NN = N * N;
  constexpr int VOL = N * N * N;
  constexpr int ROWS = NP * N;      // rows of one box
  constexpr int BUF = ROWS * N;     // elements of one box
  constexpr int CPR = G::RB / 16;   // 16-byte chunks per row
  constexpr int EPC = 16 / (int)sizeof(R);
  constexpr bool IN_SPEC = (FAM == FAM_INV);
  constexpr bool OUT_SPEC = (FAM == FAM_FWD);
  // 8-CTA clusters keep the pushed z-columns in a buffer of their own, which receives the load
  // multiplier's box first (WBOX; otherwise each thread reads its multiplier row from global
  // memory): each CTA announces (cluster arrive) that its buffer is free once its x-pass is
  // done and waits for the cluster after reading its y-lines, before pushing the results; two
  // 16 KB boxes per CTA let six CTAs share an SM
  constexpr bool SEP = (C == 8);
  constexpr bool WBOX = SEP && (UFG_C8_WBOX != 0) && (EPI & E_PRE) != 0;
  static_assert(!SEP || (EPI & E_PREP) == 0, "the fused direction update needs the box layout");
  static_assert(!SEP || ROWS == NT, "8-CTA clusters: one row per thread");
  extern __shared__ __align__(1024) unsigned char tma_smem[];
  __shared__ double red[NT / 32][2];
  __shared__ alignas(8) uint64_t bar, bar2;

  const int tid = threadIdx.x;
  const int unit = blockIdx.x / C;
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
  if (done != nullptr && A.exec_if >= 0 && *done != A.exec_if) return;  // uniform per cluster
  int rank = 0;
  if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
  // WBOX: the receive buffer holds the multiplier first, so this CTA announces it free only
  // after its x-pass; otherwise at once
  if constexpr (SEP && !WBOX) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  int t_in = t_out;
  if (A.shift < 0) t_in = (t_out == 0) ? ntau - 1 : t_out - 1;
  if (A.shift > 0) t_in = (t_out == ntau - 1) ? 0 : t_out + 1;
  // swizzled boxes need a 1024-byte aligned destination: align the dynamic region explicitly
  unsigned char* const base = tma_smem + ((1024u - (smem_addr(tma_smem) & 1023u)) & 1023u);
  R* const xs = reinterpret_cast<R*>(base);
  const R* const ws = reinterpret_cast<R*>(base) + BUF;

  // ---- TMA: this CTA's planes of x (and of the load multiplier) in one box each ----
  const bool box_pre = A.has_pre && (!SEP || WBOX);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const int row = (int)((off + (size_t)t_in * VOL + (size_t)rank * NP * NN) / N);
    mbar_expect_tx(&bar, (uint32_t)(BUF * sizeof(R)) *
                             ((box_pre ? 2u : 1u) + ((EPI & E_PREP) ? 2u : 0u)));
    tma_load_rows(xs, &A.tm_in, row, &bar);
    if constexpr ((EPI & E_PREP) != 0) {
      tma_load_rows(xs + BUF, &A.tm_r, row, &bar);
      tma_load_rows(xs + 2 * BUF, &A.tm_v, row, &bar);
    }
    if (box_pre)
      tma_load_rows(const_cast<R*>(ws), &A.tm_pre, A.pre_mode ? rank * NP * N : row, &bar);
  }
  // 8-CTA clusters: this thread's row of the multiplier, loaded while the box is in flight
  R wrow[SEP && !WBOX ? N : 1];
  if constexpr (SEP && !WBOX) {
    if (A.has_pre) {
      const R* src = A.pre_g + (size_t)rank * NP * NN + (size_t)tid * N;
      if (!A.pre_mode) src += off + (size_t)t_in * VOL;
#pragma unroll
      for (int c = 0; c < CPR; ++c) {
        R w4[EPC];
        ld16(src + c * EPC, w4);
#pragma unroll
        for (int e = 0; e < EPC; ++e) wrow[c * EPC + e] = w4[e];
      }
    }
  }
  __syncthreads();  // the mbarrier is initialised before anyone waits on it
  mbar_wait_bounded(&bar, 0u, TMA_WAIT_LIMIT, A.err);
  if (A.expire && tid == 0) mbar_expire_one_wait(&bar2, EXPIRE_LIMIT, A.err);

  R pbeta = R(0), pomega = R(0);
  R* pdst = nullptr;
  if constexpr ((EPI & E_PREP) != 0) {
    const DevScalars& sc = A.scs[A.tiles[unit].prob];
    pbeta = R(sc.beta);
    pomega = R(sc.omega);
    pdst = A.prep_out + off + (size_t)t_in * VOL + (size_t)rank * NP * NN;
  }
  // ---- x-pass: one row per thread, read as 16-byte chunks ----
  for (int r = tid; r < ROWS; r += NT) {
    R v[N];
#pragma unroll
    for (int c = 0; c < CPR; ++c) {
      const int o = G::chunk(r, c);
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[c * EPC + e] = xs[o + e];
      if constexpr ((EPI & E_PREP) != 0) {  // p' = r + beta (p - omega v), written back
        R pn[EPC];
#pragma unroll
        for (int e = 0; e < EPC; ++e) {
          pn[e] = xs[BUF + o + e] + pbeta * (v[c * EPC + e] - pomega * xs[2 * BUF + o + e]);
          v[c * EPC + e] = pn[e];
        }
        st16(pdst + r * N + c * EPC, pn);
      } else if (A.has_pre) {
        if constexpr (SEP) {
          R vc[EPC], wc[EPC];
#pragma unroll
          for (int e = 0; e < EPC; ++e) {
            vc[e] = v[c * EPC + e];
            if constexpr (WBOX) {
              wc[e] = ws[o + e];
            } else {
              wc[e] = wrow[c * EPC + e];
            }
          }
          mul_chunk(vc, wc);
#pragma unroll
          for (int e = 0; e < EPC; ++e) v[c * EPC + e] = vc[e];
        } else {
#pragma unroll
          for (int e = 0; e < EPC; ++e) v[c * EPC + e] *= ws[o + e];
        }
      }
    }
    swz_store_row<N, R>(xs, r, v, A.coef_x, IN_SPEC, OUT_SPEC);
  }
  // Clusters exchange by pushing: the y-pass stores each result straight into the CTA that owns
  // its z-column (rows [o RY, (o+1) RY) of every plane belong to CTA o), in that CTA's
  // multiplier box, so the z-pass reads local shared memory only.  The first cluster barrier
  // frees every multiplier box, the second publishes the pushed columns.
  constexpr int RY = N / C;
  R* const recv = xs + BUF;  // [plane z][row y - rank RY][x], plain layout
  if constexpr (SEP) {
    __syncthreads();  // this CTA's x-pass is complete
    if constexpr (WBOX) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    if constexpr (!WBOX) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  } else if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // ---- y-pass ----
  uint32_t rdst[C];  // shared::cluster address of every CTA's receive buffer
#pragma unroll
  for (int o = 0; o < C; ++o) rdst[o] = C > 1 ? cluster_addr(recv, o) : 0u;
  if constexpr (WBOX) {  // one line per thread, read before the wait for every receive buffer
    const int p = tid / N, x = tid - (tid / N) * N;
    R v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = xs[G::off(p * N + y, x)];
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    const int zrow = (rank * NP + p) * RY;
    line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_y, [&](int i, R val) {
      st_cluster(rdst[i / RY] + (uint32_t)(((zrow + i % RY) * N + x) * sizeof(R)), val);
    });
  }
  for (int l = tid; l < (WBOX ? 0 : NP * N); l += NT) {
    const int p = l / N, x = l - (l / N) * N;
    R v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = xs[G::off(p * N + y, x)];
    if constexpr (C > 1) {
      const int zrow = (rank * NP + p) * RY;
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_y, [&](int i, R val) {
        st_cluster(rdst[i / RY] + (uint32_t)(((zrow + i % RY) * N + x) * sizeof(R)), val);
      });
    } else {
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_y,
                                       [&](int i, R val) { xs[G::off(p * N + i, x)] = val; });
    }
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // IDBOX (identity term): this CTA's x box is free now; its z-columns of the identity
  // operand (planes of slice t_out, rows [rank RY, (rank+1) RY)) arrive there by TMA, laid out
  // like the receive buffer
  constexpr bool IDBOX = SEP && (EPI & E_IDB) != 0 && (EPI & E_ID) != 0;
  if constexpr (IDBOX) {
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar, (uint32_t)(BUF * sizeof(R)));
      tma_load_planes(xs, &A.tm_id, rank * (N / C), t_out * N, &bar);
    }
  }
  // ---- z-pass + epilogue ----
  constexpr int COLS = NN / C;
  R sgn = R(1);
  if (A.shift < 0 && t_out != 0) sgn = R(-1);
  if (A.shift > 0 && t_out != ntau - 1) sgn = R(-1);
  const R sa = sgn * R(acoef);
  const R* gid = A.id ? A.id + off : nullptr;
  const R* gpost = A.post ? A.post + off : nullptr;
  const R* gpost2 = A.post2 ? A.post2 + off : nullptr;
  const R* gU = A.U ? A.U + off : nullptr;
  const R* gV = A.V ? A.V + off : nullptr;
  const R* gdot = A.dotP ? A.dotP + off : nullptr;
  R* gout = A.out + off;
  // per-thread partial sums in the working precision (FP64 arithmetic is slow on this part and
  // a thread sums at most N terms); converted to FP64 for the block reduction
  R acc_dot = R(0), acc_self = R(0);
  for (int l = tid; l < COLS; l += NT) {
    const int q = rank * COLS + l;
    const int y = q / N, x = q - (q / N) * N;
    R v[N];
    const int yl = y - rank * RY;
    if constexpr (C > 1) {
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = recv[(z * RY + yl) * N + x];
      if constexpr (IDBOX) mbar_wait_bounded(&bar, 1u, TMA_WAIT_LIMIT, A.err);
    } else {
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = xs[G::off(z * N + y, x)];
    }
    const size_t obase = (size_t)t_out * VOL + q;
    line_op<N, R, IN_SPEC, OUT_SPEC>(v, A.coef_z, [&](int zp, R val) {
      const size_t g = obase + (size_t)zp * NN;
      if constexpr (EPI == EPI_ANY || (EPI & E_UV)) {
        R b = sgn * val;
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
      } else {
        const R* __restrict__ rid = gid;
        const R* __restrict__ rpost = gpost;
        const R* __restrict__ rpost2 = gpost2;
        const R* __restrict__ rdot = gdot;
        R* __restrict__ rout = gout;
        R b = val;
        if constexpr (EPI & E_BK) b *= __ldg(A.bkpost + zp * NN + q);
        if constexpr (EPI & E_POST) b *= __ldg(rpost + g);
        if constexpr (EPI & E_POST2) b *= __ldg(rpost2 + g);
        R o;
        if constexpr (IDBOX) {
          o = R(acoef) * fmadd(sgn, b, xs[(zp * RY + yl) * N + x]);
        } else if constexpr (EPI & E_ID) {
          o = R(acoef) * fmadd(sgn, b, __ldg(rid + g));
        } else {
          o = sa * b;  // sign folded into the scale
        }
        rout[g] = o;
        if constexpr (EPI & E_DOT) {
          if (A.want_dotP) acc_dot += o * __ldg(rdot + g);
          if (A.want_self) acc_self += o * o;
        }
      }
    });
  }
  if (A.want_dotP || A.want_self) {  // one partial pair per CTA, indexed like the plain kernel
    double pd = (double)acc_dot, ps = (double)acc_self;
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
      for (int w = 0; w < NT / 32; ++w) {
        d += red[w][0];
        q2 += red[w][1];
      }
      A.partials[2 * blockIdx.x] = d;
      A.partials[2 * blockIdx.x + 1] = q2;
    }
    if (NT == SCAL_NT && A.fop >= 0 && A.tiles != nullptr) {
      const int prob = A.tiles[unit].prob;
      last_block_update(A.fop, A.scs + prob, A.partials, A.probs[prob].st0 - A.part_base,
                        A.probs[prob].st1 - A.part_base, A.counters + prob);
    }
  }
}

}  // namespace ufg

namespace ufg {

// cuTensorMapEncodeTiled, resolved through the runtime at first use so that loading the library
// does not require the CUDA driver library (libcuda) on machines without a GPU.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <typename R>
inline cudaError_t encode_rows(CUtensorMap* tm, const void* base, long long nelem, int N,
                               int box_rows) {
  EncodeTiledFn encode = encode_tiled_fn();
  if (encode == nullptr) return cudaErrorNotSupported;  // falls back to the plain kernel
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)(nelem / N)};
  const cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(R)};
  const cuuint32_t box[2] = {(cuuint32_t)N, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const int rb = N * (int)sizeof(R);
  const CUtensorMapSwizzle sw = rb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = encode(
      tm, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D view [nelem / N^2][N][N] (planes, rows, x) with an N x box_y x N box, no swizzle
template <typename R>
inline cudaError_t encode_planes(CUtensorMap* tm, const void* base, long long nelem, int N,
                                 int box_y) {
  EncodeTiledFn encode = encode_tiled_fn();
  if (encode == nullptr) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)(nelem / ((long long)N * N))};
  const cuuint64_t strides[2] = {(cuuint64_t)N * sizeof(R), (cuuint64_t)N * N * sizeof(R)};
  const cuuint32_t box[3] = {(cuuint32_t)N, (cuuint32_t)box_y, (cuuint32_t)N};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(
      tm, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, typename R, int C, int FAM, int EPI>
inline cudaError_t tma_launch_epi(const SliceCall& c, cudaStream_t st) {
  constexpr int NP = N / C;
  constexpr int ROWS = NP * N;
  constexpr int BUF = ROWS * N;
  TmaArgs<N, R> a;
  std::memset(&a, 0, sizeof(a));
  const long long nelem = c.nelem > 0 ? c.nelem : (long long)c.ntau * N * N * N;
  cudaError_t e = encode_rows<R>(&a.tm_in, c.in, nelem, N, ROWS);
  if (e != cudaSuccess) return cudaErrorNotSupported;
  // at most one load multiplier: per site (pre) or per mode (bkpre, one slice long)
  a.has_pre = (c.pre != nullptr || c.bkpre != nullptr) ? 1 : 0;
  a.pre_mode = c.bkpre != nullptr ? 1 : 0;
  if (a.has_pre) {
    e = a.pre_mode ? encode_rows<R>(&a.tm_pre, c.bkpre, (long long)N * N * N, N, ROWS)
                   : encode_rows<R>(&a.tm_pre, c.pre, nelem, N, ROWS);
    if (e != cudaSuccess) return cudaErrorNotSupported;
  }
  tma_set_coef<N>(a.coef_x, c.coef);
  a.coef_y = a.coef_x;
  a.coef_z = a.coef_x;
  a.bkpost = static_cast<const R*>(c.bkpost);
  a.pre_g = static_cast<const R*>(a.pre_mode ? c.bkpre : c.pre);
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
  a.ntau = c.ntau;
  a.shift = c.shift;
  a.units = c.tiles != nullptr ? c.ntiles : c.ntau;
  a.err = c.err;
  a.expire = take_expired_wait(st);
  if constexpr ((EPI & E_PREP) != 0) {
    if (c.tiles == nullptr || c.scs == nullptr || c.prep_out == nullptr || a.has_pre)
      return cudaErrorInvalidValue;
    if (encode_rows<R>(&a.tm_r, c.prep_r, nelem, N, ROWS) != cudaSuccess ||
        encode_rows<R>(&a.tm_v, c.prep_v, nelem, N, ROWS) != cudaSuccess)
      return cudaErrorNotSupported;
    a.prep_out = static_cast<R*>(c.prep_out);
  }
  a.fop = c.fop;
  a.scs = c.scs;
  a.counters = c.counters;
  a.part_base = c.part_base;
  if constexpr (C == 8 && (EPI & E_IDB) != 0 && (EPI & E_ID) != 0) {
    // whole slices of one lattice (no batch tiles): planes t N .. t N + N - 1 of the 3-D view
    if (c.tiles != nullptr || c.id == nullptr || nelem % ((long long)N * N) != 0)
      return cudaErrorInvalidValue;
    if (encode_planes<R>(&a.tm_id, c.id, nelem, N, N / C) != cudaSuccess)
      return cudaErrorNotSupported;
  }
  // clusters need the second box as the z-column receive buffer; E_PREP holds p, r and v
  const size_t smem = (size_t)(((EPI & E_PREP) != 0) ? 3 : ((a.has_pre || C > 1) ? 2 : 1)) * BUF *
                          sizeof(R) +
                      1024;
  if (C == 8 && a.has_pre && a.pre_g == nullptr) return cudaErrorInvalidValue;
  auto kern = slice_tma_kernel<N, R, C, FAM, EPI>;
  static int configured = 0;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((((EPI & E_PREP) != 0) ? 3 : 2) * BUF * sizeof(R) + 1024));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  const int clusters = a.units;
  if (c.grid_out) *c.grid_out = clusters * C;
  if (C == 8 && c.fop >= 0) return cudaErrorInvalidValue;  // the fused scalar step needs 256
  return launch_k(kern, dim3(clusters * C), dim3(tma_nt<C>()), smem, st, C, a);
}

template <int N, typename R, int C, int FAM>
inline cudaError_t tma_launch_fam(const SliceCall& c, cudaStream_t st) {
  const int mask = (c.id ? E_ID : 0) | (c.post ? E_POST : 0) | (c.post2 ? E_POST2 : 0) |
                   ((c.U || c.V) ? E_UV : 0) | ((c.want_dotP || c.want_self) ? E_DOT : 0) |
                   (c.bkpost ? E_BK : 0) | (c.prep_out ? E_PREP : 0);
  if ((mask & E_PREP) != 0) {  // only the plain forward transform takes the direction update
    if constexpr (FAM == FAM_FWD && C != 8) {
      if (mask == E_PREP) return tma_launch_epi<N, R, C, FAM, E_PREP>(c, st);
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (FAM == FAM_KIN) {
    if constexpr (C == 8) {  // operands as boxes (E_PRE, E_IDB), see slice_tma_kernel
      if (c.tiles == nullptr) {
        constexpr int B = E_PRE | E_IDB;
        if (c.pre != nullptr || c.bkpre != nullptr) {
          switch (mask) {
            case E_ID: return tma_launch_epi<N, R, C, FAM, E_ID | B>(c, st);
            case E_ID | E_DOT: return tma_launch_epi<N, R, C, FAM, E_ID | E_DOT | B>(c, st);
          }
        } else {
          switch (mask) {
            case E_ID | E_POST: return tma_launch_epi<N, R, C, FAM, E_ID | E_POST | E_IDB>(c, st);
            case E_ID | E_POST | E_DOT:
              return tma_launch_epi<N, R, C, FAM, E_ID | E_POST | E_DOT | E_IDB>(c, st);
          }
        }
      }
    }
    switch (mask) {
      case E_ID: return tma_launch_epi<N, R, C, FAM, E_ID>(c, st);
      case E_ID | E_POST: return tma_launch_epi<N, R, C, FAM, E_ID | E_POST>(c, st);
      case E_ID | E_DOT: return tma_launch_epi<N, R, C, FAM, E_ID | E_DOT>(c, st);
      case E_ID | E_POST | E_DOT: return tma_launch_epi<N, R, C, FAM, E_ID | E_POST | E_DOT>(c, st);
    }
  } else if constexpr (FAM == FAM_FWD) {
    switch (mask) {
      case 0: return tma_launch_epi<N, R, C, FAM, 0>(c, st);
      case E_BK: return tma_launch_epi<N, R, C, FAM, E_BK>(c, st);
    }
  } else {
    switch (mask) {
      case 0: return tma_launch_epi<N, R, C, FAM, 0>(c, st);
      case E_POST: return tma_launch_epi<N, R, C, FAM, E_POST>(c, st);
    }
  }
  return tma_launch_epi<N, R, C, FAM, EPI_ANY>(c, st);
}

// ---- fused WCE term: inverse transform, site multiplier, forward transform -----------------
// One slice per CTA (C = 1).  With x the momentum-space vector, F the real Fourier basis, s the
// per-site multiplier sin(sigma), b the per-mode kinetic factor and the time shift S:
//   DIR 0 (the M1 term of Sec. 3):  y_t = -A sgn(t) b .* F^T( s_{t-1} .* F x_{t-1} )
//   DIR 1 (its transpose): y_t = F^T( -A sgn(t) s_t .* F( b .* x_{t+1} ) )
// x, s and (DIR 1) b arrive as TMA boxes (b through L1 instead measured 10 % slower).
// with sgn(t) = -1 except at the antiperiodic wrap.  The inverse transform's result never leaves
// shared memory: the z pass multiplies it by s in place and the forward passes follow.
template <int N, typename R>
struct M1wArgs {
  CUtensorMap tm_in;  // momentum-space input arena
  CUtensorMap tm_s;   // site multiplier arena
  CUtensorMap tm_k;   // per-mode factor (one slice), DIR 1
  CUtensorMap tm_dot; // FULL with want_dotP: the dot operand arena
  LineCoef<N, R> ci_x, ci_y, ci_z;  // inverse transform, one copy per pass (see TmaArgs)
  LineCoef<N, R> cf_x, cf_y, cf_z;  // forward transform
  const R* bk;                      // per-mode factor, DIR 0 (applied to the output)
  R* out;
  double a;
  const int* done;
  int exec_if;
  const BatchTile* tiles;
  const BatchProb* probs;
  int scale_by_A;
  int ntau;
  int* err;
  int expire;  // test hook, see TmaArgs
  // FULL (the whole operator in momentum space, see slice_m1w_kernel): out = full_scale * M x +
  // bU * U, partial sums and the batched scalar step
  const R* U;
  const R* dotP;
  double full_scale, bU;
  int want_dotP, want_self;
  double* partials;
  int fop;
  DevScalars* scs;
  unsigned* counters;
  int part_base;
};

template <int N, typename R>
constexpr int m1w_min_blocks() {
  return sizeof(R) == 4 ? 5 : (N <= 8 ? 4 : 2);  // DIR 1 (three boxes) fits 4 by shared memory
}

// Row-pair permutation of the one-CTA boxes with 64-byte rows and 16 rows per plane (FP32
// N = 16): a row's 16 words sit in banks 0-15 or 16-31 by the parity of its row index, and a
// plane is 1 KB, so the y-pass (a warp reads the same row y of planes p and p + 1) and the
// y-pass stores would hit the same banks twice.  Planes with odd p keep row y at position y ^ 1
// (the swizzle phase (r >> 1) & 3 is unchanged).  The first x-pass writes its rows to the
// permuted positions, every later pass addresses them there; the TMA boxes of multipliers and
// epilogue operands keep the plain layout.
template <int N, typename R>
constexpr bool swz_perm() {
#ifndef UFG_SWZ_PERM
#define UFG_SWZ_PERM 1
#endif
  return UFG_SWZ_PERM != 0 && N == 16 && sizeof(R) == 4;
}
// position of row r = p N + y under the permutation
template <int N, bool PERM>
__device__ __forceinline__ int prow(int r) {
  return PERM ? (r ^ ((r / N) & 1)) : r;
}

// Line passes over one swizzled slice box (all N planes in this CTA).  PERM_OUT: rows are read
// at their plain positions and written to the permuted ones (the rows r and r ^ 1 of a plane
// belong to one warp, which has read both before either is written).
template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, bool MUL, class CF,
          bool PERM_OUT = false>
__device__ __forceinline__ void swz_xpass(R* xs, const R* mul, const CF& cf) {
  using G = SwzGeom<N, R>;
  constexpr int CPR = G::RB / 16, EPC = 16 / (int)sizeof(R);
  static_assert(!PERM_OUT || (N * N) % TMA_NT == 0, "the warp-wide exchange needs whole rows");
  for (int r = threadIdx.x; r < N * N; r += TMA_NT) {
    R v[N];
#pragma unroll
    for (int c = 0; c < CPR; ++c) {
      const int o = G::chunk(r, c);
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[c * EPC + e] = MUL ? xs[o + e] * mul[o + e] : xs[o + e];
    }
    if constexpr (PERM_OUT) {
      R o[N];
      line_op<N, R, IN_SPEC, OUT_SPEC>(v, cf, [&](int i, R val) { o[i] = val; });
      __syncwarp();
      const int rp = prow<N, true>(r);
#pragma unroll
      for (int c = 0; c < CPR; ++c) {
        R* dst = xs + G::chunk(rp, c);
#pragma unroll
        for (int e = 0; e < EPC; ++e) dst[e] = o[c * EPC + e];
      }
    } else {
      swz_store_row<N, R>(xs, r, v, cf, IN_SPEC, OUT_SPEC);
    }
  }
}

template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, class CF, bool PERM = false>
__device__ __forceinline__ void swz_ypass(R* xs, const CF& cf) {
  using G = SwzGeom<N, R>;
  for (int l = threadIdx.x; l < N * N; l += TMA_NT) {
    const int p = l / N, x = l - (l / N) * N;
    R v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = xs[G::off(prow<N, PERM>(p * N + y), x)];
    line_op<N, R, IN_SPEC, OUT_SPEC>(
        v, cf, [&](int i, R val) { xs[G::off(prow<N, PERM>(p * N + i), x)] = val; });
  }
}

//
// FULL: the fermion matrix itself in the momentum basis, x = F^T x^ per slice.  With
// B_t = e^{-tau K} w_t, w_t = 1 + A sin(sigma_t) (Sec. 1), and F e^{-tau K} = b .* F:
//   DIR 0:  (M x^)_t   = x^_t + sgn(t) b .* F( w_{t-1} .* F^T x^_{t-1} )
//   DIR 1:  (M^T x^)_t = x^_t + sgn(t) F( w_t .* F^T( b .* x^_{t+1} ) )
// i.e. the same three steps with w as the site multiplier and a = 1, plus the identity term.
// Once the inverse transform has consumed the multiplier (and b) boxes, they receive x^_t and
// the dot operand's slice by TMA, overlapping the forward x and y passes.
template <int N, typename R, int DIR, bool FULL>
__global__ void __launch_bounds__(TMA_NT, (m1w_min_blocks<N, R>()))
slice_m1w_kernel(const __grid_constant__ M1wArgs<N, R> A) {
  pdl_begin();
  using G = SwzGeom<N, R>;
  constexpr int NN = N * N;
  constexpr int VOL = N * NN;
  extern __shared__ __align__(1024) unsigned char tma_smem[];
  __shared__ alignas(8) uint64_t bar, bar2;
  __shared__ double red[FULL ? TMA_NT / 32 : 1][2];
  const int tid = threadIdx.x;
  int t_out, ntau;
  size_t off = 0;
  const int* done = A.done;
  double acoef = A.a;
  if (A.tiles != nullptr) {
    const BatchTile tl = A.tiles[blockIdx.x];
    const BatchProb& pr = A.probs[tl.prob];
    t_out = tl.t0;
    ntau = pr.ntau;
    off = (size_t)pr.off;
    done = pr.done;
    if (A.scale_by_A) acoef *= pr.A;
  } else {
    t_out = blockIdx.x;
    ntau = A.ntau;
  }
  if (done != nullptr && A.exec_if >= 0 && *done != A.exec_if) return;
  const int t_in = DIR == 0 ? (t_out == 0 ? ntau - 1 : t_out - 1)
                            : (t_out == ntau - 1 ? 0 : t_out + 1);
  const R sgn = (DIR == 0 ? t_out != 0 : t_out != ntau - 1) ? R(-1) : R(1);
  const int t_s = DIR == 0 ? t_in : t_out;  // slice of the site multiplier
  unsigned char* const base = tma_smem + ((1024u - (smem_addr(tma_smem) & 1023u)) & 1023u);
  R* const xs = reinterpret_cast<R*>(base);
  R* const ss = xs + VOL;
  R* const ks = ss + VOL;
  const int row_in = (int)((off + (size_t)t_in * VOL) / N);
  R* const ds = ks;  // FULL: the dot operand's slice (third box)
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, (uint32_t)(VOL * sizeof(R)) * (DIR == 1 ? 3u : 2u));
    tma_load_rows(xs, &A.tm_in, row_in, &bar);
    tma_load_rows(ss, &A.tm_s, (int)((off + (size_t)t_s * VOL) / N), &bar);
    if (DIR == 1) tma_load_rows(ks, &A.tm_k, 0, &bar);
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0u, TMA_WAIT_LIMIT, A.err);
  if (A.expire && tid == 0) mbar_expire_one_wait(&bar2, EXPIRE_LIMIT, A.err);
  // inverse transform (spectral input); DIR 1 weights the modes by b on the way in.  With PERM
  // the slice leaves the first pass in the permuted row layout (swz_perm), the s and b boxes
  // keep the plain one.
  constexpr bool PERM = swz_perm<N, R>();
  swz_xpass<N, R, true, false, DIR == 1, LineCoef<N, R>, PERM>(xs, ks, A.ci_x);
  __syncthreads();
  swz_ypass<N, R, true, false, LineCoef<N, R>, PERM>(xs, A.ci_y);
  __syncthreads();
  const R f1 = DIR == 1 ? sgn * R(acoef) : R(1);
  for (int q = tid; q < NN; q += TMA_NT) {  // z pass, times the site multiplier, in place
    const int y = q / N, x = q - (q / N) * N;
    R v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = xs[G::off(prow<N, PERM>(z * N + y), x)];
    line_op<N, R, true, false>(v, A.ci_z, [&](int zp, R val) {
      xs[G::off(prow<N, PERM>(zp * N + y), x)] = (f1 * ss[G::off(zp * N + y, x)]) * val;
    });
  }
  __syncthreads();
  if constexpr (FULL) {  // the multiplier and b boxes are free: prefetch the epilogue operands
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int row_out = (int)((off + (size_t)t_out * VOL) / N);
      mbar_expect_tx(&bar, (uint32_t)(VOL * sizeof(R)) * (A.want_dotP ? 2u : 1u));
      tma_load_rows(ss, &A.tm_in, row_out, &bar);
      if (A.want_dotP) tma_load_rows(ds, &A.tm_dot, row_out, &bar);
    }
  }
  // forward transform (spectral output); the x-pass works on physical rows, so the permuted
  // layout stays
  swz_xpass<N, R, false, true, false>(xs, nullptr, A.cf_x);
  __syncthreads();
  swz_ypass<N, R, false, true, LineCoef<N, R>, PERM>(xs, A.cf_y);
  __syncthreads();
  const R f2 = DIR == 0 ? sgn * R(acoef) : R(1);
  R* const gout = A.out + off + (size_t)t_out * VOL;
  if constexpr (!FULL) {
    for (int q = tid; q < NN; q += TMA_NT) {
      const int y = q / N, x = q - (q / N) * N;
      R v[N];
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = xs[G::off(prow<N, PERM>(z * N + y), x)];
      line_op<N, R, false, true>(v, A.cf_z, [&](int zp, R val) {
        R o = f2 * val;
        if constexpr (DIR == 0) o *= __ldg(A.bk + zp * NN + q);
        gout[zp * NN + q] = o;
      });
    }
  } else {
    mbar_wait_bounded(&bar, 1u, TMA_WAIT_LIMIT, A.err);
    const size_t so = off + (size_t)t_out * VOL;
    const R* __restrict__ gU = A.U ? A.U + so : nullptr;
    const R fs = R(A.full_scale), bU = R(A.bU);
    R acc_dot = R(0), acc_self = R(0);
    for (int q = tid; q < NN; q += TMA_NT) {
      const int y = q / N, x = q - (q / N) * N;
      R v[N];
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = xs[G::off(prow<N, PERM>(z * N + y), x)];
      line_op<N, R, false, true>(v, A.cf_z, [&](int zp, R val) {
        const int g = zp * NN + q;
        const int os = G::off(zp * N + y, x);
        R m = f2 * val;
        if constexpr (DIR == 0) m *= __ldg(A.bk + g);
        R o = fs * (m + ss[os]);
        if (gU != nullptr) o = fmadd(bU, __ldg(gU + g), o);
        gout[g] = o;
        if (A.want_dotP) acc_dot = fmadd(o, ds[os], acc_dot);
        if (A.want_self) acc_self = fmadd(o, o, acc_self);
      });
    }
    if (A.want_dotP || A.want_self) {  // one partial pair per CTA, as the slice kernels
      double pd = (double)acc_dot, ps = (double)acc_self;
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
        for (int w = 0; w < TMA_NT / 32; ++w) {
          d += red[w][0];
          q2 += red[w][1];
        }
        A.partials[2 * blockIdx.x] = d;
        A.partials[2 * blockIdx.x + 1] = q2;
      }
      if (A.fop >= 0 && A.tiles != nullptr) {
        const int prob = A.tiles[blockIdx.x].prob;
        last_block_update(A.fop, A.scs + prob, A.partials, A.probs[prob].st0 - A.part_base,
                          A.probs[prob].st1 - A.part_base, A.counters + prob);
      } else if (A.fop >= 0) {  // one lattice: the grid's last CTA
        last_block_update(A.fop, A.scs, A.partials, 0, (int)gridDim.x, A.counters);
      }
    }
  }
}

template <int N, typename R, int DIR, bool FULL>
inline cudaError_t m1w_launch(const SliceCall& c, cudaStream_t st) {
  constexpr int VOL = N * N * N;
  M1wArgs<N, R> a;
  std::memset(&a, 0, sizeof(a));
  const long long nelem = c.nelem > 0 ? c.nelem : (long long)c.ntau * VOL;
  if (c.in == nullptr || c.pre == nullptr || c.out == nullptr || c.coef == nullptr ||
      c.coef2 == nullptr || (DIR == 1 ? c.bkpre : c.bkpost) == nullptr)
    return cudaErrorInvalidValue;
  if (encode_rows<R>(&a.tm_in, c.in, nelem, N, N * N) != cudaSuccess ||
      encode_rows<R>(&a.tm_s, c.pre, nelem, N, N * N) != cudaSuccess ||
      (DIR == 1 && encode_rows<R>(&a.tm_k, c.bkpre, VOL, N, N * N) != cudaSuccess))
    return cudaErrorNotSupported;
  a.ci_x = *reinterpret_cast<const LineCoef<N, R>*>(c.coef);
  a.ci_y = a.ci_x;
  a.ci_z = a.ci_x;
  a.cf_x = *reinterpret_cast<const LineCoef<N, R>*>(c.coef2);
  a.cf_y = a.cf_x;
  a.cf_z = a.cf_x;
  a.bk = static_cast<const R*>(c.bkpost);
  a.out = static_cast<R*>(c.out);
  a.a = c.a;
  a.done = c.done;
  a.exec_if = c.exec_if;
  a.tiles = c.tiles;
  a.probs = c.probs;
  a.scale_by_A = c.scale_by_A;
  a.ntau = c.ntau;
  a.err = c.err;
  a.expire = take_expired_wait(st);
  if constexpr (FULL) {
    if ((c.want_dotP && c.dotP == nullptr) || ((c.want_dotP || c.want_self) && !c.partials) ||
        (c.fop >= 0 && (c.scs == nullptr || c.counters == nullptr ||
                        (c.tiles == nullptr && c.part_base != 0))))
      return cudaErrorInvalidValue;
    if (c.want_dotP && encode_rows<R>(&a.tm_dot, c.dotP, nelem, N, N * N) != cudaSuccess)
      return cudaErrorNotSupported;
    a.U = static_cast<const R*>(c.U);
    a.dotP = static_cast<const R*>(c.dotP);
    a.full_scale = c.full_scale;
    a.bU = c.bU;
    a.want_dotP = c.want_dotP;
    a.want_self = c.want_self;
    a.partials = c.partials;
    a.fop = c.fop;
    a.scs = c.scs;
    a.counters = c.counters;
    a.part_base = c.part_base;
  }
  const size_t smem =
      (size_t)((DIR == 1 || (FULL && c.want_dotP)) ? 3 : 2) * VOL * sizeof(R) + 1024;
  auto kern = slice_m1w_kernel<N, R, DIR, FULL>;
  static int configured = 0;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(3 * VOL * sizeof(R) + 1024));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    configured = 1;
  }
  const int units = c.tiles != nullptr ? c.ntiles : c.ntau;
  if (c.grid_out) *c.grid_out = units;
  return launch_k(kern, dim3(units), dim3(TMA_NT), smem, st, 1, a);
}

template <int N, typename R, bool FULL>
inline cudaError_t m1w_dir(const SliceCall& c, cudaStream_t st) {
  return c.shift < 0 ? m1w_launch<N, R, 0, FULL>(c, st) : m1w_launch<N, R, 1, FULL>(c, st);
}

template <int N>
cudaError_t m1w_df_try(const SliceCall& c, cudaStream_t st);

template <int N>
inline cudaError_t slice_m1w_try(const SliceCall& c, cudaStream_t st) {
  if (!slice_m1w_supported(N, c.prec) || c.shift == 0) return cudaErrorNotSupported;
  if (c.emulate64 && c.prec == 0) return m1w_df_try<N>(c, st);
  if constexpr (N == 16) {
    if (c.prec == 1) return c.m1w_full ? m1w_dir<16, float, true>(c, st)
                                       : m1w_dir<16, float, false>(c, st);
    return c.m1w_full ? m1w_dir<16, double, true>(c, st) : m1w_dir<16, double, false>(c, st);
  } else if constexpr (N == 8) {
    return c.m1w_full ? m1w_dir<8, double, true>(c, st) : m1w_dir<8, double, false>(c, st);
  }
  return cudaErrorNotSupported;
}

// CTAs per cluster of the FP32 32^3 slice kernel: 8 (the default; a receive buffer of its own,
// six CTAs per SM) or, with UFG_TMA_C32=4, 4 (the receive buffer shared with the multiplier box,
// two cluster-wide waits, three CTAs per SM).  On the 32^3 x 512 applies: M 63.1 against 63.0 us,
// M^T 58.0 against 69.5 us.
inline int tma_c32() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("UFG_TMA_C32");
    v = (e && std::atoi(e) == 4) ? 4 : 8;
  }
  return v;
}

// Paired-line FP32 kernel (slice_pair.cuh); cudaErrorNotSupported outside what it covers.
template <int N>
cudaError_t tma_pair_try(const SliceCall& c, cudaStream_t st);

// TMA path for one N: cudaErrorNotSupported when the call is outside what it covers.
template <int N>
inline cudaError_t slice_tma_try(const SliceCall& c, cudaStream_t st) {
  if (c.bkpre != nullptr && c.pre != nullptr) return cudaErrorNotSupported;
  if (c.prec == 1) {
    const cudaError_t e = tma_pair_try<N>(c, st);
    if (e != cudaErrorNotSupported) return e;
    if constexpr (N == 32) {
      if (tma_c32() == 8 && c.fop < 0) {
        switch (c.fam) {
          case FAM_KIN: return tma_launch_fam<N, float, 8, FAM_KIN>(c, st);
          case FAM_FWD: return tma_launch_fam<N, float, 8, FAM_FWD>(c, st);
          case FAM_INV: return tma_launch_fam<N, float, 8, FAM_INV>(c, st);
        }
      }
    }
    if constexpr (N == 16 || N == 32) {
      constexpr int C = N == 32 ? 4 : 1;
      switch (c.fam) {
        case FAM_KIN: return tma_launch_fam<N, float, C, FAM_KIN>(c, st);
        case FAM_FWD: return tma_launch_fam<N, float, C, FAM_FWD>(c, st);
        case FAM_INV: return tma_launch_fam<N, float, C, FAM_INV>(c, st);
      }
    }
  } else {
    if constexpr (N == 8 || N == 16) {
      switch (c.fam) {
        case FAM_KIN: return tma_launch_fam<N, double, 1, FAM_KIN>(c, st);
        case FAM_FWD: return tma_launch_fam<N, double, 1, FAM_FWD>(c, st);
        case FAM_INV: return tma_launch_fam<N, double, 1, FAM_INV>(c, st);
      }
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace ufg
