// Register-resident 1-D line operators used by every slice kernel.
//
// The kinetic factor exp(-tau K) of the unitary-Fermi-gas fermion matrix (Sec. 1: K diagonal in
// momentum space, k_i = 2 pi n_i / N_x) is separable on the cubic lattice: exp(-tau K) = T (x) T (x) T
// where T is a real symmetric circulant N_x x N_x matrix.  Every operator applied along a line here
// (T itself, the real orthonormal Fourier basis F and its transpose) commutes with the reflection
// x -> -x (mod N), so a line v splits into an even part e (N/2+1 values) and an odd part o (N/2-1
// values) that the operator maps independently: (N/2+1)^2 + (N/2-1)^2 multiply-adds per line instead
// of N^2.
//
//   REAL input : e_0 = v_0, e_H = v_H, e_j = v_j + v_{N-j}, o_j = v_j - v_{N-j}   (H = N/2, 1<=j<H)
//   SPEC input : e_j = v_j (j = 0..H), o_j = v_{H+j}  (cosine slots, then sine slots)
//   REAL output: y_0 = E_0, y_H = E_H, y_i = E_i + O_i, y_{N-i} = E_i - O_i
//   SPEC output: y_i = E_i (i = 0..H), y_{H+i} = O_i
//
// When H = N/2 is even (N = 8, 12, 16, 32) each block splits once more.  The reflection
// x -> H - x (mod N) also commutes with every operator here; on the cosine block it pairs e_j with
// e_{H-j} and on the sine block o_j with o_{H-j}, while on the spectral side it is the sign
// (-1)^k, so cosines of even k and sines of odd k are its symmetric part.  With Q = H/2:
//
//   cosine block, REAL side : s_m = e_m + e_{H-m}, a_m = e_m - e_{H-m} (m < Q), s_Q = e_Q
//                 SPEC side : s_m = e_{2m} (m <= Q), a_m = e_{2m+1} (m < Q)
//   sine block,   REAL side : s_m = o_{m+1} + o_{H-m-1}, a_m = o_{m+1} - o_{H-m-1} (m < Q-1),
//                             s_{Q-1} = o_Q
//                 SPEC side : s_m = o_{2m+1} (m < Q), a_m = o_{2m+2} (m < Q-1)
//
// (outputs recombine the same way, e.g. E_m = U_m + W_m, E_{H-m} = U_m - W_m), leaving four
// blocks of (Q+1)^2, Q^2, Q^2 and (Q-1)^2 multiply-adds: 66 instead of 130 per line for N = 16,
// 258 instead of 514 for N = 32.
//
// The reduced matrices are built on the host in FP64 for each operator and live in the kernel's
// parameter space, so the compiler feeds them to FMA straight from the constant bank.  Layout of
// LineCoef::c: one level: ce ((H+1)^2, row-major, row = output), then co ((H-1)^2); two levels:
// the cosine-symmetric, cosine-antisymmetric, sine-symmetric and sine-antisymmetric blocks.
#pragma once
#include <cuda_runtime.h>

namespace ufg {

template <int N>
struct LineShape {
  static_assert(N >= 4 && N % 2 == 0, "line operators need an even N >= 4");
  static constexpr int H = N / 2;
  static constexpr int Q = H / 2;
  static constexpr bool TWO = (H % 2 == 0) && N >= 8;  // two-level split
  static constexpr int NC = TWO ? (Q + 1) * (Q + 1) + 2 * Q * Q + (Q - 1) * (Q - 1)
                                : (H + 1) * (H + 1) + (H - 1) * (H - 1);
  // block offsets (two levels)
  static constexpr int B_CS = 0;
  static constexpr int B_CA = (Q + 1) * (Q + 1);
  static constexpr int B_SS = B_CA + Q * Q;
  static constexpr int B_SA = B_SS + Q * Q;
};

template <int N, typename R>
struct LineCoef {
  R c[LineShape<N>::NC];
};

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two FP32 lines carried together (x: first line, y: second) so that every multiply-add and fold
// of line_op is one packed FP32x2 instruction of sm_100 and later; the coefficients of
// LineCoef<N, float2> hold each entry twice.
__device__ __forceinline__ float2 fmadd(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&d);
}

// row i of the n x n row-major block at c[off] times x
template <int n, int off, typename R, int NC>
__device__ __forceinline__ R block_row(const R (&c)[NC], const R* x, int i) {
  R acc = c[off + i * n] * x[0];
#pragma unroll
  for (int j = 1; j < n; ++j) acc = fmadd(c[off + i * n + j], x[j], acc);
  return acc;
}

// Double-float value hi + lo (|lo| <= ulp(hi) / 2, about 46 significant bits) whose arithmetic
// runs on the FP32 pipe: sums by Knuth's error-free TwoSum on both parts followed by two
// renormalisations, products by the FMA-based error-free product (Dekker's splitting replaced
// by one fused multiply-add).  GB300's FP64 pipe issues ~1/76 of its FP32 FMA rate, so an
// operation of ~20 FP32 instructions still beats one FP64 instruction by ~4x.  Every step uses
// the _rn intrinsics so that the compiler neither contracts nor reassociates them.
struct dfloat {
  float hi, lo;
};
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfloat df_renorm(float a, float b) {  // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  const dfloat t = df_two_sum(x.lo, y.lo);
  s = df_renorm(s.hi, __fadd_rn(s.lo, t.hi));
  return df_renorm(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) {
  return x + dfloat{-y.hi, -y.lo};
}
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ dfloat fmadd(dfloat a, dfloat b, dfloat c) { return a * b + c; }
__host__ __device__ __forceinline__ dfloat df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfloat x) { return (double)x.hi + (double)x.lo; }

// Applies the reduced operator to the line v[0..N) and hands every output (index, value) to st.
template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, class Store>
__device__ __forceinline__ void line_op(const R (&v)[N], const LineCoef<N, R>& cf, Store&& st) {
  using S = LineShape<N>;
  constexpr int H = S::H;
  R e[H + 1];
  R o[H - 1];  // o[j - 1] holds index j = 1 .. H-1
  if constexpr (IN_SPEC) {
#pragma unroll
    for (int j = 0; j <= H; ++j) e[j] = v[j];
#pragma unroll
    for (int j = 1; j < H; ++j) o[j - 1] = v[H + j];
  } else {
    e[0] = v[0];
    e[H] = v[H];
#pragma unroll
    for (int j = 1; j < H; ++j) {
      e[j] = v[j] + v[N - j];
      o[j - 1] = v[j] - v[N - j];
    }
  }
  if constexpr (S::TWO) {
    constexpr int Q = S::Q;
    R cs[Q + 1], ca[Q], ss[Q], sa[Q - 1 > 0 ? Q - 1 : 1];
    if constexpr (IN_SPEC) {
#pragma unroll
      for (int m = 0; m <= Q; ++m) cs[m] = e[2 * m];
#pragma unroll
      for (int m = 0; m < Q; ++m) ca[m] = e[2 * m + 1];
#pragma unroll
      for (int m = 0; m < Q; ++m) ss[m] = o[2 * m];  // k = 2m+1
#pragma unroll
      for (int m = 0; m < Q - 1; ++m) sa[m] = o[2 * m + 1];  // k = 2m+2
    } else {
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        cs[m] = e[m] + e[H - m];
        ca[m] = e[m] - e[H - m];
      }
      cs[Q] = e[Q];
#pragma unroll
      for (int m = 0; m < Q - 1; ++m) {
        ss[m] = o[m] + o[H - m - 2];  // o_{m+1} + o_{H-m-1}
        sa[m] = o[m] - o[H - m - 2];
      }
      ss[Q - 1] = o[Q - 1];  // o_Q
    }
    // rows of the four blocks, each output emitted as soon as its rows are done
    if constexpr (OUT_SPEC) {
#pragma unroll
      for (int m = 0; m <= Q; ++m) st(2 * m, block_row<Q + 1, S::B_CS>(cf.c, cs, m));
#pragma unroll
      for (int m = 0; m < Q; ++m) st(2 * m + 1, block_row<Q, S::B_CA>(cf.c, ca, m));
#pragma unroll
      for (int m = 0; m < Q; ++m) st(H + 2 * m + 1, block_row<Q, S::B_SS>(cf.c, ss, m));
#pragma unroll
      for (int m = 0; m < Q - 1; ++m) st(H + 2 * m + 2, block_row<Q - 1, S::B_SA>(cf.c, sa, m));
    } else {
      // E_m = U_m + W_m, E_{H-m} = U_m - W_m, E_Q = U_Q; O_m = Us_{m-1} + Ws_{m-1},
      // O_{H-m} = Us_{m-1} - Ws_{m-1}, O_Q = Us_{Q-1}; y_i = E_i + O_i, y_{N-i} = E_i - O_i
      {
        const R U = block_row<Q + 1, S::B_CS>(cf.c, cs, 0);
        const R W = block_row<Q, S::B_CA>(cf.c, ca, 0);
        st(0, U + W);
        st(H, U - W);
      }
#pragma unroll
      for (int m = 1; m < Q; ++m) {
        const R U = block_row<Q + 1, S::B_CS>(cf.c, cs, m);
        const R W = block_row<Q, S::B_CA>(cf.c, ca, m);
        const R Us = block_row<Q, S::B_SS>(cf.c, ss, m - 1);
        const R Ws = block_row<Q - 1, S::B_SA>(cf.c, sa, m - 1);
        const R Em = U + W, Eh = U - W, Om = Us + Ws, Oh = Us - Ws;
        st(m, Em + Om);
        st(N - m, Em - Om);
        st(H - m, Eh + Oh);
        st(H + m, Eh - Oh);  // N - (H - m)
      }
      {
        const R U = block_row<Q + 1, S::B_CS>(cf.c, cs, Q);
        const R Us = block_row<Q, S::B_SS>(cf.c, ss, Q - 1);
        st(Q, U + Us);
        st(N - Q, U - Us);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i <= H; ++i) {
      R E = cf.c[i * (H + 1)] * e[0];
#pragma unroll
      for (int j = 1; j <= H; ++j) E = fmadd(cf.c[i * (H + 1) + j], e[j], E);
      if (i == 0 || i == H) {
        st(i, E);
      } else {
        constexpr int OFF = (H + 1) * (H + 1);
        R O = cf.c[OFF + (i - 1) * (H - 1)] * o[0];
#pragma unroll
        for (int j = 2; j < H; ++j) O = fmadd(cf.c[OFF + (i - 1) * (H - 1) + j - 1], o[j - 1], O);
        if constexpr (OUT_SPEC) {
          st(i, E);
          st(H + i, O);
        } else {
          st(i, E + O);
          st(N - i, E - O);
        }
      }
    }
  }
}


// ---- column-paired form (FP32, two-level shapes) ---------------------------------------------
// Each block row y_i = sum_j c_ij x_j is evaluated as a packed FP32x2 multiply-add chain over the
// column pairs (x_{2j}, x_{2j+1}): acc = (sum over even j, sum over odd j), y_i = acc.x + acc.y,
// plus one scalar multiply-add for the last column of an odd-sized block.  A block of n columns
// costs ceil(n/2) + 1 instructions per row instead of n (N = 32: 169 instead of 258 per line),
// with no broadcast of inputs; the folds stay scalar.  LineCoefK holds every block row as its
// column pairs, followed by the odd last columns.
template <int N>
struct LineShapeK {
  using S = LineShape<N>;
  static constexpr int Q = S::Q;
  static constexpr int NCS = Q + 1, NCA = Q, NSS = Q, NSA = Q - 1;  // block sizes
  // pair offsets of the blocks and tail offsets (tails only for odd sizes)
  static constexpr int P_CS = 0;
  static constexpr int P_CA = P_CS + NCS * (NCS / 2);
  static constexpr int P_SS = P_CA + NCA * (NCA / 2);
  static constexpr int P_SA = P_SS + NSS * (NSS / 2);
  static constexpr int NP = P_SA + NSA * (NSA / 2) > 0 ? P_SA + NSA * (NSA / 2) : 1;
  static constexpr int T_CS = 0;
  static constexpr int T_CA = T_CS + (NCS % 2 ? NCS : 0);
  static constexpr int T_SS = T_CA + (NCA % 2 ? NCA : 0);
  static constexpr int T_SA = T_SS + (NSS % 2 ? NSS : 0);
  static constexpr int NT = T_SA + (NSA % 2 ? NSA : 0);
};

template <int N>
struct LineCoefK {
  float2 p[LineShapeK<N>::NP];
  float t[LineShapeK<N>::NT > 0 ? LineShapeK<N>::NT : 1];
};

// Repacks the row-major blocks of a LineCoef<N, float> (host side).
template <int N>
inline void line_coef_pairs(LineCoefK<N>& out, const LineCoef<N, float>& in) {
  using S = LineShape<N>;
  using K = LineShapeK<N>;
  const int n[4] = {K::NCS, K::NCA, K::NSS, K::NSA};
  const int src[4] = {S::B_CS, S::B_CA, S::B_SS, S::B_SA};
  const int po[4] = {K::P_CS, K::P_CA, K::P_SS, K::P_SA};
  const int to[4] = {K::T_CS, K::T_CA, K::T_SS, K::T_SA};
  for (int b = 0; b < 4; ++b) {
    const int h = n[b] / 2;
    for (int i = 0; i < n[b]; ++i) {
      const float* row = in.c + src[b] + i * n[b];
      for (int j = 0; j < h; ++j) out.p[po[b] + i * h + j] = make_float2(row[2 * j], row[2 * j + 1]);
      if (n[b] % 2) out.t[to[b] + i] = row[n[b] - 1];
    }
  }
}

// row i of a block of n columns, inputs as column pairs xp and (n odd) the last column xl
template <int n, int po, int to, int N>
__device__ __forceinline__ float block_row_k(const LineCoefK<N>& cf, const float2* xp, float xl,
                                             int i) {
  constexpr int h = n / 2;
  float r;
  if constexpr (h > 0) {
    float2 acc = cf.p[po + i * h] * xp[0];
#pragma unroll
    for (int j = 1; j < h; ++j) acc = fmadd(cf.p[po + i * h + j], xp[j], acc);
    r = acc.x + acc.y;
    if constexpr (n % 2) r = __fmaf_rn(cf.t[to + i], xl, r);
  } else {
    r = cf.t[to + i] * xl;
  }
  return r;
}

template <int n>
__device__ __forceinline__ void pack_pairs(const float* x, float2 (&xp)[n / 2 > 0 ? n / 2 : 1]) {
#pragma unroll
  for (int j = 0; j < n / 2; ++j) xp[j] = make_float2(x[2 * j], x[2 * j + 1]);
}

// line_op with the column-paired blocks (same inputs, outputs and order of emission).
template <int N, bool IN_SPEC, bool OUT_SPEC, class Store>
__device__ __forceinline__ void line_op_k(const float (&v)[N], const LineCoefK<N>& cf,
                                          Store&& st) {
  using S = LineShape<N>;
  using K = LineShapeK<N>;
  static_assert(S::TWO, "the column-paired form covers the two-level shapes");
  constexpr int H = S::H, Q = S::Q;
  float e[H + 1];
  float o[H - 1];
  if constexpr (IN_SPEC) {
#pragma unroll
    for (int j = 0; j <= H; ++j) e[j] = v[j];
#pragma unroll
    for (int j = 1; j < H; ++j) o[j - 1] = v[H + j];
  } else {
    e[0] = v[0];
    e[H] = v[H];
#pragma unroll
    for (int j = 1; j < H; ++j) {
      e[j] = v[j] + v[N - j];
      o[j - 1] = v[j] - v[N - j];
    }
  }
  float cs[Q + 1], ca[Q], ss[Q], sa[Q - 1 > 0 ? Q - 1 : 1];
  if constexpr (IN_SPEC) {
#pragma unroll
    for (int m = 0; m <= Q; ++m) cs[m] = e[2 * m];
#pragma unroll
    for (int m = 0; m < Q; ++m) ca[m] = e[2 * m + 1];
#pragma unroll
    for (int m = 0; m < Q; ++m) ss[m] = o[2 * m];
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) sa[m] = o[2 * m + 1];
  } else {
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      cs[m] = e[m] + e[H - m];
      ca[m] = e[m] - e[H - m];
    }
    cs[Q] = e[Q];
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) {
      ss[m] = o[m] + o[H - m - 2];
      sa[m] = o[m] - o[H - m - 2];
    }
    ss[Q - 1] = o[Q - 1];
  }
  float2 csp[K::NCS / 2 > 0 ? K::NCS / 2 : 1], cap[K::NCA / 2 > 0 ? K::NCA / 2 : 1];
  float2 ssp[K::NSS / 2 > 0 ? K::NSS / 2 : 1], sap[K::NSA / 2 > 0 ? K::NSA / 2 : 1];
  pack_pairs<K::NCS>(cs, csp);
  pack_pairs<K::NCA>(ca, cap);
  pack_pairs<K::NSS>(ss, ssp);
  pack_pairs<K::NSA>(sa, sap);
  const float csl = cs[K::NCS - 1], cal = ca[K::NCA - 1], ssl = ss[K::NSS - 1];
  const float sal = sa[K::NSA > 0 ? K::NSA - 1 : 0];
  auto CS = [&](int m) { return block_row_k<K::NCS, K::P_CS, K::T_CS>(cf, csp, csl, m); };
  auto CA = [&](int m) { return block_row_k<K::NCA, K::P_CA, K::T_CA>(cf, cap, cal, m); };
  auto SS = [&](int m) { return block_row_k<K::NSS, K::P_SS, K::T_SS>(cf, ssp, ssl, m); };
  auto SA = [&](int m) { return block_row_k<K::NSA, K::P_SA, K::T_SA>(cf, sap, sal, m); };
  if constexpr (OUT_SPEC) {
#pragma unroll
    for (int m = 0; m <= Q; ++m) st(2 * m, CS(m));
#pragma unroll
    for (int m = 0; m < Q; ++m) st(2 * m + 1, CA(m));
#pragma unroll
    for (int m = 0; m < Q; ++m) st(H + 2 * m + 1, SS(m));
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) st(H + 2 * m + 2, SA(m));
  } else {
    {
      const float U = CS(0), W = CA(0);
      st(0, U + W);
      st(H, U - W);
    }
#pragma unroll
    for (int m = 1; m < Q; ++m) {
      const float U = CS(m), W = CA(m), Us = SS(m - 1), Ws = SA(m - 1);
      const float Em = U + W, Eh = U - W, Om = Us + Ws, Oh = Us - Ws;
      st(m, Em + Om);
      st(N - m, Em - Om);
      st(H - m, Eh + Oh);
      st(H + m, Eh - Oh);
    }
    {
      const float U = CS(Q), Us = SS(Q - 1);
      st(Q, U + Us);
      st(N - Q, U - Us);
    }
  }
}


// line_op on a column-paired coefficient table: the same operator through line_op_k
template <int N, typename R, bool IN_SPEC, bool OUT_SPEC, class Store>
__device__ __forceinline__ void line_op(const float (&v)[N], const LineCoefK<N>& cf, Store&& st) {
  static_assert(sizeof(R) == 4, "column-paired tables are FP32");
  line_op_k<N, IN_SPEC, OUT_SPEC>(v, cf, static_cast<Store&&>(st));
}

}  // namespace ufg
