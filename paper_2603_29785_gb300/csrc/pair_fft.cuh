// Compile-time Stockham FFT over a PAIR of rows with packed FP32x2
// arithmetic (sm_100 family `add/sub/mul/fma.f32x2`).
//
// Two transforms of the same length run in lockstep: a value of the pair
// type C2 holds one complex element of each row, packed component-wise,
//   re = (Re row 0, Re row 1),  im = (Im row 0, Im row 1),
// so every butterfly add, constant multiply and twiddle multiply is one
// packed instruction for both rows (half the FP32 issue slots of two scalar
// transforms), multiplications by +-i are register renames folded into the
// following add or subtract, and the inter-stage twiddle of an item is read
// once for both rows.  The stage formula, twiddle tables and output order
// are those of fft_static.cuh (App. C DFT; Stockham autosort): stage s with
// span NS and radix R takes a_i = in[j + i M/R], multiplies by the table's
// exp(-+2 pi i i (j mod NS) / (NS R)), applies DFT_R and writes
// out[(j / NS) NS R + (j mod NS) + i NS].  Shared memory holds one C2 per
// element (16 bytes: both rows' values of that element), so each exchange is
// one 128-bit access per element pair.
#pragma once

#include "fft_core.cuh"
#include "fft_static.cuh"

namespace qtam {
namespace pr {

struct C2 {
  float2 re, im;
};

// packed FP32x2 arithmetic: padd / psub / pmul / pfma of fft_core.cuh
__device__ __forceinline__ float2 pk(float k) { return make_float2(k, k); }

// ---- complex operations on a row pair -------------------------------------
__device__ __forceinline__ C2 operator+(C2 a, C2 b) { return C2{padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ C2 operator-(C2 a, C2 b) { return C2{psub(a.re, b.re), psub(a.im, b.im)}; }
// a + S i b
template <int S> __device__ __forceinline__ C2 add_si2(C2 a, C2 b) {
  if constexpr (S > 0) {
    return C2{psub(a.re, b.im), padd(a.im, b.re)};
  } else {
    return C2{padd(a.re, b.im), psub(a.im, b.re)};
  }
}
// a k + b for a real constant k
__device__ __forceinline__ C2 fmak(C2 a, float k, C2 b) { return C2{pfma(a.re, pk(k), b.re), pfma(a.im, pk(k), b.im)}; }
__device__ __forceinline__ C2 scalek(C2 a, float k) { return C2{pmul(a.re, pk(k)), pmul(a.im, pk(k))}; }
__device__ __forceinline__ C2 negc(C2 a) { return scalek(a, -1.0f); }
// S i a
template <int S> __device__ __forceinline__ C2 mul_si(C2 a) {
  if constexpr (S > 0) {
    return C2{pmul(a.im, pk(-1.0f)), a.re};
  } else {
    return C2{a.im, pmul(a.re, pk(-1.0f))};
  }
}
// a (c + i s) for constants c, s
__device__ __forceinline__ C2 cmulk(C2 a, float c, float s) {
  return C2{pfma(a.re, pk(c), pmul(a.im, pk(-s))), pfma(a.re, pk(s), pmul(a.im, pk(c)))};
}
// stage twiddle from a pair table entry t = (c, c, s, s) holding
// exp(-2 pi i theta) = c + i s: SIGN < 0 multiplies by it, SIGN > 0 by its
// conjugate
template <int SIGN> __device__ __forceinline__ C2 twmul(C2 a, float4 t) {
  const float2 c = make_float2(t.x, t.y), s = make_float2(t.z, t.w);
  if constexpr (SIGN < 0) {
    return C2{psub(pmul(a.re, c), pmul(a.im, s)), pfma(a.re, s, pmul(a.im, c))};
  } else {
    return C2{pfma(a.im, s, pmul(a.re, c)), psub(pmul(a.im, c), pmul(a.re, s))};
  }
}

// ---- small DFTs on row pairs: a[0..R) -> DFT_R(a) in natural order --------
// (S = +1: exp(+2 pi i jk / R), synthesis, unscaled; S = -1: analysis)
template <int R, int S> struct D2;

template <int S> struct D2<2, S> {
  __device__ __forceinline__ static void run(C2* a) {
    const C2 t = a[0];
    a[0] = t + a[1];
    a[1] = t - a[1];
  }
};

// y1 = m + i h d, y2 = m - i h d with m = a0 - (a1 + a2)/2, d = a1 - a2,
// h = S sin(2 pi / 3)
template <int S> struct D2<3, S> {
  __device__ __forceinline__ static void run(C2* a) {
    constexpr float h = (float)(S * 0.86602540378443864676);
    const C2 t = a[1] + a[2], d = a[1] - a[2];
    const C2 m = fmak(t, -0.5f, a[0]);
    a[0] = a[0] + t;
    a[1] = C2{pfma(d.im, pk(-h), m.re), pfma(d.re, pk(h), m.im)};
    a[2] = C2{pfma(d.im, pk(h), m.re), pfma(d.re, pk(-h), m.im)};
  }
};

template <int S> struct D2<4, S> {
  __device__ __forceinline__ static void run(C2* a) {
    const C2 s02 = a[0] + a[2], d02 = a[0] - a[2];
    const C2 s13 = a[1] + a[3], t = a[1] - a[3];
    a[0] = s02 + s13;
    a[2] = s02 - s13;
    a[1] = add_si2<S>(d02, t);
    a[3] = add_si2<-S>(d02, t);
  }
};

// y1,4 = m1 +- i r1, y2,3 = m2 +- i r2 with t1 = a1 + a4, d1 = a1 - a4,
// t2 = a2 + a3, d2 = a2 - a3, m1 = a0 + c1 t1 + c2 t2, m2 = a0 + c2 t1 + c1 t2,
// r1 = s1 d1 + s2 d2, r2 = s2 d1 - s1 d2 (c_k = cos(2 pi k/5), s_k = S sin(2 pi k/5))
template <int S> struct D2<5, S> {
  __device__ __forceinline__ static void run(C2* a) {
    constexpr float c1 = (float)ce_cos2pi(1, 5), c2 = (float)ce_cos2pi(2, 5);
    constexpr float s1 = (float)(S * ce_sin2pi(1, 5)), s2 = (float)(S * ce_sin2pi(2, 5));
    const C2 t1 = a[1] + a[4], d1 = a[1] - a[4];
    const C2 t2 = a[2] + a[3], d2 = a[2] - a[3];
    const C2 m1 = fmak(t1, c1, fmak(t2, c2, a[0]));
    const C2 m2 = fmak(t1, c2, fmak(t2, c1, a[0]));
    const C2 r1 = fmak(d1, s1, scalek(d2, s2));
    const C2 r2 = fmak(d1, s2, scalek(d2, -s1));
    a[0] = a[0] + t1 + t2;
    a[1] = add_si2<1>(m1, r1);
    a[4] = add_si2<-1>(m1, r1);
    a[2] = add_si2<1>(m2, r2);
    a[3] = add_si2<-1>(m2, r2);
  }
};

// composite R = R1 R2 (index j = R2 j1 + j2, output k = k1 + R1 k2) with the
// inner twiddles w_R^(S j2 k1) as constants; quarter turns become renames
template <int E, int R, int S> __device__ __forceinline__ void twc(C2& x) {
  constexpr int e = E % R;
  if constexpr (e == 0) {
  } else if constexpr (4 * e == R) {
    x = mul_si<S>(x);
  } else if constexpr (2 * e == R) {
    x = negc(x);
  } else if constexpr (4 * e == 3 * R) {
    x = mul_si<-S>(x);
  } else {
    constexpr float c = (float)ce_cos2pi(e, R);
    constexpr float sn = (float)(S * ce_sin2pi(e, R));
    x = cmulk(x, c, sn);
  }
}
template <int R1, int R2, int S> struct D2Composite {
  static constexpr int R = R1 * R2;
  template <int J2, int... K1> __device__ __forceinline__ static void twcol(C2* col, std::integer_sequence<int, K1...>) {
    (twc<J2 * K1, R, S>(col[K1]), ...);
  }
  template <int J2> __device__ __forceinline__ static void column(const C2* a, C2* b) {
    C2 col[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) col[j1] = a[R2 * j1 + J2];
    D2<R1, S>::run(col);
    twcol<J2>(col, std::make_integer_sequence<int, R1>{});
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) b[J2 * R1 + k1] = col[k1];
  }
  template <int... J2> __device__ __forceinline__ static void columns(const C2* a, C2* b, std::integer_sequence<int, J2...>) {
    (column<J2>(a, b), ...);
  }
  __device__ __forceinline__ static void run(C2* a) {
    C2 b[R];
    columns(a, b, std::make_integer_sequence<int, R2>{});
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C2 row[R2];
#pragma unroll
      for (int j2 = 0; j2 < R2; ++j2) row[j2] = b[j2 * R1 + k1];
      D2<R2, S>::run(row);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = row[k2];
    }
  }
};
// prime-factor (Good-Thomas) R = R1 R2, gcd(R1, R2) = 1: input index
// (R2 n1 + R1 n2) mod R, output index (E1 k1 + E2 k2) mod R, no twiddles
template <int R1, int R2, int S> struct D2PFA {
  static constexpr int R = R1 * R2;
  static constexpr int E1 = R2 * inv_mod(R2 % R1, R1);
  static constexpr int E2 = R1 * inv_mod(R1 % R2, R2);
  __device__ __forceinline__ static void run(C2* a) {
    C2 b[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      C2 col[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) col[n1] = a[(R2 * n1 + R1 * n2) % R];
      D2<R1, S>::run(col);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) b[k1 * R2 + n2] = col[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C2 row[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) row[n2] = b[k1 * R2 + n2];
      D2<R2, S>::run(row);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[(E1 * k1 + E2 * k2) % R] = row[k2];
    }
  }
};

template <int S> struct D2<6, S> : D2PFA<2, 3, S> {};
template <int S> struct D2<8, S> : D2Composite<2, 4, S> {};
template <int S> struct D2<10, S> : D2PFA<2, 5, S> {};
template <int S> struct D2<12, S> : D2PFA<4, 3, S> {};
template <int S> struct D2<15, S> : D2PFA<3, 5, S> {};
template <int S> struct D2<16, S> : D2Composite<4, 4, S> {};
template <int S> struct D2<20, S> : D2PFA<4, 5, S> {};
template <int S> struct D2<25, S> : D2Composite<5, 5, S> {};
template <int S> struct D2<32, S> : D2Composite<4, 8, S> {};

// ---- shared memory: one C2 (float4) per element, padded e + (e >> PS) ------
template <int PS> struct PSmem {
  float4* sm;
  __device__ __forceinline__ static int addr(int e) {
    if constexpr (PS >= 30) {
      return e;
    } else {
      return e + (e >> PS);
    }
  }
  // element j + i STEP; when STEP is a multiple of the padding period the
  // padding of the run is a compile-time offset
  template <int STEP> __device__ __forceinline__ static int addr_s(int j, int i) {
    if constexpr (PS >= 30) {
      return j + i * STEP;
    } else if constexpr (STEP % (1 << PS) == 0) {
      return addr(j) + i * (STEP + (STEP >> PS));
    } else {
      return addr(j + i * STEP);
    }
  }
  template <int STEP> __device__ __forceinline__ C2 get_s(int j, int i) const {
    const float4 v = sm[addr_s<STEP>(j, i)];
    return C2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
  }
  template <int STEP> __device__ __forceinline__ void put_s(int j, int i, C2 v) const {
    sm[addr_s<STEP>(j, i)] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
  }
};

// One stage: radix R, span NS, one row pair of length M on NT threads.  The
// source / destination functors take (j, i) -> element j + i STEP.
template <int SIGN, int M, int NT, int NS, int R, class Src, class Dst>
__device__ __forceinline__ void pstage(const float4* __restrict__ tws, const Src& src, const Dst& dst, bool inplace) {
  constexpr int MR = M / R;
  constexpr int IPT = (MR + NT - 1) / NT;
  C2 a[IPT][R];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int j = threadIdx.x + q * NT;
    if (MR % NT == 0 || j < MR) {
#pragma unroll
      for (int i = 0; i < R; ++i) a[q][i] = src.template get_s<MR>(j, i);
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int i = 1; i < R; ++i) a[q][i] = twmul<SIGN>(a[q][i], __ldg(&tws[i * NS + k]));
      }
      D2<R, SIGN>::run(a[q]);
    }
  }
  if (inplace) __syncthreads();
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int j = threadIdx.x + q * NT;
    if (MR % NT == 0 || j < MR) {
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int i = 0; i < R; ++i) dst.template put_s<NS>(base, i, a[q][i]);
    }
  }
}

template <int SIGN, int M, int NT, int PS, int NS, int... Rs> struct PRun;
template <int SIGN, int M, int NT, int PS, int NS, int R> struct PRun<SIGN, M, NT, PS, NS, R> {
  template <class Store> __device__ __forceinline__ static void run(float4* sm, const float4* tws, const Store& st) {
    pstage<SIGN, M, NT, NS, R>(tws, PSmem<PS>{sm}, st, false);
  }
};
template <int SIGN, int M, int NT, int PS, int NS, int R, int R2, int... Rest>
struct PRun<SIGN, M, NT, PS, NS, R, R2, Rest...> {
  template <class Store> __device__ __forceinline__ static void run(float4* sm, const float4* tws, const Store& st) {
    const PSmem<PS> io{sm};
    pstage<SIGN, M, NT, NS, R>(tws, io, io, true);
    __syncthreads();
    PRun<SIGN, M, NT, PS, NS * R, R2, Rest...>::run(sm, tws + NS * R, st);
  }
};

// Whole pair transform: load -> shared-memory stages -> store (at least two
// stages).  `tws` points at the pair-format stage tables (stages 1..).
template <int SIGN, int M, int NT, int R0, int... Rs> struct PairFFT {
  static_assert(sizeof...(Rs) >= 1, "the pair engine runs two or more stages");
  static constexpr int PS = is_pow2<R0>() ? 4 : 30;
  static constexpr size_t smem_elems() { return PS >= 30 ? (size_t)M : (size_t)M + (M >> PS) + 1; }
  template <class Load, class Store>
  __device__ __forceinline__ static void run(float4* sm, const float4* tws, const Load& ld, const Store& st) {
    pstage<SIGN, M, NT, 1, R0>(tws, ld, PSmem<PS>{sm}, false);
    __syncthreads();
    PRun<SIGN, M, NT, PS, R0, Rs...>::run(sm, tws, st);
  }
};

}  // namespace pr
}  // namespace qtam
