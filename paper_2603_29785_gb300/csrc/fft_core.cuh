// Device FFT engine shared by the long-FFT and row kernels.
//
// A transform of length m = r_0 r_1 ... r_{S-1} (radices 2, 3, 4, 5, 8, 16)
// runs as S Stockham autosort stages inside one thread block.  Stage s with
// span Ns = r_0...r_{s-1} and radix R takes, for each butterfly j < m/R,
//   a_i = in[j + i m/R]                               (i < R)
//   a_i *= w_m^(+-i (j mod Ns) m/(Ns R))               (twiddle table)
//   b   = DFT_R(a)
//   out[(j/Ns) Ns R + (j mod Ns) + i Ns] = b_i
// so the first stage reads its inputs with unit stride across threads and the
// last stage writes its outputs with unit stride: the first stage reads global
// memory through a Load functor and the last writes global memory through a
// Store functor; only the stages in between exchange through shared memory.
// `nb` transforms (a power of two) can run side by side, interleaved as
// element (b, i) -> smem[i*nb + b].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace qtam {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using cplx = typename cvec<T>::type;

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// component-wise arithmetic of the butterflies: for float2 one packed FP32x2
// instruction (sm_100 family `add/sub/mul/fma.f32x2`) does both components;
// double2 stays scalar.  add / sub / mul carry no rounding modifier, so the
// assembler may still contract a multiply feeding an add, as for scalar code.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  float2 r;
  asm("{ .reg .b64 x, y, z; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; add.f32x2 z, x, y; mov.b64 {%0, %1}, z; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  float2 r;
  asm("{ .reg .b64 x, y, z; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; sub.f32x2 z, x, y; mov.b64 {%0, %1}, z; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  float2 r;
  asm("{ .reg .b64 x, y, z; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; mul.f32x2 z, x, y; mov.b64 {%0, %1}, z; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * b + c
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{ .reg .b64 x, y, z, w; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; mov.b64 z, {%6, %7}; "
      "fma.rn.f32x2 w, x, y, z; mov.b64 {%0, %1}, w; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return padd(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return psub(a, b); }
// a k + b, k real
__device__ __forceinline__ float2 vfmak(float2 a, float k, float2 b) { return pfma(a, make_float2(k, k), b); }
__device__ __forceinline__ float2 vscalek(float2 a, float k) { return pmul(a, make_float2(k, k)); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vfmak(double2 a, double k, double2 b) {
  return make_double2(fma(a.x, k, b.x), fma(a.y, k, b.y));
}
__device__ __forceinline__ double2 vscalek(double2 a, double k) { return make_double2(a.x * k, a.y * k); }
// a + S i b (the quarter turn is a swap: scalar)
template <int S, typename V> __device__ __forceinline__ V add_si(V a, V b) {
  return S > 0 ? mk<V>(a.x - b.y, a.y + b.x) : mk<V>(a.x + b.y, a.y - b.x);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
// multiply by S*i (S = +1 or -1)
template <int S, typename V> __device__ __forceinline__ V mul_si(V a) {
  return S > 0 ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// compile-time cos/sin of 2 pi p / q (Taylor series after quadrant reduction)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double ce_sin_q(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 24; ++k) { term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
  return sum;
}
__host__ __device__ constexpr double ce_cos_q(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 24; ++k) { term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
  return sum;
}
// angle 2 pi p/q = quadrant*pi/2 + (pi/2) rem/q
__host__ __device__ constexpr double ce_cos2pi(long p, long q) {
  long a = ((p % q) + q) % q;
  long qd = (4 * a) / q;
  long rem = 4 * a - qd * q;
  double th = 1.5707963267948966192 * (double)rem / (double)q;
  double c = ce_cos_q(th), s = ce_sin_q(th);
  return qd == 0 ? c : qd == 1 ? -s : qd == 2 ? -c : s;
}
__host__ __device__ constexpr double ce_sin2pi(long p, long q) {
  long a = ((p % q) + q) % q;
  long qd = (4 * a) / q;
  long rem = 4 * a - qd * q;
  double th = 1.5707963267948966192 * (double)rem / (double)q;
  double c = ce_cos_q(th), s = ce_sin_q(th);
  return qd == 0 ? s : qd == 1 ? c : qd == 2 ? -s : -c;
}

// ---------------------------------------------------------------------------
// small DFTs in registers: a[0..R) -> DFT_R(a) in natural order, sign S
// (S = -1: exp(-2 pi i jk/R), analysis; S = +1: synthesis, unscaled)
// ---------------------------------------------------------------------------
template <int R, int S> struct Dft;

template <int S> struct Dft<2, S> {
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    const V t = a[0];
    a[0] = vadd(t, a[1]);
    a[1] = vsub(t, a[1]);
  }
};

// y1,2 = m +- i h d with m = a0 - (a1 + a2)/2, d = a1 - a2, h = S sin(2 pi/3)
template <int S> struct Dft<3, S> {
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    using T = decltype(V::x);
    constexpr T h = (T)(S * 0.86602540378443864676);
    const V t = vadd(a[1], a[2]);
    const V d = vsub(a[1], a[2]);
    const V m = vfmak(t, (T)-0.5, a[0]);
    a[0] = vadd(a[0], t);
    a[1] = mk<V>(m.x - h * d.y, m.y + h * d.x);
    a[2] = mk<V>(m.x + h * d.y, m.y - h * d.x);
  }
};

template <int S> struct Dft<4, S> {
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    const V s02 = vadd(a[0], a[2]), d02 = vsub(a[0], a[2]);
    const V s13 = vadd(a[1], a[3]), t = vsub(a[1], a[3]);
    a[0] = vadd(s02, s13);
    a[2] = vsub(s02, s13);
    a[1] = add_si<S>(d02, t);
    a[3] = add_si<-S>(d02, t);
  }
};

// y1,4 = m1 +- i r1, y2,3 = m2 +- i r2 with t1 = a1 + a4, d1 = a1 - a4,
// t2 = a2 + a3, d2 = a2 - a3, m1 = a0 + c1 t1 + c2 t2, m2 = a0 + c2 t1 + c1 t2,
// r1 = s1 d1 + s2 d2, r2 = s2 d1 - s1 d2 (c_k = cos(2 pi k/5), s_k = S sin(2 pi k/5))
template <int S> struct Dft<5, S> {
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    using T = decltype(V::x);
    constexpr T c1 = (T)ce_cos2pi(1, 5), c2 = (T)ce_cos2pi(2, 5);
    constexpr T s1 = (T)(S * ce_sin2pi(1, 5)), s2 = (T)(S * ce_sin2pi(2, 5));
    const V t1 = vadd(a[1], a[4]), d1 = vsub(a[1], a[4]);
    const V t2 = vadd(a[2], a[3]), d2 = vsub(a[2], a[3]);
    const V m1 = vfmak(t2, c2, vfmak(t1, c1, a[0]));
    const V m2 = vfmak(t2, c1, vfmak(t1, c2, a[0]));
    const V r1 = vfmak(d1, s1, vscalek(d2, s2));
    const V r2 = vfmak(d1, s2, vscalek(d2, -s1));
    a[0] = vadd(vadd(a[0], t1), t2);
    a[1] = add_si<1>(m1, r1);
    a[4] = add_si<-1>(m1, r1);
    a[2] = add_si<1>(m2, r2);
    a[3] = add_si<-1>(m2, r2);
  }
};

// composite R = R1 * R2: index j = R2 j1 + j2, output k = k1 + R1 k2
//   b[j2][k1] = DFT_R1 over j1 of a[R2 j1 + j2];  b *= w_R^(S j2 k1);
//   y[k1 + R1 k2] = DFT_R2 over j2 of b[j2][k1]
// The inner twiddles are compile-time constants (immediate operands); the
// quarter turns among them reduce to swaps and negations.
template <int E, int R, int S, typename V> __device__ __forceinline__ void twiddle_const(V& x) {
  using T = decltype(V::x);
  constexpr int e = E % R;
  if constexpr (e == 0) {
  } else if constexpr (4 * e == R) {           // w = S i
    x = mul_si<S>(x);
  } else if constexpr (2 * e == R) {           // w = -1
    x = mk<V>(-x.x, -x.y);
  } else if constexpr (4 * e == 3 * R) {       // w = -S i
    x = mul_si<-S>(x);
  } else {
    constexpr T c = (T)ce_cos2pi(e, R);
    constexpr T sn = (T)(S * ce_sin2pi(e, R));
    x = mk<V>(x.x * c - x.y * sn, x.x * sn + x.y * c);
  }
}

template <int R1, int R2, int S> struct DftComposite {
  static constexpr int R = R1 * R2;
  template <int J2, int... K1, typename V>
  __device__ __forceinline__ static void twiddle_col(V* col, std::integer_sequence<int, K1...>) {
    (twiddle_const<J2 * K1, R, S>(col[K1]), ...);
  }
  template <int... J2, typename V>
  __device__ __forceinline__ static void columns(V* a, V* b, std::integer_sequence<int, J2...>) {
    (column<J2>(a, b), ...);
  }
  template <int J2, typename V> __device__ __forceinline__ static void column(V* a, V* b) {
    V col[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) col[j1] = a[R2 * j1 + J2];
    Dft<R1, S>::run(col);
    twiddle_col<J2>(col, std::make_integer_sequence<int, R1>{});
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) b[J2 * R1 + k1] = col[k1];
  }
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    V b[R];
    columns(a, b, std::make_integer_sequence<int, R2>{});
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      V row[R2];
#pragma unroll
      for (int j2 = 0; j2 < R2; ++j2) row[j2] = b[j2 * R1 + k1];
      Dft<R2, S>::run(row);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = row[k2];
    }
  }
};
// Prime-factor (Good-Thomas) DFT for R = R1 R2 with gcd(R1, R2) = 1: the
// input index n = (R2 n1 + R1 n2) mod R and output index
// k = (R2 (R2^-1 mod R1) k1 + R1 (R1^-1 mod R2) k2) mod R turn the DFT into
// R2 DFTs of length R1 followed by R1 DFTs of length R2 with no twiddles.
__host__ __device__ constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 1;
}
template <int R1, int R2, int S> struct DftPFA {
  static constexpr int R = R1 * R2;
  static constexpr int E1 = R2 * inv_mod(R2 % R1, R1);
  static constexpr int E2 = R1 * inv_mod(R1 % R2, R2);
  template <typename V> __device__ __forceinline__ static void run(V* a) {
    V b[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      V col[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) col[n1] = a[(R2 * n1 + R1 * n2) % R];
      Dft<R1, S>::run(col);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) b[k1 * R2 + n2] = col[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      V row[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) row[n2] = b[k1 * R2 + n2];
      Dft<R2, S>::run(row);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[(E1 * k1 + E2 * k2) % R] = row[k2];
    }
  }
};

template <int S> struct Dft<6, S> : DftPFA<2, 3, S> {};
template <int S> struct Dft<8, S> : DftComposite<2, 4, S> {};
template <int S> struct Dft<9, S> : DftComposite<3, 3, S> {};
template <int S> struct Dft<10, S> : DftPFA<2, 5, S> {};
template <int S> struct Dft<12, S> : DftPFA<4, 3, S> {};
template <int S> struct Dft<15, S> : DftPFA<3, 5, S> {};
template <int S> struct Dft<16, S> : DftComposite<4, 4, S> {};
template <int S> struct Dft<18, S> : DftPFA<2, 9, S> {};
template <int S> struct Dft<20, S> : DftPFA<4, 5, S> {};
template <int S> struct Dft<24, S> : DftPFA<8, 3, S> {};
template <int S> struct Dft<25, S> : DftComposite<5, 5, S> {};
template <int S> struct Dft<27, S> : DftComposite<3, 9, S> {};
template <int S> struct Dft<32, S> : DftComposite<4, 8, S> {};
template <int S> struct Dft<48, S> : DftPFA<16, 3, S> {};
template <int S> struct Dft<64, S> : DftComposite<8, 8, S> {};
template <int S> struct Dft<60, S> : DftPFA<4, 15, S> {};
template <int S> struct Dft<75, S> : DftPFA<3, 25, S> {};
template <int S> struct Dft<80, S> : DftPFA<16, 5, S> {};

// items held in registers per thread for one stage of radix R (~16 complex)
__host__ __device__ constexpr int ipt_for(int R) {
  return R >= 16 ? 1 : R >= 8 ? 2 : R >= 5 ? 3 : R == 4 ? 4 : R == 3 ? 5 : 8;
}

constexpr int kMaxStages = 12;

// Runtime description of one transform length: radices in stage order.
struct RadixPlan {
  int m;
  int nst;
  int r[kMaxStages];
  int pad_shift;  // smem index e -> e + (e >> pad_shift); 30 = no padding
};

template <typename V> struct SmemIO {
  V* sm;
  int nbs;
  int pad_shift;
  __device__ __forceinline__ int addr(int b, int i) const {
    int e = (i << nbs) + b;
    return e + (e >> pad_shift);
  }
  __device__ __forceinline__ V get(int b, int i) const { return sm[addr(b, i)]; }
  __device__ __forceinline__ void put(int b, int i, V v) const { sm[addr(b, i)] = v; }
};

// One Stockham stage over nb = 2^nbs interleaved transforms of length m.
// tw[t * twstride] = exp(-2 pi i t / m).  When src and dst are the same
// shared buffer (inplace) every thread holds all its items in registers
// across a barrier.
template <int R, int S, typename V, class Src, class Dst>
__device__ __forceinline__ void stockham_stage(int m, int Ns, int nbs, const V* __restrict__ tw, int twstride,
                                               const Src& src, const Dst& dst, bool inplace) {
  constexpr int IPT = ipt_for(R);
  const int mR = m / R;
  const int items = mR << nbs;
  const int bmask = (1 << nbs) - 1;
  const int tstep = (m / (Ns * R)) * twstride;
  V a[IPT][R];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int w = threadIdx.x + q * blockDim.x;
    if (w < items) {
      const int b = w & bmask, j = w >> nbs;
#pragma unroll
      for (int i = 0; i < R; ++i) a[q][i] = src.get(b, j + i * mR);
      if (Ns > 1) {
        const int k = j % Ns;
#pragma unroll
        for (int i = 1; i < R; ++i) {
          V t = __ldg(&tw[i * k * tstep]);
          if (S > 0) t.y = -t.y;
          a[q][i] = cmul(a[q][i], t);
        }
      }
      Dft<R, S>::run(a[q]);
    }
  }
  if (inplace) __syncthreads();
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int w = threadIdx.x + q * blockDim.x;
    if (w < items) {
      const int b = w & bmask, j = w >> nbs;
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int i = 0; i < R; ++i) dst.put(b, base + i * Ns, a[q][i]);
    }
  }
}

template <int S, typename V, class Src, class Dst>
__device__ __forceinline__ void stage_dispatch(int R, int m, int Ns, int nbs, const V* tw, int twstride,
                                               const Src& src, const Dst& dst, bool inplace) {
  switch (R) {
    case 16: stockham_stage<16, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
    case 8: stockham_stage<8, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
    case 5: stockham_stage<5, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
    case 4: stockham_stage<4, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
    case 3: stockham_stage<3, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
    default: stockham_stage<2, S>(m, Ns, nbs, tw, twstride, src, dst, inplace); break;
  }
}

// Whole transform: load -> [smem stages] -> store.  The caller's block size
// must cover every stage (blockDim.x * ipt_for(r_s) >= (m / r_s) << nbs).
// Ends without a trailing barrier; a caller that reuses `sm` must sync first.
template <int S, typename V, class Load, class Store>
__device__ __forceinline__ void block_fft(const RadixPlan& rp, int nbs, V* sm, const V* tw, int twstride,
                                          const Load& load, const Store& store) {
  if (rp.nst == 1) {
    stage_dispatch<S>(rp.r[0], rp.m, 1, nbs, tw, twstride, load, store, false);
    return;
  }
  SmemIO<V> io{sm, nbs, rp.pad_shift};
  stage_dispatch<S>(rp.r[0], rp.m, 1, nbs, tw, twstride, load, io, false);
  __syncthreads();
  int Ns = rp.r[0];
  for (int s = 1; s + 1 < rp.nst; ++s) {
    stage_dispatch<S>(rp.r[s], rp.m, Ns, nbs, tw, twstride, io, io, true);
    __syncthreads();
    Ns *= rp.r[s];
  }
  stage_dispatch<S>(rp.r[rp.nst - 1], rp.m, Ns, nbs, tw, twstride, io, store, false);
}

}  // namespace qtam
