// Long real FFT of each segment (step a1) and its inverse with the dual-frame
// normaliser fused in (step a7).
//
// A real segment x of N = 2n samples is read as n complex values
// z[m] = x[2m] + i x[2m+1] and transformed as an n = n1 * n2 four-step FFT:
//   column pass:  U[k1][m2] = w_n^(m2 k1) sum_m1 z[m1 n2 + m2] w_n1^(m1 k1)
//   row pass:     Z[k1 + n1 k2] = sum_m2 U[k1][m2] w_n2^(m2 k2)
// followed by the real-to-complex untangle
//   X[k] = (Z[k] + Z*[n-k]) / 2 - (i/2) w_N^k (Z[k] - Z*[n-k]),  k = 0..n
// which gives the one-sided spectrum X[f] = sum_n x[n] exp(-2 pi i f n / N)
// of App. C.  The inverse runs the same steps backwards: the untangle's
// inverse (with X_hat = A / P read through the plan's 1/P table and the DC
// and Nyquist bins taken real) feeds the row pass, then the column pass
// writes x_hat[2m] + i x_hat[2m+1] directly.
#include "fft_static.cuh"
#include "qtam_internal.h"

namespace qtam {

namespace {

// FFT engines for the four-step passes: the runtime engine takes any
// 2^a 3^b 5^c length and interleave count; the static engines fix both.
struct GenLong {
  RadixPlan rp;
  int nbs;
  static constexpr int NT = kMaxBlock;
  static constexpr int MINB = 1;
  __device__ __forceinline__ int m() const { return rp.m; }
  __device__ __forceinline__ int nb_shift() const { return nbs; }
  template <int S, typename V, class L, class St>
  __device__ __forceinline__ void run(V* sm, const V* tw, int twstride, const L& ld, const St& st) const {
    block_fft<S>(rp, nbs, sm, tw, twstride, ld, st);
  }
};
// NT_ = 0: the block spans the widest stage's items; otherwise NT_ threads and
// wider stages run in rounds
template <int M_, int NBS_, int NT_, int... Rs> struct StatLong {
  static constexpr int nrad = sizeof...(Rs);
  static constexpr int radices[nrad] = {Rs...};
  static constexpr int NT = NT_ > 0 ? NT_ : StaticThreads<M_, NBS_, Rs...>::value;
  static constexpr int MINB = NT >= 512 ? 1 : 512 / NT;   // at least 512 threads per SM
  __device__ __forceinline__ int m() const { return M_; }
  __device__ __forceinline__ int nb_shift() const { return NBS_; }
  template <int S, typename V, class L, class St>
  __device__ __forceinline__ void run(V* sm, const V* tws, int, const L& ld, const St& st) const {
    StaticFFT<S, M_, NT, NBS_, Rs...>::run(sm, tws, ld, st);
  }
  static size_t smem_bytes(size_t elem) { return StaticFFT<1, M_, NT, NBS_, Rs...>::smem_elems() * elem; }
};

template <typename V> struct LoadColumns {
  const V* zs; int n2; int c0;
  __device__ __forceinline__ V get(int b, int m1) const { return zs[(int64_t)m1 * n2 + c0 + b]; }
};
// tw4[k1 * n2 + c] = w_n^(c k1): the four-step twiddles in the layout of U,
// so a warp's loads are as contiguous as its stores.
template <typename V> struct StoreColumnsTwiddled {
  V* Us; const V* tw4; int n2; int c0;
  __device__ __forceinline__ void put(int b, int k1, V v) const {
    const int64_t e = (int64_t)k1 * n2 + c0 + b;
    Us[e] = cmul(v, __ldg(&tw4[e]));
  }
};
template <typename V> struct LoadRows {
  const V* Us; int n2; int r0;
  __device__ __forceinline__ V get(int b, int m2) const { return Us[(int64_t)(r0 + b) * n2 + m2]; }
};
template <typename V> struct StoreRowsTransposed {
  V* Zs; int n1; int r0;
  __device__ __forceinline__ void put(int b, int k2, V v) const { Zs[(int64_t)k2 * n1 + r0 + b] = v; }
};

template <class Eng, typename T>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB) k_col_forward(Eng eng, int n, int n2, const cplx<T>* __restrict__ z,
                                                          cplx<T>* __restrict__ U, const cplx<T>* __restrict__ tw4,
                                                          const cplx<T>* __restrict__ ftw) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int c0 = blockIdx.x << eng.nb_shift();
  LoadColumns<V> ld{z + seg * n, n2, c0};
  StoreColumnsTwiddled<V> stv{U + seg * n, tw4, n2, c0};
  eng.template run<-1>(sm, ftw, n / eng.m(), ld, stv);
}

template <class Eng, typename T>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB) k_row_forward(Eng eng, int n, int n1, const cplx<T>* __restrict__ U,
                                                          cplx<T>* __restrict__ Z, const cplx<T>* __restrict__ ftw) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int r0 = blockIdx.x << eng.nb_shift();
  LoadRows<V> ld{U + seg * n, eng.m(), r0};
  StoreRowsTransposed<V> stv{Z + seg * n, n1, r0};
  eng.template run<-1>(sm, ftw, n / eng.m(), ld, stv);
}

// w_N^k for k in [0, n]: table holds k <= n/2; w_N^(n-k) = -conj(w_N^k)
template <typename V> __device__ __forceinline__ V wN(const V* twN, int n, int k) {
  if (k <= (n >> 1)) return __ldg(&twN[k]);
  V t = __ldg(&twN[n - k]);
  return mk<V>(-t.x, t.y);
}

constexpr int kUntanglePairs = 4;   // (k, n-k) pairs per thread, for memory-level parallelism

template <typename T>
__global__ void k_untangle_forward(int n, const cplx<T>* __restrict__ Z, cplx<T>* __restrict__ X,
                                   const cplx<T>* __restrict__ twN) {
  using V = cplx<T>;
  const int64_t seg = blockIdx.y;
  const V* Zs = Z + seg * n;
  V* Xs = X + seg * (int64_t)(n + 1);
  const T half = (T)0.5;
  const int base = blockIdx.x * blockDim.x * kUntanglePairs + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kUntanglePairs; ++u) {
    const int k = base + u * blockDim.x;
    if (k > (n >> 1)) break;
    const int kk = n - k;                     // partner bin, in [n/2, n]
    const V zk = Zs[k];
    const V zm = Zs[kk == n ? 0 : kk];
    {
      const V a = zk, b = cconj(zm);
      const V s = a + b, d = a - b;
      const V t = cmul(__ldg(&twN[k]), d);    // w^k (a - b)
      Xs[k] = mk<V>(half * (s.x + t.y), half * (s.y - t.x));   // s/2 - (i/2) t
    }
    if (kk != k) {
      const V a = zm, b = cconj(zk);
      const V s = a + b, d = a - b;
      const V t = cmul(wN(twN, n, kk), d);
      Xs[kk] = mk<V>(half * (s.x + t.y), half * (s.y - t.x));
    }
  }
}

// Inverse untangle with the dual-frame normaliser: for the pair (k, n-k),
//   Xh = A * (1/P) (DC and Nyquist taken real),
//   Zi[k] = scale (E[k] + i O[k]),  E = (Xh[k] + conj Xh[n-k]) / 2,
//   O = (Xh[k] - conj Xh[n-k]) / 2 * w_N^(-k),
// written in natural order; coalesced reads and writes, pairs per thread.
template <typename T>
__device__ __forceinline__ cplx<T> zi_value(cplx<T> xk, cplx<T> xm, cplx<T> wk, T hs) {
  using V = cplx<T>;
  const V e = xk + cconj(xm);
  const V o = cmul(xk - cconj(xm), cconj(wk));
  return mk<V>(hs * (e.x - o.y), hs * (e.y + o.x));    // scale/2 (e + i o)
}

template <typename T>
__global__ void k_untangle_inverse(int n, const cplx<T>* __restrict__ A, const T* __restrict__ invP,
                                   cplx<T>* __restrict__ Zi, const cplx<T>* __restrict__ twN, T scale) {
  using V = cplx<T>;
  const int64_t seg = blockIdx.y;
  const V* As = A + seg * (int64_t)(n + 1);
  V* Zs = Zi + seg * n;
  const T hs = (T)0.5 * scale;
  const int base = blockIdx.x * blockDim.x * kUntanglePairs + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kUntanglePairs; ++u) {
    const int k = base + u * blockDim.x;
    if (k > (n >> 1)) break;
    const int kk = n - k;                     // in [n/2, n]
    V xk = cscale(As[k], __ldg(&invP[k]));
    V xm = cscale(As[kk], __ldg(&invP[kk]));
    if (k == 0) xk.y = (T)0;
    if (kk == n) xm.y = (T)0;
    const V wk = __ldg(&twN[k]);
    Zs[k] = zi_value<T>(xk, xm, wk, hs);
    if (kk != k && kk != n) Zs[kk] = zi_value<T>(xm, xk, mk<V>(-wk.x, wk.y), hs);   // w^(n-k) = -conj(w^k)
  }
}

// row pass of the inverse: rows k1 of Zi, read with stride n1
template <typename V> struct LoadRowsTransposed {
  const V* Zs; int n1; int r0;
  __device__ __forceinline__ V get(int b, int k2) const { return Zs[(int64_t)k2 * n1 + r0 + b]; }
};
template <typename V> struct StoreRowsTwiddledConj {
  V* Vs; const V* tw4; int n2; int r0;
  __device__ __forceinline__ void put(int b, int m2, V v) const {
    const int64_t e = (int64_t)(r0 + b) * n2 + m2;
    Vs[e] = cmul(v, cconj(__ldg(&tw4[e])));
  }
};
template <typename V> struct StoreColumns {
  V* xs; int n2; int c0;
  __device__ __forceinline__ void put(int b, int m1, V v) const { xs[(int64_t)m1 * n2 + c0 + b] = v; }
};

template <class Eng, typename T>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB) k_row_inverse(Eng eng, int n, int n1, const cplx<T>* __restrict__ Zi,
                                                          cplx<T>* __restrict__ Vb, const cplx<T>* __restrict__ tw4,
                                                          const cplx<T>* __restrict__ ftw) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int r0 = blockIdx.x << eng.nb_shift();
  LoadRowsTransposed<V> ld{Zi + seg * n, n1, r0};
  StoreRowsTwiddledConj<V> stv{Vb + seg * n, tw4, eng.m(), r0};
  eng.template run<+1>(sm, ftw, n / eng.m(), ld, stv);
}

template <class Eng, typename T>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB) k_col_inverse(Eng eng, int n, int n2, const cplx<T>* __restrict__ Vb,
                                                          cplx<T>* __restrict__ xout, const cplx<T>* __restrict__ ftw) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int c0 = blockIdx.x << eng.nb_shift();
  LoadColumns<V> ld{Vb + seg * n, n2, c0};
  StoreColumns<V> stv{xout + seg * n, n2, c0};
  eng.template run<+1>(sm, ftw, n / eng.m(), ld, stv);
}

constexpr int64_t kMaxGridY = 65535;

// Static engines for power-of-two sub-lengths (FP32): column passes
// interleave 16 columns, row passes 4 rows.  The 512-point row pass runs on
// 64 threads (its 16-point stage in two rounds) rather than 128, of which
// the 32-point stage kept half idle: the 64 s spectrum 0.0897 -> 0.0856 ms,
// the synthesis 0.0948 -> 0.0938 ms per 64 segments.
#define QTAM_LONG_CASES(X, NBS)                \
  X(32, NBS, 0, 8, 4)                          \
  X(64, NBS, 0, 16, 4)                         \
  X(128, NBS, 0, 16, 8)                        \
  X(256, NBS, 0, 16, 16)                       \
  X(512, NBS, (NBS == 2 ? 64 : 0), 16, 32)     \
  X(1024, NBS, 0, 32, 32)

template <class Eng, class K, class... Args>
void launch_pass(K kernel, const Eng& eng, size_t smem, dim3 g, cudaStream_t st, Args... args) {
  allow_smem((const void*)kernel, smem);
  kernel<<<g, Eng::NT, smem, st>>>(eng, args...);
}

// Call f(engine, smem) with the static engine for (m, nbs) when one exists
// (FP32), else with the runtime engine.
#define QTAM_CASE(M, NBS, ...)                                     \
  case M: {                                                        \
    using E = StatLong<M, NBS, __VA_ARGS__>;                       \
    f(E(), E::smem_bytes(sizeof(float2)), (const cplx<T>*)stw);    \
    return;                                                        \
  }

// Call f(engine, smem bytes, engine twiddles): the static engine for
// (m, nbs) when one exists (FP32) and its tables were built, else the
// runtime engine with the plan's length-n table.
template <typename T, class F>
void with_engine(const RadixPlan& rp, int nbs, int static_nbs, size_t gen_smem, const void* stw,
                 const cplx<T>* twn, F&& f) {
  if constexpr (sizeof(T) == 4) {
    if (stw && nbs == static_nbs && static_nbs == 4) {
      switch (rp.m) { QTAM_LONG_CASES(QTAM_CASE, 4) default: break; }
    } else if (stw && nbs == static_nbs && static_nbs == 2) {
      switch (rp.m) { QTAM_LONG_CASES(QTAM_CASE, 2) default: break; }
    }
  }
  f(GenLong{rp, nbs}, gen_smem, twn);
}
#undef QTAM_CASE

#define QTAM_RADICES(M, NBS, ...)                   \
  case M: {                                         \
    using E = StatLong<M, NBS, __VA_ARGS__>;        \
    *nst = E::nrad;                                 \
    for (int i = 0; i < E::nrad; ++i) r[i] = E::radices[i]; \
    return true;                                    \
  }

}  // namespace

bool long_static_radices(int m, int nbs, int* r, int* nst) {
  if (nbs == 4) {
    switch (m) { QTAM_LONG_CASES(QTAM_RADICES, 4) default: break; }
  } else if (nbs == 2) {
    switch (m) { QTAM_LONG_CASES(QTAM_RADICES, 2) default: break; }
  }
  return false;
}
#undef QTAM_RADICES

template <typename T>
cudaError_t launch_spectrum(const LongCfg& c, const cplx<T>* z, cplx<T>* U, cplx<T>* Z, cplx<T>* X, int64_t B,
                            const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st) {
  const cplx<T>* tw4 = static_cast<const cplx<T>*>(c.tw4);
  for (int64_t s0 = 0; s0 < B; s0 += kMaxGridY) {
    const int64_t nb = (B - s0) < kMaxGridY ? (B - s0) : kMaxGridY;
    const int64_t off = s0 * c.n;
    with_engine<T>(c.rp1, c.col_nbs, 4, c.col_smem, c.stw_col, twn, [&](auto eng, size_t smem, const cplx<T>* ftw) {
      using E = decltype(eng);
      dim3 g(c.n2 >> c.col_nbs, (unsigned)nb);
      launch_pass(k_col_forward<E, T>, eng, smem, g, st, c.n, c.n2, z + off, U + off, tw4, ftw);
    });
    with_engine<T>(c.rp2, c.row_nbs, 2, c.row_smem, c.stw_row, twn, [&](auto eng, size_t smem, const cplx<T>* ftw) {
      using E = decltype(eng);
      dim3 g(c.n1 >> c.row_nbs, (unsigned)nb);
      launch_pass(k_row_forward<E, T>, eng, smem, g, st, c.n, c.n1, (const cplx<T>*)(U + off), Z + off, ftw);
    });
    dim3 g3((unsigned)((c.n / 2 + 1 + 256 * kUntanglePairs - 1) / (256 * kUntanglePairs)), (unsigned)nb);
    k_untangle_forward<T><<<g3, 256, 0, st>>>(c.n, Z + off, X + s0 * (int64_t)(c.n + 1), twN);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_synthesis(const LongCfg& c, const cplx<T>* A, const T* invP, cplx<T>* Zi, cplx<T>* Vb,
                             cplx<T>* xout, int64_t B, const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st) {
  const cplx<T>* tw4 = static_cast<const cplx<T>*>(c.tw4);
  for (int64_t s0 = 0; s0 < B; s0 += kMaxGridY) {
    const int64_t nb = (B - s0) < kMaxGridY ? (B - s0) : kMaxGridY;
    const int64_t off = s0 * c.n;
    dim3 g0((unsigned)((c.n / 2 + 1 + 256 * kUntanglePairs - 1) / (256 * kUntanglePairs)), (unsigned)nb);
    k_untangle_inverse<T><<<g0, 256, 0, st>>>(c.n, A + s0 * (int64_t)(c.n + 1), invP, Zi + off, twN,
                                              (T)1 / (T)c.n);
    with_engine<T>(c.rp2, c.row_nbs, 2, c.row_smem, c.stw_row, twn, [&](auto eng, size_t smem, const cplx<T>* ftw) {
      using E = decltype(eng);
      dim3 g(c.n1 >> c.row_nbs, (unsigned)nb);
      launch_pass(k_row_inverse<E, T>, eng, smem, g, st, c.n, c.n1, (const cplx<T>*)(Zi + off), Vb + off, tw4, ftw);
    });
    with_engine<T>(c.rp1, c.col_nbs, 4, c.col_smem, c.stw_col, twn, [&](auto eng, size_t smem, const cplx<T>* ftw) {
      using E = decltype(eng);
      dim3 g(c.n2 >> c.col_nbs, (unsigned)nb);
      launch_pass(k_col_inverse<E, T>, eng, smem, g, st, c.n, c.n2, (const cplx<T>*)(Vb + off), xout + off, ftw);
    });
  }
  return cudaGetLastError();
}

template cudaError_t launch_spectrum<float>(const LongCfg&, const float2*, float2*, float2*, float2*, int64_t,
                                            const float2*, const float2*, cudaStream_t);
template cudaError_t launch_spectrum<double>(const LongCfg&, const double2*, double2*, double2*, double2*, int64_t,
                                             const double2*, const double2*, cudaStream_t);
template cudaError_t launch_synthesis<float>(const LongCfg&, const float2*, const float*, float2*, float2*, float2*,
                                             int64_t, const float2*, const float2*, cudaStream_t);
template cudaError_t launch_synthesis<double>(const LongCfg&, const double2*, const double*, double2*, double2*,
                                              double2*, int64_t, const double2*, const double2*, cudaStream_t);

}  // namespace qtam
