// Shared templates of the per-row kernels (included by kernels_rows.cu and
// kernels_rows_stream.cu, each translation unit instantiating its own
// kernels): envelope storage conversions, the per-row context (band limits
// and window weight), band loads and envelope stores, the band accumulation,
// the FFT engines (runtime mixed-radix and compile-time), and the forward /
// inverse row bodies.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_static.cuh"
#include "qtam_internal.h"

namespace qtam {
namespace {

// envelope storage conversions; envelopes cross HBM exactly once, so they
// are stored and loaded with the streaming (evict-first) cache policy and
// leave the L2 to the spectra and accumulators
template <typename S> __device__ __forceinline__ void stream_store(S* p, S v) {
  if constexpr (sizeof(S) == 8) {
    __stcs(reinterpret_cast<float2*>(p), *reinterpret_cast<float2*>(&v));
  } else if constexpr (sizeof(S) == 16) {
    __stcs(reinterpret_cast<double2*>(p), *reinterpret_cast<double2*>(&v));
  } else {
    __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<unsigned int*>(&v));
  }
}
template <typename S> __device__ __forceinline__ S stream_load(const S* p) {
  S v;
  if constexpr (sizeof(S) == 8) {
    *reinterpret_cast<float2*>(&v) = __ldcs(reinterpret_cast<const float2*>(p));
  } else if constexpr (sizeof(S) == 16) {
    *reinterpret_cast<double2*>(&v) = __ldcs(reinterpret_cast<const double2*>(p));
  } else {
    *reinterpret_cast<unsigned int*>(&v) = __ldcs(reinterpret_cast<const unsigned int*>(p));
  }
  return v;
}

template <typename V, int E> struct Env;
template <> struct Env<float2, ENV_F32> {
  using S = float2;
  __device__ __forceinline__ static S to(float2 v) { return v; }
  __device__ __forceinline__ static float2 from(S v) { return v; }
};
template <> struct Env<float2, ENV_BF16> {
  using S = __nv_bfloat162;
  __device__ __forceinline__ static S to(float2 v) { return __float22bfloat162_rn(v); }
  __device__ __forceinline__ static float2 from(S v) { return __bfloat1622float2(v); }
};
template <> struct Env<float2, ENV_F16> {
  using S = __half2;
  __device__ __forceinline__ static S to(float2 v) { return __float22half2_rn(v); }
  __device__ __forceinline__ static float2 from(S v) { return __half22float2(v); }
};
template <> struct Env<double2, ENV_F64> {
  using S = double2;
  __device__ __forceinline__ static S to(double2 v) { return v; }
  __device__ __forceinline__ static double2 from(S v) { return v; }
};

// Per-thread view of the row it works on.  Every call a thread makes uses
// the same interleave slot b = threadIdx.x mod 2^NBS (block sizes are whole
// warps), so the row descriptor is read once, not per element.
//
// The row's usable offsets are d in [dlo, dhi] = [-h, h] cut to bins
// 0..N/2; baseband position i holds d = i for i <= dhi and d = i - M for
// i >= M + dlo.  The weight is c W'(d) = (kw (h^2 - d^2))^2 with
// kw = sqrt(c)/h^2; with FEXACT (h < 4096) h^2 - d^2 is formed exactly in
// floating point, otherwise as the integer product (h - |d|)(h + |d|).  The
// other App. A windows (runtime engine only) read W'(|d|) from a per-plan
// table instead; positions outside the band read W'(h) and are multiplied
// by a zero bin.
template <typename T, bool FEXACT> struct RowCtx {
  int kc, h, M, dhi, mlo;
  T kw, h2;
  const T* wt;   // runtime engine only: W'(0..h) table of a non-bisquare window, or null
  T cw;          // its normalisation (c_fwd or c_inv)
  T ew;          // runtime engine only: weight where the window vanishes (dense mode), else 0
  __device__ __forceinline__ void locate(int i, bool& in, int& d) const {
    const bool lo = i <= dhi;
    in = lo || i >= mlo;
    d = lo ? i : i - M;
  }
  __device__ __forceinline__ T weight(int d) const {
    T u;
    if constexpr (FEXACT) {
      const T df = (T)d;
      u = (h2 - df * df) * kw;
    } else {
      const int a = d < 0 ? -d : d;
      if (wt) return a <= h ? cw * wt[a] : ew;
      if (a >= h) return ew;
      u = (T)(h - a) * (T)(h + a) * kw;
    }
    return u * u;
  }
};

template <typename T, bool FEXACT> struct LoadBand {
  using V = cplx<T>;
  const V* Xs;
  RowCtx<T, FEXACT> r;
  __device__ __forceinline__ V get(int, int i) const {
    bool in;
    int d;
    r.locate(i, in, d);
    const T w = r.weight(d);
    V x = mk<V>((T)0, (T)0);
    if (in) x = Xs[r.kc + d];
    return cscale(x, w);
  }
  // element e = j + s*STEP of a strided stage-0 read: the bin is k_c + e
  // (low band) or k_c + e - M (high band); both addresses are a per-item base
  // plus a compile-time offset
  template <int STEP> __device__ __forceinline__ V get_s(int, int j, int s) const {
    const int e = j + s * STEP;
    const bool lo = e <= r.dhi;
    const bool hi = e >= r.mlo;
    const V* pl = Xs + (r.kc + j);
    const V* ph = pl - r.M;
    V x = mk<V>((T)0, (T)0);
    if (lo) x = pl[s * STEP];
    if (hi) x = ph[s * STEP];
    return cscale(x, r.weight(hi ? e - r.M : e));
  }
};
template <typename V, int E> struct StoreEnvelope {
  typename Env<V, E>::S* ys;
  bool valid;
  __device__ __forceinline__ void put(int, int i, V v) const {
    if (valid) stream_store(&ys[i], Env<V, E>::to(v));
  }
};
template <typename V, int E> struct LoadEnvelope {
  const typename Env<V, E>::S* ys;
  bool valid;
  __device__ __forceinline__ V get(int, int i) const {
    return valid ? Env<V, E>::from(stream_load(&ys[i])) : mk<V>(0, 0);
  }
};

// v e^{+2 pi i (kcm i mod M) / M} (or its conjugate) from the plan's table
// twM[t] = e^{-2 pi i t / M}; kcm = k_c mod M, so kcm i < M^2 fits 32 bits
template <typename V>
__device__ __forceinline__ V carrier_rot(V v, const V* __restrict__ twM, int kcm, int i, int M, bool conj) {
  const V w = twM[(int)((unsigned)(kcm * i) % (unsigned)M)];
  const auto c = w.x, s = conj ? w.y : -w.y;
  return mk<V>(v.x * c - v.y * s, v.x * s + v.y * c);
}

// runtime-engine envelope store / load with the optional carrier (dense mode)
template <typename V, int E> struct StoreEnvelopeRT {
  typename Env<V, E>::S* ys;
  bool valid;
  int remod, kcm, M;
  const V* twM;
  __device__ __forceinline__ void put(int, int i, V v) const {
    if (remod) v = carrier_rot(v, twM, kcm, i, M, false);
    if (valid) stream_store(&ys[i], Env<V, E>::to(v));
  }
};
template <typename V, int E> struct LoadEnvelopeRT {
  const typename Env<V, E>::S* ys;
  bool valid;
  int remod, kcm, M;
  const V* twM;
  __device__ __forceinline__ V get(int, int i) const {
    V v = valid ? Env<V, E>::from(stream_load(&ys[i])) : mk<V>(0, 0);
    return remod ? carrier_rot(v, twM, kcm, i, M, true) : v;
  }
};

// *p += v when `on` (relaxed, device scope); the float2 form is one
// predicated vector reduction, so out-of-band positions cost no branch (the
// accumulator is not read in the same kernel: no ordering with other accesses)
__device__ __forceinline__ void add_if(float2* p, float2 v, bool on) {
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %3, 0; @q red.global.add.v2.f32 [%0], {%1, %2}; }"
               :: "l"(p), "f"(v.x), "f"(v.y), "r"((int)on));
}
__device__ __forceinline__ void add_if(double2* p, double2 v, bool on) {
  if (on) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
  }
}

// PRED selects the predicated vector reduction; otherwise a branch around
// the atomic (fewer live registers when the last stage holds 25 values)
template <typename T, bool FEXACT, bool PRED> struct AccumulateBand {
  using V = cplx<T>;
  V* As;
  RowCtx<T, FEXACT> r;
  __device__ __forceinline__ void put(int, int i, V v) const {
    bool in;
    int d;
    r.locate(i, in, d);
    const T w = r.weight(d);
    if constexpr (PRED) {
      add_if(&As[r.kc + d], cscale(v, w), in);
    } else if (in) {
      add_if(&As[r.kc + d], cscale(v, w), true);
    }
  }
};

// runtime-engine inverse store: accumulate v * weight(d), or (single-tile
// inverse) write v * scale / weight(d); in dense mode every bin is written once
template <typename T> struct AccumulateBandRT {
  using V = cplx<T>;
  V* As;
  RowCtx<T, false> r;
  int divide;
  T scale;
  __device__ __forceinline__ void put(int, int i, V v) const {
    bool in;
    int d;
    r.locate(i, in, d);
    const T w = r.weight(d);
    if (divide) {
      if (in) As[r.kc + d] = cscale(v, scale / w);
    } else if (in) {
      add_if(&As[r.kc + d], cscale(v, w), true);
    }
  }
};

// ---- FFT engines ----------------------------------------------------------
struct GenericEngine {
  RadixPlan rp;
  static constexpr int NBS = 0;
  static constexpr bool FEXACT = false;
  static constexpr bool PRED_RED = false;
  __device__ __forceinline__ int m() const { return rp.m; }
  template <int S, typename V, class L, class St>
  __device__ __forceinline__ void run(V* sm, const V* tw, const L& ld, const St& st) const {
    block_fft<S>(rp, 0, sm, tw, 1, ld, st);
  }
};

template <int M_, int NBS_, int MINB_, int... Rs> struct StaticEngine {
  static constexpr int M = M_;
  static constexpr int nrad = sizeof...(Rs);
  static constexpr int radices[nrad] = {Rs...};
  static constexpr int NBS = NBS_;
  static constexpr int NT = StaticThreads<M_, NBS_, Rs...>::value;
  static constexpr int MINB = MINB_;
  static_assert(M_ <= 8192, "static variants need h < 4096 for the exact float window");
  static constexpr bool FEXACT = true;
  static constexpr bool PRED_RED = radices[nrad - 1] < 25;
  __device__ __forceinline__ int m() const { return M; }
  template <int S, typename V, class L, class St>
  __device__ __forceinline__ void run(V* sm, const V* tws, const L& ld, const St& st) const {
    StaticFFT<S, M, NT, NBS, Rs...>::run(sm, tws, ld, st);
  }
  static size_t smem_bytes(size_t elem) { return StaticFFT<1, M, NT, NBS, Rs...>::smem_elems() * elem; }
};

// The same engine with an explicit block size NT_: a stage with more
// butterfly items than threads runs in rounds, so the block can be sized to
// the stages' common item count instead of the widest stage's (at M = 2400,
// 16·10·15 has 150 / 240 / 160 items: 160 threads run the 10-point stage in
// two rounds and the others in one).
template <int NT_, int M_, int NBS_, int MINB_, int... Rs> struct ThreadsEngine : StaticEngine<M_, NBS_, MINB_, Rs...> {
  static constexpr int NT = NT_;
  template <int S, typename V, class L, class St>
  __device__ __forceinline__ void run(V* sm, const V* tws, const L& ld, const St& st) const {
    StaticFFT<S, M_, NT_, NBS_, Rs...>::run(sm, tws, ld, st);
  }
};

template <typename T, bool FEXACT>
__device__ __forceinline__ RowCtx<T, FEXACT> row_ctx(const RowDev<T>* rows, int row, int M, int64_t Nr, bool valid,
                                                     bool inv, const T* wtab) {
  RowCtx<T, FEXACT> r;
  r.M = M;
  r.wt = nullptr;
  r.cw = (T)0;
  r.ew = (T)0;
  if (valid) {
    const RowDev<T> rd = rows[row];
    const int nhalf = (int)(Nr - 1);
    r.kc = rd.kc;
    r.h = rd.h;
    r.kw = inv ? rd.kw_inv : rd.kw_fwd;
    r.h2 = (T)rd.h * (T)rd.h;
    if (wtab && rd.woff >= 0) {
      r.wt = wtab + rd.woff;
      r.cw = inv ? rd.c_inv : rd.c_fwd;
    }
    r.ew = inv ? rd.eps_inv : rd.eps_fwd;
    r.dhi = min(rd.hb, nhalf - rd.kc);    // may be < 0: no non-negative offset
    r.mlo = M + max(-rd.hb, -rd.kc);      // may be > M - 1: no negative offset
    if (r.dhi < -1) r.dhi = -1;
  } else {
    r.kc = 0; r.h = 1; r.kw = 0; r.h2 = 1;
    r.dhi = -1;
    r.mlo = M;                            // nothing in band
  }
  return r;
}

template <class Eng, typename T, int E>
__device__ __forceinline__ void rows_forward_body(const Eng& eng, const RowDev<T>* __restrict__ rows, int n_rows,
                                                  int64_t Nr, const cplx<T>* __restrict__ X,
                                                  typename Env<cplx<T>, E>::S* __restrict__ y, int64_t n_units,
                                                  const cplx<T>* __restrict__ twM, const T* __restrict__ wtab) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int M = eng.m();
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_rows : 0;
  const int row = valid ? (int)(unit - seg * n_rows) : 0;
  LoadBand<T, Eng::FEXACT> ld{X + seg * Nr, row_ctx<T, Eng::FEXACT>(rows, row, M, Nr, valid, false, wtab)};
  StoreEnvelope<V, E> stv{y + (valid ? unit : 0) * M, valid};
  eng.template run<+1>(sm, twM, ld, stv);
}

template <class Eng, typename T, int E>
__device__ __forceinline__ void rows_inverse_body(const Eng& eng, const RowDev<T>* __restrict__ rows,
                                                  const int* __restrict__ row_list, int n_sel, int n_rows, int64_t Nr,
                                                  const typename Env<cplx<T>, E>::S* __restrict__ y,
                                                  cplx<T>* __restrict__ A, int64_t n_units,
                                                  const cplx<T>* __restrict__ twM, const T* __restrict__ wtab) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int M = eng.m();
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_sel : 0;
  const int row = valid ? row_list[unit - seg * n_sel] : 0;
  LoadEnvelope<V, E> ld{y + (seg * n_rows + row) * M, valid};
  AccumulateBand<T, Eng::FEXACT, Eng::PRED_RED> stv{A + seg * Nr,
                                                    row_ctx<T, Eng::FEXACT>(rows, row, M, Nr, valid, true, wtab)};
  eng.template run<-1>(sm, twM, ld, stv);
}

// The runtime-engine kernels carry the dense-mode options (carrier, division)
template <typename T, int E>
__global__ void __launch_bounds__(kMaxBlock, 1)
    k_rows_forward(GenericEngine eng, const RowDev<T>* __restrict__ rows, int n_rows, int64_t Nr,
                   const cplx<T>* __restrict__ X, typename Env<cplx<T>, E>::S* __restrict__ y, int64_t n_units,
                   const cplx<T>* __restrict__ twM, const T* __restrict__ wtab, DenseArgs<T> da) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int M = eng.m();
  const int64_t unit = blockIdx.x;
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_rows : 0;
  const int row = valid ? (int)(unit - seg * n_rows) : 0;
  const RowCtx<T, false> rc = row_ctx<T, false>(rows, row, M, Nr, valid, false, wtab);
  LoadBand<T, false> ld{X + seg * Nr, rc};
  StoreEnvelopeRT<V, E> stv{y + (valid ? unit : 0) * M, valid, da.remod, rc.kc % M, M, twM};
  eng.template run<+1>(sm, twM, ld, stv);
}
template <typename T, int E>
__global__ void __launch_bounds__(kMaxBlock, 1)
    k_rows_inverse(GenericEngine eng, const RowDev<T>* __restrict__ rows, const int* __restrict__ row_list, int n_sel,
                   int n_rows, int64_t Nr, const typename Env<cplx<T>, E>::S* __restrict__ y, cplx<T>* __restrict__ A,
                   int64_t n_units, const cplx<T>* __restrict__ twM, const T* __restrict__ wtab, DenseArgs<T> da) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int M = eng.m();
  const int64_t unit = blockIdx.x;
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_sel : 0;
  const int row = valid ? row_list[unit - seg * n_sel] : 0;
  const RowCtx<T, false> rc = row_ctx<T, false>(rows, row, M, Nr, valid, true, wtab);
  LoadEnvelopeRT<V, E> ld{y + (seg * n_rows + row) * M, valid, da.remod, rc.kc % M, M, twM};
  AccumulateBandRT<T> stv{A + seg * Nr, rc, da.divide, da.scale};
  eng.template run<-1>(sm, twM, ld, stv);
}

template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_forward_s(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                     typename Env<float2, E>::S* __restrict__ y, int64_t n_units, const float2* __restrict__ twM) {
  rows_forward_body<Eng, float, E>(Eng(), rows, n_rows, Nr, X, y, n_units, twM, nullptr);
}
template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_inverse_s(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel, int n_rows,
                     int64_t Nr, const typename Env<float2, E>::S* __restrict__ y, float2* __restrict__ A,
                     int64_t n_units, const float2* __restrict__ twM) {
  rows_inverse_body<Eng, float, E>(Eng(), rows, row_list, n_sel, n_rows, Nr, y, A, n_units, twM, nullptr);
}

// The same compile-time FFT with the weight read from the plan's window
// table (the integer-product path of RowCtx): the bisquare kernels above keep
// their exact-float formula and instruction stream untouched.
template <class Eng> struct TabEngine : Eng {
  static constexpr bool FEXACT = false;
};
template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_forward_st(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                      typename Env<float2, E>::S* __restrict__ y, int64_t n_units, const float2* __restrict__ twM,
                      const float* __restrict__ wtab) {
  rows_forward_body<TabEngine<Eng>, float, E>(TabEngine<Eng>(), rows, n_rows, Nr, X, y, n_units, twM, wtab);
}
template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_inverse_st(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel, int n_rows,
                      int64_t Nr, const typename Env<float2, E>::S* __restrict__ y, float2* __restrict__ A,
                      int64_t n_units, const float2* __restrict__ twM, const float* __restrict__ wtab) {
  rows_inverse_body<TabEngine<Eng>, float, E>(TabEngine<Eng>(), rows, row_list, n_sel, n_rows, Nr, y, A, n_units, twM,
                                              wtab);
}


// Dense tiles with the carrier, where the band spans all N/2 + 1 bins and
// M > N/2: the remodulated envelope Y e^{+2 pi i k_c n / M} is the inverse
// DFT of the weighted spectrum placed at its own bins (position i holds bin
// i, the offset from the centre is i - k_c), so neither the roll to
// baseband nor a carrier multiply is needed; the inverse reads bin i's
// analysis value at position i the same way.
template <typename T> struct LoadSpectrumAbs {
  using V = cplx<T>;
  const V* Xs;
  RowCtx<T, false> r;
  int nhalf;
  __device__ __forceinline__ V get(int, int i) const {
    V x = mk<V>((T)0, (T)0);
    if (i <= nhalf) x = Xs[i];
    return cscale(x, r.weight(i - r.kc));
  }
};
template <typename T, bool PRED> struct AccumulateAbs {
  using V = cplx<T>;
  V* As;
  RowCtx<T, false> r;
  int nhalf;
  __device__ __forceinline__ void put(int, int i, V v) const {
    const T w = r.weight(i - r.kc);
    if constexpr (PRED) {
      add_if(&As[i], cscale(v, w), i <= nhalf);
    } else if (i <= nhalf) {
      add_if(&As[i], cscale(v, w), true);
    }
  }
};

// Dense mode on a compile-time FFT (FP32 arithmetic, envelopes stored as
// EnvKind E): the weights of the
// integer-product / table path (c eps wherever the window vanishes, the band
// spanning the one-sided spectrum through hb).  ABS: tiles with the carrier
// and the floor, bins at their own positions (above); otherwise the band at
// baseband with the carrier e^{+2 pi i k_c n / M} from the plan's M-point
// table on store (its conjugate on load) when remod is set.  tws holds the
// variant's stage twiddles, twM the plan's M-point table.
template <class Eng, bool ABS, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_forward_sd(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                      typename Env<float2, E>::S* __restrict__ y, int64_t n_units, const float2* __restrict__ tws,
                      const float* __restrict__ wtab, const float2* __restrict__ twM, int remod) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  constexpr int M = Eng::M;
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_rows : 0;
  const int row = valid ? (int)(unit - seg * n_rows) : 0;
  const RowCtx<float, false> rc = row_ctx<float, false>(rows, row, M, Nr, valid, false, wtab);
  if constexpr (ABS) {
    LoadSpectrumAbs<float> ld{X + seg * Nr, rc, valid ? (int)(Nr - 1) : -1};
    StoreEnvelope<float2, E> stv{y + (valid ? unit : 0) * M, valid};
    Eng().template run<+1>(sm, tws, ld, stv);
  } else {
    LoadBand<float, false> ld{X + seg * Nr, rc};
    StoreEnvelopeRT<float2, E> stv{y + (valid ? unit : 0) * M, valid, remod, rc.kc % M, M, twM};
    Eng().template run<+1>(sm, tws, ld, stv);
  }
}
template <class Eng, bool ABS, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_inverse_sd(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel, int n_rows,
                      int64_t Nr, const typename Env<float2, E>::S* __restrict__ y, float2* __restrict__ A,
                      int64_t n_units,
                      const float2* __restrict__ tws, const float* __restrict__ wtab, const float2* __restrict__ twM,
                      int remod) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  constexpr int M = Eng::M;
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t seg = valid ? unit / n_sel : 0;
  const int row = valid ? row_list[unit - seg * n_sel] : 0;
  const RowCtx<float, false> rc = row_ctx<float, false>(rows, row, M, Nr, valid, true, wtab);
  if constexpr (ABS) {
    LoadEnvelope<float2, E> ld{y + (seg * n_rows + row) * M, valid};
    AccumulateAbs<float, Eng::PRED_RED> acc{A + seg * Nr, rc, valid ? (int)(Nr - 1) : -1};
    Eng().template run<-1>(sm, tws, ld, acc);
  } else {
    LoadEnvelopeRT<float2, E> ld{y + (seg * n_rows + row) * M, valid, remod, rc.kc % M, M, twM};
    AccumulateBand<float, false, Eng::PRED_RED> acc{A + seg * Nr, rc};
    Eng().template run<-1>(sm, tws, ld, acc);
  }
}

// ---- registry entries of compile-time variants (FP32 compute) ----------------
template <class Eng, int E>
cudaError_t fwd_launch(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                       const float2* twM, cudaStream_t st) {
  const int64_t units = B * n_rows;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_forward_s<Eng, E>, smem);
  k_rows_forward_s<Eng, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, n_rows, Nr, X, static_cast<typename Env<float2, E>::S*>(y), units, twM);
  return cudaGetLastError();
}
template <class Eng, int E>
cudaError_t inv_launch(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                       const void* y, float2* A, int64_t B, const float2* twM, cudaStream_t st) {
  const int64_t units = B * n_sel;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_inverse_s<Eng, E>, smem);
  k_rows_inverse_s<Eng, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, row_list, n_sel, n_rows, Nr, static_cast<const typename Env<float2, E>::S*>(y), A, units, twM);
  return cudaGetLastError();
}

template <class Eng>
cudaError_t fwd_launch_tab(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                           const float2* twM, cudaStream_t st, const float* wtab) {
  const int64_t units = B * n_rows;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_forward_st<Eng, ENV_F32>, smem);
  k_rows_forward_st<Eng, ENV_F32><<<(unsigned)blocks, Eng::NT, smem, st>>>(rows, n_rows, Nr, X,
                                                                            static_cast<float2*>(y), units, twM, wtab);
  return cudaGetLastError();
}
template <class Eng>
cudaError_t inv_launch_tab(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                           const void* y, float2* A, int64_t B, const float2* twM, cudaStream_t st,
                           const float* wtab) {
  const int64_t units = B * n_sel;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_inverse_st<Eng, ENV_F32>, smem);
  k_rows_inverse_st<Eng, ENV_F32><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, row_list, n_sel, n_rows, Nr, static_cast<const float2*>(y), A, units, twM, wtab);
  return cudaGetLastError();
}

// mode: 0 baseband tiles, 1 baseband tiles with the carrier, 2 tiles spanning
// the spectrum with the carrier (bins at their own positions); env: EnvKind
// of the stored envelopes (F32, BF16 or F16)
template <class Eng, bool ABS, int E>
cudaError_t fwd_launch_dense_k(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                               const float2* tws, cudaStream_t st, const float* wtab, const float2* twM, int remod) {
  const int64_t units = B * n_rows;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_forward_sd<Eng, ABS, E>, smem);
  k_rows_forward_sd<Eng, ABS, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, n_rows, Nr, X, static_cast<typename Env<float2, E>::S*>(y), units, tws, wtab, twM, remod);
  return cudaGetLastError();
}
template <class Eng, int E>
cudaError_t fwd_launch_dense_e(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                               const float2* tws, cudaStream_t st, const float* wtab, const float2* twM, int mode) {
  return mode == 2 ? fwd_launch_dense_k<Eng, true, E>(rows, n_rows, Nr, X, y, B, tws, st, wtab, twM, 0)
                   : fwd_launch_dense_k<Eng, false, E>(rows, n_rows, Nr, X, y, B, tws, st, wtab, twM, mode);
}
template <class Eng>
cudaError_t fwd_launch_dense(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                             const float2* tws, cudaStream_t st, const float* wtab, const float2* twM, int mode,
                             int env) {
  switch (env) {
    case ENV_BF16: return fwd_launch_dense_e<Eng, ENV_BF16>(rows, n_rows, Nr, X, y, B, tws, st, wtab, twM, mode);
    case ENV_F16: return fwd_launch_dense_e<Eng, ENV_F16>(rows, n_rows, Nr, X, y, B, tws, st, wtab, twM, mode);
    default: return fwd_launch_dense_e<Eng, ENV_F32>(rows, n_rows, Nr, X, y, B, tws, st, wtab, twM, mode);
  }
}
template <class Eng, bool ABS, int E>
cudaError_t inv_launch_dense_k(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                               const void* y, float2* A, int64_t B, const float2* tws, cudaStream_t st,
                               const float* wtab, const float2* twM, int remod) {
  const int64_t units = B * n_sel;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_inverse_sd<Eng, ABS, E>, smem);
  k_rows_inverse_sd<Eng, ABS, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, row_list, n_sel, n_rows, Nr, static_cast<const typename Env<float2, E>::S*>(y), A, units, tws, wtab, twM,
      remod);
  return cudaGetLastError();
}
template <class Eng, int E>
cudaError_t inv_launch_dense_e(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                               const void* y, float2* A, int64_t B, const float2* tws, cudaStream_t st,
                               const float* wtab, const float2* twM, int mode) {
  return mode == 2
             ? inv_launch_dense_k<Eng, true, E>(rows, row_list, n_sel, n_rows, Nr, y, A, B, tws, st, wtab, twM, 0)
             : inv_launch_dense_k<Eng, false, E>(rows, row_list, n_sel, n_rows, Nr, y, A, B, tws, st, wtab, twM, mode);
}
template <class Eng>
cudaError_t inv_launch_dense(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                             const void* y, float2* A, int64_t B, const float2* tws, cudaStream_t st,
                             const float* wtab, const float2* twM, int mode, int env) {
  switch (env) {
    case ENV_BF16:
      return inv_launch_dense_e<Eng, ENV_BF16>(rows, row_list, n_sel, n_rows, Nr, y, A, B, tws, st, wtab, twM, mode);
    case ENV_F16:
      return inv_launch_dense_e<Eng, ENV_F16>(rows, row_list, n_sel, n_rows, Nr, y, A, B, tws, st, wtab, twM, mode);
    default:
      return inv_launch_dense_e<Eng, ENV_F32>(rows, row_list, n_sel, n_rows, Nr, y, A, B, tws, st, wtab, twM, mode);
  }
}

template <class Eng> RowVariant make_variant(const char* name) {
  RowVariant v;
  v.M = Eng::M;
  v.rows_per_block = 1 << Eng::NBS;
  v.threads = Eng::NT;
  v.smem = Eng::smem_bytes(sizeof(float2));
  v.name = name;
  v.nst = Eng::nrad;
  for (int i = 0; i < Eng::nrad; ++i) v.r[i] = Eng::radices[i];
  v.fwd[ENV_F32] = fwd_launch<Eng, ENV_F32>;
  v.fwd[ENV_F64] = nullptr;
  v.fwd[ENV_BF16] = fwd_launch<Eng, ENV_BF16>;
  v.fwd[ENV_F16] = fwd_launch<Eng, ENV_F16>;
  v.inv[ENV_F32] = inv_launch<Eng, ENV_F32>;
  v.inv[ENV_F64] = nullptr;
  v.inv[ENV_BF16] = inv_launch<Eng, ENV_BF16>;
  v.inv[ENV_F16] = inv_launch<Eng, ENV_F16>;
  v.fwd_tab = nullptr;
  v.inv_tab = nullptr;
  v.fwd_dense = nullptr;
  v.inv_dense = nullptr;
  return v;
}
template <class Eng> RowVariant make_variant_tab(const char* name) {
  RowVariant v = make_variant<Eng>(name);
  v.fwd_tab = fwd_launch_tab<Eng>;
  v.inv_tab = inv_launch_tab<Eng>;
  return v;
}
// the table variant plus the dense-mode kernels
template <class Eng> RowVariant make_variant_dense(const char* name) {
  RowVariant v = make_variant_tab<Eng>(name);
  v.fwd_dense = fwd_launch_dense<Eng>;
  v.inv_dense = inv_launch_dense<Eng>;
  return v;
}

}  // namespace
}  // namespace qtam
