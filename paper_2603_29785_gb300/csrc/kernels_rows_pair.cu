// Row-pair kernels of the QTAM transform pair: each thread block transforms
// two consecutive (segment, plane/row) windows together on the packed FP32x2
// engine of pair_fft.cuh (both rows' values of an element share one 64-bit
// register pair per component, one shared-memory slot and one twiddle read).
//
// Forward (steps a2-a4; Sec. III demodulation, App. A): the first stage
// gathers each row's band from the L2-resident spectrum, applies the
// bisquare window (Eq. gwpy_window_formula, the scale c_k / sqrt(M N) folded
// into it) and places offset d at baseband position d mod M; the length-M
// inverse DFT runs over shared memory; the last stage writes both envelope
// rows with unit stride.
//
// Inverse (steps a5-a6; Eq. qtam_canonical_inverse, App. C synthesis): the
// first stage reads both envelope rows, the length-M forward DFT runs, and
// the last stage keeps each row's band offsets |d| <= h, weights them by
// c_k W'(d) sqrt(N/M) and adds them into the spectrum accumulator
// A[k_c + d] with predicated vector reductions.
//
// The arithmetic is that of the one-row compile-time kernels (same stage
// formula, tables and window evaluation); only its packing differs.
#include "pair_fft.cuh"
#include "rows_common.cuh"

namespace qtam {
namespace {

using pr::C2;

// PairEngine<M, min blocks per SM, radices...>: one row pair per block
template <int M_, int MINB_, int... Rs> struct PairEngine {
  static constexpr int M = M_;
  static constexpr int nrad = sizeof...(Rs);
  static constexpr int radices[nrad] = {Rs...};
  static constexpr int NT = StaticThreads<M_, 0, Rs...>::value;
  static constexpr int MINB = MINB_;
  template <int SIGN> using Fft = pr::PairFFT<SIGN, M_, NT, Rs...>;
  static size_t smem_bytes() { return Fft<1>::smem_elems() * sizeof(float4); }
};

// bisquare weights of both rows at offsets d = (d0, d1): (kw (h^2 - d^2))^2,
// h^2 - d^2 exact in FP32 (h < 4096)
__device__ __forceinline__ float2 pair_weight(float2 d, float2 h2, float2 kw) {
  const float2 u = pmul(psub(h2, pmul(d, d)), kw);
  return pmul(u, u);
}

// First forward stage: element e of each row is offset d = e (e <= dhi) or
// d = e - M (e >= mlo) from its centre bin, zero in between.  x0 / x1 point
// at the rows' centre bins k_c in their segments' spectra.
template <int M> struct PairBand {
  const float2* x0;
  const float2* x1;
  int dhi0, mlo0, dhi1, mlo1;
  float2 h2, kw;
  template <int STEP> __device__ __forceinline__ C2 get_s(int j, int i) const {
    const int e = j + i * STEP;
    const bool lo0 = e <= dhi0, hi0 = e >= mlo0, lo1 = e <= dhi1, hi1 = e >= mlo1;
    const float2* p0 = x0 + j;
    const float2* p1 = x1 + j;
    float2 v0 = make_float2(0.f, 0.f), v1 = v0;
    if (lo0) v0 = p0[i * STEP];
    if (hi0) v0 = p0[i * STEP - M];
    if (lo1) v1 = p1[i * STEP];
    if (hi1) v1 = p1[i * STEP - M];
    const float2 w = pair_weight(make_float2((float)(hi0 ? e - M : e), (float)(hi1 ? e - M : e)), h2, kw);
    return C2{make_float2(v0.x * w.x, v1.x * w.y), make_float2(v0.y * w.x, v1.y * w.y)};
  }
};

// Last forward stage: both envelope rows, unit stride, streaming stores
template <int E> struct PairStoreEnv {
  typename Env<float2, E>::S* y0;
  typename Env<float2, E>::S* y1;
  bool v0, v1;
  template <int STEP> __device__ __forceinline__ void put_s(int base, int i, C2 v) const {
    const int e = base + i * STEP;
    if (v0) stream_store(&y0[e], Env<float2, E>::to(make_float2(v.re.x, v.im.x)));
    if (v1) stream_store(&y1[e], Env<float2, E>::to(make_float2(v.re.y, v.im.y)));
  }
};

// First inverse stage: both envelope rows
template <int E> struct PairLoadEnv {
  const typename Env<float2, E>::S* y0;
  const typename Env<float2, E>::S* y1;
  bool v0, v1;
  template <int STEP> __device__ __forceinline__ C2 get_s(int j, int i) const {
    const int e = j + i * STEP;
    const float2 a = v0 ? Env<float2, E>::from(stream_load(&y0[e])) : make_float2(0.f, 0.f);
    const float2 b = v1 ? Env<float2, E>::from(stream_load(&y1[e])) : make_float2(0.f, 0.f);
    return C2{make_float2(a.x, b.x), make_float2(a.y, b.y)};
  }
};

// Last inverse stage: position e of each row holds offset d = e or e - M;
// in-band offsets are weighted and reduced into A[k_c + d] (A0 / A1 point at
// the rows' centre bins in their segments' accumulators)
template <int M> struct PairAccum {
  float2* A0;
  float2* A1;
  int dhi0, mlo0, dhi1, mlo1;
  float2 h2, kw;
  template <int STEP> __device__ __forceinline__ void put_s(int base, int i, C2 v) const {
    const int e = base + i * STEP;
    const bool lo0 = e <= dhi0, hi0 = e >= mlo0, lo1 = e <= dhi1, hi1 = e >= mlo1;
    const int d0 = hi0 ? e - M : e, d1 = hi1 ? e - M : e;
    const float2 w = pair_weight(make_float2((float)d0, (float)d1), h2, kw);
    add_if(&A0[d0], make_float2(v.re.x * w.x, v.im.x * w.x), lo0 || hi0);
    add_if(&A1[d1], make_float2(v.re.y * w.y, v.im.y * w.y), lo1 || hi1);
  }
};

template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_forward_p(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                     typename Env<float2, E>::S* __restrict__ y, int64_t n_units, const float4* __restrict__ tws) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* sm = reinterpret_cast<float4*>(smraw);
  constexpr int M = Eng::M;
  const int64_t u0 = 2 * (int64_t)blockIdx.x, u1 = u0 + 1;
  const bool v0 = u0 < n_units, v1 = u1 < n_units;
  const int64_t s0 = v0 ? u0 / n_rows : 0, s1 = v1 ? u1 / n_rows : 0;
  const int r0 = v0 ? (int)(u0 - s0 * n_rows) : 0, r1 = v1 ? (int)(u1 - s1 * n_rows) : 0;
  const RowCtx<float, true> c0 = row_ctx<float, true>(rows, r0, M, Nr, v0, false, nullptr);
  const RowCtx<float, true> c1 = row_ctx<float, true>(rows, r1, M, Nr, v1, false, nullptr);
  const PairBand<M> ld{X + s0 * Nr + c0.kc, X + s1 * Nr + c1.kc, c0.dhi, c0.mlo, c1.dhi, c1.mlo,
                       make_float2(c0.h2, c1.h2), make_float2(c0.kw, c1.kw)};
  const PairStoreEnv<E> st{y + (v0 ? u0 : 0) * M, y + (v1 ? u1 : 0) * M, v0, v1};
  Eng::template Fft<+1>::run(sm, tws, ld, st);
}

template <class Eng, int E>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_inverse_p(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel, int n_rows,
                     int64_t Nr, const typename Env<float2, E>::S* __restrict__ y, float2* __restrict__ A,
                     int64_t n_units, const float4* __restrict__ tws) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* sm = reinterpret_cast<float4*>(smraw);
  constexpr int M = Eng::M;
  const int64_t u0 = 2 * (int64_t)blockIdx.x, u1 = u0 + 1;
  const bool v0 = u0 < n_units, v1 = u1 < n_units;
  const int64_t s0 = v0 ? u0 / n_sel : 0, s1 = v1 ? u1 / n_sel : 0;
  const int r0 = v0 ? row_list[u0 - s0 * n_sel] : 0, r1 = v1 ? row_list[u1 - s1 * n_sel] : 0;
  const RowCtx<float, true> c0 = row_ctx<float, true>(rows, r0, M, Nr, v0, true, nullptr);
  const RowCtx<float, true> c1 = row_ctx<float, true>(rows, r1, M, Nr, v1, true, nullptr);
  const PairLoadEnv<E> ld{y + (s0 * n_rows + r0) * M, y + (s1 * n_rows + r1) * M, v0, v1};
  const PairAccum<M> acc{A + s0 * Nr + c0.kc, A + s1 * Nr + c1.kc, c0.dhi, c0.mlo, c1.dhi, c1.mlo,
                         make_float2(c0.h2, c1.h2), make_float2(c0.kw, c1.kw)};
  Eng::template Fft<-1>::run(sm, tws, ld, acc);
}

template <class Eng, int E>
cudaError_t fwd_launch_p(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, void* y, int64_t B,
                         const float2* tw, cudaStream_t st) {
  const int64_t units = B * n_rows;
  const int64_t blocks = (units + 1) / 2;
  const size_t smem = Eng::smem_bytes();
  allow_smem((const void*)k_rows_forward_p<Eng, E>, smem);
  k_rows_forward_p<Eng, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, n_rows, Nr, X, static_cast<typename Env<float2, E>::S*>(y), units, reinterpret_cast<const float4*>(tw));
  return cudaGetLastError();
}
template <class Eng, int E>
cudaError_t inv_launch_p(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                         const void* y, float2* A, int64_t B, const float2* tw, cudaStream_t st) {
  const int64_t units = B * n_sel;
  const int64_t blocks = (units + 1) / 2;
  const size_t smem = Eng::smem_bytes();
  allow_smem((const void*)k_rows_inverse_p<Eng, E>, smem);
  k_rows_inverse_p<Eng, E><<<(unsigned)blocks, Eng::NT, smem, st>>>(
      rows, row_list, n_sel, n_rows, Nr, static_cast<const typename Env<float2, E>::S*>(y), A, units,
      reinterpret_cast<const float4*>(tw));
  return cudaGetLastError();
}

template <class Eng> RowVariant make_variant_pair(const char* name) {
  RowVariant v;
  v.M = Eng::M;
  v.rows_per_block = 2;
  v.threads = Eng::NT;
  v.smem = Eng::smem_bytes();
  v.name = name;
  v.nst = Eng::nrad;
  for (int i = 0; i < Eng::nrad; ++i) v.r[i] = Eng::radices[i];
  v.fwd[ENV_F32] = fwd_launch_p<Eng, ENV_F32>;
  v.fwd[ENV_F64] = nullptr;
  v.fwd[ENV_BF16] = fwd_launch_p<Eng, ENV_BF16>;
  v.fwd[ENV_F16] = fwd_launch_p<Eng, ENV_F16>;
  v.inv[ENV_F32] = inv_launch_p<Eng, ENV_F32>;
  v.inv[ENV_F64] = nullptr;
  v.inv[ENV_BF16] = inv_launch_p<Eng, ENV_BF16>;
  v.inv[ENV_F16] = inv_launch_p<Eng, ENV_F16>;
  v.fwd_tab = nullptr;
  v.inv_tab = nullptr;
  v.fwd_dense = nullptr;
  v.inv_dense = nullptr;
  v.tw_pair = 1;
  return v;
}

#define QTAM_VP(M, MINB, ...) \
  make_variant_pair<PairEngine<M, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " row pair minblk " #MINB)
const RowVariant kPairVariants[] = {
    QTAM_VP(4800, 2, 16, 20, 15),
    QTAM_VP(4800, 2, 16, 15, 20),
};
#undef QTAM_VP

}  // namespace

int pair_row_variant_count() { return (int)(sizeof(kPairVariants) / sizeof(kPairVariants[0])); }
const RowVariant* pair_row_variant(int i) {
  return i >= 0 && i < pair_row_variant_count() ? &kPairVariants[i] : nullptr;
}

}  // namespace qtam
