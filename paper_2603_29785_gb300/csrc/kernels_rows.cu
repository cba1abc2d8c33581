// Per-row kernels of the QTAM transform pair: one thread block per
// (segment, plane/row) window.
//
// Forward (steps a2-a4; Sec. III demodulation, App. A): the first FFT stage
// gathers the row's band straight from the L2-resident spectrum, applies the
// bisquare window (Eq. gwpy_window_formula) on the fly and places offset d at
// baseband position d mod M (the roll by -k_c, crop and symmetric zero-pad);
// the short inverse FFT of length M runs in shared memory; the last stage
// writes the envelope row to HBM with unit stride, scaled by
// c_k / sqrt(M N) = c_k * sqrt(M/N) * (1/M).
//
// Inverse (steps a5-a6; Eq. qtam_canonical_inverse, App. C synthesis): the
// first stage reads the envelope row, the short forward FFT runs in shared
// memory, and the last stage keeps only the band offsets |d| <= h, re-scales
// by sqrt(N/M), weights by c_k W'(d) and adds the result into the spectrum
// accumulator A[k_c + d] with vector atomics (A stays L2-resident).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "qtam_internal.h"

namespace qtam {

namespace {

template <typename T> __device__ __forceinline__ T bisquare(int a, int h, T inv_h2) {
  const T u = (T)(h - a) * (T)(h + a) * inv_h2;   // 1 - (d/h)^2 without cancellation
  return u * u;
}

// envelope storage conversions
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

// band offset of baseband position i (i = d mod M), or a sentinel outside the band
__device__ __forceinline__ int band_offset(int i, int h, int M) {
  return i <= h ? i : (i >= M - h ? i - M : INT32_MIN);
}

template <typename T> struct LoadBand {
  using V = cplx<T>;
  const V* Xs; int kc; int h; int M; int nhalf; T c; T inv_h2;
  __device__ __forceinline__ V get(int, int i) const {
    const int d = band_offset(i, h, M);
    const int f = kc + d;
    if (d == INT32_MIN || f < 0 || f > nhalf) return mk<V>((T)0, (T)0);
    const int a = d < 0 ? -d : d;
    return cscale(Xs[f], c * bisquare<T>(a, h, inv_h2));
  }
};
template <typename V, int E> struct StoreEnvelope {
  typename Env<V, E>::S* ys;
  __device__ __forceinline__ void put(int, int i, V v) const { ys[i] = Env<V, E>::to(v); }
};

template <typename T, int E>
__global__ void __launch_bounds__(kMaxBlock) k_rows_forward(RadixPlan rp, const RowDev<T>* __restrict__ rows, int n_rows,
                                                       int64_t Nr, const cplx<T>* __restrict__ X,
                                                       typename Env<cplx<T>, E>::S* __restrict__ y,
                                                       const cplx<T>* __restrict__ twM) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t bid = blockIdx.x;
  const int64_t seg = bid / n_rows;
  const int row = (int)(bid - seg * n_rows);
  const RowDev<T> rd = rows[row];
  LoadBand<T> ld{X + seg * Nr, rd.kc, rd.h, rp.m, (int)(Nr - 1), rd.c_fwd, rd.inv_h2};
  StoreEnvelope<V, E> stv{y + bid * rp.m};
  block_fft<+1>(rp, 0, sm, twM, 1, ld, stv);
}

template <typename V, int E> struct LoadEnvelope {
  const typename Env<V, E>::S* ys;
  __device__ __forceinline__ V get(int, int i) const { return Env<V, E>::from(ys[i]); }
};

template <typename V> __device__ __forceinline__ void add_to(V* p, V v);
template <> __device__ __forceinline__ void add_to<float2>(float2* p, float2 v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void add_to<double2>(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

template <typename T> struct AccumulateBand {
  using V = cplx<T>;
  V* As; int kc; int h; int M; int nhalf; T c; T inv_h2;
  __device__ __forceinline__ void put(int, int i, V v) const {
    const int d = band_offset(i, h, M);
    const int f = kc + d;
    if (d == INT32_MIN || f < 0 || f > nhalf) return;
    const int a = d < 0 ? -d : d;
    add_to(&As[f], cscale(v, c * bisquare<T>(a, h, inv_h2)));
  }
};

template <typename T, int E>
__global__ void __launch_bounds__(kMaxBlock) k_rows_inverse(RadixPlan rp, const RowDev<T>* __restrict__ rows,
                                                       const int* __restrict__ row_list, int n_sel, int n_rows,
                                                       int64_t Nr, const typename Env<cplx<T>, E>::S* __restrict__ y,
                                                       cplx<T>* __restrict__ A, const cplx<T>* __restrict__ twM) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t bid = blockIdx.x;
  const int64_t seg = bid / n_sel;
  const int row = row_list[bid - seg * n_sel];
  const RowDev<T> rd = rows[row];
  LoadEnvelope<V, E> ld{y + (seg * n_rows + row) * rp.m};
  AccumulateBand<T> stv{A + seg * Nr, rd.kc, rd.h, rp.m, (int)(Nr - 1), rd.c_inv, rd.inv_h2};
  block_fft<-1>(rp, 0, sm, twM, 1, ld, stv);
}

}  // namespace

template <typename T>
cudaError_t launch_rows_forward(const RowCfg& c, const RowDev<T>* rows, int n_rows, int64_t Nr, const cplx<T>* X,
                                void* y, int env, int64_t B, const cplx<T>* twM, cudaStream_t st) {
  const int64_t blocks = B * n_rows;
  if (blocks == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    switch (env) {
      case ENV_BF16:
        allow_smem((const void*)k_rows_forward<T, ENV_BF16>, c.smem);
        k_rows_forward<T, ENV_BF16><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, n_rows, Nr, X, static_cast<__nv_bfloat162*>(y), twM);
        break;
      case ENV_F16:
        allow_smem((const void*)k_rows_forward<T, ENV_F16>, c.smem);
        k_rows_forward<T, ENV_F16><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, n_rows, Nr, X, static_cast<__half2*>(y), twM);
        break;
      default:
        allow_smem((const void*)k_rows_forward<T, ENV_F32>, c.smem);
        k_rows_forward<T, ENV_F32><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, n_rows, Nr, X, static_cast<float2*>(y), twM);
    }
  } else {
    allow_smem((const void*)k_rows_forward<T, ENV_F64>, c.smem);
    k_rows_forward<T, ENV_F64><<<(unsigned)blocks, c.threads, c.smem, st>>>(c.rp, rows, n_rows, Nr, X,
                                                                          static_cast<double2*>(y), twM);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_inverse(const RowCfg& c, const RowDev<T>* rows, const int* row_list, int n_sel, int n_rows,
                                int64_t Nr, const void* y, int env, cplx<T>* A, int64_t B, const cplx<T>* twM,
                                cudaStream_t st) {
  const int64_t blocks = B * n_sel;
  if (blocks == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    switch (env) {
      case ENV_BF16:
        allow_smem((const void*)k_rows_inverse<T, ENV_BF16>, c.smem);
        k_rows_inverse<T, ENV_BF16><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, row_list, n_sel, n_rows, Nr, static_cast<const __nv_bfloat162*>(y), A, twM);
        break;
      case ENV_F16:
        allow_smem((const void*)k_rows_inverse<T, ENV_F16>, c.smem);
        k_rows_inverse<T, ENV_F16><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, row_list, n_sel, n_rows, Nr, static_cast<const __half2*>(y), A, twM);
        break;
      default:
        allow_smem((const void*)k_rows_inverse<T, ENV_F32>, c.smem);
        k_rows_inverse<T, ENV_F32><<<(unsigned)blocks, c.threads, c.smem, st>>>(
            c.rp, rows, row_list, n_sel, n_rows, Nr, static_cast<const float2*>(y), A, twM);
    }
  } else {
    allow_smem((const void*)k_rows_inverse<T, ENV_F64>, c.smem);
    k_rows_inverse<T, ENV_F64><<<(unsigned)blocks, c.threads, c.smem, st>>>(
        c.rp, rows, row_list, n_sel, n_rows, Nr, static_cast<const double2*>(y), A, twM);
  }
  return cudaGetLastError();
}

template cudaError_t launch_rows_forward<float>(const RowCfg&, const RowDev<float>*, int, int64_t, const float2*, void*,
                                                int, int64_t, const float2*, cudaStream_t);
template cudaError_t launch_rows_forward<double>(const RowCfg&, const RowDev<double>*, int, int64_t, const double2*,
                                                 void*, int, int64_t, const double2*, cudaStream_t);
template cudaError_t launch_rows_inverse<float>(const RowCfg&, const RowDev<float>*, const int*, int, int, int64_t,
                                                const void*, int, float2*, int64_t, const float2*, cudaStream_t);
template cudaError_t launch_rows_inverse<double>(const RowCfg&, const RowDev<double>*, const int*, int, int, int64_t,
                                                 const void*, int, double2*, int64_t, const double2*, cudaStream_t);

}  // namespace qtam
