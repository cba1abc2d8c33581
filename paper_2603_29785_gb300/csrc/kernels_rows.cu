// Per-row kernels of the QTAM transform pair: each thread block transforms
// 2^NBS (segment, plane/row) windows.
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
//
// The FFT itself is either the runtime engine (any 2^a 3^b 5^c length) or a
// compile-time engine registered below for the lengths the workloads use.
#include "rows_common.cuh"

namespace qtam {
namespace {

// StaticEngine<M, log2 rows per block, min blocks per SM, radices...>; the
// first variant listed for a length is the default before tuning.
// QTAM_VT: also built for window tables (the first such variant of a length
// is the default of non-bisquare plans).
#define QTAM_V(M, NBS, MINB, ...) \
  make_variant<StaticEngine<M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB)
#define QTAM_VT(M, NBS, MINB, ...) \
  make_variant_tab<StaticEngine<M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB)
const RowVariant kVariants[] = {
    QTAM_VT(4800, 0, 4, 16, 20, 15),
    QTAM_V(4800, 0, 3, 16, 20, 15),
    QTAM_V(4800, 0, 3, 16, 15, 20),
    QTAM_V(4800, 0, 2, 16, 20, 15),
    QTAM_V(4800, 0, 3, 8, 6, 10, 10),
    QTAM_V(4800, 0, 2, 16, 12, 25),
    QTAM_VT(2400, 0, 3, 16, 10, 15),
    QTAM_V(2400, 1, 2, 16, 10, 15),
    QTAM_V(2400, 0, 4, 16, 10, 15),
    QTAM_VT(1200, 1, 2, 16, 15, 5),
    QTAM_V(1200, 2, 2, 16, 3, 25),
    QTAM_VT(600, 3, 2, 8, 3, 25),
    QTAM_V(600, 2, 2, 8, 15, 5),
    QTAM_VT(500, 3, 2, 4, 5, 25),
    QTAM_VT(300, 3, 2, 12, 25),
    QTAM_V(300, 4, 2, 4, 3, 25),
    QTAM_VT(150, 4, 2, 6, 25),
    QTAM_VT(75, 5, 2, 3, 25),
    QTAM_VT(8192, 0, 1, 16, 16, 32),
    QTAM_V(8192, 0, 1, 32, 16, 16),
    QTAM_V(8192, 0, 1, 16, 32, 16),
};
#undef QTAM_V
#undef QTAM_VT

template <typename V, int E>
__global__ void k_scale_rows(typename Env<V, E>::S* __restrict__ y, const float* __restrict__ gain, int64_t n_rows,
                             int M) {
  // one block-stride loop per row; rows with gain 1 are left untouched
  for (int64_t r = blockIdx.x; r < n_rows; r += gridDim.x) {
    const float g = gain[r];
    if (g == 1.0f) continue;
    typename Env<V, E>::S* row = y + r * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      V v = Env<V, E>::from(row[i]);
      v.x *= g;
      v.y *= g;
      row[i] = Env<V, E>::to(v);
    }
  }
}

// Per (segment, plane) pair: energy = sum |Y|^2 and peak = max |Y|^2 over
// the K*M envelope values (App. A optimal-plane selection).  Each pair is
// split over kMetricChunks blocks so the read of Y runs at HBM speed; FP32
// envelopes are squared in FP32 and summed in FP32 partials of at most 8
// terms (relative error <= ~5e-7) before FP64 accumulation (the FP64 pipe is
// slow on this part); FP64 envelopes stay in FP64.  Blocks combine with a
// double atomicAdd and an integer atomicMax on the (non-negative) float bits;
// both outputs are zeroed by the launcher first.
constexpr int kMetricChunks = 64;

template <typename V, int E>
__global__ void __launch_bounds__(256) k_plane_metrics(const typename Env<V, E>::S* __restrict__ y, int64_t per_plane,
                                                       double* __restrict__ energy, float* __restrict__ peak) {
  using R = decltype(V().x);
  const int64_t pair = blockIdx.x / kMetricChunks;
  const int part = (int)(blockIdx.x - pair * kMetricChunks);
  const int64_t len = (per_plane + kMetricChunks - 1) / kMetricChunks;
  const int64_t b0 = part * len, b1 = min(per_plane, b0 + len);
  const typename Env<V, E>::S* p = y + pair * per_plane;
  double e = 0.0;
  float mx = 0.0f;
  for (int64_t i0 = b0 + threadIdx.x; i0 < b1; i0 += 8 * (int64_t)blockDim.x) {
    R es = (R)0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      if (i < b1) {
        const V v = Env<V, E>::from(stream_load(&p[i]));
        const R a2 = v.x * v.x + v.y * v.y;
        es += a2;
        mx = fmaxf(mx, (float)a2);
      }
    }
    e += (double)es;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double se[8];
  __shared__ float sm[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    se[w] = e;
    sm[w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double et = 0.0;
    float mt = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      et += se[k];
      mt = fmaxf(mt, sm[k]);
    }
    atomicAdd(&energy[pair], et);
    atomicMax(reinterpret_cast<int*>(&peak[pair]), __float_as_int(mt));
  }
}

}  // namespace

cudaError_t launch_plane_metrics(const void* y, int env, int64_t pairs, int64_t per_plane, double* energy, float* peak,
                                 cudaStream_t st) {
  if (pairs == 0) return cudaSuccess;
  cudaError_t e0 = cudaMemsetAsync(energy, 0, (size_t)pairs * sizeof(double), st);
  if (e0 == cudaSuccess) e0 = cudaMemsetAsync(peak, 0, (size_t)pairs * sizeof(float), st);
  if (e0 != cudaSuccess) return e0;
  const unsigned grid = (unsigned)(pairs * kMetricChunks);
  switch (env) {
    case ENV_F64:
      k_plane_metrics<double2, ENV_F64><<<grid, 256, 0, st>>>(static_cast<const double2*>(y), per_plane, energy, peak);
      break;
    case ENV_BF16:
      k_plane_metrics<float2, ENV_BF16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat162*>(y), per_plane, energy, peak);
      break;
    case ENV_F16:
      k_plane_metrics<float2, ENV_F16><<<grid, 256, 0, st>>>(static_cast<const __half2*>(y), per_plane, energy, peak);
      break;
    default:
      k_plane_metrics<float2, ENV_F32><<<grid, 256, 0, st>>>(static_cast<const float2*>(y), per_plane, energy, peak);
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_rows(void* y, int env, const float* gain, int64_t n_rows, int M, cudaStream_t st) {
  if (n_rows == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)(n_rows < 65535 ? n_rows : 65535);
  switch (env) {
    case ENV_F64: k_scale_rows<double2, ENV_F64><<<blocks, 256, 0, st>>>(static_cast<double2*>(y), gain, n_rows, M); break;
    case ENV_BF16:
      k_scale_rows<float2, ENV_BF16><<<blocks, 256, 0, st>>>(static_cast<__nv_bfloat162*>(y), gain, n_rows, M);
      break;
    case ENV_F16: k_scale_rows<float2, ENV_F16><<<blocks, 256, 0, st>>>(static_cast<__half2*>(y), gain, n_rows, M); break;
    default: k_scale_rows<float2, ENV_F32><<<blocks, 256, 0, st>>>(static_cast<float2*>(y), gain, n_rows, M);
  }
  return cudaGetLastError();
}

// the dense-mode variants follow the ones registered here
// and the row-pair variants follow those
constexpr int kMainVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
int row_variant_count() {
  return kMainVariants + dense_row_variant_count() + pair_row_variant_count() + tuned_row_variant_count();
}
const RowVariant* row_variant(int i) {
  if (i < 0) return nullptr;
  if (i < kMainVariants) return &kVariants[i];
  i -= kMainVariants;
  if (i < dense_row_variant_count()) return dense_row_variant(i);
  i -= dense_row_variant_count();
  if (i < pair_row_variant_count()) return pair_row_variant(i);
  return tuned_row_variant(i - pair_row_variant_count());
}

template <typename T>
cudaError_t launch_rows_forward(const RowCfg& c, const RowDev<T>* rows, int n_rows, int64_t Nr, const cplx<T>* X,
                                void* y, int env, int64_t B, const cplx<T>* twM, cudaStream_t st, const T* wtab) {
  const int64_t units = B * n_rows;
  if (units == 0) return cudaSuccess;
  DenseArgs<T> da;
  da.remod = c.remod;
  if constexpr (sizeof(T) == 4) {
    if (const RowVariant* v = row_variant(c.variant)) {
      const float2* stw = static_cast<const float2*>(c.stw);
      if (c.dense) {
        if (v->fwd_dense)
          return v->fwd_dense(rows, n_rows, Nr, X, y, B, stw, st, wtab, twM, c.dense == 2 ? 2 : c.remod, env);
      } else {
        if (!wtab) return v->fwd[env](rows, n_rows, Nr, X, y, B, stw, st);
        if (env == ENV_F32 && v->fwd_tab) return v->fwd_tab(rows, n_rows, Nr, X, y, B, stw, st, wtab);
      }
    }
  }
  GenericEngine eng{c.rp};
  const unsigned blocks = (unsigned)units;
  if constexpr (sizeof(T) == 4) {
    switch (env) {
      case ENV_BF16:
        allow_smem((const void*)k_rows_forward<T, ENV_BF16>, c.smem);
        k_rows_forward<T, ENV_BF16><<<blocks, c.threads, c.smem, st>>>(eng, rows, n_rows, Nr, X,
                                                                       static_cast<__nv_bfloat162*>(y), units, twM, wtab, da);
        break;
      case ENV_F16:
        allow_smem((const void*)k_rows_forward<T, ENV_F16>, c.smem);
        k_rows_forward<T, ENV_F16><<<blocks, c.threads, c.smem, st>>>(eng, rows, n_rows, Nr, X,
                                                                      static_cast<__half2*>(y), units, twM, wtab, da);
        break;
      default:
        allow_smem((const void*)k_rows_forward<T, ENV_F32>, c.smem);
        k_rows_forward<T, ENV_F32><<<blocks, c.threads, c.smem, st>>>(eng, rows, n_rows, Nr, X,
                                                                      static_cast<float2*>(y), units, twM, wtab, da);
    }
  } else {
    allow_smem((const void*)k_rows_forward<T, ENV_F64>, c.smem);
    k_rows_forward<T, ENV_F64><<<blocks, c.threads, c.smem, st>>>(eng, rows, n_rows, Nr, X,
                                                                  static_cast<double2*>(y), units, twM, wtab, da);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_inverse(const RowCfg& c, const RowDev<T>* rows, const int* row_list, int n_sel, int n_rows,
                                int64_t Nr, const void* y, int env, cplx<T>* A, int64_t B, const cplx<T>* twM,
                                cudaStream_t st, const T* wtab, DenseArgs<T> da) {
  const int64_t units = B * n_sel;
  da.remod = c.remod;
  if (units == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (const RowVariant* v = da.divide ? nullptr : row_variant(c.variant)) {
      const float2* stw = static_cast<const float2*>(c.stw);
      if (c.dense) {
        if (v->inv_dense)
          return v->inv_dense(rows, row_list, n_sel, n_rows, Nr, y, A, B, stw, st, wtab, twM, c.dense == 2 ? 2 : c.remod,
                              env);
      } else {
        if (!wtab) return v->inv[env](rows, row_list, n_sel, n_rows, Nr, y, A, B, stw, st);
        if (env == ENV_F32 && v->inv_tab) return v->inv_tab(rows, row_list, n_sel, n_rows, Nr, y, A, B, stw, st, wtab);
      }
    }
  }
  GenericEngine eng{c.rp};
  const unsigned blocks = (unsigned)units;
  if constexpr (sizeof(T) == 4) {
    switch (env) {
      case ENV_BF16:
        allow_smem((const void*)k_rows_inverse<T, ENV_BF16>, c.smem);
        k_rows_inverse<T, ENV_BF16><<<blocks, c.threads, c.smem, st>>>(
            eng, rows, row_list, n_sel, n_rows, Nr, static_cast<const __nv_bfloat162*>(y), A, units, twM, wtab, da);
        break;
      case ENV_F16:
        allow_smem((const void*)k_rows_inverse<T, ENV_F16>, c.smem);
        k_rows_inverse<T, ENV_F16><<<blocks, c.threads, c.smem, st>>>(
            eng, rows, row_list, n_sel, n_rows, Nr, static_cast<const __half2*>(y), A, units, twM, wtab, da);
        break;
      default:
        allow_smem((const void*)k_rows_inverse<T, ENV_F32>, c.smem);
        k_rows_inverse<T, ENV_F32><<<blocks, c.threads, c.smem, st>>>(
            eng, rows, row_list, n_sel, n_rows, Nr, static_cast<const float2*>(y), A, units, twM, wtab, da);
    }
  } else {
    allow_smem((const void*)k_rows_inverse<T, ENV_F64>, c.smem);
    k_rows_inverse<T, ENV_F64><<<blocks, c.threads, c.smem, st>>>(
        eng, rows, row_list, n_sel, n_rows, Nr, static_cast<const double2*>(y), A, units, twM, wtab, da);
  }
  return cudaGetLastError();
}

template cudaError_t launch_rows_forward<float>(const RowCfg&, const RowDev<float>*, int, int64_t, const float2*, void*,
                                                int, int64_t, const float2*, cudaStream_t, const float*);
template cudaError_t launch_rows_forward<double>(const RowCfg&, const RowDev<double>*, int, int64_t, const double2*,
                                                 void*, int, int64_t, const double2*, cudaStream_t, const double*);
template cudaError_t launch_rows_inverse<float>(const RowCfg&, const RowDev<float>*, const int*, int, int, int64_t,
                                                const void*, int, float2*, int64_t, const float2*, cudaStream_t,
                                                const float*, DenseArgs<float>);
template cudaError_t launch_rows_inverse<double>(const RowCfg&, const RowDev<double>*, const int*, int, int, int64_t,
                                                 const void*, int, double2*, int64_t, const double2*, cudaStream_t,
                                                 const double*, DenseArgs<double>);

}  // namespace qtam
