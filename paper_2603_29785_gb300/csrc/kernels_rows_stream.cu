// Row kernels of the streaming path (overlap-save): the compile-time FFTs of
// the default variants with a store that writes only a chunk's central
// envelope columns, rotated by the chunk's carrier phase, straight into the
// caller's map (forward), and a load that assembles a chunk's envelope from
// the map history and the newly pushed columns, rotated back (inverse).  This
// replaces the chunk envelope scratch and the separate crop / re-chunk passes
// when the plan's variant has these instantiations (FP32 envelopes, bisquare
// windows).
#include <cstring>

#include "rows_common.cuh"

namespace qtam {
namespace {

// map row at the chunk's first kept column; columns Gm .. Gm + Hn - 1 of the
// chunk are stored, multiplied by the chunk's phase
template <typename V, int E> struct StoreCrop {
  typename Env<V, E>::S* out;
  int Gm, Hn;
  V ph;
  bool valid;
  __device__ __forceinline__ void put(int, int n, V v) const {
    const unsigned k = (unsigned)(n - Gm);
    if (valid && k < (unsigned)Hn)
      stream_store(&out[k], Env<V, E>::to(mk<V>(v.x * ph.x - v.y * ph.y, v.x * ph.y + v.y * ph.x)));
  }
};

// a chunk's envelope column n is history column i Hn + n (n < split) or new
// column i Hn + n - hcols; both bases are set up per thread.  The load is
// unconditional (the bases of an invalid unit still point into the buffers)
// so a butterfly's loads issue back to back, and default-cached: each map
// column is read again by the neighbouring chunk about one chunk (25 MB)
// later, within the L2.
template <typename V, int E> struct LoadChunk {
  const typename Env<V, E>::S* hb;
  const typename Env<V, E>::S* yb;
  int split;
  V ph;
  bool valid;
  __device__ __forceinline__ V get(int, int n) const {
    const typename Env<V, E>::S* p = n < split ? hb + n : yb + (n - split);
    const V v = Env<V, E>::from(*p);
    const V r = mk<V>(v.x * ph.x - v.y * ph.y, v.x * ph.y + v.y * ph.x);
    return valid ? r : mk<V>(0, 0);
  }
};

template <class Eng>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_forward_crop_s(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                          float2* __restrict__ y, int64_t pitch, int Gm, int Hn, const float2* __restrict__ phase,
                          int64_t n_units, const float2* __restrict__ twM) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t chunk = valid ? unit / n_rows : 0;
  const int row = valid ? (int)(unit - chunk * n_rows) : 0;
  LoadBand<float, Eng::FEXACT> ld{X + chunk * Nr, row_ctx<float, Eng::FEXACT>(rows, row, Eng::M, Nr, valid, false,
                                                                           nullptr)};
  StoreCrop<float2, ENV_F32> st{y + row * pitch + chunk * Hn, Gm, Hn, valid ? phase[unit] : mk<float2>(0, 0), valid};
  Eng().template run<+1>(sm, twM, ld, st);
}

template <class Eng>
__global__ void __launch_bounds__(Eng::NT, Eng::MINB)
    k_rows_inverse_chunk_s(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel,
                           int n_rows, int64_t Nr, const float2* __restrict__ hist, int hcols,
                           const float2* __restrict__ ynew, int64_t pitch, int Hn, const float2* __restrict__ phase,
                           float2* __restrict__ A, int64_t n_units, const float2* __restrict__ twM) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int64_t unit = ((int64_t)blockIdx.x << Eng::NBS) + (threadIdx.x & ((1 << Eng::NBS) - 1));
  const bool valid = unit < n_units;
  const int64_t chunk = valid ? unit / n_sel : 0;
  const int row = valid ? row_list[unit - chunk * n_sel] : 0;
  const int64_t c0 = chunk * Hn;   // the chunk's first column in [history | new columns]
  const int split = (int)max((int64_t)0, (int64_t)hcols - c0);
  LoadChunk<float2, ENV_F32> ld{hist + (int64_t)row * hcols + c0, ynew + row * pitch + max((int64_t)0, c0 - hcols),
                                split, valid ? phase[chunk * n_rows + row] : mk<float2>(0, 0), valid};
  AccumulateBand<float, Eng::FEXACT, Eng::PRED_RED> acc{
      A + chunk * Nr, row_ctx<float, Eng::FEXACT>(rows, row, Eng::M, Nr, valid, true, nullptr)};
  Eng().template run<-1>(sm, twM, ld, acc);
}

template <class Eng>
cudaError_t fwd_crop_launch(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, float2* y,
                            int64_t pitch, int Gm, int Hn, const float2* phase, int64_t B, const float2* twM,
                            cudaStream_t st) {
  const int64_t units = B * n_rows;
  if (units == 0) return cudaSuccess;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_forward_crop_s<Eng>, smem);
  k_rows_forward_crop_s<Eng><<<(unsigned)blocks, Eng::NT, smem, st>>>(rows, n_rows, Nr, X, y, pitch, Gm, Hn, phase,
                                                                     units, twM);
  return cudaGetLastError();
}

template <class Eng>
cudaError_t inv_chunk_launch(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                             const float2* hist, int hcols, const float2* ynew, int64_t pitch, int Hn,
                             const float2* phase, float2* A, int64_t B, const float2* twM, cudaStream_t st) {
  const int64_t units = B * n_sel;
  if (units == 0) return cudaSuccess;
  const int64_t blocks = (units + (1 << Eng::NBS) - 1) >> Eng::NBS;
  const size_t smem = Eng::smem_bytes(sizeof(float2));
  allow_smem((const void*)k_rows_inverse_chunk_s<Eng>, smem);
  k_rows_inverse_chunk_s<Eng><<<(unsigned)blocks, Eng::NT, smem, st>>>(rows, row_list, n_sel, n_rows, Nr, hist, hcols,
                                                                      ynew, pitch, Hn, phase, A, units, twM);
  return cudaGetLastError();
}

// same names as the variant registry, so a plan's variant finds its entry
#define QTAM_VS(M, NBS, MINB, ...)                                                                        \
  StreamRowFns {                                                                                        \
    #M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB,                                            \
        fwd_crop_launch<StaticEngine<M, NBS, MINB, __VA_ARGS__>>,                                       \
        inv_chunk_launch<StaticEngine<M, NBS, MINB, __VA_ARGS__>>                                        \
  }
#define QTAM_VS_NT(NT, M, NBS, MINB, ...)                                                                 \
  StreamRowFns {                                                                                          \
    #M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB " threads " #NT,                              \
        fwd_crop_launch<ThreadsEngine<NT, M, NBS, MINB, __VA_ARGS__>>,                                     \
        inv_chunk_launch<ThreadsEngine<NT, M, NBS, MINB, __VA_ARGS__>>                                     \
  }
const StreamRowFns kStreamFns[] = {
    QTAM_VS(4800, 0, 4, 16, 20, 15), QTAM_VS(2400, 0, 3, 16, 10, 15), QTAM_VS(1200, 1, 2, 16, 15, 5),
    QTAM_VS(600, 3, 2, 8, 3, 25),    QTAM_VS(500, 3, 2, 4, 5, 25),    QTAM_VS(300, 3, 2, 12, 25),
    QTAM_VS(150, 4, 2, 6, 25),       QTAM_VS(75, 5, 2, 3, 25),        QTAM_VS(8192, 0, 1, 16, 16, 32),
    // the preferred defaults of kernels_rows_tuned.cu
    QTAM_VS(1200, 0, 8, 10, 12, 10), QTAM_VS(600, 1, 8, 25, 24),      QTAM_VS(300, 1, 12, 15, 20),
    QTAM_VS(150, 3, 4, 10, 15),      QTAM_VS(8192, 0, 2, 16, 8, 8, 8),
    QTAM_VS_NT(160, 2400, 0, 6, 16, 10, 15),
};
#undef QTAM_VS
#undef QTAM_VS_NT

}  // namespace

const StreamRowFns* stream_row_fns(const char* variant_name) {
  if (!variant_name) return nullptr;
  for (const StreamRowFns& f : kStreamFns)
    if (std::strcmp(f.name, variant_name) == 0) return &f;
  return nullptr;
}

}  // namespace qtam
