// Internal declarations shared by the host plan code and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "fft_core.cuh"
#include "../../include/qtam.h"

struct qtam_plan_s;

namespace qtam {

constexpr int kMaxBlock = 512;   // threads per block of every FFT kernel

// Opt a kernel into more than 48 KB of dynamic shared memory when needed.
inline cudaError_t allow_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// One (plane, row) window on the device.  W_k(d) = c (((h-|d|)(h+|d|)) / h^2)^2.
template <typename T> struct RowDev {
  int kc;     // centre bin k_c
  int h;      // half-width
  T c_fwd;    // c_k / sqrt(M N): window normalisation times the forward renormalisation
  T c_inv;    // c_k sqrt(N / M): window normalisation times the synthesis re-scaling
  T inv_h2;   // 1 / h^2
  T kw_fwd;   // sqrt(c_fwd) / h^2: window weight c_fwd W'(d) = (kw_fwd (h^2 - d^2))^2
  T kw_inv;   // sqrt(c_inv) / h^2
  int woff;   // offset of this row's W'(0..h) in the plan's window table; -1: bisquare formula
  int hb;     // half-width of the loaded band: h, or N/2 in dense mode (every bin)
  T eps_fwd;  // dense mode: c_fwd eps, the weight wherever the window vanishes (else 0)
  T eps_inv;  // dense mode: c_inv eps
};

// Runtime-engine options of the dense mode: remodulate multiplies the
// envelopes by exp(+2 pi i k_c n / M) on store (and by its conjugate on load);
// divide turns the inverse store into X[k_c + d] = v * scale / weight(d)
// (the single-tile inverse) instead of accumulating v * weight(d).
template <typename T> struct DenseArgs {
  int remod = 0;
  int divide = 0;
  T scale = (T)0;
};

// Long real FFT of N = 2n samples as an n = n1 * n2 four-step complex FFT.
struct LongCfg {
  const void* stw_col = nullptr;   // stage twiddle tables of the static column engine (or null)
  const void* stw_row = nullptr;   // ... of the static row engine
  const void* tw4 = nullptr;       // [n1][n2] four-step twiddles w_n^(k1 c), layout of the column-pass output
  int n;        // N / 2
  int n1, n2;   // column length n1 (stride n2), row length n2
  int col_nbs;  // log2 of columns per column-pass block
  int row_nbs;  // log2 of rows per row-pass block
  RadixPlan rp1, rp2;
  int col_threads, row_threads;
  size_t col_smem, row_smem;
};

struct RowCfg {
  RadixPlan rp;  // radices of M (runtime engine)
  int threads;
  size_t smem;
  int variant;   // index of a compile-time row-kernel variant, -1 = runtime engine
  int remod = 0; // dense mode: remodulated envelopes
  int dense = 0; // stopband floor or carrier: only the variants' dense kernels serve the plan;
                 // 2: floor and carrier (tiles span the spectrum, bins at their own positions)
  const void* stw = nullptr;   // stage twiddle tables of that variant
  // tensor-core short DFT (M = 8192): DFT-64 block operand, its conjugate
  // transpose (the inverse rows), DFT-128 cosine and sine operands; used
  // when `tensor` is set
  int tensor = 0;
  const void* tcA = nullptr;
  const void* tcAi = nullptr;
  const void* tcG = nullptr;
};

enum EnvKind { ENV_F32 = 0, ENV_F64 = 1, ENV_BF16 = 2, ENV_F16 = 3 };

// Tensor-core rows (kernels_tc.cu): M must be 8192, FP32 compute.
bool tc_forward_supported(int M);
cudaError_t launch_rows_forward_tc(const RowCfg& c, const RowDev<float>* rows, int n_rows, int64_t Nr,
                                   const float2* X, void* y, int env, int64_t B, cudaStream_t st, const float* wtab);
// Tensor-core inverse rows (accumulate into A, zeroed by the caller).  False
// (nothing launched) when y is not 16-byte aligned: the CUDA-core rows then
// serve; otherwise *err holds the launch status.
bool launch_rows_inverse_tc(const RowCfg& c, const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows,
                            int64_t Nr, const void* y, int env, float2* A, int64_t B, cudaStream_t st,
                            const float* wtab, cudaError_t* err);

// A compile-time row-kernel variant (FP32 compute): fixed M, radix sequence,
// rows per block and occupancy target.  fwd/inv are indexed by EnvKind.
using RowFwdFn = cudaError_t (*)(const RowDev<float>*, int, int64_t, const float2*, void*, int64_t, const float2*,
                                 cudaStream_t);
using RowInvFn = cudaError_t (*)(const RowDev<float>*, const int*, int, int, int64_t, const void*, float2*, int64_t,
                                 const float2*, cudaStream_t);
// the same with the plan's window table (non-bisquare windows), FP32 envelopes
using RowFwdTabFn = cudaError_t (*)(const RowDev<float>*, int, int64_t, const float2*, void*, int64_t, const float2*,
                                    cudaStream_t, const float*);
using RowInvTabFn = cudaError_t (*)(const RowDev<float>*, const int*, int, int, int64_t, const void*, float2*, int64_t,
                                    const float2*, cudaStream_t, const float*);
// dense mode (FP32 arithmetic; envelopes F32, BF16 or F16 by EnvKind env):
// the weights with the stopband floor over the whole one-sided spectrum;
// mode 0 baseband tiles, 1 with the carrier on store / load, 2 floor and
// carrier (bins placed at their own positions)
using RowFwdDenseFn = cudaError_t (*)(const RowDev<float>*, int, int64_t, const float2*, void*, int64_t, const float2*,
                                      cudaStream_t, const float*, const float2* twM, int mode, int env);
using RowInvDenseFn = cudaError_t (*)(const RowDev<float>*, const int*, int, int, int64_t, const void*, float2*, int64_t,
                                      const float2*, cudaStream_t, const float*, const float2* twM, int mode, int env);
struct RowVariant {
  int M;
  int rows_per_block;
  int threads;
  size_t smem;
  const char* name;
  int nst;       // radix sequence of the compile-time FFT
  int r[kMaxStages];
  RowFwdFn fwd[4];
  RowInvFn inv[4];
  RowFwdTabFn fwd_tab;   // null unless built for window tables (FP32 envelopes only)
  RowInvTabFn inv_tab;
  RowFwdDenseFn fwd_dense;   // null unless built for the dense mode
  RowInvDenseFn inv_dense;
  int tw_pair = 0;   // stage tables in the row-pair format (c, c, s, s) per entry (kernels_rows_pair.cu)
  int preferred = 0;   // default of its length for bisquare plans ahead of the other variants
};
// the dense-mode variants live in their own translation unit (kernels_rows_dense.cu)
int dense_row_variant_count();
const RowVariant* dense_row_variant(int i);
// the row-pair variants (packed FP32x2, two rows per block) in kernels_rows_pair.cu
int pair_row_variant_count();
const RowVariant* pair_row_variant(int i);
// variants added after measurement (kernels_rows_tuned.cu): balanced radices for
// the short lengths, a four-stage sequence at M = 8192
int tuned_row_variant_count();
const RowVariant* tuned_row_variant(int i);
// Fused streaming row kernels (kernels_rows_stream.cu) of a compile-time
// variant, looked up by the variant's name: forward with the crop-and-phase
// store into the map, inverse with the history/new-columns chunk load.
using StreamFwdFn = cudaError_t (*)(const RowDev<float>* rows, int n_rows, int64_t Nr, const float2* X, float2* y,
                                    int64_t pitch, int Gm, int Hn, const float2* phase, int64_t B, const float2* twM,
                                    cudaStream_t st);
using StreamInvFn = cudaError_t (*)(const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows, int64_t Nr,
                                    const float2* hist, int hcols, const float2* ynew, int64_t pitch, int Hn,
                                    const float2* phase, float2* A, int64_t B, const float2* twM, cudaStream_t st);
struct StreamRowFns {
  const char* name;
  StreamFwdFn fwd;
  StreamInvFn inv;
};
const StreamRowFns* stream_row_fns(const char* variant_name);

// Streaming steps with the fused row kernels (qtam_api.cu, used by
// qtam_stream.cu).  *used is false (and nothing is launched) when the plan
// has no fused kernels: F32 compute and envelopes, bisquare windows, a
// compile-time variant with a fused entry.  phase is [b][P K] complex FP32.
qtam_status stream_forward_fused(qtam_plan_s* pl, const void* x, int64_t b, void* ymap, int64_t pitch, int Gm, int Hn,
                                 const void* phase, void* ws, size_t wsb, cudaStream_t st, bool* used);
qtam_status stream_inverse_fused(qtam_plan_s* pl, const void* hist, int hcols, const void* ynew, int64_t pitch, int Hn,
                                 const void* phase, int64_t b, uint64_t mask, void* x, void* ws, size_t wsb,
                                 cudaStream_t st, bool* used);

int row_variant_count();
// per (segment, plane) pair: energy = sum |Y|^2 (FP64), peak = max |Y|^2 over K*M values
cudaError_t launch_plane_metrics(const void* y, int env, int64_t pairs, int64_t per_plane, double* energy, float* peak,
                                 cudaStream_t st);
// y[r][*] *= gain[r] for r < n_rows (device gains), envelope storage kind env
cudaError_t launch_scale_rows(void* y, int env, const float* gain, int64_t n_rows, int M, cudaStream_t st);
const RowVariant* row_variant(int i);   // nullptr when out of range

// ---- launchers (kernels_long.cu) ----
// z: [B][n] complex view of the real input; U: [B][n]; Z: [B][n]; X: [B][n+1]
template <typename T>
cudaError_t launch_spectrum(const LongCfg& c, const cplx<T>* z, cplx<T>* U, cplx<T>* Z, cplx<T>* X, int64_t B,
                            const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st);
// A: [B][n+1] accumulated spectrum; invP: [n+1]; Zi, V: [B][n] scratch (V may alias A's
// buffer: A is consumed before V is written); xout: [B][n] complex view of the output
template <typename T>
cudaError_t launch_synthesis(const LongCfg& c, const cplx<T>* A, const T* invP, cplx<T>* Zi, cplx<T>* V,
                             cplx<T>* xout, int64_t B, const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st);

// ---- launchers (kernels_rows.cu) ----
// X: [B][Nr] spectrum -> y: [B][R][M] envelopes (R = P*K rows)
template <typename T>
cudaError_t launch_rows_forward(const RowCfg& c, const RowDev<T>* rows, int n_rows, int64_t Nr, const cplx<T>* X,
                                void* y, int env, int64_t B, const cplx<T>* twM, cudaStream_t st,
                                const T* wtab = nullptr);
// y rows listed in row_list -> atomically accumulated into A: [B][Nr] (must be zeroed)
template <typename T>
cudaError_t launch_rows_inverse(const RowCfg& c, const RowDev<T>* rows, const int* row_list, int n_sel, int n_rows,
                                int64_t Nr, const void* y, int env, cplx<T>* A, int64_t B, const cplx<T>* twM,
                                cudaStream_t st, const T* wtab = nullptr, DenseArgs<T> da = DenseArgs<T>());

// radix sequence of the static long-FFT engine used for a pass of length m
// with 2^nbs interleaved transforms (FP32); false when the runtime engine runs
bool long_static_radices(int m, int nbs, int* r, int* nst);

// Stage twiddle tables of a compile-time radix sequence r[0..nst), stage 0
// has none: for s >= 1 with NS = r_0 ... r_{s-1}, entries [i][k] (k fastest)
// = exp(-2 pi i ik / (NS r_s)), i < r_s, k < NS.  Interleaved (re, im), FP64.
inline void stage_twiddles(const int* r, int nst, double* out_or_null, size_t* count) {
  size_t n = 0, ns = (size_t)r[0];
  const double two_pi = 6.283185307179586476925286766559;
  for (int s = 1; s < nst; ++s) {
    const size_t span = ns * (size_t)r[s];
    for (int i = 0; i < r[s]; ++i)
      for (size_t k = 0; k < ns; ++k) {
        if (out_or_null) {
          const size_t e = ((size_t)i * k) % span;
          const double ang = two_pi * (double)e / (double)span;
          out_or_null[2 * n] = std::cos(ang);
          out_or_null[2 * n + 1] = -std::sin(ang);
        }
        ++n;
      }
    ns = span;
  }
  *count = n;
}

// ---- host helpers (qtam_api.cu) ----
void set_last_error(const std::string& msg);   // message for qtam_last_error()
int plan_device(const qtam_plan_s* plan);      // device of a plan, -1 when host-only

}  // namespace qtam
