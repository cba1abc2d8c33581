// Streaming QTAM over a continuous signal: overlap-save on top of the
// segment transform (qtam_forward / qtam_inverse).
//
// The paper motivates signals of hours (Sec. I) but fixes no streaming
// scheme; this one keeps every property of the segment transform it can.
// Chunks of the plan's length N advance by `hop` samples; each chunk's
// transform is circular, so its first and last G = (N - hop)/2 samples
// carry the wrap and only the central hop*M/N envelope columns are kept.
// hop and G are whole multiples of N / gcd(N, M), so chunk boundaries fall
// on envelope columns.  Demodulation (Sec. III) references each chunk's
// envelopes to the chunk's own first sample; a chunk starting a samples
// into the stream is multiplied by exp(-2 pi i k_c a / N) per row, which
// re-references it to the stream origin (the carrier phase of the shift
// theorem), so the stitched map is continuous across chunks.  The inverse
// re-chunks the map the same way, undoes the phase, applies the canonical
// dual (Eq. qtam_canonical_inverse) and keeps each chunk's central samples.
//
// Kernels: input chunk gather (history + new samples), envelope crop with
// the phase, map re-chunking with the conjugate phase.  All three are plain
// HBM copies, one block per (chunk, row) for the envelope ones, with the
// phase computed once per block from the integer k_c * a mod N in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/qtam.h"
#include "qtam_internal.h"

namespace {

// ---- element access for the four envelope storage types -------------------
template <typename S> struct Cx;
template <> struct Cx<float2> {
  __device__ static float2 rot(float2 v, double c, double s) {
    const float cf = (float)c, sf = (float)s;
    return make_float2(v.x * cf - v.y * sf, v.x * sf + v.y * cf);
  }
};
template <> struct Cx<double2> {
  __device__ static double2 rot(double2 v, double c, double s) {
    return make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
};
template <> struct Cx<__nv_bfloat162> {
  __device__ static __nv_bfloat162 rot(__nv_bfloat162 v, double c, double s) {
    const float2 f = __bfloat1622float2(v);
    return __float22bfloat162_rn(Cx<float2>::rot(f, c, s));
  }
};
template <> struct Cx<__half2> {
  __device__ static __half2 rot(__half2 v, double c, double s) {
    const float2 f = __half22float2(v);
    return __float22half2_rn(Cx<float2>::rot(f, c, s));
  }
};

// exp(sign * 2 pi i kc a / N) with kc a reduced mod N in integers.  FP64
// is a slow pipe on this part, so one thread evaluates it and the block
// reads it from shared memory.
__device__ __forceinline__ void carrier_phase(int64_t kc, int64_t a, int64_t N, double sign, double& c, double& s) {
  __shared__ double cs[2];
  if (threadIdx.x == 0) {
    int64_t am = a % N;
    if (am < 0) am += N;
    const int64_t m = (kc * am) % N;
    sincospi(sign * 2.0 * (double)m / (double)N, &cs[1], &cs[0]);
  }
  __syncthreads();
  c = cs[0];
  s = cs[1];
}

// chunks[i][t] = cat[i*hop + t], cat = [hist (nh samples) | xnew]
template <typename T>
__global__ void k_stream_gather_x(const T* __restrict__ hist, int64_t nh, const T* __restrict__ xnew, int64_t hop,
                                  int64_t N, int64_t total, T* __restrict__ chunks) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, t = e - i * N, g = i * hop + t;
    chunks[e] = g < nh ? hist[g] : xnew[g - nh];
  }
}

// y[r][i*Hn + j] = env[i][r][Gm + j] * exp(-2 pi i kc[r] (a0 + i hop) / N)
template <typename S>
__global__ void k_stream_crop(const S* __restrict__ env, int R, int M, int Gm, int Hn, const int* __restrict__ kc,
                              int64_t N, int64_t a0, int64_t hop, S* __restrict__ y, int64_t pitch) {
  const int64_t ir = blockIdx.x;
  const int64_t i = ir / R;
  const int r = (int)(ir - i * R);
  double c, s;
  carrier_phase(kc[r], a0 + i * hop, N, -1.0, c, s);
  const S* src = env + ir * M + Gm;
  S* dst = y + r * pitch + i * Hn;
  for (int j = threadIdx.x; j < Hn; j += blockDim.x) dst[j] = Cx<S>::rot(__ldcs(src + j), c, s);
}

// env[i][r][n] = cat[r][i*Hn + n] * exp(+2 pi i kc[r] (a0 + i hop) / N),
// cat[r] = [hist[r] (hcols columns) | ynew[r] (row pitch `pitch`)]
template <typename S>
__global__ void k_stream_gather_y(const S* __restrict__ hist, int hcols, const S* __restrict__ ynew, int64_t pitch,
                                  int R, int M, int Hn, const int* __restrict__ kc, int64_t N, int64_t a0, int64_t hop,
                                  S* __restrict__ env) {
  const int64_t ir = blockIdx.x;
  const int64_t i = ir / R;
  const int r = (int)(ir - i * R);
  double c, s;
  carrier_phase(kc[r], a0 + i * hop, N, 1.0, c, s);
  const S* h = hist + (int64_t)r * hcols;
  const S* yr = ynew + r * pitch;
  S* dst = env + ir * M;
  const int64_t c0 = i * Hn;
  for (int n = threadIdx.x; n < M; n += blockDim.x) {
    const int64_t col = c0 + n;
    const S v = col < hcols ? h[col] : yr[col - hcols];
    dst[n] = Cx<S>::rot(v, c, s);
  }
}

// phase[i][r] = exp(sign 2 pi i kc[r] (a0 + i hop) / N): the per-(chunk, row)
// factors of the fused streaming kernels, one FP64 evaluation each
__global__ void k_stream_phases(const int* __restrict__ kc, int R, int64_t b, int64_t N, int64_t a0, int64_t hop,
                                double sign, float2* __restrict__ phase) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b * R) return;
  const int64_t i = e / R;
  const int r = (int)(e - i * R);
  int64_t am = (a0 + i * hop) % N;
  if (am < 0) am += N;
  const int64_t m = ((int64_t)kc[r] * am) % N;
  double s, c;
  sincospi(sign * 2.0 * (double)m / (double)N, &s, &c);
  phase[e] = make_float2((float)c, (float)s);
}

template <typename S>
cudaError_t crop(const void* env, int64_t b, int R, int M, int Gm, int Hn, const int* kc, int64_t N, int64_t a0,
                 int64_t hop, void* y, int64_t pitch, cudaStream_t st) {
  k_stream_crop<S><<<(unsigned)(b * R), 256, 0, st>>>(static_cast<const S*>(env), R, M, Gm, Hn, kc, N, a0, hop,
                                                      static_cast<S*>(y), pitch);
  return cudaGetLastError();
}

template <typename S>
cudaError_t gather_y(const void* hist, int hcols, const void* ynew, int64_t pitch, int64_t b, int R, int M, int Hn,
                     const int* kc, int64_t N, int64_t a0, int64_t hop, void* env, cudaStream_t st) {
  k_stream_gather_y<S><<<(unsigned)(b * R), 256, 0, st>>>(static_cast<const S*>(hist), hcols,
                                                          static_cast<const S*>(ynew), pitch, R, M, Hn, kc, N, a0,
                                                          hop, static_cast<S*>(env));
  return cudaGetLastError();
}

qtam_status sfail(qtam_status s, const std::string& msg) {
  qtam::set_last_error(msg);
  return s;
}
qtam_status sfail_cuda(cudaError_t e, const char* where) {
  qtam::set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
  return QTAM_ERR_CUDA;
}

struct DevScope {
  int prev = -1;
  bool ok = false;
  explicit DevScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

struct qtam_stream_s {
  qtam_plan_t plan = nullptr;
  int device = -1;
  int64_t N = 0;
  int M = 0, R = 0, env = QTAM_DTYPE_F32;
  size_t rs = 4, es = 8;  // real and envelope element sizes
  int64_t hop = 0, G = 0, q = 0, bmax = 1;
  int Hn = 0, Gm = 0;
  int64_t pos = 0, cpos = 0;
  void* hx[2] = {nullptr, nullptr};
  int cx = 0;
  void* hy[2] = {nullptr, nullptr};
  int cy = 0;
  void* chunks = nullptr;
  void* envb = nullptr;
  void* ws = nullptr;
  size_t wsb = 0;
  int* kc = nullptr;
  float2* phase = nullptr;   // [max_chunks][R] phases of the fused kernels
  size_t bytes = 0;
};

namespace {

void free_stream(qtam_stream_s* s) {
  if (!s) return;
  if (s->device >= 0) {
    DevScope g(s->device);
    for (void* p : {s->hx[0], s->hx[1], s->hy[0], s->hy[1], s->chunks, s->envb, s->ws, (void*)s->kc, (void*)s->phase})
      cudaFree(p);
  }
  delete s;
}

qtam_status salloc(qtam_stream_s* s, void** p, size_t bytes) {
  if (bytes == 0) return QTAM_OK;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return sfail(QTAM_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->bytes += bytes;
  return QTAM_OK;
}

cudaError_t launch_crop(const qtam_stream_s* s, int64_t b, int64_t a0, void* y, int64_t pitch, cudaStream_t st) {
  switch (s->env) {
    case QTAM_DTYPE_F64: return crop<double2>(s->envb, b, s->R, s->M, s->Gm, s->Hn, s->kc, s->N, a0, s->hop, y, pitch, st);
    case QTAM_DTYPE_BF16:
      return crop<__nv_bfloat162>(s->envb, b, s->R, s->M, s->Gm, s->Hn, s->kc, s->N, a0, s->hop, y, pitch, st);
    case QTAM_DTYPE_F16: return crop<__half2>(s->envb, b, s->R, s->M, s->Gm, s->Hn, s->kc, s->N, a0, s->hop, y, pitch, st);
    default: return crop<float2>(s->envb, b, s->R, s->M, s->Gm, s->Hn, s->kc, s->N, a0, s->hop, y, pitch, st);
  }
}

cudaError_t launch_gather_y(const qtam_stream_s* s, const void* ynew, int64_t pitch, int64_t b, int64_t a0,
                            cudaStream_t st) {
  const void* h = s->hy[s->cy];
  const int hc = 2 * s->Gm;
  switch (s->env) {
    case QTAM_DTYPE_F64:
      return gather_y<double2>(h, hc, ynew, pitch, b, s->R, s->M, s->Hn, s->kc, s->N, a0, s->hop, s->envb, st);
    case QTAM_DTYPE_BF16:
      return gather_y<__nv_bfloat162>(h, hc, ynew, pitch, b, s->R, s->M, s->Hn, s->kc, s->N, a0, s->hop, s->envb, st);
    case QTAM_DTYPE_F16:
      return gather_y<__half2>(h, hc, ynew, pitch, b, s->R, s->M, s->Hn, s->kc, s->N, a0, s->hop, s->envb, st);
    default: return gather_y<float2>(h, hc, ynew, pitch, b, s->R, s->M, s->Hn, s->kc, s->N, a0, s->hop, s->envb, st);
  }
}

cudaError_t launch_phases(const qtam_stream_s* s, int64_t b, int64_t a0, double sign, cudaStream_t st) {
  const int64_t n = b * s->R;
  k_stream_phases<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->kc, s->R, b, s->N, a0, s->hop, sign, s->phase);
  return cudaGetLastError();
}

cudaError_t launch_gather_x(const qtam_stream_s* s, const void* xnew, int64_t b, cudaStream_t st) {
  const int64_t total = b * s->N;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (s->rs == 8)
    k_stream_gather_x<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(s->hx[s->cx]), 2 * s->G,
                                                      static_cast<const double*>(xnew), s->hop, s->N, total,
                                                      static_cast<double*>(s->chunks));
  else
    k_stream_gather_x<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(s->hx[s->cx]), 2 * s->G,
                                                     static_cast<const float*>(xnew), s->hop, s->N, total,
                                                     static_cast<float*>(s->chunks));
  return cudaGetLastError();
}

}  // namespace

extern "C" {

qtam_status qtam_stream_create(qtam_plan_t plan, int64_t hop, int64_t max_chunks, qtam_stream_t* out) {
  if (!plan || !out || hop < 0 || max_chunks < 1) return sfail(QTAM_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  const int dev = qtam::plan_device(plan);
  qtam_plan_info_t info;
  qtam_status st = qtam_plan_info(plan, &info);
  if (st != QTAM_OK) return st;
  const int64_t N = info.length, M = info.n_out;
  const int64_t q = N / std::gcd(N, M);
  if (hop == 0) {
    const int64_t G = (N / 4) / q * q;
    hop = N - 2 * G;
  }
  if (hop > N || hop % q || (N - hop) % (2 * q))
    return sfail(QTAM_ERR_INVALID_ARG, "hop must be a multiple of N/gcd(N,M) <= N, with (N-hop)/2 one too");
  const int R = info.n_planes * info.rows_per_plane;
  if (max_chunks * (int64_t)R > (int64_t)INT32_MAX) return sfail(QTAM_ERR_INVALID_ARG, "max_chunks too large");
  if (dev < 0) return sfail(QTAM_ERR_NO_DEVICE, "the plan is host-only");
  qtam_stream_s* s = new (std::nothrow) qtam_stream_s();
  if (!s) return sfail(QTAM_ERR_OUT_OF_MEMORY, "host allocation");
  s->plan = plan;
  s->device = dev;
  s->N = N;
  s->M = (int)M;
  s->R = R;
  s->env = info.envelope_dtype;
  s->rs = info.compute_dtype == QTAM_DTYPE_F64 ? 8 : 4;
  s->es = s->env == QTAM_DTYPE_F64 ? 16 : (s->env == QTAM_DTYPE_F32 ? 8 : 4);
  s->hop = hop;
  s->G = (N - hop) / 2;
  s->q = q;
  s->Hn = (int)(hop * M / N);
  s->Gm = (int)(s->G * M / N);
  s->bmax = max_chunks;
  std::vector<int64_t> kc64(R);
  std::vector<int> kc(R);
  if ((st = qtam_plan_rows(plan, nullptr, kc64.data(), nullptr, nullptr)) != QTAM_OK) {
    s->device = -1;
    free_stream(s);
    return st;
  }
  // the chunk re-reference exp(-/+ 2 pi i k_c a / N) is computed from these
  // centres; remodulated tiles already refer their columns to absolute time,
  // so their factor is 1 (centre 0)
  for (int r = 0; r < R; ++r) kc[r] = info.remodulate ? 0 : (int)kc64[r];
  size_t wsb = 0;
  qtam_workspace_size(plan, max_chunks, &wsb);
  s->wsb = wsb;
  DevScope g(dev);
  if (!g.ok) {
    s->device = -1;
    free_stream(s);
    return sfail(QTAM_ERR_CUDA, "cudaSetDevice failed");
  }
  const size_t hxb = (size_t)(2 * s->G) * s->rs, hyb = (size_t)R * (size_t)(2 * s->Gm) * s->es;
  if ((st = salloc(s, &s->hx[0], hxb)) != QTAM_OK || (st = salloc(s, &s->hx[1], hxb)) != QTAM_OK ||
      (st = salloc(s, &s->hy[0], hyb)) != QTAM_OK || (st = salloc(s, &s->hy[1], hyb)) != QTAM_OK ||
      (st = salloc(s, &s->chunks, (size_t)max_chunks * N * s->rs)) != QTAM_OK ||
      (st = salloc(s, &s->envb, (size_t)max_chunks * R * M * s->es)) != QTAM_OK ||
      (st = salloc(s, &s->ws, wsb)) != QTAM_OK ||
      (st = salloc(s, reinterpret_cast<void**>(&s->kc), (size_t)R * sizeof(int))) != QTAM_OK ||
      (st = salloc(s, reinterpret_cast<void**>(&s->phase), (size_t)max_chunks * R * sizeof(float2))) != QTAM_OK) {
    free_stream(s);
    return st;
  }
  cudaError_t e = cudaMemcpy(s->kc, kc.data(), (size_t)R * sizeof(int), cudaMemcpyHostToDevice);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    if (hxb) e = cudaMemset(s->hx[i], 0, hxb);
    if (e == cudaSuccess && hyb) e = cudaMemset(s->hy[i], 0, hyb);
  }
  if (e != cudaSuccess) {
    free_stream(s);
    return sfail_cuda(e, "stream setup");
  }
  *out = s;
  return QTAM_OK;
}

qtam_status qtam_stream_info(qtam_stream_t s, qtam_stream_info_t* o) {
  if (!s || !o) return sfail(QTAM_ERR_INVALID_ARG, "NULL argument");
  std::memset(o, 0, sizeof(*o));
  o->hop = s->hop;
  o->guard = s->G;
  o->quantum = s->q;
  o->hop_cols = s->Hn;
  o->guard_cols = s->Gm;
  o->max_chunks = s->bmax;
  o->samples_in = s->pos;
  o->columns_in = s->cpos;
  o->device_bytes = (int64_t)s->bytes;
  return QTAM_OK;
}

qtam_status qtam_stream_forward(qtam_stream_t s, const void* x, int64_t n, void* y, void* stream) {
  if (!s || n < 0 || n % s->hop) return sfail(QTAM_ERR_INVALID_ARG, "n must be a non-negative multiple of hop");
  if (n == 0) return QTAM_OK;
  if (!x || !y) return sfail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevScope g(s->device);
  if (!g.ok) return sfail(QTAM_ERR_CUDA, "cudaSetDevice failed");
  const int64_t J = n / s->hop, pitch = J * s->Hn, nh = 2 * s->G;
  for (int64_t done = 0; done < J;) {
    const int64_t b = std::min(s->bmax, J - done);
    const char* xb = static_cast<const char*>(x) + (size_t)(done * s->hop) * s->rs;
    cudaError_t e = launch_gather_x(s, xb, b, st);
    if (e != cudaSuccess) return sfail_cuda(e, "stream gather");
    void* yout = static_cast<char*>(y) + (size_t)(done * s->Hn) * s->es;
    bool used = false;
    if (s->env == QTAM_DTYPE_F32) {   // fused: the row kernel stores the kept columns with the phase
      if ((e = launch_phases(s, b, s->pos - nh, -1.0, st)) != cudaSuccess) return sfail_cuda(e, "stream phases");
      qtam_status q = qtam::stream_forward_fused(s->plan, s->chunks, b, yout, pitch, s->Gm, s->Hn, s->phase, s->ws,
                                                 s->wsb, st, &used);
      if (q != QTAM_OK) return q;
    }
    if (!used) {
      qtam_status q = qtam_forward(s->plan, s->chunks, b, s->envb, s->ws, s->wsb, stream);
      if (q != QTAM_OK) return q;
      e = launch_crop(s, b, s->pos - nh, yout, pitch, st);
      if (e != cudaSuccess) return sfail_cuda(e, "stream crop");
    }
    if (nh > 0) {  // history <- last 2G samples of [history | this step's samples]
      const int64_t nn = b * s->hop;
      char* dst = static_cast<char*>(s->hx[1 - s->cx]);
      if (nn >= nh) {
        e = cudaMemcpyAsync(dst, xb + (size_t)(nn - nh) * s->rs, (size_t)nh * s->rs, cudaMemcpyDeviceToDevice, st);
      } else {
        e = cudaMemcpyAsync(dst, static_cast<const char*>(s->hx[s->cx]) + (size_t)nn * s->rs, (size_t)(nh - nn) * s->rs,
                            cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dst + (size_t)(nh - nn) * s->rs, xb, (size_t)nn * s->rs, cudaMemcpyDeviceToDevice, st);
      }
      if (e != cudaSuccess) return sfail_cuda(e, "stream history");
      s->cx = 1 - s->cx;
    }
    s->pos += b * s->hop;
    done += b;
  }
  return QTAM_OK;
}

qtam_status qtam_stream_inverse(qtam_stream_t s, const void* y, int64_t n_cols, uint64_t plane_mask, void* x,
                                void* stream) {
  if (!s || n_cols < 0 || n_cols % s->Hn)
    return sfail(QTAM_ERR_INVALID_ARG, "n_cols must be a non-negative multiple of the hop's column count");
  if (n_cols == 0) return QTAM_OK;
  if (!x || !y) return sfail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevScope g(s->device);
  if (!g.ok) return sfail(QTAM_ERR_CUDA, "cudaSetDevice failed");
  const int64_t J = n_cols / s->Hn, hc = 2 * (int64_t)s->Gm;
  for (int64_t done = 0; done < J;) {
    const int64_t b = std::min(s->bmax, J - done);
    const char* yb = static_cast<const char*>(y) + (size_t)(done * s->Hn) * s->es;
    const int64_t a0 = (s->cpos / s->Hn) * s->hop - 3 * s->G;
    cudaError_t e = cudaSuccess;
    bool used = false;
    if (s->env == QTAM_DTYPE_F32) {   // fused: the row kernel reads history and new columns with the phase
      if ((e = launch_phases(s, b, a0, 1.0, st)) != cudaSuccess) return sfail_cuda(e, "stream phases");
      qtam_status q = qtam::stream_inverse_fused(s->plan, s->hy[s->cy], 2 * s->Gm, yb, n_cols, s->Hn, s->phase, b,
                                                 plane_mask, s->chunks, s->ws, s->wsb, st, &used);
      if (q != QTAM_OK) return q;
    }
    if (!used) {
      e = launch_gather_y(s, yb, n_cols, b, a0, st);
      if (e != cudaSuccess) return sfail_cuda(e, "stream re-chunk");
      qtam_status q = qtam_inverse(s->plan, s->envb, b, plane_mask, s->chunks, s->ws, s->wsb, stream);
      if (q != QTAM_OK) return q;
    }
    e = cudaMemcpy2DAsync(static_cast<char*>(x) + (size_t)(done * s->hop) * s->rs, (size_t)s->hop * s->rs,
                          static_cast<const char*>(s->chunks) + (size_t)s->G * s->rs, (size_t)s->N * s->rs,
                          (size_t)s->hop * s->rs, (size_t)b, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return sfail_cuda(e, "stream output");
    if (hc > 0) {  // history <- last 2Gm columns of every row of [history | this step's columns]
      const int64_t nc = b * s->Hn;
      char* dst = static_cast<char*>(s->hy[1 - s->cy]);
      const size_t hp = (size_t)hc * s->es, yp = (size_t)n_cols * s->es;
      if (nc >= hc) {
        e = cudaMemcpy2DAsync(dst, hp, yb + (size_t)(nc - hc) * s->es, yp, hp, (size_t)s->R, cudaMemcpyDeviceToDevice, st);
      } else {
        e = cudaMemcpy2DAsync(dst, hp, static_cast<const char*>(s->hy[s->cy]) + (size_t)nc * s->es, hp,
                              (size_t)(hc - nc) * s->es, (size_t)s->R, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpy2DAsync(dst + (size_t)(hc - nc) * s->es, hp, yb, yp, (size_t)nc * s->es, (size_t)s->R,
                                cudaMemcpyDeviceToDevice, st);
      }
      if (e != cudaSuccess) return sfail_cuda(e, "stream history");
      s->cy = 1 - s->cy;
    }
    s->cpos += b * s->Hn;
    done += b;
  }
  return QTAM_OK;
}

qtam_status qtam_stream_reset(qtam_stream_t s, void* stream) {
  if (!s) return sfail(QTAM_ERR_INVALID_ARG, "stream is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevScope g(s->device);
  const size_t hxb = (size_t)(2 * s->G) * s->rs, hyb = (size_t)s->R * (size_t)(2 * s->Gm) * s->es;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    if (hxb) e = cudaMemsetAsync(s->hx[i], 0, hxb, st);
    if (e == cudaSuccess && hyb) e = cudaMemsetAsync(s->hy[i], 0, hyb, st);
  }
  if (e != cudaSuccess) return sfail_cuda(e, "stream reset");
  s->pos = s->cpos = 0;
  s->cx = s->cy = 0;
  return QTAM_OK;
}

qtam_status qtam_stream_destroy(qtam_stream_t s) {
  if (!s) return QTAM_OK;
  {
    DevScope g(s->device);
    cudaDeviceSynchronize();
  }
  free_stream(s);
  return QTAM_OK;
}

}  // extern "C"
