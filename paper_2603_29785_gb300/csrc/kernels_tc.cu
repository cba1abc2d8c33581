// Tensor-core (tcgen05) kernels: a BF16 GEMM tile check that exercises the
// descriptors, tensor-memory allocation, MMA, commit and loads on their own,
// and the tensor-core short DFT of the forward and inverse row kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <string>

#include "../../include/qtam.h"
#include "qtam_internal.h"
#include "tc_sm100.cuh"

namespace qtam {
namespace {

__device__ int g_tc_timeouts = 0;   // bounded tensor-core waits that ran out (read by qtam_tc_status)

// One CTA of 128 threads: D[128][N] = (+/-A)[128][K] (+/-B)[N][K]^T with A, B
// row-major BF16 in global memory, packed into the core-matrix layout in
// shared memory, one MMA per K = 16, the accumulator in tensor memory.
// flags bit 3 issues no MMA and no commit, so the completion wait runs out
// after wait_cycles: the timeout path (counter, TMEM freed, clean return).
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm_check(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, float* __restrict__ D, int N,
                    int K, uint32_t flags, long long wait_cycles) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  unsigned char* sA = sm;
  unsigned char* sB = sm + 128 * K * 2;
  const int K8 = K >> 3;
  if (flags & 4u) {   // A in the M-major layout: 8 consecutive rows of one column per 16 bytes
    for (int ch = threadIdx.x; ch < 16 * K; ch += blockDim.x) {
      const int k = ch / 16, g = ch - k * 16;
      __align__(16) uint16_t v[8];
      for (int i = 0; i < 8; ++i) v[i] = A[(size_t)(8 * g + i) * K + k];
      *reinterpret_cast<uint4*>(sA + tc::cm_offset_mn(8 * g, k, K)) = *reinterpret_cast<const uint4*>(v);
    }
  } else {
    for (int ch = threadIdx.x; ch < 128 * K8; ch += blockDim.x) {
      const int row = ch / K8, k8 = ch - row * K8;
      *reinterpret_cast<uint4*>(sA + tc::cm_offset(row, k8 * 8, K)) =
          *reinterpret_cast<const uint4*>(A + (size_t)row * K + k8 * 8);
    }
  }
  for (int ch = threadIdx.x; ch < N * K8; ch += blockDim.x) {
    const int row = ch / K8, k8 = ch - row * K8;
    *reinterpret_cast<uint4*>(sB + tc::cm_offset(row, k8 * 8, K)) =
        *reinterpret_cast<const uint4*>(B + (size_t)row * K + k8 * 8);
  }
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tslot, ncols);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tslot;
  const bool issue = !(flags & 8u);
  if (threadIdx.x == 0 && issue) {
    const uint32_t idesc = tc::make_idesc_bf16(128, N, flags & 1u, flags & 2u, flags & 4u);
    const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB), sbo = (uint32_t)K8 * 128u;
    for (int s = 0; s < K / 16; ++s)
      tc::mma_bf16(tbase, tc::make_sdesc(a0 + 256u * s, 128u, sbo), tc::make_sdesc(b0 + 256u * s, 128u, sbo), idesc,
                   s > 0);
    tc::mma_commit(&mbar);
  }
  bool ok = tc::mbar_wait_bounded(&mbar, 0, wait_cycles);
  tc::fence_after_sync();
  if (ok) {
    const int row = threadIdx.x;   // warp w reads lanes 32w .. 32w+31
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) D[(size_t)row * N + c0 + j] = v[j];
    }
  } else {
    if (threadIdx.x == 0) atomicAdd(&g_tc_timeouts, 1);
    if (issue) tc::mbar_wait_bounded(&mbar, 0, wait_cycles);   // give an MMA still in flight a last chance
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// ---- tensor-core short DFT of the row kernels (M = 8192 = 64 x 128) ----------
//
// Forward rows (steps a2-a4), two rows per CTA iteration.  With j = 128 j1 +
// j2 and n = n1 + 64 n2 the length-8192 inverse DFT of the windowed band Z
// factors into (four-step):
//   D[n1][j2]  = sum_j1 e^{+2 pi i j1 n1/64} Z[128 j1 + j2]     GEMM A (tensor cores)
//   D'[n1][j2] = D[n1][j2] e^{+2 pi i j2 n1/8192}               twiddle (FP32, CUDA cores)
//   Y[n1+64n2] = sum_j2 D'[n1][j2] e^{+2 pi i j2 n2/128}        GEMM B (tensor cores)
// Complex products are real GEMMs on (re, im) blocks with BF16 operands and
// FP32 accumulation in tensor memory:
//   GEMM A (one per row r of the pair): M = 128 (j2), K = 128 (j1 of Re Z,
//           j1 of Im Z), N = 128 (Re D for n1 < 64, Im D); A = Z^T written by
//           the band gather, B = the DFT-64 block matrix (constant).  A lane
//           (thread) of the result holds whole complex values D[n1][j2].
//   GEMM B: M = 128 rows (64 r + n1), K = 128 per part, N = 128 + 128
//           (Re Y, Im Y): Re Y = Re D' Gr - Im D' Gi, Im Y = Re D' Gi + Im D' Gr
//           with Gr, Gi the cosine / sine DFT-128 matrices (constant, the
//           minus sign through the MMA's negate-A bit); D' is stored M-major,
//           so the thread owning column j2 writes 8 rows per 16-byte store.
// Shared memory: DFT-64 block 32 KB, Gr 32 KB, Gi 32 KB, a 64 KB buffer for
// Z and one for D'.  Tensor memory: 512 columns, D of row r in 128 r ..
// 128 r + 127, Y in 256..511.
// Pipeline per pair i: GEMM A(i) runs while the CUDA cores store the
// envelopes of pair i-1 from the Y columns; the twiddle pass turns D into D';
// GEMM B(i) runs while the CUDA cores gather pair i+1 into Z.
constexpr int kTcM = 8192;
constexpr int kTcThreads = 512;
constexpr size_t kTcSmem = 7 * 32768;   // constants (96 KB) + Z buffer (64 KB) + D' buffer (64 KB)

template <int E> struct TcEnv;
template <> struct TcEnv<ENV_F32> {
  using S = float2;
  __device__ static S to(float a, float b) { return make_float2(a, b); }
};
template <> struct TcEnv<ENV_BF16> {
  using S = __nv_bfloat162;
  __device__ static S to(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <> struct TcEnv<ENV_F16> {
  using S = __half2;
  __device__ static S to(float a, float b) { return __floats2half2_rn(a, b); }
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Per-row metadata of a pair (a four-slot ring in shared memory, filled two
// pairs ahead by threads 0 and 1): the unit's validity and envelope offset
// and the band parameters, so that the band gather (forward), the envelope
// loads and the accumulation (inverse) start without dependent reads of the
// row list and the row table.
struct TcMeta {
  long long yoff;   // (seg * n_rows + row) * M (forward: 0), or -1 when the pair has no such unit
  long long aoff;   // seg * Nr + k_c: the row's centre bin in the spectrum
  int h, woff, dhi, mlo;
  float kw, cw;     // kw and c of the direction (forward kw_fwd, c_fwd; inverse kw_inv, c_inv)
};

// the row-list read of unit (pair pk, row r): first step of a metadata fill
__device__ __forceinline__ bool tc_meta_unit(int64_t pk, int r, int64_t n_pairs, int64_t n_units, int n_sel,
                                             const int* __restrict__ row_list, int64_t& seg, int& row) {
  const int64_t u = 2 * pk + r;
  if (pk >= n_pairs || u >= n_units) return false;
  seg = u / n_sel;
  row = row_list[u - seg * n_sel];
  return true;
}
__device__ __forceinline__ TcMeta tc_meta_make(bool valid, int64_t seg, int row, const RowDev<float>& rd, int n_rows,
                                               int64_t Nr, bool inv) {
  TcMeta m;
  m.yoff = valid ? (inv ? (seg * n_rows + row) * (int64_t)kTcM : 0) : -1;
  m.aoff = seg * Nr + rd.kc;
  m.h = rd.h;
  m.woff = rd.woff;
  m.dhi = (int)min((int64_t)rd.h, Nr - 1 - rd.kc);
  m.mlo = kTcM + max(-rd.h, -rd.kc);
  m.kw = inv ? rd.kw_inv : rd.kw_fwd;
  m.cw = inv ? rd.c_inv : rd.c_fwd;
  return m;
}
// the forward's unit (pair pk, row r): segment and row without a row list
__device__ __forceinline__ bool tc_meta_unit_fwd(int64_t pk, int r, int64_t n_pairs, int64_t n_units, int n_rows,
                                                 int64_t& seg, int& row) {
  const int64_t u = 2 * pk + r;
  if (pk >= n_pairs || u >= n_units) return false;
  seg = u / n_rows;
  row = (int)(u - seg * n_rows);
  return true;
}

// Band gather + window of one pair of rows into Z (GEMM A's B operand,
// [256 c = 128 r + j2][128 k = Re j1 | Im j1]).  Thread (r, j2, h) =
// ((tid >> 7) & 1, tid & 127, tid >> 8) loads Z[r][128 j1 + j2] for j1 in
// 32 h .. 32 h + 31: a warp's loads are 32 consecutive bins, its 16-byte
// stores one core-matrix row each.
__device__ __forceinline__ void tc_fill_z(unsigned char* sZ, const TcMeta* meta, const float2* __restrict__ X,
                                          const float* __restrict__ wtab) {
  const int tid = threadIdx.x;
  const int r = (tid >> 7) & 1, j2 = tid & 127, h0 = 4 * (tid >> 8);
  const TcMeta m = meta[r];
  const bool valid = m.yoff >= 0;
  const int dhi = m.dhi, mlo = m.mlo;
  const float2* Xs = X + m.aoff;
  const bool tab = wtab != nullptr && m.woff >= 0;
  const unsigned c = 128u * r + j2;
#pragma unroll 2
  for (int o = h0; o < h0 + 4; ++o) {
    // octets wholly outside the band (for every lane of the warp) are zeros
    const int jmin = 1024 * o + j2;
    if (!__any_sync(0xffffffffu, valid && (jmin <= dhi || jmin + 896 >= mlo))) {
      *reinterpret_cast<uint4*>(sZ + tc::cm_offset(c, 8 * o, 128)) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(sZ + tc::cm_offset(c, 64 + 8 * o, 128)) = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = 128 * (8 * o + e) + j2;
      const bool lo = j <= dhi, hi = j >= mlo;
      const int d = lo ? j : j - kTcM;
      float2 v = make_float2(0.f, 0.f);
      if (valid && (lo || hi)) v = Xs[d];
      const int a = min(d < 0 ? -d : d, m.h);
      float w;
      if (tab) {
        w = m.cw * wtab[m.woff + a];
      } else {
        const float uu = (float)((m.h - a) * (m.h + a)) * m.kw;
        w = uu * uu;
      }
      re[e] = v.x * w;
      im[e] = v.y * w;
    }
    *reinterpret_cast<uint4*>(sZ + tc::cm_offset(c, 8 * o, 128)) = make_uint4(
        pack_bf16(re[0], re[1]), pack_bf16(re[2], re[3]), pack_bf16(re[4], re[5]), pack_bf16(re[6], re[7]));
    *reinterpret_cast<uint4*>(sZ + tc::cm_offset(c, 64 + 8 * o, 128)) = make_uint4(
        pack_bf16(im[0], im[1]), pack_bf16(im[2], im[3]), pack_bf16(im[4], im[5]), pack_bf16(im[6], im[7]));
  }
}

// Envelopes of pair pr from tensor memory (Re Y in columns 256.., Im Y in
// 384..) to y[u][n1 + 64 n2]; lanes are rows 64 r + n1, so a warp's stores
// are 32 consecutive envelope samples.  Each warp owns 32 values of n2 and
// stores them in two halves (q = q0 .. q1 - 1 of 2), so the kernel can issue
// one half under GEMM A and the other after the twiddle instead of one
// burst of stores from every SM at once.
template <int E>
__device__ __forceinline__ void tc_store_y(uint32_t tbase, int64_t pr, int64_t n_units,
                                           typename TcEnv<E>::S* __restrict__ y, int q0, int q1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q4 = warp & 3, quarter = warp >> 2;   // lane quarter, quarter of the n2 range
  const int r = q4 >> 1, n1 = 32 * (q4 & 1) + lane;
  const int64_t u = 2 * pr + r;
  if (u >= n_units) return;   // r is uniform per warp: whole warps skip the collective loads
  typename TcEnv<E>::S* yu = y + u * kTcM + n1;
  const uint32_t lrow = (uint32_t)(32 * q4) << 16;
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const int n20 = 32 * quarter + 16 * q;
    float vr[16], vi[16];
    tc::tmem_ld16_nowait(tbase + lrow + 256u + (uint32_t)n20, vr);
    tc::tmem_ld16_nowait(tbase + lrow + 384u + (uint32_t)n20, vi);
    tc::tmem_wait_ld(vr, vi);
#pragma unroll
    for (int e = 0; e < 16; ++e) __stcs(yu + 64 * (n20 + e), TcEnv<E>::to(vr[e], vi[e]));
  }
}

template <int E>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_rows_forward_tc(const RowDev<float>* __restrict__ rows, int n_rows, int64_t Nr, const float2* __restrict__ X,
                      typename TcEnv<E>::S* __restrict__ y, int64_t n_units, const uint4* __restrict__ tabA,
                      const uint4* __restrict__ tabG, const float* __restrict__ wtab) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbarA, mbarB;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ TcMeta smeta[4][2];          // pair of iteration i in slot i & 3
  unsigned char* sA = sm;                 // DFT-64 block, [128 n][128 k] K-major (GEMM A's B)
  unsigned char* sGr = sm + 32768;        // [128 n2][128 j2]
  unsigned char* sGi = sm + 65536;
  unsigned char* sZ = sm + 98304;         // Z^T of the next pair: row r at 32 KB r, [128 j2][128 k] K-major
  unsigned char* sDp = sm + 163840;       // D' of the current pair, [128 m][256 k] M-major
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 2048; i += kTcThreads) reinterpret_cast<uint4*>(sA)[i] = tabA[i];
  for (int i = tid; i < 4096; i += kTcThreads) reinterpret_cast<uint4*>(sGr)[i] = tabG[i];
  if (warp == 0) {   // 512 columns: one CTA per SM (the shared memory admits no second one)
    tc::tmem_alloc(&tslot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbarA, 1);
    tc::mbar_init(&mbarB, 1);
    abort_flag = 0;
  }
  // twiddle pass: warp (q4, cg) handles lanes j2 = 32 q4 + lane of row
  // r = cg >> 1, n1 = 32 (cg & 1) .. + 31; the twiddle e^{2 pi i n1 j2 / 8192}
  // is evaluated from the exact integer n1 j2 with the SFU sine/cosine
  // (absolute error ~1e-6, far below the BF16 rounding of the result)
  const int q4 = warp & 3, cg = warp >> 2;
  const int j2 = 32 * q4 + lane, rr = cg >> 1, nb = 32 * (cg & 1);
  constexpr float kAng = 6.28318530717958647692f / (float)kTcM;
  const int64_t n_pairs = (n_units + 1) >> 1;
  int64_t pr = blockIdx.x;
  if (tid < 4) {   // metadata of the first two pairs (iterations 0 and 1)
    const int it = tid >> 1, r = tid & 1;
    int64_t seg = 0;
    int row = 0;
    const bool ok = tc_meta_unit_fwd(pr + it * (int64_t)gridDim.x, r, n_pairs, n_units, n_rows, seg, row);
    smeta[it][r] = tc_meta_make(ok, seg, row, rows[row], n_rows, Nr, false);
  }
  __syncthreads();
  if (pr < n_pairs) tc_fill_z(sZ, smeta[0], X, wtab);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t aA = tc::smem_addr(sA), aGr = tc::smem_addr(sGr), aGi = tc::smem_addr(sGi);
  const uint32_t aZ = tc::smem_addr(sZ), aDp = tc::smem_addr(sDp);
  uint32_t phA = 0, phB = 0;
  bool pendA = false, pendB = false;
  int64_t prev = -1;

  for (int it = 0; pr < n_pairs; pr += gridDim.x, ++it) {
    // metadata of the pair two iterations ahead: the row-table read now, the
    // slot written after the twiddle
    int64_t mseg = 0;
    int mrow = 0;
    bool mok = false;
    RowDev<float> mrd;
    if (tid < 2) {
      mok = tc_meta_unit_fwd(pr + 2 * (int64_t)gridDim.x, tid, n_pairs, n_units, n_rows, mseg, mrow);
      mrd = rows[mrow];
    }
    // ---- GEMM A: D_r[tmem 128 r ..] = Z_r^T * DFT64^T, r = 0, 1 ----
    if (tid == 0) {
      const uint32_t idesc = tc::make_idesc_bf16(128, 128);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int s = 0; s < 8; ++s)
          tc::mma_bf16(tbase + 128u * r, tc::make_sdesc(aZ + 32768u * r + 256u * s, 128u, 2048u),
                       tc::make_sdesc(aA + 256u * s, 128u, 2048u), idesc, s > 0);
      tc::mma_commit(&mbarA);
    }
    pendA = true;
    // ... overlapped with the first half of the previous pair's envelope stores (Y columns are not
    // touched by GEMM A)
    if (prev >= 0) tc_store_y<E>(tbase, prev, n_units, y, 0, 1);
    if (!tc::mbar_wait_bounded(&mbarA, phA, tc::kWaitCycles)) abort_flag = 1;
    tc::fence_after_sync();
    __syncthreads();
    if (abort_flag) break;
    phA ^= 1u;
    pendA = false;
    // ---- twiddle: D -> D' ([128 m = 64 r + n1][256 k = Re j2 | Im j2], M-major) ----
    {
      const uint32_t lrow = (uint32_t)(32 * q4) << 16;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int n10 = nb + 16 * h;
        float vr[16], vi[16];
        tc::tmem_ld16_nowait(tbase + lrow + (uint32_t)(128 * rr + n10), vr);
        tc::tmem_ld16_nowait(tbase + lrow + (uint32_t)(128 * rr + 64 + n10), vi);
        tc::tmem_wait_ld(vr, vi);
        float orr[16], oi[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float ty, tx;
          __sincosf(kAng * (float)((n10 + e) * j2), &ty, &tx);
          orr[e] = fmaf(vr[e], tx, -vi[e] * ty);
          oi[e] = fmaf(vr[e], ty, vi[e] * tx);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int m0 = 64 * rr + n10 + 8 * g;
          *reinterpret_cast<uint4*>(sDp + tc::cm_offset_mn(m0, j2, 256)) =
              make_uint4(pack_bf16(orr[8 * g], orr[8 * g + 1]), pack_bf16(orr[8 * g + 2], orr[8 * g + 3]),
                         pack_bf16(orr[8 * g + 4], orr[8 * g + 5]), pack_bf16(orr[8 * g + 6], orr[8 * g + 7]));
          *reinterpret_cast<uint4*>(sDp + tc::cm_offset_mn(m0, 128 + j2, 256)) =
              make_uint4(pack_bf16(oi[8 * g], oi[8 * g + 1]), pack_bf16(oi[8 * g + 2], oi[8 * g + 3]),
                         pack_bf16(oi[8 * g + 4], oi[8 * g + 5]), pack_bf16(oi[8 * g + 6], oi[8 * g + 7]));
        }
      }
    }
    // the second half of the previous pair's stores, before GEMM B overwrites the Y columns
    if (prev >= 0) tc_store_y<E>(tbase, prev, n_units, y, 1, 2);
    if (tid < 2) smeta[(it + 2) & 3][tid] = tc_meta_make(mok, mseg, mrow, mrd, n_rows, Nr, false);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- GEMM B: Re Y [tmem 256..383], Im Y [384..511] ----
    if (tid == 0) {
      const uint32_t id = tc::make_idesc_bf16(128, 128, false, false, true),
                     idn = tc::make_idesc_bf16(128, 128, true, false, true);   // D' is M-major
      const uint32_t tRe = tbase + 256u, tIm = tbase + 384u;
#pragma unroll
      for (int s = 0; s < 8; ++s) {   // Re D' * Gr, Re D' * Gi
        const uint64_t a = tc::make_sdesc(aDp + 256u * s, 128u, 4096u);
        tc::mma_bf16(tRe, a, tc::make_sdesc(aGr + 256u * s, 128u, 2048u), id, s > 0);
        tc::mma_bf16(tIm, a, tc::make_sdesc(aGi + 256u * s, 128u, 2048u), id, s > 0);
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {   // - Im D' * Gi, + Im D' * Gr
        const uint64_t a = tc::make_sdesc(aDp + 256u * (8 + s), 128u, 4096u);
        tc::mma_bf16(tRe, a, tc::make_sdesc(aGi + 256u * s, 128u, 2048u), idn, 1u);
        tc::mma_bf16(tIm, a, tc::make_sdesc(aGr + 256u * s, 128u, 2048u), id, 1u);
      }
      tc::mma_commit(&mbarB);
    }
    pendB = true;
    // ... overlapped with the next pair's band gather (GEMM A has finished reading Z)
    const int64_t nx = pr + gridDim.x;
    if (nx < n_pairs) tc_fill_z(sZ, smeta[(it + 1) & 3], X, wtab);
    if (!tc::mbar_wait_bounded(&mbarB, phB, tc::kWaitCycles)) abort_flag = 1;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_flag) break;
    phB ^= 1u;
    pendB = false;
    prev = pr;
  }
  if (!abort_flag && prev >= 0) tc_store_y<E>(tbase, prev, n_units, y, 0, 2);
  if (abort_flag) {
    if (tid == 0) atomicAdd(&g_tc_timeouts, 1);
    if (pendA) tc::mbar_wait_bounded(&mbarA, phA, tc::kWaitCycles);
    if (pendB) tc::mbar_wait_bounded(&mbarB, phB, tc::kWaitCycles);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// ---- tensor-core analysis DFT of the inverse rows (M = 8192) -----------------
//
// Inverse rows (steps a5-a6), two rows per CTA iteration.  The synthesis
// needs S[j] = sum_n y[n] e^{-2 pi i j n/8192} of each envelope row; with
// n = n1 + 64 n2 and j = 128 j1 + j2 it factors into
//   E[n1][j2]      = sum_n2 y[n1 + 64 n2] e^{-2 pi i j2 n2/128}   GEMM B' (tensor cores)
//   E'[n1][j2]     = E[n1][j2] e^{-2 pi i j2 n1/8192}             twiddle (FP32)
//   S[128 j1 + j2] = sum_n1 E'[n1][j2] e^{-2 pi i j1 n1/64}       GEMM A' (tensor cores)
// and the band accumulation A[k_c + d] += c_k sqrt(N/M) W'(d) S[d mod M] for
// |d| <= h (the weight c_inv W').
//   GEMM B' (the pair): M = 128 rows (64 r + n1), K = 128 + 128 (Re y, Im y
//           over n2), N = 128 + 128: Re E = Re y Gr + Im y Gi, Im E = Im y Gr
//           - Re y Gi (the minus sign through the negate-A bit).  The
//           envelopes are the M-major A operand: 8 consecutive samples n1 of
//           one n2 fill one 16-byte row of a core matrix.
//   GEMM A' (per row r): M = 128 (j2), K = 128 (Re E', Im E' over n1), N =
//           128 (Re S, Im S over j1); E'^T is the M-major A operand written
//           by the twiddle pass, B the conjugate DFT-64 block matrix.  A lane
//           of the result holds S at bins j2 + 128 j1, so a warp's reductions
//           go to 32 consecutive bins.
// Shared memory: conjugate DFT-64 block 32 KB, Gr 32 KB, Gi 32 KB, 64 KB for
// the next pair's envelopes, 64 KB for E'^T.  Tensor memory: S of row r in
// 128 r .. 128 r + 127, E in 256..511.
// Pipeline per pair i: GEMM B'(i) runs while the CUDA cores accumulate pair
// i-1 from the S columns; GEMM A'(i) runs while they store pair i+1's
// envelopes into sY, whose loads were issued under the earlier phases.

// 8 consecutive complex envelope samples (16-byte aligned): load() issues the
// 16-byte loads, pack() turns them into 8 BF16 real parts and 8 BF16
// imaginary parts, packed in order
template <int E> struct TcLoad;
template <> struct TcLoad<ENV_F32> {
  struct Raw { float4 v[4]; };
  __device__ static void load(const float2* p, Raw& w) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int t = 0; t < 4; ++t) w.v[t] = __ldcs(q + t);
  }
  __device__ static void pack(const Raw& w, uint4& re, uint4& im) {
    re = make_uint4(pack_bf16(w.v[0].x, w.v[0].z), pack_bf16(w.v[1].x, w.v[1].z), pack_bf16(w.v[2].x, w.v[2].z),
                    pack_bf16(w.v[3].x, w.v[3].z));
    im = make_uint4(pack_bf16(w.v[0].y, w.v[0].w), pack_bf16(w.v[1].y, w.v[1].w), pack_bf16(w.v[2].y, w.v[2].w),
                    pack_bf16(w.v[3].y, w.v[3].w));
  }
};
template <> struct TcLoad<ENV_BF16> {   // already BF16: regroup the halves, no rounding
  struct Raw { uint4 v[2]; };
  __device__ static void load(const __nv_bfloat162* p, Raw& w) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    w.v[0] = __ldcs(q);
    w.v[1] = __ldcs(q + 1);
  }
  __device__ static void pack(const Raw& w, uint4& re, uint4& im) {
    const uint4 a = w.v[0], b = w.v[1];
    re = make_uint4(__byte_perm(a.x, a.y, 0x5410), __byte_perm(a.z, a.w, 0x5410), __byte_perm(b.x, b.y, 0x5410),
                    __byte_perm(b.z, b.w, 0x5410));
    im = make_uint4(__byte_perm(a.x, a.y, 0x7632), __byte_perm(a.z, a.w, 0x7632), __byte_perm(b.x, b.y, 0x7632),
                    __byte_perm(b.z, b.w, 0x7632));
  }
};
template <> struct TcLoad<ENV_F16> {
  struct Raw { uint4 v[2]; };
  __device__ static void load(const __half2* p, Raw& w) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    w.v[0] = __ldcs(q);
    w.v[1] = __ldcs(q + 1);
  }
  __device__ static void pack(const Raw& w, uint4& re, uint4& im) {
    const uint32_t u[8] = {w.v[0].x, w.v[0].y, w.v[0].z, w.v[0].w, w.v[1].x, w.v[1].y, w.v[1].z, w.v[1].w};
    uint32_t rr[4], ii[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u[2 * t]));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u[2 * t + 1]));
      rr[t] = pack_bf16(a.x, b.x);
      ii[t] = pack_bf16(a.y, b.y);
    }
    re = make_uint4(rr[0], rr[1], rr[2], rr[3]);
    im = make_uint4(ii[0], ii[1], ii[2], ii[3]);
  }
};

// *p += v when `on` (one predicated vector reduction; A is not read here)
__device__ __forceinline__ void red_add_if(float2* p, float v0, float v1, bool on) {
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %3, 0; @q red.global.add.v2.f32 [%0], {%1, %2}; }" ::"l"(p), "f"(v0),
               "f"(v1), "r"((int)on));
}

// Envelopes of pair pr into sY ([128 m = 64 r + n1][256 k = Re n2 | Im n2],
// M-major), one row r at a time: tc_load_row issues the loads into
// registers, tc_store_row packs and stores them, so the loads can be in
// flight while other work runs.  Item (r, n2, octet o) holds samples 8 o +
// 64 n2 .. + 7; the 8 lanes of a quarter warp take 8 consecutive n2 of one
// octet, so their 16-byte stores fill one core matrix (no bank conflicts)
// and each lane reads whole 32-byte sectors.
template <int E>
__device__ __forceinline__ void tc_load_row(const typename TcEnv<E>::S* yr, typename TcLoad<E>::Raw (&raw)[2]) {
  if (!yr) return;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int i = threadIdx.x + kTcThreads * t;   // 0 .. 1023
    TcLoad<E>::load(yr + 8 * ((i >> 3) & 7) + 64 * ((i & 7) + 8 * (i >> 6)), raw[t]);
  }
}

template <int E>
__device__ __forceinline__ void tc_store_row(unsigned char* sY, int r, bool valid,
                                             const typename TcLoad<E>::Raw (&raw)[2]) {
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int i = threadIdx.x + kTcThreads * t;
    const int n2 = (i & 7) + 8 * (i >> 6), o = (i >> 3) & 7;
    uint4 re = make_uint4(0u, 0u, 0u, 0u), im = re;
    if (valid) TcLoad<E>::pack(raw[t], re, im);
    const int m = 64 * r + 8 * o;
    *reinterpret_cast<uint4*>(sY + tc::cm_offset_mn(m, n2, 256)) = re;
    *reinterpret_cast<uint4*>(sY + tc::cm_offset_mn(m, 128 + n2, 256)) = im;
  }
}

// Band accumulation of a pair from tensor memory (S of row r in columns
// 128 r: Re over j1, 128 r + 64: Im), its rows described by meta[0..1].
// Warp (q4, quarter) reads lanes j2 = 32 q4 + lane of row r = quarter >> 1,
// j1 in 32 (quarter & 1) .. + 31; blocks of 16 j1 wholly outside the band
// are skipped by the whole warp.
__device__ __forceinline__ void tc_accumulate(uint32_t tbase, const TcMeta* meta, float2* __restrict__ A,
                                              const float* __restrict__ wtab) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q4 = warp & 3, quarter = warp >> 2;
  const int r = quarter >> 1, jb = 32 * (quarter & 1), j2 = 32 * q4 + lane;
  const TcMeta m = meta[r];
  if (m.yoff < 0) return;   // r is uniform per warp
  float2* As = A + m.aoff;
  const bool tab = wtab != nullptr && m.woff >= 0;
  const float h2 = (float)m.h * (float)m.h;   // exact: h < 4096
  const uint32_t lrow = (uint32_t)(32 * q4) << 16;
#pragma unroll 1
  for (int q = 0; q < 2; ++q) {
    const int j10 = jb + 16 * q;
    if (!(128 * j10 + 32 * q4 <= m.dhi || 128 * (j10 + 15) + 32 * q4 + 31 >= m.mlo)) continue;
    float vr[16], vi[16];
    tc::tmem_ld16_nowait(tbase + lrow + (uint32_t)(128 * r + j10), vr);
    tc::tmem_ld16_nowait(tbase + lrow + (uint32_t)(128 * r + 64 + j10), vi);
    tc::tmem_wait_ld(vr, vi);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int j = 128 * (j10 + e) + j2;
      const bool lo = j <= m.dhi, hi = j >= m.mlo;
      const int d = lo ? j : j - kTcM;
      float w;
      if (tab) {
        w = m.cw * wtab[m.woff + min(d < 0 ? -d : d, m.h)];
      } else {
        const float df = (float)d;
        const float t = (h2 - df * df) * m.kw;
        w = t * t;
      }
      red_add_if(As + d, vr[e] * w, vi[e] * w, lo || hi);
    }
  }
}

template <int E>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_rows_inverse_tc(const RowDev<float>* __restrict__ rows, const int* __restrict__ row_list, int n_sel, int n_rows,
                      int64_t Nr, const typename TcEnv<E>::S* __restrict__ y, float2* __restrict__ A, int64_t n_units,
                      const uint4* __restrict__ tabAi, const uint4* __restrict__ tabG, const float* __restrict__ wtab) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbarA, mbarB;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ TcMeta smeta[4][2];      // pair of iteration i in slot i & 3
  unsigned char* sAi = sm;            // conjugate DFT-64 block, [128 n][128 k] K-major (GEMM A''s B)
  unsigned char* sGr = sm + 32768;    // [128 j2][128 n2]
  unsigned char* sGi = sm + 65536;
  unsigned char* sY = sm + 98304;     // envelopes of the next pair, [128 m][256 k] M-major
  unsigned char* sE = sm + 163840;    // E'^T of the current pair: row r at 32 KB r, [128 j2][128 k] M-major
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 2048; i += kTcThreads) reinterpret_cast<uint4*>(sAi)[i] = tabAi[i];
  for (int i = tid; i < 4096; i += kTcThreads) reinterpret_cast<uint4*>(sGr)[i] = tabG[i];
  if (warp == 0) {
    tc::tmem_alloc(&tslot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbarA, 1);
    tc::mbar_init(&mbarB, 1);
    abort_flag = 0;
  }
  // twiddle pass: warp (q4, cg) takes lanes m = 32 q4 + lane = 64 r + n1 and
  // columns j2 in 32 cg .. 32 cg + 31; e^{-2 pi i n1 j2 / 8192} from the
  // exact integer n1 j2 with the SFU sine/cosine
  const int q4 = warp & 3, cg = warp >> 2;
  const int m = 32 * q4 + lane, rr = m >> 6, n1 = m & 63;
  constexpr float kAng = 6.28318530717958647692f / (float)kTcM;
  const int64_t n_pairs = (n_units + 1) >> 1;
  int64_t pr = blockIdx.x;
  // metadata of the first two pairs (iterations 0 and 1)
  if (tid < 4) {
    const int it = tid >> 1, r = tid & 1;
    int64_t seg = 0;
    int row = 0;
    const bool ok = tc_meta_unit(pr + it * (int64_t)gridDim.x, r, n_pairs, n_units, n_sel, row_list, seg, row);
    smeta[it][r] = tc_meta_make(ok, seg, row, rows[ok ? row : 0], n_rows, Nr, true);
  }
  __syncthreads();
  typename TcLoad<E>::Raw raw[2];
  if (pr < n_pairs) {
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      const long long yo = smeta[0][r].yoff;
      const typename TcEnv<E>::S* yr = yo >= 0 ? y + yo : nullptr;
      tc_load_row<E>(yr, raw);
      tc_store_row<E>(sY, r, yr != nullptr, raw);
    }
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t aAi = tc::smem_addr(sAi), aGr = tc::smem_addr(sGr), aGi = tc::smem_addr(sGi);
  const uint32_t aY = tc::smem_addr(sY), aE = tc::smem_addr(sE);
  uint32_t phA = 0, phB = 0;
  bool pendA = false, pendB = false;
  int prev_slot = -1;

  for (int it = 0; pr < n_pairs; pr += gridDim.x, ++it) {
    // ---- GEMM B': Re E [tmem 256..383], Im E [384..511] ----
    if (tid == 0) {
      const uint32_t id = tc::make_idesc_bf16(128, 128, false, false, true),
                     idn = tc::make_idesc_bf16(128, 128, true, false, true);   // y is M-major
      const uint32_t tRe = tbase + 256u, tIm = tbase + 384u;
#pragma unroll
      for (int s = 0; s < 8; ++s) {   // + Re y * Gr, - Re y * Gi
        const uint64_t a = tc::make_sdesc(aY + 256u * s, 128u, 4096u);
        tc::mma_bf16(tRe, a, tc::make_sdesc(aGr + 256u * s, 128u, 2048u), id, s > 0);
        tc::mma_bf16(tIm, a, tc::make_sdesc(aGi + 256u * s, 128u, 2048u), idn, s > 0);
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {   // + Im y * Gi, + Im y * Gr
        const uint64_t a = tc::make_sdesc(aY + 256u * (8 + s), 128u, 4096u);
        tc::mma_bf16(tRe, a, tc::make_sdesc(aGi + 256u * s, 128u, 2048u), id, 1u);
        tc::mma_bf16(tIm, a, tc::make_sdesc(aGr + 256u * s, 128u, 2048u), id, 1u);
      }
      tc::mma_commit(&mbarB);
    }
    pendB = true;
    // The next pair's envelopes are loaded a row at a time, each row's loads
    // in flight under other work (all CTAs would otherwise load at once and
    // leave the memory idle between bursts): row 0 under the accumulation
    // below, stored once GEMM B' has released sY; row 1 under the twiddle,
    // stored under GEMM A'.
    const int64_t nx = pr + gridDim.x;
    const long long yo0 = smeta[(it + 1) & 3][0].yoff, yo1 = smeta[(it + 1) & 3][1].yoff;
    const typename TcEnv<E>::S* ynx0 = nx < n_pairs && yo0 >= 0 ? y + yo0 : nullptr;
    const typename TcEnv<E>::S* ynx1 = nx < n_pairs && yo1 >= 0 ? y + yo1 : nullptr;
    // metadata of the pair two iterations ahead: the row-list read now, the
    // row-table read after GEMM B', the slot written after the twiddle
    int64_t mseg = 0;
    int mrow = 0;
    bool mok = false;
    if (tid < 2) mok = tc_meta_unit(pr + 2 * (int64_t)gridDim.x, tid, n_pairs, n_units, n_sel, row_list, mseg, mrow);
    tc_load_row<E>(ynx0, raw);
    // ... overlapped with the previous pair's band accumulation (S columns are not touched by GEMM B')
    if (prev_slot >= 0) tc_accumulate(tbase, smeta[prev_slot], A, wtab);
    if (!tc::mbar_wait_bounded(&mbarB, phB, tc::kWaitCycles)) abort_flag = 1;
    tc::fence_after_sync();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_flag) break;
    phB ^= 1u;
    pendB = false;
    RowDev<float> mrd;
    if (tid < 2) mrd = rows[mok ? mrow : 0];
    if (nx < n_pairs) tc_store_row<E>(sY, 0, ynx0 != nullptr, raw);
    tc_load_row<E>(ynx1, raw);
    // ---- twiddle: E -> E'^T (row rr at 32 KB rr, [128 j2][128 k = Re n1 | Im n1], M-major) ----
    {
      const uint32_t lrow = (uint32_t)(32 * q4) << 16;
      unsigned char* sEr = sE + 32768 * rr;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int j20 = 32 * cg + 16 * h;
        float vr[16], vi[16];
        tc::tmem_ld16_nowait(tbase + lrow + 256u + (uint32_t)j20, vr);
        tc::tmem_ld16_nowait(tbase + lrow + 384u + (uint32_t)j20, vi);
        tc::tmem_wait_ld(vr, vi);
        float orr[16], oi[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float ts, tcs;
          __sincosf(kAng * (float)(n1 * (j20 + e)), &ts, &tcs);
          orr[e] = fmaf(vr[e], tcs, vi[e] * ts);
          oi[e] = fmaf(vi[e], tcs, -vr[e] * ts);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int jg = j20 + 8 * g;
          *reinterpret_cast<uint4*>(sEr + tc::cm_offset_mn(jg, n1, 128)) =
              make_uint4(pack_bf16(orr[8 * g], orr[8 * g + 1]), pack_bf16(orr[8 * g + 2], orr[8 * g + 3]),
                         pack_bf16(orr[8 * g + 4], orr[8 * g + 5]), pack_bf16(orr[8 * g + 6], orr[8 * g + 7]));
          *reinterpret_cast<uint4*>(sEr + tc::cm_offset_mn(jg, 64 + n1, 128)) =
              make_uint4(pack_bf16(oi[8 * g], oi[8 * g + 1]), pack_bf16(oi[8 * g + 2], oi[8 * g + 3]),
                         pack_bf16(oi[8 * g + 4], oi[8 * g + 5]), pack_bf16(oi[8 * g + 6], oi[8 * g + 7]));
        }
      }
    }
    if (tid < 2) smeta[(it + 2) & 3][tid] = tc_meta_make(mok, mseg, mrow, mrd, n_rows, Nr, true);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- GEMM A': S_r [tmem 128 r ..] = E'_r^T * conj(DFT64)^T, r = 0, 1 ----
    if (tid == 0) {
      const uint32_t idesc = tc::make_idesc_bf16(128, 128, false, false, true);   // E'^T is M-major
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int s = 0; s < 8; ++s)
          tc::mma_bf16(tbase + 128u * r, tc::make_sdesc(aE + 32768u * r + 256u * s, 128u, 2048u),
                       tc::make_sdesc(aAi + 256u * s, 128u, 2048u), idesc, s > 0);
      tc::mma_commit(&mbarA);
    }
    pendA = true;
    // ... overlapped with the store of the next pair's row 1 (GEMM B' has finished reading sY)
    if (nx < n_pairs) tc_store_row<E>(sY, 1, ynx1 != nullptr, raw);
    if (!tc::mbar_wait_bounded(&mbarA, phA, tc::kWaitCycles)) abort_flag = 1;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_flag) break;
    phA ^= 1u;
    pendA = false;
    prev_slot = it & 3;
  }
  if (!abort_flag && prev_slot >= 0) tc_accumulate(tbase, smeta[prev_slot], A, wtab);
  if (abort_flag) {
    if (tid == 0) atomicAdd(&g_tc_timeouts, 1);
    if (pendA) tc::mbar_wait_bounded(&mbarA, phA, tc::kWaitCycles);
    if (pendB) tc::mbar_wait_bounded(&mbarB, phB, tc::kWaitCycles);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

}  // namespace

bool tc_forward_supported(int M) { return M == kTcM; }

cudaError_t launch_rows_forward_tc(const RowCfg& c, const RowDev<float>* rows, int n_rows, int64_t Nr,
                                   const float2* X, void* y, int env, int64_t B, cudaStream_t st, const float* wtab) {
  const int64_t units = B * n_rows;
  if (units == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t pairs = (units + 1) / 2;
  const unsigned grid = (unsigned)std::min<int64_t>(pairs, (int64_t)std::max(sms, 1));
  const uint4* A = static_cast<const uint4*>(c.tcA);
  const uint4* G = static_cast<const uint4*>(c.tcG);
  cudaError_t e;
  switch (env) {
    case ENV_BF16:
      if ((e = allow_smem((const void*)k_rows_forward_tc<ENV_BF16>, kTcSmem)) != cudaSuccess) return e;
      k_rows_forward_tc<ENV_BF16><<<grid, kTcThreads, kTcSmem, st>>>(
          rows, n_rows, Nr, X, static_cast<__nv_bfloat162*>(y), units, A, G, wtab);
      break;
    case ENV_F16:
      if ((e = allow_smem((const void*)k_rows_forward_tc<ENV_F16>, kTcSmem)) != cudaSuccess) return e;
      k_rows_forward_tc<ENV_F16><<<grid, kTcThreads, kTcSmem, st>>>(rows, n_rows, Nr, X, static_cast<__half2*>(y),
                                                                    units, A, G, wtab);
      break;
    default:
      if ((e = allow_smem((const void*)k_rows_forward_tc<ENV_F32>, kTcSmem)) != cudaSuccess) return e;
      k_rows_forward_tc<ENV_F32><<<grid, kTcThreads, kTcSmem, st>>>(rows, n_rows, Nr, X, static_cast<float2*>(y),
                                                                    units, A, G, wtab);
  }
  return cudaGetLastError();
}


bool launch_rows_inverse_tc(const RowCfg& c, const RowDev<float>* rows, const int* row_list, int n_sel, int n_rows,
                            int64_t Nr, const void* y, int env, float2* A, int64_t B, cudaStream_t st,
                            const float* wtab, cudaError_t* err) {
  *err = cudaSuccess;
  if (!c.tcAi || (reinterpret_cast<uintptr_t>(y) & 15)) return false;   // 16-byte envelope loads
  const int64_t units = B * n_sel;
  if (units == 0) return true;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t pairs = (units + 1) / 2;
  const unsigned grid = (unsigned)std::min<int64_t>(pairs, (int64_t)std::max(sms, 1));
  const uint4* Ai = static_cast<const uint4*>(c.tcAi);
  const uint4* G = static_cast<const uint4*>(c.tcG);
  cudaError_t e;
  switch (env) {
    case ENV_BF16:
      if ((e = allow_smem((const void*)k_rows_inverse_tc<ENV_BF16>, kTcSmem)) != cudaSuccess) break;
      k_rows_inverse_tc<ENV_BF16><<<grid, kTcThreads, kTcSmem, st>>>(
          rows, row_list, n_sel, n_rows, Nr, static_cast<const __nv_bfloat162*>(y), A, units, Ai, G, wtab);
      e = cudaGetLastError();
      break;
    case ENV_F16:
      if ((e = allow_smem((const void*)k_rows_inverse_tc<ENV_F16>, kTcSmem)) != cudaSuccess) break;
      k_rows_inverse_tc<ENV_F16><<<grid, kTcThreads, kTcSmem, st>>>(
          rows, row_list, n_sel, n_rows, Nr, static_cast<const __half2*>(y), A, units, Ai, G, wtab);
      e = cudaGetLastError();
      break;
    default:
      if ((e = allow_smem((const void*)k_rows_inverse_tc<ENV_F32>, kTcSmem)) != cudaSuccess) break;
      k_rows_inverse_tc<ENV_F32><<<grid, kTcThreads, kTcSmem, st>>>(
          rows, row_list, n_sel, n_rows, Nr, static_cast<const float2*>(y), A, units, Ai, G, wtab);
      e = cudaGetLastError();
  }
  *err = e;
  return true;
}

}  // namespace qtam

extern "C" {

qtam_status qtam_tc_gemm_check(const void* A, const void* B, float* D, int32_t N, int32_t K, int32_t flags,
                               void* stream) {
  if (!A || !B || !D) {
    qtam::set_last_error("NULL buffer");
    return QTAM_ERR_INVALID_ARG;
  }
  if (N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16 || (flags & ~15)) {
    qtam::set_last_error("N and K must be multiples of 16 in [16, 256]; flags in {0..15}");
    return QTAM_ERR_INVALID_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) {
    qtam::set_last_error("A and B must be 16-byte aligned");
    return QTAM_ERR_INVALID_ARG;
  }
  // operands plus 32 KB of slack past B, so no descriptor reading of a
  // mis-sized operand can leave the CTA's shared memory
  const size_t smem = (size_t)(128 + N) * K * 2 + 32768;
  cudaError_t e = qtam::allow_smem((const void*)qtam::k_tc_gemm_check, smem);
  if (e == cudaSuccess) {
    const long long wait_cycles = (flags & 8) ? 2000000LL : qtam::tc::kWaitCycles;   // ~1 ms for the timeout test
    qtam::k_tc_gemm_check<<<1, 128, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint16_t*>(A), static_cast<const uint16_t*>(B), D, N, K, (uint32_t)flags, wait_cycles);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    qtam::set_last_error(std::string("tc gemm check: ") + cudaGetErrorString(e));
    return QTAM_ERR_CUDA;
  }
  return QTAM_OK;
}

qtam_status qtam_tc_status(int32_t* timeouts) {
  if (!timeouts) {
    qtam::set_last_error("NULL argument");
    return QTAM_ERR_INVALID_ARG;
  }
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, qtam::g_tc_timeouts, sizeof(int));
  if (e != cudaSuccess) {
    qtam::set_last_error(std::string("tc status: ") + cudaGetErrorString(e));
    return QTAM_ERR_CUDA;
  }
  *timeouts = v;
  return QTAM_OK;
}

}  // extern "C"
