// Tensor-core (tcgen05) kernels: a BF16 GEMM tile check that exercises the
// descriptors, tensor-memory allocation, MMA, commit and loads on their own,
// and the tensor-core short DFT of the row kernels.
#include <cuda_bf16.h>

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
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm_check(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, float* __restrict__ D, int N,
                    int K, uint32_t flags) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  unsigned char* sA = sm;
  unsigned char* sB = sm + 128 * K * 2;
  const int K8 = K >> 3;
  for (int ch = threadIdx.x; ch < 128 * K8; ch += blockDim.x) {
    const int row = ch / K8, k8 = ch - row * K8;
    *reinterpret_cast<uint4*>(sA + tc::cm_offset(row, k8 * 8, K)) =
        *reinterpret_cast<const uint4*>(A + (size_t)row * K + k8 * 8);
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
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::make_idesc_bf16(128, N, flags & 1u, flags & 2u);
    const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB), sbo = (uint32_t)K8 * 128u;
    for (int s = 0; s < K / 16; ++s)
      tc::mma_bf16(tbase, tc::make_sdesc(a0 + 256u * s, 128u, sbo), tc::make_sdesc(b0 + 256u * s, 128u, sbo), idesc,
                   s > 0);
    tc::mma_commit(&mbar);
  }
  bool ok = tc::mbar_wait_bounded(&mbar, 0, tc::kWaitCycles);
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
    tc::mbar_wait_bounded(&mbar, 0, tc::kWaitCycles);   // give an MMA still in flight a last chance
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

}  // namespace
}  // namespace qtam

extern "C" {

qtam_status qtam_tc_gemm_check(const void* A, const void* B, float* D, int32_t N, int32_t K, int32_t flags,
                               void* stream) {
  if (!A || !B || !D) {
    qtam::set_last_error("NULL buffer");
    return QTAM_ERR_INVALID_ARG;
  }
  if (N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16 || (flags & ~3)) {
    qtam::set_last_error("N and K must be multiples of 16 in [16, 256]; flags in {0..3}");
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
    qtam::k_tc_gemm_check<<<1, 128, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint16_t*>(A), static_cast<const uint16_t*>(B), D, N, K, (uint32_t)flags);
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
