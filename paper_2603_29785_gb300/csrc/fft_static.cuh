// Compile-time specialised Stockham engine: the same stage formula as
// fft_core.cuh's runtime engine, with the length, the radix sequence, the
// stage spans, the block size and the shared-memory padding all template
// constants.  Index arithmetic then reduces to shifts and multiplies by
// constants, every butterfly array has a constant size, and no stage is
// selected at run time, so the kernels built on it stay in registers.
#pragma once

#include "fft_core.cuh"

namespace qtam {

template <int... Rs> struct RList {};

template <int A, int... Rest> struct MaxOf { static constexpr int value = A > MaxOf<Rest...>::value ? A : MaxOf<Rest...>::value; };
template <int A> struct MaxOf<A> { static constexpr int value = A; };

template <int M, int NBS, int... Rs> struct StaticThreads {
  // the widest stage's items spread over at most 512 threads, whole warps
  static constexpr int items = MaxOf<((M / Rs) << NBS)...>::value;
  static constexpr int per = (items + 511) / 512;
  static constexpr int raw = (items + per - 1) / per;
  static constexpr int value = (raw + 31) / 32 * 32;
};

template <int R> __host__ __device__ constexpr bool is_pow2() { return (R & (R - 1)) == 0; }

// One stage: radix R, span NS, over 2^NBS interleaved transforms of length M,
// NT threads.  tw[t * twstride] = exp(-2 pi i t / M).
template <int SIGN, int M, int NT, int NBS, int NS, int R, typename V, class Src, class Dst>
__device__ __forceinline__ void sstage(const V* __restrict__ tw, int twstride, const Src& src, const Dst& dst,
                                       bool inplace) {
  constexpr int MR = M / R;
  constexpr int ITEMS = MR << NBS;
  constexpr int IPT = (ITEMS + NT - 1) / NT;
  constexpr int TSTEP = M / (NS * R);
  constexpr int BMASK = (1 << NBS) - 1;
  V a[IPT][R];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int w = threadIdx.x + q * NT;
    if (ITEMS % NT == 0 || w < ITEMS) {
      const int b = w & BMASK, j = w >> NBS;
#pragma unroll
      for (int i = 0; i < R; ++i) a[q][i] = src.get(b, j + i * MR);
      if constexpr (NS > 1) {
        const int k = j % NS;
        const int t0 = k * TSTEP * twstride;
#pragma unroll
        for (int i = 1; i < R; ++i) {
          V t = __ldg(&tw[i * t0]);
          if (SIGN > 0) t.y = -t.y;
          a[q][i] = cmul(a[q][i], t);
        }
      }
      Dft<R, SIGN>::run(a[q]);
    }
  }
  if (inplace) __syncthreads();
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int w = threadIdx.x + q * NT;
    if (ITEMS % NT == 0 || w < ITEMS) {
      const int b = w & BMASK, j = w >> NBS;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int i = 0; i < R; ++i) dst.put(b, base + i * NS, a[q][i]);
    }
  }
}

template <typename V, int NBS, int PS> struct SSmem {
  V* sm;
  __device__ __forceinline__ static int addr(int b, int i) {
    const int e = (i << NBS) + b;
    return e + (e >> PS);
  }
  __device__ __forceinline__ V get(int b, int i) const { return sm[addr(b, i)]; }
  __device__ __forceinline__ void put(int b, int i, V v) const { sm[addr(b, i)] = v; }
};

template <int SIGN, int M, int NT, int NBS, int PS, int NS, int... Rs> struct SRun;

// last stage: smem -> store
template <int SIGN, int M, int NT, int NBS, int PS, int NS, int R> struct SRun<SIGN, M, NT, NBS, PS, NS, R> {
  template <typename V, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tw, int twstride, const Store& st) {
    SSmem<V, NBS, PS> io{sm};
    sstage<SIGN, M, NT, NBS, NS, R>(tw, twstride, io, st, false);
  }
};
// middle stage: smem -> smem
template <int SIGN, int M, int NT, int NBS, int PS, int NS, int R, int R2, int... Rest>
struct SRun<SIGN, M, NT, NBS, PS, NS, R, R2, Rest...> {
  template <typename V, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tw, int twstride, const Store& st) {
    SSmem<V, NBS, PS> io{sm};
    sstage<SIGN, M, NT, NBS, NS, R>(tw, twstride, io, io, true);
    __syncthreads();
    SRun<SIGN, M, NT, NBS, PS, NS * R, R2, Rest...>::run(sm, tw, twstride, st);
  }
};

// Whole transform: load -> (smem stages) -> store.  Block size must be NT.
template <int SIGN, int M, int NT, int NBS, int R0, int... Rs> struct StaticFFT {
  static constexpr int PS = is_pow2<R0>() ? 4 : 30;
  static constexpr int nst = 1 + sizeof...(Rs);
  static constexpr size_t smem_elems() {
    if (nst == 1) return 0;
    const size_t e = (size_t)M << NBS;
    return e + (e >> PS) + 1;
  }
  template <typename V, class Load, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tw, int twstride, const Load& ld, const Store& st) {
    if constexpr (sizeof...(Rs) == 0) {
      sstage<SIGN, M, NT, NBS, 1, R0>(tw, twstride, ld, st, false);
    } else {
      SSmem<V, NBS, PS> io{sm};
      sstage<SIGN, M, NT, NBS, 1, R0>(tw, twstride, ld, io, false);
      __syncthreads();
      SRun<SIGN, M, NT, NBS, PS, R0, Rs...>::run(sm, tw, twstride, st);
    }
  }
};

}  // namespace qtam
