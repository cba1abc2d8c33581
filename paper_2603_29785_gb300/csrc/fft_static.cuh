// Compile-time specialised Stockham engine: the same stage formula as
// fft_core.cuh's runtime engine, with the length, the radix sequence, the
// stage spans, the block size and the shared-memory padding all template
// constants.  Index arithmetic then reduces to shifts and multiplies by
// constants, every butterfly array has a constant size, and no stage is
// selected at run time, so the kernels built on it stay in registers.
#pragma once

#include <type_traits>

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
// NT threads.  Twiddles come from the stage's own table laid out [i][k]
// (k fastest): tws[i * NS + k] = exp(-2 pi i (i k) / (NS R)), so the threads
// of a warp (consecutive k) read consecutive entries.
template <int SIGN, int M, int NT, int NBS, int NS, int R, typename V, class Src, class Dst>
__device__ __forceinline__ void sstage(const V* __restrict__ tws, const Src& src, const Dst& dst, bool inplace) {
  constexpr int MR = M / R;
  constexpr int ITEMS = MR << NBS;
  constexpr int IPT = (ITEMS + NT - 1) / NT;
  constexpr int BMASK = (1 << NBS) - 1;
  V a[IPT][R];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int w = threadIdx.x + q * NT;
    if (ITEMS % NT == 0 || w < ITEMS) {
      const int b = w & BMASK, j = w >> NBS;
#pragma unroll
      for (int i = 0; i < R; ++i) a[q][i] = src.template get_s<MR>(b, j, i);
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int i = 1; i < R; ++i) {
          V t = __ldg(&tws[i * NS + k]);
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
      for (int i = 0; i < R; ++i) dst.template put_s<NS>(b, base, i, a[q][i]);
    }
  }
}

template <typename V, int NBS, int PS> struct SSmem {
  V* sm;
  __device__ __forceinline__ static int addr(int b, int i) {
    const int e = (i << NBS) + b;
    return e + (e >> PS);
  }
  // address of element j + i*STEP: when STEP * 2^NBS is a multiple of the
  // padding period the padding of the whole run is a compile-time offset
  template <int STEP> __device__ __forceinline__ static int addr_s(int b, int j, int i) {
    constexpr int E = STEP << NBS;
    if constexpr (PS >= 30) {
      return (j << NBS) + b + i * E;
    } else if constexpr (E % (1 << PS) == 0) {
      return addr(b, j) + i * (E + (E >> PS));
    } else {
      return addr(b, j + i * STEP);
    }
  }
  __device__ __forceinline__ V get(int b, int i) const { return sm[addr(b, i)]; }
  __device__ __forceinline__ void put(int b, int i, V v) const { sm[addr(b, i)] = v; }
  template <int STEP> __device__ __forceinline__ V get_s(int b, int j, int i) const { return sm[addr_s<STEP>(b, j, i)]; }
  template <int STEP> __device__ __forceinline__ void put_s(int b, int j, int i, V v) const {
    sm[addr_s<STEP>(b, j, i)] = v;
  }
};

// Strided accessors for the global-memory functors: element j + i*STEP.  A
// functor that defines its own get_s (e.g. to fold the stride into
// addresses) is used as is.
template <class F, class = void> struct HasGetS : std::false_type {};
template <class F>
struct HasGetS<F, std::void_t<decltype(&F::template get_s<1>)>> : std::true_type {};

template <class F> struct Strided : F {
  template <int STEP> __device__ __forceinline__ auto get_s(int b, int j, int i) const {
    if constexpr (HasGetS<F>::value) {
      return F::template get_s<STEP>(b, j, i);
    } else {
      return F::get(b, j + i * STEP);
    }
  }
  template <int STEP, typename V> __device__ __forceinline__ void put_s(int b, int j, int i, V v) const {
    F::put(b, j + i * STEP, v);
  }
};

template <int SIGN, int M, int NT, int NBS, int PS, int NS, int... Rs> struct SRun;

// last stage: smem -> store
template <int SIGN, int M, int NT, int NBS, int PS, int NS, int R> struct SRun<SIGN, M, NT, NBS, PS, NS, R> {
  template <typename V, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tws, const Store& st) {
    SSmem<V, NBS, PS> io{sm};
    sstage<SIGN, M, NT, NBS, NS, R>(tws, io, st, false);
  }
};
// middle stage: smem -> smem; the next stage's table follows this one's
template <int SIGN, int M, int NT, int NBS, int PS, int NS, int R, int R2, int... Rest>
struct SRun<SIGN, M, NT, NBS, PS, NS, R, R2, Rest...> {
  template <typename V, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tws, const Store& st) {
    SSmem<V, NBS, PS> io{sm};
    sstage<SIGN, M, NT, NBS, NS, R>(tws, io, io, true);
    __syncthreads();
    SRun<SIGN, M, NT, NBS, PS, NS * R, R2, Rest...>::run(sm, tws + NS * R, st);
  }
};


// Whole transform: load -> (smem stages) -> store.  Block size must be NT.
// `tws` points at the stage tables of this radix sequence (stages 1..).
template <int SIGN, int M, int NT, int NBS, int R0, int... Rs> struct StaticFFT {
  static constexpr int PS = is_pow2<R0>() ? 4 : 30;
  static constexpr int nst = 1 + sizeof...(Rs);
  static constexpr int radices[nst] = {R0, Rs...};
  static constexpr size_t smem_elems() {
    if (nst == 1) return 0;
    const size_t e = (size_t)M << NBS;
    return e + (e >> PS) + 1;
  }
  template <typename V, class Load, class Store>
  __device__ __forceinline__ static void run(V* sm, const V* tws, const Load& ld0, const Store& st0) {
    const Strided<Load> ld{ld0};
    const Strided<Store> st{st0};
    if constexpr (sizeof...(Rs) == 0) {
      sstage<SIGN, M, NT, NBS, 1, R0>(tws, ld, st, false);
    } else {
      SSmem<V, NBS, PS> io{sm};
      sstage<SIGN, M, NT, NBS, 1, R0>(tws, ld, io, false);
      __syncthreads();
      SRun<SIGN, M, NT, NBS, PS, R0, Rs...>::run(sm, tws, st);
    }
  }
};

}  // namespace qtam
