// Long real FFT of each segment (step a1) and its inverse with the dual-frame
// normaliser fused in (step a7).
//
// A real segment x of N = 2n samples is read as n complex values
// z[m] = x[2m] + i x[2m+1] and transformed as an n = n1 * n2 four-step FFT:
//   column pass:  U[k1][m2] = w_n^(m2 k1) sum_m1 z[m1 n2 + m2] w_n1^(m1 k1)
//   row pass:     Z[k1 + n1 k2] = sum_m2 U[k1][m2] w_n2^(m2 k2)
// followed by the real-to-complex untangle
//   X[k] = (Z[k] + Z*[n-k]) / 2 - (i/2) w_N^k (Z[k] - Z*[n-k]),  k = 0..n
// which gives the one-sided spectrum X[f] = sum_n x[n] exp(-2 pi i f n / N)
// of App. C.  The inverse runs the same steps backwards: the untangle's
// inverse (with X_hat = A / P read through the plan's 1/P table and the DC
// and Nyquist bins taken real) feeds the row pass, then the column pass
// writes x_hat[2m] + i x_hat[2m+1] directly.
#include "qtam_internal.h"

namespace qtam {

namespace {

template <typename V> struct LoadColumns {
  const V* zs; int n2; int c0;
  __device__ __forceinline__ V get(int b, int m1) const { return zs[(int64_t)m1 * n2 + c0 + b]; }
};
template <typename V> struct StoreColumnsTwiddled {
  V* Us; const V* twn; int n2; int c0;
  __device__ __forceinline__ void put(int b, int k1, V v) const {
    const int c = c0 + b;
    Us[(int64_t)k1 * n2 + c] = cmul(v, __ldg(&twn[(int64_t)c * k1]));
  }
};
template <typename V> struct LoadRows {
  const V* Us; int n2; int r0;
  __device__ __forceinline__ V get(int b, int m2) const { return Us[(int64_t)(r0 + b) * n2 + m2]; }
};
template <typename V> struct StoreRowsTransposed {
  V* Zs; int n1; int r0;
  __device__ __forceinline__ void put(int b, int k2, V v) const { Zs[(int64_t)k2 * n1 + r0 + b] = v; }
};

template <typename T>
__global__ void __launch_bounds__(kMaxBlock) k_col_forward(RadixPlan rp, int n, int n2, int nbs, const cplx<T>* __restrict__ z,
                                                      cplx<T>* __restrict__ U, const cplx<T>* __restrict__ twn) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int c0 = blockIdx.x << nbs;
  LoadColumns<V> ld{z + seg * n, n2, c0};
  StoreColumnsTwiddled<V> stv{U + seg * n, twn, n2, c0};
  block_fft<-1>(rp, nbs, sm, twn, n / rp.m, ld, stv);
}

template <typename T>
__global__ void __launch_bounds__(kMaxBlock) k_row_forward(RadixPlan rp, int n, int n1, int nbs, const cplx<T>* __restrict__ U,
                                                      cplx<T>* __restrict__ Z, const cplx<T>* __restrict__ twn) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int r0 = blockIdx.x << nbs;
  LoadRows<V> ld{U + seg * n, rp.m, r0};
  StoreRowsTransposed<V> stv{Z + seg * n, n1, r0};
  block_fft<-1>(rp, nbs, sm, twn, n / rp.m, ld, stv);
}

// w_N^k for k in [0, n]: table holds k <= n/2; w_N^(n-k) = -conj(w_N^k)
template <typename V> __device__ __forceinline__ V wN(const V* twN, int n, int k) {
  if (k <= (n >> 1)) return __ldg(&twN[k]);
  V t = __ldg(&twN[n - k]);
  return mk<V>(-t.x, t.y);
}

template <typename T>
__global__ void k_untangle_forward(int n, const cplx<T>* __restrict__ Z, cplx<T>* __restrict__ X,
                                   const cplx<T>* __restrict__ twN) {
  using V = cplx<T>;
  const int64_t seg = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > (n >> 1)) return;
  const V* Zs = Z + seg * n;
  V* Xs = X + seg * (int64_t)(n + 1);
  const int kk = n - k;                     // partner bin, in [n/2, n]
  const V zk = Zs[k];
  const V zm = Zs[kk == n ? 0 : kk];
  const T half = (T)0.5;
  {
    const V a = zk, b = cconj(zm);
    const V s = a + b, d = a - b;
    const V t = cmul(__ldg(&twN[k]), d);    // w^k (a - b)
    Xs[k] = mk<V>(half * (s.x + t.y), half * (s.y - t.x));   // s/2 - (i/2) t
  }
  if (kk != k) {
    const V a = zm, b = cconj(zk);
    const V s = a + b, d = a - b;
    const V t = cmul(wN(twN, n, kk), d);
    Xs[kk] = mk<V>(half * (s.x + t.y), half * (s.y - t.x));
  }
}

// Inverse row pass input: Zi[k] = scale (E[k] + i O[k]) with
//   E = (Xh[k] + conj Xh[n-k]) / 2,  O = (Xh[k] - conj Xh[n-k]) / 2 * w_N^(-k),
//   Xh = A * (1/P), DC and Nyquist taken real.
template <typename T> struct LoadUntangleInverse {
  using V = cplx<T>;
  const V* As; const T* invP; const V* twN; int n; int n1; int r0; T scale;
  __device__ __forceinline__ V get(int b, int k2) const {
    const int k = r0 + b + n1 * k2;          // 0 <= k < n
    const int kk = n - k;                    // 1 <= kk <= n
    V xk = cscale(As[k], __ldg(&invP[k]));
    V xm = cscale(As[kk], __ldg(&invP[kk]));
    if (k == 0) xk.y = (T)0;
    if (kk == n) xm.y = (T)0;
    const V e = xk + cconj(xm);
    const V o = cmul(xk - cconj(xm), cconj(wN(twN, n, k)));
    const T hs = (T)0.5 * scale;
    return mk<V>(hs * (e.x - o.y), hs * (e.y + o.x));    // scale/2 (e + i o)
  }
};
template <typename V> struct StoreRowsTwiddledConj {
  V* Vs; const V* twn; int n2; int r0;
  __device__ __forceinline__ void put(int b, int m2, V v) const {
    const int r = r0 + b;
    Vs[(int64_t)r * n2 + m2] = cmul(v, cconj(__ldg(&twn[(int64_t)r * m2])));
  }
};
template <typename V> struct StoreColumns {
  V* xs; int n2; int c0;
  __device__ __forceinline__ void put(int b, int m1, V v) const { xs[(int64_t)m1 * n2 + c0 + b] = v; }
};

template <typename T>
__global__ void __launch_bounds__(kMaxBlock) k_row_inverse(RadixPlan rp, int n, int n1, int nbs, const cplx<T>* __restrict__ A,
                                                      const T* __restrict__ invP, cplx<T>* __restrict__ Vb,
                                                      const cplx<T>* __restrict__ twn, const cplx<T>* __restrict__ twN,
                                                      T scale) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int r0 = blockIdx.x << nbs;
  LoadUntangleInverse<T> ld{A + seg * (int64_t)(n + 1), invP, twN, n, n1, r0, scale};
  StoreRowsTwiddledConj<V> stv{Vb + seg * n, twn, rp.m, r0};
  block_fft<+1>(rp, nbs, sm, twn, n / rp.m, ld, stv);
}

template <typename T>
__global__ void __launch_bounds__(kMaxBlock) k_col_inverse(RadixPlan rp, int n, int n2, int nbs, const cplx<T>* __restrict__ Vb,
                                                      cplx<T>* __restrict__ xout, const cplx<T>* __restrict__ twn) {
  using V = cplx<T>;
  extern __shared__ unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t seg = blockIdx.y;
  const int c0 = blockIdx.x << nbs;
  LoadColumns<V> ld{Vb + seg * n, n2, c0};
  StoreColumns<V> stv{xout + seg * n, n2, c0};
  block_fft<+1>(rp, nbs, sm, twn, n / rp.m, ld, stv);
}

constexpr int64_t kMaxGridY = 65535;

}  // namespace

template <typename T>
cudaError_t launch_spectrum(const LongCfg& c, const cplx<T>* z, cplx<T>* U, cplx<T>* Z, cplx<T>* X, int64_t B,
                            const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st) {
  for (int64_t s0 = 0; s0 < B; s0 += kMaxGridY) {
    const int64_t nb = (B - s0) < kMaxGridY ? (B - s0) : kMaxGridY;
    const int64_t off = s0 * c.n;
    dim3 g1(c.n2 >> c.col_nbs, (unsigned)nb);
    allow_smem((const void*)k_col_forward<T>, c.col_smem);
    k_col_forward<T><<<g1, c.col_threads, c.col_smem, st>>>(c.rp1, c.n, c.n2, c.col_nbs, z + off, U + off, twn);
    dim3 g2(c.n1 >> c.row_nbs, (unsigned)nb);
    allow_smem((const void*)k_row_forward<T>, c.row_smem);
    k_row_forward<T><<<g2, c.row_threads, c.row_smem, st>>>(c.rp2, c.n, c.n1, c.row_nbs, U + off, Z + off, twn);
    dim3 g3((unsigned)((c.n / 2 + 1 + 255) / 256), (unsigned)nb);
    k_untangle_forward<T><<<g3, 256, 0, st>>>(c.n, Z + off, X + s0 * (int64_t)(c.n + 1), twN);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_synthesis(const LongCfg& c, const cplx<T>* A, const T* invP, cplx<T>* Vb, cplx<T>* xout, int64_t B,
                             const cplx<T>* twn, const cplx<T>* twN, cudaStream_t st) {
  for (int64_t s0 = 0; s0 < B; s0 += kMaxGridY) {
    const int64_t nb = (B - s0) < kMaxGridY ? (B - s0) : kMaxGridY;
    const int64_t off = s0 * c.n;
    dim3 g2(c.n1 >> c.row_nbs, (unsigned)nb);
    allow_smem((const void*)k_row_inverse<T>, c.row_smem);
    k_row_inverse<T><<<g2, c.row_threads, c.row_smem, st>>>(c.rp2, c.n, c.n1, c.row_nbs, A + s0 * (int64_t)(c.n + 1),
                                                            invP, Vb + off, twn, twN, (T)1 / (T)c.n);
    dim3 g1(c.n2 >> c.col_nbs, (unsigned)nb);
    allow_smem((const void*)k_col_inverse<T>, c.col_smem);
    k_col_inverse<T><<<g1, c.col_threads, c.col_smem, st>>>(c.rp1, c.n, c.n2, c.col_nbs, Vb + off, xout + off, twn);
  }
  return cudaGetLastError();
}

template cudaError_t launch_spectrum<float>(const LongCfg&, const float2*, float2*, float2*, float2*, int64_t,
                                            const float2*, const float2*, cudaStream_t);
template cudaError_t launch_spectrum<double>(const LongCfg&, const double2*, double2*, double2*, double2*, int64_t,
                                             const double2*, const double2*, cudaStream_t);
template cudaError_t launch_synthesis<float>(const LongCfg&, const float2*, const float*, float2*, float2*, int64_t,
                                             const float2*, const float2*, cudaStream_t);
template cudaError_t launch_synthesis<double>(const LongCfg&, const double2*, const double*, double2*, double2*, int64_t,
                                              const double2*, const double2*, cudaStream_t);

}  // namespace qtam
