// Host side of the QTAM library: plan construction (filter-bank geometry,
// FP64 frame operator, twiddle tables, launch shapes) and the C ABI.
//
// Geometry follows App. A of the paper: a log grid of centre frequencies per
// Q-plane, window length proportional to f_k N_t / Q clamped at
// L_max = 2 floor(ceil(N_t Delta f_max) / 2) + 1 (Delta f_max = largest gap
// between neighbouring centres, or a manual clamp), centre bin k_c = f_k N_t
// (Eq. support), bisquare windows (Eq. gwpy_window_formula; Hann, Kaiser,
// Tukey and Planck-taper as the App. A alternatives) and an envelope
// length M no shorter than the largest window (Sec. III, lossless
// decimation).  Where the paper leaves a constant open the choices are:
// h = max(1, min(floor(f T q_width / Q), h_max)) with q_width = sqrt(11);
// k_c rounds half away from zero; M = smallest 2^a 3^b 5^c >= max L;
// c_k normalises the untruncated window to unit energy (L2, default), to
// 1 / sum W'^2 (PAPER) or 1 (NONE); windows are cut to 0 <= f <= N/2.
//
// The frame operator P[f] = sum_k W_k[f]^2 (App. C) and its inverse on the
// kept set F_tau = {P > 0, P >= tau max P} are the only FP64 arithmetic of
// the library, done here once per plan (and once per new plane mask).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qtam.h"
#include "qtam_internal.h"
#include "tc_sm100.cuh"

using namespace qtam;

namespace {

thread_local std::string g_last_error;

qtam_status fail(qtam_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
qtam_status fail_cuda(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return QTAM_ERR_CUDA;
}

constexpr int kMaxSmem = 227 * 1024;
constexpr int kMaxThreads = 512;  // must match the kernels' __launch_bounds__

bool factor235(int64_t m, int& a, int& b, int& c) {
  a = b = c = 0;
  if (m < 1) return false;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  while (m % 5 == 0) { m /= 5; ++c; }
  return m == 1;
}

bool make_radix_plan(int m, RadixPlan& rp) {
  int a, b, c;
  if (m < 2 || !factor235(m, a, b, c)) return false;
  std::vector<int> rs;
  while (a >= 4) { rs.push_back(16); a -= 4; }
  if (a == 3) rs.push_back(8);
  else if (a == 2) rs.push_back(4);
  else if (a == 1) rs.push_back(2);
  for (int i = 0; i < c; ++i) rs.push_back(5);
  for (int i = 0; i < b; ++i) rs.push_back(3);
  if ((int)rs.size() > kMaxStages) return false;
  std::memset(&rp, 0, sizeof(rp));
  rp.m = m;
  rp.nst = (int)rs.size();
  for (int i = 0; i < rp.nst; ++i) rp.r[i] = rs[i];
  const int r0 = rs[0];
  rp.pad_shift = (r0 & (r0 - 1)) == 0 ? 4 : 30;
  return true;
}

int threads_for(const RadixPlan& rp, int nbs) {
  int t = 32;
  for (int s = 0; s < rp.nst; ++s) {
    const int items = (rp.m / rp.r[s]) << nbs;
    const int ipt = ipt_for(rp.r[s]);
    t = std::max(t, (items + ipt - 1) / ipt);
  }
  return (t + 31) / 32 * 32;
}

size_t smem_for(const RadixPlan& rp, int nbs, size_t elem) {
  if (rp.nst <= 1) return 0;
  const size_t e = (size_t)rp.m << nbs;
  return (e + (e >> rp.pad_shift) + 1) * elem;
}

int64_t smooth_at_least(int64_t n) {
  for (int64_t m = std::max<int64_t>(1, n);; ++m) {
    int a, b, c;
    if (factor235(m, a, b, c)) return m;
  }
}

// unnormalised bisquare W'(d) = (1 - (d/h)^2)^2, |d| <= h
inline double bisq(int64_t d, int64_t h) {
  const int64_t a = d < 0 ? -d : d;
  if (a > h) return 0.0;
  const double u = (double)((h - a) * (h + a)) / ((double)h * (double)h);
  return u * u;
}

// modified Bessel function I0 from its power series sum_k ((x/2)^k / k!)^2
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

// unnormalised window W'(d), |d| <= h, of the App. A family (u = |d|/h):
// bisquare (1-u^2)^2; Hann (1+cos(pi u))/2; Kaiser I0(beta sqrt(1-u^2))/I0(beta);
// Tukey and Planck-taper flat on u <= 1-a, tapering over the outer fraction a.
// The Planck taper uses the continuous exponent Z = a/t - a/(a-t), t = 1-u.
double window_profile(int64_t d, int64_t h, int win, double prm) {
  const int64_t a = d < 0 ? -d : d;
  if (a > h) return 0.0;
  if (win == QTAM_WIN_BISQUARE) return bisq(d, h);
  const double pi = 3.14159265358979323846;
  const double u = (double)a / (double)h;
  switch (win) {
    case QTAM_WIN_HANN: return 0.5 * (1.0 + std::cos(pi * u));
    case QTAM_WIN_KAISER: return bessel_i0(prm * std::sqrt(std::max(0.0, 1.0 - u * u))) / bessel_i0(prm);
    case QTAM_WIN_TUKEY:
      if (prm <= 0 || u <= 1.0 - prm) return 1.0;
      return 0.5 * (1.0 + std::cos(pi * (u - (1.0 - prm)) / prm));
    case QTAM_WIN_PLANCK: {
      const double t = 1.0 - u;
      if (t <= 0) return 0.0;
      if (prm <= 0 || t >= prm) return 1.0;
      const double z = prm / t - prm / (prm - t);
      return 1.0 / (std::exp(std::min(700.0, std::max(-700.0, z))) + 1.0);
    }
    default: return 0.0;
  }
}

struct MaskEntry {
  void* invP = nullptr;   // [Nr] T
  int* rows = nullptr;    // selected row indices
  int n_sel = 0;
  int64_t kept = 0;
  double kappa = 0;
};

}  // namespace

struct qtam_plan_s {
  // description
  double fs = 0;
  int64_t N = 0;
  std::vector<double> q;
  double fmin = 0, fmax = 0;
  int K = 0;
  int norm = QTAM_NORM_L2;
  double q_width = 0;
  double max_window_hz = 0;
  std::vector<int> window;          // per plane (QTAM_WIN_*)
  std::vector<double> window_param; // per plane
  int compute = QTAM_DTYPE_F32;
  int env = QTAM_DTYPE_F32;
  int short_dft = QTAM_SHORT_DFT_CUDA;
  double eps = 0;        // dense mode: stopband floor of every window
  int remod = 0;         // dense mode: envelopes carry the carrier
  double tau = 0;
  // geometry
  int P = 0;
  int64_t n = 0, Nr = 0;
  int M = 0;
  int64_t h_max = 0;
  int Lmax = 0;
  int64_t band_bins = 0;
  std::vector<double> f, c;
  std::vector<int64_t> kc;
  std::vector<int> h;
  std::vector<std::vector<double>> Pplane;  // per-plane frame operator
  // device
  int device = -1;
  LongCfg lc{};
  RowCfg rc{};
  void* d_rows = nullptr;
  void* d_twM = nullptr;
  void* d_twn = nullptr;
  void* d_twN = nullptr;
  void* d_tw4 = nullptr;
  void* d_wtab = nullptr;   // W'(0..h) per distinct half-width, non-bisquare windows only
  void* d_tcA = nullptr;    // tensor-core short DFT operands (short_dft = TENSOR)
  void* d_tcAi = nullptr;
  void* d_tcG = nullptr;
  void* d_ones = nullptr;   // dense mode: 1/P := 1 for the single-tile inverse
  size_t device_bytes = 0;
  std::map<int, void*> variant_tw;   // stage twiddle tables per row-kernel variant
  void* d_stw_col = nullptr;
  void* d_stw_row = nullptr;
  std::mutex mu;
  std::map<uint64_t, MaskEntry> masks;
  // host round trip pipeline: copy-in and copy-out streams and their events,
  // created on first use; one round trip at a time per plan (rt_mu)
  std::mutex rt_mu;
  cudaStream_t rt_in = nullptr, rt_out = nullptr, rt_cs = nullptr;
  std::vector<cudaEvent_t> rt_ev;

  size_t real_size() const { return compute == QTAM_DTYPE_F64 ? 8 : 4; }
  size_t cplx_size() const { return 2 * real_size(); }
  size_t env_size() const {
    return env == QTAM_DTYPE_F64 ? 16 : (env == QTAM_DTYPE_F32 ? 8 : 4);
  }
  uint64_t all_mask() const { return P >= 64 ? ~0ull : ((1ull << P) - 1); }
  double wprof(int64_t d, int64_t hk, int p) const { return window_profile(d, hk, window[p], window_param[p]); }
  // the window with the dense mode's floor: eps wherever the window vanishes
  double wdense(int64_t d, int64_t hk, int p) const {
    const double w = wprof(d, hk, p);
    return (eps > 0 && !(w > 0)) ? eps : w;
  }
  bool all_bisquare() const {
    for (int w : window)
      if (w != QTAM_WIN_BISQUARE) return false;
    return true;
  }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T> void fill_twiddles(std::vector<T>& v, int64_t len, int64_t count) {
  // e^{-2 pi i t / len}, t < count, evaluated in FP64
  v.resize(2 * count);
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t t = 0; t < count; ++t) {
    const double ang = two_pi * (double)t / (double)len;
    v[2 * t] = (T)std::cos(ang);
    v[2 * t + 1] = (T)(-std::sin(ang));
  }
}

qtam_status upload(void** dst, const void* src, size_t bytes, size_t& total) {
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return fail(QTAM_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  total += bytes;
  e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy");
  return QTAM_OK;
}

// Build (or find) the normaliser and row list for a plane mask.  Called with plan->mu held.
qtam_status build_mask(qtam_plan_s* pl, uint64_t mask, MaskEntry** out) {
  auto it = pl->masks.find(mask);
  if (it != pl->masks.end()) {
    *out = &it->second;
    return QTAM_OK;
  }
  std::vector<double> Pm(pl->Nr, 0.0);
  std::vector<int> rows;
  for (int p = 0; p < pl->P; ++p) {
    if (!((mask >> p) & 1ull)) continue;
    for (int64_t f = 0; f < pl->Nr; ++f) Pm[f] += pl->Pplane[p][f];
    for (int k = 0; k < pl->K; ++k) rows.push_back(p * pl->K + k);
  }
  double pmax = 0;
  for (double v : Pm) pmax = std::max(pmax, v);
  MaskEntry e;
  std::vector<double> inv(pl->Nr, 0.0);
  for (int64_t f = 0; f < pl->Nr; ++f) {
    if (Pm[f] > 0 && Pm[f] >= pl->tau * pmax) {
      inv[f] = 1.0 / Pm[f];
      ++e.kept;
    }
  }
  if (e.kept == 0) return fail(QTAM_ERR_NO_COVERAGE, "the selected planes cover no frequency bin");
  // kappa = max over kept bins of max_k W_k / P
  std::vector<double> wmax(pl->Nr, 0.0);
  for (int r : rows) {
    const int64_t hk = pl->h[r], kc = pl->kc[r];
    const int64_t lo = pl->eps > 0 ? -kc : -hk, hi = pl->eps > 0 ? pl->Nr - 1 - kc : hk;
    for (int64_t d = lo; d <= hi; ++d) {
      const int64_t fb = kc + d;
      if (fb < 0 || fb >= pl->Nr) continue;
      wmax[fb] = std::max(wmax[fb], pl->c[r] * pl->wdense(d, hk, r / pl->K));
    }
  }
  for (int64_t f = 0; f < pl->Nr; ++f)
    if (inv[f] > 0) e.kappa = std::max(e.kappa, wmax[f] * inv[f]);
  e.n_sel = (int)rows.size();
  if (pl->device >= 0) {
    size_t tot = 0;
    qtam_status s;
    if (pl->compute == QTAM_DTYPE_F64) {
      s = upload(&e.invP, inv.data(), inv.size() * sizeof(double), tot);
    } else {
      std::vector<float> invf(inv.begin(), inv.end());
      s = upload(&e.invP, invf.data(), invf.size() * sizeof(float), tot);
    }
    if (s != QTAM_OK) return s;
    s = upload(reinterpret_cast<void**>(&e.rows), rows.data(), rows.size() * sizeof(int), tot);
    if (s != QTAM_OK) {
      cudaFree(e.invP);
      return s;
    }
    pl->device_bytes += tot;
  }
  auto res = pl->masks.emplace(mask, e);
  *out = &res.first->second;
  return QTAM_OK;
}

bool choose_long(int64_t n, bool dbl, LongCfg& lc) {
  if (n < 4 || n > (int64_t)1 << 26) return false;
  const size_t elem = dbl ? 16 : 8;
  double best = 1e30;
  bool found = false;
  for (int64_t n1 = 2; n1 <= n / 2; ++n1) {
    if (n % n1) continue;
    const int64_t n2 = n / n1;
    RadixPlan r1, r2;
    if (!make_radix_plan((int)n1, r1) || !make_radix_plan((int)n2, r2)) continue;
    const int cmax = dbl ? 3 : 4, rmax = dbl ? 1 : 2;
    int cn = cmax, rn = rmax;
    while (cn > 0 && (n2 % (1 << cn) || threads_for(r1, cn) > kMaxThreads || smem_for(r1, cn, elem) > (size_t)kMaxSmem)) --cn;
    while (rn > 0 && (n1 % (1 << rn) || threads_for(r2, rn) > kMaxThreads || smem_for(r2, rn, elem) > (size_t)kMaxSmem)) --rn;
    const int t1 = threads_for(r1, cn), t2 = threads_for(r2, rn);
    const size_t s1 = smem_for(r1, cn, elem), s2 = smem_for(r2, rn, elem);
    if (t1 > kMaxThreads || t2 > kMaxThreads || s1 > (size_t)kMaxSmem || s2 > (size_t)kMaxSmem) continue;
    // prefer balanced splits and full-width column groups
    const double score = std::fabs(std::log2((double)n1) - std::log2((double)n2) + 1.0) + (cmax - cn) * 2.0 +
                         (rmax - rn) * 1.0;
    if (score < best) {
      best = score;
      found = true;
      lc.n = (int)n;
      lc.n1 = (int)n1;
      lc.n2 = (int)n2;
      lc.col_nbs = cn;
      lc.row_nbs = rn;
      lc.rp1 = r1;
      lc.rp2 = r2;
      lc.col_threads = t1;
      lc.row_threads = t2;
      lc.col_smem = s1;
      lc.row_smem = s2;
    }
  }
  return found;
}

// Build the stage twiddle tables of a compile-time radix sequence in FP64,
// round to float once and upload them; `pair` writes each entry (c, s) as
// (c, c, s, s), the layout of the row-pair kernels (one value per row lane).
qtam_status upload_stage_table(const int* r, int nst, void** dst, size_t& total, bool pair = false) {
  size_t n = 0;
  stage_twiddles(r, nst, nullptr, &n);
  if (n == 0) n = 1;
  std::vector<double> d(2 * n, 0.0);
  stage_twiddles(r, nst, d.data(), &n);
  std::vector<float> f;
  if (pair) {
    f.reserve(4 * n);
    for (size_t t = 0; t < n; ++t) {
      const float c = (float)d[2 * t], s = (float)d[2 * t + 1];
      f.insert(f.end(), {c, c, s, s});
    }
  } else {
    f.assign(d.begin(), d.end());
  }
  return upload(dst, f.data(), f.size() * sizeof(float), total);
}

// round to the nearest BF16, ties to even (finite inputs)
uint16_t to_bf16(double x) {
  const float f = (float)x;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

// Constant operands of the tensor-core four-step (M = 64 x 128),
// FP64-evaluated and rounded once, in the K-major core-matrix layout:
//  A: DFT-64 block matrix as GEMM A's B operand, row n1 (Re D) or 64 + n1
//     (Im D), column j1 (times Re Z) or 64 + j1 (times Im Z):
//     [cos, -sin; sin, cos] of 2 pi j1 n1 / 64;
//  Ai: the conjugate block matrix as the inverse GEMM A''s B operand, row j1
//     (Re S) or 64 + j1 (Im S), column n1 (times Re E') or 64 + n1 (Im E'):
//     [cos, sin; -sin, cos] of 2 pi j1 n1 / 64;
//  G: cosine then sine DFT-128 matrices [n2][j2] of 2 pi j2 n2 / 128.
qtam_status upload_tc_tables(qtam_plan_s* pl, size_t& tot) {
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<uint16_t> A(128 * 128), Ai(128 * 128), G(2 * 128 * 128);
  for (int c = 0; c < 128; ++c)
    for (int k = 0; k < 128; ++k) {
      const int a = c & 63, part = c >> 6, b = k & 63, comp = k >> 6;
      const double th = two_pi * (double)((a * b) % 64) / 64.0;
      const double co = std::cos(th), si = std::sin(th);
      A[qtam::tc::cm_offset(c, k, 128) / 2] = to_bf16(part == 0 ? (comp == 0 ? co : -si) : (comp == 0 ? si : co));
      Ai[qtam::tc::cm_offset(c, k, 128) / 2] = to_bf16(part == 0 ? (comp == 0 ? co : si) : (comp == 0 ? -si : co));
    }
  for (int n2 = 0; n2 < 128; ++n2)
    for (int j2 = 0; j2 < 128; ++j2) {
      const double th = two_pi * (double)((j2 * n2) % 128) / 128.0;
      G[qtam::tc::cm_offset(n2, j2, 128) / 2] = to_bf16(std::cos(th));
      G[128 * 128 + qtam::tc::cm_offset(n2, j2, 128) / 2] = to_bf16(std::sin(th));
    }
  qtam_status s;
  if ((s = upload(&pl->d_tcA, A.data(), A.size() * 2, tot)) != QTAM_OK) return s;
  if ((s = upload(&pl->d_tcAi, Ai.data(), Ai.size() * 2, tot)) != QTAM_OK) return s;
  if ((s = upload(&pl->d_tcG, G.data(), G.size() * 2, tot)) != QTAM_OK) return s;
  pl->rc.tcA = pl->d_tcA;
  pl->rc.tcAi = pl->d_tcAi;
  pl->rc.tcG = pl->d_tcG;
  return QTAM_OK;
}

template <typename T> qtam_status upload_tables(qtam_plan_s* pl) {
  std::vector<T> tw;
  size_t tot = 0;
  qtam_status s;
  fill_twiddles(tw, pl->M, pl->M);
  if ((s = upload(&pl->d_twM, tw.data(), tw.size() * sizeof(T), tot)) != QTAM_OK) return s;
  fill_twiddles(tw, pl->n, pl->n);
  if ((s = upload(&pl->d_twn, tw.data(), tw.size() * sizeof(T), tot)) != QTAM_OK) return s;
  fill_twiddles(tw, pl->N, pl->n / 2 + 1);
  if ((s = upload(&pl->d_twN, tw.data(), tw.size() * sizeof(T), tot)) != QTAM_OK) return s;
  {  // four-step twiddles in [k1][c] layout: w_n^(k1 c), exponent reduced mod n in integers
    const int64_t n1 = pl->lc.n1, n2 = pl->lc.n2;
    std::vector<T> t4(2 * (size_t)pl->n);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t k1 = 0; k1 < n1; ++k1)
      for (int64_t c = 0; c < n2; ++c) {
        const int64_t e = (k1 * c) % pl->n;
        const double ang = two_pi * (double)e / (double)pl->n;
        t4[2 * (k1 * n2 + c)] = (T)std::cos(ang);
        t4[2 * (k1 * n2 + c) + 1] = (T)(-std::sin(ang));
      }
    if ((s = upload(&pl->d_tw4, t4.data(), t4.size() * sizeof(T), tot)) != QTAM_OK) return s;
    pl->lc.tw4 = pl->d_tw4;
  }
  std::vector<RowDev<T>> rows(pl->P * pl->K);
  const double sMN = std::sqrt((double)pl->M * (double)pl->N), sNM = std::sqrt((double)pl->N / (double)pl->M);
  for (size_t r = 0; r < rows.size(); ++r) {
    rows[r].kc = (int)pl->kc[r];
    rows[r].h = pl->h[r];
    rows[r].c_fwd = (T)(pl->c[r] / sMN);
    rows[r].c_inv = (T)(pl->c[r] * sNM);
    rows[r].inv_h2 = (T)(1.0 / ((double)pl->h[r] * (double)pl->h[r]));
    rows[r].kw_fwd = (T)(std::sqrt(pl->c[r] / sMN) / ((double)pl->h[r] * (double)pl->h[r]));
    rows[r].kw_inv = (T)(std::sqrt(pl->c[r] * sNM) / ((double)pl->h[r] * (double)pl->h[r]));
    rows[r].woff = -1;
    rows[r].hb = pl->eps > 0 ? (int)pl->n : pl->h[r];
    rows[r].eps_fwd = (T)(pl->eps > 0 ? pl->c[r] / sMN * pl->eps : 0.0);
    rows[r].eps_inv = (T)(pl->eps > 0 ? pl->c[r] * sNM * pl->eps : 0.0);
  }
  if (pl->eps > 0) {
    std::vector<T> ones(pl->Nr, (T)1);
    if ((s = upload(&pl->d_ones, ones.data(), ones.size() * sizeof(T), tot)) != QTAM_OK) return s;
  }
  if (!pl->all_bisquare()) {
    // one W'(0..h) table per distinct (window, parameter, half-width), read by
    // the runtime engine; bisquare rows of a mixed bank keep the formula
    std::map<std::tuple<int, double, int>, int> off;
    std::vector<T> tab;
    for (size_t r = 0; r < rows.size(); ++r) {
      const int p = (int)r / pl->K, hk = pl->h[r];
      if (pl->window[p] == QTAM_WIN_BISQUARE) continue;
      const auto key = std::make_tuple(pl->window[p], pl->window_param[p], hk);
      auto it = off.find(key);
      if (it == off.end()) {
        if (tab.size() + hk + 1 > (size_t)INT32_MAX) return fail(QTAM_ERR_UNSUPPORTED_SIZE, "window tables too large");
        it = off.emplace(key, (int)tab.size()).first;
        for (int a = 0; a <= hk; ++a) tab.push_back((T)pl->wdense(a, hk, p));
      }
      rows[r].woff = it->second;
    }
    if ((s = upload(&pl->d_wtab, tab.data(), tab.size() * sizeof(T), tot)) != QTAM_OK) return s;
  }
  if ((s = upload(&pl->d_rows, rows.data(), rows.size() * sizeof(RowDev<T>), tot)) != QTAM_OK) return s;
  if (pl->rc.tensor && (s = upload_tc_tables(pl, tot)) != QTAM_OK) return s;
  if (sizeof(T) == 4) {
    for (int v = 0; v < row_variant_count(); ++v) {
      const RowVariant* rv = row_variant(v);
      if (rv->M != pl->M) continue;
      void* p = nullptr;
      if ((s = upload_stage_table(rv->r, rv->nst, &p, tot, rv->tw_pair != 0)) != QTAM_OK) return s;
      pl->variant_tw[v] = p;
    }
    int r[kMaxStages], nst = 0;
    if (long_static_radices(pl->lc.n1, pl->lc.col_nbs, r, &nst)) {
      if ((s = upload_stage_table(r, nst, &pl->d_stw_col, tot)) != QTAM_OK) return s;
      pl->lc.stw_col = pl->d_stw_col;
    }
    if (long_static_radices(pl->lc.n2, pl->lc.row_nbs, r, &nst)) {
      if ((s = upload_stage_table(r, nst, &pl->d_stw_row, tot)) != QTAM_OK) return s;
      pl->lc.stw_row = pl->d_stw_row;
    }
    auto it = pl->variant_tw.find(pl->rc.variant);
    pl->rc.stw = it == pl->variant_tw.end() ? nullptr : it->second;
    if (pl->rc.variant >= 0 && !pl->rc.stw) pl->rc.variant = -1;
  }
  pl->device_bytes += tot;
  return QTAM_OK;
}

// A compile-time row variant serves a plan of its length with FP32 compute;
// plans with a non-bisquare window need a variant built for window tables
// and FP32 envelopes, dense-mode plans (stopband floor or carrier) one built
// with the dense kernels (any envelope storage).
bool variant_usable(const qtam_plan_s* pl, int id) {
  const RowVariant* v = row_variant(id);
  if (!v || v->M != pl->M || pl->compute != QTAM_DTYPE_F32) return false;
  if (pl->eps > 0 || pl->remod) return v->fwd_dense != nullptr;   // F32, BF16 or F16 envelopes
  return pl->all_bisquare() || (v->fwd_tab != nullptr && pl->env == QTAM_DTYPE_F32);
}

void free_plan(qtam_plan_s* pl) {
  if (!pl) return;
  if (pl->device >= 0) {
    DeviceGuard g(pl->device);
    cudaFree(pl->d_rows);
    cudaFree(pl->d_twM);
    cudaFree(pl->d_twn);
    cudaFree(pl->d_twN);
    cudaFree(pl->d_tw4);
    cudaFree(pl->d_wtab);
    cudaFree(pl->d_tcA);
    cudaFree(pl->d_tcAi);
    cudaFree(pl->d_tcG);
    cudaFree(pl->d_ones);
    cudaFree(pl->d_stw_col);
    cudaFree(pl->d_stw_row);
    for (auto& kv : pl->variant_tw) cudaFree(kv.second);
    for (cudaEvent_t e : pl->rt_ev) cudaEventDestroy(e);
    if (pl->rt_in) cudaStreamDestroy(pl->rt_in);
    if (pl->rt_out) cudaStreamDestroy(pl->rt_out);
    if (pl->rt_cs) cudaStreamDestroy(pl->rt_cs);
    for (auto& kv : pl->masks) {
      cudaFree(kv.second.invP);
      cudaFree(kv.second.rows);
    }
  }
  delete pl;
}

qtam_status check_mask(const qtam_plan_s* pl, uint64_t& mask) {
  if (mask == 0) mask = pl->all_mask();
  if (mask & ~pl->all_mask()) return fail(QTAM_ERR_INVALID_ARG, "plane_mask selects planes the plan does not have");
  return QTAM_OK;
}

size_t ws_bytes(const qtam_plan_s* pl, int64_t B) {
  const size_t cs = pl->cplx_size();
  const size_t r0 = ((size_t)B * pl->Nr * cs + 255) / 256 * 256;
  return r0 + (size_t)B * pl->n * cs;
}

struct Regions {
  void* r0;  // [B][Nr] complex: U (stride n) then X / A (stride Nr)
  void* r1;  // [B][n] complex: Z / V
};
Regions split_ws(const qtam_plan_s* pl, void* ws, int64_t B) {
  const size_t cs = pl->cplx_size();
  const size_t r0 = ((size_t)B * pl->Nr * cs + 255) / 256 * 256;
  return Regions{ws, static_cast<char*>(ws) + r0};
}

qtam_status common_checks(const qtam_plan_s* pl, int64_t batch) {
  if (!pl) return fail(QTAM_ERR_INVALID_ARG, "plan is NULL");
  if (pl->device < 0) return fail(QTAM_ERR_NO_DEVICE, "host-only plan (device = -1) cannot run transforms");
  if (batch < 0) return fail(QTAM_ERR_INVALID_ARG, "batch < 0");
  if (batch * (int64_t)pl->P * pl->K > INT32_MAX) return fail(QTAM_ERR_UNSUPPORTED_SIZE, "batch * rows exceeds 2^31-1");
  return QTAM_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T>
qtam_status run_spectrum(qtam_plan_s* pl, const void* x, int64_t B, void* X, void* ws, cudaStream_t st) {
  using V = cplx<T>;
  Regions rg = split_ws(pl, ws, B);
  cudaError_t e = launch_spectrum<T>(pl->lc, static_cast<const V*>(x), static_cast<V*>(rg.r0), static_cast<V*>(rg.r1),
                                     static_cast<V*>(X), B, static_cast<const V*>(pl->d_twn),
                                     static_cast<const V*>(pl->d_twN), st);
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "spectrum launch");
}

template <typename T> qtam_status run_envelopes(qtam_plan_s* pl, const void* X, int64_t B, void* y, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (pl->rc.tensor) {
      cudaError_t e = launch_rows_forward_tc(pl->rc, static_cast<const RowDev<float>*>(pl->d_rows), pl->P * pl->K,
                                             pl->Nr, static_cast<const float2*>(X), y, pl->env, B, st,
                                             static_cast<const float*>(pl->d_wtab));
      if (e != cudaSuccess) return fail_cuda(e, "tensor-core envelopes");
      return QTAM_OK;
    }
  }
  using V = cplx<T>;
  cudaError_t e = launch_rows_forward<T>(pl->rc, static_cast<const RowDev<T>*>(pl->d_rows), pl->P * pl->K, pl->Nr,
                                         static_cast<const V*>(X), y, pl->env, B, static_cast<const V*>(pl->d_twM), st,
                                         static_cast<const T*>(pl->d_wtab));
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "envelope launch");
}

template <typename T>
qtam_status run_accumulate(qtam_plan_s* pl, const void* y, int64_t B, const MaskEntry* me, void* A, cudaStream_t st) {
  using V = cplx<T>;
  cudaError_t e = cudaMemsetAsync(A, 0, (size_t)B * pl->Nr * sizeof(V), st);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
  if constexpr (sizeof(T) == 4) {
    if (pl->rc.tensor &&
        launch_rows_inverse_tc(pl->rc, static_cast<const RowDev<float>*>(pl->d_rows), me->rows, me->n_sel,
                               pl->P * pl->K, pl->Nr, y, pl->env, static_cast<float2*>(A), B, st,
                               static_cast<const float*>(pl->d_wtab), &e))
      return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "tensor-core accumulate");
  }
  e = launch_rows_inverse<T>(pl->rc, static_cast<const RowDev<T>*>(pl->d_rows), me->rows, me->n_sel, pl->P * pl->K,
                             pl->Nr, y, pl->env, static_cast<V*>(A), B, static_cast<const V*>(pl->d_twM), st,
                             static_cast<const T*>(pl->d_wtab));
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "accumulate launch");
}

template <typename T>
qtam_status run_synthesize(qtam_plan_s* pl, const void* A, int64_t B, const MaskEntry* me, void* x, void* ws,
                           cudaStream_t st) {
  using V = cplx<T>;
  Regions rg = split_ws(pl, ws, B);
  // Zi in region 1, V in region 0 (region 0 may hold A, which the untangle consumes first)
  cudaError_t e = launch_synthesis<T>(pl->lc, static_cast<const V*>(A), static_cast<const T*>(me->invP),
                                      static_cast<V*>(rg.r1), static_cast<V*>(rg.r0), static_cast<V*>(x), B,
                                      static_cast<const V*>(pl->d_twn), static_cast<const V*>(pl->d_twN), st);
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "synthesis launch");
}

qtam_status get_mask(qtam_plan_s* pl, uint64_t mask, MaskEntry** me) {
  qtam_status s = check_mask(pl, mask);
  if (s != QTAM_OK) return s;
  DeviceGuard g(pl->device);
  std::lock_guard<std::mutex> lk(pl->mu);
  return build_mask(pl, mask, me);
}

}  // namespace

namespace qtam {
namespace {
const StreamRowFns* fused_fns(const qtam_plan_s* pl) {
  if (pl->compute != QTAM_DTYPE_F32 || pl->env != QTAM_DTYPE_F32 || !pl->all_bisquare() || pl->rc.tensor ||
      pl->eps > 0 || pl->remod || pl->device < 0)
    return nullptr;
  const RowVariant* v = row_variant(pl->rc.variant);
  return v && pl->rc.stw ? stream_row_fns(v->name) : nullptr;
}
}  // namespace

qtam_status stream_forward_fused(qtam_plan_s* pl, const void* x, int64_t b, void* ymap, int64_t pitch, int Gm, int Hn,
                                 const void* phase, void* ws, size_t wsb, cudaStream_t st, bool* used) {
  *used = false;
  const StreamRowFns* f = fused_fns(pl);
  if (!f || b == 0) return QTAM_OK;
  if (wsb < ws_bytes(pl, b)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  DeviceGuard g(pl->device);
  Regions rg = split_ws(pl, ws, b);
  qtam_status s = run_spectrum<float>(pl, x, b, rg.r0, ws, st);
  if (s != QTAM_OK) return s;
  cudaError_t e = f->fwd(static_cast<const RowDev<float>*>(pl->d_rows), pl->P * pl->K, pl->Nr,
                         static_cast<const float2*>(rg.r0), static_cast<float2*>(ymap), pitch, Gm, Hn,
                         static_cast<const float2*>(phase), b, static_cast<const float2*>(pl->rc.stw), st);
  if (e != cudaSuccess) return fail_cuda(e, "fused stream forward");
  *used = true;
  return QTAM_OK;
}

qtam_status stream_inverse_fused(qtam_plan_s* pl, const void* hist, int hcols, const void* ynew, int64_t pitch, int Hn,
                                 const void* phase, int64_t b, uint64_t mask, void* x, void* ws, size_t wsb,
                                 cudaStream_t st, bool* used) {
  *used = false;
  const StreamRowFns* f = fused_fns(pl);
  if (!f || b == 0) return QTAM_OK;
  if (wsb < ws_bytes(pl, b)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  MaskEntry* me = nullptr;
  qtam_status s = get_mask(pl, mask, &me);
  if (s != QTAM_OK) return s;
  DeviceGuard g(pl->device);
  Regions rg = split_ws(pl, ws, b);
  cudaError_t e = cudaMemsetAsync(rg.r0, 0, (size_t)b * pl->Nr * sizeof(float2), st);
  if (e == cudaSuccess)
    e = f->inv(static_cast<const RowDev<float>*>(pl->d_rows), me->rows, me->n_sel, pl->P * pl->K, pl->Nr,
               static_cast<const float2*>(hist), hcols, static_cast<const float2*>(ynew), pitch, Hn,
               static_cast<const float2*>(phase), static_cast<float2*>(rg.r0), b,
               static_cast<const float2*>(pl->rc.stw), st);
  if (e != cudaSuccess) return fail_cuda(e, "fused stream inverse");
  if ((s = run_synthesize<float>(pl, rg.r0, b, me, x, ws, st)) != QTAM_OK) return s;
  *used = true;
  return QTAM_OK;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }
int plan_device(const qtam_plan_s* plan) { return plan ? plan->device : -1; }
}  // namespace qtam

extern "C" {

void qtam_plan_desc_init(qtam_plan_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->window = QTAM_WIN_BISQUARE;
  d->norm = QTAM_NORM_L2;
  d->q_width = 0.0;
  d->max_window_hz = 0.0;
  d->n_out = 0;
  d->compute_dtype = QTAM_DTYPE_F32;
  d->envelope_dtype = QTAM_DTYPE_F32;
  d->p_floor_rel = -1.0;
}

qtam_status qtam_plan(const qtam_plan_desc* d, int device, qtam_plan_t* out) {
  if (!d || !out) return fail(QTAM_ERR_INVALID_ARG, "desc or out is NULL");
  *out = nullptr;
  if (!(d->sample_rate > 0) || d->length <= 0 || d->length % 2) return fail(QTAM_ERR_INVALID_ARG, "sample_rate > 0 and an even length > 0 are required");
  if (!d->q || d->n_q < 1 || d->n_q > 64) return fail(QTAM_ERR_INVALID_ARG, "1 to 64 Q values are required");
  for (int i = 0; i < d->n_q; ++i)
    if (!(d->q[i] > 0)) return fail(QTAM_ERR_INVALID_ARG, "Q values must be > 0");
  if (d->rows_per_plane < 1) return fail(QTAM_ERR_INVALID_ARG, "rows_per_plane >= 1 required");
  if (!(d->f_min > 0) || !(d->f_max >= d->f_min)) return fail(QTAM_ERR_INVALID_ARG, "0 < f_min <= f_max required");
  if (d->rows_per_plane > 1 && !(d->f_max > d->f_min)) return fail(QTAM_ERR_INVALID_ARG, "f_max > f_min required for K > 1");
  for (int i = 0; i < d->n_q; ++i) {
    const int w = d->plane_window ? d->plane_window[i] : d->window;
    const double a = d->plane_window_param ? d->plane_window_param[i] : d->window_param;
    if (w < QTAM_WIN_BISQUARE || w > QTAM_WIN_PLANCK) return fail(QTAM_ERR_INVALID_ARG, "unknown window");
    if (!std::isfinite(a)) return fail(QTAM_ERR_INVALID_ARG, "window_param must be finite");
    if (w == QTAM_WIN_KAISER && !(a >= 0 && a <= 100)) return fail(QTAM_ERR_INVALID_ARG, "Kaiser beta must lie in [0, 100]");
    if ((w == QTAM_WIN_TUKEY || w == QTAM_WIN_PLANCK) && !(a >= 0 && a <= 1))
      return fail(QTAM_ERR_INVALID_ARG, "taper fraction must lie in [0, 1]");
  }
  if (d->norm < QTAM_NORM_L2 || d->norm > QTAM_NORM_NONE) return fail(QTAM_ERR_INVALID_ARG, "unknown norm");
  if (d->compute_dtype != QTAM_DTYPE_F32 && d->compute_dtype != QTAM_DTYPE_F64) return fail(QTAM_ERR_INVALID_ARG, "compute_dtype must be F32 or F64");
  if (d->compute_dtype == QTAM_DTYPE_F64 && d->envelope_dtype != QTAM_DTYPE_F64) return fail(QTAM_ERR_INVALID_ARG, "F64 compute stores F64 envelopes");
  if (d->compute_dtype == QTAM_DTYPE_F32 && d->envelope_dtype == QTAM_DTYPE_F64) return fail(QTAM_ERR_INVALID_ARG, "F64 envelopes need F64 compute");
  if (d->envelope_dtype < 0 || d->envelope_dtype > QTAM_DTYPE_F16) return fail(QTAM_ERR_INVALID_ARG, "unknown envelope dtype");
  if (d->max_window_hz < 0 || d->n_out < 0) return fail(QTAM_ERR_INVALID_ARG, "max_window_hz and n_out must be >= 0");
  if (d->length > ((int64_t)1 << 27)) return fail(QTAM_ERR_UNSUPPORTED_SIZE, "length above 2^27");
  if (d->short_dft != QTAM_SHORT_DFT_CUDA && d->short_dft != QTAM_SHORT_DFT_TENSOR &&
      d->short_dft != QTAM_SHORT_DFT_AUTO)
    return fail(QTAM_ERR_INVALID_ARG, "unknown short_dft");
  if (!std::isfinite(d->stopband_eps) || d->stopband_eps < 0 || (d->remodulate != 0 && d->remodulate != 1))
    return fail(QTAM_ERR_INVALID_ARG, "stopband_eps must be finite and >= 0, remodulate 0 or 1");
  if ((d->stopband_eps > 0 || d->remodulate) && d->short_dft == QTAM_SHORT_DFT_TENSOR)
    return fail(QTAM_ERR_UNSUPPORTED_SIZE, "the dense mode runs on the CUDA cores, not the tensor-core short DFT");
  if (d->short_dft == QTAM_SHORT_DFT_TENSOR && (d->compute_dtype != QTAM_DTYPE_F32 || d->n_out != 8192))
    return fail(QTAM_ERR_UNSUPPORTED_SIZE, "the tensor-core short DFT needs n_out = 8192 and F32 compute");

  qtam_plan_s* pl = new (std::nothrow) qtam_plan_s();
  if (!pl) return fail(QTAM_ERR_OUT_OF_MEMORY, "host allocation");
  pl->fs = d->sample_rate;
  pl->N = d->length;
  pl->q.assign(d->q, d->q + d->n_q);
  pl->fmin = d->f_min;
  pl->fmax = d->f_max;
  pl->K = d->rows_per_plane;
  pl->norm = d->norm;
  pl->q_width = d->q_width > 0 ? d->q_width : std::sqrt(11.0);
  pl->max_window_hz = d->max_window_hz;
  for (int i = 0; i < d->n_q; ++i) {
    const int w = d->plane_window ? d->plane_window[i] : d->window;
    const double a = d->plane_window_param ? d->plane_window_param[i] : d->window_param;
    pl->window.push_back(w);
    pl->window_param.push_back(w == QTAM_WIN_HANN || w == QTAM_WIN_BISQUARE ? 0.0 : a);
  }
  pl->compute = d->compute_dtype;
  pl->env = d->envelope_dtype;
  pl->short_dft = d->short_dft;
  pl->eps = d->stopband_eps;
  pl->remod = d->remodulate;
  pl->tau = d->p_floor_rel >= 0 ? d->p_floor_rel : (pl->compute == QTAM_DTYPE_F64 ? 0.0 : 1e-6);
  pl->P = d->n_q;
  pl->n = pl->N / 2;
  pl->Nr = pl->n + 1;

  // --- grid and widths (App. A) ---
  const double T = (double)pl->N / pl->fs;
  std::vector<double> grid(pl->K);
  for (int k = 0; k < pl->K; ++k)
    grid[k] = pl->K == 1 ? pl->fmin : pl->fmin * std::pow(pl->fmax / pl->fmin, (double)k / (double)(pl->K - 1));
  double dfmax = 0;
  if (pl->max_window_hz > 0) dfmax = pl->max_window_hz;
  else
    for (int k = 0; k + 1 < pl->K; ++k) dfmax = std::max(dfmax, grid[k + 1] - grid[k]);
  pl->h_max = dfmax > 0 ? (int64_t)std::ceil(T * dfmax) / 2 : ((int64_t)1 << 40);
  const int R = pl->P * pl->K;
  pl->f.resize(R);
  pl->c.resize(R);
  pl->kc.resize(R);
  pl->h.resize(R);
  int64_t Lmax = 0;
  for (int p = 0; p < pl->P; ++p) {
    for (int k = 0; k < pl->K; ++k) {
      const int r = p * pl->K + k;
      const double fk = grid[k];
      pl->f[r] = fk;
      pl->kc[r] = (int64_t)std::floor(fk * T + 0.5);
      int64_t hi = (int64_t)std::floor(fk * T * pl->q_width / pl->q[p]);
      hi = std::max<int64_t>(1, std::min(hi, pl->h_max));
      if (hi > (int64_t)1 << 28) {
        free_plan(pl);
        return fail(QTAM_ERR_UNSUPPORTED_SIZE, "window half-width too large");
      }
      pl->h[r] = (int)hi;
      double s2 = 0;
      for (int64_t dd = -hi; dd <= hi; ++dd) {
        const double w = pl->wprof(dd, hi, p);
        s2 += w * w;
      }
      pl->c[r] = pl->norm == QTAM_NORM_L2 ? 1.0 / std::sqrt(s2) : (pl->norm == QTAM_NORM_PAPER ? 1.0 / s2 : 1.0);
      Lmax = std::max<int64_t>(Lmax, 2 * hi + 1);
      if (pl->kc[r] > pl->n + hi || pl->kc[r] < -hi) {
        free_plan(pl);
        return fail(QTAM_ERR_INVALID_ARG, "a window lies wholly above Nyquist");
      }
    }
  }
  if (pl->eps > 0) Lmax = std::max<int64_t>(Lmax, pl->Nr);   // every tile spans the one-sided spectrum
  pl->Lmax = (int)Lmax;
  if (d->n_out > 0) {
    if (d->n_out < Lmax) {
      free_plan(pl);
      return fail(QTAM_ERR_ALIASING, "n_out is shorter than the largest window");
    }
    pl->M = d->n_out;
  } else {
    pl->M = (int)smooth_at_least(Lmax);
  }

  // --- frame operator per plane (App. C), FP64 ---
  pl->Pplane.assign(pl->P, std::vector<double>(pl->Nr, 0.0));
  pl->band_bins = 0;
  for (int r = 0; r < R; ++r) {
    const int p = r / pl->K;
    const int64_t hk = pl->h[r], kcr = pl->kc[r];
    const int64_t lo = pl->eps > 0 ? -kcr : -hk, hi = pl->eps > 0 ? pl->Nr - 1 - kcr : hk;
    for (int64_t dd = lo; dd <= hi; ++dd) {
      const int64_t fb = kcr + dd;
      if (fb < 0 || fb >= pl->Nr) continue;
      const double w = pl->c[r] * pl->wdense(dd, hk, p);
      pl->Pplane[p][fb] += w * w;
      ++pl->band_bins;
    }
  }

  // --- launch shapes ---
  const bool dbl = pl->compute == QTAM_DTYPE_F64;
  if (!make_radix_plan(pl->M, pl->rc.rp)) {
    free_plan(pl);
    return fail(QTAM_ERR_UNSUPPORTED_SIZE, "n_out must have no prime factor other than 2, 3, 5");
  }
  pl->rc.threads = threads_for(pl->rc.rp, 0);
  pl->rc.smem = smem_for(pl->rc.rp, 0, pl->cplx_size());
  pl->rc.variant = -1;
  if (pl->short_dft == QTAM_SHORT_DFT_AUTO) {
    // the tensor cores where their BF16 rounding is inside the plan's accuracy
    // class (BF16 envelopes) and they serve the length; CUDA cores otherwise
    const bool tc_ok = tc_forward_supported(pl->M) && pl->compute == QTAM_DTYPE_F32 &&
                       pl->env == QTAM_DTYPE_BF16 && pl->eps <= 0 && !pl->remod;
    pl->short_dft = tc_ok ? QTAM_SHORT_DFT_TENSOR : QTAM_SHORT_DFT_CUDA;
  }
  pl->rc.tensor = pl->short_dft == QTAM_SHORT_DFT_TENSOR && tc_forward_supported(pl->M);
  pl->rc.remod = pl->remod;
  pl->rc.dense = (pl->eps > 0 && pl->remod) ? 2 : (pl->eps > 0 || pl->remod) ? 1 : 0;
  if (!dbl) {
    // the first usable variant marked preferred for this length, else the
    // first registered usable one
    for (int pass = 0; pass < 2 && pl->rc.variant < 0; ++pass)
      for (int v = 0; v < row_variant_count(); ++v)
        if (variant_usable(pl, v) && (pass == 1 || row_variant(v)->preferred)) {
          pl->rc.variant = v;
          break;
        }
  }
  if (pl->rc.threads > kMaxThreads || pl->rc.smem > (size_t)kMaxSmem) {
    free_plan(pl);
    return fail(QTAM_ERR_UNSUPPORTED_SIZE, "n_out too large for one thread block");
  }
  if (!choose_long(pl->n, dbl, pl->lc)) {
    free_plan(pl);
    return fail(QTAM_ERR_UNSUPPORTED_SIZE, "length/2 must be a product of 2, 3, 5 between 4 and 2^26");
  }

  pl->device = device;
  if (device >= 0) {
    DeviceGuard g(device);
    if (!g.ok) {
      pl->device = -1;
      free_plan(pl);
      return fail(QTAM_ERR_CUDA, "cudaSetDevice failed");
    }
    qtam_status s = dbl ? upload_tables<double>(pl) : upload_tables<float>(pl);
    if (s != QTAM_OK) {
      free_plan(pl);
      return s;
    }
  }
  MaskEntry* me = nullptr;
  {
    std::lock_guard<std::mutex> lk(pl->mu);
    qtam_status s;
    if (device >= 0) {
      DeviceGuard g(device);
      s = build_mask(pl, pl->all_mask(), &me);
    } else {
      s = build_mask(pl, pl->all_mask(), &me);
    }
    if (s != QTAM_OK) {
      free_plan(pl);
      return s;
    }
  }
  *out = pl;
  return QTAM_OK;
}

qtam_status qtam_plan_info(qtam_plan_t pl, qtam_plan_info_t* o) {
  if (!pl || !o) return fail(QTAM_ERR_INVALID_ARG, "NULL argument");
  std::memset(o, 0, sizeof(*o));
  o->length = pl->N;
  o->n_bins = pl->Nr;
  o->n_planes = pl->P;
  o->rows_per_plane = pl->K;
  o->n_out = pl->M;
  o->h_max = (int32_t)std::min<int64_t>(pl->h_max, INT32_MAX);
  o->max_window = pl->Lmax;
  o->compute_dtype = pl->compute;
  o->envelope_dtype = pl->env;
  o->fft_n1 = pl->lc.n1;
  o->fft_n2 = pl->lc.n2;
  o->envelope_bytes_per_segment = (int64_t)pl->P * pl->K * pl->M * (int64_t)pl->env_size();
  o->band_bins = pl->band_bins;
  o->p_floor_rel = pl->tau;
  std::lock_guard<std::mutex> lk(pl->mu);
  auto it = pl->masks.find(pl->all_mask());
  if (it != pl->masks.end()) {
    o->kappa = it->second.kappa;
    o->kept_bins = it->second.kept;
  }
  o->device_bytes = (int64_t)pl->device_bytes;
  o->row_variant = pl->rc.variant;
  o->short_dft = pl->rc.tensor ? QTAM_SHORT_DFT_TENSOR : QTAM_SHORT_DFT_CUDA;
  o->stopband_eps = pl->eps;
  o->remodulate = pl->remod;
  return QTAM_OK;
}

qtam_status qtam_plan_variants(qtam_plan_t pl, int32_t* ids, int32_t capacity, int32_t* count) {
  if (!pl || !count || capacity < 0 || (capacity > 0 && !ids)) return fail(QTAM_ERR_INVALID_ARG, "bad argument");
  int32_t n = 0;
  auto push = [&](int32_t id) {
    if (n < capacity) ids[n] = id;
    ++n;
  };
  push(-1);
  for (int v = 0; v < row_variant_count(); ++v)
    if (variant_usable(pl, v)) push(v);
  *count = n;
  return QTAM_OK;
}

qtam_status qtam_plan_set_variant(qtam_plan_t pl, int32_t id) {
  if (!pl) return fail(QTAM_ERR_INVALID_ARG, "plan is NULL");
  if (id != -1) {
    if (!variant_usable(pl, id))
      return fail(QTAM_ERR_INVALID_ARG, "variant does not match the plan's envelope length, dtype or window");
  }
  if (id >= 0 && pl->device >= 0) {
    auto it = pl->variant_tw.find(id);
    if (it == pl->variant_tw.end()) return fail(QTAM_ERR_INVALID_ARG, "variant tables were not built for this plan");
    pl->rc.stw = it->second;
  }
  pl->rc.variant = id;
  return QTAM_OK;
}

qtam_status qtam_variant_describe(int32_t id, char* name, size_t capacity, int32_t* threads, int32_t* rows_per_block) {
  if (id == -1) {
    if (name && capacity) std::snprintf(name, capacity, "runtime mixed-radix engine");
    if (threads) *threads = 0;
    if (rows_per_block) *rows_per_block = 1;
    return QTAM_OK;
  }
  const RowVariant* v = row_variant(id);
  if (!v) return fail(QTAM_ERR_INVALID_ARG, "unknown variant");
  if (name && capacity) std::snprintf(name, capacity, "%s", v->name);
  if (threads) *threads = v->threads;
  if (rows_per_block) *rows_per_block = v->rows_per_block;
  return QTAM_OK;
}

qtam_status qtam_plan_rows(qtam_plan_t pl, double* f, int64_t* kc, int32_t* h, double* c) {
  if (!pl) return fail(QTAM_ERR_INVALID_ARG, "plan is NULL");
  const size_t R = pl->f.size();
  for (size_t r = 0; r < R; ++r) {
    if (f) f[r] = pl->f[r];
    if (kc) kc[r] = pl->kc[r];
    if (h) h[r] = pl->h[r];
    if (c) c[r] = pl->c[r];
  }
  return QTAM_OK;
}

qtam_status qtam_frame_operator(qtam_plan_t pl, uint64_t mask, double* p_out) {
  if (!pl || !p_out) return fail(QTAM_ERR_INVALID_ARG, "NULL argument");
  qtam_status s = check_mask(pl, mask);
  if (s != QTAM_OK) return s;
  std::fill(p_out, p_out + pl->Nr, 0.0);
  for (int p = 0; p < pl->P; ++p)
    if ((mask >> p) & 1ull)
      for (int64_t fb = 0; fb < pl->Nr; ++fb) p_out[fb] += pl->Pplane[p][fb];
  return QTAM_OK;
}

qtam_status qtam_workspace_size(qtam_plan_t pl, int64_t batch, size_t* bytes) {
  if (!pl || !bytes || batch < 0) return fail(QTAM_ERR_INVALID_ARG, "bad argument");
  *bytes = ws_bytes(pl, batch);
  return QTAM_OK;
}

qtam_status qtam_stage_spectrum(qtam_plan_t pl, const void* x, int64_t B, void* X, void* ws, size_t wsb, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!x || !X || !ws) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  if (!aligned(x, pl->cplx_size()) || !aligned(X, pl->cplx_size()) || !aligned(ws, 256))
    return fail(QTAM_ERR_INVALID_ARG, "x and X must be aligned to a complex element, workspace to 256 bytes");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pl->compute == QTAM_DTYPE_F64 ? run_spectrum<double>(pl, x, B, X, ws, st) : run_spectrum<float>(pl, x, B, X, ws, st);
}

qtam_status qtam_stage_envelopes(qtam_plan_t pl, const void* X, int64_t B, void* y, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!X || !y) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(X, pl->cplx_size()) || !aligned(y, pl->env_size())) return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pl->compute == QTAM_DTYPE_F64 ? run_envelopes<double>(pl, X, B, y, st) : run_envelopes<float>(pl, X, B, y, st);
}

qtam_status qtam_stage_accumulate(qtam_plan_t pl, const void* y, int64_t B, uint64_t mask, void* A, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK) return s;
  MaskEntry* me = nullptr;
  if ((s = get_mask(pl, mask, &me)) != QTAM_OK || B == 0) return s;
  if (!y || !A) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(A, pl->cplx_size()) || !aligned(y, pl->env_size())) return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pl->compute == QTAM_DTYPE_F64 ? run_accumulate<double>(pl, y, B, me, A, st) : run_accumulate<float>(pl, y, B, me, A, st);
}

qtam_status qtam_stage_synthesize(qtam_plan_t pl, const void* A, int64_t B, uint64_t mask, void* x, void* ws, size_t wsb,
                                  void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK) return s;
  MaskEntry* me = nullptr;
  if ((s = get_mask(pl, mask, &me)) != QTAM_OK || B == 0) return s;
  if (!A || !x || !ws) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  if (!aligned(A, pl->cplx_size()) || !aligned(x, pl->cplx_size()) || !aligned(ws, 256))
    return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pl->compute == QTAM_DTYPE_F64 ? run_synthesize<double>(pl, A, B, me, x, ws, st)
                                       : run_synthesize<float>(pl, A, B, me, x, ws, st);
}

qtam_status qtam_forward(qtam_plan_t pl, const void* x, int64_t B, void* y, void* ws, size_t wsb, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!x || !y || !ws) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  if (!aligned(x, pl->cplx_size()) || !aligned(y, pl->env_size()) || !aligned(ws, 256))
    return fail(QTAM_ERR_INVALID_ARG, "x must be aligned to two samples, y to one envelope element, workspace to 256 bytes");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Regions rg = split_ws(pl, ws, B);
  if (pl->compute == QTAM_DTYPE_F64) {
    if ((s = run_spectrum<double>(pl, x, B, rg.r0, ws, st)) != QTAM_OK) return s;
    return run_envelopes<double>(pl, rg.r0, B, y, st);
  }
  if ((s = run_spectrum<float>(pl, x, B, rg.r0, ws, st)) != QTAM_OK) return s;
  return run_envelopes<float>(pl, rg.r0, B, y, st);
}

qtam_status qtam_inverse(qtam_plan_t pl, const void* y, int64_t B, uint64_t mask, void* x, void* ws, size_t wsb,
                         void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK) return s;
  MaskEntry* me = nullptr;
  if ((s = get_mask(pl, mask, &me)) != QTAM_OK || B == 0) return s;
  if (!x || !y || !ws) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  if (!aligned(x, pl->cplx_size()) || !aligned(y, pl->env_size()) || !aligned(ws, 256))
    return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Regions rg = split_ws(pl, ws, B);
  if (pl->compute == QTAM_DTYPE_F64) {
    if ((s = run_accumulate<double>(pl, y, B, me, rg.r0, st)) != QTAM_OK) return s;
    return run_synthesize<double>(pl, rg.r0, B, me, x, ws, st);
  }
  if ((s = run_accumulate<float>(pl, y, B, me, rg.r0, st)) != QTAM_OK) return s;
  return run_synthesize<float>(pl, rg.r0, B, me, x, ws, st);
}

qtam_status qtam_inverse_single_tile(qtam_plan_t pl, const void* y, int64_t B, int32_t plane, int32_t row, void* x,
                                     void* ws, size_t wsb, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK) return s;
  if (!(pl->eps > 0) || pl->M < pl->Nr)
    return fail(QTAM_ERR_INVALID_ARG, "the single-tile inverse needs the dense mode (stopband_eps > 0)");
  if (plane < 0 || plane >= pl->P || row < 0 || row >= pl->K) return fail(QTAM_ERR_INVALID_ARG, "no such tile");
  MaskEntry* me = nullptr;
  if ((s = get_mask(pl, pl->all_mask(), &me)) != QTAM_OK || B == 0) return s;
  if (!x || !y || !ws) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  if (!aligned(x, pl->cplx_size()) || !aligned(y, pl->env_size()) || !aligned(ws, 256))
    return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Regions rg = split_ws(pl, ws, B);
  const int* one_row = me->rows + (plane * pl->K + row);   // the all-planes row list is 0 .. P K - 1
  const double scale = (double)pl->N / (double)pl->M;
  cudaError_t e;
  if (pl->compute == QTAM_DTYPE_F64) {
    DenseArgs<double> da;
    da.divide = 1;
    da.scale = scale;
    e = launch_rows_inverse<double>(pl->rc, static_cast<const RowDev<double>*>(pl->d_rows), one_row, 1, pl->P * pl->K,
                                    pl->Nr, y, pl->env, static_cast<double2*>(rg.r0), B,
                                    static_cast<const double2*>(pl->d_twM), st, static_cast<const double*>(pl->d_wtab),
                                    da);
    if (e != cudaSuccess) return fail_cuda(e, "single-tile launch");
    e = launch_synthesis<double>(pl->lc, static_cast<const double2*>(rg.r0), static_cast<const double*>(pl->d_ones),
                                 static_cast<double2*>(rg.r1), static_cast<double2*>(rg.r0), static_cast<double2*>(x),
                                 B, static_cast<const double2*>(pl->d_twn), static_cast<const double2*>(pl->d_twN), st);
  } else {
    DenseArgs<float> da;
    da.divide = 1;
    da.scale = (float)scale;
    e = launch_rows_inverse<float>(pl->rc, static_cast<const RowDev<float>*>(pl->d_rows), one_row, 1, pl->P * pl->K,
                                   pl->Nr, y, pl->env, static_cast<float2*>(rg.r0), B,
                                   static_cast<const float2*>(pl->d_twM), st, static_cast<const float*>(pl->d_wtab), da);
    if (e != cudaSuccess) return fail_cuda(e, "single-tile launch");
    e = launch_synthesis<float>(pl->lc, static_cast<const float2*>(rg.r0), static_cast<const float*>(pl->d_ones),
                                static_cast<float2*>(rg.r1), static_cast<float2*>(rg.r0), static_cast<float2*>(x), B,
                                static_cast<const float2*>(pl->d_twn), static_cast<const float2*>(pl->d_twN), st);
  }
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "synthesis launch");
}

qtam_status qtam_roundtrip_host(qtam_plan_t pl, const void* x_host, int64_t B, uint64_t mask, void* xhat_host,
                                void* x_dev, void* y_dev, void* xhat_dev, void* ws, size_t wsb, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!x_host || !xhat_host || !x_dev || !y_dev || !xhat_dev) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (wsb < ws_bytes(pl, B)) return fail(QTAM_ERR_WORKSPACE, "workspace too small");
  DeviceGuard g(pl->device);
  std::lock_guard<std::mutex> lk(pl->rt_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  constexpr int kChunks = 10;
  cudaError_t e = cudaSuccess;
  if (!pl->rt_in) {
    e = cudaStreamCreateWithFlags(&pl->rt_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->rt_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->rt_cs, cudaStreamNonBlocking);
    for (int i = 0; i < 2 * kChunks + 2 && e == cudaSuccess; ++i) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) pl->rt_ev.push_back(ev);
    }
    if (e != cudaSuccess) return fail_cuda(e, "round-trip streams");
  }
  // chunk c holds segments [bound[c], bound[c + 1]); copies of neighbouring
  // chunks overlap the transforms of chunk c.  Inner
  // chunks carry about 16 MB of input (smaller ones pay per-chunk launch and
  // tail costs; measured best on the 64 s workload); the first and last
  // chunks are cut to about B/16 segments, since their copies cannot overlap
  // anything
  const size_t xs = (size_t)pl->N * pl->real_size();
  std::vector<int64_t> bound{0};
  {
    const int64_t by_bytes = (int64_t)((size_t)B * xs / (16u << 20));
    if (by_bytes < 2) {
      bound.push_back(B);
    } else {
      const int64_t edge = std::max<int64_t>(1, B / 16);
      const int64_t inner = B - 2 * edge;
      const int64_t ni = std::max<int64_t>(
          1, std::min<int64_t>({(int64_t)kChunks - 2, inner, (int64_t)((size_t)inner * xs / (16u << 20))}));
      bound.push_back(edge);
      for (int64_t i = 1; i <= ni; ++i) bound.push_back(edge + inner * i / ni);
      bound.push_back(B);
    }
  }
  const int C = (int)bound.size() - 1;
  const size_t ys = (size_t)pl->P * pl->K * pl->M * pl->env_size();
  // Odd chunks run on a second library-owned stream with their own half of
  // the workspace when two chunk workspaces fit, so a chunk's first kernels
  // fill the last waves of the one before (short chunks leave the GPU half
  // idle in their tails); even chunks stay on the caller's stream.
  int64_t maxnb = 0;
  for (int c = 0; c < C; ++c) maxnb = std::max<int64_t>(maxnb, bound[c + 1] - bound[c]);
  const size_t slot = (ws_bytes(pl, maxnb) + 255) / 256 * 256;
  const bool two = C > 1 && 2 * slot <= wsb && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0;
  auto chunk_stream = [&](int c) { return (two && (c & 1)) ? pl->rt_cs : st; };
  auto chunk_ws = [&](int c) { return (two && (c & 1)) ? static_cast<void*>(static_cast<char*>(ws) + slot) : ws; };
  const size_t chunk_wsb = two ? slot : wsb;
  cudaEvent_t ev_start = pl->rt_ev[0], ev_end = pl->rt_ev[1];
  cudaEvent_t* ev_in = &pl->rt_ev[2];
  cudaEvent_t* ev_done = &pl->rt_ev[2 + kChunks];
  auto seg0 = [&](int c) { return bound[c]; };
  if ((e = cudaEventRecord(ev_start, st)) != cudaSuccess) return fail_cuda(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(pl->rt_in, ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(pl->rt_out, ev_start, 0)) != cudaSuccess ||
      (two && (e = cudaStreamWaitEvent(pl->rt_cs, ev_start, 0)) != cudaSuccess))
    return fail_cuda(e, "cudaStreamWaitEvent");
  for (int c = 0; c < C; ++c) {
    const int64_t s0 = seg0(c), nb = seg0(c + 1) - s0;
    e = cudaMemcpyAsync(static_cast<char*>(x_dev) + s0 * xs, static_cast<const char*>(x_host) + s0 * xs, nb * xs,
                        cudaMemcpyHostToDevice, pl->rt_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[c], pl->rt_in);
    if (e != cudaSuccess) return fail_cuda(e, "host-to-device copy");
  }
  for (int c = 0; c < C; ++c) {
    const int64_t s0 = seg0(c), nb = seg0(c + 1) - s0;
    cudaStream_t cs = chunk_stream(c);
    if ((e = cudaStreamWaitEvent(cs, ev_in[c], 0)) != cudaSuccess) return fail_cuda(e, "cudaStreamWaitEvent");
    void* xc = static_cast<char*>(x_dev) + s0 * xs;
    void* yc = static_cast<char*>(y_dev) + s0 * ys;
    void* hc = static_cast<char*>(xhat_dev) + s0 * xs;
    if ((s = qtam_forward(pl, xc, nb, yc, chunk_ws(c), chunk_wsb, cs)) != QTAM_OK) return s;
    if ((s = qtam_inverse(pl, yc, nb, mask, hc, chunk_ws(c), chunk_wsb, cs)) != QTAM_OK) return s;
    if ((e = cudaEventRecord(ev_done[c], cs)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(pl->rt_out, ev_done[c], 0)) != cudaSuccess)
      return fail_cuda(e, "chunk ordering");
    e = cudaMemcpyAsync(static_cast<char*>(xhat_host) + s0 * xs, hc, nb * xs, cudaMemcpyDeviceToHost, pl->rt_out);
    if (e != cudaSuccess) return fail_cuda(e, "device-to-host copy");
  }
  if ((e = cudaEventRecord(ev_end, pl->rt_out)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ev_end, 0)) != cudaSuccess)
    return fail_cuda(e, "round-trip join");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
  return QTAM_OK;
}

qtam_status qtam_plane_metrics(qtam_plan_t pl, const void* y, int64_t B, double* energy, float* peak, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!y || !energy || !peak) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(y, pl->env_size()) || !aligned(energy, 8) || !aligned(peak, 4)) return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  if (B * pl->P > 0x7fffffff) return fail(QTAM_ERR_UNSUPPORTED_SIZE, "too many (segment, plane) pairs");
  DeviceGuard g(pl->device);
  cudaError_t e = launch_plane_metrics(y, pl->env, B * pl->P, (int64_t)pl->K * pl->M, energy, peak,
                                       static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "plane_metrics launch");
}

qtam_status qtam_scale_rows(qtam_plan_t pl, void* y, int64_t B, const float* gain, void* stream) {
  qtam_status s = common_checks(pl, B);
  if (s != QTAM_OK || B == 0) return s;
  if (!y || !gain) return fail(QTAM_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(y, pl->env_size()) || !aligned(gain, 4)) return fail(QTAM_ERR_INVALID_ARG, "misaligned buffer");
  DeviceGuard g(pl->device);
  cudaError_t e = launch_scale_rows(y, pl->env, gain, B * (int64_t)pl->P * pl->K, pl->M, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? QTAM_OK : fail_cuda(e, "scale_rows launch");
}

qtam_status qtam_batched_workspace_size(const qtam_group* g, int32_t n, size_t* bytes) {
  if (!bytes || n < 0 || (n > 0 && !g)) return fail(QTAM_ERR_INVALID_ARG, "bad argument");
  size_t mx = 256;
  for (int32_t i = 0; i < n; ++i) {
    if (!g[i].plan || g[i].batch < 0) return fail(QTAM_ERR_INVALID_ARG, "group with NULL plan or negative batch");
    mx = std::max(mx, ws_bytes(g[i].plan, g[i].batch));
  }
  *bytes = mx;
  return QTAM_OK;
}

namespace {
qtam_status check_groups(const qtam_group* g, int32_t n, size_t wsb) {
  if (n < 0 || (n > 0 && !g)) return fail(QTAM_ERR_INVALID_ARG, "bad group list");
  int dev = -2;
  for (int32_t i = 0; i < n; ++i) {
    qtam_status s = common_checks(g[i].plan, g[i].batch);
    if (s != QTAM_OK) return s;
    if (dev != -2 && g[i].plan->device != dev) return fail(QTAM_ERR_INVALID_ARG, "groups on different devices");
    dev = g[i].plan->device;
    if (g[i].batch > 0 && (!g[i].in || !g[i].out)) return fail(QTAM_ERR_INVALID_ARG, "group with NULL buffer");
    if (wsb < ws_bytes(g[i].plan, g[i].batch)) return fail(QTAM_ERR_WORKSPACE, "workspace too small for a group");
  }
  return QTAM_OK;
}
}  // namespace

qtam_status qtam_forward_batched(const qtam_group* g, int32_t n, void* ws, size_t wsb, void* stream) {
  qtam_status s = check_groups(g, n, wsb);
  if (s != QTAM_OK) return s;
  for (int32_t i = 0; i < n; ++i)
    if ((s = qtam_forward(g[i].plan, g[i].in, g[i].batch, g[i].out, ws, wsb, stream)) != QTAM_OK) return s;
  return QTAM_OK;
}

qtam_status qtam_inverse_batched(const qtam_group* g, int32_t n, uint64_t mask, void* ws, size_t wsb, void* stream) {
  qtam_status s = check_groups(g, n, wsb);
  if (s != QTAM_OK) return s;
  for (int32_t i = 0; i < n; ++i)
    if ((s = qtam_inverse(g[i].plan, g[i].in, g[i].batch, mask, g[i].out, ws, wsb, stream)) != QTAM_OK) return s;
  return QTAM_OK;
}

qtam_status qtam_destroy(qtam_plan_t pl) {
  free_plan(pl);
  return QTAM_OK;
}

const char* qtam_status_string(qtam_status s) {
  switch (s) {
    case QTAM_OK: return "ok";
    case QTAM_ERR_INVALID_ARG: return "invalid argument";
    case QTAM_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case QTAM_ERR_ALIASING: return "n_out shorter than the largest window (aliasing)";
    case QTAM_ERR_NO_COVERAGE: return "no frequency bin is covered";
    case QTAM_ERR_OUT_OF_MEMORY: return "out of memory";
    case QTAM_ERR_CUDA: return "CUDA error";
    case QTAM_ERR_TIMEOUT: return "device wait timed out";
    case QTAM_ERR_NO_DEVICE: return "host-only plan";
    case QTAM_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

const char* qtam_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
