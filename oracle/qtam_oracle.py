"""FP64 CPU oracle of the QTAM analysis/synthesis pair (arXiv 2603.29785).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the library: geometry, windows, the frame
operator and both transforms are written out again here from the paper, in
float64, with numpy's FFT as the only library step (the FFT is itself pinned
against a naive O(N^2) DFT by the tests).

What is computed, in the paper's notation
-----------------------------------------
x       real segment of N samples at rate fs, duration T = N / fs (the paper's N_t)
X[f]    one-sided DFT, f = 0 .. N/2                      (App. C, DFT definition)
f_k     centre frequencies, log grid per plane             (App. A, frequency grid)
k_c     centre bin round(f_k T)                            (Eq. support: k_c = f N_t)
h       window half-width (the paper's Delta k_f)          (Eq. support; App. A clamp)
W_k[f]  c_k (1 - ((f - k_c)/h)^2)^2 on |f - k_c| <= h      (Eq. gwpy_window_formula)
M       envelope length (the paper's N_out)                (Sec. III, demodulation)
Y_k[n]  sqrt(M/N) * IDFT_M of the band shifted to baseband (Sec. III; App. C,
        "QTAM demodulation" normalisation)
P[f]    sum_k W_k[f]^2, the diagonal frame operator        (App. C)
x_hat   irfft( sum_k T~_k W_k / P )                        (Eq. qtam_canonical_inverse)

Readings where the paper is silent or garbled (each is a plan option or a
documented choice; the same list is kept in the design notes):
  C1  log grid with both endpoints: f_k = fmin (fmax/fmin)^(k/(K-1)).
  C2  h_ideal = floor(f_k T q_width / Q), q_width = sqrt(11) (rms half-width of
      the bisquare's square is h/sqrt(11), so Q = f / sigma_f).
  C3  Delta f_max = largest gap between consecutive centres; h_max =
      floor(ceil(T Delta f_max) / 2)  (L_max = 2 h_max + 1, App. A clamp);
      h = max(1, min(h_ideal, h_max)).  A manual clamp in Hz replaces Delta f_max.
  C4  c_k = (sum_d W'(d)^2)^(-1/2) over the untruncated window ("L2", default);
      "paper" = 1 / sum_d W'(d)^2 (Eq. gwpy_window_and_normalization read
      literally); "none" = 1.
  C5  M = smallest 2^a 3^b 5^c >= max_k L_k (lossless iff M >= L); N_in = N.
  C6  windows are truncated to 0 <= f <= N/2 (no Hermitian folding).
  C7  k_c rounds half away from zero.
  C8  the inverse divides by P only on F_tau = {f : P[f] > 0, P[f] >= tau max P}
      and sets X_hat = 0 elsewhere: the round trip is the orthogonal projection
      of x onto F_tau.
  C9  a plane mask selects the planes whose rows are synthesised and whose
      windows enter P.
  D1  dense mode (Sec. III alternative inversion; App. A regularisation):
      with stopband_eps > 0 every window is W' where W' > 0 and eps wherever
      it vanishes (outside |d| <= h, and at the edge points |d| = h where the
      printed window is exactly zero although the text wants it strictly
      non-zero), so each tile spans all N/2 + 1 bins
      (M >= N/2 + 1 for a lossless tile) and any single tile inverts by
      spectral division, x = irfft( T~_k / W_k ) (the equation after
      Eq. qtam_window_formula).  c_k keeps its value from the band.  With
      remodulate the envelope is multiplied by exp(+2 pi i k_c n / M), the
      carrier the demodulation removed: the tile is then the plain inverse
      DFT of the unshifted filtered spectrum X W_k (the undemodulated,
      "standard" tile, here on M columns).
  S1  streaming (the paper motivates hours-long signals, Sec. I, without
      fixing a scheme): overlap-save with chunks of the plan's length N, hop H
      and guard G = (N - H)/2 on each side; each chunk keeps its central
      H M / N envelope columns.  H and G are multiples of N / gcd(N, M) so
      that column and sample boundaries coincide.  A chunk starting a samples
      after the stream origin has its envelopes multiplied by
      exp(-2 pi i k_c a / N), so every chunk is demodulated against the same
      time origin and the map is continuous across chunks (the inverse
      multiplies by the conjugate).  A remodulated tile (D1) already carries
      its carrier exp(+2 pi i k_c n / M) on absolute time: a circular shift
      of x by a samples only shifts its columns, so its re-reference factor
      is 1.  The stream is preceded by
      2G zeros; map column c is time c N/M - G, and the streaming inverse
      (re-chunk the map the same way, keep each chunk's central H samples)
      returns sample s at time s - 2G.

Parity of every function here is pinned by the ``-m "not gpu"`` oracle tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NORMS = ("l2", "paper", "none")


# ----------------------------------------------------------------------------
# geometry (App. A: frequency grid, window length, clamp)
# ----------------------------------------------------------------------------
def smooth_length(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5 (reading C5)."""
    m = max(1, int(n))
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def log_grid(fmin: float, fmax: float, K: int) -> np.ndarray:
    """Log-spaced centre frequencies, both endpoints included (App. A grid, reading C1)."""
    if K == 1:
        return np.array([float(fmin)])
    k = np.arange(K, dtype=np.float64)
    return fmin * (fmax / fmin) ** (k / (K - 1))


def round_half_away(v: float) -> int:
    """k_c = f N_t is not an integer (Eq. support); round half away from zero (C7)."""
    return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)


@dataclass
class Geometry:
    fs: float
    N: int
    qs: tuple
    fmin: float
    fmax: float
    K: int
    norm: str
    q_width: float
    h_max: int              # clamp half-width (App. A), or a huge value when unclamped
    M: int                  # envelope length N_out
    f: np.ndarray           # [P, K] centre frequencies
    kc: np.ndarray          # [P, K] centre bins
    h: np.ndarray           # [P, K] half-widths
    c: np.ndarray           # [P, K] window normalisation c_k
    window: object = "bisquare"       # one name, or one per plane (composite bank)
    window_param: object = 0.0        # one value, or one per plane
    eps: float = 0.0                  # stopband floor of every window (reading D1)
    remodulate: bool = False          # envelopes carry the carrier again (reading D1)
    extra: dict = field(default_factory=dict)

    def plane_window(self, p: int):
        """(window name, shape parameter) of plane p: a plane of the bank is a
        (Q, window, parameter) configuration (App. A, composite filter bank)."""
        w = self.window if isinstance(self.window, str) else self.window[p]
        a = self.window_param if np.ndim(self.window_param) == 0 else self.window_param[p]
        return w, float(a)

    @property
    def P(self) -> int:
        return len(self.qs)

    @property
    def T(self) -> float:
        return self.N / self.fs

    @property
    def Nr(self) -> int:
        return self.N // 2 + 1

    @property
    def L(self) -> np.ndarray:
        return 2 * self.h + 1


def bisquare_profile(d: np.ndarray, h: int) -> np.ndarray:
    """Unnormalised bisquare W'(d) = (1 - (d/h)^2)^2 for |d| <= h, else 0.

    Eq. gwpy_window_formula.  (1 - (d/h)^2) is formed as (h-|d|)(h+|d|)/h^2 with
    the product taken exactly in integers, so values near the window edge carry
    no cancellation error.
    """
    d = np.asarray(d, dtype=np.int64)
    a = np.abs(d)
    num = (h - a) * (h + a)                       # exact integer
    u = num.astype(np.float64) / float(h * h)
    return np.where(a <= h, u * u, 0.0)


WINDOWS = ("bisquare", "hann", "kaiser", "tukey", "planck")


def window_profile(d: np.ndarray, h: int, window: str = "bisquare", param: float = 0.0) -> np.ndarray:
    """Unnormalised spectral window W'(d), |d| <= h, of App. A with u = d/h:

    bisquare  (1 - u^2)^2                              (Eq. gwpy_window_formula)
    hann      (1 + cos(pi u)) / 2
    kaiser    I0(beta sqrt(1 - u^2)) / I0(beta),        param = beta
    tukey     1 on |u| <= 1 - a; (1 + cos(pi (|u| - (1 - a)) / a)) / 2 beyond,  param = a
    planck    1 on |u| <= 1 - a; 1 / (exp(Z) + 1) beyond with t = 1 - |u|,
              Z = a / t - a / (a - t),  param = a
    The printed Planck exponent adds both terms; taken literally the window would
    jump from 1 to 0 at the plateau edge, so the standard continuous form (the
    second term with the opposite sign) is used.
    """
    if window == "bisquare":
        return bisquare_profile(d, h)
    d = np.asarray(d, dtype=np.int64)
    a = np.abs(d)
    u = a.astype(np.float64) / float(h)
    w = np.zeros(u.shape)
    inside = a <= h
    if window == "hann":
        w = 0.5 * (1.0 + np.cos(np.pi * u))
    elif window == "kaiser":
        beta = float(param)
        w = np.i0(beta * np.sqrt(np.clip(1.0 - u * u, 0.0, None))) / np.i0(beta)
    elif window == "tukey":
        al = float(param)
        w = np.ones(u.shape)
        if al > 0:
            edge = u > 1.0 - al
            w[edge] = 0.5 * (1.0 + np.cos(np.pi * (u[edge] - (1.0 - al)) / al))
    elif window == "planck":
        al = float(param)
        w = np.ones(u.shape)
        t = 1.0 - u
        edge = (t < al) & (t > 0)
        if al > 0:
            z = al / t[edge] - al / (al - t[edge])
            w[edge] = 1.0 / (np.exp(np.clip(z, -700, 700)) + 1.0)
        w[t <= 0] = 0.0
    else:
        raise ValueError(window)
    return np.where(inside, w, 0.0)


def window_norm(h: int, norm: str, window: str = "bisquare", param: float = 0.0) -> float:
    """c_k of Eq. gwpy_window_and_normalization under reading C4."""
    d = np.arange(-h, h + 1)
    s2 = float(np.sum(window_profile(d, h, window, param) ** 2))
    if norm == "l2":
        return 1.0 / math.sqrt(s2)
    if norm == "paper":
        return 1.0 / s2
    if norm == "none":
        return 1.0
    raise ValueError(norm)


def geometry(fs, N, qs, fmin, fmax, K, norm="l2", q_width=math.sqrt(11.0),
             max_window_hz=0.0, n_out=0, window="bisquare", window_param=0.0,
             stopband_eps=0.0, remodulate=False) -> Geometry:
    """Plan the filter bank: grid, centre bins, half-widths, c_k and M.

    App. A (grid f_k, L_k^ideal proportional to f_k N_t / Q, automatic clamp
    L_max = 2 floor(ceil(N_t Delta f_max)/2) + 1, L_k = min(L_k^ideal, L_max))
    and Sec. IV's minimal output length, under readings C1-C5.
    """
    N = int(N)
    if N <= 0 or N % 2:
        raise ValueError("N must be a positive even integer")
    T = N / fs
    grid = log_grid(fmin, fmax, K)
    if max_window_hz > 0:
        df_max = float(max_window_hz)
    elif K >= 2:
        df_max = float(np.max(np.diff(grid)))
    else:
        df_max = math.inf
    if math.isinf(df_max):
        h_max = 1 << 62
    else:
        h_max = int(math.ceil(T * df_max)) // 2
    P = len(qs)
    if not isinstance(window, str) and len(window) != P:
        raise ValueError("one window per plane is required")
    if np.ndim(window_param) != 0 and len(window_param) != P:
        raise ValueError("one window parameter per plane is required")
    f = np.zeros((P, K))
    kc = np.zeros((P, K), dtype=np.int64)
    h = np.zeros((P, K), dtype=np.int64)
    c = np.zeros((P, K))
    for p, Q in enumerate(qs):
        for k in range(K):
            f[p, k] = grid[k]
            kc[p, k] = round_half_away(grid[k] * T)
            h_ideal = int(math.floor(grid[k] * T * q_width / Q))
            h[p, k] = max(1, min(h_ideal, h_max))
            wname = window if isinstance(window, str) else window[p]
            wpar = window_param if np.ndim(window_param) == 0 else window_param[p]
            c[p, k] = window_norm(int(h[p, k]), norm, wname, float(wpar))
    Lmax = int(np.max(2 * h + 1))
    if stopband_eps < 0:
        raise ValueError("stopband_eps must be >= 0")
    if stopband_eps > 0:
        Lmax = max(Lmax, N // 2 + 1)          # every tile spans the whole one-sided spectrum
    if n_out:
        if n_out < Lmax:
            raise ValueError("n_out shorter than the largest window: aliasing")
        M = int(n_out)
    else:
        M = smooth_length(Lmax)
    return Geometry(fs=float(fs), N=N, qs=tuple(float(q) for q in qs), fmin=float(fmin),
                    fmax=float(fmax), K=int(K), norm=norm, q_width=float(q_width),
                    h_max=int(h_max), M=M, f=f, kc=kc, h=h, c=c,
                    window=window if isinstance(window, str) else tuple(window),
                    window_param=float(window_param) if np.ndim(window_param) == 0
                    else tuple(float(a) for a in window_param),
                    eps=float(stopband_eps), remodulate=bool(remodulate))


def row_weight(g: Geometry, p: int, k: int, d: np.ndarray) -> np.ndarray:
    """c_k W_k at offsets d from the centre: the window where it is positive
    and the stopband floor eps wherever it vanishes -- outside |d| <= h and at
    the support's edge points, where the printed window is exactly zero
    (reading D1; eps = 0 by default)."""
    d = np.asarray(d, dtype=np.int64)
    w = window_profile(d, int(g.h[p, k]), *g.plane_window(p))
    if g.eps > 0:
        w = np.where(w > 0, w, g.eps)
    return g.c[p, k] * w


def carrier(g: Geometry, p: int, k: int) -> np.ndarray:
    """exp(+2 pi i k_c n / M), n = 0..M-1 (k_c n reduced mod M in integers)."""
    n = np.arange(g.M, dtype=np.int64)
    return np.exp(2j * np.pi * np.mod(int(g.kc[p, k]) * n, g.M) / g.M)


def window(g: Geometry, p: int, k: int) -> np.ndarray:
    """Dense W_k[f], f = 0..N/2, truncated to the one-sided band (reading C6)."""
    fbin = np.arange(g.Nr)
    return row_weight(g, p, k, fbin - g.kc[p, k])


def frame_operator(g: Geometry, planes=None) -> np.ndarray:
    """P[f] = sum_k |W_k[f]|^2 over the selected planes (App. C, frame operator)."""
    planes = range(g.P) if planes is None else planes
    Pf = np.zeros(g.Nr)
    for p in planes:
        for k in range(g.K):
            Pf += window(g, p, k) ** 2
    return Pf


def kept_bins(Pf: np.ndarray, tau: float) -> np.ndarray:
    """F_tau = {f : P[f] > 0 and P[f] >= tau max P} (reading C8)."""
    return (Pf > 0) & (Pf >= tau * np.max(Pf))


# ----------------------------------------------------------------------------
# transforms
# ----------------------------------------------------------------------------
def spectrum(x: np.ndarray) -> np.ndarray:
    """X[f] = sum_n x[n] exp(-2 pi i f n / N), f = 0..N/2 (App. C, DFT)."""
    return np.fft.rfft(np.asarray(x, dtype=np.float64))


def band(g: Geometry, p: int, k: int):
    """Offsets d in [-h, h] whose bins k_c + d lie in 0..N/2, and those bins
    (every bin 0..N/2 in dense mode, reading D1)."""
    hk = int(g.h[p, k])
    if g.eps > 0:
        fb = np.arange(g.Nr)
        return fb - g.kc[p, k], fb
    d = np.arange(-hk, hk + 1)
    fb = g.kc[p, k] + d
    ok = (fb >= 0) & (fb <= g.N // 2)
    return d[ok], fb[ok]


def forward_row(g: Geometry, X: np.ndarray, p: int, k: int) -> np.ndarray:
    """Envelope Y_k[n], n = 0..M-1, of one row (Sec. III demodulation; App. A).

    1. filter:   S'_k[d] = W_k[k_c + d] X[k_c + d]     (element-wise product)
    2. shift:    roll by -k_c so the band sits at baseband, Z[d mod M] = S'_k[d]
                 (crop to the band, zero-pad symmetrically to M)
    3. IFFT of length M and renormalise by sqrt(N_out / N_in) = sqrt(M/N):
                 Y_k[n] = sqrt(M/N) * (1/M) sum_j Z[j] exp(+2 pi i j n / M)
    """
    d, fb = band(g, p, k)
    Z = np.zeros(g.M, dtype=np.complex128)
    Z[d % g.M] = row_weight(g, p, k, d) * X[fb]
    Y = np.fft.ifft(Z) * math.sqrt(g.M / g.N)
    return Y * carrier(g, p, k) if g.remodulate else Y


def forward(g: Geometry, x: np.ndarray) -> np.ndarray:
    """QTAM analysis of one segment: Y[p, k, n] complex128 of shape [P, K, M]."""
    X = spectrum(x)
    Y = np.zeros((g.P, g.K, g.M), dtype=np.complex128)
    for p in range(g.P):
        for k in range(g.K):
            Y[p, k] = forward_row(g, X, p, k)
    return Y


def accumulate(g: Geometry, Y: np.ndarray, planes=None) -> np.ndarray:
    """A[f] = sum_k W_k^*[f] T~_k[f]: the numerator of Eq. qtam_canonical_inverse.

    Each row's tile spectrum is recovered from the envelope by an FFT of length
    M, re-scaled by sqrt(N_in/N_out) = sqrt(N/M) and shifted back from baseband
    to its carrier k_c (App. C, synthesis step), then weighted by the window.
    """
    planes = range(g.P) if planes is None else planes
    A = np.zeros(g.Nr, dtype=np.complex128)
    for p in planes:
        for k in range(g.K):
            y = Y[p, k] * np.conj(carrier(g, p, k)) if g.remodulate else Y[p, k]
            S = np.fft.fft(y) * math.sqrt(g.N / g.M)
            d, fb = band(g, p, k)
            A[fb] += row_weight(g, p, k, d) * S[d % g.M]
    return A


def real_ifft(Xh: np.ndarray, N: int) -> np.ndarray:
    """Inverse of the one-sided DFT for a real signal; the imaginary parts of
    the DC and Nyquist bins are dropped (the real signal's spectrum is
    Hermitian there)."""
    Xh = np.array(Xh, dtype=np.complex128)
    Xh[0] = Xh[0].real
    Xh[N // 2] = Xh[N // 2].real
    return np.fft.irfft(Xh, n=N)


def inverse(g: Geometry, Y: np.ndarray, planes=None, tau: float = 0.0) -> np.ndarray:
    """Canonical dual-frame synthesis (Eq. qtam_canonical_inverse; App. C):
    x_hat = F^-1{ A[f] / P[f] } on F_tau, 0 elsewhere (reading C8)."""
    A = accumulate(g, Y, planes)
    Pf = frame_operator(g, planes)
    keep = kept_bins(Pf, tau)
    Xh = np.zeros(g.Nr, dtype=np.complex128)
    Xh[keep] = A[keep] / Pf[keep]
    return real_ifft(Xh, g.N)


def inverse_single_tile(g: Geometry, Y: np.ndarray, p: int, k: int) -> np.ndarray:
    """Reconstruction from the one tile (p, k) by spectral division (the
    equation after Eq. qtam_window_formula): the tile spectrum shifted back to
    its carrier, T~_k[f] = sqrt(N/M) FFT_M(Y_k)[f - k_c], divided by c_k W_k[f]
    on every bin; needs the dense mode (eps > 0, M >= N/2 + 1)."""
    if g.eps <= 0 or g.M < g.Nr:
        raise ValueError("the single-tile inverse needs stopband_eps > 0 and M >= N/2 + 1")
    y = Y[p, k] * np.conj(carrier(g, p, k)) if g.remodulate else Y[p, k]
    S = np.fft.fft(y) * math.sqrt(g.N / g.M)
    d, fb = band(g, p, k)
    Xh = np.zeros(g.Nr, dtype=np.complex128)
    Xh[fb] = S[d % g.M] / row_weight(g, p, k, d)
    return real_ifft(Xh, g.N)


def projection(g: Geometry, x: np.ndarray, planes=None, tau: float = 0.0) -> np.ndarray:
    """x_proj = irfft(X 1[F_tau]): what an exact round trip returns (App. C
    exact reconstruction where P > 0; reading C8 elsewhere)."""
    X = spectrum(x)
    keep = kept_bins(frame_operator(g, planes), tau)
    return real_ifft(np.where(keep, X, 0.0), g.N)


def kappa(g: Geometry, planes=None, tau: float = 0.0) -> float:
    """Worst amplification of the dual frame on F_tau: max_f (max_k W_k[f]) / P[f]."""
    planes = range(g.P) if planes is None else planes
    Pf = frame_operator(g, planes)
    Wmax = np.zeros(g.Nr)
    for p in planes:
        for k in range(g.K):
            Wmax = np.maximum(Wmax, window(g, p, k))
    keep = kept_bins(Pf, tau)
    return float(np.max(Wmax[keep] / Pf[keep]))


# ----------------------------------------------------------------------------
# optimal-plane selection (App. A, multi-Q bank: "optimal selection" mode)
# ----------------------------------------------------------------------------
def plane_metrics(Y: np.ndarray):
    """Per Q-plane signal-quality metrics of one segment's envelopes Y[P, K, M]:
    total energy sum_{k,n} |Y|^2 and peak pixel intensity max_{k,n} |Y|^2, and
    the plane each criterion selects (App. A: full scan vs optimal selection,
    chosen independently for every signal)."""
    e = np.sum(np.abs(Y) ** 2, axis=(1, 2))
    pk = np.max(np.abs(Y) ** 2, axis=(1, 2))
    return e, pk, int(np.argmax(e)), int(np.argmax(pk))


# ----------------------------------------------------------------------------
# streaming (reading S1): overlap-save over a continuous signal
# ----------------------------------------------------------------------------
def stream_quantum(g: Geometry) -> int:
    """Smallest sample count whose envelope column count is whole: N / gcd(N, M)."""
    return g.N // math.gcd(g.N, g.M)


def stream_layout(g: Geometry, hop: int):
    """(G, Hn, Gm): guard samples, kept columns per chunk, guard columns."""
    q = stream_quantum(g)
    if hop <= 0 or hop > g.N or hop % q or (g.N - hop) % (2 * q):
        raise ValueError("hop must be a positive multiple of the column quantum with (N - hop)/2 one too")
    G = (g.N - hop) // 2
    return G, hop * g.M // g.N, G * g.M // g.N


def stream_phase(g: Geometry, a: int) -> np.ndarray:
    """[P, K] factors exp(-2 pi i k_c a / N) that re-reference the envelopes of a
    chunk starting at stream sample a to the stream origin (k_c a reduced mod N
    in integers first); 1 for remodulated tiles, whose carrier
    exp(+2 pi i k_c n / M) already refers column n to absolute time
    (reading S1)."""
    if g.remodulate:
        return np.ones(g.kc.shape, dtype=np.complex128)
    m = np.mod(g.kc.astype(np.int64) * int(a), g.N)
    return np.exp(-2j * np.pi * m / g.N)


def stream_forward(g: Geometry, x: np.ndarray, hop: int) -> np.ndarray:
    """Envelope map [P, K, J Hn] of a stream of J hops: chunk i is the N samples
    starting at stream sample a = i hop - 2G (the stream is preceded by 2G
    zeros); its envelopes, re-referenced by stream_phase(a), give columns
    Gm .. Gm + Hn - 1 as map columns i Hn .. (i + 1) Hn - 1."""
    G, Hn, Gm = stream_layout(g, hop)
    x = np.asarray(x, dtype=np.float64)
    if x.size % hop:
        raise ValueError("the stream must be a whole number of hops")
    J = x.size // hop
    xp = np.concatenate([np.zeros(2 * G), x])
    out = np.zeros((g.P, g.K, J * Hn), dtype=np.complex128)
    for i in range(J):
        Y = forward(g, xp[i * hop: i * hop + g.N]) * stream_phase(g, i * hop - 2 * G)[:, :, None]
        out[:, :, i * Hn:(i + 1) * Hn] = Y[:, :, Gm:Gm + Hn]
    return out


def stream_inverse(g: Geometry, Ymap: np.ndarray, hop: int, planes=None, tau: float = 0.0) -> np.ndarray:
    """Samples [J hop] from an envelope map of J Hn columns: chunk i takes the
    map columns i Hn - 2 Gm .. i Hn - 2 Gm + M - 1 (zeros before the map),
    which belong to the chunk starting at sample a = i hop - 3G of the forward
    stream's time axis; it is taken back to its own origin (conjugate of
    stream_phase(a)), inverted with Eq. qtam_canonical_inverse, and gives its
    central hop samples G .. G + hop - 1."""
    G, Hn, Gm = stream_layout(g, hop)
    if Ymap.shape[2] % Hn:
        raise ValueError("the map must be a whole number of chunks")
    J = Ymap.shape[2] // Hn
    Yp = np.concatenate([np.zeros((g.P, g.K, 2 * Gm), dtype=np.complex128), Ymap], axis=2)
    out = np.zeros(J * hop)
    for i in range(J):
        Yi = Yp[:, :, i * Hn: i * Hn + g.M] * np.conj(stream_phase(g, i * hop - 3 * G))[:, :, None]
        xh = inverse(g, Yi, planes=planes, tau=tau)
        out[i * hop:(i + 1) * hop] = xh[G:G + hop]
    return out
