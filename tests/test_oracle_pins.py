"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a naive definition, a closed form, an
identity the paper proves (App. C), a worked number the paper prints
(tests/golden/paper_shapes.json) or a hand derivation from its formulas
(tests/golden/geometry_hand.json).  None of them re-calls the oracle to make
its own expected value.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import synth


def naive_dft(x, sign=-1):
    """Textbook O(N^2) DFT, X[f] = sum_n x[n] exp(sign 2 pi i f n / N)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    idx = np.arange(n)
    E = np.exp(sign * 2j * np.pi * np.outer(idx, idx) / n)
    return E @ x


def small_geom(N=512, fs=64.0, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, **kw):
    return O.geometry(fs, N, qs, fmin, fmax, K, **kw)


# --------------------------------------------------------------------------- P1
@pytest.mark.parametrize("N", [2, 4, 6, 8, 10, 12, 16, 18, 20, 30, 32, 48, 50, 64, 90, 96, 14, 22, 26, 34])
def test_spectrum_is_naive_dft(N):
    x = synth.white(N, N).astype(np.float32).astype(np.float64)
    X = O.spectrum(x)
    ref = naive_dft(x)[: N // 2 + 1]
    assert X.shape == (N // 2 + 1,)
    assert np.max(np.abs(X - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref))) * N


@pytest.mark.parametrize("M", [3, 5, 8, 15, 16, 25, 48, 75, 100])
def test_short_transforms_are_naive(M):
    z = synth.white(1, M) + 1j * synth.white(2, M)
    assert np.allclose(np.fft.ifft(z) * M, naive_dft(z, +1), atol=1e-12)
    assert np.allclose(np.fft.fft(z), naive_dft(z, -1), atol=1e-12)


@pytest.mark.parametrize("N", [4, 8, 14, 32, 64])
def test_real_ifft_matches_hermitian_formula(N):
    rng = synth.rng(N)
    Xh = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
    n = np.arange(N)
    ref = np.full(N, Xh[0].real) + Xh[N // 2].real * (-1.0) ** n
    for f in range(1, N // 2):
        ref += 2 * np.real(Xh[f] * np.exp(2j * np.pi * f * n / N))
    ref /= N
    assert np.allclose(O.real_ifft(Xh, N), ref, atol=1e-13)


# --------------------------------------------------------------------------- geometry
def test_paper_shapes(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_shapes.json")))
    for e in g["one_sided_lengths"]:
        assert O.spectrum(np.zeros(e["N"])).size == e["bins"]
    # App. A clamp: L_max = 2 floor(ceil(N_t df)/2) + 1 equals the printed
    # minimal length n = ceil(N_t df) + 1 whenever ceil(N_t df) is even.
    for e, df in zip(g["minimal_lengths"], (111.25, 157.5)):
        T = e["duration_s"]
        N = int(round(T * 4096)) & ~1
        geo = O.geometry(4096.0, N, (1.0,), 20.0, 2048.0, 16, max_window_hz=df)
        assert int(np.max(geo.L)) == e["n_min"]


def test_geometry_hand_derivations(golden_dir):
    cases = json.load(open(os.path.join(golden_dir, "geometry_hand.json")))["cases"]
    c1, c2 = cases
    g = O.geometry(c1["fs"], c1["N"], c1["qs"], c1["fmin"], c1["fmax"], c1["K"])
    assert g.h_max == c1["h_max"] and int(g.L.max()) == c1["max_L"] and g.M == c1["M"]
    for k, v in c1["kc"].items():
        assert g.kc[0, int(k)] == v
    for k, v in c1["h"].items():
        assert g.h[0, int(k)] == v
    Pf = O.frame_operator(g)
    zero = np.nonzero(Pf == 0)[0]
    assert zero.size == c1["n_zero_bins"]
    for b in c1["zero_coverage_bins"]:
        assert Pf[b] == 0 and Pf[b - 1] > 0 and Pf[b + 1] > 0
    assert np.all(Pf[: c1["zero_coverage_below"] + 1] == 0) and Pf[c1["zero_coverage_below"] + 1] > 0
    assert np.all(Pf[c1["zero_coverage_from"]:] == 0) and Pf[c1["zero_coverage_from"] - 1] > 0

    g = O.geometry(c2["fs"], c2["N"], c2["qs"], c2["fmin"], c2["fmax"], c2["K"])
    assert g.h_max == c2["h_max"] and int(g.L.max()) == c2["max_L"] and g.M == c2["M"]
    assert g.kc[0, -1] == c2["kc_top"] == g.N // 2
    assert g.h[0, 0] == c2["row0_q4_h"]


def test_smooth_length_brute_force():
    def smooth(m):
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        return m == 1
    for n in range(1, 5000, 7):
        m = O.smooth_length(n)
        assert m >= n and smooth(m) and not any(smooth(j) for j in range(n, m))


def test_bisquare_shape_and_moments():
    for h in (1, 2, 7, 33, 1061):
        d = np.arange(-h - 3, h + 4)
        w = O.bisquare_profile(d, h)
        assert w[d == 0][0] == 1.0
        assert np.all(w[np.abs(d) >= h] == 0)
        assert np.allclose(w, w[::-1])
        # (1 - u^2)^2 sampled exactly at u = 1/2
        if h % 2 == 0:
            assert w[d == h // 2][0] == pytest.approx(0.5625, abs=1e-15)
    # sum of W'^2 -> h * int_{-1}^{1} (1-u^2)^4 du = h * 256/315;
    # rms half-width of W'^2 -> h / sqrt(11) (reading C2)
    h = 20000
    d = np.arange(-h, h + 1)
    w2 = O.bisquare_profile(d, h) ** 2
    assert np.sum(w2) / h == pytest.approx(256 / 315, rel=1e-4)
    assert math.sqrt(np.sum(d ** 2 * w2) / np.sum(w2)) / h == pytest.approx(1 / math.sqrt(11), rel=1e-4)


def test_window_norms():
    g = small_geom(norm="l2")
    for p in range(g.P):
        for k in range(g.K):
            hk = int(g.h[p, k])
            w = g.c[p, k] * O.bisquare_profile(np.arange(-hk, hk + 1), hk)
            assert np.sum(w ** 2) == pytest.approx(1.0, rel=1e-13)
    gp = small_geom(norm="paper")
    for p in range(gp.P):
        for k in range(gp.K):
            hk = int(gp.h[p, k])
            s = np.sum(O.bisquare_profile(np.arange(-hk, hk + 1), hk) ** 2)
            assert gp.c[p, k] * s == pytest.approx(1.0, rel=1e-13)
    assert np.all(small_geom(norm="none").c == 1.0)


def test_grid_and_widths_follow_formulas():
    g = small_geom()
    T = g.N / g.fs
    r = (g.fmax / g.fmin) ** (1 / (g.K - 1))
    for k in range(g.K):
        assert g.f[0, k] == pytest.approx(g.fmin * r ** k, rel=1e-14)
    assert g.f[0, 0] == pytest.approx(g.fmin) and g.f[0, -1] == pytest.approx(g.fmax)
    gap = g.fmax - g.fmax / r
    assert g.h_max == math.ceil(T * gap) // 2
    for p, q in enumerate(g.qs):
        for k in range(g.K):
            assert g.h[p, k] == max(1, min(int(g.f[p, k] * T * math.sqrt(11) / q), g.h_max))
            assert abs(g.kc[p, k] - g.f[p, k] * T) <= 0.5


# --------------------------------------------------------------------------- identities (App. C)
def _rand_x(N, seed=0):
    return synth.white(seed, N)


def test_dense_tile_relation_bruteforce_time_domain():
    """P6: with M | N, Y_k[n] = sqrt(N/M) exp(-2 pi i k_c n / M) T_k[n N / M],
    T_k the dense tile computed here by brute-force circular convolution of x
    with the row's complex atom (Eq. gwpy_convolution_prd)."""
    N, fs = 64, 64.0
    g = O.geometry(fs, N, (2.0, 5.0), 3.0, 24.0, 5, n_out=16)
    assert N % g.M == 0
    x = _rand_x(N, 3)
    Y = O.forward(g, x)
    n = np.arange(N)
    for p in range(g.P):
        for k in range(g.K):
            # atom g_k[m] = (1/N) sum_f W_k[f] exp(+2 pi i f m / N), one-sided W
            W = np.zeros(N)
            hk = int(g.h[p, k])
            for f in range(N // 2 + 1):
                d = f - int(g.kc[p, k])
                if abs(d) <= hk:
                    W[f] = g.c[p, k] * (1 - (d / hk) ** 2) ** 2
            atom = np.array([np.sum(W * np.exp(2j * np.pi * np.arange(N) * m / N)) for m in n]) / N
            Tk = np.array([np.sum(x * atom[(tau - n) % N]) for tau in n])
            step = N // g.M
            for j in range(g.M):
                ref = math.sqrt(N / g.M) * np.exp(-2j * np.pi * g.kc[p, k] * j / g.M) * Tk[j * step]
                assert abs(Y[p, k, j] - ref) <= 1e-12 * (1 + abs(ref))


def test_round_trip_fp64_is_projection():
    """P2: x_hat = x_proj (App. C exact reconstruction where P > 0)."""
    for g, seed in ((small_geom(), 1), (O.geometry(4096, 16384, (8,), 20, 1024, 64), 2)):
        x = _rand_x(g.N, seed)
        xh = O.inverse(g, O.forward(g, x))
        xp = O.projection(g, x)
        assert np.linalg.norm(xh - xp) / np.linalg.norm(xp) < 1e-12
        # a signal already inside F_0 comes back exactly
        xh2 = O.inverse(g, O.forward(g, xp))
        assert np.linalg.norm(xh2 - xp) / np.linalg.norm(xp) < 1e-12


def test_round_trip_fp64_config1_signal():
    g = O.geometry(4096, 16384, (8,), 20, 1024, 64)
    x = synth.white_sine_gaussian_segment(0).astype(np.float64)
    xp = O.projection(g, x)
    xh = O.inverse(g, O.forward(g, x))
    assert np.linalg.norm(xh - xp) / np.linalg.norm(xp) < 1e-12
    # the sine-Gaussian at 150 Hz lies inside the covered band: its energy survives
    sg = synth.sine_gaussian(g.N, g.fs, 150.0, 9.0, 5.0, 2.0)
    sgp = O.projection(g, sg)
    assert np.linalg.norm(sgp - sg) / np.linalg.norm(sg) < 1e-6


def test_linearity():
    """P3: T(a x1 + b x2) = a T(x1) + b T(x2) (Sec. III)."""
    g = small_geom()
    x1, x2 = _rand_x(g.N, 4), _rand_x(g.N, 5)
    a, b = 0.75, -2.5
    lhs = O.forward(g, a * x1 + b * x2)
    rhs = a * O.forward(g, x1) + b * O.forward(g, x2)
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * 10 * np.max(np.abs(lhs))


def test_parseval_per_row_and_frame_energy():
    """P5: sum_n |Y_k|^2 = (1/N) sum_f |W_k X|^2 (App. C, energy preservation),
    and summed over rows (1/N) sum_f P[f] |X[f]|^2 (frame operator S = T*T)."""
    g = small_geom()
    x = _rand_x(g.N, 6)
    X = np.fft.rfft(x)
    Y = O.forward(g, x)
    for p in range(g.P):
        for k in range(g.K):
            e_row = np.sum(np.abs(Y[p, k]) ** 2)
            e_ref = np.sum(np.abs(O.window(g, p, k) * X) ** 2) / g.N
            assert e_row == pytest.approx(e_ref, rel=1e-12)
    Pf = O.frame_operator(g)
    assert np.sum(np.abs(Y) ** 2) == pytest.approx(np.sum(Pf * np.abs(X) ** 2) / g.N, rel=1e-12)
    # frame bounds on the kept set
    keep = O.kept_bins(Pf, 0.0)
    Xk = np.where(keep, X, 0)
    e = np.sum(np.abs(O.forward(g, O.real_ifft(Xk, g.N))) ** 2)
    e_x = np.sum(np.abs(Xk) ** 2) / g.N
    assert Pf[keep].min() * e_x * (1 - 1e-12) <= e <= Pf[keep].max() * e_x * (1 + 1e-12)


def test_adjoint_dot_product():
    """<T x, y> = <x, T* y> with T* the synthesis without the 1/P division:
    T* y = irfft(omega A), omega = 1 at DC and Nyquist, 1/2 elsewhere (the
    one-sided storage of a real signal's spectrum)."""
    g = small_geom()
    x = _rand_x(g.N, 7)
    rng = synth.rng(8)
    y = rng.standard_normal((g.P, g.K, g.M)) + 1j * rng.standard_normal((g.P, g.K, g.M))
    lhs = np.real(np.sum(np.conj(O.forward(g, x)) * y))
    A = O.accumulate(g, y)
    omega = np.full(g.Nr, 0.5)
    omega[0] = omega[-1] = 1.0
    Ts_y = O.real_ifft(omega * A, g.N)
    rhs = float(np.dot(x, Ts_y))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_shift_invariance_one_decimation_step():
    """P7: shifting x by N/M samples moves every envelope by one column with
    the carrier phase exp(-2 pi i k_c / M) (Sec. III, AM demodulation)."""
    N = 512
    g = O.geometry(64.0, N, (4.0, 8.0), 3.0, 30.0, 12, n_out=64)
    assert N % g.M == 0
    s = N // g.M
    x = _rand_x(N, 9)
    Y = O.forward(g, x)
    Ys = O.forward(g, np.roll(x, s))
    ph = np.exp(-2j * np.pi * g.kc / g.M)[..., None]
    assert np.max(np.abs(Ys - ph * np.roll(Y, 1, axis=-1))) <= 1e-12 * np.max(np.abs(Y))


def test_shift_invariance_general_shift():
    g = small_geom()
    x = _rand_x(g.N, 10)
    s = 37
    Ys = O.forward(g, np.roll(x, s))
    # multiply each band bin by exp(-2 pi i (k_c + d) s / N) and re-synthesise the envelope
    X = np.fft.rfft(x) * np.exp(-2j * np.pi * np.arange(g.Nr) * s / g.N)
    for p in range(g.P):
        for k in range(g.K):
            assert np.allclose(O.forward_row(g, X, p, k), Ys[p, k], atol=1e-12)


def test_tone_peaks_on_its_row():
    """P4: a cosine on row k's centre bin has ||Y_j|| proportional to W_j[k_c]
    (closed form); under 'none' normalisation the own row (W' = 1) wins."""
    g = O.geometry(4096, 16384, (8,), 20, 1024, 64, norm="none")
    n = np.arange(g.N)
    for k in range(0, g.K, 5):
        b = int(g.kc[0, k])
        x = np.cos(2 * np.pi * b * n / g.N)
        E = np.sum(np.abs(O.forward(g, x)[0]) ** 2, axis=-1)
        assert int(np.argmax(E)) == k
        # closed form |X[b]| = N/2 -> sum_n |Y_j|^2 = W_j[b]^2 N / 4
        assert E[k] == pytest.approx(g.N / 4, rel=1e-12)
    gl = O.geometry(4096, 16384, (8,), 20, 1024, 64, norm="l2")
    for k in range(0, gl.K, 7):
        b = int(gl.kc[0, k])
        E = np.sum(np.abs(O.forward(gl, np.cos(2 * np.pi * b * n / gl.N))[0]) ** 2, axis=-1)
        assert int(np.argmax(E)) == k


def test_masked_inverse_drops_rows_keeps_normaliser():
    """P8: inverting row-zeroed envelopes equals A/P with those rows left out
    of A only; a single-plane mask uses that plane's P (reading C9)."""
    g = small_geom()
    x = _rand_x(g.N, 11)
    Y = O.forward(g, x)
    Ym = Y.copy()
    Ym[0, 2:5] = 0
    Ym[1, 7] = 0
    xm = O.inverse(g, Ym)
    # by linearity: contributions of the zeroed rows, divided by the full P
    Yz = np.zeros_like(Y)
    Yz[0, 2:5] = Y[0, 2:5]
    Yz[1, 7] = Y[1, 7]
    Az = O.accumulate(g, Yz)
    Pf = O.frame_operator(g)
    keep = O.kept_bins(Pf, 0.0)
    missing = O.real_ifft(np.where(keep, Az / np.where(keep, Pf, 1), 0), g.N)
    assert np.allclose(xm, O.inverse(g, Y) - missing, atol=1e-12)
    # one plane alone is a valid dual on its own coverage
    x1 = O.inverse(g, Y, planes=[1])
    assert np.linalg.norm(x1 - O.projection(g, x, planes=[1])) < 1e-11 * np.linalg.norm(x)


def test_floor_tau_projection():
    g = small_geom()
    x = _rand_x(g.N, 12)
    for tau in (1e-6, 1e-3, 0.1):
        xh = O.inverse(g, O.forward(g, x), tau=tau)
        xp = O.projection(g, x, tau=tau)
        assert np.linalg.norm(xh - xp) <= 1e-12 * np.linalg.norm(x)
    Pf = O.frame_operator(g)
    assert O.kept_bins(Pf, 0.1).sum() < O.kept_bins(Pf, 0.0).sum()


def test_windows_truncated_at_band_edges():
    """Reading C6: bins outside 0..N/2 are dropped, c_k stays that of the full window."""
    g = O.geometry(64.0, 256, (1.0,), 1.0, 32.0, 6)
    assert g.kc[0, -1] == g.N // 2 and g.kc[0, 0] - g.h[0, 0] < 0
    for k in (0, g.K - 1):
        d, fb = O.band(g, 0, k)
        assert fb.min() >= 0 and fb.max() <= g.N // 2
        assert d.size < g.L[0, k]


# --------------------------------------------------------------------------- optimal-plane selection
def test_plane_energy_is_per_plane_frame_identity():
    """Energy of plane p = (1/N) sum_f P_p[f] |X[f]|^2 (App. C frame operator of
    that plane alone), which the metric must reproduce."""
    g = small_geom()
    x = _rand_x(g.N, 21)
    X = np.fft.rfft(x)
    e, pk, best_e, best_p = O.plane_metrics(O.forward(g, x))
    for p in range(g.P):
        ref = np.sum(O.frame_operator(g, planes=[p]) * np.abs(X) ** 2) / g.N
        assert e[p] == pytest.approx(ref, rel=1e-12)
    assert best_e == int(np.argmax(e)) and best_p == int(np.argmax(pk))


def test_plane_peak_of_a_tone_closed_form():
    """A cosine on row k's centre bin gives |Y_k[n]|^2 = W_k[b]^2 N / (4 M) on every
    column (one spectral line, shifted to DC): the peak of each plane is that value
    on its strongest row."""
    g = O.geometry(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, norm="none")
    b = int(g.kc[0, 5])
    x = np.cos(2 * np.pi * b * np.arange(g.N) / g.N)
    e, pk, _, _ = O.plane_metrics(O.forward(g, x))
    for p in range(g.P):
        wmax = max(O.window(g, p, k)[b] for k in range(g.K))
        assert pk[p] == pytest.approx(wmax ** 2 * g.N / (4 * g.M), rel=1e-12)


# --------------------------------------------------------------------------- window family (App. A)
def test_window_family_special_cases_and_moments():
    """Closed forms: Tukey a=1 is Hann, Tukey a=0 and Kaiser beta=0 are the
    rectangle, sum of Hann^2 -> 3h/4 (int_{-1}^{1} cos^4(pi u/2) du = 3/4),
    Planck-taper is continuous (plateau 1, -> 0 at the edge, monotone in between)."""
    h = 4000
    d = np.arange(-h, h + 1)
    hann = O.window_profile(d, h, "hann")
    assert np.allclose(O.window_profile(d, h, "tukey", 1.0), hann, atol=1e-15)
    assert np.all(O.window_profile(d, h, "tukey", 0.0) == 1.0)
    assert np.allclose(O.window_profile(d, h, "kaiser", 0.0), 1.0, atol=1e-15)
    assert np.sum(hann ** 2) / h == pytest.approx(0.75, rel=1e-3)
    assert hann[h] == 1.0 and hann[0] == pytest.approx(0.0, abs=1e-15)
    k = O.window_profile(d, h, "kaiser", 8.0)
    assert k[h] == pytest.approx(1.0) and k[0] == pytest.approx(1.0 / np.i0(8.0))
    pl = O.window_profile(d, h, "planck", 0.25)
    half = pl[h:]                      # d = 0 .. h
    assert np.all(half[: int(0.75 * h)] == 1.0) and half[-1] == 0.0
    assert np.all(np.diff(half) <= 1e-15)                     # non-increasing away from the centre
    assert np.max(np.abs(np.diff(half))) < 0.01               # continuous: no jump at the plateau edge
    # the taper is symmetric about its midpoint: w(t) + w(a - t) = 1, t = 1 - |u|
    t = 0.1
    u1, u2 = 1 - t, 1 - (0.25 - t)
    w1 = O.window_profile(np.array([int(round(u1 * h))]), h, "planck", 0.25)[0]
    w2 = O.window_profile(np.array([int(round(u2 * h))]), h, "planck", 0.25)[0]
    assert w1 + w2 == pytest.approx(1.0, abs=2e-3)


def test_kaiser_window_integral_closed_form():
    """Kaiser window (App. A): int_{-1}^{1} I0(beta sqrt(1 - u^2)) du = 2 sinh(beta) / beta,
    so the trapezoid sum of W'(d) = I0(beta sqrt(1 - (d/h)^2)) / I0(beta) over
    |d| <= h, divided by h, tends to 2 sinh(beta) / (beta I0(beta)) with an
    O(1/h^2) error.  Fixes the interior shape, not only the end points (an
    argument beta (1 - u^2) misses it by 9-25 %)."""
    h = 4000
    d = np.arange(-h, h + 1)
    for beta in (2.0, 6.0, 8.0):
        w = O.window_profile(d, h, "kaiser", beta)
        trap = (np.sum(w) - 0.5 * (w[0] + w[-1])) / h
        closed = 2.0 * math.sinh(beta) / (beta * float(np.i0(beta)))
        assert trap == pytest.approx(closed, rel=1e-7), beta


def test_kappa_hand_case():
    """kappa = max over kept bins of (max_k W_k) / P.  Two rows far apart, both
    clamped to h = 3 (T = 1 s, manual clamp 7 Hz: h_max = floor(ceil(7) / 2)):
    each kept bin sees one window, P = W^2 there, so kappa = 1 / min W over the
    kept bins = 1 / (c W'(2)) with W'(2) = ((9 - 4) / 9)^2 = 25/81 (W'(3) = 0 is
    not kept) and c = (sum W'^2)^(-1/2) = (6561 / 16003)^(1/2): kappa = sqrt(16003) / 25."""
    g = O.geometry(4096.0, 4096, (8.0,), 100.0, 1000.0, 2, max_window_hz=7.0)
    assert list(g.h.ravel()) == [3, 3] and list(g.kc.ravel()) == [100, 1000]
    assert O.kappa(g) == pytest.approx(math.sqrt(16003.0) / 25.0, rel=1e-13)


@pytest.mark.parametrize("window,param", [("hann", 0.0), ("kaiser", 6.0), ("tukey", 0.5), ("planck", 0.3)])
def test_window_family_frame_identities(window, param):
    """App. C holds for any window: round trip = projection, frame energy identity."""
    g = small_geom(window=window, window_param=param)
    x = _rand_x(g.N, 31)
    Y = O.forward(g, x)
    assert np.linalg.norm(O.inverse(g, Y) - O.projection(g, x)) < 1e-12 * np.linalg.norm(x)
    X = np.fft.rfft(x)
    assert np.sum(np.abs(Y) ** 2) == pytest.approx(np.sum(O.frame_operator(g) * np.abs(X) ** 2) / g.N, rel=1e-12)
    for p in range(g.P):
        for k in range(g.K):
            hk = int(g.h[p, k])
            w = g.c[p, k] * O.window_profile(np.arange(-hk, hk + 1), hk, window, param)
            assert np.sum(w ** 2) == pytest.approx(1.0, rel=1e-12)


def test_composite_bank_planes_are_single_window_transforms():
    """A plane of the composite bank (App. A: Q x window x parameter) is the
    one-plane transform with that plane's configuration; the bank's frame
    operator is the sum of its planes' operators, and the bank inverts to the
    projection onto its kept bins."""
    qs = (4.0, 4.0, 8.0, 8.0)
    wins = ("bisquare", "tukey", "kaiser", "planck")
    prms = (0.0, 0.5, 6.0, 0.3)
    g = O.geometry(64.0, 512, qs, 3.0, 30.0, 12, window=wins, window_param=prms)
    x = _rand_x(g.N, 44)
    Y = O.forward(g, x)
    Pf = np.zeros(g.Nr)
    for p in range(g.P):
        g1 = O.geometry(64.0, 512, (qs[p],), 3.0, 30.0, 12, window=wins[p], window_param=prms[p], n_out=g.M)
        assert g.plane_window(p) == (wins[p], prms[p])
        assert np.array_equal(g1.h[0], g.h[p]) and np.allclose(g1.c[0], g.c[p], rtol=1e-15)
        assert np.allclose(O.forward(g1, x)[0], Y[p], rtol=0, atol=1e-14 * np.max(np.abs(Y)))
        Pf += O.frame_operator(g1)
    assert np.allclose(O.frame_operator(g), Pf, rtol=1e-14, atol=0)
    assert np.linalg.norm(O.inverse(g, Y) - O.projection(g, x)) < 1e-12 * np.linalg.norm(x)
    # the same name on every plane equals the single-window geometry
    gs = O.geometry(64.0, 512, qs, 3.0, 30.0, 12, window="hann")
    gb = O.geometry(64.0, 512, qs, 3.0, 30.0, 12, window=("hann",) * 4, window_param=(0.0,) * 4)
    assert np.array_equal(gs.c, gb.c) and np.allclose(O.forward(gs, x), O.forward(gb, x), rtol=0, atol=0)
    with pytest.raises(ValueError):
        O.geometry(64.0, 512, qs, 3.0, 30.0, 12, window=("hann", "tukey"))


# --------------------------------------------------------------------------- streaming (reading S1)
def _stream_geom(remodulate=False):
    # N = 1024 at 256 Hz, M = 96 (gcd 32 -> quantum 32 samples = 3 columns)
    return O.geometry(256.0, 1024, (6.0, 12.0), 2.0, 100.0, 20, n_out=96, remodulate=remodulate)


def test_stream_layout_rules():
    g = _stream_geom()
    assert O.stream_quantum(g) == 32
    assert O.stream_layout(g, 512) == (256, 48, 24)
    assert O.stream_layout(g, 1024) == (0, 96, 0)
    for bad in (0, 500, 2048, 544):        # not a quantum multiple / too long / odd guard count
        with pytest.raises(ValueError):
            O.stream_layout(g, bad)


@pytest.mark.parametrize("remodulate", [False, True])
def test_stream_of_a_periodic_signal_tiles_the_circular_transform(remodulate):
    """A stream repeating one segment x0 is, away from the zero prefix, the
    segment's circular transform tiled with the guard offset: map column c equals
    Y0 column (c - Gm) mod M, and the streaming inverse returns the projection
    of x0 delayed by 2G (shift invariance in whole columns, App. C).  For
    remodulated tiles the same holds with no re-reference phase, since their
    carrier already refers each column to absolute time."""
    g = _stream_geom(remodulate)
    hop = 512
    G, Hn, Gm = O.stream_layout(g, hop)
    x0 = _rand_x(g.N, 51)
    reps = 6
    x = np.tile(x0, reps)
    Ymap = O.stream_forward(g, x, hop)
    Y0 = O.forward(g, x0)
    c0 = 2 * Hn                                   # chunks 0, 1 see the zero prefix
    cols = np.arange(c0, Ymap.shape[2])
    assert np.allclose(Ymap[:, :, cols], Y0[:, :, (cols - Gm) % g.M], rtol=0, atol=1e-12 * np.max(np.abs(Y0)))
    xh = O.stream_inverse(g, Ymap, hop)
    s0 = (2 + 2 * Gm // Hn + 2) * hop             # chunks whose envelopes come from clean map columns
    s = np.arange(s0, xh.size)
    xp0 = O.projection(g, x0)
    assert np.allclose(xh[s], xp0[(s - 2 * G) % g.N], rtol=0, atol=1e-12 * np.max(np.abs(xp0)))


def test_stream_without_guard_is_chunkwise():
    g = _stream_geom()
    x = _rand_x(3 * g.N, 52)
    Ymap = O.stream_forward(g, x, g.N)
    for i in range(3):
        Yi = O.forward(g, x[i * g.N:(i + 1) * g.N])
        assert np.array_equal(Ymap[:, :, i * g.M:(i + 1) * g.M], Yi)
        assert np.allclose(O.stream_inverse(g, Ymap, g.N)[i * g.N:(i + 1) * g.N], O.inverse(g, Yi), rtol=0,
                           atol=1e-13 * np.max(np.abs(x)))


# --------------------------------------------------------------------------- dense mode (reading D1)
def _dense_geom(eps=1e-6, remodulate=False, **kw):
    # N = 512: N/2 + 1 = 257 bins, M = 270 (smallest 2^a 3^b 5^c >= 257)
    return O.geometry(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, stopband_eps=eps, remodulate=remodulate, **kw)


def test_dense_geometry_spans_the_spectrum():
    g = _dense_geom()
    assert g.M == 270 and g.M >= g.Nr
    d, fb = O.band(g, 0, 3)
    assert np.array_equal(fb, np.arange(g.Nr))
    w = O.row_weight(g, 0, 3, d)
    hk = int(g.h[0, 3])
    assert np.all(w[np.abs(d) >= hk] == g.c[0, 3] * 1e-6) and np.all(w > 0)     # edge points too
    assert np.allclose(w[np.abs(d) < hk], g.c[0, 3] * O.bisquare_profile(d[np.abs(d) < hk], hk), rtol=1e-15)
    assert np.array_equal(g.c, O.geometry(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, n_out=270).c)
    with pytest.raises(ValueError):
        O.geometry(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, stopband_eps=1e-6, n_out=256)


@pytest.mark.parametrize("remodulate", [False, True])
def test_single_tile_inverse_recovers_the_signal(remodulate):
    """With a non-zero stopband every tile is element-wise invertible: each
    single tile gives back x (the equation after Eq. qtam_window_formula)."""
    g = _dense_geom(remodulate=remodulate)
    x = _rand_x(g.N, 61)
    Y = O.forward(g, x)
    for p, k in ((0, 0), (0, 6), (1, 11), (1, 4)):
        assert np.linalg.norm(O.inverse_single_tile(g, Y, p, k) - x) < 1e-8 * np.linalg.norm(x)
    # the frame inverse is exact too (P > 0 on every bin); bins that only the
    # floor covers have P ~ (c eps)^2, which lifts FP64 rounding by ~1/eps
    assert np.linalg.norm(O.inverse(g, Y) - x) < 1e-9 * np.linalg.norm(x)
    with pytest.raises(ValueError):
        O.inverse_single_tile(small_geom(), O.forward(small_geom(), x), 0, 0)


def test_remodulated_tile_is_the_unshifted_filtered_spectrum():
    """T_k = Y_k exp(+2 pi i k_c n / M) is sqrt(M/N) IDFT_M of X W_k placed at
    the absolute bins f (no roll): the undemodulated tile."""
    g = _dense_geom(remodulate=True)
    x = _rand_x(g.N, 62)
    X = np.fft.rfft(x)
    Y = O.forward(g, x)
    for p, k in ((0, 2), (1, 9)):
        V = np.zeros(g.M, dtype=np.complex128)
        V[:g.Nr] = O.window(g, p, k) * X
        assert np.allclose(np.fft.fft(Y[p, k]) / np.sqrt(g.M / g.N), V, rtol=0, atol=1e-12 * np.max(np.abs(V)))


def test_small_stopband_barely_changes_the_tile():
    """eps of the order of the working precision leaves the forward transform
    as it was (Sec. III: negligible impact): the change is bounded by eps."""
    g0 = O.geometry(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, n_out=270)
    g1 = _dense_geom(eps=1e-9)
    x = _rand_x(g0.N, 63)
    Y0, Y1 = O.forward(g0, x), O.forward(g1, x)
    assert np.linalg.norm(Y1 - Y0) <= 1e-9 * np.max(g1.c) * np.linalg.norm(np.fft.rfft(x)) * np.sqrt(g1.P * g1.K)
    assert np.linalg.norm(Y1 - Y0) > 0


def test_all_ones_window_tile_is_the_analytic_signal():
    """Textbook special case: one row whose window is 1 on every bin (a
    rectangle, Tukey a = 0, with floor eps = 1 outside), c = 1, the carrier
    restored, M = N.  The tile is (1/N) sum_{f=0}^{N/2} X[f] e^{2 pi i f n / N},
    so 2 Re T[n] = x[n] + (X[0] + X[N/2] (-1)^n) / N -- checked against x."""
    N = 512
    g = O.geometry(64.0, N, (1.0,), 7.0, 7.0, 1, norm="none", window="tukey", window_param=0.0,
                   stopband_eps=1.0, remodulate=True, n_out=N)
    assert g.M == N and g.c[0, 0] == 1.0
    x = _rand_x(N, 71) + 0.3            # a DC offset so the correction term matters
    X = np.fft.rfft(x)
    T = O.forward(g, x)[0, 0]
    n = np.arange(N)
    expect = 0.5 * (x + (X[0].real + X[-1].real * (-1.0) ** n) / N)
    assert np.allclose(T.real, expect, rtol=0, atol=1e-13 * np.max(np.abs(x)))
