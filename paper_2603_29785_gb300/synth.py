"""Seeded synthetic strain for tests and benchmarks.

Gravitational-wave-shaped inputs with the shapes of the paper's workloads:
whitened Gaussian noise, sine-Gaussian glitches and Newtonian chirps.  This
module holds no Q-transform arithmetic: it only makes input segments, which
both the CUDA path and the CPU oracle then read.  Every generator draws from
``numpy.random.Generator(PCG64(seed))`` and returns float32, the storage type
of the library's input; the oracle reads the same float32 values as float64.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def white(seed: int, n: int, sigma: float = 1.0) -> np.ndarray:
    """Unit-variance white Gaussian noise (float64 before the final cast)."""
    return sigma * rng(seed).standard_normal(int(n))


def sine_gaussian(n: int, fs: float, f0: float, q: float, amp: float, t0: float) -> np.ndarray:
    """amp * exp(-(t-t0)^2 / tau^2) * sin(2 pi f0 (t - t0)), tau = q / (sqrt(2) pi f0)."""
    t = np.arange(int(n)) / fs
    tau = q / (math.sqrt(2.0) * math.pi * f0)
    return amp * np.exp(-((t - t0) / tau) ** 2) * np.sin(2 * math.pi * f0 * (t - t0))


def tukey(n: int, alpha: float) -> np.ndarray:
    """Tukey (tapered cosine) window of length n with taper fraction alpha."""
    if n <= 1 or alpha <= 0:
        return np.ones(max(n, 0))
    x = np.arange(n) / (n - 1)
    w = np.ones(n)
    a2 = alpha / 2
    lo = x < a2
    hi = x > 1 - a2
    w[lo] = 0.5 * (1 + np.cos(math.pi * (x[lo] / a2 - 1)))
    w[hi] = 0.5 * (1 + np.cos(math.pi * ((x[hi] - 1) / a2 + 1)))
    return w


def newtonian_chirp(n: int, fs: float, f_lo: float, f_hi: float, t_c: float, duration: float) -> np.ndarray:
    """Unit-amplitude-scale Newtonian chirp, f(t) = f_lo ((t_c - t)/(t_c - t_s))^(-3/8).

    Starts at t_s = t_c - duration with f_lo, stops where f reaches f_hi;
    amplitude grows as f^(2/3); both ends Tukey-tapered.
    """
    t = np.arange(int(n)) / fs
    t_s = t_c - duration
    tau0 = duration
    t_end = t_c - tau0 * (f_hi / f_lo) ** (-8.0 / 3.0)
    on = (t >= t_s) & (t < t_end)
    tau = np.where(on, t_c - t, tau0)
    f = f_lo * (tau / tau0) ** (-3.0 / 8.0)
    # phase = 2 pi * integral f dt = -2 pi f_lo tau0^(3/8) (8/5) tau^(5/8) + const
    phase = -2 * math.pi * f_lo * tau0 ** 0.375 * 1.6 * tau ** 0.625
    h = np.where(on, (f / f_lo) ** (2.0 / 3.0) * np.cos(phase), 0.0)
    idx = np.nonzero(on)[0]
    if idx.size:
        h[idx] *= tukey(idx.size, 0.1)
    return h


def psd_coloured(f: np.ndarray) -> np.ndarray:
    """Smooth one-sided PSD shape: f^-4 below 40 Hz (capped at 10 Hz), flat
    from 40 to 300 Hz, rising as f^2 above 300 Hz."""
    f = np.asarray(f, dtype=np.float64)
    s = np.ones_like(f)
    lo = f < 40
    s[lo] = (np.maximum(f[lo], 10.0) / 40.0) ** -4
    hi = f > 300
    s[hi] = (f[hi] / 300.0) ** 2
    return s


def whiten(strain: np.ndarray, fs: float, psd) -> np.ndarray:
    """Divide the spectrum by sqrt(PSD) (the analytic PSD the noise was coloured with)."""
    n = strain.size
    F = np.fft.rfft(strain)
    return np.fft.irfft(F / np.sqrt(psd(np.fft.rfftfreq(n, 1 / fs))), n=n)


def colour(white_noise: np.ndarray, fs: float, psd) -> np.ndarray:
    n = white_noise.size
    F = np.fft.rfft(white_noise)
    return np.fft.irfft(F * np.sqrt(psd(np.fft.rfftfreq(n, 1 / fs))), n=n)


def coloured_chirp_segment(seed: int, n: int = 262144, fs: float = 4096.0, snr: float = 20.0,
                           f_lo: float = 20.0, f_hi: float = 400.0, chirp_s: float = 8.0,
                           t_c: float | None = None) -> np.ndarray:
    """64 s-style segment: coloured Gaussian noise plus a Newtonian chirp, then
    whitened by the analytic PSD.  The chirp is scaled so that its whitened
    energy sqrt(sum h_w^2) equals ``snr`` against unit-variance white noise."""
    T = n / fs
    if t_c is None:
        t_c = T - 2.0
    noise = colour(white(seed, n), fs, psd_coloured)
    h = newtonian_chirp(n, fs, f_lo, f_hi, t_c, chirp_s)
    h_w = whiten(h, fs, psd_coloured)
    e = math.sqrt(float(np.sum(h_w ** 2)))
    a = snr / e if e > 0 else 0.0
    return whiten(noise + a * h, fs, psd_coloured).astype(np.float32)


def white_sine_gaussian_segment(seed: int, n: int = 16384, fs: float = 4096.0, f0: float = 150.0,
                                q: float = 9.0, amp: float = 5.0, t0: float = 2.0) -> np.ndarray:
    """4 s-style segment: white N(0,1) noise plus one sine-Gaussian."""
    return (white(seed, n) + sine_gaussian(n, fs, f0, q, amp, t0)).astype(np.float32)


def glitchy_segment(seed: int, n: int, fs: float, rate_hz: float = 0.25, chirp: bool = False,
                    snr_range=(8.0, 50.0), f0_range=(30.0, 1500.0), q_range=(4.0, 40.0)) -> np.ndarray:
    """Whitened Gaussian noise with Poisson sine-Gaussian glitches (f0 log-uniform,
    Q uniform, SNR uniform) and optionally one chirp (SNR 20)."""
    g = rng(seed)
    T = n / fs
    x = g.standard_normal(n)
    for _ in range(int(g.poisson(rate_hz * T))):
        f0 = math.exp(g.uniform(math.log(f0_range[0]), math.log(min(f0_range[1], 0.45 * fs))))
        q = g.uniform(*q_range)
        t0 = g.uniform(0, T)
        s = sine_gaussian(n, fs, f0, q, 1.0, t0)
        e = math.sqrt(float(np.sum(s ** 2)))
        if e > 0:
            x += g.uniform(*snr_range) * s / e
    if chirp:
        dur = min(8.0, 0.75 * T)
        h = newtonian_chirp(n, fs, 20.0, min(400.0, 0.45 * fs), T * 0.9, dur)
        e = math.sqrt(float(np.sum(h ** 2)))
        if e > 0:
            x += 20.0 * h / e
    return x.astype(np.float32)


def batch(fn, seeds, **kw) -> np.ndarray:
    """Stack one segment per seed into a [B, N] float32 array."""
    return np.stack([fn(int(s), **kw) for s in seeds]) if len(seeds) else np.zeros((0, kw.get("n", 0)), np.float32)
