"""Dense mode (reading D1) through the C ABI against the FP64 oracle: tiles
spanning the one-sided spectrum with a stopband floor, the remodulated
(undemodulated) tile, and the single-tile inverse by spectral division.

Tolerances from the arithmetic: the forward is the ordinary FP32 path (1e-6
Frobenius, 1e-5 element-wise of the largest).  The single-tile inverse divides
the stopband bins by c eps, lifting the envelopes' rounding (u ~ 6e-8 in FP32,
1e-16 in FP64) by about sqrt(L/M)/eps: with eps = 1e-3 in FP32 that is a few
1e-6 relative, bound 1e-4; with eps = 1e-6 in FP64 a few 1e-11, bound 1e-8."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CFGS = [
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12),                 # M = 270
    dict(fs=4096.0, N=8192, qs=(4.0, 8.0, 16.0), fmin=20.0, fmax=2048.0, K=64),     # M = 4320
]


def _make(c, compute, eps, remod, window="bisquare", n_out=0, envelope=None):
    p = qtam.Plan(c["fs"], c["N"], c["qs"], c["fmin"], c["fmax"], c["K"], compute=compute, stopband_eps=eps,
                  remodulate=remod, window=window, n_out=n_out, envelope=envelope, device=0)
    g = O.geometry(c["fs"], c["N"], c["qs"], c["fmin"], c["fmax"], c["K"], stopband_eps=eps, remodulate=remod,
                   window=window, n_out=n_out)
    assert p.M == g.M and p.M >= g.Nr
    return p, g


@pytest.mark.parametrize("i", range(len(CFGS)))
@pytest.mark.parametrize("remod", [False, True])
@pytest.mark.parametrize("window", ["bisquare", "hann"])
def test_dense_forward_and_single_tile_fp32(i, remod, window):
    c = CFGS[i]
    p, g = _make(c, "f32", 1e-3, remod, window)
    B = 2
    gen = (lambda b: synth.white(300 + b, c["N"])) if c["fs"] < 1000 else \
        (lambda b: synth.glitchy_segment(300 + b, c["N"], c["fs"]))
    x = np.stack([gen(b) for b in range(B)]).astype(np.float32)
    y = p.forward(torch.from_numpy(x).cuda())
    Y = y.cpu().numpy().astype(np.complex128)
    for b in range(B):
        ref = O.forward(g, x[b].astype(np.float64))
        assert _rel(Y[b], ref) < 1e-6
        assert np.max(np.abs(Y[b] - ref)) <= 1e-5 * np.max(np.abs(ref))
    for pl, k in ((0, 0), (g.P - 1, g.K - 1), (1, g.K // 2)):
        xs = p.inverse_single_tile(y, pl, k).cpu().numpy().astype(np.float64)
        for b in range(B):
            xo = O.inverse_single_tile(g, Y[b], pl, k)        # the oracle's division of the GPU's own tile
            assert _rel(xs[b], xo) < 1e-4, (pl, k)
            assert _rel(xs[b], x[b].astype(np.float64)) < 1e-4, (pl, k)
    xh = p.inverse(y).cpu().numpy().astype(np.float64)
    for b in range(B):
        assert _rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < 1e-5


@pytest.mark.parametrize("eps,remod,window", [(1e-3, False, "bisquare"), (1e-3, True, "hann"),
                                              (0.0, True, "bisquare")])
def test_dense_compile_time_variants_match_oracle(eps, remod, window):
    """M = 4320 has compile-time variants with the dense kernels: each of them
    and the runtime engine against the oracle, forward and accumulated inverse
    (odd batch).  Floor alone: baseband tiles; floor and carrier: bins at
    their own positions; carrier alone: baseband tiles times the carrier."""
    c = CFGS[1]
    p, g = _make(c, "f32", eps, remod, window, n_out=4320)
    ids = qtam.qtam_plan_variants(p.handle)
    assert p.info["row_variant"] >= 0 and len(ids) == 4
    B = 3
    x = np.stack([synth.glitchy_segment(700 + b, c["N"], c["fs"], chirp=True) for b in range(B)]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    refs = [O.forward(g, xb.astype(np.float64)) for xb in x]
    projs = [O.projection(g, xb.astype(np.float64), tau=p.info["p_floor_rel"]) for xb in x]
    for v in ids:
        qtam.qtam_plan_set_variant(p.handle, v)
        y = p.forward(xd)
        Y = y.cpu().numpy().astype(np.complex128)
        xh = p.inverse(y).cpu().numpy().astype(np.float64)
        for b in range(B):
            assert _rel(Y[b], refs[b]) < 1e-6, v
            assert np.max(np.abs(Y[b] - refs[b])) <= 1e-5 * np.max(np.abs(refs[b])), v
            assert _rel(xh[b], projs[b]) < 1e-5, v


@pytest.mark.parametrize("env", ["bf16", "f16"])
def test_dense_16bit_envelopes_on_compile_time_variants(env):
    """Dense tiles (floor and carrier) stored as BF16 / FP16 by the dense
    variants, against the oracle at 16-bit storage accuracy: forward 1e-2
    (BF16 keeps 8 significand bits, u = 2e-3; FP16 11 bits), the canonical
    inverse of the stored tiles 2e-2 of the projection."""
    c = CFGS[1]
    p, g = _make(c, "f32", 1e-3, True, envelope=env)
    assert p.info["row_variant"] >= 0
    B = 2
    x = np.stack([synth.glitchy_segment(720 + b, c["N"], c["fs"], chirp=True) for b in range(B)]).astype(np.float32)
    y = p.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    a = y.float().cpu().numpy().astype(np.float64)
    Y = a[..., 0] + 1j * a[..., 1]
    xh = p.inverse(y).cpu().numpy().astype(np.float64)
    for b in range(B):
        ref = O.forward(g, x[b].astype(np.float64))
        assert _rel(Y[b], ref) < 1e-2
        assert _rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < 2e-2


@pytest.mark.parametrize("remod", [False, True])
def test_dense_single_tile_fp64(remod):
    c = CFGS[1]
    p, g = _make(c, "f64", 1e-6, remod)
    x = synth.white_sine_gaussian_segment(4)[: c["N"]].astype(np.float64)
    y = p.forward(torch.from_numpy(x[None]).cuda())
    Y = y.cpu().numpy()[0]
    assert _rel(Y, O.forward(g, x)) < 1e-13
    for pl, k in ((0, 3), (2, 40)):
        xs = p.inverse_single_tile(y, pl, k).cpu().numpy()[0]
        assert _rel(xs, x) < 1e-8
        assert _rel(xs, O.inverse_single_tile(g, Y, pl, k)) < 1e-8


def test_single_tile_needs_dense_mode():
    p = qtam.Plan(4096.0, 8192, (8.0,), 20.0, 2048.0, 32, device=0)
    y = p.envelope_tensor(1)
    with pytest.raises(qtam.QtamError):
        p.inverse_single_tile(y, 0, 0)
    q = qtam.Plan(4096.0, 8192, (8.0,), 20.0, 2048.0, 32, stopband_eps=1e-3, device=0)
    with pytest.raises(qtam.QtamError):
        q.inverse_single_tile(q.envelope_tensor(1), 0, 32)          # row out of range


def test_all_ones_window_tile_is_the_analytic_signal_gpu():
    """The oracle pin's special case on the GPU (runtime engine, dense mode)."""
    N = 512
    p = qtam.Plan(64.0, N, (1.0,), 7.0, 7.0, 1, norm="none", window="tukey", window_param=0.0, stopband_eps=1.0,
                  remodulate=True, n_out=N, device=0)
    x = (synth.white(72, N) + 0.3).astype(np.float32)
    T = p.forward(torch.from_numpy(x[None]).cuda()).cpu().numpy()[0, 0, 0].astype(np.complex128)
    xd = x.astype(np.float64)
    X = np.fft.rfft(xd)
    n = np.arange(N)
    expect = 0.5 * (xd + (X[0].real + X[-1].real * (-1.0) ** n) / N)
    assert np.max(np.abs(T.real - expect)) <= 1e-6 * np.max(np.abs(xd))
