"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances (FP32 compute), from the arithmetic: unit roundoff u = 6e-8; a
mixed-radix FFT of length m has rms relative error ~ u sqrt(log2 m), the long
FFT ~ u sqrt(log2 n), and the on-the-fly window ~ 3u, so the forward's
relative Frobenius error is ~ 4e-7: bound 1e-6.  Element-wise, every
coefficient must sit within 1e-5 of the segment's largest magnitude.  The
round trip is bounded by 1e-5 relative to the oracle's projection onto the
kept bins (the stated FP32 target).  FP64 compute: 1e-12 / 1e-13.
"""
import math

import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_FROB = {"f32": 1e-6, "f64": 1e-13}
FWD_ELEM = {"f32": 1e-5, "f64": 1e-12}
RT = {"f32": 1e-5, "f64": 1e-12}


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def env_np(p, y):
    if p.envelope in ("bf16", "f16"):
        y = host(y.float()).astype(np.float64)
        return y[..., 0] + 1j * y[..., 1]
    y = host(y)
    return y.astype(np.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def elem_ok(a, b, tol):
    return np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def geom_of(p):
    return O.geometry(p._args["fs"], p._args["N"], p._args["qs"], p._args["fmin"], p._args["fmax"], p._args["K"],
                      norm=p._args.get("norm", "l2"), max_window_hz=p._args.get("max_window_hz", 0.0),
                      n_out=p._args.get("n_out", 0), window=p._args.get("window", "bisquare"),
                      window_param=p._args.get("window_param", 0.0))


def make(fs, N, qs, fmin, fmax, K, compute="f32", envelope=None, **kw):
    p = qtam.Plan(fs, N, qs, fmin, fmax, K, compute=compute, envelope=envelope, device=0, **kw)
    p._args = dict(fs=fs, N=N, qs=qs, fmin=fmin, fmax=fmax, K=K, **kw)
    return p


SMALL = [
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12),
    dict(fs=64.0, N=256, qs=(1.0,), fmin=1.0, fmax=32.0, K=6),             # windows cut at DC and Nyquist
    dict(fs=256.0, N=1024, qs=(6.0, 12.0), fmin=2.0, fmax=100.0, K=20, n_out=96),
    dict(fs=64.0, N=512, qs=(2.0,), fmin=3.0, fmax=32.0, K=7, norm="none", max_window_hz=2.0),
    dict(fs=4096.0, N=6144, qs=(8.0, 40.0), fmin=30.0, fmax=1500.0, K=33),  # N/2 = 3 * 2^10
    dict(fs=1000.0, N=3000, qs=(3.0, 30.0), fmin=5.0, fmax=490.0, K=40),    # N/2 = 1500 = 2^2 3 5^3
]


# ---------------------------------------------------------------------------- stages
# powers of two from 2048 to 262144 samples run on thread-block clusters (one
# per segment, 1 to 16 CTAs); the others on the three-pass kernels
@pytest.mark.parametrize("N", [256, 512, 2048, 3000, 4096, 6144, 8192, 16384, 24576, 32768, 65536, 131072,
                               262144, 524288])
def test_spectrum_stage(N):
    p = make(4096.0, N, (8.0,), 30.0, 1000.0, 8, max_window_hz=20.0)
    B = 3
    x = np.stack([synth.white(s, N) for s in range(B)]).astype(np.float32)
    X = host(p.spectrum(dev(x))).astype(np.complex128)
    for b in range(B):
        ref = O.spectrum(x[b].astype(np.float64))
        assert rel(X[b], ref) < 1e-6
        assert elem_ok(X[b], ref, 1e-5)


@pytest.mark.parametrize("i", range(len(SMALL)))
def test_envelopes_stage_from_oracle_spectrum(i):
    p = make(**SMALL[i])
    g = geom_of(p)
    x = synth.white(100 + i, g.N)
    X = O.spectrum(x)
    y = env_np(p, p.envelopes(dev(X[None].astype(np.complex64))))[0]
    ref = np.stack([[O.forward_row(g, X, a, b) for b in range(g.K)] for a in range(g.P)])
    assert rel(y, ref) < FWD_FROB["f32"]
    assert elem_ok(y, ref, FWD_ELEM["f32"])


@pytest.mark.parametrize("i", range(len(SMALL)))
def test_accumulate_stage_from_oracle_envelopes(i):
    p = make(**SMALL[i])
    g = geom_of(p)
    rng = synth.rng(7 + i)
    Y = rng.standard_normal((g.P, g.K, g.M)) + 1j * rng.standard_normal((g.P, g.K, g.M))
    A = host(p.accumulate(dev(Y[None].astype(np.complex64)))).astype(np.complex128)[0]
    ref = O.accumulate(g, Y)
    assert rel(A, ref) < 1e-6
    assert elem_ok(A, ref, 1e-5)


@pytest.mark.parametrize("i", range(len(SMALL)))
def test_synthesize_stage_from_oracle_accumulator(i):
    p = make(**SMALL[i])
    g = geom_of(p)
    Y = O.forward(g, synth.white(40 + i, g.N))
    A = O.accumulate(g, Y)
    x = host(p.synthesize(dev(A[None].astype(np.complex64))))[0].astype(np.float64)
    ref = O.inverse(g, Y, tau=p.info["p_floor_rel"])
    assert rel(x, ref) < 1e-5


# ---------------------------------------------------------------------------- whole path
@pytest.mark.parametrize("i", range(len(SMALL)))
def test_forward_and_roundtrip_small(i):
    p = make(**SMALL[i])
    g = geom_of(p)
    B = 3
    x = np.stack([synth.white(200 + 10 * i + b, g.N) for b in range(B)]).astype(np.float32)
    y = p.forward(dev(x))
    Yg = env_np(p, y)
    xh = host(p.inverse(y)).astype(np.float64)
    tau = p.info["p_floor_rel"]
    for b in range(B):
        xb = x[b].astype(np.float64)
        ref = O.forward(g, xb)
        assert rel(Yg[b], ref) < FWD_FROB["f32"]
        assert elem_ok(Yg[b], ref, FWD_ELEM["f32"])
        assert rel(xh[b], O.projection(g, xb, tau=tau)) < RT["f32"]


WINDOWS = [("hann", 0.0), ("kaiser", 8.0), ("tukey", 0.5), ("planck", 0.3)]


@pytest.mark.parametrize("win,prm", WINDOWS)
@pytest.mark.parametrize("i", [0, 1, 2, 4])
def test_window_family_forward_and_roundtrip(win, prm, i):
    """App. A's alternative windows: per-plan W' tables read by the runtime engine."""
    p = make(**SMALL[i], window=win, window_param=prm)
    assert p.info["row_variant"] == -1
    g = geom_of(p)
    B = 2
    x = np.stack([synth.white(700 + 10 * i + b, g.N) for b in range(B)]).astype(np.float32)
    y = p.forward(dev(x))
    Yg = env_np(p, y)
    xh = host(p.inverse(y)).astype(np.float64)
    tau = p.info["p_floor_rel"]
    for b in range(B):
        xb = x[b].astype(np.float64)
        ref = O.forward(g, xb)
        assert rel(Yg[b], ref) < FWD_FROB["f32"]
        assert elem_ok(Yg[b], ref, FWD_ELEM["f32"])
        assert rel(xh[b], O.projection(g, xb, tau=tau)) < RT["f32"]


@pytest.mark.parametrize("win,prm", WINDOWS)
def test_window_family_float64(win, prm):
    """FP64 with an explicit floor tau = 1e-10: the Planck taper's edge weights
    fall like exp(-a h), so without a floor its frame operator keeps bins with
    P ~ 1e-32 max P and the canonical inverse divides rounding noise by them."""
    tau = 1e-10
    p = make(4096.0, 16384, (8.0,), 20.0, 1024.0, 64, compute="f64", window=win, window_param=prm, p_floor_rel=tau)
    g = geom_of(p)
    assert p.info["kept_bins"] == int(O.kept_bins(O.frame_operator(g), tau).sum())
    x = synth.white_sine_gaussian_segment(3).astype(np.float64)
    y = p.forward(dev(x[None]))
    Y = env_np(p, y)[0]
    ref = O.forward(g, x)
    assert rel(Y, ref) < FWD_FROB["f64"]
    assert elem_ok(Y, ref, FWD_ELEM["f64"])
    assert rel(host(p.inverse(y))[0], O.projection(g, x, tau=tau)) < RT["f64"]


def test_composite_bank_forward_roundtrip_and_optimal_plane():
    """Planes scanning Q x window x parameter in one plan (bisquare planes keep the
    formula, the others read their tables), one launch per stage."""
    wins = ("bisquare", "tukey", "kaiser", "planck", "hann", "bisquare")
    prms = (0.0, 0.5, 6.0, 0.3, 0.0, 0.0)
    p = make(4096.0, 32768, (8.0, 8.0, 8.0, 16.0, 16.0, 32.0), 20.0, 2048.0, 128, window=wins, window_param=prms)
    g = geom_of(p)
    x = np.stack([synth.glitchy_segment(900 + b, g.N, 4096.0, chirp=(b == 0)) for b in range(2)]).astype(np.float32)
    y = p.forward(dev(x))
    Yg = env_np(p, y)
    xh = host(p.inverse(y)).astype(np.float64)
    e, pk, _, _ = p.plane_metrics(y)
    tau = p.info["p_floor_rel"]
    for b in range(2):
        xb = x[b].astype(np.float64)
        ref = O.forward(g, xb)
        assert rel(Yg[b], ref) < FWD_FROB["f32"]
        assert elem_ok(Yg[b], ref, FWD_ELEM["f32"])
        assert rel(xh[b], O.projection(g, xb, tau=tau)) < RT["f32"]
        eo, po, _, _ = O.plane_metrics(ref)
        assert np.allclose(host(e)[b], eo, rtol=2e-6)
        assert np.allclose(host(pk)[b], po, rtol=5e-6)


def test_window_family_full_size_sampled_rows():
    """64 s, five planes, 128 rows, Kaiser beta = 8 (M = 4800, runtime engine)."""
    p = make(4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128, window="kaiser", window_param=8.0)
    g = geom_of(p)
    x = synth.coloured_chirp_segment(5)[None]
    y = p.forward(dev(x))
    Y = env_np(p, y)[0]
    X = O.spectrum(x[0].astype(np.float64))
    rows = [(0, 0), (0, 127), (1, 64), (3, 100), (4, 127)]
    big = max(np.max(np.abs(O.forward_row(g, X, a, k))) for a, k in rows)
    for a, k in rows:
        ref = O.forward_row(g, X, a, k)
        assert rel(Y[a, k], ref) < FWD_FROB["f32"], (a, k)
        assert np.max(np.abs(Y[a, k] - ref)) <= FWD_ELEM["f32"] * big
    xh = host(p.inverse(y))[0].astype(np.float64)
    assert rel(xh, O.projection(g, x[0].astype(np.float64), tau=p.info["p_floor_rel"])) < RT["f32"]


def test_batch_zero_is_noop():
    p = make(**SMALL[0])
    x = torch.zeros((0, p.N), dtype=torch.float32, device="cuda")
    y = p.forward(x)
    assert y.shape[0] == 0
    assert p.inverse(y).shape == (0, p.N)


def test_config1_float64_roundtrip():
    """4 s at 4096 Hz, white noise + sine-Gaussian, Q=8, 64 rows 20-1024 Hz, FP64."""
    p = make(4096.0, 16384, (8.0,), 20.0, 1024.0, 64, compute="f64")
    g = geom_of(p)
    x = synth.white_sine_gaussian_segment(0).astype(np.float64)
    y = p.forward(dev(x[None]))
    Y = env_np(p, y)[0]
    ref = O.forward(g, x)
    assert rel(Y, ref) < FWD_FROB["f64"]
    assert elem_ok(Y, ref, FWD_ELEM["f64"])
    xh = host(p.inverse(y))[0]
    assert rel(xh, O.projection(g, x)) < RT["f64"]
    assert p.info["p_floor_rel"] == 0.0


@pytest.fixture(scope="module")
def cfg2():
    """64 s at 4096 Hz, Q in {4,8,16,32,64}, 128 rows 20-2048 Hz, FP32, coloured+whitened noise + chirp."""
    p = make(4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128)
    g = geom_of(p)
    x = np.stack([synth.coloured_chirp_segment(s) for s in range(2)])
    return p, g, x


def test_config2_forward_sampled_rows(cfg2):
    p, g, x = cfg2
    y = p.forward(dev(x))
    Y = env_np(p, y)
    rows = [(0, 0), (0, 127), (1, 64), (2, 5), (3, 100), (4, 127), (4, 0), (2, 126)]
    for b in range(x.shape[0]):
        X = O.spectrum(x[b].astype(np.float64))
        big = max(np.max(np.abs(O.forward_row(g, X, a, k))) for a, k in rows)
        for a, k in rows:
            ref = O.forward_row(g, X, a, k)
            assert rel(Y[b, a, k], ref) < FWD_FROB["f32"], (a, k)
            assert np.max(np.abs(Y[b, a, k] - ref)) <= FWD_ELEM["f32"] * big


def test_config2_forward_every_row_every_variant(cfg2):
    """Every (plane, row) envelope of both 64 s segments against the oracle,
    element by element, for each compile-time 4800-point variant and the
    runtime engine: a phase or index error that cancels in the round trip, or
    that the energy identity cannot see, shows up here (Sec. III demodulation)."""
    p, g, x = cfg2
    refs = [O.forward(g, x[b].astype(np.float64)) for b in range(x.shape[0])]
    xd = dev(x)
    variants = qtam.qtam_plan_variants(p.handle)
    assert len(variants) >= 4, variants
    chosen = p.info["row_variant"]
    try:
        for v in variants:
            qtam.qtam_plan_set_variant(p.handle, v)
            Y = env_np(p, p.forward(xd))
            name = qtam.qtam_variant_describe(v)["name"]
            for b, ref in enumerate(refs):
                big = np.max(np.abs(ref))
                for a in range(g.P):
                    for k in range(g.K):
                        assert rel(Y[b, a, k], ref[a, k]) < FWD_FROB["f32"], (name, b, a, k)
                assert np.max(np.abs(Y[b] - ref)) <= FWD_ELEM["f32"] * big, name
    finally:
        qtam.qtam_plan_set_variant(p.handle, chosen)


def test_config2_roundtrip(cfg2):
    p, g, x = cfg2
    xh = host(p.inverse(p.forward(dev(x)))).astype(np.float64)
    tau = p.info["p_floor_rel"]
    for b in range(x.shape[0]):
        xp = O.projection(g, x[b].astype(np.float64), tau=tau)
        assert rel(xh[b], xp) < RT["f32"]


def test_config2_energy_identity(cfg2):
    """sum |Y|^2 = (1/N) sum_f P[f] |X[f]|^2 at full size (App. C frame operator)."""
    p, g, x = cfg2
    Y = env_np(p, p.forward(dev(x[:1])))[0]
    X = O.spectrum(x[0].astype(np.float64))
    Pf = p.frame_operator(0)
    assert np.sum(np.abs(Y) ** 2) == pytest.approx(np.sum(Pf * np.abs(X) ** 2) / g.N, rel=1e-5)


def test_linearity_and_shift_invariance_gpu():
    N = 16384
    p = make(4096.0, N, (8.0, 16.0), 20.0, 1024.0, 48, n_out=512)
    x1, x2 = synth.white(1, N), synth.white(2, N)
    a, b = 0.5, -1.75
    xs = np.stack([x1, x2, a * x1 + b * x2, np.roll(x1, N // 512)]).astype(np.float32)
    Y = env_np(p, p.forward(dev(xs)))
    lhs, rhs = Y[2], a * Y[0] + b * Y[1]
    assert rel(lhs, rhs) < 2e-6
    ph = np.exp(-2j * np.pi * p.geometry.kc / p.M)[..., None]
    assert rel(Y[3], ph * np.roll(Y[0], 1, axis=-1)) < 2e-6


def test_masked_and_plane_inverse():
    p = make(**SMALL[0])
    g = geom_of(p)
    x = synth.white(77, g.N).astype(np.float32)
    y = p.forward(dev(x[None]))
    Y = env_np(p, y)[0]
    tau = p.info["p_floor_rel"]
    ym = y.clone()
    ym[0, 0, 2:5] = 0
    ym[0, 1, 7] = 0
    Ym = Y.copy()
    Ym[0, 2:5] = 0
    Ym[1, 7] = 0
    xm = host(p.inverse(ym))[0]
    assert rel(xm, O.inverse(g, Ym, tau=tau)) < RT["f32"]
    x1 = host(p.inverse(y, plane_mask=0b10))[0]
    assert rel(x1, O.inverse(g, Y, planes=[1], tau=tau)) < RT["f32"]


@pytest.mark.parametrize("env,tol_f,tol_rt", [("bf16", 1e-2, 1e-2), ("f16", 2e-3, 2e-3)])
def test_16bit_envelopes(env, tol_f, tol_rt):
    p = make(4096.0, 32768, (8.0, 16.0, 32.0), 20.0, 2048.0, 128, envelope=env)
    g = geom_of(p)
    x = synth.glitchy_segment(3, 32768, 4096.0, chirp=True)
    y = p.forward(dev(x[None]))
    Y = env_np(p, y)[0]
    xd = x.astype(np.float64)
    assert rel(Y, O.forward(g, xd)) < tol_f
    xh = host(p.inverse(y))[0]
    assert rel(xh, O.projection(g, xd, tau=p.info["p_floor_rel"])) < tol_rt


@pytest.mark.parametrize("B", [2, 11, 20])
def test_roundtrip_host_entry(B):
    """Host round trip, pipelined over up to 8 chunks (uneven for B = 11, 20):
    every segment comes back as the oracle's projection, and the envelopes
    left on the device are the plain forward's."""
    p = make(**SMALL[4])
    g = geom_of(p)
    x = np.stack([synth.white(300 + b, g.N) for b in range(B)]).astype(np.float32)
    xh_pinned = torch.empty((B, g.N), dtype=torch.float32).pin_memory()
    x_pinned = torch.from_numpy(x).pin_memory()
    x_dev = torch.empty((B, g.N), dtype=torch.float32, device="cuda")
    xh_dev = torch.empty_like(x_dev)
    y_dev = p.envelope_tensor(B)
    ws, wsb = p.workspace(B)
    for _ in range(2):                      # the second call reuses the plan's streams and events
        xh_pinned.zero_()
        qtam.qtam_roundtrip_host(p.handle, x_pinned, B, 0, xh_pinned, x_dev, y_dev, xh_dev, ws, wsb)
        xh = xh_pinned.numpy().astype(np.float64)
        for b in range(B):
            assert rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < RT["f32"]
    assert torch.equal(y_dev, p.forward(torch.from_numpy(x).cuda()))


def test_roundtrip_host_pipelined_chunks(cfg2):
    """50 segments of 64 s (1 MiB each): three uneven chunks of the host round
    trip; every segment equals the device path and sampled ones the oracle."""
    p, g, _ = cfg2
    B = 50
    x = np.stack([synth.white(900 + b, g.N) for b in range(B)]).astype(np.float32)
    x_pinned = torch.from_numpy(x).pin_memory()
    xh_pinned = torch.empty((B, g.N), dtype=torch.float32).pin_memory()
    x_dev = torch.empty((B, g.N), dtype=torch.float32, device="cuda")
    xh_dev = torch.empty_like(x_dev)
    y_dev = p.envelope_tensor(B)
    ws, wsb = p.workspace(B)
    qtam.qtam_roundtrip_host(p.handle, x_pinned, B, 0, xh_pinned, x_dev, y_dev, xh_dev, ws, wsb)
    xd = torch.from_numpy(x).cuda()
    yd = p.forward(xd)
    assert torch.equal(y_dev, yd)
    ref = host(p.inverse(yd)).astype(np.float64)
    xh = xh_pinned.numpy().astype(np.float64)
    assert max(rel(xh[b], ref[b]) for b in range(B)) < 1e-6     # the inverse accumulates with float atomics
    for b in (0, 17, 49):
        assert rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < RT["f32"]


def test_device_errors_are_reported():
    p = make(**SMALL[0])
    with pytest.raises(qtam.QtamError) as e:
        qtam.qtam_forward(p.handle, 0, 1, 0, 0, 0)
    assert e.value.status == 1
    ws, wsb = p.workspace(4)
    x = torch.zeros((4, p.N), dtype=torch.float32, device="cuda")
    y = p.envelope_tensor(4)
    with pytest.raises(qtam.QtamError) as e:
        qtam.qtam_forward(p.handle, x, 4, y, ws, 16)
    assert e.value.status == 9


def test_plane_metrics_and_optimal_plane():
    """Optimal-plane selection: per-plane energy and peak of the envelopes match the
    oracle and select the same plane for every segment."""
    p = make(4096.0, 32768, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 64)
    g = geom_of(p)
    B = 4
    x = np.stack([synth.glitchy_segment(40 + b, g.N, 4096.0, chirp=True) for b in range(B)])
    y = p.forward(dev(x))
    energy, peak, best_e, best_p = p.plane_metrics(y)
    torch.cuda.synchronize()
    Yg = env_np(p, y)
    for b in range(B):
        e, pk, be, bp = O.plane_metrics(O.forward(g, x[b].astype(np.float64)))
        assert np.allclose(energy[b].cpu().numpy(), e, rtol=2e-6)
        assert np.allclose(peak[b].cpu().numpy(), pk, rtol=5e-6)
        e_gpu, pk_gpu, _, _ = O.plane_metrics(Yg[b])          # same reduction of the GPU envelopes
        # FP32 squares summed in short FP32 partials, then FP64 (relative error <= ~5e-7)
        assert np.allclose(energy[b].cpu().numpy(), e_gpu, rtol=1e-6)
        assert int(best_e[b]) == int(np.argmax(e_gpu)) and int(best_p[b]) == int(np.argmax(pk_gpu))


def test_edge_M_equals_largest_window():
    """M = L_max exactly (45): every baseband position holds a band offset."""
    p = make(64.0, 512, (4.0, 8.0), 3.0, 29.0, 12)
    g = geom_of(p)
    assert p.M == int(g.L.max()) == 45
    x = synth.white(61, g.N).astype(np.float32)
    y = p.forward(dev(x[None]))
    Y = env_np(p, y)[0]
    ref = O.forward(g, x.astype(np.float64))
    assert rel(Y, ref) < FWD_FROB["f32"]
    xh = host(p.inverse(y))[0]
    assert rel(xh, O.projection(g, x.astype(np.float64), tau=p.info["p_floor_rel"])) < RT["f32"]


def test_edge_single_row_unclamped():
    """K = 1: no neighbouring centre, so no clamp; one window of half-width 44."""
    p = make(64.0, 512, (6.0,), 10.0, 10.0, 1)
    g = geom_of(p)
    assert g.K == 1 and int(g.h[0, 0]) == 44
    x = synth.white(62, g.N).astype(np.float32)
    y = p.forward(dev(x[None]))
    assert rel(env_np(p, y)[0], O.forward(g, x.astype(np.float64))) < FWD_FROB["f32"]
    xh = host(p.inverse(y))[0]
    assert rel(xh, O.projection(g, x.astype(np.float64), tau=p.info["p_floor_rel"])) < RT["f32"]


def test_edge_batch_above_grid_y_limit():
    """65540 segments: the long-FFT launches split the batch at 65535 grid rows."""
    p = make(256.0, 256, (2.0,), 20.0, 60.0, 2)
    g = geom_of(p)
    B = 65540
    rng = synth.rng(63)
    x = rng.standard_normal((B, g.N)).astype(np.float32)
    xd = dev(x)
    y = p.forward(xd)
    xh = p.inverse(y)
    torch.cuda.synchronize()
    tau = p.info["p_floor_rel"]
    for b in (0, 65534, 65535, 65536, B - 1):
        xb = x[b].astype(np.float64)
        assert rel(y[b].cpu().numpy().astype(np.complex128), O.forward(g, xb)) < FWD_FROB["f32"], b
        assert rel(xh[b].cpu().numpy().astype(np.float64), O.projection(g, xb, tau=tau)) < RT["f32"], b


def test_edge_maximum_length():
    """The largest accepted segment, N = 2^27 (9.1 hours at 4096 Hz: a long FFT
    of 2^26 complex points), two segments so the second starts 2^27 samples
    in; the manual clamp keeps every window at h = 2048 (M = 4320).  Every row
    of both segments and the second segment's round trip against the
    oracle."""
    N = 2 ** 27
    p = make(4096.0, N, (8.0,), 20.0, 1024.0, 8, max_window_hz=0.125)
    g = geom_of(p)
    assert p.N == N and p.M == g.M == 4320 and int(g.h.max()) == 2048
    B = 2
    x = np.stack([synth.white(70 + b, N) for b in range(B)]).astype(np.float32)
    xd = dev(x)
    y = p.forward(xd)
    xh = p.inverse(y)
    torch.cuda.synchronize()
    Y = env_np(p, y)
    for b in range(B):
        X = O.spectrum(x[b].astype(np.float64))
        for k in range(g.K):
            ref = O.forward_row(g, X, 0, k)
            assert rel(Y[b, 0, k], ref) < FWD_FROB["f32"], (b, k)
        del X
    xb = x[1].astype(np.float64)
    assert rel(host(xh[1:])[0], O.projection(g, xb, tau=p.info["p_floor_rel"])) < RT["f32"]


def test_edge_one_bin_windows():
    """Rows whose ideal half-width rounds to 0 get h = 1 (reading C3b): the
    bisquare is then a single bin (W' = 1 at k_c, 0 at k_c +/- 1); three such
    rows beside wider ones, M = 15."""
    p = make(64.0, 256, (40.0,), 2.0, 20.0, 6)
    g = geom_of(p)
    assert [int(h) for h in g.h[0]] == [1, 1, 1, 2, 4, 6] and p.M == g.M == 15
    B = 3
    x = np.stack([synth.white(80 + b, g.N) for b in range(B)]).astype(np.float32)
    y = p.forward(dev(x))
    Yg = env_np(p, y)
    xh = host(p.inverse(y)).astype(np.float64)
    for b in range(B):
        xb = x[b].astype(np.float64)
        ref = O.forward(g, xb)
        assert rel(Yg[b], ref) < FWD_FROB["f32"]
        assert elem_ok(Yg[b], ref, FWD_ELEM["f32"])
        assert rel(xh[b], O.projection(g, xb, tau=p.info["p_floor_rel"])) < RT["f32"]
