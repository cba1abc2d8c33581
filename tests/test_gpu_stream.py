"""Streaming (overlap-save) analysis and synthesis through the C ABI against the
FP64 oracle's stream_forward / stream_inverse (reading S1)."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    torch.cuda.synchronize()
    if t.dtype in (torch.bfloat16, torch.float16):
        a = t.float().cpu().numpy().astype(np.float64)
        return a[..., 0] + 1j * a[..., 1]
    return t.cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SMALL = dict(fs=256.0, N=1024, qs=(6.0, 12.0), fmin=2.0, fmax=100.0, K=20, n_out=96)   # quantum 32 samples


def _plan(cfg, **kw):
    c = dict(cfg)
    p = qtam.Plan(c.pop("fs"), c.pop("N"), c.pop("qs"), c.pop("fmin"), c.pop("fmax"), c.pop("K"), device=0, **c, **kw)
    g = O.geometry(cfg["fs"], cfg["N"], cfg["qs"], cfg["fmin"], cfg["fmax"], cfg["K"], n_out=cfg.get("n_out", 0),
                   max_window_hz=cfg.get("max_window_hz", 0.0))
    return p, g


def _push(s, x, pieces):
    out, o = [], 0
    for k in pieces:
        out.append(s.forward(x[o:o + k * s.hop]))
        o += k * s.hop
    return torch.cat(out, dim=2)


@pytest.mark.parametrize("hop", [512, 256, 1024])
def test_stream_forward_and_inverse_match_oracle(hop):
    p, g = _plan(SMALL)
    s = qtam.Stream(p, hop=hop, max_chunks=3)
    J = 12 * (1024 // hop)
    x = synth.glitchy_segment(7, J * hop, 256.0, chirp=True).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    pieces = [3, 1, 5] + [1] * (J - 9)
    Y = _push(s, xd, pieces)
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    Yg = _np(Y)
    assert Yg.shape == Yo.shape
    assert _rel(Yg, Yo) < 1e-6
    assert np.max(np.abs(Yg - Yo)) <= 1e-5 * np.max(np.abs(Yo))
    # inverse of the GPU's own map, pushed in other pieces, against the oracle's inverse of that map
    cols = s.hop_cols
    parts, o = [], 0
    for k in [2, 4] + [1] * (J - 6):
        parts.append(s.inverse(Y[:, :, o:o + k * cols].contiguous()))
        o += k * cols
    xh = _np(torch.cat(parts))
    xo = O.stream_inverse(g, Yg, hop, tau=p.info["p_floor_rel"])
    assert _rel(xh, xo) < 1e-5
    info = qtam.qtam_stream_info(s.handle)
    assert info["samples_in"] == J * hop and info["columns_in"] == J * cols


def test_stream_is_independent_of_push_sizes_and_resets():
    """The forward map is bitwise independent of how the stream is pushed."""
    p, _ = _plan(SMALL)
    x = torch.from_numpy(synth.white(3, 40 * 512).astype(np.float32)).cuda()
    a = qtam.Stream(p, hop=512, max_chunks=40)
    b = qtam.Stream(p, hop=512, max_chunks=2)
    Ya = a.forward(x)
    Yb = _push(b, x, [1, 7, 2, 30])
    assert torch.equal(Ya, Yb)
    a.reset()
    assert torch.equal(a.forward(x), Ya)
    xa = a.inverse(Ya)
    xb = _push_inv(b, Ya, [5, 5, 30])
    # the inverse accumulates rows with float atomics (order-dependent rounding)
    assert float((xa - xb).norm() / xa.norm()) < 1e-6


def _push_inv(s, Y, pieces):
    out, o = [], 0
    for k in pieces:
        out.append(s.inverse(Y[:, :, o:o + k * s.hop_cols].contiguous()))
        o += k * s.hop_cols
    return torch.cat(out)


def test_stream_periodic_signal_round_trip_is_delayed_projection():
    """A periodic stream inverts, past the start-up chunks, to the segment's
    projection delayed by 2G (exact up to FP32 rounding)."""
    p, g = _plan(SMALL)
    s = qtam.Stream(p, hop=512, max_chunks=4)
    x0 = synth.white(11, g.N)
    x = np.tile(x0, 10).astype(np.float32)
    Y = s.forward(torch.from_numpy(x).cuda())
    xh = _np(s.inverse(Y))
    G = s.guard
    st = 8 * 512
    idx = np.arange(st, xh.size)
    xp0 = O.projection(g, x0.astype(np.float32).astype(np.float64), tau=p.info["p_floor_rel"])
    assert _rel(xh[idx], xp0[(idx - 2 * G) % g.N]) < 1e-5


def test_stream_float64_and_bf16():
    p, g = _plan(SMALL, compute="f64")
    s = qtam.Stream(p, hop=512, max_chunks=4)
    x = synth.glitchy_segment(5, 16 * 512, 256.0).astype(np.float64)
    Y = s.forward(torch.from_numpy(x).cuda())
    Yo = O.stream_forward(g, x, 512)
    assert _rel(_np(Y), Yo) < 1e-13
    assert _rel(_np(s.inverse(Y)), O.stream_inverse(g, Yo, 512)) < 1e-12
    pb, _ = _plan(SMALL, envelope="bf16")
    sb = qtam.Stream(pb, hop=512, max_chunks=4)
    Yb = _np(sb.forward(torch.from_numpy(x.astype(np.float32)).cuda()))
    assert _rel(Yb, Yo) < 1e-2


def test_stream_full_size_chunks():
    """64 s chunks at 4096 Hz (N = 2^18, M = 4800, quantum 4096 samples), hop
    32 s: an 8-hop (256 s) stream of coloured noise with a chirp."""
    cfg = dict(fs=4096.0, N=262144, qs=(4.0, 8.0, 16.0, 32.0, 64.0), fmin=20.0, fmax=2048.0, K=128)
    p, g = _plan(cfg)
    s = qtam.Stream(p, hop=131072, max_chunks=3)
    assert s.guard == 65536 and s.hop_cols == 2400
    x = np.concatenate([synth.coloured_chirp_segment(20 + i)[:131072] for i in range(8)]).astype(np.float32)
    Y = s.forward(torch.from_numpy(x).cuda())
    Yg = _np(Y)
    Yo = O.stream_forward(g, x.astype(np.float64), 131072)
    assert _rel(Yg, Yo) < 1e-6
    assert np.max(np.abs(Yg - Yo)) <= 1e-5 * np.max(np.abs(Yo))
    xh = _np(s.inverse(Y))
    xo = O.stream_inverse(g, Yg, 131072, tau=p.info["p_floor_rel"])
    assert _rel(xh, xo) < 1e-5


def test_stream_fused_row_kernels_m600():
    """N = 32768 chunks at 4096 Hz, Q {8,16,32} x 128 rows (M = 600, quantum 4096
    samples): the compile-time variant's fused streaming kernels (crop-and-phase
    store, history/new-columns load) against the oracle, push-size invariance
    and a plane-masked inverse."""
    cfg = dict(fs=4096.0, N=32768, qs=(8.0, 16.0, 32.0), fmin=20.0, fmax=2048.0, K=128)
    p, g = _plan(cfg)
    assert p.M == 600 and p.info["row_variant"] >= 0
    hop = 16384
    J = 12
    x = np.concatenate([synth.glitchy_segment(40 + i, hop, 4096.0, chirp=(i % 3 == 0)) for i in range(J)])
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    s1 = qtam.Stream(p, hop=hop, max_chunks=5)
    s2 = qtam.Stream(p, hop=hop, max_chunks=12)
    Y = _push(s1, xd, [2, 5, 1, 4])
    assert torch.equal(Y, s2.forward(xd))
    Yg = _np(Y)
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    assert _rel(Yg, Yo) < 1e-6
    assert np.max(np.abs(Yg - Yo)) <= 1e-5 * np.max(np.abs(Yo))
    xh = _np(_push_inv(s1, Y, [3, 3, 6]))
    tau = p.info["p_floor_rel"]
    assert _rel(xh, O.stream_inverse(g, Yg, hop, tau=tau)) < 1e-5
    xm = _np(s2.inverse(Y, plane_mask=0b010))
    assert _rel(xm, O.stream_inverse(g, Yg, hop, planes=[1], tau=tau)) < 1e-5


def test_stream_fused_row_kernels_m8192_cuda_cores():
    """M = 8192 on CUDA cores: the four-stage default variant's fused
    streaming kernels against the oracle's stream at FP32 accuracy."""
    cfg = dict(fs=4096.0, N=32768, qs=(8.0, 16.0), fmin=20.0, fmax=2048.0, K=32, n_out=8192)
    p, g = _plan(cfg, short_dft="cuda")
    assert p.M == 8192
    assert qtam.qtam_variant_describe(p.info["row_variant"])["name"] == "8192:16, 8, 8, 8 rows/blk 2^0 minblk 2"
    hop = 16384
    s = qtam.Stream(p, hop=hop, max_chunks=4)
    x = synth.glitchy_segment(23, 6 * hop, 4096.0, chirp=True).astype(np.float32)
    Y = _push(s, torch.from_numpy(x).cuda(), [2, 1, 3])
    Yg = _np(Y)
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    assert _rel(Yg, Yo) < 1e-6
    xh = _np(s.inverse(Y.contiguous()))
    assert _rel(xh, O.stream_inverse(g, Yg, hop, tau=p.info["p_floor_rel"])) < 1e-5


def test_stream_fused_row_kernels_m2400_threads_160():
    """32 s chunks at 4096 Hz (M = 2400): the 160-thread default variant's
    fused streaming kernels against the oracle's stream at FP32 accuracy."""
    cfg = dict(fs=4096.0, N=131072, qs=(8.0, 16.0, 32.0), fmin=20.0, fmax=2048.0, K=128)
    p, g = _plan(cfg)
    assert p.M == 2400
    assert qtam.qtam_variant_describe(p.info["row_variant"])["name"] == "2400:16, 10, 15 rows/blk 2^0 minblk 6 threads 160"
    hop = 65536
    s = qtam.Stream(p, hop=hop, max_chunks=3)
    x = synth.glitchy_segment(29, 5 * hop, 4096.0, chirp=True).astype(np.float32)
    Y = _push(s, torch.from_numpy(x).cuda(), [2, 1, 2])
    Yg = _np(Y)
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    assert _rel(Yg, Yo) < 1e-6
    xh = _np(s.inverse(Y.contiguous()))
    assert _rel(xh, O.stream_inverse(g, Yg, hop, tau=p.info["p_floor_rel"])) < 1e-5


def test_stream_over_tensor_core_plan():
    """A stream over a plan with the tensor-core short DFT (M = 8192, both
    directions on tcgen05) against the oracle's stream, at the BF16 bound of
    the tensor-core rows (relative 1e-2)."""
    cfg = dict(fs=4096.0, N=32768, qs=(8.0, 16.0), fmin=20.0, fmax=2048.0, K=32, n_out=8192)
    t0 = qtam.qtam_tc_status()
    p, g = _plan(cfg, short_dft="tensor")
    hop = 16384
    s = qtam.Stream(p, hop=hop, max_chunks=4)
    J = 6
    x = synth.glitchy_segment(17, J * hop, 4096.0, chirp=True).astype(np.float32)
    Y = _push(s, torch.from_numpy(x).cuda(), [2, 1, 3])
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    Yg = _np(Y)
    assert Yg.shape == Yo.shape
    assert _rel(Yg, Yo) < 1e-2
    xh = _np(s.inverse(Y.contiguous()))
    xo = O.stream_inverse(g, Yg, hop, tau=p.info["p_floor_rel"])
    assert _rel(xh, xo) < 2e-2
    assert qtam.qtam_tc_status() == t0


@pytest.mark.parametrize("cfg,kw,hop", [
    (SMALL, dict(remodulate=True), 512),                                           # carrier alone
    (SMALL, dict(remodulate=True, envelope="bf16"), 512),                          # carrier, 16-bit map (phase kernels)
    (dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, n_out=320),
     dict(remodulate=True, stopband_eps=1e-3), 256),                               # dense: floor and carrier
])
def test_stream_over_remodulated_plans(cfg, kw, hop):
    """Remodulated tiles carry their carrier on absolute time, so the stream
    re-references their chunks by 1 (reading S1): forward map and streaming
    inverse against the oracle's stream of the same plan.  A BF16 map goes
    through the unfused phase kernels and is held to BF16 accuracy; its
    inverse is compared with the oracle's inverse of the stored map."""
    c = dict(cfg)
    kw = dict(kw)
    env = kw.pop("envelope", "f32")
    p = qtam.Plan(c.pop("fs"), c.pop("N"), c.pop("qs"), c.pop("fmin"), c.pop("fmax"), c.pop("K"), device=0,
                  envelope=env, **c, **kw)
    g = O.geometry(cfg["fs"], cfg["N"], cfg["qs"], cfg["fmin"], cfg["fmax"], cfg["K"], n_out=cfg.get("n_out", 0),
                   **kw)
    assert p.M == g.M and p.info["remodulate"] == 1
    s = qtam.Stream(p, hop=hop, max_chunks=3)
    J = 10
    x = synth.glitchy_segment(9, J * hop, cfg["fs"]).astype(np.float32) if cfg["fs"] > 100 else \
        synth.white(9, J * hop).astype(np.float32)
    Y = _push(s, torch.from_numpy(x).cuda(), [3, 1, 4, 2])
    Yo = O.stream_forward(g, x.astype(np.float64), hop)
    Yg = _np(Y)
    assert Yg.shape == Yo.shape
    assert _rel(Yg, Yo) < (1e-2 if env == "bf16" else 1e-6)
    xh = _np(s.inverse(Y.contiguous()))
    xo = O.stream_inverse(g, Yg, hop, tau=p.info["p_floor_rel"])
    assert _rel(xh, xo) < 1e-5
