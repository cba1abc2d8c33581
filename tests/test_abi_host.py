"""The C-ABI library loads, exports every symbol include/qtam.h declares, and
its host-side plan logic (App. A geometry, FP64 frame operator, argument
checks) agrees with the oracle.  No GPU is needed: plans are made host-only
(device = -1), and no transform is launched."""
import math

import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam


@pytest.fixture(scope="module")
def L():
    return qtam.lib()


def test_library_exports_every_header_symbol(L):
    names = qtam.header_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
        assert n in qtam.SIGNATURES, n


def test_status_strings(L):
    for s in range(10):
        assert qtam.qtam_status_string(s) not in ("", "unknown status")


CASES = [
    dict(fs=4096, N=16384, qs=(8,), fmin=20, fmax=1024, K=64),
    dict(fs=4096, N=262144, qs=(4, 8, 16, 32, 64), fmin=20, fmax=2048, K=128),
    dict(fs=4096, N=32768, qs=(8, 16, 32), fmin=20, fmax=2048, K=128),
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12),
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, norm="paper"),
    dict(fs=64.0, N=512, qs=(2.0,), fmin=3.0, fmax=32.0, K=7, norm="none", max_window_hz=2.0),
    dict(fs=256.0, N=1024, qs=(6.0, 12.0), fmin=2.0, fmax=100.0, K=20, n_out=96),
    dict(fs=16384, N=16384 * 2, qs=(8, 16, 32), fmin=20, fmax=2048, K=128),
    # the App. A window family
    dict(fs=4096, N=32768, qs=(8, 16, 32), fmin=20, fmax=2048, K=128, window="hann"),
    dict(fs=4096, N=32768, qs=(8, 16, 32), fmin=20, fmax=2048, K=128, window="kaiser", window_param=8.0),
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, window="tukey", window_param=0.5),
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, window="planck", window_param=0.3,
         norm="paper"),
    dict(fs=4096, N=16384, qs=(8,), fmin=20, fmax=1024, K=64, window="tukey", window_param=1.0),
    dict(fs=4096, N=16384, qs=(8,), fmin=20, fmax=1024, K=64, window="planck", window_param=0.0),
    dict(fs=4096, N=16384, qs=(8,), fmin=20, fmax=1024, K=64, window="kaiser", window_param=0.0),
    # composite bank: planes scan Q x window x parameter
    dict(fs=4096, N=32768, qs=(8, 8, 8, 16, 16), fmin=20, fmax=2048, K=128,
         window=("bisquare", "tukey", "kaiser", "planck", "hann"), window_param=(0.0, 0.5, 6.0, 0.3, 0.0)),
    # dense mode: stopband floor, tiles spanning the one-sided spectrum
    dict(fs=64.0, N=512, qs=(4.0, 8.0), fmin=3.0, fmax=30.0, K=12, stopband_eps=1e-6),
    dict(fs=4096, N=8192, qs=(4, 8, 16), fmin=20, fmax=2048, K=64, stopband_eps=1e-5, remodulate=True,
         window="hann"),
]


def _both(c):
    kw = dict(norm=c.get("norm", "l2"), max_window_hz=c.get("max_window_hz", 0.0), n_out=c.get("n_out", 0),
              window=c.get("window", "bisquare"), window_param=c.get("window_param", 0.0),
              stopband_eps=c.get("stopband_eps", 0.0), remodulate=c.get("remodulate", False))
    g = O.geometry(c["fs"], c["N"], c["qs"], c["fmin"], c["fmax"], c["K"], **kw)
    p = qtam.Plan(c["fs"], c["N"], c["qs"], c["fmin"], c["fmax"], c["K"], device=-1, **kw)
    return g, p


@pytest.mark.parametrize("i", range(len(CASES)))
def test_geometry_matches_oracle(i):
    g, p = _both(CASES[i])
    assert p.M == g.M
    # the largest tile support: 2h + 1, or the whole one-sided spectrum in dense mode
    assert p.info["max_window"] == (max(int(g.L.max()), g.Nr) if g.eps > 0 else int(g.L.max()))
    assert p.info["h_max"] == min(g.h_max, 2**31 - 1)
    assert np.array_equal(p.geometry.kc, g.kc)
    assert np.array_equal(p.geometry.h, g.h)
    assert np.allclose(p.geometry.f, g.f, rtol=1e-14, atol=0)
    assert np.allclose(p.geometry.c, g.c, rtol=1e-12, atol=0)


@pytest.mark.parametrize("i", range(len(CASES)))
def test_frame_operator_and_floor_match_oracle(i):
    g, p = _both(CASES[i])
    Pl = p.frame_operator(0)
    Po = O.frame_operator(g)
    assert np.max(np.abs(Pl - Po)) <= 1e-12 * np.max(Po)
    tau = p.info["p_floor_rel"]
    assert tau == 1e-6
    assert p.info["kept_bins"] == int(O.kept_bins(Po, tau).sum())
    assert p.info["kappa"] == pytest.approx(O.kappa(g, tau=tau), rel=1e-9)
    if g.P > 1:
        P1 = p.frame_operator(0b10)
        assert np.max(np.abs(P1 - O.frame_operator(g, planes=[1]))) <= 1e-12 * np.max(Po)
    assert p.info["band_bins"] == sum(O.band(g, a, b)[0].size for a in range(g.P) for b in range(g.K))


def test_plan_info_sizes():
    g, p = _both(CASES[1])
    assert p.info["envelope_bytes_per_segment"] == 5 * 128 * 4800 * 8
    assert p.info["fft_n1"] * p.info["fft_n2"] == g.N // 2
    assert p.info["device_bytes"] == 0          # host-only: nothing uploaded
    ws = qtam.qtam_workspace_size(p.handle, 64)
    assert ws >= 64 * (g.N // 2 + g.Nr) * 8


def _err(fn):
    with pytest.raises(qtam.QtamError) as e:
        fn()
    return e.value.status


def test_argument_errors():
    assert _err(lambda: qtam.Plan(4096, 16383, (8,), 20, 1024, 64, device=-1)) == 1          # odd N
    assert _err(lambda: qtam.Plan(4096, 16384, (), 20, 1024, 64, device=-1)) == 1            # no planes
    assert _err(lambda: qtam.Plan(4096, 16384, (8,), 2000, 1024, 64, device=-1)) == 1        # fmin > fmax
    assert _err(lambda: qtam.Plan(4096, 16384, (8,), 20, 1024, 64, n_out=100, device=-1)) == 3   # aliasing
    assert _err(lambda: qtam.Plan(4096, 16384, (8,), 20, 1024, 64, n_out=251, device=-1)) == 2   # 251 is prime
    assert _err(lambda: qtam.Plan(4096, 16384, (8,), 20, 1024, 64, compute="f64", envelope="bf16", device=-1)) == 1
    assert _err(lambda: qtam.Plan(4096, 16384 + 14, (8,), 20, 1024, 64, device=-1)) == 2     # N/2 = 8199 = 3*2733
    p = qtam.Plan(4096, 16384, (8,), 20, 1024, 64, device=-1)
    assert _err(lambda: qtam.qtam_forward(p.handle, 0, 1, 0, 0, 0, 0)) == 8    # host-only plan
    assert _err(lambda: qtam.qtam_frame_operator(p.handle, 0b110, p.Nr)) == 1  # plane 1, 2 do not exist
    assert _err(lambda: qtam.qtam_workspace_size(p.handle, -1)) == 1


def test_window_argument_errors_and_variants():
    base = (4096, 16384, (8,), 20, 1024, 64)
    assert _err(lambda: qtam.Plan(*base, window="kaiser", window_param=-1.0, device=-1)) == 1
    assert _err(lambda: qtam.Plan(*base, window="tukey", window_param=1.5, device=-1)) == 1
    assert _err(lambda: qtam.Plan(*base, window="planck", window_param=float("nan"), device=-1)) == 1
    d = qtam.make_desc(*base)
    d.window = 7
    assert _err(lambda: qtam.qtam_plan(d, -1)) == 1
    # compile-time row variants: the bisquare kernels evaluate the window formula; other windows use the
    # variants built for window tables
    b = qtam.Plan(4096.0, 262144, (4, 8, 16, 32, 64), 20.0, 2048.0, 128, device=-1)
    h = qtam.Plan(4096.0, 262144, (4, 8, 16, 32, 64), 20.0, 2048.0, 128, window="hann", device=-1)
    vb, vh = qtam.qtam_plan_variants(b.handle), qtam.qtam_plan_variants(h.handle)
    assert len(vb) > 2 and b.info["row_variant"] >= 0
    # non-bisquare windows: the variants built for window tables (FP32 envelopes) only
    assert vh[0] == -1 and 2 <= len(vh) < len(vb) and set(vh) <= set(vb) and h.info["row_variant"] == vh[1]
    assert _err(lambda: qtam.qtam_plan_set_variant(h.handle, [v for v in vb if v not in vh][0])) == 1
    hb = qtam.Plan(4096.0, 262144, (4, 8), 20.0, 2048.0, 128, window="hann", envelope="bf16", device=-1)
    assert qtam.qtam_plan_variants(hb.handle) == [-1]                    # 16-bit envelopes: runtime engine
    m = qtam.Plan(4096.0, 262144, (4, 8), 20.0, 2048.0, 128, window=("bisquare", "tukey"), window_param=(0, 0.5),
                  device=-1)
    assert qtam.qtam_plan_variants(m.handle) == vh
    assert _err(lambda: qtam.Plan(*base[:2], (8, 16), *base[3:], window=("hann", "tukey"),
                                  window_param=(0.0, 2.0), device=-1)) == 1
    with pytest.raises(ValueError):
        qtam.Plan(*base[:2], (8, 16), *base[3:], window=("hann",), device=-1)


def test_stream_argument_errors():
    """Streaming (overlap-save) layout rules are checked before anything is
    allocated: hop and guard on the column quantum N / gcd(N, M)."""
    p = qtam.Plan(256.0, 1024, (6.0, 12.0), 2.0, 100.0, 20, n_out=96, device=-1)   # quantum 32
    for hop in (500, 2048, 544, -32):
        assert _err(lambda: qtam.qtam_stream_create(p.handle, hop, 4)) == 1
    assert _err(lambda: qtam.qtam_stream_create(p.handle, 512, 0)) == 1
    assert _err(lambda: qtam.qtam_stream_create(p.handle, 512, 4)) == 8        # host-only plan
    assert _err(lambda: qtam.qtam_stream_create(p.handle, 0, 4)) == 8          # default hop is valid


def test_tensor_short_dft_options():
    base = (4096.0, 32768, (8.0, 16.0), 20.0, 2048.0, 64)
    p = qtam.Plan(*base, n_out=8192, short_dft="tensor", device=-1)
    assert p.info["short_dft"] == 1 and p.M == 8192
    vs = qtam.qtam_plan_variants(p.handle)                 # runtime engine + the compile-time inverse variants
    assert vs[0] == -1 and len(vs) >= 4
    assert all(qtam.qtam_variant_describe(v)["name"].startswith("8192:") for v in vs[1:])
    assert qtam.Plan(*base, device=-1).info["short_dft"] == 0
    assert _err(lambda: qtam.Plan(*base, short_dft="tensor", device=-1)) == 2                    # M = 600
    assert _err(lambda: qtam.Plan(*base, n_out=8192, short_dft="tensor", compute="f64", device=-1)) == 2
    d = qtam.make_desc(*base)
    d.short_dft = 5
    assert _err(lambda: qtam.qtam_plan(d, -1)) == 1


def test_short_dft_auto_picks_the_engine_per_plan():
    """AUTO: tensor cores where their BF16 rounding is inside the plan's
    accuracy class (M = 8192, F32 compute, BF16 envelopes, no dense mode),
    CUDA cores otherwise; never an error where the CUDA cores serve."""
    base = (4096.0, 32768, (8.0, 16.0), 20.0, 2048.0, 64)
    auto = lambda **kw: qtam.Plan(*base, short_dft="auto", device=-1, **kw).info["short_dft"]
    assert auto(n_out=8192, envelope="bf16") == 1
    assert auto(n_out=8192) == 0                                # FP32 envelopes: FP32-accurate engine
    assert auto(n_out=8192, envelope="f16") == 0                # FP16 storage is more accurate than BF16 operands
    assert auto(envelope="bf16") == 0                           # M = 600: no tensor-core length
    assert auto(n_out=8192, compute="f64", envelope="f64") == 0
    assert auto(n_out=8192, envelope="bf16", remodulate=True) == 0


def test_dense_mode_options():
    base = (4096.0, 8192, (8.0,), 20.0, 2048.0, 32)
    p = qtam.Plan(*base, stopband_eps=1e-6, p_floor_rel=0.0, device=-1)
    assert p.M == 4320 and p.info["max_window"] == 4097            # smallest 2^a 3^b 5^c >= N/2 + 1
    assert p.info["stopband_eps"] == 1e-6 and p.info["remodulate"] == 0
    assert p.info["kept_bins"] == 4097 and p.info["band_bins"] == 32 * 4097   # P > 0 on every bin
    vs = qtam.qtam_plan_variants(p.handle)                          # runtime engine + the dense variants
    assert vs[0] == -1 and len(vs) == 4 and p.info["row_variant"] == vs[1]
    names = [qtam.qtam_variant_describe(v)["name"] for v in vs[1:]]
    assert all(n.startswith("4320:") for n in names)
    assert qtam.qtam_plan_variants(qtam.Plan(*base, stopband_eps=1e-6, n_out=4800, device=-1).handle) == [-1]
    assert qtam.qtam_plan_variants(qtam.Plan(*base, stopband_eps=1e-6, envelope="bf16", device=-1).handle) == vs
    assert qtam.qtam_plan_variants(qtam.Plan(*base, stopband_eps=1e-6, compute="f64", device=-1).handle) == [-1]
    r = qtam.Plan(*base, remodulate=True, n_out=4320, device=-1)     # carrier alone: dense kernels too
    assert r.info["remodulate"] == 1 and r.info["stopband_eps"] == 0.0
    assert len(qtam.qtam_plan_variants(r.handle)) == 4
    assert _err(lambda: qtam.Plan(*base, stopband_eps=1e-6, n_out=4000, device=-1)) == 3    # aliasing
    assert _err(lambda: qtam.Plan(*base, stopband_eps=-1.0, device=-1)) == 1
    assert _err(lambda: qtam.Plan(*base, n_out=8192, stopband_eps=1e-6, short_dft="tensor", device=-1)) == 2
    d = qtam.make_desc(*base)
    d.remodulate = 2
    assert _err(lambda: qtam.qtam_plan(d, -1)) == 1
    q = qtam.Plan(*base, device=-1)
    assert _err(lambda: qtam.qtam_inverse_single_tile(q.handle, 0, 1, 0, 0, 0, 0, 0, 0)) == 8   # host-only plan


def test_f64_defaults():
    p = qtam.Plan(4096, 16384, (8,), 20, 1024, 64, compute="f64", device=-1)
    assert p.info["p_floor_rel"] == 0.0 and p.info["envelope_bytes_per_segment"] == 64 * 250 * 16
    g = O.geometry(4096, 16384, (8,), 20, 1024, 64)
    assert p.info["kept_bins"] == int((O.frame_operator(g) > 0).sum())


def test_binding_rejects_mismatched_tensors():
    """The ABI sees raw pointers, so the binding checks every tensor's shape,
    dtype, device and layout before a call."""
    torch = pytest.importorskip("torch")
    p = qtam.Plan(64.0, 512, (4.0, 8.0), 3.0, 30.0, 12, device=-1)
    with pytest.raises(ValueError):
        p.envelopes(torch.zeros(p.Nr, dtype=torch.complex64))            # 1-D, CPU
    with pytest.raises(ValueError):
        p.forward(torch.zeros((2, p.N), dtype=torch.float32))             # CPU tensor
    with pytest.raises(ValueError):
        p.inverse(torch.zeros((1, p.P, p.K, p.M + 1), dtype=torch.complex64))
    with pytest.raises(ValueError):
        p.synthesize(torch.zeros((1, p.Nr), dtype=torch.complex128))


def test_batched_workspace_is_largest_group():
    a = qtam.Plan(4096.0, 4096, (8.0, 16.0, 32.0), 20.0, 2048.0, 128, device=-1)
    b = qtam.Plan(4096.0, 32768, (8.0, 16.0, 32.0), 20.0, 2048.0, 128, device=-1)
    ga = (a.handle, 0, 0, 7)
    gb = (b.handle, 0, 0, 3)
    want = max(qtam.qtam_workspace_size(a.handle, 7), qtam.qtam_workspace_size(b.handle, 3))
    assert qtam.qtam_batched_workspace_size([ga, gb]) == want
    with pytest.raises(qtam.QtamError):
        qtam.qtam_forward_batched([ga, gb], 0, want, stream=0)   # host-only plans cannot run
    with pytest.raises(qtam.QtamError):
        qtam.qtam_batched_workspace_size([(a.handle, 0, 0, -1)])


def test_tuned_defaults_per_length():
    """Bisquare plans at M = 1200, 600, 300, 150 start on their preferred
    balanced-radix variant, M = 2400 on its 160-thread one and M = 8192 on
    its four-stage one; a window-table
    plan of the same length keeps the first table-capable variant; M = 4800
    keeps its first registered one."""
    want = {32: "2400:16, 10, 15 rows/blk 2^0 minblk 6 threads 160",
            16: "1200:10, 12, 10 rows/blk 2^0 minblk 8", 8: "600:25, 24 rows/blk 2^1 minblk 8",
            4: "300:15, 20 rows/blk 2^1 minblk 12", 2: "150:10, 15 rows/blk 2^3 minblk 4"}
    for dur, name in want.items():
        p = qtam.Plan(4096.0, 4096 * dur, (8.0, 16.0, 32.0), 20.0, 2048.0, 128, device=-1)
        assert qtam.qtam_variant_describe(p.info["row_variant"])["name"] == name
        assert p.info["row_variant"] in qtam.qtam_plan_variants(p.handle)
        h = qtam.Plan(4096.0, 4096 * dur, (8.0, 16.0, 32.0), 20.0, 2048.0, 128, window="hann", device=-1)
        assert h.info["row_variant"] == qtam.qtam_plan_variants(h.handle)[1]
    b = qtam.Plan(4096.0, 262144, (4, 8, 16, 32, 64), 20.0, 2048.0, 128, device=-1)
    assert qtam.qtam_variant_describe(b.info["row_variant"])["name"] == "4800:16, 20, 15 rows/blk 2^0 minblk 4"
    # M = 8192 on CUDA cores: the four-stage sequence at two blocks per SM
    e = qtam.Plan(4096.0, 262144, (4, 8, 16, 32, 64), 20.0, 2048.0, 128, n_out=8192, device=-1)
    assert qtam.qtam_variant_describe(e.info["row_variant"])["name"] == "8192:16, 8, 8, 8 rows/blk 2^0 minblk 2"
