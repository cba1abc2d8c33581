"""Tensor-core short DFT (M = 8192 as a 64 x 128 four-step on tcgen05 with BF16
operands) against the FP64 oracle.

Tolerance from the arithmetic: BF16 keeps 8 significand bits (unit roundoff
u = 2^-9 = 2e-3).  The windowed band, the DFT matrices and the twiddled
intermediate are each rounded once, and FP32 accumulation adds nothing
comparable, so the envelopes' relative Frobenius error is a few 1e-3: bound
1e-2; every coefficient within 3e-2 of the segment's largest."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(y):
    torch.cuda.synchronize()
    if y.dtype in (torch.bfloat16, torch.float16):
        a = y.float().cpu().numpy().astype(np.float64)
        return a[..., 0] + 1j * a[..., 1]
    return y.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("K,qs,B,window,prm", [
    (128, (8.0, 16.0, 32.0), 2, "bisquare", 0.0),
    (65, (8.0,), 1, "bisquare", 0.0),          # odd number of rows: the last pair has one
    (64, (8.0, 16.0), 1, "hann", 0.0),         # window table path
    (32, (4.0,), 3, "kaiser", 6.0),
])
def test_tensor_forward_matches_oracle(K, qs, B, window, prm):
    fs, N = 4096.0, 32768
    t0 = qtam.qtam_tc_status()
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, n_out=8192, short_dft="tensor", window=window, window_param=prm,
                  device=0)
    g = O.geometry(fs, N, qs, 20.0, 2048.0, K, n_out=8192, window=window, window_param=prm)
    x = np.stack([synth.glitchy_segment(60 + b, N, fs, chirp=True) for b in range(B)])
    Y = _np(p.forward(torch.from_numpy(x).cuda()))
    for b in range(B):
        ref = O.forward(g, x[b].astype(np.float64))
        assert _rel(Y[b], ref) < 1e-2
        assert np.max(np.abs(Y[b] - ref)) <= 3e-2 * np.max(np.abs(ref))
    assert qtam.qtam_tc_status() == t0              # no tensor-core wait ran out


def test_tensor_forward_full_size_and_roundtrip():
    """64 s segments (N = 2^18, Q {4..64} x 128 rows, largest window 4693 bins)
    with M = 8192: sampled rows against the oracle, the CUDA-core inverse of the
    tensor-core envelopes against the oracle's projection, 16-bit envelopes."""
    fs, N, qs = 4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0)
    t0 = qtam.qtam_tc_status()
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, 128, n_out=8192, short_dft="tensor", device=0)
    g = O.geometry(fs, N, qs, 20.0, 2048.0, 128, n_out=8192)
    x = np.stack([synth.coloured_chirp_segment(s) for s in range(2)])
    y = p.forward(torch.from_numpy(x).cuda())
    Y = _np(y)
    rows = [(0, 0), (0, 127), (1, 64), (2, 5), (3, 100), (4, 127)]
    for b in range(2):
        X = O.spectrum(x[b].astype(np.float64))
        big = max(np.max(np.abs(O.forward_row(g, X, a, k))) for a, k in rows)
        for a, k in rows:
            ref = O.forward_row(g, X, a, k)
            assert _rel(Y[b, a, k], ref) < 1e-2, (a, k)
            assert np.max(np.abs(Y[b, a, k] - ref)) <= 3e-2 * big
    xh = p.inverse(y).cpu().numpy().astype(np.float64)
    for b in range(2):
        assert _rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < 2e-2
    for env in ("bf16", "f16"):
        q = qtam.Plan(fs, N, qs, 20.0, 2048.0, 128, n_out=8192, short_dft="tensor", envelope=env, device=0)
        Yq = _np(q.forward(torch.from_numpy(x).cuda()))
        assert _rel(Yq, Y) < 1e-2
    assert qtam.qtam_tc_status() == t0
