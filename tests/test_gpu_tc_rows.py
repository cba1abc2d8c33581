"""Tensor-core short DFT (M = 8192 as a 64 x 128 four-step on tcgen05 with BF16
operands), forward and inverse rows, against the FP64 oracle.

Tolerance from the arithmetic: BF16 keeps 8 significand bits (unit roundoff
u = 2^-9 = 2e-3).  Forward: the windowed band, the DFT matrices and the
twiddled intermediate are each rounded once; inverse: the envelopes, the DFT
matrices and the twiddled intermediate.  FP32 accumulation adds nothing
comparable, so the relative Frobenius error is a few 1e-3: bound 1e-2; every
coefficient within 3e-2 of the largest."""
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
    with M = 8192: every row against the oracle, the tensor-core inverse of
    the tensor-core envelopes against the oracle's projection, 16-bit
    envelopes."""
    fs, N, qs = 4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0)
    t0 = qtam.qtam_tc_status()
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, 128, n_out=8192, short_dft="tensor", device=0)
    g = O.geometry(fs, N, qs, 20.0, 2048.0, 128, n_out=8192)
    x = np.stack([synth.coloured_chirp_segment(s) for s in range(2)])
    y = p.forward(torch.from_numpy(x).cuda())
    Y = _np(y)
    for b in range(2):
        ref = O.forward(g, x[b].astype(np.float64))
        big = np.max(np.abs(ref))
        for a in range(g.P):
            for k in range(g.K):
                assert _rel(Y[b, a, k], ref[a, k]) < 1e-2, (b, a, k)
        assert np.max(np.abs(Y[b] - ref)) <= 3e-2 * big
    xh = p.inverse(y).cpu().numpy().astype(np.float64)
    for b in range(2):
        assert _rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < 2e-2
    for env in ("bf16", "f16"):
        q = qtam.Plan(fs, N, qs, 20.0, 2048.0, 128, n_out=8192, short_dft="tensor", envelope=env, device=0)
        Yq = _np(q.forward(torch.from_numpy(x).cuda()))
        assert _rel(Yq, Y) < 1e-2
    assert qtam.qtam_tc_status() == t0


def _masked_planes(mask, P):
    return None if mask == 0 else [i for i in range(P) if (mask >> i) & 1]


@pytest.mark.parametrize("K,qs,B,window,prm,mask", [
    (128, (8.0, 16.0, 32.0), 2, "bisquare", 0.0, 0),
    (65, (8.0,), 1, "bisquare", 0.0, 0),              # odd number of rows: the last pair has one
    (64, (8.0, 16.0, 32.0), 2, "hann", 0.0, 0b101),   # window table, plane subset (row list)
    (32, (4.0,), 3, "kaiser", 6.0, 0),
])
def test_tensor_accumulate_matches_oracle(K, qs, B, window, prm, mask):
    """The inverse rows alone: A[f] = sum_k W_k(f) sqrt(N/M) FFT_M(Y_k) on the
    tensor cores, fed the oracle's own envelopes, against the oracle's A."""
    fs, N = 4096.0, 32768
    t0 = qtam.qtam_tc_status()
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, n_out=8192, short_dft="tensor", window=window, window_param=prm,
                  device=0)
    g = O.geometry(fs, N, qs, 20.0, 2048.0, K, n_out=8192, window=window, window_param=prm)
    x = [synth.glitchy_segment(80 + b, N, fs, chirp=True).astype(np.float64) for b in range(B)]
    Y = np.stack([O.forward(g, xb) for xb in x])
    A = p.accumulate(torch.from_numpy(Y.astype(np.complex64)).cuda(), plane_mask=mask)
    torch.cuda.synchronize()
    A = A.cpu().numpy().astype(np.complex128)
    planes = _masked_planes(mask, len(qs))
    for b in range(B):
        ref = O.accumulate(g, Y[b], planes)
        assert _rel(A[b], ref) < 1e-2
        assert np.max(np.abs(A[b] - ref)) <= 3e-2 * np.max(np.abs(ref))
        assert _rel(A[b], ref) > 1e-5                  # BF16 operands: the tensor-core rows ran
    assert qtam.qtam_tc_status() == t0


def test_tensor_inverse_envelope_dtypes_and_unaligned_pointer():
    """16-bit envelopes go through the tensor-core inverse too; an envelope
    pointer that is not 16-byte aligned takes the CUDA-core rows (FP32
    accuracy)."""
    fs, N, qs, K = 4096.0, 32768, (8.0, 16.0), 64
    g = O.geometry(fs, N, qs, 20.0, 2048.0, K, n_out=8192)
    x = synth.glitchy_segment(91, N, fs, chirp=True).astype(np.float64)
    Y = O.forward(g, x)[None]
    ref = O.accumulate(g, Y[0])
    for env, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, n_out=8192, short_dft="tensor", envelope=env, device=0)
        y = torch.from_numpy(np.stack([Y.real, Y.imag], axis=-1).astype(np.float32)).to(dt).cuda()
        A = p.accumulate(y).cpu().numpy().astype(np.complex128)[0]
        assert _rel(A, ref) < 1e-2, env
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, n_out=8192, short_dft="tensor", device=0)
    flat = torch.zeros(Y.size + 1, dtype=torch.complex64, device="cuda")
    y_off = flat[1:].view(Y.shape)                     # 8 bytes past a 16-byte boundary
    assert y_off.data_ptr() % 16 == 8
    y_off.copy_(torch.from_numpy(Y.astype(np.complex64)))
    A = p.accumulate(y_off).cpu().numpy().astype(np.complex128)[0]
    assert _rel(A, ref) < 1e-5


def test_short_dft_auto_engine_and_accuracy():
    """short_dft = AUTO takes the tensor cores for an M = 8192 plan with BF16
    envelopes (their rounding is inside that plan's accuracy class: bound
    1e-2 against the oracle) and the CUDA cores for FP32 envelopes (FP32
    bound 1e-6), forward and round trip."""
    fs, N, qs, K = 4096.0, 32768, (8.0, 16.0), 64
    g = O.geometry(fs, N, qs, 20.0, 2048.0, K, n_out=8192)
    x = np.stack([synth.glitchy_segment(70 + b, N, fs, chirp=True) for b in range(2)])
    xd = torch.from_numpy(x).cuda()
    refs = [O.forward(g, x[b].astype(np.float64)) for b in range(2)]
    for env, engine, bound, rt in (("bf16", 1, 1e-2, 2e-2), ("f32", 0, 1e-6, 1e-5)):
        p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, n_out=8192, short_dft="auto", envelope=env, device=0)
        assert p.info["short_dft"] == engine, env
        y = p.forward(xd)
        Y = _np(y)
        for b in range(2):
            assert _rel(Y[b], refs[b]) < bound, env
        xh = p.inverse(y).cpu().numpy().astype(np.float64)
        for b in range(2):
            assert _rel(xh[b], O.projection(g, x[b].astype(np.float64), tau=p.info["p_floor_rel"])) < rt, env
