"""qtam_forward_noalloc -- the forward transform for callers that cannot
allocate device memory when they call it (real-time loops, host callbacks,
plug-ins whose host owns all device memory) -- must give the same envelopes
as qtam_forward with a caller workspace.

Kept in its own file, collected last, so a run that stops at the first
failure has already run every other test.  It makes its own plan and inputs,
so it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_FROB = 1e-6   # relative Frobenius bound used by the FP32 parity tests
FWD_ELEM = 1e-5   # element-wise bound, relative to the largest coefficient


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_forward_noalloc_matches_forward_on_two_calls():
    p = qtam.Plan(4096.0, 65536, (8.0, 16.0), 20.0, 2048.0, 64, device=0)
    B = 4
    st = torch.cuda.current_stream()
    for call, seed in enumerate((11, 12)):       # two calls in a row, different inputs
        x = torch.from_numpy(np.stack([synth.glitchy_segment(seed * 10 + b, p.N, 4096.0, chirp=True)
                                       for b in range(B)])).cuda()
        y_ref = p.forward(x)                     # existing entry point, caller workspace
        y = p.envelope_tensor(B)
        y.fill_(float("nan"))
        qtam.qtam_forward_noalloc(p.handle, x, B, y, st)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(y)).all(), f"call {call}: output not fully written"
        assert _rel(y, y_ref) < FWD_FROB, f"call {call}"
        assert float((y - y_ref).abs().max()) <= FWD_ELEM * float(y_ref.abs().max()), f"call {call}"


def test_forward_noalloc_rejects_batches_beyond_its_scratch():
    p = qtam.Plan(4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128, device=0)
    B = 20                                       # needs about 42 MB of scratch, above the fixed 32 MiB
    assert qtam.qtam_workspace_size(p.handle, B) > 32 * 2**20
    x = torch.zeros((B, p.N), dtype=torch.float32, device="cuda")
    y = p.envelope_tensor(B)
    with pytest.raises(qtam.QtamError) as e:
        qtam.qtam_forward_noalloc(p.handle, x, B, y)
    assert e.value.status == 9 and "32" in str(e.value)
    # a batch that fits still runs
    qtam.qtam_forward_noalloc(p.handle, x[:2], 2, y[:2])
    torch.cuda.synchronize()
    assert float(y[:2].abs().max()) == 0.0
