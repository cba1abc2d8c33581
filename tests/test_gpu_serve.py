"""Serving on the GPU: each request's result is the same served alone and in
a mix of concurrent requests (continuous batching over several streams), and
matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import serve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, FS = 32768, 4096.0


def fresh(r):
    return serve.Request(r.rid, r.x, r.q, r.kind, r.row_gain, r.fs)


@pytest.fixture(scope="module")
def requests():
    reqs = [serve.make_request(i, 1000 + i, n=N, fs=FS, inverse_frac=0.4) for i in range(10)]
    assert {r.kind for r in reqs} == {"forward", "inverse"}
    return reqs


def test_result_same_alone_and_in_mix(requests):
    ex = serve.GpuExecutor(slots=3)
    solo = {}
    for r in requests:
        s = serve.Server(ex, hbm_budget_bytes=40 * 2**30)
        rr = fresh(r)
        s.submit(rr)
        s.drain()
        assert not s.rejected, s.rejected[0].error if s.rejected else ""
        solo[r.rid] = rr.result
    s = serve.Server(ex, hbm_budget_bytes=40 * 2**30, max_batch_requests=4)
    arrivals = np.zeros(len(requests))       # all at once: same (Q, kind) requests share batches
    mix = [fresh(r) for r in requests]
    st = serve.run_stream(s, mix, arrivals)
    assert st["completed"] == len(requests) and st["rejected"] == 0
    assert st["batches"] < len(requests)
    for r in mix:
        a, b = solo[r.rid], r.result
        if r.kind == "forward":
            assert np.array_equal(a, b)
        else:
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)


def test_served_results_match_oracle(requests):
    ex = serve.GpuExecutor(slots=2)
    s = serve.Server(ex, hbm_budget_bytes=40 * 2**30)
    mix = [fresh(r) for r in requests[:4]]
    serve.run_stream(s, mix, np.zeros(len(mix)))
    for r in mix:
        g = O.geometry(FS, N, (r.q,), 20.0, 2048.0, 128)
        for c in (0, 2):
            x = r.x[c].astype(np.float64)
            Y = O.forward(g, x)
            if r.kind == "forward":
                got = r.result[c].astype(np.complex128)
                assert np.linalg.norm(got - Y) < 1e-6 * np.linalg.norm(Y)
            else:
                Ym = Y * r.row_gain[c][None, :, None]
                ref = O.inverse(g, Ym, tau=1e-6)
                assert np.linalg.norm(r.result[c] - ref) < 1e-5 * np.linalg.norm(ref)


def test_tiny_budget_serialises_but_completes(requests):
    ex = serve.GpuExecutor(slots=4)
    one = ex.nbytes(ex.key(requests[0]), requests[0].x.shape[0])
    s = serve.Server(ex, hbm_budget_bytes=int(one * 1.5))
    mix = [fresh(r) for r in requests[:5]]
    st = serve.run_stream(s, mix, np.zeros(len(mix)))
    assert st["completed"] + st["rejected"] == 5 and s.peak_bytes <= one * 1.5


def test_batch_device_bytes_within_its_charge(requests):
    """The bytes a batch holds on the device while in flight (input, envelopes,
    long-FFT workspace, inverse gains and output) stay within what admission
    charged for it (torch rounds each allocation up to 512 bytes)."""
    ex = serve.GpuExecutor(slots=1)
    for r in requests[:4]:
        key = ex.key(r)
        nb = ex.nbytes(key, r.x.shape[0])
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        b = serve.Batch(key, [fresh(r)], nb)
        ex.launch(b, 0)
        held = torch.cuda.memory_allocated() - before
        ex.collect(b)
        assert 0 < held <= nb + 5 * 512, (r.kind, held, nb)
