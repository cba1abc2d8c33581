"""Serving loop logic on the host: admission by an HBM budget, continuous
batching, rejection, and failure injection (a fake executor raises on the
host; no GPU is involved)."""
import threading
import time

import numpy as np
import pytest

from paper_2603_29785_gb300 import serve


class FakeExecutor(serve.Executor):
    def __init__(self, slots=2, per_segment=100, polls=2, fail_rids=()):
        self.slots = slots
        self.per = per_segment
        self.polls = polls
        self.fail = set(fail_rids)
        self.launched = []

    def nbytes(self, key, n):
        return n * self.per

    def launch(self, b, slot):
        if any(r.rid in self.fail for r in b.requests):
            raise RuntimeError("injected launch failure")
        b.handle = [0]
        self.launched.append((slot, [r.rid for r in b.requests]))

    def poll(self, b):
        b.handle[0] += 1
        return b.handle[0] >= self.polls

    def collect(self, b):
        for r in b.requests:
            r.result = r.x * 2


def req(rid, q=8.0, kind="forward", c=1, n=16):
    return serve.Request(rid, np.full((c, n), rid, np.float32), q, kind)


def test_budget_caps_bytes_in_flight():
    ex = FakeExecutor(slots=4, per_segment=100)
    s = serve.Server(ex, hbm_budget_bytes=250, max_batch_requests=1)
    for i in range(10):
        s.submit(req(i))
    s.drain(timeout=5)
    assert len(s.done) == 10 and not s.rejected
    assert s.peak_bytes <= 250
    assert all(np.array_equal(r.result, r.x * 2) for r in s.done)


def test_same_key_requests_share_a_batch():
    ex = FakeExecutor(slots=1)
    s = serve.Server(ex, hbm_budget_bytes=10**9, max_batch_requests=8)
    for i in range(6):
        s.submit(req(i, q=8.0))
    s.submit(req(6, q=16.0))
    s.drain(timeout=5)
    assert ex.launched[0][1] == [0, 1, 2, 3, 4, 5]
    assert ex.launched[1][1] == [6]


def test_oversized_request_is_rejected_others_served():
    ex = FakeExecutor(per_segment=100)
    s = serve.Server(ex, hbm_budget_bytes=150)
    s.submit(req(0, c=2))          # 200 bytes > budget
    s.submit(req(1))
    s.drain(timeout=5)
    assert [r.rid for r in s.rejected] == [0] and "budget" in s.rejected[0].error
    assert [r.rid for r in s.done] == [1]


def test_injected_launch_failure_fails_only_its_batch():
    ex = FakeExecutor(fail_rids={3})
    s = serve.Server(ex, hbm_budget_bytes=10**9, max_batch_requests=1)
    for i in range(6):
        s.submit(req(i))
    s.drain(timeout=5)
    assert [r.rid for r in s.rejected] == [3] and "injected" in s.rejected[0].error
    assert sorted(r.rid for r in s.done) == [0, 1, 2, 4, 5]


def test_arrivals_during_work_join_later_batches_and_stats():
    ex = FakeExecutor(slots=1, polls=40)          # slow device: arrivals pile up behind it
    s = serve.Server(ex, hbm_budget_bytes=10**9, max_batch_requests=4)
    stop = threading.Event()

    def producer():
        for i in range(40):
            s.submit(req(i, q=8.0 + (i % 2) * 8))
            time.sleep(0.0005)
        stop.set()

    th = threading.Thread(target=producer)
    th.start()
    while not stop.is_set() or s.pending() or s.inflight:
        if not s.step():
            time.sleep(0.0001)
    th.join()
    st = s.stats()
    assert st["completed"] == 40 and st["rejected"] == 0
    assert st["batches"] < 40                       # requests were batched together
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]


def test_poisson_arrivals_and_request_recipe():
    a = serve.poisson_arrivals(200.0, 2.0, seed=1)
    assert 300 < a.size < 500 and np.all(np.diff(a) > 0)
    kinds = [serve.make_request(i, i, n=4096, rows=16).kind for i in range(40)]
    assert 0 < kinds.count("inverse") < 20
    r = next(serve.make_request(i, i, n=4096, rows=16) for i in range(100)
             if serve.make_request(i, i, n=4096, rows=16).kind == "inverse")
    zeroed = (r.row_gain == 0).mean(axis=1)
    assert np.all((zeroed >= 0.05) & (zeroed <= 0.35)) and r.x.shape == (3, 4096)


def test_batch_charge_counts_the_long_fft_workspace():
    """The HBM charge of a batch is the sum of the tensors it allocates, the
    long-FFT workspace included (qtam_workspace_size of the batch), for every
    batch size and both request kinds (host-only plan, no GPU)."""
    from paper_2603_29785_gb300 import qtam
    p = qtam.Plan(4096.0, 32768, (8.0,), 20.0, 2048.0, 128, device=-1)
    for kind in ("forward", "inverse"):
        for B in (1, 3, 8):
            a = serve.batch_allocations(p, kind, B)
            assert a["workspace"] == qtam.qtam_workspace_size(p.handle, B) > 0
            assert a["y"] == B * p.info["envelope_bytes_per_segment"]
            assert set(a) == ({"x", "y", "workspace"} | ({"gain", "xh"} if kind == "inverse" else set()))
