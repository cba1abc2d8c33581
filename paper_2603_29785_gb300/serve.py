"""Continuous-batching request loop for QTAM transforms on one GPU.

Requests (strain windows on one or more channels, a Q value, and either
"forward" -> envelopes, or "inverse" -> the reconstruction from the envelopes
with some rows zeroed) arrive at any time.  The server loop

  1. admits pending requests oldest-first while the bytes they need on the
     device fit the HBM budget and an execution slot (stream) is free,
  2. groups the admitted requests by (plan, kind) into one batch -- requests
     that arrive while other batches run join the next batch --
  3. launches each batch asynchronously on its own stream (copy in, QTAM
     kernels, copy out), so batches overlap on the device,
  4. polls completion events, hands results back and frees budget and slot.

Plans (geometry, twiddles, normalisers) stay resident in a PlanCache.  The
executor interface separates the scheduling logic from the device work so
admission, batching and failure handling are testable without a GPU.
"""
from __future__ import annotations

import collections
import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    x: np.ndarray                   # [C, N] float32, one row per channel
    q: float
    kind: str = "forward"           # "forward" | "inverse"
    row_gain: np.ndarray | None = None   # [C, K] gains for "inverse" (0 = row zeroed)
    fs: float = 4096.0
    t_arrival: float = 0.0
    t_admit: float | None = None
    t_done: float | None = None
    result: np.ndarray | None = None
    error: str | None = None

    @property
    def samples(self) -> int:
        return int(self.x.shape[0] * self.x.shape[1])

    @property
    def latency(self) -> float | None:
        return None if self.t_done is None else self.t_done - self.t_arrival


@dataclass
class Batch:
    key: tuple
    requests: list
    nbytes: int
    handle: object = None


class Executor:
    """Device work for one batch: bytes it needs, async launch, poll, collect."""

    slots = 1

    def key(self, req: Request) -> tuple:
        return (req.fs, req.x.shape[1], req.q, req.kind)

    def nbytes(self, key: tuple, n_segments: int) -> int:
        raise NotImplementedError

    def launch(self, batch: Batch, slot: int):
        raise NotImplementedError

    def poll(self, batch: Batch) -> bool:
        raise NotImplementedError

    def collect(self, batch: Batch) -> None:
        raise NotImplementedError


_ENV_BYTES = {"f32": 8, "f64": 16, "bf16": 4, "f16": 4}


def batch_allocations(plan, kind: str, n_segments: int) -> dict:
    """Device bytes one batch of `n_segments` allocates, per tensor: the input
    samples, the envelopes, the long-FFT workspace (qtam_workspace_size), and
    for an inverse the row gains and the reconstruction.  The executor charges
    their sum against the HBM budget and allocates exactly these tensors."""
    from . import qtam
    B = int(n_segments)
    out = {"x": B * plan.N * 4,
           "y": B * plan.P * plan.K * plan.M * _ENV_BYTES[plan.envelope],
           "workspace": qtam.qtam_workspace_size(plan.handle, B)}
    if kind == "inverse":
        out["gain"] = B * plan.P * plan.K * 4
        out["xh"] = B * plan.N * 4
    return out


class GpuExecutor(Executor):
    """Runs batches with the library's C entry points on `slots` CUDA streams."""

    def __init__(self, f_min=20.0, f_max=2048.0, rows_per_plane=128, slots=4, device=0, tune=False):
        import torch

        from . import batch as qbatch

        self.torch = torch
        self.device = device
        self.slots = slots
        self.cache = qbatch.PlanCache((1.0,), f_min, f_max, rows_per_plane, device=device)
        self.plans = {}
        self.K = rows_per_plane
        self.f_min, self.f_max = f_min, f_max
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        # per-slot pinned staging (input samples, output samples or envelopes),
        # grown on demand and reused: a slot's buffers are free again once its
        # batch has been collected, and pinning per batch would cost milliseconds
        self.pin_in = [None] * slots
        self.pin_out = [None] * slots
        self.tune = tune

    def plan(self, fs, N, q):
        from . import qtam
        key = (float(fs), int(N), float(q))
        p = self.plans.get(key)
        if p is None:
            p = qtam.Plan(fs, N, (q,), self.f_min, self.f_max, self.K, device=self.device)
            self.plans[key] = p
        return p

    def nbytes(self, key, n_segments):
        fs, N, q, kind = key
        return sum(batch_allocations(self.plan(fs, N, q), kind, n_segments).values())

    def _pinned(self, pool, slot, shape, dtype):
        """A pinned host tensor of `shape` and `dtype` on the slot's reusable bytes."""
        t = self.torch
        n = int(np.prod(shape)) * t.empty((), dtype=dtype).element_size()
        buf = pool[slot]
        if buf is None or buf.numel() < n:
            buf = t.empty(max(n, 16), dtype=t.uint8).pin_memory()
            pool[slot] = buf
        return buf[:n].view(dtype).view(shape)

    def launch(self, batch, slot):
        from . import qtam
        t = self.torch
        fs, N, q, kind = batch.key
        p = self.plan(fs, N, q)
        st = self.streams[slot]
        B = sum(r.x.shape[0] for r in batch.requests)
        dev = f"cuda:{self.device}"
        x_host = self._pinned(self.pin_in, slot, (B, N), t.float32)
        xs = x_host.numpy()
        o = 0
        for r in batch.requests:
            xs[o:o + r.x.shape[0]] = r.x
            o += r.x.shape[0]
        with t.cuda.stream(st):
            # every device tensor of the batch is allocated here, on the batch's
            # stream, and released when the batch is collected: the bytes in
            # flight are exactly what admission charged (batch_allocations)
            x = x_host.to(dev, non_blocking=True)
            y = p.envelope_tensor(B)
            ws = t.empty(max(qtam.qtam_workspace_size(p.handle, B), 256), dtype=t.uint8, device=dev)
            qtam.qtam_forward(p.handle, x, B, y, ws, ws.numel(), st)
            if kind == "inverse":
                g = np.concatenate([r.row_gain if r.row_gain is not None else np.ones((r.x.shape[0], p.K), np.float32)
                                    for r in batch.requests]).astype(np.float32).reshape(B, 1, p.K)
                gain = t.from_numpy(g).pin_memory().to(dev, non_blocking=True)
                qtam.qtam_scale_rows(p.handle, y, B, gain, st)
                xh = t.empty((B, N), dtype=t.float32, device=dev)
                qtam.qtam_inverse(p.handle, y, B, 0, xh, ws, ws.numel(), st)
                out = self._pinned(self.pin_out, slot, (B, N), t.float32)
                out.copy_(xh, non_blocking=True)
                keep = (x, y, ws, gain, xh)
            else:
                out = self._pinned(self.pin_out, slot, tuple(y.shape), y.dtype)
                out.copy_(y, non_blocking=True)
                keep = (x, y, ws)
            ev = t.cuda.Event()
            ev.record(st)
        used = sum(v.numel() * v.element_size() for v in keep)
        if used > batch.nbytes:
            raise RuntimeError(f"batch allocated {used} device bytes, {batch.nbytes} were charged")
        batch.handle = (ev, out, keep)

    def poll(self, batch):
        return batch.handle[0].query()

    def collect(self, batch):
        ev, out, _ = batch.handle
        ev.synchronize()
        res = out.numpy()
        o = 0
        for r in batch.requests:
            c = r.x.shape[0]
            r.result = res[o:o + c].copy()
            o += c
        batch.handle = None


class Server:
    """Admission by HBM budget + continuous batching over an Executor."""

    def __init__(self, executor: Executor, hbm_budget_bytes: int, max_batch_requests: int = 32,
                 clock=time.perf_counter):
        self.ex = executor
        self.budget = int(hbm_budget_bytes)
        self.max_batch = max_batch_requests
        self.clock = clock
        self._pending = collections.deque()
        self._lock = threading.Lock()
        self.inflight = {}            # slot -> Batch
        self.inflight_bytes = 0
        self.done = []
        self.rejected = []
        self.peak_bytes = 0
        self.batches = 0

    # -- producer side (any thread) ------------------------------------------
    def submit(self, req: Request):
        if not req.t_arrival:
            req.t_arrival = self.clock()
        with self._lock:
            self._pending.append(req)

    def pending(self) -> int:
        with self._lock:
            return len(self._pending)

    # -- server loop (one thread) ---------------------------------------------
    def _free_slot(self):
        for s in range(self.ex.slots):
            if s not in self.inflight:
                return s
        return None

    def _admit(self):
        """Form one batch from the oldest pending request's (plan, kind) bucket."""
        slot = self._free_slot()
        if slot is None:
            return False
        with self._lock:
            if not self._pending:
                return False
            head = self._pending[0]
            key = self.ex.key(head)
            one = self.ex.nbytes(key, head.x.shape[0])
            if one > self.budget:
                self._pending.popleft()
                head.error = f"request needs {one} bytes, more than the HBM budget {self.budget}"
                head.t_done = self.clock()
                self.rejected.append(head)
                return True
            free = self.budget - self.inflight_bytes
            chosen, nbytes, segs = [], 0, 0
            rest = collections.deque()
            while self._pending and len(chosen) < self.max_batch:
                r = self._pending.popleft()
                if self.ex.key(r) == key:
                    need = self.ex.nbytes(key, segs + r.x.shape[0])
                    if need <= free:
                        chosen.append(r)
                        segs += r.x.shape[0]
                        nbytes = need
                        continue
                    rest.append(r)
                    break
                rest.append(r)
            while rest:
                self._pending.appendleft(rest.pop())
        if not chosen:
            return False                  # head waits until in-flight work frees budget
        now = self.clock()
        for r in chosen:
            r.t_admit = now
        b = Batch(key, chosen, nbytes)
        try:
            self.ex.launch(b, slot)
        except Exception as e:            # a failed launch fails its requests, not the server
            for r in chosen:
                r.error = f"launch failed: {e}"
                r.t_done = self.clock()
                self.rejected.append(r)
            return True
        self.inflight[slot] = b
        self.inflight_bytes += nbytes
        self.peak_bytes = max(self.peak_bytes, self.inflight_bytes)
        self.batches += 1
        return True

    def _complete(self):
        finished = [s for s, b in self.inflight.items() if self.ex.poll(b)]
        for s in finished:
            b = self.inflight.pop(s)
            try:
                self.ex.collect(b)
                err = None
            except Exception as e:
                err = f"collect failed: {e}"
            now = self.clock()
            for r in b.requests:
                r.t_done = now
                if err:
                    r.error = err
                    self.rejected.append(r)
                else:
                    self.done.append(r)
            self.inflight_bytes -= b.nbytes
        return bool(finished)

    def step(self) -> bool:
        """One loop iteration; True if anything happened."""
        progressed = self._complete()
        while self._admit():
            progressed = True
        return progressed

    def drain(self, timeout: float = 60.0):
        t0 = self.clock()
        while (self.pending() or self.inflight) and self.clock() - t0 < timeout:
            if not self.step():
                time.sleep(0.0002)

    # -- statistics ----------------------------------------------------------
    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.done], dtype=np.float64)
        samples = sum(r.samples for r in self.done)
        if len(self.done):
            t0 = min(r.t_arrival for r in self.done)
            t1 = max(r.t_done for r in self.done)
        else:
            t0 = t1 = 0.0
        return {
            "completed": len(self.done), "rejected": len(self.rejected), "batches": self.batches,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_ms": float(lat.max() * 1e3) if lat.size else None,
            "msamples_per_s": samples / max(t1 - t0, 1e-9) / 1e6 if lat.size else 0.0,
            "peak_inflight_bytes": self.peak_bytes,
        }


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times of a seeded Poisson process."""
    g = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


def make_request(rid: int, seed: int, n_channels=3, n=32768, fs=4096.0, qs=(8.0, 16.0, 32.0), inverse_frac=0.2,
                 rows=128) -> Request:
    """A serving request: `n_channels` whitened strain windows with glitches and
    a chirp, a Q drawn from `qs`, and with probability `inverse_frac` an
    inverse request whose envelope has 10-30 % of its rows zeroed."""
    from . import synth
    g = synth.rng(seed)
    x = np.stack([synth.glitchy_segment(seed * 7 + c, n, fs, chirp=(c == 0)) for c in range(n_channels)])
    q = float(g.choice(np.asarray(qs)))
    if g.uniform() < inverse_frac:
        gain = np.ones((n_channels, rows), np.float32)
        for c in range(n_channels):
            k = int(round(g.uniform(0.1, 0.3) * rows))
            gain[c, g.choice(rows, size=k, replace=False)] = 0.0
        return Request(rid, x, q, "inverse", gain, fs)
    return Request(rid, x, q, "forward", None, fs)


def run_stream(server: Server, requests, arrivals, realtime=True):
    """Feed requests at their arrival times (seconds from now) and serve them."""
    t0 = server.clock()
    heap = [(a, i) for i, a in enumerate(arrivals)]
    heapq.heapify(heap)
    while heap or server.pending() or server.inflight:
        now = server.clock() - t0
        while heap and (heap[0][0] <= now or not realtime):
            a, i = heapq.heappop(heap)
            r = requests[i]
            r.t_arrival = t0 + a if realtime else server.clock()
            server.submit(r)
        if not server.step():
            time.sleep(0.0002)
    return server.stats()
