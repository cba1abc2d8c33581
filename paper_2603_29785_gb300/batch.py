"""Uneven batches: many segments of different lengths and sample rates.

Segments are grouped by (sample rate, length); each group gets its own plan
(same Q planes, rows and frequency range) and is transformed with the
batched C entry points, which enqueue every group on one stream with one
shared workspace.  ``UnevenBatch.capture()`` records the forward and inverse
of all groups into a single CUDA graph, so a whole uneven batch is one graph
launch; inside the graph the groups are spread over several forked streams
(one workspace each), so independent groups run concurrently and fill each
other's last waves.  Row-kernel launch shapes come from the autotuner.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import qtam
from . import tune as qtune


@dataclass
class Group:
    fs: float
    N: int
    index: list                    # positions of this group's segments in the caller's list
    plan: "qtam.Plan" = None
    x: object = None               # [b, N] device input
    y: object = None               # [b, P, K, M] device envelopes
    xh: object = None              # [b, N] device reconstruction


class PlanCache:
    """Plans keyed by (fs, N, planes, rows, band, options), kept resident."""

    def __init__(self, qs, f_min, f_max, rows_per_plane, device=0, **opts):
        self.qs, self.f_min, self.f_max, self.K = tuple(qs), f_min, f_max, rows_per_plane
        self.device, self.opts = device, opts
        self._plans = {}

    def get(self, fs: float, N: int) -> "qtam.Plan":
        key = (float(fs), int(N))
        p = self._plans.get(key)
        if p is None:
            p = qtam.Plan(fs, N, self.qs, self.f_min, self.f_max, self.K, device=self.device, **self.opts)
            self._plans[key] = p
        return p

    def __len__(self):
        return len(self._plans)

    def plans(self):
        return list(self._plans.values())


class UnevenBatch:
    """Forward + inverse of a fixed list of uneven segments, optionally as one CUDA graph."""

    def __init__(self, segments, sample_rates, cache: PlanCache, tune: bool = True, plane_mask: int = 0):
        import torch

        self.cache = cache
        self.plane_mask = plane_mask
        self.n = len(segments)
        keys = {}
        for i, (x, fs) in enumerate(zip(segments, sample_rates)):
            keys.setdefault((float(fs), int(len(x))), []).append(i)
        # largest groups first: the long transforms dominate
        self.groups = [Group(fs, N, idx) for (fs, N), idx in sorted(keys.items(), key=lambda kv: -kv[0][1])]
        dev = f"cuda:{cache.device}"
        self.samples = int(sum(len(x) for x in segments))
        for g in self.groups:
            g.plan = cache.get(g.fs, g.N)
            b = len(g.index)
            g.x = torch.from_numpy(np.stack([np.asarray(segments[i], np.float32) for i in g.index])).to(dev)
            g.y = g.plan.envelope_tensor(b)
            g.xh = torch.empty((b, g.N), dtype=torch.float32, device=dev)
            if tune:
                qtune.tune(g.plan, b)
        self.fwd = [(g.plan.handle, g.x, g.y, len(g.index)) for g in self.groups]
        self.inv = [(g.plan.handle, g.y, g.xh, len(g.index)) for g in self.groups]
        self.ws_bytes = max(qtam.qtam_batched_workspace_size(self.fwd), qtam.qtam_batched_workspace_size(self.inv))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.graph = None
        self._stream_ws = {}
        self.envelope_bytes = sum(int(g.y.numel() * g.y.element_size()) for g in self.groups)

    # -- eager ---------------------------------------------------------------
    def forward(self, stream=None):
        qtam.qtam_forward_batched(self.fwd, self.ws, self.ws_bytes, stream)

    def inverse(self, stream=None):
        qtam.qtam_inverse_batched(self.inv, self.plane_mask, self.ws, self.ws_bytes, stream)

    def roundtrip(self, stream=None):
        self.forward(stream)
        self.inverse(stream)

    # -- graph ---------------------------------------------------------------
    def _lanes(self, n_streams):
        """Split the groups over n_streams lanes (balanced by envelope bytes),
        each lane with its own workspace."""
        import torch
        lanes = [[] for _ in range(n_streams)]
        load = [0] * n_streams
        for g in sorted(self.groups, key=lambda g: -int(g.y.numel())):
            i = load.index(min(load))
            lanes[i].append(g)
            load[i] += int(g.y.numel())
        out = []
        for i, lane in enumerate(lanes):
            if not lane:
                continue
            need = max(qtam.qtam_workspace_size(g.plan.handle, len(g.index)) for g in lane)
            ws = self._stream_ws.get(i)
            if ws is None or ws.numel() < need:
                ws = torch.empty(need, dtype=torch.uint8, device=self.ws.device)
                self._stream_ws[i] = ws
            out.append((lane, ws))
        return out

    def capture(self, n_streams: int = 4):
        """Record forward + inverse of every group into one CUDA graph.  The
        groups are spread over n_streams forked streams (each with its own
        workspace) so independent groups run concurrently and fill each
        other's last waves; n_streams = 1 records them in order."""
        import torch

        self.roundtrip()                      # first call outside capture: tables and attributes exist
        torch.cuda.synchronize()
        lanes = self._lanes(max(1, n_streams))
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        side = [torch.cuda.Stream() for _ in lanes]
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for lane_stream in side:
                    lane_stream.wait_stream(s)            # fork
                for (lane, ws), lane_stream in zip(lanes, side):
                    with torch.cuda.stream(lane_stream):
                        for grp in lane:
                            b = len(grp.index)
                            qtam.qtam_forward(grp.plan.handle, grp.x, b, grp.y, ws, ws.numel(), lane_stream)
                            qtam.qtam_inverse(grp.plan.handle, grp.y, b, self.plane_mask, grp.xh, ws, ws.numel(),
                                              lane_stream)
                for lane_stream in side:
                    s.wait_stream(lane_stream)            # join
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    # -- results -------------------------------------------------------------
    def envelopes(self, i):
        """Envelope tensor [P, K, M] of segment i (a view)."""
        for g in self.groups:
            if i in g.index:
                return g.y[g.index.index(i)]
        raise IndexError(i)

    def reconstruction(self, i):
        for g in self.groups:
            if i in g.index:
                return g.xh[g.index.index(i)]
        raise IndexError(i)


def uneven_workload(n_segments=512, durations=(1, 2, 4, 8, 16, 32), rates=(4096.0, 16384.0), seed=0,
                    max_seconds=None):
    """Seeded uneven segments: lengths uniform over `durations`, half the
    segments at each rate, whitened noise + sine-Gaussian glitches, a chirp in
    every other segment.  Returns (list of float32 arrays, list of rates)."""
    from . import synth

    g = synth.rng(seed)
    dur = g.choice(np.asarray(durations, float), size=n_segments)
    if max_seconds is not None:
        dur = np.minimum(dur, max_seconds)
    fs = np.where(np.arange(n_segments) % 2 == 0, rates[0], rates[-1])
    segs = [synth.glitchy_segment(seed * 100003 + i, int(d * f), float(f), chirp=(i % 4 < 2))
            for i, (d, f) in enumerate(zip(dur, fs))]
    return segs, [float(f) for f in fs]
