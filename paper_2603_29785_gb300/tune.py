"""Autotuner for the row kernels' launch shapes.

Every plan can run its per-row transforms with the runtime mixed-radix engine
or with any compile-time variant built for its envelope length M (radix
sequence, rows per block, occupancy target; see ``qtam_plan_variants``).  All
variants compute the same numbers; ``tune`` times each one on the plan's own
shapes (the envelope stage and the accumulation stage, CUDA events on the
current stream, synthetic inputs), keeps the fastest with
``qtam_plan_set_variant`` and caches the choice in a JSON file keyed by GPU,
geometry, batch and envelope dtype.
"""
from __future__ import annotations

import json
import os
import threading

from . import qtam

_lock = threading.Lock()


def default_cache_path() -> str:
    return os.environ.get("QTAM_TUNE_CACHE", os.path.join(os.path.dirname(qtam._build.lib_path()), "tune_cache.json"))


def _key(plan: "qtam.Plan", batch: int) -> str:
    import torch
    name = torch.cuda.get_device_name(plan.device).replace(" ", "_")
    i, d = plan.info, plan._desc
    # the plan's kind: window (band_bins tells composite banks apart), dense-mode options, short-DFT engine
    kind = f"w{d.window}:{d.window_param}:{i['band_bins']}|eps{d.stopband_eps}|rm{d.remodulate}|sd{d.short_dft}"
    return f"{name}|N{plan.N}|P{plan.P}|K{plan.K}|M{plan.M}|B{batch}|{plan.compute}/{plan.envelope}|{kind}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    tmp = path + ".tmp"
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(plan: "qtam.Plan", batch: int, reps: int = 5, warmup: int = 2, cache_path: str | None = None,
         use_cache: bool = True) -> dict:
    """Select the fastest row-kernel variant for `plan` at `batch` segments.

    Returns {"variant": id, "name": ..., "timings": {id: (fwd_ms, inv_ms)}, "cached": bool}.
    """
    import torch

    cache_path = cache_path or default_cache_path()
    key = _key(plan, batch)
    variants = qtam.qtam_plan_variants(plan.handle)
    if use_cache:
        with _lock:
            hit = _load(cache_path).get(key)
        if hit is not None and hit["variant"] in variants:
            qtam.qtam_plan_set_variant(plan.handle, hit["variant"])
            return dict(hit, cached=True)
    if len(variants) == 1:
        return {"variant": variants[0], "name": qtam.qtam_variant_describe(variants[0])["name"], "timings": {},
                "cached": False}
    dev = f"cuda:{plan.device}"
    gen = torch.Generator(device=dev).manual_seed(1234)
    x = torch.randn((batch, plan.N), generator=gen, device=dev, dtype=plan.real_dtype())
    X = plan.spectrum(x)
    y = plan.envelopes(X)
    st = torch.cuda.current_stream(plan.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    timings = {}
    for v in variants:
        qtam.qtam_plan_set_variant(plan.handle, v)
        for _ in range(warmup):
            plan.envelopes(X)
            plan.accumulate(y)
        tf = ti = 0.0
        for _ in range(reps):
            ev[0].record(st)
            plan.envelopes(X)
            ev[1].record(st)
            plan.accumulate(y)
            ev[2].record(st)
            ev[2].synchronize()
            tf += ev[0].elapsed_time(ev[1])
            ti += ev[1].elapsed_time(ev[2])
        timings[v] = (tf / reps, ti / reps)
    best = min(timings, key=lambda v: sum(timings[v]))
    qtam.qtam_plan_set_variant(plan.handle, best)
    res = {"variant": best, "name": qtam.qtam_variant_describe(best)["name"],
           "timings": {str(k): [round(a, 4), round(b, 4)] for k, (a, b) in timings.items()}}
    with _lock:
        data = _load(cache_path)
        data[key] = res
        try:
            _save(cache_path, data)
        except OSError:
            pass
    return dict(res, cached=False)
