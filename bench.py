"""Benchmark: QTAM forward + inverse throughput on GB300.

Workload (one step = one pass of the whole path over one batch): 64 segments
of 64 s at 4096 Hz (N = 262144) of coloured-then-whitened Gaussian noise with
a Newtonian chirp (SNR 20), Q-planes {4, 8, 16, 32, 64} x 128 log rows from
20 to 2048 Hz, envelopes M = 4800, FP32.  A step runs the long FFT, the
envelope kernel, the accumulation kernel and the synthesis (1/P + inverse
long FFT) through the library's C ABI.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on the host instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "QTAM fwd+inv Msamples/s and HBM-roofline % at FP32 vs FP64-oracle error; p99 latency"
UNIT = "Msamples/s"
WORKLOAD = dict(fs=4096.0, N=262144, qs=(4.0, 8.0, 16.0, 32.0, 64.0), fmin=20.0, fmax=2048.0, K=128)
WORKLOAD_NAME = "64 s @ 4096 Hz segments, Q {4,8,16,32,64} x 128 log rows 20-2048 Hz, M=4800, FP32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=64, help="segments per GPU per step")
    ap.add_argument("--impl", default="qtam", choices=["qtam", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the serving, batched and precision legs of the default line")
    ap.add_argument("--serving-seconds", type=float, default=12.0,
                    help="seconds of arrivals of the serving leg in the default line")
    ap.add_argument("--cpu-sample-segments", type=int, default=4)
    ap.add_argument("--variant", type=int, default=None,
                    help="row-kernel variant id (default: chosen by the autotuner)")
    ap.add_argument("--workload", default="64s", choices=["64s", "batched", "serving", "precision", "latency", "stream", "dense", "bank"],
                    help="64s: the headline workload (default); batched: 512 uneven segments in one graph; "
                         "serving: Poisson request stream; precision: envelope dtype sweep; "
                         "stream: overlap-save over a continuous signal; dense: stopband-floored tiles + "
                         "single-tile inverse; bank: Q x window composite bank with optimal-plane metrics")
    ap.add_argument("--duration", type=float, default=60.0, help="seconds of arrivals for --workload serving")
    return ap.parse_args()


def rank_seeds(rank: int, per_rank: int):
    """Distinct input seeds per rank: each rank transforms its own segments
    (weak scaling, replicas; no data crosses ranks)."""
    return [rank * per_rank + i for i in range(per_rank)]


def reduce_max(value: float, dist, device=None) -> float:
    """Max of a per-rank value over all ranks (the job time is the slowest
    rank's); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------- inputs
def make_inputs(seeds):
    from paper_2603_29785_gb300 import synth
    return np.stack([synth.coloured_chirp_segment(int(s), n=WORKLOAD["N"], fs=WORKLOAD["fs"]) for s in seeds])


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s) and its source."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    """Time the FP64 CPU oracle (as it stands) on the host cores: each step is
    one segment per core (distinct seeds), forward + inverse, in spawned
    worker processes warmed before timing; a host that cannot spawn
    processes runs one segment per step on one thread."""
    if rank != 0:
        return
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import qtam_oracle as O
    g = O.geometry(WORKLOAD["fs"], WORKLOAD["N"], WORKLOAD["qs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["K"])
    tau = 1e-6
    ncores = os.cpu_count() or 1
    times, note = [], None
    try:
        x = make_inputs(range(ncores))
        with cf.ProcessPoolExecutor(max_workers=ncores, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_warm, range(ncores)))
            for s in range(max(0, min(args.warmup, 1)) + args.steps):
                t0 = time.perf_counter()
                list(ex.map(_oracle_segment_seconds, [x[b] for b in range(ncores)], [tau] * ncores))
                if s >= min(args.warmup, 1):
                    times.append(time.perf_counter() - t0)
        per_step, cores = ncores, ncores
        sample = f"{ncores} segments of the workload per step, one per worker process, forward + inverse, numpy FP64"
    except Exception as e:     # no process spawning: one segment per step on one thread
        note = str(e)[:200]
        x = make_inputs([0])[0].astype(np.float64)
        times = []
        for s in range(max(0, min(args.warmup, 1)) + args.steps):
            t0 = time.perf_counter()
            O.inverse(g, O.forward(g, x), tau=tau)
            if s >= min(args.warmup, 1):
                times.append(time.perf_counter() - t0)
        per_step, cores = 1, 1
        sample = "1 segment of the workload per step (forward + inverse, numpy FP64, one thread)"
    total = sum(times)
    value = args.steps * per_step * WORKLOAD["N"] / total / 1e6
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if note:
        cb["all_cores_unavailable"] = note
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "segments_per_step": per_step, "N": WORKLOAD["N"], "M": g.M},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measured_traffic(kernel: str):
    """DRAM bytes per full-size launch from the committed ncu capture, or None
    when the kernel sources changed since the counters were taken."""
    import hashlib
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        h = hashlib.sha256()
        for f in ("kernels_rows.cu", "rows_common.cuh", "fft_static.cuh", "fft_core.cuh", "qtam_internal.h"):
            h.update(open(os.path.join(ROOT, "paper_2603_29785_gb300", "csrc", f), "rb").read())
        if h.hexdigest() != tr.get("source_sha256"):
            return None
        return tr.get(kernel, {}).get("bytes_per_launch_full")
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------- GPU arm
def _oracle_segment_seconds(x, tau):
    """Forward + inverse of one segment by the oracle as it stands (worker of
    the all-cores timing; top level so a spawned process can import it)."""
    from oracle import qtam_oracle as O
    t0 = time.perf_counter()
    g = O.geometry(WORKLOAD["fs"], WORKLOAD["N"], WORKLOAD["qs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["K"])
    O.inverse(g, O.forward(g, np.asarray(x, dtype=np.float64)), tau=tau)
    return time.perf_counter() - t0


def _warm(_):
    from oracle import qtam_oracle  # noqa: F401  (imports numpy and the oracle once per worker)
    return os.getpid()


def cpu_all_cores(x_host, tau, ncores):
    """The oracle on every host core: one segment per worker process (spawned,
    so safe after the CUDA context exists), workers warmed before timing."""
    import concurrent.futures as cf
    import multiprocessing as mp
    nseg = min(ncores, x_host.shape[0])
    with cf.ProcessPoolExecutor(max_workers=nseg, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_warm, range(nseg)))
        t0 = time.perf_counter()
        list(ex.map(_oracle_segment_seconds, [x_host[b] for b in range(nseg)], [tau] * nseg))
        dt = time.perf_counter() - t0
    return {"value": nseg * WORKLOAD["N"] / dt / 1e6, "unit": UNIT, "cores": nseg, "kind": "oracle",
            "sample": f"{nseg} segments of the workload, one per worker process, forward + inverse, numpy FP64"}


def cpu_baseline_leg(p, x_host, xh_gpu, y_gpu, nseg):
    """Oracle on a bounded sample (nseg segments): timing + GPU-vs-oracle error."""
    from oracle import qtam_oracle as O
    g = O.geometry(WORKLOAD["fs"], WORKLOAD["N"], WORKLOAD["qs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["K"])
    tau = p.info["p_floor_rel"]
    t0 = time.perf_counter()
    errs_f, errs_rt = [], []
    outs = []
    for b in range(nseg):
        xb = x_host[b].astype(np.float64)
        Y = O.forward(g, xb)
        xr = O.inverse(g, Y, tau=tau)
        outs.append((Y, xr))
    dt = time.perf_counter() - t0
    for b, (Y, xr) in enumerate(outs):
        errs_f.append(float(np.linalg.norm(y_gpu[b] - Y) / np.linalg.norm(Y)))
        xp = xr  # oracle inverse of its own forward = projection onto F_tau
        errs_rt.append(float(np.linalg.norm(xh_gpu[b] - xp) / np.linalg.norm(xp)))
    one = {"value": nseg * WORKLOAD["N"] / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{nseg} segments of the workload, forward + inverse, numpy FP64, one thread"}
    try:
        allc = cpu_all_cores(x_host, tau, os.cpu_count() or 1)
        allc["single_thread"] = one
        base = allc
    except Exception as e:          # a host without process spawning keeps the one-thread number
        one["all_cores_unavailable"] = str(e)[:200]
        base = one
    return (base,
            {"forward_rel_err_max": max(errs_f), "roundtrip_rel_err_max": max(errs_rt),
             "segments_checked": nseg, "tolerance": {"forward": 1e-6, "roundtrip": 1e-5}})


def run_gpu(args, rank, world, local):
    import torch
    from paper_2603_29785_gb300 import qtam

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B = args.batch
    seeds = rank_seeds(rank, B)
    x_host = make_inputs(seeds)
    p = qtam.Plan(WORKLOAD["fs"], WORKLOAD["N"], WORKLOAD["qs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["K"],
                  device=local)
    if args.variant is not None:
        qtam.qtam_plan_set_variant(p.handle, args.variant)
        chosen = qtam.qtam_variant_describe(args.variant)
    else:
        from paper_2603_29785_gb300 import tune as qtune
        chosen = qtune.tune(p, B)
    N, Nr, M, P, K = p.N, p.Nr, p.M, p.P, p.K
    dev = f"cuda:{local}"
    x = torch.from_numpy(x_host).to(dev)
    X = torch.empty((B, Nr), dtype=torch.complex64, device=dev)
    A = torch.empty((B, Nr), dtype=torch.complex64, device=dev)
    y = p.envelope_tensor(B)
    xh = torch.empty((B, N), dtype=torch.float32, device=dev)
    ws, wsb = p.workspace(B)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    st = torch.cuda.current_stream()
    h = p.handle

    def step():
        qtam.qtam_stage_spectrum(h, x, B, X, ws, wsb, st)
        ev[1].record(st)
        qtam.qtam_stage_envelopes(h, X, B, y, st)
        ev[2].record(st)
        qtam.qtam_stage_accumulate(h, y, B, 0, A, st)
        ev[3].record(st)
        qtam.qtam_stage_synthesize(h, A, B, 0, xh, ws, wsb, st)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for _ in range(args.warmup):
        flush.zero_()
        ev[0].record(st)
        step()
        ev[4].record(st)
    torch.cuda.synchronize()
    stage_ms = np.zeros(4)
    total_ms = 0.0
    step_ms = []
    # the sampler runs from the timed loop through the e2e and per-segment
    # legs (the GPU is busy throughout), so the record holds more than the one
    # sample a ~25 ms loop would give at 50 ms intervals
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        ev[0].record(st)
        step()
        ev[4].record(st)
        ev[4].synchronize()
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        stage_ms += t
        step_ms.append(ev[0].elapsed_time(ev[4]))
        total_ms += step_ms[-1]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_per_step = reduce_max(total_ms / args.steps, dist, dev)
    samples_per_step = world * B * N
    value = samples_per_step / (ms_per_step * 1e-3) / 1e6

    # ---- end to end through the C ABI with host buffers (pinned) ----
    x_pin = torch.from_numpy(x_host).pin_memory()
    xh_pin = torch.empty((B, N), dtype=torch.float32).pin_memory()
    for _ in range(2):
        qtam.qtam_roundtrip_host(h, x_pin, B, 0, xh_pin, x, y, xh, ws, wsb, st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        qtam.qtam_roundtrip_host(h, x_pin, B, 0, xh_pin, x, y, xh, ws, wsb, st)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dist, dev)
    e2e = {"value": samples_per_step / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": B * N * 4,
           "d2h_bytes_per_step": B * N * 4, "ms_per_step": e2e_s * 1e3}

    # ---- the plain per-segment path on the same GPU and plan: one qtam_forward +
    # qtam_inverse call pair per segment (the same kernels at batch 1: the same numbers) ----
    def per_segment():
        for b in range(B):
            qtam.qtam_forward(h, x[b:b + 1], 1, y[b:b + 1], ws, wsb, st)
            qtam.qtam_inverse(h, y[b:b + 1], 1, 0, xh[b:b + 1], ws, wsb, st)

    for _ in range(2):
        per_segment()
    ps_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev[0].record(st)
        per_segment()
        ev[4].record(st)
        ev[4].synchronize()
        ps_ms += ev[0].elapsed_time(ev[4])
    ps_ms = reduce_max(ps_ms / args.steps, dist, dev)
    clk = clocks.stop()
    clk["window"] = "timed loop, e2e and per-segment legs"
    per_seg = {"value": round(samples_per_step / (ps_ms * 1e-3) / 1e6, 2), "unit": UNIT, "ms_per_step": round(ps_ms, 4),
               "path": "the same segments, one qtam_forward + qtam_inverse call pair per segment"}

    # ---- roofline of the dominant kernel (envelope kernel: writes B*P*K*M complex64) ----
    hbm_peak, peak_src = hbm_peak_gbs()
    env_bytes = B * P * K * M * 8
    x_bytes = B * N * 4
    stage_bytes = [x_bytes, env_bytes, env_bytes, x_bytes]       # algorithmic HBM bytes per stage launch
    stage_names = ["spectrum (long R2C FFT)", "envelopes (k_rows_forward)", "accumulate (k_rows_inverse)",
                   "synthesize (1/P + long C2R FFT)"]
    stage_avg_ms = stage_ms / args.steps
    kernels = {}
    for nm, b, t in zip(stage_names, stage_bytes, stage_avg_ms):
        kernels[nm] = {"ms": round(float(t), 4), "alg_bytes": int(b), "GB_s": round(b / (t * 1e-3) / 1e9, 1)}
    dom = int(np.argmax(stage_avg_ms[1:3])) + 1
    achieved = stage_bytes[dom] / (stage_avg_ms[dom] * 1e-3) / 1e9
    traffic = measured_traffic(["", "k_rows_forward", "k_rows_inverse"][dom])
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": traffic, "kernel": stage_names[dom],
                "peak_source": peak_src}
    fwdinv_bytes = 2 * (env_bytes + x_bytes)
    path_frac = fwdinv_bytes / (ms_per_step * 1e-3) / 1e9 / hbm_peak

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "segments_per_gpu": B, "N": N, "M": M, "planes": P,
                   "rows_per_plane": K, "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "row_variant": chosen["name"]},
        "roofline": roofline,
        "path_hbm_frac": round(path_frac, 4),
        "stages": kernels,
        "e2e": e2e,
        "per_segment_path": per_seg,
        # per step: k_col_forward, k_row_forward, k_untangle_forward (spectrum), k_rows_forward_s
        # (envelopes), k_rows_inverse_s (accumulate; the zeroing is a memset, not a kernel),
        # k_untangle_inverse, k_row_inverse, k_col_inverse (synthesis) -- as the ncu launch list shows
        "gpu_launches": 8 * args.steps,
        "clocks": clk,
        # latency of one whole step (64 segments forward + inverse), over the timed steps
        "latency": {"step_p50_ms": round(float(np.percentile(step_ms, 50)), 4),
                    "step_p99_ms": round(float(np.percentile(step_ms, 99)), 4),
                    "step_max_ms": round(float(np.max(step_ms)), 4)},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        # the metric's p99 latency under load, and the batched and precision
        # configurations, as extra keys of the same line
        sv = serving_leg(local, args.serving_seconds)
        line["serving"] = dict(sv["serving"], config=sv["config"], clocks=sv["clocks"])
        line["latency"]["serving_p50_ms"] = sv["serving"]["p50_ms"]
        line["latency"]["serving_p99_ms"] = sv["serving"]["p99_ms"]
        bl = batched_leg(argparse.Namespace(steps=max(3, min(args.steps, 10)), warmup=3), local)
        line["batched"] = bl
        line["precision"] = precision_leg(argparse.Namespace(steps=max(3, min(args.steps, 10))), local, B)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nseg = max(1, min(args.cpu_sample_segments, B))
        torch.cuda.synchronize()
        yv = y[:nseg].cpu().numpy().astype(np.complex128)
        xv = xh[:nseg].cpu().numpy().astype(np.float64)
        cb, acc = cpu_baseline_leg(p, x_host, xv, yv, nseg)
        line["cpu_baseline"] = cb
        line["accuracy"] = acc
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- other workloads
def _clock_wrap(fn, local):
    clocks = ClockSampler(local)
    clocks.start()
    try:
        out = fn()
    finally:
        clk = clocks.stop()
    return out, clk


def batched_leg(args, local):
    """512 uneven segments (1-32 s, 4096/16384 Hz), Q {8,16,32} x 128 rows:
    forward + inverse of all segments captured as one CUDA graph, against the
    plain path (one forward + one inverse call per segment, no graph)."""
    import torch
    from paper_2603_29785_gb300 import batch as qb
    torch.cuda.set_device(local)
    segs, rates = qb.uneven_workload(512, seed=0)
    cache = qb.PlanCache((8.0, 16.0, 32.0), 20.0, 2048.0, 128, device=local)
    ub = qb.UnevenBatch(segs, rates, cache, tune=True)
    ub.capture(n_streams=1)
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ub.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        ub.replay()
    e1.record(st)
    e1.synchronize()
    ms_one_stream = e0.elapsed_time(e1) / args.steps
    ub.capture(n_streams=4)
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ub.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        e0.record(st)
        for _ in range(args.steps):
            ub.replay()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps
    ms, clk = _clock_wrap(timed, local)
    # plain per-segment path: one forward and one inverse per segment, eager
    per = []
    for g in ub.groups:
        for j in range(len(g.index)):
            per.append((g.plan, g.x[j:j + 1], g.y[j:j + 1], g.xh[j:j + 1]))

    def plain():
        for p, x, y, xh in per:
            p.forward(x, y)
            p.inverse(y, x=xh)
    plain()
    torch.cuda.synchronize()
    e0.record(st)
    reps = max(1, min(3, args.steps))
    for _ in range(reps):
        plain()
    e1.record(st)
    e1.synchronize()
    ms_plain = e0.elapsed_time(e1) / reps
    bytes_alg = 2 * (ub.envelope_bytes + ub.samples * 4)
    peak, src = hbm_peak_gbs()
    gbs = bytes_alg / (ms * 1e-3) / 1e9
    return {"value": round(ub.samples / ms / 1e3, 2), "unit": UNIT, "ms_per_step": round(ms, 4),
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "512 segments, 1-32 s, half 4096 Hz / half 16384 Hz, Q {8,16,32} x 128 rows 20-2048 Hz",
                       "groups": len(ub.groups), "graph_streams": 4, "samples": ub.samples,
                       "envelope_bytes": ub.envelope_bytes, "l2": "inputs+envelopes (1.4 GB) larger than L2"},
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "peak_source": src,
                         "bytes": "2 x (envelopes + input samples) per replay: forward writes and inverse reads "
                                  "every envelope, forward reads and inverse writes every sample"},
            "per_segment_plain_path": {"value": round(ub.samples / ms_plain / 1e3, 2), "ms_per_step": round(ms_plain, 3),
                                       "launches": "2 calls per segment, no graph"},
            "speedup_vs_plain": round(ms_plain / ms, 2),
            "graph_one_stream": {"value": round(ub.samples / ms_one_stream / 1e3, 2),
                                 "ms_per_step": round(ms_one_stream, 4)},
            "clocks": clk}


def run_batched(args, local):
    b = batched_leg(args, local)
    line = {"metric": "QTAM fwd+inv Msamples/s, uneven batch in one CUDA graph", "value": b.pop("value"),
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "path_hbm_frac": b["roofline"]["frac"]}
    line.update(b)
    print(json.dumps(line), flush=True)


def run_stream(args, local):
    """Overlap-save streaming of a continuous 4096 Hz signal through 64 s chunks
    (Q {4..64} x 128 rows, M = 4800) with a 32 s hop: every step pushes 16 hops
    (512 s of new samples) forward, then pushes the resulting map columns
    through the streaming inverse."""
    import torch
    from paper_2603_29785_gb300 import qtam, synth, tune as qtune
    torch.cuda.set_device(local)
    W = WORKLOAD
    p = qtam.Plan(W["fs"], W["N"], W["qs"], W["fmin"], W["fmax"], W["K"], device=local)
    qtune.tune(p, 16)
    hop, per = 131072, 16
    s = qtam.Stream(p, hop=hop, max_chunks=per)
    n = hop * per
    x = torch.from_numpy(np.concatenate([synth.coloured_chirp_segment(100 + i)[:hop] for i in range(per)])
                         .astype(np.float32)).cuda()
    y = s._map_tensor(per * s.hop_cols)
    xh = torch.empty(n, dtype=torch.float32, device=x.device)
    st = torch.cuda.current_stream()

    def step():
        qtam.qtam_stream_forward(s.handle, x, n, y, st)
        qtam.qtam_stream_inverse(s.handle, y, per * s.hop_cols, 0, xh, st)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def timed():
        tf = 0.0
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(st)
        for _ in range(args.steps):
            ev[0].record(st)
            qtam.qtam_stream_forward(s.handle, x, n, y, st)
            ev[1].record(st)
            qtam.qtam_stream_inverse(s.handle, y, per * s.hop_cols, 0, xh, st)
        t1.record(st)
        t1.synchronize()
        return t0.elapsed_time(t1) / args.steps
    ms, clk = _clock_wrap(timed, local)
    # forward alone, same pushes
    torch.cuda.synchronize()
    ev[0].record(st)
    for _ in range(args.steps):
        qtam.qtam_stream_forward(s.handle, x, n, y, st)
    ev[1].record(st)
    ev[1].synchronize()
    ms_f = ev[0].elapsed_time(ev[1]) / args.steps
    # algorithmic bytes: the kept map columns written (forward) and read (inverse), samples in and out
    kept = p.P * p.K * per * s.hop_cols * 8
    peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    line = {"metric": "QTAM streaming fwd+inv Msamples/s of continuous signal", "value": round(n / ms / 1e3, 2),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "continuous 4096 Hz stream, 64 s chunks (N=262144, M=4800), hop 32 s, "
                                   "Q {4,8,16,32,64} x 128 rows, 16 hops (512 s) per push",
                       "hop": hop, "guard": s.guard, "hop_cols": s.hop_cols, "samples_per_step": n,
                       "l2": "each step moves > 1 GB of envelopes"},
            "forward_only": {"value": round(n / ms_f / 1e3, 2), "ms_per_step": round(ms_f, 4)},
            "kept_map_hbm_frac": round(2 * kept / (ms * 1e-3) / 1e9 / peak, 4),
            "overlap_cost": "each 32 s of signal is transformed as part of two 64 s chunks (2x the segment work)",
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_dense(args, local):
    """Dense mode: 2 s @ 4096 Hz segments (N = 8192), Q {4,8,16} x 64 rows
    20-2048 Hz, stopband floor eps = 1e-3, remodulated (undemodulated) tiles of
    M = 4320 >= N/2 + 1 columns (the compile-time variants built for the dense
    mode, tuned); forward of every tile, the single-tile inverse from one
    mid-band tile per segment (spectral division), and the canonical dual
    inverse of all tiles."""
    import torch
    from oracle import qtam_oracle as O
    from paper_2603_29785_gb300 import qtam, synth
    torch.cuda.set_device(local)
    from paper_2603_29785_gb300 import tune as qtune
    fs, N, qs, K, eps = 4096.0, 8192, (4.0, 8.0, 16.0), 64, 1e-3
    B = args.batch * 4
    p = qtam.Plan(fs, N, qs, 20.0, 2048.0, K, stopband_eps=eps, remodulate=True, device=local)
    tuned = qtune.tune(p, B)      # the compile-time variants built for the dense mode (M = 4320)
    xh_ = np.stack([synth.glitchy_segment(500 + b, N, fs, chirp=(b % 2 == 0)) for b in range(B)]).astype(np.float32)
    x = torch.from_numpy(xh_).cuda()
    y = p.forward(x)
    xs = p.inverse_single_tile(y, 1, K // 2)
    torch.cuda.synchronize()
    g = O.geometry(fs, N, qs, 20.0, 2048.0, K, stopband_eps=eps, remodulate=True)
    ef = max(float(np.linalg.norm(y[b].cpu().numpy() - O.forward(g, xh_[b].astype(np.float64)))
                   / np.linalg.norm(O.forward(g, xh_[b].astype(np.float64)))) for b in range(2))
    es = max(float(np.linalg.norm(xs[b].cpu().numpy() - xh_[b]) / np.linalg.norm(xh_[b])) for b in range(2))
    st = torch.cuda.current_stream()
    ws, wsb = p.workspace(B)
    for _ in range(max(3, args.warmup)):
        qtam.qtam_forward(p.handle, x, B, y, ws, wsb, st)
        qtam.qtam_inverse_single_tile(p.handle, y, B, 1, K // 2, xs, ws, wsb, st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    xd = torch.empty_like(x)

    def timed():
        tf = ti = td = 0.0
        for _ in range(args.steps):
            ev[0].record(st)
            qtam.qtam_forward(p.handle, x, B, y, ws, wsb, st)
            ev[1].record(st)
            qtam.qtam_inverse_single_tile(p.handle, y, B, 1, K // 2, xs, ws, wsb, st)
            ev[2].record(st)
            qtam.qtam_inverse(p.handle, y, B, 0, xd, ws, wsb, st)
            ev[3].record(st)
            ev[3].synchronize()
            tf += ev[0].elapsed_time(ev[1])
            ti += ev[1].elapsed_time(ev[2])
            td += ev[2].elapsed_time(ev[3])
        return tf / args.steps, ti / args.steps, td / args.steps
    (ms_f, ms_i, ms_d), clk = _clock_wrap(timed, local)
    env_bytes = B * p.info["envelope_bytes_per_segment"]
    line = {"metric": "QTAM dense mode: tiles Msamples/s and single-tile inverse Msamples/s",
            "value": round(B * N / ms_f / 1e3, 2), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms_f, 4), "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "2 s @ 4096 Hz segments, Q {4,8,16} x 64 rows 20-2048 Hz, stopband eps 1e-3, "
                                   "remodulated tiles, M = %d" % p.M, "segments": B,
                       "l2": "envelopes %.2f GB per step, larger than L2" % (env_bytes / 1e9)},
            "forward_GB_s": round(env_bytes / (ms_f * 1e-3) / 1e9, 1),
            "single_tile_inverse": {"value": round(B * N / ms_i / 1e3, 2), "ms_per_step": round(ms_i, 4),
                                    "tile": [1, K // 2], "rel_err_vs_input": es},
            "canonical_inverse": {"value": round(B * N / ms_d / 1e3, 2), "ms_per_step": round(ms_d, 4)},
            "row_variant": tuned["name"],
            "forward_rel_err_vs_oracle": ef, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_bank(args, local):
    """Composite bank (App. A): the 64 s workload with one App. A window per
    plane -- (Q 4, bisquare), (8, Tukey 0.5), (16, Kaiser 8), (32, Hann),
    (64, Planck-taper 0.3) -- forward + inverse, then the per-plane energy /
    peak of every segment (optimal-plane selection), against the same
    transform with the bisquare on every plane."""
    import torch
    from paper_2603_29785_gb300 import qtam, tune as qtune
    torch.cuda.set_device(local)
    W = WORKLOAD
    B = args.batch
    wins = ("bisquare", "tukey", "kaiser", "hann", "planck")
    prms = (0.0, 0.5, 8.0, 0.0, 0.3)
    x = torch.from_numpy(make_inputs(range(B))).cuda()
    st = torch.cuda.current_stream()
    out = {}
    for label, kw in (("bank", dict(window=wins, window_param=prms)), ("bisquare", {})):
        p = qtam.Plan(W["fs"], W["N"], W["qs"], W["fmin"], W["fmax"], W["K"], device=local, **kw)
        qtune.tune(p, B)
        y = p.forward(x)
        xh = p.inverse(y)
        energy = torch.empty((B, p.P), dtype=torch.float64, device=x.device)
        peak = torch.empty((B, p.P), dtype=torch.float32, device=x.device)
        ws, wsb = p.workspace(B)
        for _ in range(max(3, args.warmup)):
            qtam.qtam_forward(p.handle, x, B, y, ws, wsb, st)
            qtam.qtam_inverse(p.handle, y, B, 0, xh, ws, wsb, st)
            qtam.qtam_plane_metrics(p.handle, y, B, energy, peak, st)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(st)
        for _ in range(args.steps):
            qtam.qtam_forward(p.handle, x, B, y, ws, wsb, st)
            qtam.qtam_inverse(p.handle, y, B, 0, xh, ws, wsb, st)
        ev[1].record(st)
        for _ in range(args.steps):
            qtam.qtam_plane_metrics(p.handle, y, B, energy, peak, st)
        ev[2].record(st)
        ev[2].synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        ms_m = ev[1].elapsed_time(ev[2]) / args.steps
        env_bytes = B * p.info["envelope_bytes_per_segment"]
        out[label] = {"msamples_per_s": round(B * W["N"] / ms / 1e3, 1), "ms_per_step": round(ms, 4),
                      "row_variant": qtam.qtam_variant_describe(p.info["row_variant"])["name"],
                      "plane_metrics_ms": round(ms_m, 4),
                      "plane_metrics_GB_s": round(env_bytes / (ms_m * 1e-3) / 1e9, 1),
                      "best_plane_by_energy_seg0": int(torch.argmax(energy[0]).item())}
    line = {"metric": "QTAM composite bank (Q x window) fwd+inv Msamples/s and optimal-plane metrics",
            "value": out["bank"]["msamples_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME + "; plane windows " + ", ".join(
                f"{w}{'' if a == 0 else ' ' + str(a)}" for w, a in zip(wins, prms)), "segments": B},
            "bank": out["bank"], "bisquare_all_planes": out["bisquare"]}
    print(json.dumps(line), flush=True)


def serving_leg(local, duration):
    """Poisson arrivals (200/s) of 3-channel 8 s @ 4096 Hz requests, Q in
    {8,16,32}, 20 % inverse of row-zeroed envelopes; 40 GB HBM budget."""
    import torch
    from paper_2603_29785_gb300 import serve
    torch.cuda.set_device(local)
    pool = [serve.make_request(i, 5000 + i) for i in range(256)]
    arrivals = serve.poisson_arrivals(200.0, duration, seed=7)
    reqs = [serve.Request(i, pool[i % len(pool)].x, pool[i % len(pool)].q, pool[i % len(pool)].kind,
                          pool[i % len(pool)].row_gain) for i in range(len(arrivals))]
    ex = serve.GpuExecutor(slots=4, device=local)
    warm = serve.Server(ex, hbm_budget_bytes=40 * 2**30)
    serve.run_stream(warm, [serve.Request(-i - 1, r.x, r.q, r.kind, r.row_gain) for i, r in enumerate(pool[:32])],
                     np.zeros(32), realtime=False)
    srv = serve.Server(ex, hbm_budget_bytes=40 * 2**30, max_batch_requests=32)
    st, clk = _clock_wrap(lambda: serve.run_stream(srv, reqs, arrivals), local)
    st["target_p99_ms"] = 100.0
    return {"config": {"workload": "Poisson 200 req/s, 3 x 8 s @ 4096 Hz per request, Q {8,16,32} x 128 rows, "
                                   "20 % inverse of row-zeroed envelopes", "duration_s": duration,
                       "hbm_budget_gb": 40, "streams": ex.slots, "max_batch_requests": 32},
            "serving": st, "clocks": clk}


def run_serving(args, local):
    sv = serving_leg(local, args.duration)
    line = {"metric": "QTAM serving p50/p99 latency (ms) and Msamples/s", "value": round(sv["serving"]["p99_ms"], 3),
            "unit": "ms p99", "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic"}
    line.update(sv)
    print(json.dumps(line), flush=True)


def precision_leg(args, local, B):
    """Precision sweep on the 64 s workload: envelope storage FP32 / BF16 / FP16
    at M = 4800 (CUDA-core FFTs), and at M = 8192 the CUDA-core runtime engine
    against the tensor-core short DFT (64 x 128 four-step on tcgen05, BF16
    operands, both directions): error against the FP64 oracle (2 segments),
    fwd+inv throughput, and the envelope and accumulation stages alone (64
    segments)."""
    import torch
    from oracle import qtam_oracle as O
    from paper_2603_29785_gb300 import qtam, tune as qtune
    torch.cuda.set_device(local)
    W = WORKLOAD
    x_host = make_inputs(range(B))
    refs = {}
    for n_out in (0, 8192):
        g = O.geometry(W["fs"], W["N"], W["qs"], W["fmin"], W["fmax"], W["K"], n_out=n_out)
        rr = []
        for b in range(2):
            xb = x_host[b].astype(np.float64)
            Y = O.forward(g, xb)
            rr.append((Y, O.inverse(g, Y, tau=1e-6)))
        refs[n_out] = rr
    x = torch.from_numpy(x_host).cuda()
    st = torch.cuda.current_stream()
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    out = []
    for env, n_out, sd in (("f32", 0, "cuda"), ("bf16", 0, "cuda"), ("f16", 0, "cuda"), ("f32", 8192, "cuda"),
                           ("f32", 8192, "tensor"), ("bf16", 8192, "tensor")):
        p = qtam.Plan(W["fs"], W["N"], W["qs"], W["fmin"], W["fmax"], W["K"], envelope=env, n_out=n_out,
                      short_dft=sd, device=local)
        qtune.tune(p, B)          # CUDA-core variants (the inverse, and the forward of "cuda" plans)
        y = p.forward(x)
        xh = p.inverse(y)
        torch.cuda.synchronize()
        yv = y[:2].float().cpu().numpy() if env != "f32" else y[:2].cpu().numpy()
        if env != "f32":
            yv = yv[..., 0] + 1j * yv[..., 1]
        rr = refs[n_out]
        ef = max(float(np.linalg.norm(yv[b] - rr[b][0]) / np.linalg.norm(rr[b][0])) for b in range(2))
        er = max(float(np.linalg.norm(xh[b].cpu().numpy() - rr[b][1]) / np.linalg.norm(rr[b][1])) for b in range(2))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for _ in range(3):
            p.forward(x, y); p.inverse(y, x=xh)
        e[0].record(st)
        for _ in range(args.steps):
            p.forward(x, y); p.inverse(y, x=xh)
        e[1].record(st)
        e[1].synchronize()
        ms = e[0].elapsed_time(e[1]) / args.steps
        X = p.spectrum(x)
        qtam.qtam_stage_envelopes(p.handle, X, B, y, st)
        e[2].record(st)
        for _ in range(args.steps):
            qtam.qtam_stage_envelopes(p.handle, X, B, y, st)
        e[3].record(st)
        e[3].synchronize()
        ms_env = e[2].elapsed_time(e[3]) / args.steps
        A = p.accumulate(y)
        e[4].record(st)
        for _ in range(args.steps):
            qtam.qtam_stage_accumulate(p.handle, y, B, 0, A, st)
        e[5].record(st)
        e[5].synchronize()
        ms_acc = e[4].elapsed_time(e[5]) / args.steps
        item = {"envelope": env, "M": p.M, "short_dft": sd, "forward_rel_err": ef, "roundtrip_rel_err": er,
                "msamples_per_s": round(B * W["N"] / ms / 1e3, 1), "ms_per_step": round(ms, 4),
                "envelope_stage_ms": round(ms_env, 4), "accumulate_stage_ms": round(ms_acc, 4),
                "envelope_stage_GB_s": round(B * p.info["envelope_bytes_per_segment"] / (ms_env * 1e-3) / 1e9, 1),
                "envelope_bytes_per_segment": p.info["envelope_bytes_per_segment"]}
        pk_hbm, _ = hbm_peak_gbs()
        item["envelope_stage_hbm_frac"] = round(item["envelope_stage_GB_s"] / pk_hbm, 4)
        item["accumulate_stage_hbm_frac"] = round(
            B * p.info["envelope_bytes_per_segment"] / (ms_acc * 1e-3) / 1e9 / pk_hbm, 4)
        if sd == "tensor":
            # two tcgen05 GEMMs per pair of rows in each direction: 128x256x128 +
            # 4 x 128x128x128 multiply-adds
            flops = B * p.P * p.K / 2 * 2 * (128 * 256 * 128 + 4 * 128 * 128 * 128)
            tf = flops / (ms_env * 1e-3) / 1e12
            tfi = flops / (ms_acc * 1e-3) / 1e12
            pk = float(peaks.get("bf16_tflops", 1900.0))
            item["tensor"] = {"achieved_tflops": round(tf, 1), "peak_tflops": pk, "frac": round(tf / pk, 4),
                              "inverse_achieved_tflops": round(tfi, 1), "inverse_frac": round(tfi / pk, 4),
                              "peak_source": "measured" if "bf16_tflops" in peaks else "fallback"}
        out.append(item)
    return out


def run_precision(args, local):
    out = precision_leg(args, local, args.batch)
    line = {"metric": "QTAM precision sweep: error vs FP64 oracle and Msamples/s per envelope dtype and short-DFT engine",
            "value": out[0]["msamples_per_s"], "unit": UNIT, "n_gpus": 1, "dtype": "f32 compute",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "segments": args.batch}, "precision": out}
    print(json.dumps(line), flush=True)


def run_latency(args, local):
    """Single-segment forward+inverse latency: the 4 s FP64 case (white noise +
    sine-Gaussian, Q=8, 64 rows 20-1024 Hz) and one 64 s FP32 segment."""
    import torch
    from paper_2603_29785_gb300 import qtam, synth, tune as qtune
    torch.cuda.set_device(local)
    cases = [("4 s @ 4096 Hz, Q=8, 64 rows, FP64", dict(fs=4096.0, N=16384, qs=(8.0,), fmin=20.0, fmax=1024.0, K=64),
              "f64", synth.white_sine_gaussian_segment(0).astype(np.float64)),
             ("64 s @ 4096 Hz, Q {4..64}, 128 rows, FP32", WORKLOAD, "f32", make_inputs([0])[0])]
    res = []
    st = torch.cuda.current_stream()
    for name, w, dt, xn in cases:
        p = qtam.Plan(w["fs"], w["N"], w["qs"], w["fmin"], w["fmax"], w["K"], compute=dt, device=local)
        if dt == "f32":
            qtune.tune(p, 1)
        x = torch.from_numpy(xn[None]).cuda()
        y = p.forward(x)
        xh = p.inverse(y)
        ts = []
        for i in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            p.forward(x, y)
            p.inverse(y, x=xh)
            e1.record(st)
            e1.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        res.append({"case": name, "dtype": dt, "median_ms": round(float(np.median(ts)), 4),
                    "p99_ms": round(float(np.percentile(ts, 99)), 4), "M": p.M})
    line = {"metric": "QTAM single-segment fwd+inv latency", "value": res[0]["median_ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "latency": res}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batched":
        return run_batched(args, local) if rank == 0 else None
    if args.workload == "serving":
        return run_serving(args, local) if rank == 0 else None
    if args.workload == "precision":
        return run_precision(args, local) if rank == 0 else None
    if args.workload == "bank":
        return run_bank(args, local) if rank == 0 else None
    if args.workload == "dense":
        return run_dense(args, local) if rank == 0 else None
    if args.workload == "stream":
        return run_stream(args, local) if rank == 0 else None
    if args.workload == "latency":
        return run_latency(args, local) if rank == 0 else None
    run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
