"""ctypes binding of libqtam.so (the C ABI declared in include/qtam.h).

Argument marshalling only: every step of the transforms runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  The
module-level functions carry the C names (``qtam_plan``, ``qtam_forward``,
``qtam_inverse`` ...); ``Plan`` wraps them with output allocation.

If the library cannot be loaded (not built, or built for another machine)
every entry point raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

QTAM_OK = 0
STATUS = {
    0: "QTAM_OK", 1: "QTAM_ERR_INVALID_ARG", 2: "QTAM_ERR_UNSUPPORTED_SIZE", 3: "QTAM_ERR_ALIASING",
    4: "QTAM_ERR_NO_COVERAGE", 5: "QTAM_ERR_OUT_OF_MEMORY", 6: "QTAM_ERR_CUDA", 7: "QTAM_ERR_TIMEOUT",
    8: "QTAM_ERR_NO_DEVICE", 9: "QTAM_ERR_WORKSPACE",
}
NORM = {"l2": 0, "paper": 1, "none": 2}
WINDOW = {"bisquare": 0, "hann": 1, "kaiser": 2, "tukey": 3, "planck": 4}
SHORT_DFT = {"cuda": 0, "tensor": 1, "auto": 2}
DTYPE = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}
ENV_BYTES = {"f32": 8, "f64": 16, "bf16": 4, "f16": 4}


class QtamError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class qtam_plan_desc(ctypes.Structure):
    _fields_ = [
        ("sample_rate", ctypes.c_double), ("length", ctypes.c_int64), ("q", ctypes.POINTER(ctypes.c_double)),
        ("n_q", ctypes.c_int32), ("f_min", ctypes.c_double), ("f_max", ctypes.c_double),
        ("rows_per_plane", ctypes.c_int32), ("window", ctypes.c_int32), ("norm", ctypes.c_int32),
        ("q_width", ctypes.c_double), ("max_window_hz", ctypes.c_double), ("n_out", ctypes.c_int32),
        ("compute_dtype", ctypes.c_int32), ("envelope_dtype", ctypes.c_int32), ("p_floor_rel", ctypes.c_double),
        ("window_param", ctypes.c_double), ("plane_window", ctypes.POINTER(ctypes.c_int32)),
        ("plane_window_param", ctypes.POINTER(ctypes.c_double)), ("short_dft", ctypes.c_int32),
        ("stopband_eps", ctypes.c_double), ("remodulate", ctypes.c_int32),
    ]


class qtam_stream_info_t(ctypes.Structure):
    _fields_ = [
        ("hop", ctypes.c_int64), ("guard", ctypes.c_int64), ("quantum", ctypes.c_int64),
        ("hop_cols", ctypes.c_int32), ("guard_cols", ctypes.c_int32), ("max_chunks", ctypes.c_int64),
        ("samples_in", ctypes.c_int64), ("columns_in", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
    ]


class qtam_group(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("input", ctypes.c_void_p), ("output", ctypes.c_void_p),
                ("batch", ctypes.c_int64)]


class qtam_plan_info_t(ctypes.Structure):
    _fields_ = [
        ("length", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("n_planes", ctypes.c_int32),
        ("rows_per_plane", ctypes.c_int32), ("n_out", ctypes.c_int32), ("h_max", ctypes.c_int32),
        ("max_window", ctypes.c_int32), ("compute_dtype", ctypes.c_int32), ("envelope_dtype", ctypes.c_int32),
        ("fft_n1", ctypes.c_int32), ("fft_n2", ctypes.c_int32), ("envelope_bytes_per_segment", ctypes.c_int64),
        ("band_bins", ctypes.c_int64), ("p_floor_rel", ctypes.c_double), ("kappa", ctypes.c_double),
        ("kept_bins", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("row_variant", ctypes.c_int32),
        ("short_dft", ctypes.c_int32), ("stopband_eps", ctypes.c_double), ("remodulate", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
SIGNATURES = {
    "qtam_plan_desc_init": (None, [ctypes.POINTER(qtam_plan_desc)]),
    "qtam_plan": (ctypes.c_int, [ctypes.POINTER(qtam_plan_desc), ctypes.c_int, ctypes.POINTER(_P)]),
    "qtam_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(qtam_plan_info_t)]),
    "qtam_plan_rows": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "qtam_frame_operator": (ctypes.c_int, [_P, _U64, _P]),
    "qtam_workspace_size": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_SZ)]),
    "qtam_plan_variants": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "qtam_plan_set_variant": (ctypes.c_int, [_P, ctypes.c_int32]),
    "qtam_variant_describe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_char_p, _SZ, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "qtam_forward": (ctypes.c_int, [_P, _P, _I64, _P, _P, _SZ, _P]),
    "qtam_inverse": (ctypes.c_int, [_P, _P, _I64, _U64, _P, _P, _SZ, _P]),
    "qtam_stage_spectrum": (ctypes.c_int, [_P, _P, _I64, _P, _P, _SZ, _P]),
    "qtam_stage_envelopes": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "qtam_stage_accumulate": (ctypes.c_int, [_P, _P, _I64, _U64, _P, _P]),
    "qtam_stage_synthesize": (ctypes.c_int, [_P, _P, _I64, _U64, _P, _P, _SZ, _P]),
    "qtam_roundtrip_host": (ctypes.c_int, [_P, _P, _I64, _U64, _P, _P, _P, _P, _P, _SZ, _P]),
    "qtam_inverse_single_tile": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int32, ctypes.c_int32, _P, _P, _SZ, _P]),
    "qtam_forward_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "qtam_scale_rows": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "qtam_plane_metrics": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "qtam_batched_workspace_size": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_SZ)]),
    "qtam_forward_batched": (ctypes.c_int, [_P, ctypes.c_int32, _P, _SZ, _P]),
    "qtam_inverse_batched": (ctypes.c_int, [_P, ctypes.c_int32, _U64, _P, _SZ, _P]),
    "qtam_stream_create": (ctypes.c_int, [_P, _I64, _I64, ctypes.POINTER(_P)]),
    "qtam_stream_info": (ctypes.c_int, [_P, ctypes.POINTER(qtam_stream_info_t)]),
    "qtam_stream_forward": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "qtam_stream_inverse": (ctypes.c_int, [_P, _P, _I64, _U64, _P, _P]),
    "qtam_stream_reset": (ctypes.c_int, [_P, _P]),
    "qtam_stream_destroy": (ctypes.c_int, [_P]),
    "qtam_tc_gemm_check": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
    "qtam_tc_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "qtam_destroy": (ctypes.c_int, [_P]),
    "qtam_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qtam_last_error": (ctypes.c_char_p, []),
}


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libqtam.so (building it in-tree first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.lib_path()
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libqtam.so not found at {path}; run paper_2603_29785_gb300/build.py")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(status: int):
    if status != QTAM_OK:
        raise QtamError(status, lib().qtam_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(f"cannot pass {type(t)} as a pointer")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------------------
# C-named entry points (thin marshalling)
# ----------------------------------------------------------------------------
def make_desc(sample_rate, length, qs, f_min, f_max, rows_per_plane, norm="l2", q_width=0.0, max_window_hz=0.0,
              n_out=0, compute="f32", envelope=None, p_floor_rel=-1.0, window="bisquare", window_param=0.0,
              short_dft="cuda", stopband_eps=0.0, remodulate=False):
    d = qtam_plan_desc()
    lib().qtam_plan_desc_init(ctypes.byref(d))
    qarr = (ctypes.c_double * len(qs))(*[float(q) for q in qs])
    d.sample_rate = float(sample_rate)
    d.length = int(length)
    d.q = ctypes.cast(qarr, ctypes.POINTER(ctypes.c_double))
    d.n_q = len(qs)
    d.f_min, d.f_max = float(f_min), float(f_max)
    d.rows_per_plane = int(rows_per_plane)
    d.norm = NORM[norm]
    d.q_width = float(q_width)
    d.max_window_hz = float(max_window_hz)
    d.n_out = int(n_out)
    d.compute_dtype = DTYPE[compute]
    d.envelope_dtype = DTYPE[envelope or compute]
    d.p_floor_rel = float(p_floor_rel)
    keep = [qarr]  # arrays the struct points to live as long as the struct
    if isinstance(window, str):
        d.window = WINDOW[window]
    else:                      # composite bank: one window per plane
        warr = (ctypes.c_int32 * len(window))(*[WINDOW[w] for w in window])
        d.plane_window = ctypes.cast(warr, ctypes.POINTER(ctypes.c_int32))
        keep.append(warr)
        if len(window) != len(qs):
            raise ValueError("one window per plane is required")
    if np.ndim(window_param) == 0:
        d.window_param = float(window_param)
    else:
        parr = (ctypes.c_double * len(window_param))(*[float(a) for a in window_param])
        d.plane_window_param = ctypes.cast(parr, ctypes.POINTER(ctypes.c_double))
        keep.append(parr)
        if len(window_param) != len(qs):
            raise ValueError("one window parameter per plane is required")
    d.short_dft = SHORT_DFT[short_dft]
    d.stopband_eps = float(stopband_eps)
    d.remodulate = int(bool(remodulate))
    d._keep = keep
    return d


def qtam_plan(desc: qtam_plan_desc, device: int) -> int:
    h = _P()
    _check(lib().qtam_plan(ctypes.byref(desc), int(device), ctypes.byref(h)))
    return h.value


def qtam_plan_info(plan) -> dict:
    o = qtam_plan_info_t()
    _check(lib().qtam_plan_info(plan, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in qtam_plan_info_t._fields_}


def qtam_plan_rows(plan, n_rows: int) -> dict:
    f = np.zeros(n_rows, np.float64)
    kc = np.zeros(n_rows, np.int64)
    h = np.zeros(n_rows, np.int32)
    c = np.zeros(n_rows, np.float64)
    _check(lib().qtam_plan_rows(plan, f.ctypes.data, kc.ctypes.data, h.ctypes.data, c.ctypes.data))
    return {"f": f, "kc": kc, "h": h, "c": c}


def qtam_frame_operator(plan, plane_mask: int, n_bins: int) -> np.ndarray:
    out = np.zeros(n_bins, np.float64)
    _check(lib().qtam_frame_operator(plan, int(plane_mask), out.ctypes.data))
    return out


def qtam_workspace_size(plan, batch: int) -> int:
    s = _SZ()
    _check(lib().qtam_workspace_size(plan, int(batch), ctypes.byref(s)))
    return s.value


def qtam_plan_variants(plan) -> list[int]:
    n = ctypes.c_int32()
    _check(lib().qtam_plan_variants(plan, None, 0, ctypes.byref(n)))
    ids = np.zeros(max(1, n.value), np.int32)
    _check(lib().qtam_plan_variants(plan, ids.ctypes.data, n.value, ctypes.byref(n)))
    return [int(v) for v in ids[: n.value]]


def qtam_plan_set_variant(plan, variant: int):
    _check(lib().qtam_plan_set_variant(plan, int(variant)))


def qtam_variant_describe(variant: int) -> dict:
    buf = ctypes.create_string_buffer(128)
    t, r = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().qtam_variant_describe(int(variant), buf, 128, ctypes.byref(t), ctypes.byref(r)))
    return {"id": int(variant), "name": buf.value.decode(), "threads": t.value, "rows_per_block": r.value}


def qtam_forward(plan, x, batch, y, workspace, workspace_bytes, stream=None):
    _check(lib().qtam_forward(plan, _ptr(x), int(batch), _ptr(y), _ptr(workspace), int(workspace_bytes), _stream(stream)))


def qtam_inverse(plan, y, batch, plane_mask, x, workspace, workspace_bytes, stream=None):
    _check(lib().qtam_inverse(plan, _ptr(y), int(batch), int(plane_mask), _ptr(x), _ptr(workspace),
                              int(workspace_bytes), _stream(stream)))


def qtam_inverse_single_tile(plan, y, batch, plane, row, x, workspace, workspace_bytes, stream=None):
    _check(lib().qtam_inverse_single_tile(plan, _ptr(y), int(batch), int(plane), int(row), _ptr(x), _ptr(workspace),
                                          int(workspace_bytes), _stream(stream)))


def qtam_stage_spectrum(plan, x, batch, X, workspace, workspace_bytes, stream=None):
    _check(lib().qtam_stage_spectrum(plan, _ptr(x), int(batch), _ptr(X), _ptr(workspace), int(workspace_bytes),
                                     _stream(stream)))


def qtam_stage_envelopes(plan, X, batch, y, stream=None):
    _check(lib().qtam_stage_envelopes(plan, _ptr(X), int(batch), _ptr(y), _stream(stream)))


def qtam_stage_accumulate(plan, y, batch, plane_mask, A, stream=None):
    _check(lib().qtam_stage_accumulate(plan, _ptr(y), int(batch), int(plane_mask), _ptr(A), _stream(stream)))


def qtam_stage_synthesize(plan, A, batch, plane_mask, x, workspace, workspace_bytes, stream=None):
    _check(lib().qtam_stage_synthesize(plan, _ptr(A), int(batch), int(plane_mask), _ptr(x), _ptr(workspace),
                                       int(workspace_bytes), _stream(stream)))


def qtam_roundtrip_host(plan, x_host, batch, plane_mask, xhat_host, x_dev, y_dev, xhat_dev, workspace,
                        workspace_bytes, stream=None):
    _check(lib().qtam_roundtrip_host(plan, _ptr(x_host), int(batch), int(plane_mask), _ptr(xhat_host), _ptr(x_dev),
                                     _ptr(y_dev), _ptr(xhat_dev), _ptr(workspace), int(workspace_bytes),
                                     _stream(stream)))


def qtam_forward_noalloc(plan, x, batch, y, stream=None):
    """qtam_forward with the library's fixed scratch array instead of a
    caller workspace (for callers that cannot allocate at call time)."""
    _check(lib().qtam_forward_noalloc(plan, _ptr(x), int(batch), _ptr(y), _stream(stream)))


def qtam_plane_metrics(plan, y, batch, energy, peak, stream=None):
    _check(lib().qtam_plane_metrics(plan, _ptr(y), int(batch), _ptr(energy), _ptr(peak), _stream(stream)))


def qtam_scale_rows(plan, y, batch, gain, stream=None):
    _check(lib().qtam_scale_rows(plan, _ptr(y), int(batch), _ptr(gain), _stream(stream)))


def make_groups(groups) -> ctypes.Array:
    """groups: iterable of (plan handle, input tensor/pointer, output tensor/pointer, batch)."""
    groups = list(groups)
    arr = (qtam_group * max(1, len(groups)))()
    for i, (plan, inp, out, batch) in enumerate(groups):
        arr[i].plan = plan
        arr[i].input = _ptr(inp)
        arr[i].output = _ptr(out)
        arr[i].batch = int(batch)
    return arr, len(groups)


def qtam_batched_workspace_size(groups) -> int:
    arr, n = make_groups(groups)
    s = _SZ()
    _check(lib().qtam_batched_workspace_size(arr, n, ctypes.byref(s)))
    return s.value


def qtam_forward_batched(groups, workspace, workspace_bytes, stream=None):
    arr, n = make_groups(groups)
    _check(lib().qtam_forward_batched(arr, n, _ptr(workspace), int(workspace_bytes), _stream(stream)))


def qtam_inverse_batched(groups, plane_mask, workspace, workspace_bytes, stream=None):
    arr, n = make_groups(groups)
    _check(lib().qtam_inverse_batched(arr, n, int(plane_mask), _ptr(workspace), int(workspace_bytes),
                                      _stream(stream)))


def qtam_destroy(plan):
    if plan:
        lib().qtam_destroy(plan)


def qtam_stream_create(plan, hop: int = 0, max_chunks: int = 8) -> int:
    h = _P()
    _check(lib().qtam_stream_create(plan, int(hop), int(max_chunks), ctypes.byref(h)))
    return h.value


def qtam_stream_info(s) -> dict:
    o = qtam_stream_info_t()
    _check(lib().qtam_stream_info(s, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in qtam_stream_info_t._fields_}


def qtam_stream_forward(s, x, n, y, stream=None):
    _check(lib().qtam_stream_forward(s, _ptr(x), int(n), _ptr(y), _stream(stream)))


def qtam_stream_inverse(s, y, n_cols, plane_mask, x, stream=None):
    _check(lib().qtam_stream_inverse(s, _ptr(y), int(n_cols), int(plane_mask), _ptr(x), _stream(stream)))


def qtam_stream_reset(s, stream=None):
    _check(lib().qtam_stream_reset(s, _stream(stream)))


def qtam_stream_destroy(s):
    if s:
        lib().qtam_stream_destroy(s)


def qtam_tc_gemm_check(A, B, D, N, K, flags=0, stream=None):
    _check(lib().qtam_tc_gemm_check(_ptr(A), _ptr(B), _ptr(D), int(N), int(K), int(flags), _stream(stream)))


def qtam_tc_status() -> int:
    v = ctypes.c_int32()
    _check(lib().qtam_tc_status(ctypes.byref(v)))
    return v.value


def qtam_status_string(status: int) -> str:
    return lib().qtam_status_string(int(status)).decode()


def _require(t, shape, dtypes, device, name):
    """Reject a tensor whose shape, dtype, device or layout does not match
    what the C entry point will read or write (the ABI sees raw pointers)."""
    ok = (hasattr(t, "is_cuda") and t.is_cuda and t.device.index == device and t.dtype in dtypes
          and t.is_contiguous() and t.dim() == len(shape)
          and all(s is None or int(d) == s for d, s in zip(t.shape, shape)))
    if not ok:
        want = "[" + ", ".join("batch" if s is None else str(s) for s in shape) + "]"
        got = (tuple(t.shape), getattr(t, "dtype", None), getattr(t, "device", None)) if hasattr(t, "shape") else type(t)
        raise ValueError(f"{name} must be a contiguous cuda:{device} tensor {want} of {dtypes}; got {got}")


# ----------------------------------------------------------------------------
# convenience wrapper
# ----------------------------------------------------------------------------
@dataclass
class Geometry:
    f: np.ndarray
    kc: np.ndarray
    h: np.ndarray
    c: np.ndarray


class Plan:
    """A QTAM plan on one device, with torch-allocated outputs and workspace.

    Plan(sample_rate, length, qs, f_min, f_max, rows_per_plane, ...,
         compute="f32" | "f64", envelope="f32" | "bf16" | "f16" | "f64",
         device=0)   (device=-1: host-only, geometry queries only)
    """

    def __init__(self, sample_rate, length, qs, f_min, f_max, rows_per_plane, norm="l2", q_width=0.0,
                 max_window_hz=0.0, n_out=0, compute="f32", envelope=None, p_floor_rel=-1.0, device=0,
                 window="bisquare", window_param=0.0, short_dft="cuda", stopband_eps=0.0, remodulate=False):
        self.compute = compute
        self.envelope = envelope or compute
        self.device = int(device)
        self._desc = make_desc(sample_rate, length, qs, f_min, f_max, rows_per_plane, norm, q_width, max_window_hz,
                               n_out, compute, self.envelope, p_floor_rel, window, window_param, short_dft,
                               stopband_eps, remodulate)
        self.handle = qtam_plan(self._desc, self.device)
        self.info = qtam_plan_info(self.handle)
        self.N = self.info["length"]
        self.Nr = self.info["n_bins"]
        self.P = self.info["n_planes"]
        self.K = self.info["rows_per_plane"]
        self.M = self.info["n_out"]
        r = qtam_plan_rows(self.handle, self.P * self.K)
        shp = (self.P, self.K)
        self.geometry = Geometry(r["f"].reshape(shp), r["kc"].reshape(shp), r["h"].reshape(shp), r["c"].reshape(shp))
        self._ws = {}

    def __del__(self):
        try:
            qtam_destroy(self.handle)
        except Exception:
            pass

    # -- helpers ------------------------------------------------------------
    def frame_operator(self, plane_mask: int = 0) -> np.ndarray:
        return qtam_frame_operator(self.handle, plane_mask, self.Nr)

    def workspace(self, batch: int):
        import torch
        need = qtam_workspace_size(self.handle, batch)
        ws = self._ws.get(self.device)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
            self._ws[self.device] = ws
        return ws, ws.numel()

    def real_dtype(self):
        import torch
        return torch.float64 if self.compute == "f64" else torch.float32

    def envelope_tensor(self, batch: int):
        import torch
        dev = f"cuda:{self.device}"
        shp = (batch, self.P, self.K, self.M)
        if self.envelope == "f32":
            return torch.empty(shp, dtype=torch.complex64, device=dev)
        if self.envelope == "f64":
            return torch.empty(shp, dtype=torch.complex128, device=dev)
        dt = torch.bfloat16 if self.envelope == "bf16" else torch.float16
        return torch.empty(shp + (2,), dtype=dt, device=dev)

    def _check_x(self, x):
        if x.dim() == 1:
            x = x.unsqueeze(0)
        _require(x, (None, self.N), (self.real_dtype(),), self.device, "x")
        return x

    def complex_dtype(self):
        import torch
        return torch.complex128 if self.compute == "f64" else torch.complex64

    def _check_y(self, y):
        import torch
        if self.envelope in ("bf16", "f16"):
            dt = torch.bfloat16 if self.envelope == "bf16" else torch.float16
            _require(y, (None, self.P, self.K, self.M, 2), (dt,), self.device, "y")
        else:
            _require(y, (None, self.P, self.K, self.M), (self.complex_dtype(),), self.device, "y")
        return y

    def _check_spec(self, X, name):
        _require(X, (None, self.Nr), (self.complex_dtype(),), self.device, name)
        return X

    # -- transforms ---------------------------------------------------------
    def forward(self, x, y=None, stream=None):
        x = self._check_x(x)
        B = x.shape[0]
        y = self.envelope_tensor(B) if y is None else self._check_y(y)
        if y.shape[0] != B:
            raise ValueError("x and y batch sizes differ")
        ws, wsb = self.workspace(B)
        qtam_forward(self.handle, x, B, y, ws, wsb, stream)
        return y

    def inverse(self, y, plane_mask: int = 0, x=None, stream=None):
        import torch
        self._check_y(y)
        B = y.shape[0]
        x = torch.empty((B, self.N), dtype=self.real_dtype(), device=y.device) if x is None else self._check_x(x)
        if x.shape[0] != B:
            raise ValueError("x and y batch sizes differ")
        ws, wsb = self.workspace(B)
        qtam_inverse(self.handle, y, B, plane_mask, x, ws, wsb, stream)
        return x

    def inverse_single_tile(self, y, plane: int, row: int, x=None, stream=None):
        """Dense mode: reconstruct every segment from its one tile (plane, row)."""
        import torch
        self._check_y(y)
        B = y.shape[0]
        x = torch.empty((B, self.N), dtype=self.real_dtype(), device=y.device) if x is None else self._check_x(x)
        ws, wsb = self.workspace(B)
        qtam_inverse_single_tile(self.handle, y, B, plane, row, x, ws, wsb, stream)
        return x

    def plane_metrics(self, y, stream=None):
        """(energy [B, P] float64, peak [B, P] float32, best plane by energy [B],
        best plane by peak [B]) -- optimal-plane selection per segment."""
        import torch
        self._check_y(y)
        B = y.shape[0]
        energy = torch.empty((B, self.P), dtype=torch.float64, device=y.device)
        peak = torch.empty((B, self.P), dtype=torch.float32, device=y.device)
        qtam_plane_metrics(self.handle, y, B, energy, peak, stream)
        return energy, peak, energy.argmax(dim=1), peak.argmax(dim=1)

    def scale_rows(self, y, gain, stream=None):
        """y[b, p, k, :] *= gain[b, p, k] in place (gain: CUDA float32 [batch, P, K])."""
        self._check_y(y)
        B = y.shape[0]
        _require(gain, (B, self.P, self.K), (__import__("torch").float32,), self.device, "gain")
        qtam_scale_rows(self.handle, y, B, gain, stream)
        return y

    def spectrum(self, x, stream=None):
        import torch
        x = self._check_x(x)
        B = x.shape[0]
        cdt = torch.complex128 if self.compute == "f64" else torch.complex64
        X = torch.empty((B, self.Nr), dtype=cdt, device=x.device)
        ws, wsb = self.workspace(B)
        qtam_stage_spectrum(self.handle, x, B, X, ws, wsb, stream)
        return X

    def envelopes(self, X, stream=None):
        self._check_spec(X, "X")
        B = X.shape[0]
        y = self.envelope_tensor(B)
        qtam_stage_envelopes(self.handle, X, B, y, stream)
        return y

    def accumulate(self, y, plane_mask: int = 0, stream=None):
        import torch
        self._check_y(y)
        B = y.shape[0]
        A = torch.empty((B, self.Nr), dtype=self.complex_dtype(), device=y.device)
        qtam_stage_accumulate(self.handle, y, B, plane_mask, A, stream)
        return A

    def synthesize(self, A, plane_mask: int = 0, stream=None):
        import torch
        self._check_spec(A, "A")
        B = A.shape[0]
        x = torch.empty((B, self.N), dtype=self.real_dtype(), device=A.device)
        ws, wsb = self.workspace(B)
        qtam_stage_synthesize(self.handle, A, B, plane_mask, x, ws, wsb, stream)
        return x


class Stream:
    """Overlap-save streaming over a continuous signal with a device plan.

    Stream(plan, hop=0, max_chunks=8): hop = 0 picks N/2 on the column
    quantum grid.  forward(x) takes a 1-D device tensor of a multiple of hop
    samples and returns the new map columns [P, K, n/hop*Hn]; inverse(y)
    takes map columns and returns samples.  Map column c of the whole stream
    is time c*N/M - guard; inverse sample s is time s - 2*guard.
    """

    def __init__(self, plan: Plan, hop: int = 0, max_chunks: int = 8):
        self.plan = plan
        self.handle = qtam_stream_create(plan.handle, hop, max_chunks)
        self.info = qtam_stream_info(self.handle)
        self.hop = self.info["hop"]
        self.guard = self.info["guard"]
        self.hop_cols = self.info["hop_cols"]

    def __del__(self):
        try:
            qtam_stream_destroy(self.handle)
        except Exception:
            pass

    def _map_tensor(self, cols):
        import torch
        p = self.plan
        dev = f"cuda:{p.device}"
        shp = (p.P, p.K, cols)
        if p.envelope == "f32":
            return torch.empty(shp, dtype=torch.complex64, device=dev)
        if p.envelope == "f64":
            return torch.empty(shp, dtype=torch.complex128, device=dev)
        dt = torch.bfloat16 if p.envelope == "bf16" else torch.float16
        return torch.empty(shp + (2,), dtype=dt, device=dev)

    def forward(self, x, stream=None):
        p = self.plan
        _require(x, (None,), (p.real_dtype(),), p.device, "x")
        n = int(x.shape[0])
        if n % self.hop:
            raise ValueError(f"push a multiple of hop = {self.hop} samples; got {n}")
        y = self._map_tensor(n // self.hop * self.hop_cols)
        qtam_stream_forward(self.handle, x, n, y, stream)
        return y

    def inverse(self, y, plane_mask: int = 0, stream=None):
        import torch
        p = self.plan
        if p.envelope in ("bf16", "f16"):
            dt = torch.bfloat16 if p.envelope == "bf16" else torch.float16
            _require(y, (p.P, p.K, None, 2), (dt,), p.device, "y")
        else:
            _require(y, (p.P, p.K, None), (p.complex_dtype(),), p.device, "y")
        cols = int(y.shape[2])
        if cols % self.hop_cols:
            raise ValueError(f"push a multiple of {self.hop_cols} map columns; got {cols}")
        x = torch.empty((cols // self.hop_cols * self.hop,), dtype=p.real_dtype(), device=y.device)
        qtam_stream_inverse(self.handle, y, cols, plane_mask, x, stream)
        return x

    def reset(self, stream=None):
        qtam_stream_reset(self.handle, stream)


def header_symbols(header_path: str | None = None) -> list[str]:
    """Names of the functions include/qtam.h declares."""
    import re
    if header_path is None:
        header_path = os.path.join(_build.ROOT, "include", "qtam.h")
    txt = open(header_path).read()
    return sorted(set(re.findall(r"QTAM_API\s+[\w\s\*]+?\b(qtam_\w+)\s*\(", txt)))
