"""GB300-native running max-min filter: Python binding of ``libmmf.so``.

This module only marshals arguments for the C ABI declared in
``include/mmf.h``; every step of the filter runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or the tensors are not on a CUDA device,
calls raise.

Build the library with ``python -m paper_cs_0610046_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = ["MMFError", "load", "filter1d", "filter1d_host", "filter1d_w3", "argfilter1d", "output_length",
           "device_status", "set_wait_fault", "dispatch_set", "dispatch_get", "dispatch_autotune", "BatchPlan", "filter2d", "filter2d_workspace", "Server", "n_outputs", "DTYPES", "KERNELS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
# MMF_CHECKED=1 selects the range-checked build (see build.py).
LIB_PATH = os.path.join(_HERE, "libmmf_checked.so" if os.environ.get("MMF_CHECKED") == "1" else "libmmf.so")

MMF_OK = 0
STATUS_NAMES = {0: "MMF_OK", 1: "MMF_EINVAL", 2: "MMF_ENOMEM", 3: "MMF_ECUDA", 4: "MMF_EBUSY",
                5: "MMF_ETIMEOUT", 6: "MMF_ECLOSED", 7: "MMF_ENOTIMPL", 8: "MMF_EDEVICE"}
DTYPES = {torch.float32: 0, torch.float64: 1, torch.int16: 2, torch.uint8: 3}
MODES = {"valid": 0, "envelope": 1, "centered_clipped": 1}
KERNELS = {"auto": 0, "blockscan": 1, "slide": 2, "wedge": 3, "front": 4}

_I64 = ctypes.c_int64
_VP = ctypes.c_void_p
_INT = ctypes.c_int

_lock = threading.Lock()
_lib = None


class MMFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load ``libmmf.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                                   "`python -m paper_cs_0610046_gb300.build`")
            lib = ctypes.CDLL(LIB_PATH)
            lib.mmf_last_error.restype = ctypes.c_char_p
            lib.mmf_version.restype = ctypes.c_char_p
            lib.mmf_output_length.argtypes = [_I64, _I64, _INT]
            lib.mmf_output_length.restype = _I64
            lib.mmf_filter1d.argtypes = [_VP, _I64, _I64, _INT, _INT, _VP, _VP, _VP]
            lib.mmf_filter1d.restype = _INT
            lib.mmf_filter1d_ex.argtypes = [_VP, _I64, _I64, _INT, _INT, _VP, _VP, _VP, _INT]
            lib.mmf_filter1d_ex.restype = _INT
            lib.mmf_device_status.argtypes = [ctypes.POINTER(ctypes.c_uint32), _INT]
            lib.mmf_device_status.restype = _INT
            _declare_more(lib)
            _lib = lib
    return _lib


def _declare_more(lib) -> None:
    """Signatures of the entry points added beyond the 1D filter."""
    for name, args in _EXTRA_SIGNATURES.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = args[0]
            f.restype = args[1]


_P64 = ctypes.POINTER(ctypes.c_int64)
_EXTRA_SIGNATURES: dict = {
    "mmf_batch_plan_create": ([_P64, _P64, _P64, _I64, _INT, _INT, ctypes.POINTER(_VP)], _INT),
    "mmf_batch_plan_destroy": ([_VP], None),
    "mmf_batch_plan_out_offsets": ([_VP, _P64], _INT),
    "mmf_batch_plan_sizes": ([_VP, _P64, _P64, _P64], _INT),
    "mmf_batch_plan_set_segment": ([_VP, _INT, _INT], _INT),
    "mmf_batch_plan_get_segment": ([_VP, _INT, ctypes.POINTER(_INT)], _INT),
    "mmf_batch_plan_autotune": ([_VP, _VP, _VP, _VP, _VP], _INT),
    "mmf_filter1d_batched": ([_VP, _VP, _VP, _VP, _VP], _INT),
    "mmf_filter1d_per_series": ([_VP, _VP, _VP, _VP, _VP], _INT),
    "mmf_lb_keogh_batched": ([_VP, _VP, _VP, _I64, _VP, _VP], _INT),
    "mmf_server_create": ([ctypes.c_size_t, _INT, _INT, ctypes.POINTER(_VP)], _INT),
    "mmf_server_destroy": ([_VP], None),
    "mmf_stream_open": ([_VP, _I64, ctypes.POINTER(ctypes.c_uint64)], _INT),
    "mmf_stream_push": ([_VP, ctypes.c_uint64, _VP, _I64, _VP, _VP, _P64, ctypes.POINTER(ctypes.c_uint64)], _INT),
    "mmf_ticket_wait": ([_VP, ctypes.c_uint64, _INT], _INT),
    "mmf_stream_push_batch": ([_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _P64], _INT),
    "mmf_ticket_wait_batch": ([_VP, _I64, _VP, _INT], _INT),
    "mmf_stream_close": ([_VP, ctypes.c_uint64, _INT], _INT),
    "mmf_filter1d_host": ([_VP, _I64, _I64, _INT, _INT, _VP, _VP, _I64, _VP], _INT),
    "mmf_argfilter1d": ([_VP, _I64, _I64, _INT, _VP, _VP, _VP, _VP, _VP], _INT),
    "mmf_argfilter1d_ex": ([_VP, _I64, _I64, _INT, _VP, _VP, _VP, _VP, _VP, _INT], _INT),
    "mmf_filter1d_w3": ([_VP, _I64, _INT, _VP, _VP, _VP, _VP], _INT),
    "mmf_stream_snapshot": ([_VP, ctypes.c_uint64, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _INT], _INT),
    "mmf_stream_snapshot_wedge": ([_VP, ctypes.c_uint64, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _INT],
                                  _INT),
    "mmf_stream_restore": ([_VP, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)], _INT),
    "mmf_server_pause": ([_VP, _INT], _INT),
    "mmf_test_set_wait_fault": ([_INT, _I64], _INT),
    "mmf_test_set_input_clip": ([_I64], _INT),
    "mmf_dispatch_set": ([_INT, _I64, _I64, _INT], _INT),
    "mmf_dispatch_get": ([_INT, _I64, _I64, ctypes.POINTER(_INT)], _INT),
    "mmf_dispatch_autotune": ([_VP, _I64, _I64, _INT, _VP, _VP, _VP, ctypes.POINTER(_INT)], _INT),
    "mmf_batch_plan_set_knobs": ([_VP, _I64, _INT], _INT),
    "mmf_batch_plan_get_knobs": ([_VP, _P64, ctypes.POINTER(_INT)], _INT),
    "mmf_filter2d_workspace": ([_I64, _I64, _I64, _I64, _I64, _INT, _INT, ctypes.POINTER(ctypes.c_size_t)], _INT),
    "mmf_filter2d_separable": ([_VP, _I64, _I64, _I64, _I64, _I64, _I64, _INT, _INT, _VP, _VP, _VP,
                                ctypes.c_size_t, _VP], _INT),
}


def check(status: int) -> None:
    if status != MMF_OK:
        raise MMFError(status, load().mmf_last_error().decode(errors="replace"))


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensor(t: torch.Tensor, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in DTYPES:
        raise TypeError(f"{name}: unsupported dtype {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def output_length(n: int, w_or_r: int, mode: str = "valid") -> int:
    return int(load().mmf_output_length(n, w_or_r, MODES[mode]))


def filter1d(x: torch.Tensor, w: int, mode: str = "valid", out_max=None, out_min=None,
             kernel: str = "auto", stream=None, want_max: bool = True, want_min: bool = True):
    """Running max and min of every window of ``x`` (1D, CUDA tensor).

    ``mode="valid"``: windows [j, j+w), n-w+1 outputs.  ``mode="envelope"``:
    ``w`` is the radius r and the windows are [i-r, i+r] clipped to the array,
    n outputs.  Returns ``(max, min)`` (either may be None if not wanted).
    """
    _check_tensor(x, "x")
    lib = load()
    x = x.reshape(-1)
    m = int(lib.mmf_output_length(x.numel(), w, MODES[mode]))
    if m < 0:
        raise MMFError(1, f"invalid window {w} for mode {mode}")
    if want_max and out_max is None:
        out_max = torch.empty(m, dtype=x.dtype, device=x.device)
    if want_min and out_min is None:
        out_min = torch.empty(m, dtype=x.dtype, device=x.device)
    for o, nm in ((out_max, "out_max"), (out_min, "out_min")):
        if o is not None:
            _check_tensor(o, nm)
            if o.dtype != x.dtype or o.numel() < m:
                raise ValueError(f"{nm} must hold {m} elements of {x.dtype}")
    with torch.cuda.device(x.device):
        check(lib.mmf_filter1d_ex(_ptr(x), x.numel(), w, DTYPES[x.dtype], MODES[mode],
                                  _ptr(out_max), _ptr(out_min), _VP(_stream_handle(stream)),
                                  KERNELS[kernel]))
    return out_max, out_min


def filter1d_host(x: torch.Tensor, w: int, mode: str = "valid", out_max=None, out_min=None, chunk: int = 0,
                  stream=None, device=None):
    """The filter of a HOST (CPU) tensor through the chunked upload / filter /
    download pipeline on ``device`` (default: the current CUDA device).
    Outputs are CPU tensors (pinned memory is fastest); returns (max, min).
    Synchronise ``stream`` (default: the current stream) before reading."""
    if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype not in DTYPES:
        raise TypeError("x must be a CPU tensor of a supported dtype")
    x = x.reshape(-1)
    if not x.is_contiguous():
        raise ValueError("x must be contiguous")
    lib = load()
    m = int(lib.mmf_output_length(x.numel(), w, MODES[mode]))
    if m < 0:
        raise MMFError(1, f"invalid window {w} for mode {mode}")
    if out_max is None:
        out_max = torch.empty(m, dtype=x.dtype, pin_memory=True)
    if out_min is None:
        out_min = torch.empty(m, dtype=x.dtype, pin_memory=True)
    for o in (out_max, out_min):
        if o.is_cuda or o.dtype != x.dtype or o.numel() < m or not o.is_contiguous():
            raise ValueError(f"outputs must be contiguous CPU tensors of {m} elements")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        check(lib.mmf_filter1d_host(ctypes.c_void_p(x.data_ptr()), x.numel(), w, DTYPES[x.dtype], MODES[mode],
                                    ctypes.c_void_p(out_max.data_ptr()), ctypes.c_void_p(out_min.data_ptr()), chunk,
                                    _VP(_stream_handle(stream))))
    return out_max, out_min


def argfilter1d(x: torch.Tensor, w: int, stream=None, out=None, kernel: str = "auto"):
    """Positions (int64) of the maximum and minimum of every window
    [j, j+w) of ``x``, leftmost among equal values, and the values:
    returns ``(argmax, argmin, max, min)``.  ``kernel``: "auto"/"blockscan"
    (any w) or "wedge" (w <= 496).  ``out``: optional tuple of the four
    output tensors (at least n-w+1 elements each)."""
    _check_tensor(x, "x")
    lib = load()
    x = x.reshape(-1)
    m = int(lib.mmf_output_length(x.numel(), w, MODES["valid"]))
    if m < 0:
        raise MMFError(1, f"invalid window {w}")
    if out is not None:
        am, an, vm, vn = out
        for t, dt in ((am, torch.int64), (an, torch.int64), (vm, x.dtype), (vn, x.dtype)):
            if not (t.is_cuda and t.is_contiguous()) or t.dtype != dt or t.numel() < m:
                raise ValueError(f"outputs must be contiguous CUDA tensors of {m} elements ({dt})")
    else:
        am = torch.empty(m, dtype=torch.int64, device=x.device)
        an = torch.empty(m, dtype=torch.int64, device=x.device)
        vm = torch.empty(m, dtype=x.dtype, device=x.device)
        vn = torch.empty(m, dtype=x.dtype, device=x.device)
    with torch.cuda.device(x.device):
        check(lib.mmf_argfilter1d_ex(_ptr(x), x.numel(), w, DTYPES[x.dtype], _ptr(vm), _ptr(vn), _ptr(am), _ptr(an),
                                     _VP(_stream_handle(stream)), KERNELS[kernel]))
    return am, an, vm, vn


def filter1d_w3(x: torch.Tensor, out_max=None, out_min=None, count: bool = False, stream=None):
    """Window-3 max and min by the two-comparison scheme (``mmf_filter1d_w3``):
    returns ``(max, min)``, or ``(max, min, comparisons)`` with ``count``."""
    _check_tensor(x, "x")
    lib = load()
    x = x.reshape(-1)
    m = max(0, x.numel() - 2)
    mx = out_max if out_max is not None else torch.empty(m, dtype=x.dtype, device=x.device)
    mn = out_min if out_min is not None else torch.empty(m, dtype=x.dtype, device=x.device)
    for t in (mx, mn):
        _check_tensor(t, "output")
        if t.dtype != x.dtype or t.numel() < m:
            raise ValueError(f"outputs must be {x.dtype} tensors of at least {m} elements")
    cnt = torch.zeros(1, dtype=torch.int64, device=x.device) if count else None
    with torch.cuda.device(x.device):
        check(lib.mmf_filter1d_w3(_ptr(x), x.numel(), DTYPES[x.dtype], _ptr(mx), _ptr(mn),
                                  _ptr(cnt) if count else None, _VP(_stream_handle(stream))))
    return (mx, mn, cnt) if count else (mx, mn)


def _i64_array(xs):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int64))
    return a, a.ctypes.data_as(_P64)


class BatchPlan:
    """Many independent series in one buffer, filtered by one persistent
    launch per kernel group replayed from a CUDA graph (``mmf_filter1d_batched``).

    ``lengths``/``windows`` per series (windows are radii in envelope mode);
    ``in_offsets`` (optional) places each series in the input buffer, else
    the series are packed back to back."""

    def __init__(self, lengths, windows, dtype=torch.float32, mode: str = "valid", in_offsets=None):
        lib = load()
        self._lib = lib
        self.dtype = dtype
        self.mode = mode
        self._len, plen = _i64_array(lengths)
        self._w, pw = _i64_array(windows)
        if self._len.shape != self._w.shape:
            raise ValueError("lengths and windows differ in size")
        poff = None
        if in_offsets is not None:
            self._off, poff = _i64_array(in_offsets)
        self.nseries = int(self._len.size)
        h = _VP()
        check(lib.mmf_batch_plan_create(poff, plen, pw, self.nseries, DTYPES[dtype], MODES[mode], ctypes.byref(h)))
        self._h = h
        a, b = ctypes.c_int64(), ctypes.c_int64()
        items = (ctypes.c_int64 * 4)()
        check(lib.mmf_batch_plan_sizes(self._h, ctypes.byref(a), ctypes.byref(b), items))
        self.in_len, self.out_len = int(a.value), int(b.value)
        self.items_per_group = list(items)

    def out_offsets(self):
        """Start of each series' outputs, then out_len: series s has its
        n_out outputs from off[s] (on a 32-byte boundary), then padding."""
        import numpy as np
        off = np.zeros(self.nseries + 1, dtype=np.int64)
        check(self._lib.mmf_batch_plan_out_offsets(self._h, off.ctypes.data_as(_P64)))
        return off

    def _check_input(self, x):
        _check_tensor(x, "x")
        if x.dtype != self.dtype or x.numel() < self.in_len:
            raise ValueError(f"input must hold {self.in_len} elements of {self.dtype}")

    def _outs(self, x, out_max, out_min):
        # Zero-filled: the padding between series (outputs start on 32-byte
        # boundaries) is never written and reads as 0.
        if out_max is None:
            out_max = torch.zeros(self.out_len, dtype=x.dtype, device=x.device)
        if out_min is None:
            out_min = torch.zeros(self.out_len, dtype=x.dtype, device=x.device)
        for o, nm in ((out_max, "out_max"), (out_min, "out_min")):
            _check_tensor(o, nm)
            if o.dtype != x.dtype or o.numel() < self.out_len:
                raise ValueError(f"{nm} must hold {self.out_len} elements of {x.dtype}")
        return out_max, out_min

    def __call__(self, x, out_max=None, out_min=None, stream=None):
        self._check_input(x)
        out_max, out_min = self._outs(x, out_max, out_min)
        with torch.cuda.device(x.device):
            check(self._lib.mmf_filter1d_batched(self._h, _ptr(x), _ptr(out_max), _ptr(out_min),
                                                 _VP(_stream_handle(stream))))
        return out_max, out_min

    def per_series(self, x, out_max=None, out_min=None, stream=None):
        """The plain form: one mmf_filter1d launch per series."""
        self._check_input(x)
        out_max, out_min = self._outs(x, out_max, out_min)
        with torch.cuda.device(x.device):
            check(self._lib.mmf_filter1d_per_series(self._h, _ptr(x), _ptr(out_max), _ptr(out_min),
                                                    _VP(_stream_handle(stream))))
        return out_max, out_min

    def lb_keogh(self, x, query, out=None, stream=None):
        """Lower bound of the time-warping distance of ``query`` and every
        series from the series' envelope (an envelope plan whose series all
        have the query's length): float64 tensor of nseries."""
        _check_tensor(x, "x")
        _check_tensor(query, "query")
        if query.dtype != self.dtype or x.dtype != self.dtype:
            raise ValueError(f"x and query must be {self.dtype}")
        if out is None:
            out = torch.empty(self.nseries, dtype=torch.float64, device=x.device)
        elif not (isinstance(out, torch.Tensor) and out.is_cuda and out.is_contiguous()) or \
                out.dtype != torch.float64 or out.numel() < self.nseries:
            raise ValueError(f"out must be a contiguous CUDA tensor of {self.nseries} float64 values")
        with torch.cuda.device(x.device):
            check(self._lib.mmf_lb_keogh_batched(self._h, _ptr(x), _ptr(query), query.numel(), _ptr(out),
                                                 _VP(_stream_handle(stream))))
        return out

    def autotune(self, x, out_max=None, out_min=None, stream=None):
        self._check_input(x)
        out_max, out_min = self._outs(x, out_max, out_min)
        with torch.cuda.device(x.device):
            check(self._lib.mmf_batch_plan_autotune(self._h, _ptr(x), _ptr(out_max), _ptr(out_min),
                                                    _VP(_stream_handle(stream))))
        return self.segments()

    def segments(self):
        out = []
        for g in range(4):
            v = ctypes.c_int()
            check(self._lib.mmf_batch_plan_get_segment(self._h, g, ctypes.byref(v)))
            out.append(int(v.value))
        return out

    def set_segment(self, group: int, tiles: int):
        check(self._lib.mmf_batch_plan_set_segment(self._h, group, tiles))

    def knobs(self):
        """Tuned knobs beside the segments: ``short_cut`` (series of at most
        this many elements take one warp each) and ``slide_max`` (windows up
        to this take the register slide)."""
        sc, sl = ctypes.c_int64(), ctypes.c_int()
        check(self._lib.mmf_batch_plan_get_knobs(self._h, ctypes.byref(sc), ctypes.byref(sl)))
        return {"short_cut": int(sc.value), "slide_max": int(sl.value), "segments": self.segments()}

    def set_knobs(self, short_cut: int, slide_max: int):
        check(self._lib.mmf_batch_plan_set_knobs(self._h, int(short_cut), int(slide_max)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mmf_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filter2d_workspace(n: int, H: int, W: int, wy: int, wx: int, dtype: torch.dtype, fuse: int = -1) -> int:
    """Bytes of workspace filter2d needs for n dense images of H x W."""
    need = ctypes.c_size_t(0)
    check(load().mmf_filter2d_workspace(n, H, W, wy, wx, DTYPES[dtype], fuse, ctypes.byref(need)))
    return need.value


def filter2d(x: torch.Tensor, wy: int, wx: int, fuse: int = -1, out_max=None, out_min=None,
             workspace=None, stream=None):
    """Separable 2D max/min filter, valid windows wy x wx, of images
    ``x`` shaped (H, W) or (N, H, W) (last dim contiguous; rows may be
    padded).  Returns ``(max, min)`` shaped (N, H-wy+1, W-wx+1)."""
    if x.dim() == 2:
        x = x.unsqueeze(0)
    if x.dim() != 3 or not x.is_cuda or x.dtype not in DTYPES or x.stride(2) != 1:
        raise TypeError("x must be a CUDA tensor (N, H, W) with unit column stride")
    n, H, W = x.shape
    pitch = x.stride(1)
    if n > 1 and x.stride(0) != H * pitch:
        raise ValueError("images must be stacked at H * pitch")
    lib = load()
    Ho, Wo = max(0, H - wy + 1), max(0, W - wx + 1)
    if out_max is None:
        out_max = torch.empty((n, Ho, Wo), dtype=x.dtype, device=x.device)
    if out_min is None:
        out_min = torch.empty((n, Ho, Wo), dtype=x.dtype, device=x.device)
    need = ctypes.c_size_t(0)
    check(lib.mmf_filter2d_workspace(n, H, W, wy, wx, DTYPES[x.dtype], fuse, ctypes.byref(need)))
    if need.value and (workspace is None or workspace.numel() * workspace.element_size() < need.value):
        workspace = torch.empty(need.value, dtype=torch.uint8, device=x.device)
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    with torch.cuda.device(x.device):
        check(lib.mmf_filter2d_separable(_ptr(x), n, H, W, pitch, wy, wx, DTYPES[x.dtype], fuse,
                                         _ptr(out_max), _ptr(out_min), _ptr(workspace),
                                         wbytes, _VP(_stream_handle(stream))))
    return out_max, out_min


class ServerStats(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_int64), ("elements", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("queued", ctypes.c_int64), ("device_bytes_used", ctypes.c_int64),
                ("p50_queue_ms", ctypes.c_double), ("p99_queue_ms", ctypes.c_double),
                ("p50_service_ms", ctypes.c_double), ("p99_service_ms", ctypes.c_double),
                ("max_hold_ms", ctypes.c_double)]


_NP_DTYPES = {"float32": 0, "float64": 1, "int16": 2, "uint8": 3}


class Server:
    """Streaming service (``mmf_server_*``): zero-latency running max-min of
    many concurrent streams with continuous batching on the device.

    Chunks and outputs are numpy arrays in host memory (pinned arrays, e.g.
    from ``torch.empty(..., pin_memory=True).numpy()``, copy faster); they must
    stay alive until their ticket is waited for."""

    def __init__(self, budget_bytes: int = 1 << 30, max_batch: int = 256, dtype: str = "float32"):
        lib = load()
        self._lib = lib
        self.dtype = dtype
        h = _VP()
        check(lib.mmf_server_create(budget_bytes, max_batch, _NP_DTYPES[dtype], ctypes.byref(h)))
        self._h = h
        self._keep = {}
        lib.mmf_server_stats.argtypes = [_VP, _INT, ctypes.POINTER(ServerStats)]
        lib.mmf_server_stats.restype = _INT

    def open(self, w: int) -> int:
        sid = ctypes.c_uint64(0)
        check(self._lib.mmf_stream_open(self._h, w, ctypes.byref(sid)))
        return int(sid.value)

    def push(self, sid: int, chunk, out_max=None, out_min=None):
        """Queue ``chunk`` (1D numpy array); returns ``(ticket, n_out)``.
        ``out_max``/``out_min`` must hold n_out elements (see n_outputs)."""
        import numpy as np
        assert chunk.dtype == np.dtype(self.dtype) and chunk.flags["C_CONTIGUOUS"]
        n_out = ctypes.c_int64(0)
        t = ctypes.c_uint64(0)
        p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        check(self._lib.mmf_stream_push(self._h, sid, p(chunk), chunk.size, p(out_max), p(out_min),
                                        ctypes.byref(n_out), ctypes.byref(t)))
        self._keep[int(t.value)] = (chunk, out_max, out_min)
        return int(t.value), int(n_out.value)

    def wait(self, ticket: int, timeout_ms: int = 60_000) -> None:
        check(self._lib.mmf_ticket_wait(self._h, ticket, timeout_ms))
        self._keep.pop(ticket, None)

    def push_batch(self, sids, chunk_ptrs, lens, max_ptrs=None, min_ptrs=None):
        """Queue many chunks in one call (``mmf_stream_push_batch``).  All
        arguments are equal-length numpy arrays: stream ids (uint64), host
        addresses of the chunks and of their outputs (uint64, e.g.
        ``arr.ctypes.data`` plus byte offsets) and lengths (int64).  The
        caller keeps the memory alive until the tickets are waited for.
        Returns ``(tickets, n_out)`` as numpy arrays."""
        import numpy as np
        sids = np.ascontiguousarray(sids, dtype=np.uint64)
        chunk_ptrs = np.ascontiguousarray(chunk_ptrs, dtype=np.uint64)
        lens = np.ascontiguousarray(lens, dtype=np.int64)
        k = sids.size
        tickets = np.empty(k, dtype=np.uint64)
        n_out = np.empty(k, dtype=np.int64)
        done = ctypes.c_int64(0)
        p = lambda a: None if a is None else ctypes.c_void_p(np.ascontiguousarray(a, dtype=np.uint64).ctypes.data)
        mp, np_ = (None if max_ptrs is None else np.ascontiguousarray(max_ptrs, dtype=np.uint64),
                   None if min_ptrs is None else np.ascontiguousarray(min_ptrs, dtype=np.uint64))
        check(self._lib.mmf_stream_push_batch(self._h, k, p(sids), p(chunk_ptrs), ctypes.c_void_p(lens.ctypes.data),
                                              p(mp), p(np_), ctypes.c_void_p(n_out.ctypes.data),
                                              ctypes.c_void_p(tickets.ctypes.data), ctypes.byref(done)))
        return tickets, n_out

    def wait_batch(self, tickets, timeout_ms: int = 60_000) -> None:
        import numpy as np
        t = np.ascontiguousarray(tickets, dtype=np.uint64)
        check(self._lib.mmf_ticket_wait_batch(self._h, t.size, ctypes.c_void_p(t.ctypes.data), timeout_ms))
        for x in t.tolist():
            self._keep.pop(int(x), None)

    def close_stream(self, sid: int, timeout_ms: int = 60_000) -> None:
        check(self._lib.mmf_stream_close(self._h, sid, timeout_ms))

    def snapshot(self, sid: int, timeout_ms: int = 60_000, wedge: bool = False) -> bytes:
        """The stream's state as bytes: window, 64-bit count and the last w-1
        samples, or (wedge=True) only the samples of its monotonic wedge."""
        fn = self._lib.mmf_stream_snapshot_wedge if wedge else self._lib.mmf_stream_snapshot
        n = ctypes.c_size_t()
        check(fn(self._h, sid, None, 0, ctypes.byref(n), timeout_ms))
        buf = ctypes.create_string_buffer(n.value)
        check(fn(self._h, sid, buf, n.value, ctypes.byref(n), timeout_ms))
        return buf.raw[:n.value]

    def restore(self, state: bytes) -> int:
        """A new stream in the state of a snapshot; returns its id."""
        sid = ctypes.c_uint64()
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        check(self._lib.mmf_stream_restore(self._h, buf, len(state), ctypes.byref(sid)))
        return int(sid.value)

    def pause(self, paused: bool = True) -> None:
        check(self._lib.mmf_server_pause(self._h, 1 if paused else 0))

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        check(self._lib.mmf_server_stats(self._h, 1 if reset else 0, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mmf_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def n_outputs(count_before: int, chunk_len: int, w: int) -> int:
    """Outputs of a chunk of chunk_len samples pushed after count_before
    samples to a stream with window w (windows ending inside the chunk)."""
    return max(0, count_before + chunk_len - w + 1) - max(0, count_before - w + 1)


_KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


def dispatch_set(dtype, n: int, w: int, kernel: str) -> None:
    """Entry of the AUTO dispatch table for the bucket of (dtype, n, w)
    (``kernel="auto"`` removes it)."""
    check(load().mmf_dispatch_set(DTYPES[dtype], int(n), int(w), KERNELS[kernel]))


def dispatch_get(dtype, n: int, w: int) -> str:
    """The kernel that ``kernel="auto"`` takes for valid windows of w over n."""
    k = ctypes.c_int()
    check(load().mmf_dispatch_get(DTYPES[dtype], int(n), int(w), ctypes.byref(k)))
    return _KERNEL_NAMES[int(k.value)]


def dispatch_autotune(x: torch.Tensor, w: int, out_max=None, out_min=None, stream=None) -> str:
    """Times every kernel that can filter ``x`` at window w and stores the
    fastest in the dispatch table (synchronises the stream); returns it."""
    _check_tensor(x, "x")
    lib = load()
    x = x.reshape(-1)
    m = int(lib.mmf_output_length(x.numel(), w, MODES["valid"]))
    if out_max is None:
        out_max = torch.empty(max(m, 1), dtype=x.dtype, device=x.device)
    if out_min is None:
        out_min = torch.empty(max(m, 1), dtype=x.dtype, device=x.device)
    k = ctypes.c_int()
    with torch.cuda.device(x.device):
        check(lib.mmf_dispatch_autotune(_ptr(x), x.numel(), int(w), DTYPES[x.dtype], _ptr(out_max), _ptr(out_min),
                                        _VP(_stream_handle(stream)), ctypes.byref(k)))
    return _KERNEL_NAMES[int(k.value)]


def set_wait_fault(starve_copies: bool, wait_limit_cycles: int = 0) -> None:
    """Test hook (``mmf_test_set_wait_fault``): block-scan kernels launched
    while it is on issue no input copies, so their pipeline waits run out
    after ``wait_limit_cycles`` SM clocks and set bit 0 of the status word."""
    check(load().mmf_test_set_wait_fault(1 if starve_copies else 0, int(wait_limit_cycles)))


def device_status(reset: bool = True) -> int:
    """Device status word (bit 0: a bounded wait ran out); syncs the device."""
    v = ctypes.c_uint32(0)
    check(load().mmf_device_status(ctypes.byref(v), 1 if reset else 0))
    return int(v.value)
