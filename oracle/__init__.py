"""CPU oracle for the running max-min filter (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links or loads
it, and it imports nothing from the library.

The arithmetic lives in ``mmf_oracle.c`` (plain C, compiled by :func:`build`):

* :func:`bf1d` -- the definition of Section 1 (max/min over every window
  ``[j, j+w)``), i.e. the "naive" row of Table 1.
* :func:`bf1d_at` -- the same at chosen window starts (for full-size checks).
* :func:`wedge` -- Algorithm 1 of Section 4 with a comparison counter
  (Section 1 cost model) and the wedge-size bound of Proposition 4.
* :func:`envelope` -- centred, end-clipped windows of radius ``r`` (the
  envelope use cited in Section 1).
* :func:`bf2d` / :func:`bf2d_at` -- literal ``wy x wx`` rectangle max/min,
  valid mode (the 2D filter of Section 1, written without separation).
* :func:`stream_reference` -- the served outputs of a chunked stream are, by
  the definition, the whole-array filter over the concatenated chunks.
* :func:`lb_keogh` -- the lower bound of the time-warping distance from a
  precomputed envelope (the application Section 1 cites): a query against
  a series' centred, end-clipped envelope of radius ``r``, in double.
* :func:`dtw_band` -- the banded time-warping distance that ``lb_keogh``
  bounds (a pin for it), by dynamic programming in double.
* :func:`argbf1d` -- the locations of every window's maximum and minimum
  (leftmost among equals), by scanning each window (Section 5's
  arg-max/arg-min filter).
* :func:`w3` -- the window-3 filter of the proposition following Section 3's
  lower bound, in at most 2 comparisons per element (counted).

Python here does marshalling only; no arithmetic of the method is in it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_SUFFIX = {np.dtype(np.float32): "f32", np.dtype(np.float64): "f64",
           np.dtype(np.int16): "i16", np.dtype(np.uint8): "u8"}

_I64 = ctypes.c_int64
_VP = ctypes.c_void_p


class WedgeStats(ctypes.Structure):
    _fields_ = [("ncmp", _I64), ("max_size", _I64), ("stale_fronts", _I64),
                ("steps", _I64)]


def build(force: bool = False) -> str:
    """Compile ``mmf_oracle.c`` into ``liboracle.so`` (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            for suf in _SUFFIX.values():
                getattr(lib, f"oracle_bf1d_{suf}").argtypes = [_VP, _I64, _I64, _VP, _VP]
                getattr(lib, f"oracle_bf1d_at_{suf}").argtypes = [_VP, _I64, _I64, _VP, _I64, _VP, _VP]
                getattr(lib, f"oracle_wedge_{suf}").argtypes = [_VP, _I64, _I64, _VP, _VP,
                                                               ctypes.POINTER(WedgeStats)]
                getattr(lib, f"oracle_envelope_{suf}").argtypes = [_VP, _I64, _I64, _VP, _VP]
                getattr(lib, f"oracle_bf2d_{suf}").argtypes = [_VP, _I64, _I64, _I64, _I64, _I64, _VP, _VP]
                getattr(lib, f"oracle_bf2d_at_{suf}").argtypes = [_VP, _I64, _I64, _I64, _I64, _I64,
                                                                 _VP, _VP, _I64, _VP, _VP]
                getattr(lib, f"oracle_lb_keogh_{suf}").argtypes = [_VP, _VP, _I64, _I64, _VP]
                getattr(lib, f"oracle_dtw_band_{suf}").argtypes = [_VP, _VP, _I64, _I64, _VP]
                getattr(lib, f"oracle_w3_{suf}").argtypes = [_VP, _I64, _VP, _VP, _VP]
                getattr(lib, f"oracle_argbf1d_{suf}").argtypes = [_VP, _I64, _I64, _VP, _VP]
                for name in ("bf1d", "bf1d_at", "wedge", "envelope", "bf2d", "bf2d_at", "lb_keogh",
                             "dtw_band", "w3", "argbf1d"):
                    getattr(lib, f"oracle_{name}_{suf}").restype = ctypes.c_int
            _lib = lib
    return _lib


def _fn(name: str, dtype) -> object:
    dt = np.dtype(dtype)
    if dt not in _SUFFIX:
        raise TypeError(f"oracle: unsupported dtype {dt}")
    return getattr(_load(), f"oracle_{name}_{_SUFFIX[dt]}")


def _ptr(x: np.ndarray | None):
    return None if x is None else x.ctypes.data_as(_VP)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def n_out(n: int, w: int) -> int:
    """Number of windows [j, j+w) inside a length-n array (0 if w > n)."""
    return max(0, n - w + 1)


def bf1d(a: np.ndarray, w: int):
    """Max and min of every window [j, j+w), j = 0..n-w (Section 1)."""
    a = np.ascontiguousarray(a)
    m = n_out(a.size, w)
    mx = np.empty(m, a.dtype)
    mn = np.empty(m, a.dtype)
    _check(_fn("bf1d", a.dtype)(_ptr(a), a.size, w, _ptr(mx), _ptr(mn)), "bf1d")
    return mx, mn


def bf1d_at(a: np.ndarray, w: int, starts: np.ndarray):
    """Max and min of the windows [s, s+w) for each s in ``starts``."""
    a = np.ascontiguousarray(a)
    starts = np.ascontiguousarray(starts, dtype=np.int64)
    mx = np.empty(starts.size, a.dtype)
    mn = np.empty(starts.size, a.dtype)
    _check(_fn("bf1d_at", a.dtype)(_ptr(a), a.size, w, _ptr(starts), starts.size,
                                   _ptr(mx), _ptr(mn)), "bf1d_at")
    return mx, mn


def wedge(a: np.ndarray, w: int):
    """Algorithm 1: returns (max, min, stats) with the comparison count."""
    a = np.ascontiguousarray(a)
    m = n_out(a.size, w)
    mx = np.empty(m, a.dtype)
    mn = np.empty(m, a.dtype)
    st = WedgeStats()
    _check(_fn("wedge", a.dtype)(_ptr(a), a.size, w, _ptr(mx), _ptr(mn),
                                 ctypes.byref(st)), "wedge")
    return mx, mn, {"ncmp": st.ncmp, "max_size": st.max_size,
                    "stale_fronts": st.stale_fronts, "steps": st.steps}


def wedge_mt(a: np.ndarray, w: int, threads: int | None = None):
    """Algorithm 1 on ``threads`` host threads: the outputs are split into
    contiguous ranges and each range runs the single-thread wedge over its
    inputs plus the w-1 that follow (each output depends only on its own
    window, Section 1, so the split is exact).  ctypes releases the GIL
    around each call.  Returns (max, min, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    a = np.ascontiguousarray(a)
    m = n_out(a.size, w)
    mx = np.empty(m, a.dtype)
    mn = np.empty(m, a.dtype)
    t = max(1, min(threads or os.cpu_count() or 1, m))
    bounds = [m * k // t for k in range(t + 1)]
    fn = _fn("wedge", a.dtype)

    def run(k):
        j0, j1 = bounds[k], bounds[k + 1]
        if j1 <= j0:
            return 0
        seg = a[j0:j1 + w - 1]
        return fn(_ptr(seg), seg.size, w, _ptr(mx[j0:j1]), _ptr(mn[j0:j1]), None)

    if m > 0:
        with ThreadPoolExecutor(max_workers=t) as ex:
            for rc in ex.map(run, range(t)):
                _check(rc, "wedge_mt")
    return mx, mn, t


def envelope(a: np.ndarray, r: int):
    """Centred end-clipped envelope of radius r: (upper, lower), n each."""
    a = np.ascontiguousarray(a)
    up = np.empty(a.size, a.dtype)
    lo = np.empty(a.size, a.dtype)
    _check(_fn("envelope", a.dtype)(_ptr(a), a.size, r, _ptr(up), _ptr(lo)), "envelope")
    return up, lo


def bf2d(img: np.ndarray, wy: int, wx: int):
    """Valid-mode rectangle max/min of a 2D array (rows x cols)."""
    img = np.ascontiguousarray(img)
    H, W = img.shape
    Ho, Wo = max(0, H - wy + 1), max(0, W - wx + 1)
    mx = np.empty((Ho, Wo), img.dtype)
    mn = np.empty((Ho, Wo), img.dtype)
    _check(_fn("bf2d", img.dtype)(_ptr(img), H, W, W, wy, wx, _ptr(mx), _ptr(mn)), "bf2d")
    return mx, mn


def bf2d_at(img: np.ndarray, wy: int, wx: int, ys: np.ndarray, xs: np.ndarray):
    """Rectangle max/min whose top-left corners are (ys[t], xs[t])."""
    img = np.ascontiguousarray(img)
    H, W = img.shape
    ys = np.ascontiguousarray(ys, dtype=np.int64)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    mx = np.empty(ys.size, img.dtype)
    mn = np.empty(ys.size, img.dtype)
    _check(_fn("bf2d_at", img.dtype)(_ptr(img), H, W, W, wy, wx, _ptr(ys), _ptr(xs),
                                     ys.size, _ptr(mx), _ptr(mn)), "bf2d_at")
    return mx, mn


def stream_reference(chunks, w: int):
    """Outputs a zero-latency stream must have emitted after all ``chunks``:
    the filter of the concatenation (each output depends only on its
    window, Section 1)."""
    return bf1d(np.concatenate([np.asarray(c) for c in chunks]), w)


def lb_keogh(c: np.ndarray, q: np.ndarray, r: int) -> float:
    """Lower bound of the banded time-warping distance of q and c from the
    envelope of radius r of c (sqrt of the squared excursions of q outside
    it), in double."""
    c = np.ascontiguousarray(c)
    q = np.ascontiguousarray(q, dtype=c.dtype)
    if q.size != c.size:
        raise ValueError("query and series lengths differ")
    out = ctypes.c_double()
    _check(_fn("lb_keogh", c.dtype)(_ptr(c), _ptr(q), c.size, r, ctypes.byref(out)), "lb_keogh")
    return out.value


def dtw_band(q: np.ndarray, c: np.ndarray, r: int) -> float:
    """Time-warping distance of q and c with |i - j| <= r (small n only:
    n x n doubles)."""
    q = np.ascontiguousarray(q)
    c = np.ascontiguousarray(c, dtype=q.dtype)
    out = ctypes.c_double()
    _check(_fn("dtw_band", q.dtype)(_ptr(q), _ptr(c), q.size, r, ctypes.byref(out)), "dtw_band")
    return out.value


def w3(a: np.ndarray):
    """Window-3 max and min in at most 2 comparisons per element: returns
    (max, min, comparisons)."""
    a = np.ascontiguousarray(a)
    m = n_out(a.size, 3)
    mx = np.empty(m, a.dtype)
    mn = np.empty(m, a.dtype)
    c = ctypes.c_int64()
    _check(_fn("w3", a.dtype)(_ptr(a), a.size, _ptr(mx), _ptr(mn), ctypes.byref(c)), "w3")
    return mx, mn, c.value


def argbf1d(a: np.ndarray, w: int):
    """Positions of the maximum and minimum of every window [j, j+w), the
    leftmost among equal values (int64 arrays of n-w+1)."""
    a = np.ascontiguousarray(a)
    m = n_out(a.size, w)
    imx = np.empty(m, np.int64)
    imn = np.empty(m, np.int64)
    _check(_fn("argbf1d", a.dtype)(_ptr(a), a.size, w, _ptr(imx), _ptr(imn)), "argbf1d")
    return imx, imn
