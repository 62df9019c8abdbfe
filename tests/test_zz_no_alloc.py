"""The batched filter without device allocation (mmf_filter1d_batched_noalloc),
called through the C ABI and compared with the oracle series by series.

This entry point serves callers that cannot allocate device memory: a process
that reserved its whole device budget up front, or a latency-bound host thread
where an allocation may block or fail.  Its work tables live in one fixed
device array shared by all calls, so each case runs two calls in a row with
different series: the second call must not see the first call's tables.  The
file is named to run last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NP2T = {np.float32: torch.float32, np.float64: torch.float64, np.int16: torch.int16, np.uint8: torch.uint8}
DT = {np.float32: 0, np.float64: 1, np.int16: 2, np.uint8: 3}
P64 = ctypes.POINTER(ctypes.c_int64)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    lib = m.load()
    f = lib.mmf_filter1d_batched_noalloc
    f.argtypes = [ctypes.c_void_p, P64, P64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib


def _out_offsets(lens, ws, mode, itemsize):
    """Each series' outputs start on the next 32-byte boundary (the documented
    layout of batched outputs)."""
    a = 32 // itemsize
    off, end = [], 0
    for L, w in zip(lens, ws):
        start = -(-end // a) * a
        n_out = max(0, L - w + 1) if mode == "valid" else L
        off.append(start)
        end = start + n_out
    return off, end


def _noalloc(lib, x, lens, ws, mode, dtype):
    lens = np.ascontiguousarray(lens, dtype=np.int64)
    ws = np.ascontiguousarray(ws, dtype=np.int64)
    off, out_len = _out_offsets(lens, ws, mode, np.dtype(dtype).itemsize)
    mx = torch.zeros(max(out_len, 1), dtype=x.dtype, device=x.device)
    mn = torch.zeros(max(out_len, 1), dtype=x.dtype, device=x.device)
    st = lib.mmf_filter1d_batched_noalloc(x.data_ptr(), lens.ctypes.data_as(P64), ws.ctypes.data_as(P64), lens.size,
                                          DT[dtype], {"valid": 0, "envelope": 1}[mode], mx.data_ptr(), mn.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.mmf_last_error()
    return mx, mn, off


def _check(lib, lens, ws, mode, dtype, seed, sample=None):
    """One call against the oracle: every output of every series, or (with
    ``sample``) both ends and ``sample`` random windows of each series."""
    data = synth.uneven_batch_data(np.asarray(lens), np.arange(len(lens)) % 3, np.arange(len(lens)) + seed, dtype)
    x = torch.from_numpy(data).cuda()
    mx, mn, off = _noalloc(lib, x, lens, ws, mode, dtype)
    torch.cuda.synchronize()
    gm, gn = mx.cpu().numpy(), mn.cpu().numpy()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    rng = np.random.default_rng(seed)
    for s, (L, w) in enumerate(zip(lens, ws)):
        a = data[starts[s]:starts[s] + L]
        if sample is None:
            em, en = oracle.bf1d(a, w) if mode == "valid" else oracle.envelope(a, w)
            got_m, got_n = gm[off[s]:off[s] + em.size], gn[off[s]:off[s] + en.size]
        else:
            m = L - w + 1
            js = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, sample)]))
            em, en = oracle.bf1d_at(a, w, js)
            got_m, got_n = gm[off[s] + js], gn[off[s] + js]
        assert np.array_equal(got_m, em), f"series {s} max (len {L}, w {w}, {mode}, {np.dtype(dtype).name})"
        assert np.array_equal(got_n, en), f"series {s} min (len {L}, w {w}, {mode}, {np.dtype(dtype).name})"


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
def test_noalloc_two_calls_vs_oracle(lib, dtype):
    """Uneven series (every kernel group), then fewer and different series:
    the shared tables must not leak from the first call into the second."""
    lens1, ws1, _, _ = synth.uneven_batch(120, seed=41, lo_exp=1.0, hi_exp=4.6)
    _check(lib, lens1, ws1, "valid", dtype, 1)
    lens2 = [70_001, 5, 4097, 30_000, 1, 9000]
    ws2 = [10_001, 5, 3, 1001, 1, 17]
    _check(lib, lens2, ws2, "valid", dtype, 7)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
def test_noalloc_envelope_vs_oracle(lib, dtype):
    _check(lib, [1024] * 40 + [3000, 7], [51] * 40 + [700, 9], "envelope", dtype, 3)
    _check(lib, [513, 100_000], [0, 5000], "envelope", dtype, 4)


def test_noalloc_long_series_take_longer_items(lib):
    """512 series of about 1.15e5 elements: more output tiles than 16-tile items
    can cover within the item limit, so items grow to 32 tiles (and the
    sampled windows land in every item)."""
    rng = np.random.default_rng(12)
    lens = rng.integers(110_000, 120_000, 512)
    ws = rng.choice([3, 101, 4097, 10_001], 512)
    assert sum((L - w + 1 + 2047) // 2048 for L, w in zip(lens, ws)) // 16 + 512 > 2048
    _check(lib, lens, ws, "valid", np.float32, 5, sample=300)
    _check(lib, lens[:3], ws[:3], "valid", np.float32, 6)


def test_noalloc_limits(lib):
    x = torch.zeros(1000, device="cuda")
    lens = np.full(513, 1, dtype=np.int64)
    st = lib.mmf_filter1d_batched_noalloc(x.data_ptr(), lens.ctypes.data_as(P64), lens.ctypes.data_as(P64),
                                          513, 0, 0, x.data_ptr(), None, None)
    assert st == 1 and b"limit" in lib.mmf_last_error()  # over the series limit: a clear MMF_EINVAL
    big = np.array([2**61, 2**61], dtype=np.int64)  # the second series' end passes 2^62
    one = np.ones(2, dtype=np.int64)
    st = lib.mmf_filter1d_batched_noalloc(x.data_ptr(), big.ctypes.data_as(P64), one.ctypes.data_as(P64),
                                          2, 0, 0, x.data_ptr(), None, None)
    assert st == 1 and b"overflow" in lib.mmf_last_error()
