"""The batched filter without device allocation (mmf_filter1d_batched_noalloc),
called through the C ABI, against the plan-based batched filter.

This entry point serves callers that cannot allocate device memory (a fixed
memory pool reserved up front, real-time paths, host callbacks); its work
tables live in one fixed device array shared by all calls.  Two calls in a
row with different series check that each call re-initialises the shared
tables.  The file is named to run last."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _noalloc(lib, x, lens, ws, mode, out_len):
    f = lib.mmf_filter1d_batched_noalloc
    P64 = ctypes.POINTER(ctypes.c_int64)
    f.argtypes = [ctypes.c_void_p, P64, P64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    lens = np.ascontiguousarray(lens, dtype=np.int64)
    ws = np.ascontiguousarray(ws, dtype=np.int64)
    # Zero-filled like the plan's own buffers: the padding between series
    # is never written, so both keep zeros there.
    mx = torch.zeros(out_len, dtype=x.dtype, device=x.device)
    mn = torch.zeros(out_len, dtype=x.dtype, device=x.device)
    st = f(x.data_ptr(), lens.ctypes.data_as(P64), ws.ctypes.data_as(P64), lens.size,
           {torch.float32: 0, torch.float64: 1}[x.dtype], {"valid": 0, "envelope": 1}[mode],
           mx.data_ptr(), mn.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.mmf_last_error()
    return mx, mn


def _case(mmf, lens, ws, mode, dtype, seed):
    data = synth.uneven_batch_data(np.asarray(lens), np.arange(len(lens)) % 3, np.arange(len(lens)) + seed,
                                   np.float32 if dtype == torch.float32 else np.float64)
    x = torch.from_numpy(data).cuda()
    plan = mmf.BatchPlan(lens, ws, dtype, mode)
    em, en = plan(x)
    gm, gn = _noalloc(mmf.load(), x, lens, ws, mode, plan.out_len)
    torch.cuda.synchronize()
    plan.close()
    # Every output is an input element: the two paths agree bit for bit.
    assert torch.equal(gm, em) and torch.equal(gn, en)


def test_noalloc_matches_plan_two_calls(mmf):
    lens1, ws1, _, _ = synth.uneven_batch(200, seed=41, lo_exp=2.0, hi_exp=5.0)
    _case(mmf, lens1, ws1, "valid", torch.float32, 1)
    # Second call: fewer, different series; the shared tables must not leak.
    lens2 = [70_001, 5, 4097, 300_000, 1]
    ws2 = [10_001, 5, 3, 1001, 1]
    _case(mmf, lens2, ws2, "valid", torch.float32, 7)


def test_noalloc_envelope_f64_and_limits(mmf):
    _case(mmf, [1024] * 40, [51] * 40, "envelope", torch.float64, 3)
    lib = mmf.load()
    x = torch.zeros(1000, device="cuda")
    lens = np.full(513, 1, dtype=np.int64)
    P64 = ctypes.POINTER(ctypes.c_int64)
    st = lib.mmf_filter1d_batched_noalloc(x.data_ptr(), lens.ctypes.data_as(P64), lens.ctypes.data_as(P64),
                                          513, 0, 0, x.data_ptr(), None, None)
    assert st == 1  # over the series limit: a clear MMF_EINVAL
    assert b"limit" in lib.mmf_last_error()
