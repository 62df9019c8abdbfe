"""The device-side timeout path of the block-scan kernels, made to run out on
purpose without any fault: with the test hook on, the kernels issue none of
their input copies, so no transaction ever reaches a pipeline barrier, every
bounded wait runs out after a short limit, the expiring warps report bit 0 of
the device status word, finish their work item without waiting again (every
warp still takes every barrier of the item), and all warps of each CTA leave
together at the item's end, at a barrier that ORs their failure flags.  The
test checks that each call returns, that the status bit is set, and that the
context is still usable afterwards (a normal call then matches the oracle);
the outputs of a failed call are unspecified."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

LIMIT = 200_000  # SM clocks, about 0.1 ms


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _sentinel(n, dtype):
    if dtype.is_floating_point:
        return torch.full((n,), float("nan"), dtype=dtype, device="cuda")
    return torch.full((n,), 77, dtype=dtype, device="cuda")


CASES = [  # (dtype, window or radius, mode): every block mode and both consumer forms
    (torch.float32, 3, "valid"), (torch.float32, 5, "valid"), (torch.float32, 101, "valid"),
    (torch.float32, 1001, "valid"), (torch.float32, 5001, "valid"), (torch.float32, 51, "envelope"),
    (torch.float64, 3, "valid"), (torch.float64, 5, "valid"), (torch.float64, 101, "valid"),
    (torch.float64, 5001, "valid"), (torch.int16, 101, "valid"), (torch.uint8, 9000, "valid"),
]


def test_starved_waits_run_out_and_every_cta_leaves(mmf):
    a = synth.random_walk(300_000, 5, np.float64)
    mmf.device_status(reset=True)
    try:
        mmf.set_wait_fault(True, LIMIT)
        for dtype, w, mode in CASES:
            x = torch.from_numpy(a).to("cuda").to(dtype) if dtype.is_floating_point else \
                torch.from_numpy((a * 10).astype(np.int64) % 200).to("cuda").to(dtype)
            m = mmf.output_length(x.numel(), w, mode)
            om, on = _sentinel(m, dtype), _sentinel(m, dtype)
            mmf.filter1d(x, w, mode=mode, out_max=om, out_min=on)
            torch.cuda.synchronize()
            assert mmf.device_status(reset=True) & 1, f"no timeout reported ({dtype}, {mode} {w})"
        # The advancing front (tickets, published tile aggregates): items
        # whose producers failed still find their flags set, so no wait
        # runs beyond the first.
        for w in (2049, 20_001):
            xf = torch.from_numpy(a).to("cuda").float()
            mmf.filter1d(xf, w, kernel="front")
            torch.cuda.synchronize()
            assert mmf.device_status(reset=True) & 1, f"no timeout reported (front, w {w})"
        # A batched plan: ticketed work items, long series only (block scans).
        lens = [40_000, 70_001, 5_000, 120_000]
        ws = [3, 1001, 17, 10_001]
        plan = mmf.BatchPlan(lens, ws, torch.float32)
        xb = torch.from_numpy(synth.random_walk(sum(lens), 6, np.float32)).cuda()
        bm, bn = _sentinel(plan.out_len, torch.float32), _sentinel(plan.out_len, torch.float32)
        plan(xb, bm, bn)
        torch.cuda.synchronize()
        assert mmf.device_status(reset=True) & 1
        plan.close()
        # The 2D row pass (block scans over rows); the column pass that follows
        # reads an unwritten workspace, which is allowed to give any values.
        img = torch.rand(2, 300, 700, device="cuda")
        mmf.filter2d(img, 5, 40, fuse=0)
        torch.cuda.synchronize()
        assert mmf.device_status(reset=True) & 1
    finally:
        mmf.set_wait_fault(False)
    # The context is usable and the status word clean after normal calls.
    x = torch.from_numpy(a.astype(np.float32)).cuda()
    for w in (3, 101, 5001):
        mx, mn = mmf.filter1d(x, w)
        em, en = oracle.bf1d(a.astype(np.float32), w)
        assert np.array_equal(mx.cpu().numpy(), em) and np.array_equal(mn.cpu().numpy(), en)
    assert mmf.device_status(reset=True) == 0
