"""The range-checked build (``python -m paper_cs_0610046_gb300.build --checked``,
loaded with ``MMF_CHECKED=1``): the block-scan and short-series kernels check
every input copy and direct load against the launch's readable bound and
record bit 2 of the device status word instead of reading past it.

The test hook ``mmf_test_set_input_clip`` tells the kernels a bound below what
they read (the bytes past it are still inside the caller's buffer, so nothing
outside it is touched in either build): the checked build must flag it, and
the ordinary build, whose copies fall back to bounded direct loads, must
still give the oracle's outputs."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
CHECKED = os.environ.get("MMF_CHECKED") == "1"


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _run_clipped(mmf, x, w, clip):
    lib = mmf.load()
    mmf.device_status(reset=True)
    try:
        assert lib.mmf_test_set_input_clip(clip) == 0
        mx, mn = mmf.filter1d(x, w)
        torch.cuda.synchronize()
        st = mmf.device_status(reset=True)
    finally:
        lib.mmf_test_set_input_clip(0)
    return mx, mn, st


@pytest.mark.skipif(not CHECKED, reason="range checks are compiled into the checked build only")
@pytest.mark.parametrize("w", [3, 101, 1001, 5001])
def test_checked_build_flags_reads_past_the_bound(mmf, w):
    a = synth.random_walk(1 << 20, seed=w, dtype=np.float32)
    x = torch.from_numpy(a).cuda()
    _, _, st = _run_clipped(mmf, x, w, 1 << 19)
    assert st & 4, f"no range error recorded (status {st})"
    mx, mn = mmf.filter1d(x, w)  # unclipped: correct and clean
    em, en = oracle.bf1d(a, w)
    assert np.array_equal(mx.cpu().numpy(), em) and np.array_equal(mn.cpu().numpy(), en)
    assert mmf.device_status(reset=True) == 0


@pytest.mark.skipif(CHECKED, reason="the checked build skips the clipped reads by design")
@pytest.mark.parametrize("w", [3, 101, 1001, 5001])
def test_clipped_bound_changes_nothing_unchecked(mmf, w):
    """A smaller readable bound only moves slices from bulk copies to bounded
    direct loads: same outputs, no error."""
    a = synth.random_walk((1 << 20) + 13, seed=w, dtype=np.float32)
    x = torch.from_numpy(a).cuda()
    mx, mn, st = _run_clipped(mmf, x, w, 1 << 19)
    assert st == 0
    em, en = oracle.bf1d(a, w)
    assert np.array_equal(mx.cpu().numpy(), em) and np.array_equal(mn.cpu().numpy(), en)
