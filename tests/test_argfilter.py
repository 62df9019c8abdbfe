"""GPU parity of the arg-max/arg-min filter (chunked wedge with ties kept in
the deques) against the oracle's scan of every window: positions bit for
bit (leftmost among equal extremes), values bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _check(mmf, a, w, off=0):
    big = torch.from_numpy(a).cuda()
    x = big[off:]
    am, an, vm, vn = mmf.argfilter1d(x, w)
    torch.cuda.synchronize()
    emx, emn = oracle.argbf1d(a[off:], w)
    vmx, vmn = oracle.bf1d(a[off:], w)
    assert np.array_equal(am.cpu().numpy(), emx), f"argmax w={w}"
    assert np.array_equal(an.cpu().numpy(), emn), f"argmin w={w}"
    assert np.array_equal(vm.cpu().numpy(), vmx) and np.array_equal(vn.cpu().numpy(), vmn)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
@pytest.mark.parametrize("w", [1, 2, 3, 17, 100, 257, 496])
def test_argfilter_matches_oracle(mmf, dtype, w):
    a = synth.random_walk(40_009, seed=w, dtype=dtype)
    _check(mmf, a, w)


@pytest.mark.parametrize("w", [2, 3, 8, 64, 496])
def test_argfilter_ties(mmf, w):
    """Long runs of equal values (coarse u8, constant stretches, plateaus
    between monotone runs): the leftmost position of every tied extreme."""
    u = (synth.uniform(30_000, seed=w, dtype=np.uint8) // 64).astype(np.uint8)
    _check(mmf, u, w)
    p = np.repeat(synth.random_walk(3000, seed=w, dtype=np.float32), 10)
    _check(mmf, p, w)
    c = np.full(5000, 3.5, np.float32)
    _check(mmf, c, w)
    m = synth.monotone(20_000, w, np.float32)
    _check(mmf, m, w)
    _check(mmf, m[::-1].copy(), w)


def test_argfilter_sizes_views_and_limits(mmf):
    for n, w in [(1, 1), (5, 5), (6, 5), (7, 2), (4099, 3), (100, 99)]:
        _check(mmf, synth.uniform(n, seed=n, dtype=np.float32), w)
    _check(mmf, synth.random_walk(20_003, seed=4, dtype=np.float32), 33, off=3)
    x = torch.zeros(1000, device="cuda")
    with pytest.raises(mmf.MMFError):
        mmf.argfilter1d(x, 497)
    am, an, vm, vn = mmf.argfilter1d(x[:10], 11)
    assert am.numel() == 0
    assert mmf.device_status() == 0
