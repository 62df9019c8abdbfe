"""GPU parity of the arg-max/arg-min filter against the oracle's scan of every
window: positions bit for bit (leftmost among equal extremes), values bit for
bit.  Two kernels: block scans over (value, position) pairs (the default, any
window; windows above the 2048-position tile take per-tile carries) and the
chunked wedge with ties kept in the deques (windows up to 496)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TILE = 2048  # positions per CTA of the block-scan kernel


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _check(mmf, a, w, off=0, kernel="auto"):
    big = torch.from_numpy(a).cuda()
    x = big[off:]
    am, an, vm, vn = mmf.argfilter1d(x, w, kernel=kernel)
    torch.cuda.synchronize()
    emx, emn = oracle.argbf1d(a[off:], w)
    vmx, vmn = oracle.bf1d(a[off:], w)
    assert np.array_equal(am.cpu().numpy(), emx), f"argmax w={w} {kernel}"
    assert np.array_equal(an.cpu().numpy(), emn), f"argmin w={w} {kernel}"
    assert np.array_equal(vm.cpu().numpy(), vmx) and np.array_equal(vn.cpu().numpy(), vmn)


def _kernels(w):
    return ["blockscan", "wedge"] if w <= 496 else ["blockscan"]


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
@pytest.mark.parametrize("w", [1, 2, 3, 17, 100, 257, 496, 1025, TILE - 1, TILE, TILE + 1, 5000])
def test_argfilter_matches_oracle(mmf, dtype, w):
    a = synth.random_walk(40_009, seed=w, dtype=dtype)
    for k in _kernels(w):
        _check(mmf, a, w, kernel=k)


@pytest.mark.parametrize("w", [2, 3, 8, 64, 496, 700, TILE + 1, 4097])
def test_argfilter_ties(mmf, w):
    """Long runs of equal values (coarse u8, constant stretches, plateaus
    between monotone runs): the leftmost position of every tied extreme,
    also where the ties straddle tiles and blocks."""
    u = (synth.uniform(30_000, seed=w, dtype=np.uint8) // 64).astype(np.uint8)
    p = np.repeat(synth.random_walk(3000, seed=w, dtype=np.float32), 10)
    c = np.full(max(5000, 3 * w), 3.5, np.float32)
    m = synth.monotone(20_000, w, np.float32)
    for k in _kernels(w):
        _check(mmf, u, w, kernel=k)
        _check(mmf, p, w, kernel=k)
        _check(mmf, c, w, kernel=k)
        _check(mmf, m, w, kernel=k)
        _check(mmf, m[::-1].copy(), w, kernel=k)


def test_argfilter_infinities(mmf):
    """-inf / +inf in the data equal the block-scan identities: the real
    positions still win (leftmost among the tied infinities)."""
    a = synth.uniform(12_000, seed=5, dtype=np.float32)
    a[::7] = -np.inf
    a[3::11] = np.inf
    a[5000:9000] = -np.inf
    for w in (1, 3, 31, 2100, 4500):
        _check(mmf, a, w, kernel="blockscan")


def test_argfilter_sizes_views_and_limits(mmf):
    for n, w in [(1, 1), (5, 5), (6, 5), (7, 2), (4099, 3), (100, 99), (2049, 2049), (4097, 2049), (6000, 2500)]:
        for k in _kernels(w):
            _check(mmf, synth.uniform(n, seed=n, dtype=np.float32), w, kernel=k)
    _check(mmf, synth.random_walk(20_003, seed=4, dtype=np.float32), 33, off=3)
    _check(mmf, synth.random_walk(20_003, seed=4, dtype=np.float32), 2600, off=5)
    x = torch.zeros(1000, device="cuda")
    with pytest.raises(mmf.MMFError):
        mmf.argfilter1d(x, 497, kernel="wedge")
    with pytest.raises(mmf.MMFError):
        mmf.argfilter1d(x, 3, kernel="slide")
    am, an, vm, vn = mmf.argfilter1d(x[:10], 11)
    assert am.numel() == 0
    assert mmf.device_status() == 0


@pytest.mark.parametrize("w", [3, 1001, 65537])
def test_argfilter_full_size_sampled(mmf, w):
    """n = 2^30 f32 random walk (the measured stream size), in the measured
    launch configuration; 300 sampled outputs plus the first and last."""
    n = 1 << 30
    x = synth.torch_by_name("random_walk", n, 91, torch.device("cuda"))
    am, an, vm, vn = mmf.argfilter1d(x, w)
    torch.cuda.synchronize()
    m = n - w + 1
    rng = np.random.default_rng(w)
    idx = np.concatenate([[0, 1, m - 2, m - 1], rng.integers(0, m, 300)])
    pick = torch.from_numpy(idx).cuda()
    outs = [t[pick] for t in (am, an, vm, vn)]
    am_s, an_s, vm_s, vn_s = (t.cpu().numpy() for t in outs)
    for q, j in enumerate(idx):
        seg = x[j:j + w].cpu().numpy()
        emx, emn = oracle.argbf1d(seg, w)
        vmx, vmn = oracle.bf1d(seg, w)
        assert am_s[q] == j + emx[0] and an_s[q] == j + emn[0], f"w={w} j={j}"
        assert vm_s[q] == vmx[0] and vn_s[q] == vmn[0]
    # Properties at every output: the value at the reported position, and the
    # position inside the window.
    js = torch.arange(m, device="cuda")
    assert torch.equal(x[am], vm) and torch.equal(x[an], vn)
    assert bool(((am >= js) & (am < js + w)).all()) and bool(((an >= js) & (an < js + w)).all())
    del x, am, an, vm, vn, js
    torch.cuda.empty_cache()


def test_argfilter_positions_beyond_2_31(mmf):
    """u8 stream of 2^31 + 5000 elements: positions above 2^31 (64-bit index
    arithmetic), a small and a multi-tile window, sampled near the end."""
    n = (1 << 31) + 5000
    g = torch.Generator(device="cuda")
    g.manual_seed(77)
    x = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
    for w in (5, 4500):
        am, an, vm, vn = mmf.argfilter1d(x, w)
        torch.cuda.synchronize()
        m = n - w + 1
        idx = np.concatenate([np.arange(m - 40, m), np.arange((1 << 31) - 20, (1 << 31) + 20), [0, 12345]])
        pick = torch.from_numpy(idx).cuda()
        am_s, an_s, vm_s, vn_s = (t[pick].cpu().numpy() for t in (am, an, vm, vn))
        for q, j in enumerate(idx):
            seg = x[j:j + w].cpu().numpy()
            emx, emn = oracle.argbf1d(seg, w)
            assert am_s[q] == j + emx[0] and an_s[q] == j + emn[0], f"w={w} j={j}"
            assert vm_s[q] == seg[emx[0]] and vn_s[q] == seg[emn[0]]
        del am, an, vm, vn
    del x
    torch.cuda.empty_cache()


def test_argfilter_window_above_2_30(mmf):
    """w = 2^30 + 1 (64-bit positions inside the kernel) on a u8 array of
    2^30 + 100 elements of 128 with planted extremes, whose leftmost positions
    follow from where they lie: a 255 at 2^29 (in every window), 0 at 5 and
    at 2^30 + 20, a 255 at 2^30 + 50 (never leftmost)."""
    n, w = (1 << 30) + 100, (1 << 30) + 1
    x = torch.full((n,), 128, dtype=torch.uint8, device="cuda")
    x[1 << 29] = 255
    x[(1 << 30) + 50] = 255
    x[5] = 0
    x[(1 << 30) + 20] = 0
    am, an, vm, vn = mmf.argfilter1d(x, w)
    torch.cuda.synchronize()
    m = n - w + 1
    exp_max = np.full(m, 1 << 29)
    exp_min = np.array([5 if j <= 5 else (j if j + w - 1 < (1 << 30) + 20 else (1 << 30) + 20) for j in range(m)])
    exp_vmin = np.array([0 if (j <= 5 or j + w - 1 >= (1 << 30) + 20) else 128 for j in range(m)])
    assert np.array_equal(am.cpu().numpy(), exp_max)
    assert np.array_equal(an.cpu().numpy(), exp_min)
    assert bool((vm == 255).all()) and np.array_equal(vn.cpu().numpy(), exp_vmin.astype(np.uint8))
    del x, am, an, vm, vn
    torch.cuda.empty_cache()
