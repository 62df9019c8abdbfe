"""GPU parity of the chunked monotonic-wedge kernel (Algorithm 1 per thread
chunk, Section 4) against the CPU oracle, through mmf_filter1d_ex with
MMF_KERNEL_WEDGE.  Bit-exact: every output is an input element."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DTYPES = [np.float32, np.float64, np.int16, np.uint8]
MAX_W = 496  # MMF_WEDGE_MAX_WINDOW


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(gm, gn, emx, emn, what):
    for got, exp, side in ((gm, emx, "max"), (gn, emn, "min")):
        assert got.shape == exp.shape, what
        if not np.array_equal(got, exp):
            bad = np.nonzero(got != exp)[0]
            raise AssertionError(f"{side} mismatch {what}: {bad.size} bad, first {bad[:8]}")


def _check(mmf, a, w):
    mx, mn = mmf.filter1d(_gpu(a), w, kernel="wedge")
    torch.cuda.synchronize()
    emx, emn = oracle.bf1d(a, w)
    _same(mx.cpu().numpy(), mn.cpu().numpy(), emx, emn, f"w={w} n={a.size} {a.dtype}")


@pytest.mark.parametrize("w", [1, 2, 3, 4, 7, 8, 9, 15, 16, 17, 31, 64, 101, 255, 256, 257, 400, MAX_W])
@pytest.mark.parametrize("dist", ["uniform", "random_walk", "piecewise_monotone"])
def test_windows_f32(mmf, w, dist):
    a = synth.by_name(dist, 200_003, seed=w, dtype=np.float32)
    _check(mmf, a, w)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("w", [2, 5, 33, 129, MAX_W])
def test_dtypes(mmf, dtype, w):
    a = synth.random_walk(100_001, seed=w, dtype=dtype)
    _check(mmf, a, w)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_and_monotone(mmf, dtype):
    """Long runs of equal values and strictly monotone stretches: the cases
    where U or L keep many entries (Proposition 3 and its tied variant)."""
    rng = np.random.default_rng(5)
    a = np.repeat(rng.integers(0, 4, 6000), rng.integers(1, 60, 6000)).astype(dtype)
    for w in (3, 50, 300):
        _check(mmf, a, w)
    up = np.arange(70_000) % 120
    _check(mmf, up.astype(dtype), 97)
    _check(mmf, up[::-1].copy().astype(dtype), 97)


@pytest.mark.parametrize("dtype", DTYPES)
def test_edge_sizes(mmf, dtype):
    """n around the chunk and 8-element group boundaries, w = n, w > n."""
    for n in (1, 2, 7, 8, 9, 15, 16, 17, 63, 64, 65, 1000, 4097):
        a = synth.uniform(n, n, dtype)
        for w in {1, 2, min(n, 5), n}:
            if w <= MAX_W:
                _check(mmf, a, w)
    x = _gpu(synth.uniform(10, 1, dtype))
    mx, mn = mmf.filter1d(x, 11, kernel="wedge")
    assert mx.numel() == 0 and mn.numel() == 0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("off", [1, 3])
def test_unaligned_views(mmf, dtype, off):
    """Views whose start is not 16-byte aligned take the scalar load/store
    path of the kernel."""
    a = synth.random_walk(50_000, seed=off, dtype=dtype)
    x = _gpu(a)[off:]
    w = 77
    m = x.numel() - w + 1
    ob = torch.empty(m + 8, dtype=x.dtype, device="cuda")
    nb = torch.empty(m + 8, dtype=x.dtype, device="cuda")
    mmf.filter1d(x, w, out_max=ob[off:off + m], out_min=nb[off:off + m], kernel="wedge")
    torch.cuda.synchronize()
    emx, emn = oracle.bf1d(a[off:], w)
    _same(ob[off:off + m].cpu().numpy(), nb[off:off + m].cpu().numpy(), emx, emn, f"off={off}")


def test_single_side(mmf):
    a = synth.uniform(30_000, 9, np.float32)
    x = _gpu(a)
    emx, emn = oracle.bf1d(a, 40)
    mx, mn = mmf.filter1d(x, 40, kernel="wedge", want_min=False)
    assert mn is None and np.array_equal(mx.cpu().numpy(), emx)
    mx, mn = mmf.filter1d(x, 40, kernel="wedge", want_max=False)
    assert mx is None and np.array_equal(mn.cpu().numpy(), emn)


def test_limits_are_errors(mmf):
    x = _gpu(synth.uniform(5000, 2, np.float32))
    with pytest.raises(mmf.MMFError):
        mmf.filter1d(x, MAX_W + 1, kernel="wedge")
    with pytest.raises(mmf.MMFError):
        mmf.filter1d(x, 5, mode="envelope", kernel="wedge")
    assert mmf.device_status(reset=True) == 0


def test_same_as_blockscan_sine(mmf):
    """The paper's sine input: the wedge and the block-scan kernels agree
    with each other and with the definition."""
    a = synth.sine(1_000_000, np.float64)
    x = _gpu(a)
    for w in (10, 300):
        wm, wn = mmf.filter1d(x, w, kernel="wedge")
        bm, bn = mmf.filter1d(x, w, kernel="blockscan")
        assert torch.equal(wm, bm) and torch.equal(wn, bn)
        emx, emn = oracle.bf1d(a, w)
        _same(wm.cpu().numpy(), wn.cpu().numpy(), emx, emn, f"sine w={w}")


@pytest.mark.parametrize("w", [3, 31, MAX_W])
def test_full_size_sampled(mmf, w):
    """n = 2^30 piecewise-monotone f32 (the long-stream size, the launch the
    benchmark times): equal to the block-scan kernel everywhere and to the
    definition at sampled windows, including every chunk boundary region."""
    n = 1 << 30
    x = synth.torch_by_name("piecewise_monotone", n, seed=31, device="cuda")
    wm, wn = mmf.filter1d(x, w, kernel="wedge")
    bm, bn = mmf.filter1d(x, w, kernel="blockscan")
    torch.cuda.synchronize()
    assert torch.equal(wm, bm) and torch.equal(wn, bn)
    m = n - w + 1
    rng = np.random.default_rng(w)
    starts = np.concatenate([rng.integers(0, m, size=4000), [0, 1, m - 1, m - 2]]).astype(np.int64)
    a = x.cpu().numpy()
    emx, emn = oracle.bf1d_at(a, w, starts)
    idx = torch.from_numpy(starts).cuda()
    _same(wm[idx].cpu().numpy(), wn[idx].cpu().numpy(), emx, emn, f"sampled w={w}")
    del x, wm, wn, bm, bn
    torch.cuda.empty_cache()
