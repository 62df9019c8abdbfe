"""GPU parity of the 1D filter (mmf_filter1d through the C ABI) against the
CPU oracle: bit-exact for every dtype, since a max or min returns an input."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NP2T = {np.float32: torch.float32, np.float64: torch.float64, np.int16: torch.int16, np.uint8: torch.uint8}
DTYPES = [np.float32, np.float64, np.int16, np.uint8]


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _expect(a, w):
    # The definition for modest sizes, Algorithm 1 (pinned to it) for large w.
    if a.size * w <= 4e8:
        return oracle.bf1d(a, w)
    mx, mn, _ = oracle.wedge(a, w)
    return mx, mn


def _check(mmf, a, w, mode="valid", kernel="auto"):
    x = _gpu(a)
    mx, mn = mmf.filter1d(x, w, mode=mode, kernel=kernel)
    torch.cuda.synchronize()
    if mode == "valid":
        emx, emn = _expect(a, w)
    else:
        emx, emn = oracle.envelope(a, w)
    gm, gn = mx.cpu().numpy(), mn.cpu().numpy()
    assert gm.shape == emx.shape
    if not np.array_equal(gm, emx):
        bad = np.nonzero(gm != emx)[0]
        raise AssertionError(f"max mismatch w={w} n={a.size}: {bad.size} bad, first {bad[:8]}")
    if not np.array_equal(gn, emn):
        bad = np.nonzero(gn != emn)[0]
        raise AssertionError(f"min mismatch w={w} n={a.size}: {bad.size} bad, first {bad[:8]}")


WINDOWS = [1, 2, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33, 101, 255, 256, 257, 258, 511, 512, 513, 1001, 1024, 1025,
           2047, 2048, 2049, 4095, 4096, 4097, 4098, 8193, 12289]


@pytest.mark.parametrize("w", WINDOWS)
def test_f32_windows_random_walk(mmf, w):
    a = synth.random_walk(61_237, seed=w, dtype=np.float32)
    _check(mmf, a, w)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("kernel", ["slide", "blockscan"])
@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 15, 16, 17])
def test_small_windows_each_kernel(mmf, dtype, kernel, w):
    """Windows up to 17 (9 for types other than f32) through the register
    slide and through the block scan (blocks inside a thread), bit-exact."""
    if kernel == "slide" and dtype != np.float32 and w > 9:
        pytest.skip("the register slide covers w <= 9 for this type")
    a = synth.random_walk(30_011, seed=w, dtype=dtype)
    _check(mmf, a, w, kernel=kernel)
    off = synth.uniform(10_007, seed=w, dtype=dtype)
    x = _gpu(off)[3:]
    mx, mn = mmf.filter1d(x, w, kernel=kernel)
    emx, emn = oracle.bf1d(off[3:], w)
    assert np.array_equal(mx.cpu().numpy(), emx) and np.array_equal(mn.cpu().numpy(), emn)


def test_slide_rejects_large_window(mmf):
    x = torch.zeros(100, device="cuda")
    with pytest.raises(mmf.MMFError):
        mmf.filter1d(x, 18, kernel="slide")
    with pytest.raises(mmf.MMFError):
        mmf.filter1d(x.double(), 10, kernel="slide")
    with pytest.raises(mmf.MMFError):
        mmf.filter1d(x.to(torch.int16), 10, kernel="slide")


@pytest.mark.parametrize("w", [2, 4, 5, 9, 33, 127, 128, 129, 130, 1023, 1024, 1025, 1026, 2049, 3075])
def test_f64_windows(mmf, w):
    a = synth.piecewise_monotone(23_457, seed=w, dtype=np.float64)
    _check(mmf, a, w)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dist", synth.DISTS)
@pytest.mark.parametrize("w", [3, 31, 1001, 5000])
def test_dtypes_distributions(mmf, dtype, dist, w):
    a = synth.by_name(dist, 40_003, seed=7, dtype=dtype)
    _check(mmf, a, w)


@pytest.mark.parametrize("dtype", DTYPES)
def test_edge_sizes(mmf, dtype):
    for n, w in [(1, 1), (2, 1), (2, 2), (3, 2), (7, 7), (4096, 4096), (4097, 4096), (4097, 2),
                 (8192, 4097), (8193, 8193), (100, 99), (12_345, 12_345), (5, 3)]:
        a = synth.uniform(n, seed=n + w, dtype=dtype)
        _check(mmf, a, w)


def test_empty_and_oversized_window(mmf):
    x = torch.zeros(0, device="cuda")
    mx, mn = mmf.filter1d(x, 3)
    assert mx.numel() == 0 and mn.numel() == 0
    x = torch.arange(10, device="cuda", dtype=torch.float32)
    mx, mn = mmf.filter1d(x, 11)
    assert mx.numel() == 0


def test_monotone_and_constant(mmf):
    a = synth.monotone(50_000, 3, np.float32)
    x = _gpu(a)
    for w in (3, 1000, 5000):
        mx, mn = mmf.filter1d(x, w)
        assert np.array_equal(mx.cpu().numpy(), a[w - 1:])
        assert np.array_equal(mn.cpu().numpy(), a[: a.size - w + 1])
    c = torch.full((9999,), 2.5, device="cuda")
    mx, mn = mmf.filter1d(c, 77)
    assert bool((mx == 2.5).all()) and bool((mn == 2.5).all())


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("off", [1, 2, 3, 5, 7, 13])
@pytest.mark.parametrize("w,kernel", [(3, "auto"), (3, "blockscan"), (257, "auto"), (1001, "auto"),
                                      (5000, "auto")])
def test_unaligned_input_and_output(mmf, dtype, off, w, kernel):
    """Sub-tensor views whose start is not 16-byte aligned, through each
    kernel path (register slide, blocks in a thread, across lanes, per warp,
    tile aggregates): inputs are realigned after the copy and outputs are
    moved across lanes to whole 16-byte stores.  The offsets reach every
    distance to the next 16-byte boundary for each type; the elements around
    the output view stay untouched."""
    a = synth.random_walk(30_000, seed=off + w, dtype=dtype)
    big = _gpu(a)
    x = big[off:]
    m = x.numel() - w + 1
    obuf = torch.zeros(m + 2 * off, dtype=x.dtype, device="cuda")
    nbuf = torch.zeros(m + 2 * off, dtype=x.dtype, device="cuda")
    mmf.filter1d(x, w, out_max=obuf[off:off + m], out_min=nbuf[off:off + m], kernel=kernel)
    torch.cuda.synchronize()
    emx, emn = oracle.bf1d(a[off:], w)
    ob, nb = obuf.cpu().numpy(), nbuf.cpu().numpy()
    assert np.array_equal(ob[off:off + m], emx)
    assert np.array_equal(nb[off:off + m], emn)
    assert not ob[:off].any() and not ob[off + m:].any()
    assert not nb[:off].any() and not nb[off + m:].any()


@pytest.mark.parametrize("dtype", DTYPES)
def test_unaligned_max_only(mmf, dtype):
    """One output side, not 16-byte aligned."""
    a = synth.uniform(20_011, seed=3, dtype=dtype)
    x = _gpu(a)
    m = x.numel() - 1001 + 1
    obuf = torch.zeros(m + 1, dtype=x.dtype, device="cuda")
    mmf.filter1d(x, 1001, out_max=obuf[1:], want_min=False)
    emx, _ = oracle.bf1d(a, 1001)
    ob = obuf.cpu().numpy()
    assert np.array_equal(ob[1:], emx) and ob[0] == 0


def test_single_side_outputs(mmf):
    a = synth.uniform(20_000, 4, np.float32)
    x = _gpu(a)
    mx, mn = mmf.filter1d(x, 55, want_min=False)
    assert mn is None
    emx, emn = oracle.bf1d(a, 55)
    assert np.array_equal(mx.cpu().numpy(), emx)
    mx, mn = mmf.filter1d(x, 55, want_max=False)
    assert mx is None and np.array_equal(mn.cpu().numpy(), emn)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("r", [0, 1, 51, 700, 5000, 100_000])
def test_envelope(mmf, dtype, r):
    a = synth.random_walk(9_001, seed=r, dtype=dtype)
    _check(mmf, a, r, mode="envelope")


def test_envelope_unaligned_short_series(mmf):
    a = synth.znorm_walks(3, 1024, 33)
    flat = a.reshape(-1)
    big = _gpu(flat)
    for s in range(3):
        x = big[s * 1024 + 1:(s + 1) * 1024]
        up, lo = mmf.filter1d(x, 51, mode="envelope")
        eup, elo = oracle.envelope(flat[s * 1024 + 1:(s + 1) * 1024], 51)
        assert np.array_equal(up.cpu().numpy(), eup) and np.array_equal(lo.cpu().numpy(), elo)


def test_sine_wave_paper_input(mmf):
    a = synth.sine(1_000_000, np.float64)
    for w in (10, 1000, 30_000):
        _check(mmf, a, w)


def test_device_status_clean(mmf):
    assert mmf.device_status(reset=True) == 0


@pytest.mark.parametrize("w", [3, 31, 1001, 65537])
def test_full_size_long_stream_sampled(mmf, w):
    """n = 2^30 fp32 (the long-stream workload), same launch as the bench:
    sampled windows against the definition (a million random starts for
    small windows, about 2e9 / w for large ones, plus the ends and a stride
    through every CTA's range), plus the bracketing property max >= min on
    every output."""
    n = 1 << 30
    x = synth.torch_by_name("random_walk", n, seed=22, device="cuda")
    mx, mn = mmf.filter1d(x, w)
    torch.cuda.synchronize()
    m = n - w + 1
    assert bool((mx >= mn).all())
    rng = np.random.default_rng(w)
    starts = np.concatenate([rng.integers(0, m, size=min(1_000_000, 2_000_000_000 // w)), [0, 1, m - 1, m - 2],
                             np.arange(0, m, 4096 * 152 * 7)[:400]]).astype(np.int64)
    a = x.cpu().numpy()
    emx, emn = oracle.bf1d_at(a, w, starts)
    idx = torch.from_numpy(starts).cuda()
    assert np.array_equal(mx[idx].cpu().numpy(), emx)
    assert np.array_equal(mn[idx].cpu().numpy(), emn)
    del x, mx, mn
    torch.cuda.empty_cache()
    assert mmf.device_status(reset=True) == 0


@pytest.mark.parametrize("w", [2049, 4097, 4200, 6145, 8193])
def test_long_items_large_windows(mmf, w):
    """Windows of 1-4 whole tiles with items of many tiles (few CTAs per
    series): the sliding range of whole tiles between j and k advances
    across many output tiles of one item."""
    a = synth.random_walk(8_000_000, seed=w, dtype=np.float32)
    _check(mmf, a, w)
    b = synth.piecewise_monotone(700_001, seed=w, dtype=np.float32)
    _check(mmf, b, w)


@pytest.mark.parametrize("mode,w", [("valid", 3), ("valid", 1001), ("valid", 70_001), ("envelope", 0),
                                    ("envelope", 51), ("envelope", 40_000)])
def test_host_pipeline_equals_oracle(mmf, mode, w):
    """Host arrays through the chunked pipeline (small chunks, so many of
    them, with windows shorter and longer than a chunk) equal the oracle."""
    a = synth.random_walk(300_007, seed=w + 1, dtype=np.float32)
    x = torch.from_numpy(a)
    mx, mn = mmf.filter1d_host(x, w, mode=mode, chunk=20_000)
    torch.cuda.current_stream().synchronize()
    emx, emn = oracle.bf1d(a, w) if mode == "valid" else oracle.envelope(a, w)
    assert np.array_equal(mx.numpy(), emx) and np.array_equal(mn.numpy(), emn)


def test_host_pipeline_types_and_calls_in_a_row(mmf):
    for dtype in DTYPES:
        a = synth.uniform(50_001, seed=9, dtype=dtype)
        x = torch.from_numpy(a)
        outs = [mmf.filter1d_host(x, w, chunk=4096) for w in (2, 257)]
        torch.cuda.current_stream().synchronize()
        for (mx, mn), w in zip(outs, (2, 257)):
            emx, emn = oracle.bf1d(a, w)
            assert np.array_equal(mx.numpy(), emx) and np.array_equal(mn.numpy(), emn)
    assert mmf.device_status() == 0
