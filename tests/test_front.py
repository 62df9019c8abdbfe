"""GPU parity of the advancing-front block scan (MMF_KERNEL_FRONT), a
schedule for windows of a tile or more: output tiles go to the CTAs of a
cooperative grid round-robin, and the aggregates of the whole tiles inside
each window come from the CTAs that read those tiles a round ahead.  Compared
with the oracle's Algorithm 1 (pinned to the definition) at every output, and
with the per-range block scan."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NP2T = {np.float32: torch.float32, np.int16: torch.int16, np.uint8: torch.uint8}
TILE = {np.float32: 2048, np.int16: 4096, np.uint8: 4096}


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _data(dtype, n, seed, dist="random_walk"):
    a = synth.by_name(dist, n, seed, np.float64 if dtype != np.float32 else np.float32)
    if dtype == np.float32:
        return a
    scale = 20.0 if dtype == np.uint8 else 300.0
    v = np.rint(a * scale).astype(np.int64)
    lo, hi = (0, 255) if dtype == np.uint8 else (-32768, 32767)
    return (np.mod(v - lo, hi - lo + 1) + lo).astype(dtype)


def _run(mmf, a, w, kernel, mode="valid"):
    x = torch.from_numpy(a).cuda()
    mx, mn = mmf.filter1d(x, w, mode=mode, kernel=kernel)
    torch.cuda.synchronize()
    return mx.cpu().numpy(), mn.cpu().numpy()


@pytest.mark.parametrize("dtype", [np.float32, np.int16, np.uint8])
@pytest.mark.parametrize("tiles_plus", [(1, 0), (1, 1), (2, 5), (4, 1000), (8, 0), (8, 1), (31, 77), (32, 1)])
def test_front_equals_algorithm1(mmf, dtype, tiles_plus):
    """Windows of q whole tiles plus a remainder (q = 1 .. 32), ragged
    lengths, several distributions: every output equals the oracle's."""
    q, extra = tiles_plus
    w = q * TILE[dtype] + extra + 1
    for dist, n in (("random_walk", 40 * TILE[dtype] * 4 + 777), ("uniform", w + 5 * TILE[dtype] + 3),
                    ("piecewise_monotone", 3 * w + 12_345)):
        a = _data(dtype, n, seed=q * 31 + extra, dist=dist)
        gm, gn = _run(mmf, a, w, "front")
        em, en, _ = oracle.wedge(a, w)
        assert np.array_equal(gm, em), f"max {np.dtype(dtype).name} w={w} {dist} n={n}"
        assert np.array_equal(gn, en), f"min {np.dtype(dtype).name} w={w} {dist} n={n}"
    assert mmf.device_status() == 0


@pytest.mark.parametrize("r", [1024, 1500, 20_000, 40_000])
def test_front_envelope(mmf, r):
    """Centred windows clipped at both ends (virtual identities before and
    after the series, so the first and last tiles are partly outside)."""
    a = synth.random_walk(600_001, seed=r, dtype=np.float32)
    gm, gn = _run(mmf, a, r, "front", mode="envelope")
    em, en = oracle.envelope(a[:200_000], r)
    assert np.array_equal(gm[:150_000], em[:150_000]) and np.array_equal(gn[:150_000], en[:150_000])
    bm, bn = _run(mmf, a, r, "blockscan", mode="envelope")
    assert np.array_equal(gm, bm) and np.array_equal(gn, bn)
    tail_m, tail_n = oracle.envelope(a[-200_000:], r)
    assert np.array_equal(gm[-150_000:], tail_m[-150_000:]) and np.array_equal(gn[-150_000:], tail_n[-150_000:])


@pytest.mark.parametrize("w", [16_385, 65_537, 65_538, 100_001])
def test_front_long_series_vs_ranges(mmf, w):
    """Many more rounds than CTAs (2^26 elements): the front, the per-range
    schedule and the automatic choice agree at every output; sampled windows
    against the definition."""
    n = 1 << 26
    x = synth.torch_by_name("random_walk", n, seed=w, device="cuda")
    fm, fn = mmf.filter1d(x, w, kernel="front")
    bm, bn = mmf.filter1d(x, w, kernel="blockscan")
    am, an = mmf.filter1d(x, w)  # the automatic choice (the per-range schedule)
    torch.cuda.synchronize()
    assert torch.equal(fm, bm) and torch.equal(fn, bn)
    assert torch.equal(am, fm) and torch.equal(an, fn)
    m = n - w + 1
    rng = np.random.default_rng(w)
    starts = np.concatenate([rng.integers(0, m, 20_000), [0, 1, m - 2, m - 1]]).astype(np.int64)
    em, en = oracle.bf1d_at(x.cpu().numpy(), w, starts)
    idx = torch.from_numpy(starts).cuda()
    assert np.array_equal(fm[idx].cpu().numpy(), em) and np.array_equal(fn[idx].cpu().numpy(), en)
    assert mmf.device_status() == 0


def test_front_refusals(mmf):
    """The front takes windows of a tile or more and not f64."""
    x = torch.rand(100_000, device="cuda")
    with pytest.raises(mmf.MMFError) as e:
        mmf.filter1d(x, 2048, kernel="front")  # w - 1 < one tile
    assert e.value.status == 7
    with pytest.raises(mmf.MMFError) as e:
        mmf.filter1d(x.double(), 5000, kernel="front")
    assert e.value.status == 7
    mx, mn = mmf.filter1d(x, 2049, kernel="front")
    em, en, _ = oracle.wedge(x.cpu().numpy(), 2049)
    assert np.array_equal(mx.cpu().numpy(), em) and np.array_equal(mn.cpu().numpy(), en)
