"""GPU parity of the batched filter (plan + persistent launches + graph)
against the oracle, series by series; bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NP2T = {np.float32: torch.float32, np.float64: torch.float64, np.int16: torch.int16, np.uint8: torch.uint8}


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _check_batch(mmf, data, lens, ws, mode="valid", in_offsets=None, dtype=np.float32, **kw):
    plan = mmf.BatchPlan(lens, ws, NP2T[dtype], mode, in_offsets=in_offsets)
    x = torch.from_numpy(data).cuda()
    mx, mn = plan(x)
    torch.cuda.synchronize()
    off = plan.out_offsets()
    gm, gn = mx.cpu().numpy(), mn.cpu().numpy()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]]) if in_offsets is None else np.asarray(in_offsets)
    for s in range(len(lens)):
        a = data[starts[s]:starts[s] + lens[s]]
        em, en = oracle.bf1d(a, ws[s]) if mode == "valid" else oracle.envelope(a, ws[s])
        # Series s's outputs start on a 32-byte boundary; padding follows.
        assert off[s] * data.itemsize % 32 == 0 and off[s] + em.size <= off[s + 1]
        assert np.array_equal(gm[off[s]:off[s] + em.size], em), f"series {s} max (len {lens[s]}, w {ws[s]})"
        assert np.array_equal(gn[off[s]:off[s] + en.size], en), f"series {s} min"
    # Replay from the cached graph and the plain per-series form agree.
    mx2, mn2 = plan(x)
    pm, pn = plan.per_series(x)
    torch.cuda.synchronize()
    assert torch.equal(mx2, mx) and torch.equal(mn2, mn)
    assert torch.equal(pm, mx) and torch.equal(pn, mn)
    plan.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
def test_uneven_batch_small(mmf, dtype):
    lens, ws, dists, seeds = synth.uneven_batch(96, seed=31, lo_exp=1.0, hi_exp=4.3)
    data = synth.uneven_batch_data(lens, dists, seeds, dtype)
    _check_batch(mmf, data, lens, ws, dtype=dtype)


def test_every_kernel_group(mmf):
    """Windows that land in each kernel group (slide, blocks in a thread,
    across lanes, per warp, tile aggregates), lengths with ragged tails."""
    ws = [1, 2, 3, 9, 10, 16, 31, 255, 256, 257, 1001, 2048, 2049, 5000, 10001]
    lens = [20_000 + 37 * i for i in range(len(ws))]
    data = synth.uneven_batch_data(np.array(lens), np.arange(len(ws)) % 3, np.arange(len(ws)) + 5)
    _check_batch(mmf, data, lens, ws)


def test_tiny_and_clipped(mmf):
    lens = [1, 2, 3, 5, 17, 100, 1000, 4096, 4097]
    ws = [1, 2, 3, 5, 17, 100, 1000, 4096, 4097]  # w == len: one output each
    data = synth.uniform(int(sum(lens)), 3, np.float32)
    _check_batch(mmf, data, lens, ws)


def test_explicit_offsets_unaligned(mmf):
    rng = np.random.default_rng(5)
    lens = rng.integers(50, 30_000, size=40)
    gaps = rng.integers(0, 7, size=40)
    offs = np.cumsum(np.concatenate([[3], lens[:-1] + gaps[:-1]]))
    total = int(offs[-1] + lens[-1] + 5)
    data = synth.random_walk(total, 9, np.float32)
    ws = np.minimum(rng.choice([3, 15, 101, 1001, 10001], size=40), lens)
    _check_batch(mmf, data, lens, ws, in_offsets=offs)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_envelope_batch(mmf, dtype):
    x = synth.znorm_walks(300, 1024, 33, dtype)
    lens = np.full(300, 1024)
    rs = np.full(300, 51)
    _check_batch(mmf, x.reshape(-1), lens, rs, mode="envelope", dtype=dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
@pytest.mark.parametrize("mode", ["valid", "envelope"])
def test_short_series_both_decompositions(mmf, dtype, mode):
    """Series short enough for the warp-per-series kernel (at most 1024
    elements, 512 for f64), windows on both sides of one lane's 32 (16 for
    f64) elements: blocks of w elements below, the lanes as blocks above.
    Ragged lengths, windows of E, E+1, 2E, 2E+1, up to the whole series;
    radii from 0 past the series' length; unaligned starts, and the last
    series ending at the buffer's end (its loads cannot read ahead)."""
    E = 16 if dtype == np.float64 else 32
    cap = 32 * E
    rng = np.random.default_rng(7 + E + (mode == "envelope"))
    lens, ws = [], []
    for n in list(rng.integers(1, cap + 1, size=120)) + [cap, cap, cap - 1, E + 1, 2 * E + 3, 1]:
        n = int(n)
        if mode == "valid":
            cand = [1, E - 1, E, E + 1, 2 * E, 2 * E + 1, 3 * E + 7, n // 2 + 1, n - 1, n]
            w = int(rng.choice([c for c in cand if 1 <= c <= n]))
        else:
            cand = [0, 1, E // 2 - 1, E // 2, E // 2 + 1, E, E + 3, n // 3, n - 1, n + 5]
            w = int(rng.choice([c for c in cand if c >= 0]))
        lens.append(n)
        ws.append(w)
    lens, ws = np.array(lens), np.array(ws)
    gaps = rng.integers(0, 7, size=len(lens))
    offs = np.cumsum(np.concatenate([[5], (lens + gaps)[:-1]]))
    total = int(offs[-1] + lens[-1])  # nothing after the last series
    data = synth.uniform(total, 11, np.float64)
    if dtype in (np.float32, np.float64):
        data = data.astype(dtype)
    else:
        lo, hi = (0, 255) if dtype == np.uint8 else (-32768, 32767)
        data = (lo + np.floor(data * (hi - lo + 1))).clip(lo, hi).astype(dtype)
    _check_batch(mmf, data, lens, ws, mode=mode, in_offsets=offs, dtype=dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("mode", ["valid", "envelope"])
def test_short_series_many_per_warp(mmf, dtype, mode):
    """Many more short series than warps (each warp takes about eight in
    turn), so a warp stages its next series in shared memory while it
    finishes the current one: windows on both sides of the lane width in
    random order (a staged series follows a lane-block one; a w-block series
    stages nothing), 16-byte aligned and unaligned starts, lengths below and
    at the maximum, every series against the oracle."""
    E = 16 if dtype == np.float64 else 32
    cap = 32 * E
    nser = 20_000
    rng = np.random.default_rng(23 + E + (mode == "envelope"))
    lens = np.where(rng.random(nser) < 0.5, cap, rng.integers(1, cap + 1, nser))
    if mode == "valid":
        ws = np.minimum(np.where(rng.random(nser) < 0.8, rng.integers(E + 1, 3 * E + 40, nser),
                                 rng.integers(1, E + 1, nser)), lens)
    else:
        ws = np.where(rng.random(nser) < 0.8, rng.integers(E // 2, 3 * E, nser), rng.integers(0, E // 2, nser))
    step = 16 // np.dtype(dtype).itemsize
    gaps = np.where(rng.random(nser) < 0.7, (-lens) % step, rng.integers(0, step, nser))  # mostly aligned starts
    offs = np.cumsum(np.concatenate([[0], (lens + gaps)[:-1]]))
    total = int(offs[-1] + lens[-1])
    data = synth.random_walk(total, 29, dtype)
    plan = mmf.BatchPlan(lens, ws, NP2T[dtype], mode, in_offsets=offs)
    x = torch.from_numpy(data).cuda()
    mx, mn = plan(x)
    torch.cuda.synchronize()
    off = plan.out_offsets()
    gm, gn = mx.cpu().numpy(), mn.cpu().numpy()
    plan.close()
    for s in range(nser):
        a = data[offs[s]:offs[s] + lens[s]]
        em, en = oracle.bf1d(a, int(ws[s])) if mode == "valid" else oracle.envelope(a, int(ws[s]))
        assert np.array_equal(gm[off[s]:off[s] + em.size], em), f"series {s} max (len {lens[s]}, w {ws[s]})"
        assert np.array_equal(gn[off[s]:off[s] + en.size], en), f"series {s} min (len {lens[s]}, w {ws[s]})"
    assert mmf.device_status() == 0


def test_segments_and_autotune(mmf, tmp_path, monkeypatch):
    monkeypatch.setenv("MMF_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    lens, ws, dists, seeds = synth.uneven_batch(64, seed=8, lo_exp=3.0, hi_exp=5.0)
    data = synth.uneven_batch_data(lens, dists, seeds, np.float32)
    plan = mmf.BatchPlan(lens, ws, torch.float32)
    x = torch.from_numpy(data).cuda()
    ref_m, ref_n = plan(x)
    for seg in (1, 3, 64):
        for g in range(4):
            plan.set_segment(g, seg)
        m, n = plan(x)
        assert torch.equal(m, ref_m) and torch.equal(n, ref_n)
    segs = plan.autotune(x)
    assert all(s >= 1 for s in segs)
    m, n = plan(x)
    torch.cuda.synchronize()
    assert torch.equal(m, ref_m) and torch.equal(n, ref_n)
    assert (tmp_path / "tune.txt").exists()
    plan2 = mmf.BatchPlan(lens, ws, torch.float32)  # picks the cached choice
    m2, n2 = plan2(x)
    assert torch.equal(m2, ref_m)
    assert mmf.device_status() == 0
