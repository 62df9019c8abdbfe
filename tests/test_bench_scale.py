"""Parity at the benchmark's sizes and launch configurations, for the kernel
paths that only the full-size workloads reach:

* the uneven batch (4096 series, lengths log-uniform in [1e3, 1e6], windows
  from {3, 15, 101, 1001, 10001}; inputs drawn on the device as the benchmark
  does): many more work items than the persistent grid, so every CTA takes
  item after item from the ticket (at the autotuned segments, at one tile per
  item, and one launch per series);
* the envelope batch (1e6 z-normalised series of 1024, r = 51) through the
  warp-per-series kernel;
* the fused 2D filter on 4096 x 4096 f32 images at 3 x 3, where the
  persistent tile kernel loops over about 13 output tiles per CTA, and the
  streaming kernel (the automatic choice) covers 64 bands of rows per image.

Outputs are compared with the oracle at sampled windows (every series' or
image's ends included); the GPU forms are compared with each other at every
output.  Bit-exact throughout."""
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


def _uneven_input(lens, dists, dev, tdt):
    """The benchmark's input: each series takes its distribution's values (a
    full-length draw per distribution) at its own offset."""
    total = int(lens.sum())
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    src = [synth.torch_by_name(d, total, 31 + i, dev, tdt) for i, d in enumerate(synth.DISTS)]
    x = src[0]
    for i in range(lens.size):
        if dists[i]:
            a, b = int(starts[i]), int(starts[i] + lens[i])
            x[a:b] = src[dists[i]][a:b]
    del src
    return x, starts


@pytest.mark.parametrize("tdt", [torch.float32, torch.float64])
def test_uneven_batch_full_size(mmf, tdt):
    dev = torch.device("cuda")
    lens, ws, dists, _ = synth.uneven_batch(4096, seed=31)
    x, starts = _uneven_input(lens, dists, dev, tdt)
    plan = mmf.BatchPlan(lens, ws, tdt)
    assert sum(plan.items_per_group) > 8 * 304  # many items per CTA of the one-wave grid
    om = torch.empty(plan.out_len, dtype=tdt, device=dev)
    on = torch.empty(plan.out_len, dtype=tdt, device=dev)
    plan.autotune(x, om, on)
    gm, gn = plan(x)
    for g in range(4):
        plan.set_segment(g, 1)
    g1m, g1n = plan(x)
    pm, pn = plan.per_series(x)
    torch.cuda.synchronize()
    assert torch.equal(g1m, gm) and torch.equal(g1n, gn), "one tile per item differs from the tuned segments"
    assert torch.equal(pm, gm) and torch.equal(pn, gn), "per-series launches differ from the batch"
    off = plan.out_offsets()
    plan.close()
    host = x.cpu().numpy()
    hm, hn = gm.cpu().numpy(), gn.cpu().numpy()
    rng = np.random.default_rng(3)
    for s in range(lens.size):
        a = host[starts[s]:starts[s] + lens[s]]
        m = int(lens[s] - ws[s] + 1)
        js = np.unique(np.concatenate([[0, 1, m - 2, m - 1], rng.integers(0, m, 24)]).clip(0, m - 1))
        em, en = oracle.bf1d_at(a, int(ws[s]), js)
        assert np.array_equal(hm[off[s] + js], em), f"series {s} max (len {lens[s]}, w {ws[s]})"
        assert np.array_equal(hn[off[s] + js], en), f"series {s} min (len {lens[s]}, w {ws[s]})"
    assert mmf.device_status() == 0


def test_envelope_batch_full_size(mmf):
    dev = torch.device("cuda")
    ns, L, r = 1_000_000, 1024, 51
    g = torch.Generator(device=dev)
    g.manual_seed(33)
    z = torch.cumsum(torch.randn(ns, L, generator=g, device=dev, dtype=torch.float64), 1)
    z = ((z - z.mean(1, keepdim=True)) / z.std(1, unbiased=False, keepdim=True)).float().reshape(-1) + 0.0
    plan = mmf.BatchPlan(np.full(ns, L), np.full(ns, r), torch.float32, "envelope")
    um, lm = plan(z)
    torch.cuda.synchronize()
    off = plan.out_offsets()
    plan.close()
    rng = np.random.default_rng(5)
    picks = np.unique(np.concatenate([[0, 1, ns - 1], rng.integers(0, ns, 3000)]))
    host = z.cpu().numpy()
    hu, hl = um.cpu().numpy(), lm.cpu().numpy()
    for s in picks:
        eu, el = oracle.envelope(host[s * L:(s + 1) * L], r)
        assert np.array_equal(hu[off[s]:off[s] + L], eu), f"series {s} upper"
        assert np.array_equal(hl[off[s]:off[s] + L], el), f"series {s} lower"


@pytest.mark.parametrize("fuse", [-1, 1, 2])
def test_2d_f32_full_size_persistent_tiles(mmf, fuse):
    """Four 4096 x 4096 f32 images at 3 x 3: the automatic choice (the
    streaming kernel), the forced tile kernel (its persistent tile loop) and
    the forced streaming kernel against the literal rectangle at every pixel
    of each image's first and last two rows and columns and at 20 000 random
    pixels, and against the two-pass form at every pixel."""
    imgs = synth.blobs2d(4, 4096, 4096, seed=41, dtype=np.float32, nblobs=200)
    x = torch.from_numpy(imgs).cuda()
    mx, mn = mmf.filter2d(x, 3, 3, fuse=fuse)
    ux, un = mmf.filter2d(x, 3, 3, fuse=0)
    torch.cuda.synchronize()
    assert torch.equal(mx, ux) and torch.equal(mn, un)
    gm, gn = mx.cpu().numpy(), mn.cpu().numpy()
    Ho, Wo = gm.shape[1], gm.shape[2]
    rng = np.random.default_rng(11)
    for k in range(imgs.shape[0]):
        border_y = np.concatenate([np.repeat([0, 1, Ho - 2, Ho - 1], Wo), np.tile(np.arange(Ho), 4)])
        border_x = np.concatenate([np.tile(np.arange(Wo), 4), np.repeat([0, 1, Wo - 2, Wo - 1], Ho)])
        ys = np.concatenate([border_y, rng.integers(0, Ho, 20_000)])
        xs = np.concatenate([border_x, rng.integers(0, Wo, 20_000)])
        em, en = oracle.bf2d_at(imgs[k], 3, 3, ys, xs)
        assert np.array_equal(gm[k][ys, xs], em), f"image {k} max"
        assert np.array_equal(gn[k][ys, xs], en), f"image {k} min"
    assert mmf.device_status() == 0
