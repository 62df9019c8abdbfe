"""GPU tests of the autotuners: a forced bad choice is replaced by the tuned
one, and outputs stay identical (every kernel computes the same exact
filter).

* Batch plans tune three knobs: the short-series cut-off (one warp per
  series against block-scan work items of a whole CTA), the register-slide
  limit (kernel choice for small windows) and the segment length per group.
* mmf_filter1d's automatic choice consults a dispatch table per (dtype,
  window bucket, length bucket) that mmf_dispatch_autotune fills."""
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


def test_plan_knobs_forced_bad_are_retuned(mmf, tmp_path, monkeypatch):
    """Envelope batch of 100 000 short series: with the warp-per-series kernel
    switched off (every series a block-scan item), the tuner brings it back;
    outputs are identical throughout and match the oracle."""
    monkeypatch.setenv("MMF_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    ns, L, r = 100_000, 1024, 51
    z = torch.from_numpy(synth.znorm_walks(ns, L, 33, np.float32).reshape(-1)).cuda()
    plan = mmf.BatchPlan(np.full(ns, L), np.full(ns, r), torch.float32, "envelope")
    ref_u, ref_l = plan(z)
    plan.set_knobs(short_cut=0, slide_max=1)
    assert plan.knobs()["short_cut"] == 0
    bu, bl = plan(z)
    knobs = (plan.autotune(z), plan.knobs())[1]
    assert knobs["short_cut"] > 0, knobs  # one warp per series wins over CTA items
    tu, tl = plan(z)
    torch.cuda.synchronize()
    assert torch.equal(bu, ref_u) and torch.equal(bl, ref_l)
    assert torch.equal(tu, ref_u) and torch.equal(tl, ref_l)
    off = plan.out_offsets()
    host = z.cpu().numpy()
    for s in (0, 1, 777, ns - 1):
        eu, el = oracle.envelope(host[s * L:(s + 1) * L], r)
        assert np.array_equal(tu.cpu().numpy()[off[s]:off[s] + L], eu)
        assert np.array_equal(tl.cpu().numpy()[off[s]:off[s] + L], el)
    assert "short" in (tmp_path / "tune.txt").read_text()
    plan2 = mmf.BatchPlan(np.full(ns, L), np.full(ns, r), torch.float32, "envelope")
    assert plan2.knobs()["short_cut"] == knobs["short_cut"]  # read back from the cache
    plan.close()
    plan2.close()


def test_plan_slide_knob_and_uneven_batch(mmf):
    """Uneven batch with small windows: every slide limit and cut-off gives
    the same outputs as the oracle (the knobs move series between kernels)."""
    lens, ws, dists, seeds = synth.uneven_batch(64, seed=12, lo_exp=2.0, hi_exp=4.5, windows=(3, 5, 9, 17, 101))
    data = synth.uneven_batch_data(lens, dists, seeds, np.float32)
    x = torch.from_numpy(data).cuda()
    plan = mmf.BatchPlan(lens, ws, torch.float32)
    ref_m, ref_n = plan(x)
    for short_cut, slide_max in ((0, 1), (256, 5), (1024, 9), (512, 17)):
        plan.set_knobs(short_cut, slide_max)
        m, n = plan(x)
        torch.cuda.synchronize()
        assert torch.equal(m, ref_m) and torch.equal(n, ref_n), (short_cut, slide_max)
    off = plan.out_offsets()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    for s in range(len(lens)):
        em, en = oracle.bf1d(data[starts[s]:starts[s] + lens[s]], ws[s])
        assert np.array_equal(ref_m.cpu().numpy()[off[s]:off[s] + em.size], em)
        assert np.array_equal(ref_n.cpu().numpy()[off[s]:off[s] + en.size], en)
    with pytest.raises(mmf.MMFError):
        plan.set_knobs(2000, 5)  # beyond the warp-per-series kernel's length
    with pytest.raises(mmf.MMFError):
        plan.set_knobs(512, 18)  # beyond the register slide's window
    plan.close()


def test_dispatch_table_forced_bad_is_retuned(mmf, tmp_path, monkeypatch):
    """The automatic choice for f32, w = 400 over 2^24 elements is forced to
    the chunked wedge (far slower there); the tuner replaces it; every choice
    gives the oracle's outputs."""
    monkeypatch.setenv("MMF_AUTOTUNE_CACHE", str(tmp_path / "dispatch.txt"))
    n, w = 1 << 24, 400
    a = synth.random_walk(n, seed=4, dtype=np.float32)
    x = torch.from_numpy(a).cuda()
    builtin = mmf.dispatch_get(torch.float32, n, w)
    assert builtin == "blockscan"
    mmf.dispatch_set(torch.float32, n, w, "wedge")
    try:
        assert mmf.dispatch_get(torch.float32, n, w) == "wedge"
        wm, wn = mmf.filter1d(x, w)  # takes the wedge now
        chosen = mmf.dispatch_autotune(x, w)
        assert chosen != "wedge", chosen
        assert mmf.dispatch_get(torch.float32, n, w) == chosen
        tm, tn = mmf.filter1d(x, w)
        torch.cuda.synchronize()
        assert torch.equal(wm, tm) and torch.equal(wn, tn)
        em, en, _ = oracle.wedge(a, w)
        assert np.array_equal(tm.cpu().numpy(), em) and np.array_equal(tn.cpu().numpy(), en)
        assert "dispatch|" in (tmp_path / "dispatch.txt").read_text()
        # An entry whose kernel cannot take a call is passed over: the wedge
        # does not compute envelopes, so AUTO keeps its rule there.
        mmf.dispatch_set(torch.float32, n, w, "wedge")
        um, ul = mmf.filter1d(x, (w - 1) // 2, mode="envelope")
        eu, el = oracle.envelope(a[:100_000], (w - 1) // 2)
        assert np.array_equal(um[:90_000].cpu().numpy(), eu[:90_000])
    finally:
        mmf.dispatch_set(torch.float32, n, w, "auto")
    assert mmf.dispatch_get(torch.float32, n, w) == builtin
    assert mmf.device_status() == 0
