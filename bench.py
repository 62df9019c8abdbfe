"""Benchmark of the running max-min filter on the long-stream workload.

Workload (one "step"): an n = 2^30 fp32 stream for each of three seeded
distributions (i.i.d. uniform[0,1), N(0,1) random walk, piecewise monotone
runs of mean length 1000), filtered at each window w in {3, 31, 1001, 65537}
-- 12 calls of mmf_filter1d, 12 * 2^30 input elements.  Inputs (4 GiB each)
are larger than L2, so no flush is needed between timed iterations.

Prints ONE JSON line.  Metric: filtered Gelem/s (input elements per second,
whole job over all ranks).  ``--impl reference`` times the CPU oracle (the
paper's Algorithm 1, single thread) on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank filters its own independent streams (weak
scaling, no data-path collective); the barrier and the max-over-ranks timing
are the only communication.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "filtered Gelem/s"
N = 1 << 30
WINDOWS = (3, 31, 1001, 65537)
DISTS = ("uniform", "random_walk", "piecewise_monotone")
SEEDS = {"uniform": 21, "random_walk": 22, "piecewise_monotone": 23}
WORKLOAD = "long 1D stream: n=2^30 fp32 x {uniform, random walk, piecewise monotone} x w in {3,31,1001,65537}"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic():
    """dram bytes per launch from a committed ncu summary (None if absent)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time(elapsed_ms, per_rank_elems, ws, device="cpu"):
    """Whole-job timing across ranks: the slowest rank's elapsed time (max
    over ranks, all_reduce on the process group when ws > 1) and the elements
    all ranks processed (each rank filters its own streams: weak scaling, no
    data exchange).  Returns (elapsed_ms, total_elements, Gelem/s)."""
    import torch
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([float(elapsed_ms)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    total = per_rank_elems * ws
    return elapsed_ms, total, total / (elapsed_ms * 1e-3) / 1e9


def run_reference(args):
    """CPU oracle (Algorithm 1 on all host cores, chunks with a w-1 halo) on a
    bounded sample per step."""
    import oracle
    import synth
    ws, rank, _ = _dist_env()
    if rank != 0:
        return 0
    oracle.build()
    sample = args.ref_sample
    data = {d: synth.by_name(d, sample, SEEDS[d], np.float32) for d in DISTS}
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.wedge_mt(data["random_walk"][: sample // 8], 101, cores)
    used = 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for d in DISTS:
            for w in WINDOWS:
                used = oracle.wedge_mt(data[d], w, cores)[2]
    dt = time.perf_counter() - t0
    elems = args.steps * len(DISTS) * len(WINDOWS) * sample
    value = elems / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "windows": list(WINDOWS), "dists": list(DISTS),
                   "reference_sample_elements": sample},
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": used, "kind": "oracle",
                         "sample": f"first {sample} elements of each distribution (numpy-seeded), "
                                   f"Algorithm 1 wedge per window on {used} threads (chunks with a "
                                   f"w-1 halo), {args.steps} steps"},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(sample: int):
    """The oracle's Algorithm 1 on the host: all cores (chunks with a w-1
    halo, one thread each) as the reported figure, one core beside it."""
    import oracle
    import synth
    oracle.build()
    a = {d: synth.by_name(d, sample, SEEDS[d], np.float32) for d in DISTS}
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    used = 1
    for d in DISTS:
        for w in WINDOWS:
            used = oracle.wedge_mt(a[d], w, cores)[2]
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    for d in DISTS:
        for w in WINDOWS:
            oracle.wedge(a[d], w)
    dt1 = time.perf_counter() - t0
    # The definition itself (the naive row of Table 1, 2w-2 comparisons per
    # output), single thread, where it is feasible: w <= 1001, on a sample
    # of min(2^20, 2^28/w) elements per distribution (about a second each).
    naive = {}
    for w in (x for x in WINDOWS if x <= 1001):
        ns = min(sample, 1 << 20, (1 << 28) // w)
        t0 = time.perf_counter()
        for d in DISTS:
            oracle.bf1d(a[d][:ns], w)
        naive[str(w)] = {"value": len(DISTS) * ns / (time.perf_counter() - t0) / 1e9, "sample": ns}
    elems = len(DISTS) * len(WINDOWS) * sample
    return {"value": elems / dt / 1e9, "unit": "Gelem/s", "cores": used, "kind": "oracle",
            "single_core_value": elems / dt1 / 1e9, "naive_single_core_by_window": naive,
            "sample": f"{sample} elements per distribution x 3 distributions x 4 windows, "
                      f"Algorithm 1 wedge split into {used} chunks with a w-1 halo on {used} threads "
                      f"({dt:.1f} s); single thread {dt1:.1f} s"}


def _events_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_extras(dev, stream, peak, reps=5, envelope_series=1_000_000):
    """Uneven batch (4096 series, f32 and f64) and envelope batch (1M series
    of 1024, r=51): one persistent launch per kernel group (graph replay)
    against one mmf_filter1d launch per series, both event-timed."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    import synth
    out = {}
    lens, ws, dists, seeds = synth.uneven_batch(4096, seed=31)
    total = int(lens.sum())
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    for tname, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        src = [synth.torch_by_name(d, total, 31 + i, dev, tdt) for i, d in enumerate(synth.DISTS)]
        # each series takes its distribution's values at its own offset
        x = src[0]
        for i in range(lens.size):
            if dists[i]:
                a, b = int(starts[i]), int(starts[i] + lens[i])
                x[a:b] = src[dists[i]][a:b]
        del src
        plan = mmf.BatchPlan(lens, ws, tdt)
        om = torch.empty(plan.out_len, dtype=tdt, device=dev)
        on = torch.empty(plan.out_len, dtype=tdt, device=dev)
        plan.autotune(x, om, on, stream)
        for _ in range(2):
            plan(x, om, on, stream)
        bms = _events_ms(lambda: plan(x, om, on, stream), reps, stream)
        plan.per_series(x, om, on, stream)
        pms = _events_ms(lambda: plan.per_series(x, om, on, stream), 2, stream)
        sz = 4 if tdt == torch.float32 else 8
        n_out = int(np.maximum(lens - ws + 1, 0).sum())  # padding between series excluded
        byts = (total + 2 * n_out) * sz
        out[f"uneven_{tname}"] = {
            "series": 4096, "elements": total, "batched_ms": bms, "per_series_ms": pms,
            "batched_over_per_series": pms / bms, "batched_Gelem_s": total / bms / 1e6,
            "batched_GBps": byts / bms / 1e6, "frac": byts / bms / 1e6 / peak,
            "tuned": plan.knobs(), "items_per_group": plan.items_per_group}
        plan.close()
        del x, om, on
    torch.cuda.empty_cache()
    out.update(envelope_extras(dev, stream, peak, reps=reps, envelope_series=envelope_series))
    return out


def envelope_extras(dev, stream, peak, reps=5, envelope_series=1_000_000):
    """Envelope batch (z-normalised random walks of 1024, r = 51) batched and
    per series, and the LB_Keogh bound of one query against the same series."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    out = {}
    ns, L, r = envelope_series, 1024, 51
    g = torch.Generator(device=dev)
    g.manual_seed(33)
    z = torch.cumsum(torch.randn(ns, L, generator=g, device=dev, dtype=torch.float64), 1)
    z = ((z - z.mean(1, keepdim=True)) / z.std(1, unbiased=False, keepdim=True)).float().reshape(-1) + 0.0
    plan = mmf.BatchPlan(np.full(ns, L), np.full(ns, r), torch.float32, "envelope")
    om = torch.empty(plan.out_len, dtype=torch.float32, device=dev)
    on = torch.empty(plan.out_len, dtype=torch.float32, device=dev)
    plan.autotune(z, om, on, stream)
    for _ in range(2):
        plan(z, om, on, stream)
    bms = _events_ms(lambda: plan(z, om, on, stream), reps, stream)
    pms = _events_ms(lambda: plan.per_series(z, om, on, stream), 1, stream)
    byts = 3 * ns * L * 4
    out["envelope_f32"] = {
        "series": ns, "length": L, "radius": r, "batched_ms": bms, "per_series_ms": pms,
        "batched_over_per_series": pms / bms, "batched_Gelem_s": ns * L / bms / 1e6,
        "batched_GBps": byts / bms / 1e6, "frac": byts / bms / 1e6 / peak, "tuned": plan.knobs()}
    # The envelope lower bound of the time-warping distance against one query
    # (same series and radius): the envelope feeds a per-series sum in the
    # kernel and is never stored.  Bytes: the series once, the query, one
    # double per series.
    qz = torch.cumsum(torch.randn(L, generator=g, device=dev, dtype=torch.float64), 0)
    qz = ((qz - qz.mean()) / qz.std(unbiased=False)).float()
    lb = torch.empty(ns, dtype=torch.float64, device=dev)
    for _ in range(2):
        plan.lb_keogh(z, qz, out=lb, stream=stream)
    lms = _events_ms(lambda: plan.lb_keogh(z, qz, out=lb, stream=stream), reps, stream)
    lbyts = ns * L * 4 + L * 4 + ns * 8
    out["lb_keogh_f32"] = {
        "series": ns, "length": L, "radius": r, "ms": lms, "Gelem_s": ns * L / lms / 1e6,
        "GBps": lbyts / lms / 1e6, "frac": lbyts / lms / 1e6 / peak,
        "envelope_batch_ms": bms, "envelope_over_lb": bms / lms}
    plan.close()
    return out


def wedge_extras(dev, stream, peak, n=1 << 30, windows=(3, 31, 101, 496), reps=3):
    """The chunked-wedge kernel (Algorithm 1 per thread chunk) beside the
    library's default kernel choice (register slide or block scan) on the same
    n = 2^30 f32 streams, each event-timed."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    import synth
    out = {}
    om = torch.empty(n, dtype=torch.float32, device=dev)
    on = torch.empty(n, dtype=torch.float32, device=dev)
    for d in DISTS:
        x = synth.torch_by_name(d, n, 91, dev)
        for w in windows:
            m = n - w + 1
            row = {}
            for k in ("wedge", "auto"):
                def f():
                    mmf.filter1d(x, w, out_max=om[:m], out_min=on[:m], kernel=k, stream=stream)
                f()
                ms = _events_ms(f, reps, stream)
                gbs = (n + 2 * m) * 4 / ms / 1e6
                row[k] = {"ms": ms, "Gelem_s": n / ms / 1e6, "GBps": gbs, "frac": gbs / peak}
            row["wedge_over_auto"] = row["auto"]["ms"] / row["wedge"]["ms"]
            if w == 3:
                # The two-comparison scheme of Section 3 with its comparisons
                # counted on the device.
                cnt = torch.zeros(1, dtype=torch.int64, device=dev)
                def h():
                    mmf.filter1d_w3(x, out_max=om[:m], out_min=on[:m], stream=stream)
                h()
                ms = _events_ms(h, reps, stream)
                gbs = (n + 2 * m) * 4 / ms / 1e6
                _, _, cnt = mmf.filter1d_w3(x, out_max=om[:m], out_min=on[:m], count=True, stream=stream)
                torch.cuda.synchronize()
                row["w3_two_comparisons"] = {"ms": ms, "Gelem_s": n / ms / 1e6, "GBps": gbs, "frac": gbs / peak,
                                             "comparisons_per_element": int(cnt.item()) / m}
            out[f"{d}_w{w}"] = row
        del x
    del om, on
    torch.cuda.empty_cache()
    return out


def arg_extras(dev, stream, peak, n=1 << 30, windows=(3, 31, 496, 1001, 65537), reps=3):
    """The arg-max / arg-min filter (values and int64 positions of both
    extremes) on the n = 2^30 f32 streams: block scans over (value, position)
    pairs, and the chunked wedge where its window limit allows.  Algorithmic
    bytes: 4 + 2 x (4 + 8) per element."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    import synth
    out = {}
    om = torch.empty(n, dtype=torch.float32, device=dev)
    on = torch.empty(n, dtype=torch.float32, device=dev)
    am = torch.empty(n, dtype=torch.int64, device=dev)
    an = torch.empty(n, dtype=torch.int64, device=dev)
    for d in DISTS:
        x = synth.torch_by_name(d, n, 91, dev)
        for w in windows:
            m = n - w + 1
            row = {}
            for k in ("blockscan", "wedge"):
                if k == "wedge" and w > 496:
                    continue
                def g():
                    mmf.argfilter1d(x, w, stream=stream, out=(am[:m], an[:m], om[:m], on[:m]), kernel=k)
                g()
                ms = _events_ms(g, reps, stream)
                gbs = (n * 4 + 2 * m * 12) / ms / 1e6
                row[k] = {"ms": ms, "Gelem_s": n / ms / 1e6, "GBps": gbs, "frac": gbs / peak}
            if "wedge" in row:
                row["blockscan_over_wedge_time"] = row["blockscan"]["ms"] / row["wedge"]["ms"]
            out[f"{d}_w{w}"] = row
        del x
    del om, on, am, an
    torch.cuda.empty_cache()
    return out


def blobs_torch(nimg, H, W, seed, dev, nblobs=200):
    """The 2D recipe (sum of Gaussian blobs + 10 % uniform noise) drawn on the
    device: each image is an outer-product sum, one GEMM."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    out = torch.empty((nimg, H, W), dtype=torch.float32, device=dev)
    ys = torch.arange(H, device=dev, dtype=torch.float32)
    xs = torch.arange(W, device=dev, dtype=torch.float32)
    for k in range(nimg):
        cy = torch.rand(nblobs, generator=g, device=dev) * H
        cx = torch.rand(nblobs, generator=g, device=dev) * W
        sig = 5 + torch.rand(nblobs, generator=g, device=dev) * 195
        amp = torch.rand(nblobs, generator=g, device=dev)
        gy = torch.exp(-0.5 * ((ys[None, :] - cy[:, None]) / sig[:, None]) ** 2) * amp[:, None]
        gx = torch.exp(-0.5 * ((xs[None, :] - cx[:, None]) / sig[:, None]) ** 2)
        img = gy.T @ gx
        rng = (img.max() - img.min()).clamp_min(1e-6)
        img += torch.rand((H, W), generator=g, device=dev) * 0.1 * rng
        out[k] = img
    return out


def filter2d_extras(dev, stream, peak, nimg=64, H=4096, W=4096, reps=3):
    """64 images of 4096 x 4096, uint8 and fp32, five windows; row pass then
    column pass (unfused) and, where the windows allow, the fused tile kernel
    and the register-streaming kernel; the fastest is the line's figure.
    Algorithmic bytes: the image once plus both outputs."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    f = blobs_torch(nimg, H, W, 41, dev)
    lo, hi = f.amin(dim=(1, 2), keepdim=True), f.amax(dim=(1, 2), keepdim=True)
    u8 = torch.round((f - lo) / (hi - lo) * 255).clamp(0, 255).to(torch.uint8)
    res = {}
    for name, x in (("u8", u8), ("f32", f)):
        sz = x.element_size()
        for wy, wx in ((3, 3), (15, 15), (63, 63), (255, 1), (1, 255)):
            Ho, Wo = H - wy + 1, W - wx + 1
            om = torch.empty((nimg, Ho, Wo), dtype=x.dtype, device=dev)
            on = torch.empty((nimg, Ho, Wo), dtype=x.dtype, device=dev)
            ws = torch.empty(max(16, mmf.filter2d_workspace(nimg, H, W, wy, wx, x.dtype, 0)),
                             dtype=torch.uint8, device=dev)
            byts = (nimg * H * W + 2 * nimg * Ho * Wo) * sz
            row = {}
            for tag, fuse in (("unfused", 0), ("fused", 1), ("packed", 2)):
                if fuse == 1 and (wy == 1 or wx == 1 or wx > 31 or wy > 31):
                    continue
                if fuse == 2 and (wy > 9 or wx > 9):
                    continue
                mmf.filter2d(x, wy, wx, fuse=fuse, out_max=om, out_min=on, workspace=ws, stream=stream)
                ms = _events_ms(lambda: mmf.filter2d(x, wy, wx, fuse=fuse, out_max=om, out_min=on, workspace=ws,
                                                     stream=stream), reps, stream)
                row[tag] = {"ms": ms, "Gpix_s": nimg * H * W / ms / 1e6,
                            "GBps": byts / ms / 1e6, "frac": byts / ms / 1e6 / peak}
            best = min(row.values(), key=lambda r: r["ms"])
            res[f"{name}_{wy}x{wx}"] = {**best, **({k: v for k, v in row.items()} if len(row) > 1 else {})}
            del om, on, ws
    del f, u8
    torch.cuda.empty_cache()
    return res


def serving_extras(dev, nstreams=10_000, seed=51, duration=0.5,
                   rates=(2_000, 10_000, 30_000, 60_000, 120_000, 240_000, 480_000, 960_000, 1_920_000)):
    """10,000 fp32 random-walk streams, windows log-uniform in [8, 4096],
    chunks log-uniform in [256, 65536] samples released by an aggregate
    Poisson process at each rate (chunks/s); chunk data and outputs live in
    pinned host memory.  The pusher hands every chunk due by now to one
    mmf_stream_push_batch call.  Reports push-to-completion p50/p99 per rate
    and the achieved rate, until the service saturates."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    import synth
    ws = synth.stream_windows(nstreams, seed)
    pool = 1 << 27
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    walk = torch.cumsum(torch.randn(pool, generator=g, device=dev, dtype=torch.float64), 0).float()
    hin = torch.empty(pool, dtype=torch.float32, pin_memory=True)
    hin.copy_(walk)
    del walk
    hout = torch.empty(2, 1 << 26, dtype=torch.float32, pin_memory=True)
    in_base, max_base, min_base = hin.data_ptr(), hout[0].data_ptr(), hout[1].data_ptr()
    osize = hout.shape[1]
    srv = mmf.Server(4 << 30, 1024, "float32")
    ids = np.array([srv.open(int(w)) for w in ws], dtype=np.uint64)
    counts = np.zeros(nstreams, dtype=np.int64)
    rows = []
    for k, rate in enumerate(rates):
        t_rel, sid, clen = synth.poisson_arrivals(nstreams, rate, duration, seed + 100 + k)
        sid = sid.astype(np.int64)
        clen = clen.astype(np.int64)
        offs = np.random.default_rng(seed + k).integers(0, pool - 65536, size=t_rel.size)
        # Samples of the stream pushed before each chunk (earlier rates included).
        order = np.argsort(sid, kind="stable")
        cs = np.cumsum(clen[order])
        first = np.searchsorted(sid[order], sid[order], side="left")
        before_sorted = cs - clen[order] - np.concatenate([[0], cs])[first]
        before = np.empty_like(before_sorted)
        before[order] = before_sorted
        before += counts[sid]
        wv = ws[sid].astype(np.int64)
        m = np.maximum(0, before + clen - wv + 1) - np.maximum(0, before - wv + 1)
        opos = np.concatenate([[0], np.cumsum(m)[:-1]]) % max(1, osize - 65536)
        cptr = (in_base + 4 * offs).astype(np.uint64)
        mptr = (max_base + 4 * opos).astype(np.uint64)
        nptr = (min_base + 4 * opos).astype(np.uint64)
        sids = ids[sid]
        tickets = []
        srv.stats(reset=True)
        t0 = time.perf_counter()
        i = 0
        while i < t_rel.size:
            j = int(np.searchsorted(t_rel, time.perf_counter() - t0, side="right"))
            if j > i:
                t, _ = srv.push_batch(sids[i:j], cptr[i:j], clen[i:j], mptr[i:j], nptr[i:j])
                tickets.append(t)
                i = j
        push_end = time.perf_counter()
        srv.wait_batch(np.concatenate(tickets))
        t1 = time.perf_counter()
        st = srv.stats(reset=True)
        np.add.at(counts, sid, clen)
        elems = int(clen.sum())
        rows.append({"offered_chunks_s": rate, "offered_Gelem_s": rate * float(clen.mean()) / 1e9,
                     "achieved_Gelem_s": elems / (t1 - t0) / 1e9, "chunks": int(t_rel.size),
                     "push_calls": len(tickets), "push_s": push_end - t0, "p50_ms": st["p50_ms"],
                     "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "batches": st["batches"],
                     "p99_queue_ms": st["p99_queue_ms"], "p99_service_ms": st["p99_service_ms"],
                     "max_hold_ms": st["max_hold_ms"]})
        if (t1 - t0) > 1.5 * duration:  # the service no longer keeps up
            break
    srv.close()
    sat = max(r["achieved_Gelem_s"] for r in rows)
    head = min(rows, key=lambda r: abs(r["achieved_Gelem_s"] - 0.5 * sat))
    return {"streams": nstreams, "rows": rows, "saturation_Gelem_s": sat,
            "headline": {"load_Gelem_s": head["achieved_Gelem_s"], "p50_ms": head["p50_ms"],
                         "p99_ms": head["p99_ms"], "note": "load nearest to half of saturation"}}


def run_only(args):
    """One extra measurement on its own (the commands of the profiles/ summaries)."""
    import torch
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    from paper_cs_0610046_gb300 import build
    build.build()
    stream = torch.cuda.current_stream()
    peak = _peaks()[0]
    if args.only == "wedge":
        r = wedge_extras(dev, stream, peak, n=(1 << 26) if args.small else (1 << 30))
    elif args.only == "arg":
        r = arg_extras(dev, stream, peak, n=(1 << 26) if args.small else (1 << 30))
    elif args.only == "batched":
        r = batched_extras(dev, stream, peak, envelope_series=100_000 if args.small else 1_000_000)
    elif args.only == "envelope":
        r = envelope_extras(dev, stream, peak, envelope_series=100_000 if args.small else 1_000_000)
    elif args.only == "filter2d":
        r = filter2d_extras(dev, stream, peak, nimg=4 if args.small else 64)
    else:
        r = serving_extras(dev, duration=0.2 if args.small else 0.5)
    print(json.dumps({args.only: r}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--ref-sample", type=int, default=1 << 24)
    ap.add_argument("--cpu-sample", type=int, default=1 << 26)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched/2D/serving measurements")
    ap.add_argument("--only", choices=["wedge", "arg", "batched", "envelope", "filter2d", "serving"],
                    help="run one extra measurement alone and print its JSON (profiling)")
    ap.add_argument("--small", action="store_true",
                    help="with --only: a smaller instance of that workload (profiling captures)")
    args = ap.parse_args()

    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)

    import torch
    import torch.distributed as dist

    import paper_cs_0610046_gb300 as mmf
    from paper_cs_0610046_gb300 import build
    import synth

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    mmf.load()
    stream = torch.cuda.current_stream()

    n = args.n
    xs = {d: synth.torch_by_name(d, n, SEEDS[d] + 1000 * rank, dev) for d in DISTS}
    omax = torch.empty(n, dtype=torch.float32, device=dev)
    omin = torch.empty(n, dtype=torch.float32, device=dev)

    def step(events=None):
        for d in DISTS:
            for w in WINDOWS:
                m = n - w + 1
                if events is not None:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                mmf.filter1d(xs[d], w, out_max=omax[:m], out_min=omin[:m], stream=stream)
                if events is not None:
                    e1.record(stream)
                    events.append((w, e0, e1))

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    sampler = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    time.sleep(0.3)
    launch_events = []
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(launch_events)
    t_end.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    per_step_elems = len(DISTS) * len(WINDOWS) * n
    elapsed_ms, total_elems, value = job_time(t_start.elapsed_time(t_end), per_step_elems * args.steps, ws, dev)

    # Roofline of the dominant kernel.  Each window maps to one kernel
    # instantiation (mode): 3 register slide, 1 sub-warp blocks, 2 warp blocks.
    # Algorithmic bytes per launch: n*4 read + 2*(n-w+1)*4 written.
    peak, peak_kind = _peaks()
    def kmode(w):  # the kernel choice of the library for f32 (16 elements per thread)
        s = w - 1
        return 3 if s <= 16 else (2 if s >= 512 else (1 if s >= 16 else 0))
    per_w = {}
    per_k = {}
    for w, e0, e1 in launch_events:
        ms = e0.elapsed_time(e1)
        b = 4.0 * n + 8.0 * (n - w + 1)
        d = per_w.setdefault(w, {"ms": [], "bytes": b})
        d["ms"].append(ms)
        k = per_k.setdefault(kmode(w), {"ms": 0.0, "bytes": 0.0, "launches": 0, "windows": set()})
        k["ms"] += ms
        k["bytes"] += b
        k["launches"] += 1
        k["windows"].add(w)
    dom = max(per_k, key=lambda m: per_k[m]["ms"])
    kd = per_k[dom]
    kname = f"mmf::blockscan_kernel<float, {dom}, false, false>"
    achieved = kd["bytes"] / (kd["ms"] * 1e-3) / 1e9
    tr = _traffic().get(kname)
    traffic = None
    if tr:
        per_elem = dict(zip(tr["windows"], tr["dram_bytes_per_elem"]))
        if all(w in per_elem for w in kd["windows"]):
            traffic = sum(per_elem[w] for w in kd["windows"]) / len(kd["windows"]) * n
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "kernel": kname,
                "kernel_windows": sorted(kd["windows"]),
                "traffic": traffic,
                "algorithmic_bytes_per_launch": kd["bytes"] / kd["launches"],
                "frac_of_8TBps": achieved / 8000.0}
    all_bytes = sum(v["bytes"] for v in per_k.values())
    all_ms = sum(v["ms"] for v in per_k.values())
    roofline["all_kernels_achieved"] = all_bytes / (all_ms * 1e-3) / 1e9
    breakdown = {str(w): {"ms": statistics.median(v["ms"]),
                          "GBps": v["bytes"] / (statistics.median(v["ms"]) * 1e-3) / 1e9,
                          "Gelem_s": n / (statistics.median(v["ms"]) * 1e-3) / 1e9,
                          "frac": v["bytes"] / (statistics.median(v["ms"]) * 1e-3) / 1e9 / peak,
                          "kernel_mode": kmode(w)}
                 for w, v in per_w.items()}

    # End to end through the C ABI with HOST buffers (mmf_filter1d_host):
    # each call uploads its stream from pinned host memory, filters it and
    # downloads both outputs, in overlapped chunks.  Every rank runs it on its
    # own streams at the same time (GPUs may share a host link); the job's
    # figure is all ranks' elements over the slowest rank's time, as above.
    e2e = None
    if not args.no_e2e:
        hx = {d: torch.empty(n, dtype=torch.float32, pin_memory=True) for d in DISTS}
        for d in DISTS:
            hx[d].copy_(xs[d])
        hmax = torch.empty(n, dtype=torch.float32, pin_memory=True)
        hmin = torch.empty(n, dtype=torch.float32, pin_memory=True)

        def e2e_step():
            for d in DISTS:
                for w in WINDOWS:
                    m = n - w + 1
                    mmf.filter1d_host(hx[d], w, out_max=hmax[:m], out_min=hmin[:m], stream=stream)

        e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        _, _, e2e_value = job_time(s0.elapsed_time(s1), per_step_elems * args.e2e_steps, ws, dev)
        e2e = {"value": e2e_value, "unit": "Gelem/s",
               "h2d_bytes_per_step": len(DISTS) * len(WINDOWS) * n * 4 * ws,
               "d2h_bytes_per_step": sum(2 * 4 * (n - w + 1) for w in WINDOWS) * len(DISTS) * ws,
               "steps": args.e2e_steps, "path": "mmf_filter1d_host (chunks of 2^26, 3 streams)"}
        del hx, hmax, hmin

    extras = {}
    if not args.no_extras and rank == 0:
        del xs
        torch.cuda.empty_cache()
        extras["wedge"] = wedge_extras(dev, stream, peak)
        extras["arg"] = arg_extras(dev, stream, peak)
        extras["batched"] = batched_extras(dev, stream, peak)
        extras["filter2d"] = filter2d_extras(dev, stream, peak)
        extras["serving"] = serving_extras(dev)

    status = mmf.device_status(reset=True)
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        cpu = cpu_baseline(args.cpu_sample)

    # The workload's own targets, carried in the line: the whole step's share
    # of HBM bandwidth on the long stream, batched over per-series launches on
    # the uneven and envelope batches, and serving p99 near half saturation.
    step_bytes = sum(4.0 * n + 8.0 * (n - w + 1) for w in WINDOWS) * len(DISTS) * ws
    step_gbps = step_bytes / (elapsed_ms / args.steps * 1e-3) / 1e9
    targets = {"long_stream_step": {"GBps": step_gbps, "frac": step_gbps / peak, "frac_of_8TBps": step_gbps / 8000.0,
                                    "target_frac_of_8TBps": 0.70}}
    b = extras.get("batched") or {}
    if b:
        targets["batched_over_per_series"] = {k: b[k]["batched_over_per_series"]
                                              for k in ("uneven_f32", "uneven_f64", "envelope_f32") if k in b}
        targets["batched_over_per_series"]["target"] = 3.0
    sv = extras.get("serving") or {}
    if sv:
        targets["serving"] = {"p99_ms": sv["headline"]["p99_ms"], "p50_ms": sv["headline"]["p50_ms"],
                              "load_Gelem_s": sv["headline"]["load_Gelem_s"],
                              "saturation_Gelem_s": sv["saturation_Gelem_s"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "windows": list(WINDOWS), "dists": list(DISTS),
                       "l2": "inputs of 4 GiB per stream exceed L2 (no flush needed)",
                       "parallelism": f"{ws} independent streams per distribution (one per GPU)"},
            "roofline": roofline, "per_window": breakdown, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": len(launch_events), "clocks": clocks, "device_status": status,
            **extras,
            # last, so that a record which keeps only the end of the line keeps it
            "targets": targets,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
