"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the filter itself: it only draws numbers.
Every generator is deterministic in its seed.  Values contain no NaN and no
negative zero (``x + 0.0`` maps -0.0 to +0.0), so a max or a min is a unique
bit pattern and GPU results can be compared bitwise with the oracle.

Recipes (the workloads of the benchmarks; the paper used Unix ``rand`` noise
and a sine wave of period 10 000 on one million doubles, Section 5):

* ``uniform``             i.i.d. uniform[0, 1)
* ``random_walk``         cumulative sum of N(0, 1) increments, summed in
                          float64, then cast
* ``piecewise_monotone``  alternating rising/falling runs (first rising), run
                          lengths Geometric(p=1e-3) on {1, 2, ...} (mean 1000),
                          steps |N(0, 1)|, x0 = 0
* ``sine``                sin(2 pi i / 10000), the paper's piecewise-monotone
                          input
* ``uneven_batch``        4096 series, lengths round(10^U(3, 6)), windows from
                          {3, 15, 101, 1001, 10001} clipped to the length,
                          distribution per series uniform over the three above
* ``znorm_walks``         random walks z-normalised per series (envelope input)
* ``blobs2d``             sums of Gaussian blobs plus 10% uniform noise
                          (2D input); uint8 by min/max quantisation

Integer dtypes are produced from the float recipe by a min/max rescale to the
type's range and rounding.
"""
from __future__ import annotations

import numpy as np

WINDOWS_BATCH = (3, 15, 101, 1001, 10001)
DISTS = ("uniform", "random_walk", "piecewise_monotone")


def _canon(x: np.ndarray) -> np.ndarray:
    if x.dtype.kind == "f":
        x += x.dtype.type(0.0)  # -0.0 -> +0.0
    return x


def _quantise(x64: np.ndarray, dtype) -> np.ndarray:
    dt = np.dtype(dtype)
    if dt.kind == "f":
        return _canon(x64.astype(dt))
    info = np.iinfo(dt)
    lo, hi = float(x64.min()), float(x64.max())
    span = hi - lo if hi > lo else 1.0
    y = np.rint((x64 - lo) / span * (info.max - info.min) + info.min)
    return np.clip(y, info.min, info.max).astype(dt)


def uniform(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _quantise(rng.random(n), dtype)


def random_walk(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _quantise(np.cumsum(rng.standard_normal(n)), dtype)


def piecewise_monotone(n: int, seed: int, dtype=np.float32, mean_run: float = 1000.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    runs = []
    total = 0
    while total < n:
        r = rng.geometric(1.0 / mean_run, size=max(16, int(2 * (n - total) / mean_run) + 16))
        runs.append(r)
        total += int(r.sum())
    runs = np.concatenate(runs)
    sign = np.where(np.arange(runs.size) % 2 == 0, 1.0, -1.0)
    steps = np.repeat(sign, runs)[:n] * np.abs(rng.standard_normal(n))
    steps[0] = 0.0
    return _quantise(np.cumsum(steps), dtype)


def sine(n: int, dtype=np.float64, period: int = 10000) -> np.ndarray:
    return _quantise(np.sin(2.0 * np.pi * np.arange(n) / period), dtype)


def by_name(dist: str, n: int, seed: int, dtype=np.float32) -> np.ndarray:
    return {"uniform": uniform, "random_walk": random_walk,
            "piecewise_monotone": piecewise_monotone}[dist](n, seed, dtype)


def monotone(n: int, seed: int, dtype=np.float32, decreasing: bool = False) -> np.ndarray:
    """Non-decreasing (or non-increasing) input with repeated values."""
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.integers(0, 3, size=n).astype(np.float64))
    if decreasing:
        x = -x
    return _quantise(x, dtype)


def uneven_batch(nseries: int, seed: int, lo_exp: float = 3.0, hi_exp: float = 6.0,
                 windows=WINDOWS_BATCH):
    """Lengths log-uniform in [10^lo_exp, 10^hi_exp], windows drawn from
    ``windows`` and clipped to the length, one distribution per series."""
    rng = np.random.default_rng(seed)
    lens = np.rint(10.0 ** rng.uniform(lo_exp, hi_exp, size=nseries)).astype(np.int64)
    ws = rng.choice(np.asarray(windows, dtype=np.int64), size=nseries)
    ws = np.minimum(ws, lens)
    dists = rng.integers(0, len(DISTS), size=nseries)
    seeds = rng.integers(0, 2**31 - 1, size=nseries)
    return lens, ws, dists, seeds


def uneven_batch_data(lens, dists, seeds, dtype=np.float32) -> np.ndarray:
    parts = [by_name(DISTS[d], int(L), int(s), dtype) for L, d, s in zip(lens, dists, seeds)]
    return np.concatenate(parts) if parts else np.empty(0, dtype)


def znorm_walks(nseries: int, length: int, seed: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal((nseries, length)), axis=1)
    mu = x.mean(axis=1, keepdims=True)
    sd = x.std(axis=1, keepdims=True)
    sd[sd == 0] = 1.0
    return _canon(((x - mu) / sd).astype(dtype))


def blobs2d(nimg: int, H: int, W: int, seed: int, dtype=np.float32, nblobs: int = 200) -> np.ndarray:
    """Sum of ``nblobs`` Gaussian blobs (centre uniform, sigma U(5, 200) px,
    amplitude U(0, 1)) plus uniform noise U(0, 0.1 * range), per image."""
    rng = np.random.default_rng(seed)
    out = np.empty((nimg, H, W), dtype=np.dtype(dtype))
    ys = np.arange(H, dtype=np.float64)
    xs = np.arange(W, dtype=np.float64)
    for k in range(nimg):
        cy = rng.uniform(0, H, nblobs)
        cx = rng.uniform(0, W, nblobs)
        sig = rng.uniform(5.0, 200.0, nblobs)
        amp = rng.uniform(0.0, 1.0, nblobs)
        gy = np.exp(-0.5 * ((ys[None, :] - cy[:, None]) / sig[:, None]) ** 2) * amp[:, None]
        gx = np.exp(-0.5 * ((xs[None, :] - cx[:, None]) / sig[:, None]) ** 2)
        img = gy.T @ gx
        rngv = float(img.max() - img.min()) or 1.0
        img += rng.uniform(0.0, 0.1 * rngv, size=(H, W))
        out[k] = _quantise(img, dtype)
    return out


def poisson_arrivals(nstreams: int, rate_chunks_per_s: float, duration_s: float, seed: int,
                     chunk_lo: int = 256, chunk_hi: int = 65536):
    """Arrival times (s), stream ids and chunk lengths of an aggregate Poisson
    process; chunk lengths log-uniform in [chunk_lo, chunk_hi]."""
    rng = np.random.default_rng(seed)
    m = rng.poisson(rate_chunks_per_s * duration_s)
    t = np.sort(rng.uniform(0.0, duration_s, size=m))
    sid = rng.integers(0, nstreams, size=m)
    clen = np.rint(10.0 ** rng.uniform(np.log10(chunk_lo), np.log10(chunk_hi), size=m)).astype(np.int64)
    return t, sid, clen


def stream_windows(nstreams: int, seed: int, lo: int = 8, hi: int = 4096) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=nstreams)).astype(np.int64)


# ---- device-side generators for full-size workloads (torch, seeded) -------

def torch_by_name(dist: str, n: int, seed: int, device, dtype=None):
    """Same recipes drawn with a seeded torch generator on ``device`` (used
    where host generation of 2^30 values would dominate the run).  The
    values differ from the numpy recipe but follow the same distribution."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dtype = dtype or torch.float32
    if dist == "uniform":
        x = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    elif dist == "random_walk":
        x = torch.cumsum(torch.randn(n, generator=g, device=device, dtype=torch.float64), 0)
    elif dist == "piecewise_monotone":
        # run lengths ~ Geometric(1e-3): floor(log(U)/log(1-p)) + 1
        p = 1e-3
        nr = int(2 * n / 1000) + 64
        u = torch.rand(nr, generator=g, device=device, dtype=torch.float64).clamp_min(1e-300)
        runs = (torch.floor(torch.log(u) / np.log1p(-p)) + 1).to(torch.int64)
        while int(runs.sum()) < n:
            u = torch.rand(nr, generator=g, device=device, dtype=torch.float64).clamp_min(1e-300)
            runs = torch.cat([runs, (torch.floor(torch.log(u) / np.log1p(-p)) + 1).to(torch.int64)])
        sign = torch.where(torch.arange(runs.numel(), device=device) % 2 == 0, 1.0, -1.0).to(torch.float64)
        steps = torch.repeat_interleave(sign, runs)[:n] * torch.randn(n, generator=g, device=device,
                                                                      dtype=torch.float64).abs()
        steps[0] = 0.0
        x = torch.cumsum(steps, 0)
    else:
        raise ValueError(dist)
    if dtype.is_floating_point:
        return x.to(dtype) + 0.0
    info = torch.iinfo(dtype)
    lo, hi = x.min(), x.max()
    span = torch.where(hi > lo, hi - lo, torch.ones_like(hi))
    return torch.round((x - lo) / span * (info.max - info.min) + info.min).clamp(info.min, info.max).to(dtype)
