"""Rounding of the f32 envelope lower bound, modelled on the CPU.

The GPU forms the LB_Keogh sum for f32 series in f32: each excursion
d = q - U (or L - q) is one f32 subtraction, d*d is added to a per-lane
partial sum by a fused multiply-add, the 32 lanes of a warp are summed by a
butterfly of five f32 additions, and warp sums are added in double.  Two
orders exist:

  * block-scan kernel (series longer than 1024): a lane sums the 16 positions
    it owns (one side per position: an excursion is above U or below L,
    never both), warps cover 512 consecutive positions;
  * short-series kernel (up to 1024): lane l sums positions 32k + l over k,
    the max side over all its positions first, then the min side; one warp
    per series;
  * short-series kernel, windows longer than 32 elements: lane l sums
    positions 32k + l over k, one term per position (the side outside the
    envelope), ascending.

Summing m non-negative terms recursively in f32 has a relative error of at
most (m-1)u (u = 2^-24), a zero term adds nothing, the butterfly adds 5u and
each term carries at most 2u from its rounded difference: 22u (about 1.3e-6)
for the block-scan order and 38u (about 2.3e-6) for both short orders before
the square root, half of that after it.  This model applies those roundings
in those orders (numpy float32, the multiply-add done exactly in double and
rounded once) and checks the result against the oracle's double sum within
the bounds, on z-normalised walks and on queries far outside every envelope
(every term non-zero and of one size, the worst case for accumulation).  The
GPU parity test's tolerance of 4e-6 on the bound lies above both."""
import numpy as np
import pytest

import oracle
import synth

U = 2.0 ** -24


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _butterfly(part):
    """part: (warps, 32) f32; the xor-shuffle sum every lane ends with."""
    p = part.copy()
    for k in (16, 8, 4, 2, 1):
        p = (p + p[:, np.arange(32) ^ k]).astype(np.float32)
    return p[:, 0]


def _excursions(c, q, r):
    up, lo = oracle.envelope(c, r)
    dmax = np.where(q > up, (q - up).astype(np.float32), np.float32(0))
    dmin = np.where(q < lo, (lo - q).astype(np.float32), np.float32(0))
    return dmax, dmin


def _blockscan_order(dmax, dmin):
    d = np.where(dmax > 0, dmax, dmin).astype(np.float32)  # one side per position
    n = d.size
    nw = -(-n // 512)
    dd = np.zeros(nw * 512, np.float32)
    dd[:n] = d
    lanes = dd.reshape(nw, 32, 16)
    part = np.zeros((nw, 32), np.float32)
    for i in range(16):
        part = _fma32(lanes[:, :, i], lanes[:, :, i], part)
    return float(np.sum(_butterfly(part).astype(np.float64)))


def _short_order(dmax, dmin):
    n = dmax.size
    assert n <= 1024
    part = np.zeros((1, 32), np.float32)
    for side in (dmax, dmin):
        ds = np.zeros(1024, np.float32)
        ds[:n] = side
        rows = ds.reshape(32, 32)  # row k holds positions 32k + lane
        for k in range(32):
            part = _fma32(rows[k][None, :], rows[k][None, :], part)
    return float(_butterfly(part)[0])


def _short_lanes_order(dmax, dmin):
    n = dmax.size
    assert n <= 1024
    d = np.zeros(1024, np.float32)
    d[:n] = np.where(dmax > 0, dmax, dmin)
    rows = d.reshape(32, 32)
    part = np.zeros((1, 32), np.float32)
    for k in range(32):
        part = _fma32(rows[k][None, :], rows[k][None, :], part)
    return float(_butterfly(part)[0])


@pytest.mark.parametrize("far", [False, True])
def test_f32_bound_rounding_within_the_derived_bounds(far):
    rng = np.random.default_rng(9)
    worst = {"blockscan": 0.0, "short": 0.0, "short_lanes": 0.0}
    for t in range(60):
        n = int(rng.integers(2, 1025)) if t % 2 else int(rng.integers(1025, 6000))
        r = int(rng.integers(0, 80))
        c, q = synth.znorm_walks(2, n, 100 + t, np.float32)
        if far:
            q = (q + np.float32(50.0 + rng.random() * 1000.0)).astype(np.float32)
        exact = oracle.lb_keogh(c, q, r) ** 2
        if exact == 0.0:
            continue
        dmax, dmin = _excursions(c, q, r)
        got = {"blockscan": _blockscan_order(dmax, dmin)}
        if n <= 1024:
            got["short"] = _short_order(dmax, dmin)
            got["short_lanes"] = _short_lanes_order(dmax, dmin)
        for kind, v in got.items():
            rel = abs(v - exact) / exact
            bound = (22 if kind == "blockscan" else 38) * U * 1.0001
            assert rel <= bound, (kind, n, r, rel, bound)
            rel_sqrt = abs(np.sqrt(v) - np.sqrt(exact)) / np.sqrt(exact)
            assert rel_sqrt <= 2e-6 and rel_sqrt <= 4e-6
            worst[kind] = max(worst[kind], rel)
    assert worst["blockscan"] > 0 and worst["short"] > 0 and worst["short_lanes"] > 0  # the model really rounds
