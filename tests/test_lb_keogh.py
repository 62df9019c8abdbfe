"""GPU parity of the envelope lower bound of the time-warping distance
(mmf_lb_keogh_batched, the envelope kernel with a fused reduction) against
the oracle, series by series.

Tolerances: i16/u8 are summed exactly in integers, so their bounds equal the
oracle's double result bit for bit.  f32 forms each squared excursion and a
per-warp sum in f32 (non-negative terms: at most 22u, about 1.3e-6, relative
before the square root in the block-scan kernel and 38u, about 2.3e-6, in the
short-series kernel, u = 2^-24; half of that after it), so the test allows
4e-6 relative on the bound.
f64 sums per warp in double and across tiles atomically (order-dependent
rounding): 1e-12 relative."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NP2T = {np.float32: torch.float32, np.float64: torch.float64, np.int16: torch.int16, np.uint8: torch.uint8}
RTOL = {np.float32: 4e-6, np.float64: 1e-12, np.int16: 0.0, np.uint8: 0.0}


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _series(dtype, nser, n, seed):
    if dtype in (np.float32, np.float64):
        return synth.znorm_walks(nser, n, seed, dtype)
    return np.stack([synth.random_walk(n, seed=seed + s, dtype=dtype) for s in range(nser)])


def _check(mmf, dtype, nser, n, r, seed=1, query=None):
    c = _series(dtype, nser, n, seed)
    q = _series(dtype, 1, n, seed + 999)[0] if query is None else query
    plan = mmf.BatchPlan(np.full(nser, n), np.full(nser, r), NP2T[dtype], "envelope")
    x = torch.from_numpy(np.ascontiguousarray(c.reshape(-1))).cuda()
    qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    lb = plan.lb_keogh(x, qd).cpu().numpy()
    plan.close()
    for s in range(nser):
        e = oracle.lb_keogh(c[s], q, r)
        tol = RTOL[dtype] * e
        assert abs(lb[s] - e) <= tol, f"series {s}: {lb[s]} vs {e} (n {n}, r {r})"
    return lb


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
@pytest.mark.parametrize("n,r", [(1024, 51), (1, 0), (7, 3), (100, 0), (2047, 5), (5000, 200), (9001, 17),
                                 (500, 40), (1000, 15), (1000, 16), (300, 299), (700, 5000)])
def test_lb_keogh_matches_oracle(mmf, dtype, n, r):
    """Lengths below, at and across tiles (ragged ends), radii that take the
    register slide (2r+1 <= 17), the scans inside a thread, across lanes and
    per warp; short series with windows within one lane's elements and
    beyond (2r+1 = 31 and 33), radii reaching past the series."""
    nser = 40 if n <= 2047 else 6
    _check(mmf, dtype, nser, n, r)


def test_lb_keogh_zero_inside_and_known_value(mmf):
    """A query equal to a series gives 0 for it; a query shifted far above
    every envelope gives the Euclidean distance to the upper envelope."""
    n, r = 3000, 25
    c = _series(np.float64, 5, n, 3)
    plan = mmf.BatchPlan(np.full(5, n), np.full(5, r), torch.float64, "envelope")
    x = torch.from_numpy(c.reshape(-1).copy()).cuda()
    lb = plan.lb_keogh(x, torch.from_numpy(c[2].copy()).cuda()).cpu().numpy()
    assert lb[2] == 0.0 and (lb[[0, 1, 3, 4]] > 0).all()
    q = np.full(n, 100.0)
    lb = plan.lb_keogh(x, torch.from_numpy(q).cuda()).cpu().numpy()
    for s in range(5):
        up, _ = oracle.envelope(c[s], r)
        e = np.sqrt(((q - up) ** 2).sum())
        assert abs(lb[s] - e) <= 1e-12 * e
    plan.close()


def test_lb_keogh_rejects(mmf):
    x = torch.zeros(300, device="cuda")
    plan = mmf.BatchPlan([100, 200], [5, 5], torch.float32, "envelope")
    with pytest.raises(mmf.MMFError):
        plan.lb_keogh(x, torch.zeros(100, device="cuda"))  # lengths differ
    plan.close()
    plan = mmf.BatchPlan([100, 100], [5, 5], torch.float32, "valid")
    with pytest.raises(mmf.MMFError):
        plan.lb_keogh(x, torch.zeros(100, device="cuda"))  # not an envelope plan
    plan.close()
    assert mmf.device_status() == 0
