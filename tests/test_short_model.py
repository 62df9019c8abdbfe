"""CPU model of the short-series kernel's decomposition, checked against the
oracle (valid windows and centred, end-clipped envelopes).

Short series are filtered with blocks of exactly w elements starting at
position 0 (van Herk/Gil-Werman's own blocks, Section 2 and Table 1), with
the identity (-inf for max, +inf for min) at every position past the
series' end.  A window [lo, lo+w-1] then covers the suffix of lo's block and
the prefix of the next block (or is one whole block), so its extreme is
op(S[lo], P[lo+w-1]).  Clipped windows follow the kernel's rules: a window
clipped at the start (lo <= 0) lies in block 0, which begins at position 0,
so it is P[hi]; a window clipped at the end (hi = n-1) is S[lo] when lo and
hi share a block (the identities after the series do not change it), else
op(S[lo], P[hi])."""
import numpy as np

import oracle
import synth


def _scans(x, w, op):
    P = x.copy()
    S = x.copy()
    for i in range(1, len(x)):
        if i % w:
            P[i] = op(P[i - 1], x[i])
    for i in range(len(x) - 2, -1, -1):
        if (i + 1) % w:
            S[i] = op(S[i + 1], x[i])
    return P, S


def _model(a, w, d, n_out, cap):
    """cap: positions held (the kernel's 32 lanes x E elements)."""
    n = len(a)
    assert n <= cap
    out = []
    for x0, op, ident in ((a.astype(np.float64), max, -np.inf), (a.astype(np.float64), min, np.inf)):
        x = np.full(cap, ident)
        x[:n] = x0
        P, S = _scans(x, w, op)
        res = np.empty(n_out)
        for o in range(n_out):
            lo = o + d
            hi = min(lo + w - 1, n - 1)
            if lo <= 0:
                assert hi < w  # block 0
                res[o] = P[hi]
            elif lo // w == hi // w:
                res[o] = S[lo]
            else:
                assert hi // w == lo // w + 1  # exactly two blocks
                res[o] = op(S[lo], P[hi])
        out.append(res)
    return out


def test_valid_windows():
    rng = np.random.default_rng(1)
    for _ in range(300):
        n = int(rng.integers(1, 257))
        w = int(rng.integers(1, n + 1))
        a = synth.random_walk(n, seed=int(rng.integers(1 << 30)), dtype=np.float32)
        if rng.random() < 0.3:
            a = rng.integers(0, 3, size=n).astype(np.float32)  # ties
        gm, gn = _model(a, w, 0, n - w + 1, 256)
        em, en = oracle.bf1d(a, w)
        assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (n, w)


def test_envelopes():
    rng = np.random.default_rng(2)
    for _ in range(300):
        n = int(rng.integers(1, 257))
        r = int(rng.integers(0, n + 3))
        a = synth.random_walk(n, seed=int(rng.integers(1 << 30)), dtype=np.float32)
        rr = min(r, n - 1)  # a radius of n-1 already covers the series from every centre
        gm, gn = _model(a, 2 * rr + 1, -rr, n, 256)
        em, en = oracle.envelope(a, r)
        assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (n, r)
