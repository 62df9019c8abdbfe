"""CPU model of the host-memory pipeline's chunking (mmf_filter1d_host),
checked against the oracle.

The outputs are cut into chunks [o0, o1) of `chunk` outputs.  Output o's
window starts at o + d (d = 0 for valid windows, -r for centred ones) and
has w elements, so a chunk needs the inputs [max(0, o0 + d), min(n, o1 - 1 +
d + w)); they are uploaded as a series of their own whose output 0 starts its
window at (o0 + d) - lo, with the identities of the filter (-inf, +inf)
wherever a window reaches outside that series, which happens only at the
true ends of the array.  Each output depends on its own window alone
(Section 1), so the chunks' outputs put side by side are the whole filter."""
import numpy as np

import oracle
import synth


def _series_filter(x, w, d, n_out):
    """The filter of one series with identities outside it."""
    out_m = np.empty(n_out)
    out_n = np.empty(n_out)
    for o in range(n_out):
        s = o + d
        win = x[max(0, s):max(0, min(len(x), s + w))]
        out_m[o] = win.max() if win.size else -np.inf
        out_n[o] = win.min() if win.size else np.inf
    return out_m, out_n


def _pipeline(a, w_or_r, mode, chunk):
    n = len(a)
    if mode == "valid":
        w, d, n_out = w_or_r, 0, max(0, n - w_or_r + 1)
    else:
        r = min(w_or_r, max(n - 1, 0))
        w, d, n_out = 2 * r + 1, -r, n
    om, on = np.empty(n_out), np.empty(n_out)
    for o0 in range(0, n_out, chunk):
        o1 = min(n_out, o0 + chunk)
        lo, hi = max(0, o0 + d), min(n, o1 - 1 + d + w)
        m, mn = _series_filter(a[lo:hi].astype(np.float64), w, (o0 + d) - lo, o1 - o0)
        om[o0:o1], on[o0:o1] = m, mn
    return om, on


def test_chunks_put_together_are_the_whole_filter():
    rng = np.random.default_rng(13)
    for _ in range(120):
        n = int(rng.integers(1, 300))
        a = synth.random_walk(n, seed=n, dtype=np.float32)
        chunk = int(rng.integers(1, 40))
        w = int(rng.integers(1, n + 1))
        gm, gn = _pipeline(a, w, "valid", chunk)
        em, en = oracle.bf1d(a, w)
        assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (n, w)
        r = int(rng.integers(0, n + 2))
        gm, gn = _pipeline(a, r, "envelope", chunk)
        em, en = oracle.envelope(a, r)
        assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (n, r)
