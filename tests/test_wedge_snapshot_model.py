"""CPU model of the wedge form of a stream snapshot, checked against the
definition on every tie pattern.

A stream's state for later outputs is its last h = min(count, w-1) samples
(every later window holds only those and later samples, Section 1).  The wedge
form keeps only the samples of the monotonic wedge of Section 4: U, the
samples strictly above every later one, and L, those strictly below every
later one (the deques of Algorithm 1 after the last step).  Restoring it
rebuilds a halo: wedge samples keep their values and every other position
takes the value of the nearest later sample of U.  The claim tested here: for
every continuation of the stream, every window that ends after the snapshot
has the same maximum and minimum with the rebuilt halo as with the true one.
The library's snapshot and restore follow these rules (its GPU tests check
continuation through the service); this model checks the rules themselves
over every array of up to 7 samples over 3 values and random continuations."""
import itertools

import numpy as np

import oracle


def wedge_sides(h):
    """Positions of U and L, oldest first (a sample leaves a side when a later
    one is at least as large for U, at least as small for L)."""
    u, l = [], []
    for k, x in enumerate(h):
        while u and not h[u[-1]] > x:
            u.pop()
        u.append(k)
        while l and not h[l[-1]] < x:
            l.pop()
        l.append(k)
    return u, l


def rebuild(h, u, l):
    out = np.zeros_like(h)
    in_u = np.zeros(len(h), bool)
    known = np.zeros(len(h), bool)
    for k in u:
        out[k] = h[k]
        in_u[k] = known[k] = True
    for k in l:
        out[k] = h[k]
        known[k] = True
    last = out[-1]
    for k in range(len(h) - 1, -1, -1):
        if in_u[k]:
            last = out[k]
        elif not known[k]:
            out[k] = last
    return out


def _later_windows_equal(h, r, w, rng):
    """Windows of w that end at or after the first sample following h."""
    for _ in range(3):
        fut = rng.integers(0, 3, size=int(rng.integers(1, w + 3))).astype(np.float32)
        a = np.concatenate([h, fut])
        b = np.concatenate([r, fut])
        ma, na = oracle.bf1d(a, w)
        mb, nb = oracle.bf1d(b, w)
        first = max(0, len(h) - w + 1)  # first window that holds a later sample
        assert np.array_equal(ma[first:], mb[first:]) and np.array_equal(na[first:], nb[first:]), (h, fut, w)


def test_wedge_is_the_algorithm_1_deques():
    """The sides equal Algorithm 1's deques after the last step, whose
    fronts are the window extremes (the oracle's wedge gives the last
    window's max and min as U's and L's fronts)."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        h = rng.integers(0, 4, size=n).astype(np.float32)
        u, l = wedge_sides(h)
        assert h[u[0]] == h.max() and h[l[0]] == h.min()
        assert all(h[u[i]] > h[u[i + 1]] for i in range(len(u) - 1))
        assert all(h[l[i]] < h[l[i + 1]] for i in range(len(l) - 1))
        assert u[-1] == l[-1] == n - 1  # the newest sample is in both
        mx, mn, _ = oracle.wedge(h, n)
        assert mx[0] == h[u[0]] and mn[0] == h[l[0]]


def test_rebuilt_halo_gives_the_same_later_outputs_exhaustive():
    rng = np.random.default_rng(11)
    for n in range(1, 8):
        for vals in itertools.product(range(3), repeat=n):
            h = np.asarray(vals, np.float32)
            u, l = wedge_sides(h)
            r = rebuild(h, u, l)
            for w in range(n + 1, n + 3):  # the halo is the last w-1 samples: w-1 >= n
                _later_windows_equal(h, r, w, rng)


def test_rebuilt_halo_random_long():
    rng = np.random.default_rng(12)
    for _ in range(40):
        n = int(rng.integers(10, 300))
        h = np.cumsum(rng.integers(-1, 2, size=n)).astype(np.float32)  # walks with many ties
        u, l = wedge_sides(h)
        r = rebuild(h, u, l)
        _later_windows_equal(h, r, n + 1, rng)
        # the wedge is far smaller than the halo on such data, never larger
        assert len(u) + len(l) <= n + 1
