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
import itertools

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


# Windows longer than a lane (w - 1 >= E): the blocks are the lanes' own E
# elements instead (the general block decomposition of Section 2 with blocks
# shorter than the window), so the prefix and suffix scans never restart
# inside a lane.  With s = w - 1 = q*E + rr, the window starting at lo (lane
# j, element e) ends in lane K = j + q (or j + q + 1 when e + rr >= E): its
# extreme is op(S[lo], aggregates of lanes j+1 .. K-1, P[hi]).  The lane
# aggregates over the q-1 and q lanes after each lane come from a doubling
# over lanes (windows of 1, 2, 4, 8, 16 lanes, two overlapping ones per
# length); lanes past the last hold identities, and so does P at hi past the
# last lane (the kernel reads an identity column there).  Positions past the
# series' end repeat its last element (every window reaching past the end
# holds that element already).  Lane j forms the outputs whose windows start
# in its own block (o = lo - d); the outputs whose windows start before
# position 0 (envelopes) take the aggregate of the lanes before hi's lane
# and P[hi].


def _lane_windows(A, q, op, ident):
    """m1[j] = op(A[j+1 .. j+q-1]), m2[j] = op(A[j+1 .. j+q]), by the
    kernel's doubling (D[k][x] = op over lanes x .. x+2^k-1, identities past
    the last lane)."""
    L = len(A)
    D = [list(A)]
    for k in range(5):
        dl = 1 << k
        D.append([op(D[k][x], D[k][x + dl] if x + dl < L else ident) for x in range(L)])

    def win(length):
        out = []
        for j in range(L):
            if length <= 0:
                out.append(ident)
            elif length >= 32:
                out.append(D[5][j + 1] if j + 1 < L else ident)
            else:
                k = length.bit_length() - 1
                p = 1 << k
                u = D[k][j + 1] if j + 1 < L else ident
                off = 1 + length - p
                v = D[k][j + off] if j + off < L else ident
                out.append(op(u, v))
        return out

    return win(q - 1), win(q)


def _model_lanes(a, w, d, n_out, E, mistake=None):
    lanes = 32
    cap = lanes * E
    n = len(a)
    assert n <= cap and w - 1 >= E
    s = w - 1
    q, rr = divmod(s, E)
    x = np.full(cap, float(a[-1]))  # the last element repeated past the end
    x[:n] = a.astype(np.float64)
    if mistake == "identity_pad_one_side":
        x[n:] = -np.inf  # right for max only
    res_all = []
    for op, ident in ((max, -np.inf), (min, np.inf)):
        P = x.copy()
        S = x.copy()
        for j in range(lanes):
            b = j * E
            for e in range(1, E):
                P[b + e] = op(P[b + e - 1], x[b + e])
            for e in range(E - 2, -1, -1):
                S[b + e] = op(S[b + e + 1], x[b + e])
        A = [S[j * E] for j in range(lanes)]
        m1, m2 = _lane_windows(A, q, op, ident)
        if mistake == "m_swapped":
            m1, m2 = m2, m1

        def Pk(K, eh):  # identity column past the last lane
            return P[K * E + eh] if K < lanes else ident

        res = np.full(n_out, np.nan)
        for j in range(lanes):
            for e in range(E):
                lo = j * E + e
                o = lo - d
                if not 0 <= o < n_out:
                    continue
                far = e >= E - rr
                K = j + q + (1 if far else 0)
                eh = e + rr - (E if far else 0)
                assert lo + s == K * E + eh
                assert np.isnan(res[o]), "an output is formed twice"
                res[o] = op(op(S[lo], m2[j] if far else m1[j]), Pk(min(K, lanes), eh))
        if d < 0:
            incl = list(itertools.accumulate(A, op))
            for o in range(min(-d, n_out)):
                hi = o + d + s
                K = min(hi // E, lanes)
                xk = incl[K - 1] if K > 0 else ident
                assert np.isnan(res[o]), "an output is formed twice"
                res[o] = op(xk, Pk(K, hi % E))
        assert not np.isnan(res).any(), "an output is never formed"
        res_all.append(res)
    return res_all


def test_lane_blocks_valid_windows():
    rng = np.random.default_rng(3)
    for E in (4, 8, 16, 32):
        cap = 32 * E
        for _ in range(40 if E < 16 else 12):
            n = int(rng.integers(E + 1, cap + 1))
            w = int(rng.integers(E + 1, n + 1))
            a = synth.random_walk(n, seed=int(rng.integers(1 << 30)), dtype=np.float32)
            if rng.random() < 0.3:
                a = rng.integers(0, 3, size=n).astype(np.float32)
            gm, gn = _model_lanes(a, w, 0, n - w + 1, E)
            em, en = oracle.bf1d(a, w)
            assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (E, n, w)


def test_lane_blocks_envelopes():
    rng = np.random.default_rng(4)
    for E in (4, 8, 16, 32):
        cap = 32 * E
        for _ in range(40 if E < 16 else 12):
            n = int(rng.integers(1, cap + 1))
            rr = int(rng.integers(0, n))
            if 2 * rr < E:
                continue  # a window of at most a lane: the other decomposition
            a = synth.random_walk(n, seed=int(rng.integers(1 << 30)), dtype=np.float32)
            gm, gn = _model_lanes(a, 2 * rr + 1, -rr, n, E)
            em, en = oracle.envelope(a, rr)
            assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (E, n, rr)


def test_lane_blocks_edges_and_planted_mistakes():
    """Windows of exactly E+1 (q = 1, rr = 0), of q whole lanes, longer than
    the series (clipped envelopes, hi past the last lane), full series; a
    swapped choice of the between-lane aggregate fails, and so does padding
    past the end with the max side's identity for both sides."""
    E = 8
    cap = 32 * E
    a = synth.random_walk(cap, seed=9, dtype=np.float32)
    for w in (E + 1, 2 * E + 1, 3 * E, 31 * E + 1, cap):
        gm, gn = _model_lanes(a, w, 0, cap - w + 1, E)
        em, en = oracle.bf1d(a, w)
        assert np.array_equal(gm, em) and np.array_equal(gn, en), w
    for n, r in ((cap, cap - 1), (cap, 40), (100, 99), (E + 3, E)):
        gm, gn = _model_lanes(a[:n], 2 * r + 1, -r, n, E)
        em, en = oracle.envelope(a[:n], r)
        assert np.array_equal(gm, em) and np.array_equal(gn, en), (n, r)
    gm, gn = _model_lanes(a, 3 * E + 5, 0, cap - 3 * E - 4, E, mistake="m_swapped")
    em, en = oracle.bf1d(a, 3 * E + 5)
    assert not (np.array_equal(gm, em) and np.array_equal(gn, en))
    gm, gn = _model_lanes(a[:100], 61, -30, 100, E, mistake="identity_pad_one_side")
    em, en = oracle.envelope(a[:100], 30)
    assert np.array_equal(gm, em) and not np.array_equal(gn, en)


def _lane_envelope_arrays(a, r, E, staged, restore):
    """The lane-block envelope with the prefix arrays addressed as the kernel
    does: [E][33] words, element e of lane j at row e, column j, and column
    32 an identity column that windows reaching past the last lane read.  A
    staged next series (128 bytes per lane: lane l's words [32l, 32l + 32) of
    the flat array) covers the min side's array before this series' prefix
    is written; the kernel then writes the identity column again (restore)."""
    lanes, ROW = 32, 33
    n = len(a)
    cap = lanes * E
    w, d, s = 2 * r + 1, -r, 2 * r
    q, rr = divmod(s, E)
    x = np.full(cap, float(a[-1]))
    x[:n] = a
    out = []
    for side, (op, ident) in enumerate(((max, -np.inf), (min, np.inf))):
        arr = np.full(E * ROW, np.nan)
        arr[32::ROW] = ident  # the identity column, written once per kernel
        if staged and side == 1:
            arr[:32 * 32] = -1e9  # the next series' staged words (below this series)
            if restore:
                arr[32::ROW] = ident
        P = x.copy()
        S = x.copy()
        for j in range(lanes):
            b = j * E
            for e in range(1, E):
                P[b + e] = op(P[b + e - 1], x[b + e])
            for e in range(E - 2, -1, -1):
                S[b + e] = op(S[b + e + 1], x[b + e])
            for e in range(E):
                arr[e * ROW + j] = P[b + e]  # the prefix pass writes columns 0..31 only
        A = [S[j * E] for j in range(lanes)]
        m1, m2 = _lane_windows(A, q, op, ident)
        incl = list(itertools.accumulate(A, op))
        res = np.empty(n)
        for o in range(n):
            lo = o + d
            if lo >= 0:
                j, e = divmod(lo, E)
                far = e >= E - rr
                K = min(j + q + (1 if far else 0), 32)
                eh = e + rr - (E if far else 0)
                res[o] = op(op(S[lo], m2[j] if far else m1[j]), arr[eh * ROW + K])
            else:
                hi = lo + s
                K = min(hi // E, 32)
                res[o] = op(incl[K - 1] if K > 0 else ident, arr[(hi % E) * ROW + K])
        out.append(res)
    return out


def test_staged_series_needs_the_identity_column_again():
    """Windows reaching past the last lane read the identity column; a staged
    copy of the next series covers it, so the kernel writes it again: with
    that, the envelope equals the oracle's; without it, the min side does not
    (the max side's array is never staged)."""
    E = 32
    a = synth.random_walk(32 * E, seed=12, dtype=np.float32).astype(np.float64)
    r = 51
    em, en = oracle.envelope(a.astype(np.float32), r)
    gm, gn = _lane_envelope_arrays(a, r, E, staged=True, restore=True)
    assert np.array_equal(gm, em) and np.array_equal(gn, en)
    gm, gn = _lane_envelope_arrays(a, r, E, staged=False, restore=False)
    assert np.array_equal(gm, em) and np.array_equal(gn, en)
    gm, gn = _lane_envelope_arrays(a, r, E, staged=True, restore=False)
    assert np.array_equal(gm, em) and not np.array_equal(gn, en)
