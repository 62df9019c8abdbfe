"""CPU model of the block-scan decomposition that the default 1D kernel uses
(Section 2's van Herk/Gil-Werman idea, Table 1), checked against the oracle.

The model takes the kernel's own choices at a reduced geometry (V elements
per thread, LANES threads per warp, NW warps per tile; the kernel has
32 lanes): per work item (a range of output tiles, positions relative to the
item's first window start), s = w-1 and

  * s < V         blocks of B = 2^floor(log2 s) inside a thread (mode 0),
  * s < W = LANES*V  the same B across lanes (mode 1),
  * s >= W        blocks of one warp slice (mode 2),

and output j is op(S_B[j], blocks strictly between, P_B[k]) with k = j+s.
For modes 0 and 1 it checks that at most one block lies between and takes
it, as the kernel does, from P_B at that block's end.  For mode 2 with
s >= T (case B) the blocks between are split as the kernel splits them: the
rest of j's tile, whole tiles kept in a sliding two-stack queue over a ring
of tile aggregates (a port of the kernel's queue, with the smallest ring the
kernel allows), the K tile of the previous step when k lies one tile
further, and the start of k's tile.  Positions outside the series hold the
identities (-inf for max, +inf for min), which is also how the centred
envelope is formed.  A wrong block size, a wrong split, an off-by-one in
the queue or a missing identity fails against the oracle."""
import numpy as np
import pytest

import oracle
import synth

GEOMETRIES = [(4, 4, 2), (2, 4, 4), (4, 2, 3)]  # (V, LANES, NW)


class TileQueue:
    """Sliding max/min of tile aggregates [c+1, c+q-1]: slots [fs, fe) hold
    suffix extremes up to fe-1, slots [fe, be) raw aggregates whose running
    extremes are (bm, bn); the older part is rebuilt in place when empty."""

    def __init__(self, ring, cap):
        self.ring, self.cap = ring, cap
        self.fs = self.fe = self.be = 1
        self.bm, self.bn = -np.inf, np.inf

    def push(self, x):
        assert x == self.be
        m, n = self.ring[x % self.cap]
        self.bm, self.bn = max(self.bm, m), min(self.bn, n)
        self.be = x + 1

    def slide(self, x):
        self.fs += 1
        self.push(x)
        if self.fs >= self.fe:
            # As the kernel's warp does it: groups of 32 slots from the newest
            # down, lane l holding slot top - l, an inclusive scan over the
            # lanes (shuffles up by 1, 2, .., 16), then the carry of the
            # slots above the group (lane 31's result of the group before).
            cm, cn = -np.inf, np.inf
            top = self.be - 1
            while top >= self.fs:
                ys = [top - l for l in range(32)]
                m = [self.ring[y % self.cap][0] if y >= self.fs else -np.inf for y in ys]
                n = [self.ring[y % self.cap][1] if y >= self.fs else np.inf for y in ys]
                d = 1
                while d < 32:
                    um, un = list(m), list(n)  # every lane reads before any writes
                    for l in range(d, 32):
                        m[l], n[l] = max(m[l], um[l - d]), min(n[l], un[l - d])
                    d <<= 1
                m = [max(v, cm) for v in m]
                n = [min(v, cn) for v in n]
                for l, y in enumerate(ys):
                    if y >= self.fs:
                        self.ring[y % self.cap] = (m[l], n[l])
                cm, cn = m[31], n[31]
                top -= 32
            self.bm, self.bn = -np.inf, np.inf
            self.fe = self.be

    def query(self):
        m, n = self.bm, self.bn
        if self.fs < self.fe:
            f = self.ring[self.fs % self.cap]
            m, n = max(m, f[0]), min(n, f[1])
        return m, n


def _block_scans(x, B, op):
    """Prefix and suffix scans restarting at every multiple of B."""
    P = x.copy()
    S = x.copy()
    for i in range(1, len(x)):
        if i % B:
            P[i] = op(P[i - 1], x[i])
    for i in range(len(x) - 2, -1, -1):
        if (i + 1) % B:
            S[i] = op(S[i + 1], x[i])
    return P, S


def _item(a, d, s, o_begin, o_end, geo):
    """Outputs [o_begin, o_end) of one item: window of output o starts at
    o + d (d = 0 valid, -r envelope) and has s+1 elements."""
    V, LANES, NW = geo
    W = LANES * V
    T = NW * W
    n = len(a)
    p0 = o_begin + d
    NC = -(-(o_end - o_begin) // T)
    q = s // T
    span = (NC + q + 2) * T  # every K tile an item can reach
    pos = p0 + np.arange(span)
    inside = (pos >= 0) & (pos < n)
    vals = np.where(inside, a[np.clip(pos, 0, n - 1)].astype(np.float64), 0.0)
    xm = np.where(inside, vals, -np.inf)
    xn = np.where(inside, vals, np.inf)
    if s < W:
        B = 1 << (s.bit_length() - 1) if s >= 1 else 1
    else:
        B = W
    out_m = np.empty(o_end - o_begin)
    out_n = np.empty(o_end - o_begin)
    for side, x, op in ((0, xm, max), (1, xn, min)):
        P, S = _block_scans(x, B, op)
        agg = [op(*x[b * B:(b + 1) * B]) if B > 1 else x[b] for b in range(span // B)]
        ring = None
        if s >= T:  # case B: the queue over tile aggregates of this item
            cap = q + 2  # the smallest ring the kernel's bound allows
            ring = [None] * cap
            tagg = lambda t: (max(xm[t * T:(t + 1) * T]), min(xn[t * T:(t + 1) * T]))
            for t in range(1, q + 1):
                ring[t % cap] = tagg(t)
            tq = TileQueue(ring, cap)
            for t in range(1, q):
                tq.push(t)
        for c in range(NC):
            if s >= T:
                between_tiles = tq.query()[side]
            for j in range(c * T, min((c + 1) * T, o_end - o_begin)):
                k = j + s
                bj, bk = j // B, k // B
                if s == 0:
                    v = x[j]
                elif s < W:
                    assert bk - bj in (1, 2), (s, B, j)  # B <= s < 2B
                    v = op(S[j], P[k])
                    if bk - bj == 2:
                        v = op(v, P[(bj + 2) * B - 1])  # the block between, at its end
                elif s < T:
                    v = op(S[j], P[k])
                    for b in range(bj + 1, bk):
                        v = op(v, agg[b])
                else:
                    tj, tk = j // T, k // T
                    assert tj == c and tk in (c + q, c + q + 1)
                    v = op(S[j], P[k])
                    for b in range(bj + 1, (tj + 1) * T // B):  # rest of j's tile
                        v = op(v, agg[b])
                    v = op(v, between_tiles)  # tiles c+1 .. c+q-1
                    if tk == c + q + 1:  # tile c+q, the previous K tile
                        v = op(v, max(xm[(c + q) * T:(c + q + 1) * T]) if side == 0
                               else min(xn[(c + q) * T:(c + q + 1) * T]))
                    for b in range(tk * T // B, bk):  # start of k's tile
                        v = op(v, agg[b])
                (out_m if side == 0 else out_n)[j] = v
            if s >= T and c + 1 < NC:
                # publish K tile c+q+1, then slide to output tile c+1's range
                ring[(c + q + 1) % cap] = tagg(c + q + 1)
                if q >= 2:
                    tq.slide(c + q)
    return out_m, out_n


def _model(a, w_or_r, mode, geo, seg_tiles):
    V, LANES, NW = geo
    T = NW * LANES * V
    n = len(a)
    if mode == "valid":
        s, d, n_out = w_or_r - 1, 0, max(0, n - w_or_r + 1)
    else:
        r = min(w_or_r, max(n - 1, 0))
        s, d, n_out = 2 * r, -r, n
    om = np.empty(n_out)
    on = np.empty(n_out)
    for ob in range(0, n_out, seg_tiles * T):
        oe = min(ob + seg_tiles * T, n_out)
        om[ob:oe], on[ob:oe] = _item(a, d, s, ob, oe, geo)
    return om, on


WINDOWS = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 47, 63, 64, 65, 95, 96, 97, 127, 128, 129, 161, 200]


@pytest.mark.parametrize("geo", GEOMETRIES)
@pytest.mark.parametrize("seg_tiles", [1, 3])
def test_valid_windows_match_the_definition(geo, seg_tiles):
    rng = np.random.default_rng(sum(geo) + seg_tiles)
    for w in WINDOWS:
        n = int(rng.integers(w, w + 400))
        for a in (synth.random_walk(n, seed=w, dtype=np.float32),
                  rng.integers(0, 4, size=n).astype(np.int16)):  # many ties
            gm, gn = _model(a, w, "valid", geo, seg_tiles)
            em, en = oracle.bf1d(a, w)
            assert np.array_equal(gm, em.astype(np.float64)), (geo, w, n)
            assert np.array_equal(gn, en.astype(np.float64)), (geo, w, n)


@pytest.mark.parametrize("geo", GEOMETRIES[:2])
def test_envelope_matches_the_definition(geo):
    rng = np.random.default_rng(7)
    for r in [0, 1, 2, 5, 8, 16, 40, 70, 100]:
        n = int(rng.integers(1, 500))
        a = synth.random_walk(n, seed=r, dtype=np.float32)  # both signs: a wrong identity shows
        gm, gn = _model(a, r, "envelope", geo, 2)
        em, en = oracle.envelope(a, r)
        assert np.array_equal(gm, em.astype(np.float64)) and np.array_equal(gn, en.astype(np.float64)), (r, n)


def test_tile_queue_is_a_sliding_window():
    """The queue alone against a brute-force window over random aggregates,
    with the smallest ring (q + 2 slots), for q = 1..9."""
    rng = np.random.default_rng(3)
    for q in list(range(1, 10)) + [33, 34, 40, 65, 66, 97]:  # the rebuild spans 1 to 3 lane groups
        vals = rng.integers(0, 5 if q < 10 else 1000, size=80 + 3 * q).astype(float)
        cap = q + 2
        ring = [None] * cap
        for t in range(1, q + 1):
            ring[t % cap] = (vals[t], vals[t])
        tq = TileQueue(ring, cap)
        for t in range(1, q):
            tq.push(t)
        for c in range(0, len(vals) - q - 2):
            lo, hi = c + 1, c + q - 1
            want = (max(vals[lo:hi + 1]), min(vals[lo:hi + 1])) if hi >= lo else (-np.inf, np.inf)
            assert tq.query() == want, (q, c)
            ring[(c + q + 1) % cap] = (vals[c + q + 1], vals[c + q + 1])
            if q >= 2:
                tq.slide(c + q)


def test_register_slide_windows():
    """The register slide (windows up to 17 for f32, 9 for the other types):
    a thread holds its V elements and the HALO that follow them; doubling
    passes p = 1, 2, .., P2/2 in place, then each window of W = P2 + r is the
    union of values i and i + r.  Every output must use only the NE = V + HALO
    values held and equal the window's extreme."""
    rng = np.random.default_rng(17)
    for V, HALO, wmax in ((16, 16, 17), (16, 8, 9), (4, 8, 9)):  # f32; i16/u8; f64
        NE = V + HALO
        for W in range(1, wmax + 1):
            P2 = 16 if W >= 16 else 8 if W >= 8 else 4 if W >= 4 else 2 if W >= 2 else 1
            assert (V - 1) + (W - P2) + P2 - 1 < NE  # the last value read stays in the thread
            x = rng.integers(-3, 4, size=(200, NE)).astype(float)
            a = x.copy()
            p = 1
            while p < P2:
                for i in range(NE - p):
                    a[:, i] = np.maximum(a[:, i], a[:, i + p])
                p <<= 1
            got = np.maximum(a[:, :V], a[:, W - P2:W - P2 + V])
            want = np.stack([x[:, i:i + W].max(axis=1) for i in range(V)], axis=1)
            assert np.array_equal(got, want), (V, HALO, W)
