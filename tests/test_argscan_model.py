"""CPU model of the block-scan arg filter's decomposition (van Herk/Gil-Werman
over (value, position) pairs, Section 2), checked against the oracle's scan of
every window.  It follows the kernel's steps with a small tile so that tiles,
blocks and their carries all occur on short inputs:

* blocks of w from position 0; out[j] = S[j] joined with Q[j], S the segmented
  suffix scan of x, Q the segmented exclusive prefix scan of y[i] = x[i+w];
* a tile holds whole blocks (w <= tile) or one tile of one block, whose parts
  of S and Q outside the tile come from per-tile aggregates scanned within
  each block;
* each thread: one forward sweep (local Q and the two summaries), a segmented
  scan of the summaries across threads, one backward sweep;
* ties: S wins against Q, the earlier position inside each scan; identities
  are -inf/+inf and tie with infinite data.

The model is its own code (no part of the GPU path); it pins the tie argument
and the carry structure on the CPU."""
import numpy as np
import pytest

import oracle
import synth

E, NT = 4, 16
TILE = E * NT


def _side(x, w, is_max):
    n = len(x)
    n_out = n - w + 1
    ident = -np.inf if is_max else np.inf

    def gt(a, b):
        return a > b if is_max else a < b

    def ge(a, b):
        return a >= b if is_max else a <= b

    def join(a, b):  # a left of b
        return b if gt(b[0], a[0]) else a

    none = (ident, 0)
    out_v = np.zeros(n_out)
    out_i = np.zeros(n_out, np.int64)
    if w > TILE:
        ntiles = -(-w // TILE)
        nbo = -(-n_out // w)  # blocks holding outputs; Q reads the block after them

        def tile_agg(b, t):  # leftmost extreme of tile t of block b, or None if empty
            lo = b * w + t * TILE
            best = None
            for i in range(lo, min(lo + TILE, (b + 1) * w, n)):
                if best is None or gt(x[i], best[0]):
                    best = (x[i], i)
            return best

        def keep_left(a, b):  # a's range left of b's
            if a is None:
                return b
            if b is None:
                return a
            return b if gt(b[0], a[0]) else a

        pre, suf = [], []
        for b in range(nbo + 1):
            aggs = [tile_agg(b, t) for t in range(ntiles)]
            p, acc = [], None
            for a in aggs:
                acc = keep_left(acc, a)
                p.append(acc)
            q, acc = [None] * ntiles, None
            for t in reversed(range(ntiles)):
                acc = keep_left(aggs[t], acc)
                q[t] = acc
            pre.append(p)
            suf.append(q)
        tiles = [(b, t) for b in range(nbo) for t in range(ntiles)]
    else:
        ntiles = 0
        length = (TILE // w) * w
        tiles = [(c, 0) for c in range(-(-n_out // length))]
    for b, t in tiles:
        if ntiles == 0:
            ln, base, r0 = length, b * length, 0
        else:
            r0 = t * TILE
            base, ln = b * w + r0, min(TILE, w - r0)
        if base >= n_out:
            continue
        xs = [x[base + p] if p < ln and base + p < n else np.nan for p in range(TILE)]
        ys = [x[base + w + p] if p < ln and base + w + p < n else np.nan for p in range(TILE)]
        cq = cs = none
        if ntiles:
            if t > 0 and pre[b + 1][t - 1] is not None:
                cq = (pre[b + 1][t - 1][0], pre[b + 1][t - 1][1] - base)
            if t + 1 < ntiles and suf[b][t + 1] is not None:
                cs = (suf[b][t + 1][0], suf[b][t + 1][1] - base)
        # Segment starts and ends among each thread's positions; past the last
        # tile of a block (phase >= w) a thread has none.
        starts, ends = [], []
        for th in range(NT):
            r = ((th * E) % w) if ntiles == 0 else r0 + th * E
            ph = [r + k if ntiles else (r + k) % w for k in range(E)]
            starts.append({k for k in range(E) if ph[k] == 0})
            ends.append({k for k in range(E) if ph[k] == w - 1})
        staged = [None] * TILE
        qsum, ssum = [], []
        for th in range(NT):
            q, s, done = none, none, False
            for k in range(E):
                p = th * E + k
                if k in starts[th]:
                    q = none
                staged[p] = q
                if gt(ys[p], q[0]):
                    q = (ys[p], w + p)
                if not done:
                    if gt(xs[p], s[0]):
                        s = (xs[p], p)
                    done = k in ends[th]
            qsum.append((q, bool(starts[th])))
            ssum.append((s, bool(ends[th])))
        for th in range(NT):
            c = cq
            for u in range(th):
                c = qsum[u][0] if qsum[u][1] else join(c, qsum[u][0])
            d = cs
            for u in range(NT - 1, th, -1):
                d = ssum[u][0] if ssum[u][1] else join(ssum[u][0], d)
            first = min(starts[th]) if starts[th] else E
            s = d
            for k in reversed(range(E)):
                p = th * E + k
                if k in ends[th]:
                    s = none
                if ge(xs[p], s[0]):
                    s = (xs[p], p)
                q = join(c, staged[p]) if k < first else staged[p]
                res = q if gt(q[0], s[0]) else s
                if p < ln and base + p < n_out:
                    out_v[base + p], out_i[base + p] = res[0], base + res[1]
    return out_v, out_i


def _check(a, w):
    f = a.astype(np.float64)
    vmx, imx = _side(f, w, True)
    vmn, imn = _side(f, w, False)
    emx, emn = oracle.argbf1d(a, w)
    bmx, bmn = oracle.bf1d(a, w)
    assert np.array_equal(imx, emx) and np.array_equal(imn, emn), f"positions w={w}"
    assert np.array_equal(vmx, bmx.astype(np.float64)) and np.array_equal(vmn, bmn.astype(np.float64))


@pytest.mark.parametrize("w", [1, 2, 3, 5, TILE - 1, TILE, TILE + 1, 3 * TILE + 7])
def test_model_random_walk(w):
    _check(synth.random_walk(700, seed=w, dtype=np.float32), w)


@pytest.mark.parametrize("w", [2, 3, 7, TILE + 1, 2 * TILE])
def test_model_ties_and_infinities(w):
    u = (synth.uniform(600, seed=w, dtype=np.uint8) // 64).astype(np.uint8)
    _check(u, w)
    _check(np.full(max(300, 3 * w), 2.5, np.float32), w)
    a = synth.uniform(500, seed=w, dtype=np.float32)
    a[::5] = -np.inf
    a[2::9] = np.inf
    a[100:260] = -np.inf
    _check(a, w)


def test_model_edges():
    for n, w in [(1, 1), (5, 5), (6, 5), (TILE + 1, TILE + 1), (2 * TILE + 1, TILE + 1)]:
        _check(synth.uniform(n, seed=n, dtype=np.float32), w)
