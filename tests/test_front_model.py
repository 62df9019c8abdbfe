"""CPU model of the advancing-front schedule of the block scan (windows of a
tile or more), checked against the oracle, and a check that its waits always
end.

Decomposition (Section 2's van Herk/Gil-Werman idea at tile granularity):
with tiles of T elements, s = w-1 = q*T + r (q >= 1), the window of output j
of output tile t is the rest of tile t from j, the whole tiles t+1..t+q-1,
and the start of tile t+q up to k = j+s (or all of tile t+q and the start of
tile t+q+1).  A grid of G CTAs takes output tiles round-robin (CTA b: rounds
t = b, b+G, b+2G, ...).  A prologue, before any round, publishes the
aggregates of tiles 1 .. q+G-1; round t waits until the aggregates of tiles
t+1..t+q-1 are published, publishes tile t+q+G (read ahead, when any later
round needs it) and forms its outputs.

The model runs the CTAs in random interleavings at reduced tile sizes,
checks that every aggregate a round takes was published by the prologue or
by an earlier round (so the waits end whatever the interleaving: no state
is reached where every CTA waits), and compares the outputs with the oracle.
A schedule in which some tile's aggregate has no publisher (no prologue)
hangs, and one that took a tile's aggregate from the wrong tile gives wrong
outputs: both fail here."""
import numpy as np
import pytest

import oracle
import synth


def _run_front(a, w, T, G, rng, mode="valid", r_env=0, mistake=None):
    n = len(a)
    s = w - 1
    q = s // T
    d = -r_env if mode == "envelope" else 0
    n_out = n if mode == "envelope" else n - w + 1
    tiles = -(-n_out // T)
    G = min(G, tiles)
    last = tiles + q - 2  # the last tile whose aggregate any round takes
    # Virtual padding: positions outside [0, n) hold identities.
    span = (tiles + q + G + 2) * T
    pos = d + np.arange(span)
    inside = (pos >= 0) & (pos < n)
    vals = np.where(inside, a[np.clip(pos, 0, n - 1)].astype(np.float64), 0.0)
    xm = np.where(inside, vals, -np.inf)
    xn = np.where(inside, vals, np.inf)

    published = {}  # tile -> (max, min, publisher: -1 for the prologue, else the round)
    out_m = np.full(n_out, np.nan)
    out_n = np.full(n_out, np.nan)

    def publish(tile, who):
        v = (xm[tile * T:(tile + 1) * T].max(), xn[tile * T:(tile + 1) * T].min())
        assert tile not in published, "a tile is published twice"
        published[tile] = (*v, who)

    if mistake != "no_prologue":
        for x in range(1, q + G):
            publish(x, -1)

    def round_steps(t):
        """One round as a generator: yields 'wait' until its aggregates are
        published, then finishes."""
        needed = list(range(t + 1, t + q))
        if mistake == "between_off_by_one":
            needed = [x - 1 for x in needed]
        while any(x not in published for x in needed):
            yield "wait"
        for x in needed:
            assert published[x][2] < t, "a round waited on a later one"
        if t + q + G <= last:
            publish(t + q + G, t)
        bm = max([published[x][0] for x in needed], default=-np.inf)
        bn = min([published[x][1] for x in needed], default=np.inf)
        o0, o1 = t * T, min((t + 1) * T, n_out)
        for j in range(o0, o1):
            k = j + s
            jm = xm[j:(t + 1) * T].max()
            jn = xn[j:(t + 1) * T].min()
            kt = k // T
            if kt == t + q:
                km, kn = xm[kt * T:k + 1].max(), xn[kt * T:k + 1].min()
            else:
                assert kt == t + q + 1
                km = max(xm[(t + q) * T:kt * T].max(), xm[kt * T:k + 1].max())  # all of K tile q, then q+1
                kn = min(xn[(t + q) * T:kt * T].min(), xn[kt * T:k + 1].min())
            out_m[j] = max(jm, bm, km)
            out_n[j] = min(jn, bn, kn)
        yield "done"

    ctas = [{"rounds": list(range(b, tiles, G)), "gen": None} for b in range(G)]
    while True:
        live = [c for c in ctas if c["gen"] is not None or c["rounds"]]
        if not live:
            break
        progressed = False
        for i in rng.permutation(len(live)):
            c = live[i]
            if c["gen"] is None:
                c["gen"] = round_steps(c["rounds"].pop(0))
            if next(c["gen"]) == "done":
                c["gen"] = None
                progressed = True
                break
            # "wait": try another CTA this round
        assert progressed, "every CTA waits: the schedule would hang"
    return out_m, out_n


@pytest.mark.parametrize("T", [8, 16])
@pytest.mark.parametrize("G", [1, 2, 3, 7])
@pytest.mark.parametrize("q,r", [(1, 0), (1, 5), (2, 3), (4, 0), (5, 7)])
def test_front_schedule_matches_oracle(T, G, q, r):
    if r >= T:
        pytest.skip("remainder below one tile")
    w = q * T + r + 1
    rng = np.random.default_rng(T * 100 + G * 10 + q + r)
    for n in (w, w + 1, w + 3 * T + 5, 11 * T + w + 2):
        a = synth.random_walk(n, seed=n + w, dtype=np.float64)
        gm, gn = _run_front(a, w, T, G, rng)
        em, en = oracle.bf1d(a, w)
        assert np.array_equal(gm, em) and np.array_equal(gn, en), (n, w, T, G)


@pytest.mark.parametrize("T,G,rr", [(8, 3, 9), (16, 2, 20), (8, 5, 33)])
def test_front_schedule_envelope(T, G, rr):
    rng = np.random.default_rng(rr)
    w = 2 * rr + 1
    a = synth.uniform(5 * T + 3, seed=rr, dtype=np.float64)
    gm, gn = _run_front(a, w, T, G, rng, mode="envelope", r_env=rr)
    em, en = oracle.envelope(a, rr)
    assert np.array_equal(gm, em) and np.array_equal(gn, en)


def test_front_schedule_planted_mistakes():
    """Planted mistakes fail: without the prologue the first q+G-1 tiles are
    published by nobody and every CTA ends up waiting; a between-range one
    tile early gives wrong outputs."""
    T, q = 8, 3
    w = q * T + 1
    a = synth.random_walk(40 * T + w, seed=1, dtype=np.float64)
    rng = np.random.default_rng(0)
    with pytest.raises(AssertionError, match="every CTA waits"):
        _run_front(a, w, T, 3, rng, mistake="no_prologue")
    em, en = oracle.bf1d(a, w)
    with pytest.raises(AssertionError):  # an early tile is not yet published, or outputs differ
        gm, gn = _run_front(a, w, T, 3, rng, mistake="between_off_by_one")
        assert np.array_equal(gm, em) and np.array_equal(gn, en)
    gm, gn = _run_front(a, w, T, 1, rng)  # the real schedule, even on one CTA
    assert np.array_equal(gm, em) and np.array_equal(gn, en)
