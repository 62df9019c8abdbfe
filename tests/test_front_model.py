"""CPU model of the advancing-front schedule of the block scan (windows of a
tile or more), checked against the oracle, and a check that its waits always
end.

Decomposition (Section 2's van Herk/Gil-Werman idea at tile granularity):
with tiles of T elements, s = w-1 = q*T + r (q >= 1), the window of output j
of output tile t is the rest of tile t from j, the whole tiles t+1..t+q-1,
and the start of tile t+q up to k = j+s (or all of tile t+q and the start of
tile t+q+1).  Work item t is output tile t, handed out in ticket order to G
CTAs, each holding up to three tickets.  An item reads tile t+q (its first K
tile) and publishes that tile's aggregate before it waits for anything; item
0 instead reads and publishes tiles 1..q.  Every later item takes the
aggregates of tiles t+1..t+q-1 from the published ones (it waits until they
are there), reads tile t+q+1 when some window reaches it (publishing it), and
reads tile t again for the suffixes.

The model runs the CTAs in random interleavings at reduced tile sizes,
checks that every published aggregate is published by an earlier ticket
(so the waits end whatever the interleaving: no state is reached where every
CTA waits), and compares the outputs with the oracle.  A schedule in which
some tile's aggregate has no earlier publisher (item 0 without its
prologue) hangs, and one that took a tile's aggregate from the wrong tile
gives wrong outputs: both fail here."""
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
    NC = -(-n_out // T)
    # Virtual padding: positions outside [0, n) hold identities.
    span = (NC + q + 2) * T
    pos = d + np.arange(span)
    inside = (pos >= 0) & (pos < n)
    vals = np.where(inside, a[np.clip(pos, 0, n - 1)].astype(np.float64), 0.0)
    xm = np.where(inside, vals, -np.inf)
    xn = np.where(inside, vals, np.inf)

    published = {}  # global tile -> (max, min, publishing ticket)
    out_m = np.full(n_out, np.nan)
    out_n = np.full(n_out, np.nan)

    def publish(tile, ticket):
        v = (xm[tile * T:(tile + 1) * T].max(), xn[tile * T:(tile + 1) * T].min())
        if tile in published:
            assert published[tile][:2] == v  # duplicates publish the same bits
        else:
            published[tile] = (*v, ticket)

    def item_steps(t):
        """The item as a generator: yields 'wait' until its aggregates are
        published, then finishes."""
        if t == 0 and mistake != "no_prologue":
            for x in range(1, q + 1):
                publish(x, t)
        else:
            publish(t + q, t)
            needed = list(range(t + 1, t + q)) if t else []
            if mistake == "between_off_by_one":
                needed = [x - 1 for x in needed]
            while any(x not in published for x in needed):
                yield "wait"
            for x in needed:
                assert published[x][2] < t, "an item waited on a later ticket"
        o0, o1 = t * T, min((t + 1) * T, n_out)
        if (o1 - 1 + s) // T >= t + q + 1:  # some window reaches tile t+q+1
            publish(t + q + 1, t)
        between = range(t + 1, t + q) if mistake != "between_off_by_one" else range(t, t + q - 1)
        if mistake == "no_prologue" and t == 0:
            between = []  # item 0 would read tiles 1..q-1 itself; here it is the only item that does not wait
        between_m = max([published.get(x, (-np.inf, np.inf))[0] for x in between], default=-np.inf)
        between_n = min([published.get(x, (-np.inf, np.inf))[1] for x in between], default=np.inf)
        for j in range(o0, o1):
            k = j + s
            jm = xm[j:(t + 1) * T].max()
            jn = xn[j:(t + 1) * T].min()
            kt = k // T
            if kt == t + q:
                km, kn = xm[kt * T:k + 1].max(), xn[kt * T:k + 1].min()
            else:
                assert kt == t + q + 1
                km = max(published[t + q][0], xm[kt * T:k + 1].max())
                kn = min(published[t + q][1], xn[kt * T:k + 1].min())
            out_m[j] = max(jm, between_m, km)
            out_n[j] = min(jn, between_n, kn)
        yield "done"

    next_ticket = 0
    ctas = []
    for _ in range(G):
        ctas.append({"queue": [], "gen": None})
    def take(c):
        nonlocal next_ticket
        while len(c["queue"]) < 3 and next_ticket < NC:
            c["queue"].append(next_ticket)
            next_ticket += 1
    for c in ctas:
        take(c)
    while True:
        live = [c for c in ctas if c["gen"] is not None or c["queue"]]
        if not live:
            break
        progressed = False
        for c in rng.permutation(len(live)):
            c = live[c]
            if c["gen"] is None:
                c["gen"] = item_steps(c["queue"].pop(0))
                take(c)
            st = next(c["gen"])
            if st == "done":
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
    """Planted mistakes fail: without item 0's prologue the tiles 1..q-1 are
    published by nobody and every CTA ends up waiting; a between-range one
    tile early gives wrong outputs."""
    T, q = 8, 3
    w = q * T + 1
    a = synth.random_walk(12 * T + w, seed=1, dtype=np.float64)
    rng = np.random.default_rng(0)
    with pytest.raises(AssertionError, match="every CTA waits"):
        _run_front(a, w, T, 2, rng, mistake="no_prologue")
    gm, gn = _run_front(a, w, T, 2, rng, mistake="between_off_by_one")
    em, en = oracle.bf1d(a, w)
    assert not (np.array_equal(gm, em) and np.array_equal(gn, en))
    gm, gn = _run_front(a, w, T, 1, rng)  # the real schedule, even on one CTA
    assert np.array_equal(gm, em) and np.array_equal(gn, en)
