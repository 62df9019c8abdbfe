"""GPU tests of the streaming service: chunked outputs equal the whole-array
oracle exactly, a stream gives the same outputs alone and in the mix, and
host-side failures (closed streams, stalls, oversize chunks) return errors
without touching the GPU's health."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _split(n, rng, lo=1, hi=5000):
    cuts = []
    pos = 0
    while pos < n:
        c = int(rng.integers(lo, hi))
        cuts.append(min(c, n - pos))
        pos += c
    return cuts


def _serve(mmf, streams, budget=1 << 28, max_batch=64, interleave=True, seed=0):
    """streams: list of (data, w, chunk lengths).  Returns per-stream outputs."""
    srv = mmf.Server(budget, max_batch, "float32")
    ids = [srv.open(w) for _, w, _ in streams]
    pos = [0] * len(streams)
    ci = [0] * len(streams)
    outs = [([], []) for _ in streams]
    pend = []
    order = np.random.default_rng(seed)
    live = list(range(len(streams)))
    while live:
        k = int(order.choice(live)) if interleave else live[0]
        data, w, cl = streams[k]
        L = cl[ci[k]]
        chunk = np.ascontiguousarray(data[pos[k]:pos[k] + L])
        m = mmf.n_outputs(pos[k], L, w)
        omax = np.empty(m, np.float32)
        omin = np.empty(m, np.float32)
        t, n_out = srv.push(ids[k], chunk, omax, omin)
        assert n_out == m
        pend.append(t)
        outs[k][0].append(omax)
        outs[k][1].append(omin)
        pos[k] += L
        ci[k] += 1
        if ci[k] == len(cl):
            live.remove(k)
    for t in pend:
        srv.wait(t)
    st = srv.stats()
    for sid in ids:
        srv.close_stream(sid)
    srv.close()
    return [(np.concatenate(a) if a else np.empty(0, np.float32),
             np.concatenate(b) if b else np.empty(0, np.float32)) for a, b in outs], st


def test_chunked_equals_whole_array(mmf):
    rng = np.random.default_rng(5)
    streams = []
    for k in range(24):
        n = int(rng.integers(1, 40_000))
        w = int(rng.choice([1, 2, 3, 8, 9, 31, 257, 1001, 4096, 5000]))
        data = synth.random_walk(n, 100 + k, np.float32)
        streams.append((data, w, _split(n, rng, 1, 7000)))
    outs, st = _serve(mmf, streams)
    for (data, w, cl), (gm, gn) in zip(streams, outs):
        em, en = oracle.stream_reference(np.split(data, np.cumsum(cl)[:-1]), w)
        assert np.array_equal(gm, em) and np.array_equal(gn, en), (len(data), w)
    assert st["chunks"] == sum(len(c) for _, _, c in streams)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # Latency splits into the wait for admission and the batch's service.
    assert st["p99_service_ms"] >= st["p50_service_ms"] > 0 and st["p99_queue_ms"] >= st["p50_queue_ms"] >= 0
    assert st["p50_queue_ms"] + st["p50_service_ms"] <= 2 * st["p99_ms"] and st["max_hold_ms"] >= 0


def test_alone_equals_in_the_mix(mmf):
    rng = np.random.default_rng(9)
    target = (synth.piecewise_monotone(30_000, 3, np.float32), 777, _split(30_000, rng, 100, 4000))
    others = [(synth.uniform(20_000, 50 + k, np.float32), int(rng.choice([5, 64, 2000])),
               _split(20_000, rng, 10, 3000)) for k in range(16)]
    alone, _ = _serve(mmf, [target])
    mixed, _ = _serve(mmf, [target] + others, max_batch=8, seed=3)
    assert np.array_equal(alone[0][0], mixed[0][0]) and np.array_equal(alone[0][1], mixed[0][1])
    em, en = oracle.bf1d(target[0], target[1])
    assert np.array_equal(alone[0][0], em) and np.array_equal(alone[0][1], en)


def test_tight_budget_admission(mmf):
    """A budget that holds only a few chunks at a time: admission waits for
    completions and every result is still exact."""
    rng = np.random.default_rng(12)
    streams = [(synth.random_walk(60_000, 7 + k, np.float32), 513, _split(60_000, rng, 4000, 16_000))
               for k in range(6)]
    outs, _ = _serve(mmf, streams, budget=1 << 20, max_batch=4)
    for (data, w, _), (gm, gn) in zip(streams, outs):
        em, en = oracle.bf1d(data, w)
        assert np.array_equal(gm, em) and np.array_equal(gn, en)


def test_host_side_faults(mmf):
    srv = mmf.Server(1 << 20, 8, "float32")
    sid = srv.open(16)
    x = synth.uniform(100_000, 1, np.float32)
    # a chunk that can never fit the budget
    big = np.ascontiguousarray(x)
    with pytest.raises(mmf.MMFError) as e:
        srv.push(sid, big, np.empty(100_000, np.float32), None)
    assert e.value.status == 2  # MMF_ENOMEM
    # a stalled service: the wait times out, then completes after resuming
    srv.pause(True)
    chunk = np.ascontiguousarray(x[:1000])
    om = np.empty(985, np.float32)
    t, m = srv.push(sid, chunk, om, None)
    with pytest.raises(mmf.MMFError) as e:
        srv.wait(t, timeout_ms=50)
    assert e.value.status == 5  # MMF_ETIMEOUT
    with pytest.raises(mmf.MMFError) as e:
        srv.close_stream(sid, timeout_ms=20)  # still pending
    assert e.value.status == 5
    srv.pause(False)
    srv.wait(t)
    assert np.array_equal(om, oracle.bf1d(chunk, 16)[0])
    # the stream was closed by the timed-out close: pushes are refused
    with pytest.raises(mmf.MMFError) as e:
        srv.push(sid, chunk, om, None)
    assert e.value.status == 6  # MMF_ECLOSED
    with pytest.raises(mmf.MMFError) as e:
        srv.push(12345, chunk, om, None)
    assert e.value.status == 6
    srv.close()
    assert mmf.device_status() == 0


def test_push_batch_equals_whole_array(mmf):
    """Chunks of many streams queued with mmf_stream_push_batch (several of a
    stream in one call, in order) and waited with mmf_ticket_wait_batch give
    the filter of each stream's concatenation."""
    rng = np.random.default_rng(17)
    ns = 40
    ws = rng.integers(1, 700, ns)
    data = [synth.random_walk(int(rng.integers(2000, 30000)), seed=100 + k, dtype=np.float32) for k in range(ns)]
    cuts = [_split(d.size, rng, 1, 3000) for d in data]
    srv = mmf.Server(1 << 28, 128, "float32")
    ids = np.array([srv.open(int(w)) for w in ws], dtype=np.uint64)
    # One flat host buffer per side for every output, laid out per chunk.
    events = []
    for k in range(ns):
        pos = 0
        for L in cuts[k]:
            events.append((k, pos, L))
            pos += L
    # A random interleaving of the streams that keeps each stream's chunks in order.
    per = {k: [e for e in events if e[0] == k] for k in range(ns)}
    seq = []
    nxt = {k: 0 for k in range(ns)}
    for _ in range(len(events)):
        live = [k for k in range(ns) if nxt[k] < len(per[k])]
        k = live[int(rng.integers(0, len(live)))]
        seq.append(per[k][nxt[k]])
        nxt[k] += 1
    m_of = [mmf.n_outputs(p, L, int(ws[k])) for k, p, L in seq]
    out_off = np.concatenate([[0], np.cumsum(m_of)])
    hmax = np.empty(max(1, int(out_off[-1])), np.float32)
    hmin = np.empty_like(hmax)
    chunks = [np.ascontiguousarray(data[k][p:p + L]) for k, p, L in seq]
    sids = np.array([ids[k] for k, _, _ in seq], dtype=np.uint64)
    cptr = np.array([c.ctypes.data for c in chunks], dtype=np.uint64)
    lens = np.array([L for _, _, L in seq], dtype=np.int64)
    mptr = np.array([hmax.ctypes.data + 4 * int(o) for o in out_off[:-1]], dtype=np.uint64)
    nptr = np.array([hmin.ctypes.data + 4 * int(o) for o in out_off[:-1]], dtype=np.uint64)
    tickets = []
    for a in range(0, len(seq), 97):  # groups of up to 97 chunks per call
        b = min(len(seq), a + 97)
        t, n_out = srv.push_batch(sids[a:b], cptr[a:b], lens[a:b], mptr[a:b], nptr[a:b])
        assert list(n_out) == m_of[a:b]
        tickets.append(t)
    srv.wait_batch(np.concatenate(tickets))
    srv.close()
    got = {k: ([], []) for k in range(ns)}
    for (k, p, L), o0, o1 in zip(seq, out_off[:-1], out_off[1:]):
        got[k][0].append(hmax[o0:o1])
        got[k][1].append(hmin[o0:o1])
    for k in range(ns):
        emx, emn = oracle.bf1d(data[k], int(ws[k]))
        assert np.array_equal(np.concatenate(got[k][0]), emx), k
        assert np.array_equal(np.concatenate(got[k][1]), emn), k


def _push_all(mmf, srv, sid, data, start, cuts, w, dtype=np.float32):
    """Pushes data[start:] in chunks of `cuts`; returns the concatenated
    outputs (max, min)."""
    mx, mn, ts = [], [], []
    pos = start
    for L in cuts:
        chunk = np.ascontiguousarray(data[pos:pos + L])
        m = mmf.n_outputs(pos, L, w)
        a = np.empty(m, dtype)
        b = np.empty(m, dtype)
        t, n_out = srv.push(sid, chunk, a, b)
        assert n_out == m
        ts.append(t)
        mx.append(a)
        mn.append(b)
        pos += L
    for t in ts:
        srv.wait(t)
    return np.concatenate(mx), np.concatenate(mn)


@pytest.mark.parametrize("w,cut_at", [(1, 5000), (2, 1), (5, 3), (257, 100), (257, 40_000), (9001, 20_000)])
def test_snapshot_restore_continues_exactly(mmf, w, cut_at):
    """A stream snapshotted after `cut_at` samples and restored as a new
    stream (on another server) gives, for the rest of the data, the outputs
    the original stream gives, and both equal the whole-array filter of the
    concatenation; snapshots before w-1 samples carry a shorter state."""
    rng = np.random.default_rng(w + cut_at)
    data = synth.random_walk(60_000, seed=w, dtype=np.float32)
    first = _split(cut_at, rng, 1, 3000)
    rest = _split(data.size - cut_at, rng, 1, 7000)
    srv = mmf.Server(1 << 26, 32, "float32")
    sid = srv.open(w)
    m0, n0 = _push_all(mmf, srv, sid, data, 0, first, w)
    state = srv.snapshot(sid)
    assert len(state) == 40 + 4 * min(cut_at, w - 1)
    m1, n1 = _push_all(mmf, srv, sid, data, cut_at, rest, w)
    srv2 = mmf.Server(1 << 26, 32, "float32")
    sid2 = srv2.restore(state)
    m2, n2 = _push_all(mmf, srv2, sid2, data, cut_at, rest, w)
    assert np.array_equal(m1, m2) and np.array_equal(n1, n2)
    emx, emn = oracle.bf1d(data, w)
    assert np.array_equal(np.concatenate([m0, m1]), emx) and np.array_equal(np.concatenate([n0, n1]), emn)
    srv.close()
    srv2.close()
    assert mmf.device_status() == 0


def test_snapshot_64bit_count_and_rejects(mmf):
    """A snapshot written by hand in the documented layout with a count past
    2^32 (an unbounded stream): the restored stream's outputs follow from its
    halo and the new samples alone.  Bad snapshots are refused on the host."""
    import struct
    w = 33
    halo = synth.uniform(w - 1, seed=1, dtype=np.float32)
    count = (1 << 40) + 12345
    state = struct.pack("<IIiiqqq", 0x53464D4D, 1, 0, 0, w, count, w - 1) + halo.tobytes()
    srv = mmf.Server(1 << 24, 8, "float32")
    sid = srv.restore(state)
    more = synth.uniform(5000, seed=2, dtype=np.float32)
    m = mmf.n_outputs(count, more.size, w)
    assert m == more.size
    a = np.empty(m, np.float32)
    b = np.empty(m, np.float32)
    t, n_out = srv.push(sid, more, a, b)
    srv.wait(t)
    emx, emn = oracle.bf1d(np.concatenate([halo, more]), w)
    assert np.array_equal(a, emx) and np.array_equal(b, emn)
    assert srv.snapshot(sid)[:40] == struct.pack("<IIiiqqq", 0x53464D4D, 1, 0, 0, w, count + more.size, w - 1)
    for bad in (state[:39], state[:-4], b"XXXX" + state[4:],
                struct.pack("<IIiiqqq", 0x53464D4D, 1, 1, 0, w, count, w - 1) + halo.tobytes(),
                struct.pack("<IIiiqqq", 0x53464D4D, 1, 0, 0, w, 3, w - 1) + halo.tobytes()):
        with pytest.raises(mmf.MMFError):
            srv.restore(bad)
    srv.close()
    assert mmf.device_status() == 0


def test_sizes_past_the_budget_are_refused_on_host(mmf):
    """Windows, chunk lengths and snapshot headers whose byte counts would
    pass 2^64 are refused before anything is copied (1 MiB budget), and the
    server keeps serving."""
    import ctypes
    import struct
    srv = mmf.Server(1 << 20, 8, "float32")
    for w in ((1 << 62) + 1, (1 << 20) + 1):
        with pytest.raises(mmf.MMFError) as e:
            srv.open(w)
        assert e.value.status == 2  # MMF_ENOMEM
    sid = srv.open(16)
    x = np.zeros(16, np.float32)
    n_out, t = ctypes.c_int64(0), ctypes.c_uint64(0)
    for n in (1 << 62, (1 << 62) + (1 << 61)):  # far past the 16 elements really there
        st = srv._lib.mmf_stream_push(srv._h, sid, ctypes.c_void_p(x.ctypes.data), n,
                                      ctypes.c_void_p(x.ctypes.data), None, ctypes.byref(n_out), ctypes.byref(t))
        assert st == 2
    for w in ((1 << 62) + 1, (1 << 61) + 1):
        for version, body in ((1, b"\0" * 64), (2, struct.pack("<qq", 1 << 60, 1 << 60) + b"\0" * 24)):
            hdr = struct.pack("<IIiiqqq", 0x53464D4D, version, 0, 0, w, w - 1, w - 1)
            with pytest.raises(mmf.MMFError) as e:
                srv.restore(hdr + body)
            assert e.value.status == 2
    # a wedge whose record count runs past the end of the buffer
    hdr = struct.pack("<IIiiqqq", 0x53464D4D, 2, 0, 0, 5, 100, 4)
    with pytest.raises(mmf.MMFError) as e:
        srv.restore(hdr + struct.pack("<qq", 4, 4) + struct.pack("<qf", 1, 1.0))
    assert e.value.status == 1  # MMF_EINVAL
    chunk = synth.uniform(1000, 3, np.float32)
    om = np.empty(985, np.float32)
    t2, m = srv.push(sid, chunk, om, None)
    srv.wait(t2)
    assert m == 985 and np.array_equal(om, oracle.bf1d(chunk, 16)[0])
    srv.close()
    assert mmf.device_status() == 0


@pytest.mark.parametrize("kind", ["random_walk", "uniform", "increasing", "decreasing", "constant", "steps"])
@pytest.mark.parametrize("w", [2, 33, 9001])
def test_wedge_snapshot_continues_exactly(mmf, kind, w):
    """A stream restored from its monotonic wedge (Section 4) continues with
    the outputs of the original: samples outside the wedge never decide a
    later window's extreme.  Ties (constant data, steps) included."""
    n, cut = 40_000, 23_456
    if kind == "increasing":
        data = np.arange(n, dtype=np.float32)
    elif kind == "decreasing":
        data = np.arange(n, 0, -1).astype(np.float32)
    elif kind == "constant":
        data = np.full(n, 2.5, np.float32)
    elif kind == "steps":
        data = np.repeat(synth.uniform(n // 100, seed=w, dtype=np.float32), 100)
    else:
        data = synth.by_name(kind, n, seed=w, dtype=np.float32)
    rng = np.random.default_rng(w)
    first = _split(cut, rng, 1, 3000)
    rest = _split(n - cut, rng, 1, 5000)
    srv = mmf.Server(1 << 26, 32, "float32")
    sid = srv.open(w)
    _push_all(mmf, srv, sid, data, 0, first, w)
    full = srv.snapshot(sid)
    wedge = srv.snapshot(sid, wedge=True)
    m1, n1 = _push_all(mmf, srv, sid, data, cut, rest, w)
    sid2 = srv.restore(wedge)
    m2, n2 = _push_all(mmf, srv, sid2, data, cut, rest, w)
    assert np.array_equal(m1, m2) and np.array_equal(n1, n2)
    if w == 9001:
        # i.i.d. noise: about ln(w) records per side; a random walk: on the
        # order of sqrt(w); monotone data: one side holds the whole window.
        if kind == "uniform":
            assert len(wedge) < len(full) // 50
        if kind == "random_walk":
            assert len(wedge) < len(full) // 5
    srv.close()
    assert mmf.device_status() == 0


def test_wedge_snapshot_rejects_bad_entries(mmf):
    import struct
    srv = mmf.Server(1 << 24, 8, "float32")
    hdr = struct.pack("<IIiiqqq", 0x53464D4D, 2, 0, 0, 5, 100, 4)
    good = hdr + struct.pack("<qq", 1, 1) + struct.pack("<qf", 1, 1.0) + struct.pack("<qf", 1, 1.0)
    sid = srv.restore(good)
    assert sid > 0
    for bad in (hdr + struct.pack("<qq", 1, 1) + struct.pack("<qf", 5, 1.0) + struct.pack("<qf", 1, 1.0),
                hdr + struct.pack("<qq", 0, 1) + struct.pack("<qf", 1, 1.0),
                hdr + struct.pack("<qq", 1, 1) + struct.pack("<qf", 1, 1.0)):
        with pytest.raises(mmf.MMFError):
            srv.restore(bad)
    srv.close()
