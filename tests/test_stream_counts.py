"""Output counts of a pushed chunk (host logic, no GPU): with zero stream
latency (Section 1) a chunk completes exactly the windows that end inside
it, so over any chunking the counts add up to the n-w+1 windows of the
whole stream, and the outputs released after each chunk are the prefix of
the whole-stream filter that the samples so far determine."""
import numpy as np

import oracle
import paper_cs_0610046_gb300 as mmf
import synth


def test_counts_follow_the_windows_that_end_in_each_chunk():
    rng = np.random.default_rng(21)
    for _ in range(200):
        n = int(rng.integers(0, 400))
        w = int(rng.integers(1, 60))
        cuts = np.sort(rng.integers(0, n + 1, size=int(rng.integers(0, 8))))
        lens = np.diff(np.concatenate([[0], cuts, [n]])).astype(int)
        data = synth.random_walk(max(n, 1), seed=n + w, dtype=np.float32)[:n]
        full_max, full_min = oracle.bf1d(data, w)
        count, released = 0, 0
        for c in lens:
            m = mmf.n_outputs(count, int(c), w)
            # windows [j, j+w) with end j+w-1 in [count, count+c)
            ends = np.arange(max(count, w - 1), count + c)
            assert m == ends.size
            count += int(c)
            released += m
            # everything released so far is the whole-stream filter's prefix
            # over the samples seen (no window waits for a later sample)
            pm, pn = oracle.bf1d(data[:count], w)
            assert np.array_equal(pm, full_max[:released]) and np.array_equal(pn, full_min[:released])
        assert released == max(0, n - w + 1)


def test_halo_state_gives_the_whole_stream_filter():
    """A stream's state is its last min(count, w-1) samples: filtering each
    chunk behind that halo (the windows that end inside the chunk) and then
    keeping the new last w-1 samples gives, chunk by chunk, exactly the
    whole-stream filter (each output depends on its own window alone)."""
    rng = np.random.default_rng(22)
    for _ in range(200):
        n = int(rng.integers(0, 400))
        w = int(rng.integers(1, 60))
        data = rng.integers(0, 5, size=n).astype(np.float32)  # ties
        halo = data[:0]
        count = 0
        got_m, got_n = [], []
        pos = 0
        while pos < n:
            c = int(rng.integers(1, 50))
            chunk = data[pos:pos + c]
            staged = np.concatenate([halo, chunk])
            m = mmf.n_outputs(count, chunk.size, w)
            if m:
                sm, sn = oracle.bf1d(staged, w)
                got_m.append(sm[-m:])  # the windows that end inside the chunk
                got_n.append(sn[-m:])
            count += chunk.size
            halo = staged[max(0, staged.size - (w - 1)):] if w > 1 else staged[:0]
            assert halo.size == min(count, w - 1)
            pos += c
        em, en = oracle.bf1d(data, w)
        gm = np.concatenate(got_m) if got_m else em[:0]
        gn = np.concatenate(got_n) if got_n else en[:0]
        assert np.array_equal(gm, em) and np.array_equal(gn, en), (n, w)
