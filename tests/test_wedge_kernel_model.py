"""CPU model of the chunked-wedge kernel's per-thread loop, checked against
the oracle's definition (values) and its leftmost-position rule (arg form).

The kernel runs Algorithm 1 (Section 4) restated so that the newest index is
in both deques after every step: at step i, if a_i > a_{i-1} the back of U
(index i-1) is dominated and popped, then U's back while a_i is strictly
larger, and i joins both deques (symmetrically for L when a_i < a_{i-1}); the
fronts whose index is i - w leave the window.  For values, a_i = a_{i-1} may
take either branch and at most one front leaves per step.  The arg form
keeps ties: an input equal to its predecessor joins both deques without a
pop, so equal earlier indices stay at the fronts (the leftmost extreme), and
both fronts may leave at once.  Deques hold the low 16 bits of chunk-local
indices and values are read from a ring of the last vcap inputs (vcap a power
of two that divides 2^16); positions are rebuilt as i - ((i - front) mod
2^16).  Each thread starts at its chunk's first window and runs w-1 warm-up
steps.  This model keeps all of that (16-bit storage, ring reads, chunk
restarts) and checks every output on exhaustive small arrays, tied random
arrays and a chunk whose indices pass 2^16."""
import itertools

import numpy as np

import oracle

M16 = 0xFFFF


def _chunk(a, j0, cnt, w, arg):
    """Outputs j0 .. j0+cnt-1 as one kernel thread forms them."""
    if w == 1:
        vals = a[j0:j0 + cnt]
        return list(vals), list(vals), list(range(j0, j0 + cnt)), list(range(j0, j0 + cnt))
    vcap = 1
    while vcap < w + 16:
        vcap <<= 1
    ring = {}  # value ring: slot -> value (only the last vcap inputs are ever read)
    x = a[j0:j0 + cnt + w - 1]

    def val(b16):
        return ring[b16 & (vcap - 1)]

    for k in range(min(len(x), vcap)):
        ring[k & (vcap - 1)] = x[k]
    U, L = [0], [0]  # 16-bit indices, front first
    uf = lf = 0
    prev = x[0]
    omx, omn, amx, amn = [], [], [], []
    nbound = max(len(U), len(L))

    for i in range(1, cnt + w - 1):
        if i + 16 < len(x):  # the kernel stages inputs ahead of use within the ring
            ring[(i + 16) & (vcap - 1)] = x[i + 16]
        ring[i & (vcap - 1)] = x[i]
        ai = x[i]
        if arg and ai == prev:
            U.append(i & M16)
            L.append(i & M16)
        elif ai > prev:
            U.pop()
            while U and ai > val(U[-1]):
                U.pop()
            U.append(i & M16)
            if len(U) == 1:
                uf = i & M16
            L.append(i & M16)
        else:
            L.pop()
            while L and ai < val(L[-1]):
                L.pop()
            L.append(i & M16)
            if len(L) == 1:
                lf = i & M16
            U.append(i & M16)
        gone = (i - w) & M16
        expired_u = uf == gone
        if expired_u:
            U.pop(0)
            uf = U[0]
        if (arg or not expired_u) and lf == gone:
            L.pop(0)
            lf = L[0]
        prev = ai
        nbound = max(nbound, len(U), len(L))
        if i >= w - 1:
            omx.append(val(uf))
            omn.append(val(lf))
            amx.append(j0 + i - ((i - uf) & M16))
            amn.append(j0 + i - ((i - lf) & M16))
    assert nbound <= w + 1  # per deque (Proposition 4 bounds the sum without ties)
    return omx, omn, amx, amn


def _model(a, w, chunk, arg):
    n_out = len(a) - w + 1
    res = ([], [], [], [])
    for j0 in range(0, n_out, chunk):
        part = _chunk(a, j0, min(chunk, n_out - j0), w, arg)
        for acc, p in zip(res, part):
            acc.extend(p)
    return [np.asarray(r) for r in res]


def _check(a, w, chunk):
    em, en = oracle.bf1d(a, w)
    ix, inn = oracle.argbf1d(a, w)
    vm, vn, _, _ = _model(a, w, chunk, arg=False)
    assert np.array_equal(vm, em) and np.array_equal(vn, en), (a, w, chunk)
    gm, gn, am, an = _model(a, w, chunk, arg=True)
    assert np.array_equal(gm, em) and np.array_equal(gn, en), (a, w, chunk)
    assert np.array_equal(am, ix) and np.array_equal(an, inn), (a, w, chunk)


def test_exhaustive_ternary_every_window_and_chunk():
    for n in range(1, 8):
        for vals in itertools.product(range(3), repeat=n):
            a = np.asarray(vals, np.float32)
            for w in range(1, n + 1):
                for chunk in (1, 2, n):
                    _check(a, w, chunk)


def test_random_tied_arrays():
    rng = np.random.default_rng(8)
    for _ in range(60):
        n = int(rng.integers(20, 400))
        w = int(rng.integers(1, min(n, 60) + 1))
        a = rng.integers(0, 4, size=n).astype(np.int16)
        _check(a, w, int(rng.integers(1, 50)))


def test_chunk_indices_past_2_16():
    """One chunk of 70 000 outputs: ring indices wrap past 2^16 and the
    positions are rebuilt from their low 16 bits."""
    rng = np.random.default_rng(3)
    w = 496
    a = np.repeat(rng.integers(0, 50, size=(70_000 + w) // 7 + 1), 7)[:70_000 + w - 1].astype(np.float32)
    _check(a, w, 70_000)
