"""CPU model of the 2D filter's column pass for windows of 10 rows or more,
checked against the oracle's 1D definition down one column.

The column pass (Section 1: the 2D filter is the 1D filter on rows, then on
columns) streams a column in tiles of 8 rows.  With s = wy-1 = 8q + r, the
window of row j = 8c + i ends at k = j + s in tile c+q (near) or c+q+1 (far)
and its extreme is op(suffix of tile c from row i, the tiles strictly
between, prefix of k's tile up to k): van Herk/Gil-Werman blocks of 8 rows
(Section 2, Table 1).  Prefixes of the last two K tiles sit in a 2-slot ring;
the aggregates of tiles c+1..c+q-1 are a two-stack queue inside a ring of
q+2 tile aggregates (older part as suffix extremes rebuilt in place, newer
part raw with a running extreme), and the far case adds tile c+q.  Rows
outside the image read as identities.  The model keeps the kernel's order of
ring writes and reads, so a ring too small for it, a queue that misses its
slide or rebuild, or a wrong near/far choice fails against the oracle."""
import numpy as np

import oracle
import synth

ROWS = 8


def _column_blocks(col, wy, op, ident):
    H = len(col)
    Ho = H - wy + 1
    s = wy - 1
    q, rr = s >> 3, s & 7
    qcap = q + 2
    assert q >= 1

    def tile(y0):
        return [col[y] if 0 <= y < H else ident for y in range(y0, y0 + ROWS)]

    rp = [[None] * ROWS for _ in range(2)]  # prefixes of the last two K tiles
    ta = [None] * qcap                       # tile aggregates (ring)

    def k_tile(x, v):
        for r in range(1, ROWS):
            v[r] = op(v[r - 1], v[r])
        rp[x & 1] = list(v)
        ta[x % qcap] = v[-1]

    for x in range(1, q + 1):
        k_tile(x, tile(x * ROWS))
    NC = -(-Ho // ROWS)
    fs = fe = be = 1
    b = ident

    def push(x):
        nonlocal b, be
        b = op(b, ta[x % qcap])
        be = x + 1

    if q >= 2:
        for x in range(1, q):
            push(x)
    out = []
    for c in range(NC):
        if c > 0 and q >= 2:
            fs += 1
            push(c + q - 1)
            if fs >= fe:
                m = ident
                for x in range(be - 1, fs - 1, -1):
                    m = op(m, ta[x % qcap])
                    ta[x % qcap] = m
                b = ident
                fe = be
        j = tile(c * ROWS)
        k_tile(c + q + 1, tile((c + q + 1) * ROWS))
        for r in range(ROWS - 2, -1, -1):
            j[r] = op(j[r + 1], j[r])
        near = op(b, ta[fs % qcap]) if fs < fe else b
        far = op(near, ta[(c + q) % qcap])
        for i in range(ROWS):
            kr = i + rr
            is_far = kr >= ROWS
            pk = rp[(c + q + (1 if is_far else 0)) & 1][kr & 7]
            out.append(op(op(j[i], far if is_far else near), pk))
    return np.asarray(out[:Ho])


def test_column_pass_matches_the_definition():
    rng = np.random.default_rng(5)
    for wy in list(range(10, 40)) + [63, 64, 65, 100, 127, 255]:
        for _ in range(3):
            H = int(rng.integers(wy, wy + 150))
            col = synth.random_walk(H, seed=int(rng.integers(1 << 30)), dtype=np.float32).astype(np.float64)
            if rng.random() < 0.4:
                col = rng.integers(0, 3, size=H).astype(np.float64)  # ties
            em, en = oracle.bf1d(col, wy)
            gm = _column_blocks(col, wy, max, -np.inf)
            gn = _column_blocks(col, wy, min, np.inf)
            assert np.array_equal(gm, em) and np.array_equal(gn, en), (wy, H)


def test_row_pass_as_one_series_over_stacked_rows():
    """The two-pass 2D filter's row pass reads all rows of all images as one
    series (rows `pitch` apart, images stacked): the 1D window starting at
    stream position r*pitch + x is row r's window at column x for x < W-wx+1;
    windows past that straddle two rows or a row's padding and are not used.
    Checked with the oracle's own 1D and 2D definitions, padding filled with
    extreme values so that a window reaching into it would show."""
    rng = np.random.default_rng(9)
    for nimg, H, W, pitch, wx in ((2, 5, 17, 17, 4), (3, 4, 20, 23, 7), (1, 6, 9, 16, 9), (2, 3, 33, 40, 1),
                                  (1, 1, 12, 12, 12)):
        imgs = synth.random_walk(nimg * H * W, seed=wx + W, dtype=np.float32).reshape(nimg, H, W)
        buf = np.empty((nimg * H, pitch), np.float32)
        buf[:, W:] = rng.choice([-1e30, 1e30], size=(nimg * H, pitch - W))
        buf[:, :W] = imgs.reshape(nimg * H, W)
        stream = buf.reshape(-1)[:(nimg * H - 1) * pitch + W]
        smax, smin = oracle.bf1d(stream, wx)
        Wo = W - wx + 1
        for k in range(nimg):
            em, en = oracle.bf2d(imgs[k], 1, wx)
            for y in range(H):
                r = k * H + y
                assert np.array_equal(smax[r * pitch:r * pitch + Wo], em[y]), (nimg, H, W, pitch, wx, k, y)
                assert np.array_equal(smin[r * pitch:r * pitch + Wo], en[y]), (nimg, H, W, pitch, wx, k, y)
