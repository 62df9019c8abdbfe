"""CPU model of the fused 2D tile kernel (windows up to 31 x 31), checked
against the oracle's literal rectangle maximum and minimum.

Per output tile of 32 x 128 pixels the kernel reads the input tile with its
halo, (32 + wy - 1) x (128 + wx - 1) elements, with 0 at positions outside the
image (they only feed outputs outside it, which are not stored).  The row
pass gives each thread runs of 8 outputs of one row from 8 + 2*P2 values
(P2 the largest power of two <= wx): doubling passes p = 1, 2, .., P2/2
leave value i as the extreme of [i, i + P2), and the window of P2 + r
elements is the union of values i and i + r (Table 1's naive windows shared
between neighbours).  The column pass does the same down runs of 8 rows of
the row-pass tiles.  This model runs those steps with the kernel's run
lengths, in-place doubling order, zero padding and store bounds, on ragged
images of several tiles, for every window of up to 31 in each direction
(a sample of pairs) and checks every stored pixel."""
import numpy as np
import pytest

import oracle

TR, TC, RUN = 32, 128, 8


def pow2_floor(w):
    return 16 if w >= 16 else 8 if w >= 8 else 4 if w >= 4 else 2 if w >= 2 else 1


def run_windows(vals, w, op):
    """vals: (..., RUN + 2*P2) values of runs; returns (..., RUN) extremes of
    windows of w, in the kernel's order (in-place doubling, then the union)."""
    P2 = pow2_floor(w)
    r = w - P2
    a = vals.copy()
    NE = a.shape[-1]
    assert NE == RUN + 2 * P2
    p = 1
    while p < P2:
        for i in range(NE - p):  # increasing i: a[i + p] still holds the previous pass
            a[..., i] = op(a[..., i], a[..., i + p])
        p <<= 1
    return op(a[..., :RUN], a[..., r:r + RUN])


def tile_model(img, wy, wx):
    H, W = img.shape
    Ho, Wo = H - wy + 1, W - wx + 1
    outs = [np.full((max(Ho, 0), max(Wo, 0)), np.nan) for _ in range(2)]
    if Ho <= 0 or Wo <= 0:
        return outs
    rows_in, cols_in = TR + wy - 1, TC + wx - 1
    NEx, NEy = RUN + 2 * pow2_floor(wx), RUN + 2 * pow2_floor(wy)
    for y0 in range(0, Ho, TR):
        for x0 in range(0, Wo, TC):
            X = np.zeros((rows_in, cols_in))
            ys, xs = min(rows_in, H - y0), min(cols_in, W - x0)
            X[:ys, :xs] = img[y0:y0 + ys, x0:x0 + xs]
            # row pass: runs of RUN outputs from NEx values (0 past cols_in)
            Xp = np.zeros((rows_in, TC + NEx))
            Xp[:, :cols_in] = X
            runs = np.stack([Xp[:, c0:c0 + NEx] for c0 in range(0, TC, RUN)], axis=1)  # (rows, runs, NEx)
            for side, op in ((0, np.maximum), (1, np.minimum)):
                R = run_windows(runs, wx, op).reshape(rows_in, TC)
                # column pass: runs of RUN rows from NEy values (0 past rows_in)
                Rp = np.zeros((TR + NEy, TC))
                Rp[:rows_in] = R
                cr = np.stack([Rp[r0:r0 + NEy].T for r0 in range(0, TR, RUN)], axis=0)  # (runs, cols, NEy)
                O = run_windows(cr, wy, op)  # (runs, cols, RUN)
                O = O.transpose(0, 2, 1).reshape(TR, TC)
                hy, hx = min(TR, Ho - y0), min(TC, Wo - x0)
                outs[side][y0:y0 + hy, x0:x0 + hx] = O[:hy, :hx]
    return outs


PAIRS = [(1, 1), (1, 2), (2, 1), (3, 3), (2, 31), (31, 2), (5, 7), (7, 5), (8, 8), (9, 15), (15, 16),
         (16, 17), (17, 30), (31, 31), (4, 23), (12, 1), (1, 29)]


@pytest.mark.parametrize("wy,wx", PAIRS)
def test_tile_model_matches_the_rectangle_definition(wy, wx):
    rng = np.random.default_rng(wy * 100 + wx)
    H = int(rng.integers(max(wy, 40), 90))   # two or three tile rows, ragged
    W = int(rng.integers(max(wx, 140), 300))  # two or three tile columns, ragged
    img = rng.integers(-5, 6, size=(H, W)).astype(np.float64)  # ties, both signs
    em, en = oracle.bf2d(img, wy, wx)
    gm, gn = tile_model(img, wy, wx)
    assert np.array_equal(gm, em) and np.array_equal(gn, en), (wy, wx, H, W)


def test_union_identity_for_every_window():
    """The window of P2 + r values is the union of two doubled values, for
    every w in 1..31 and every run position."""
    rng = np.random.default_rng(1)
    for w in range(1, 32):
        P2 = pow2_floor(w)
        vals = rng.standard_normal((50, RUN + 2 * P2))
        got = run_windows(vals, w, np.maximum)
        want = np.stack([vals[:, i:i + w].max(axis=1) for i in range(RUN)], axis=1)
        assert np.array_equal(got, want), w
