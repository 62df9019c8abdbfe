"""Pins of the CPU oracle against what the paper and the mathematics fix.

No test here re-types the oracle's loops.  Each check comes from somewhere
else: the comparison bounds of Propositions 2-4, closed forms on monotone
input, the characterisation of a maximum (an upper bound that is a member of
the window), library reductions (numpy max/min/accumulate) for the degenerate
windows, the semigroup identity of sliding maxima, negation symmetry, chunk
invariance, and separability of the 2D filter (Section 1).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DTYPES = [np.float32, np.float64, np.int16, np.uint8]


def _facts():
    with open(os.path.join(GOLDEN, "paper_facts.json")) as f:
        return json.load(f)


def _windows(a, w):
    return np.lib.stride_tricks.sliding_window_view(a, w)


def _characterises(a, w, mx, mn):
    """max_j is >= every element of [j, j+w) and equal to one of them;
    likewise min_j (definition of Section 1 by characterisation)."""
    win = _windows(a, w)
    assert mx.shape == (a.size - w + 1,) and mn.shape == mx.shape
    assert (win <= mx[:, None]).all() and (win == mx[:, None]).any(axis=1).all()
    assert (win >= mn[:, None]).all() and (win == mn[:, None]).any(axis=1).all()


# ---------------------------------------------------------------- exhaustive

def test_exhaustive_permutations_wedge_equals_definition():
    """All permutations of n <= 7 and every w: Algorithm 1 equals the
    definition, uses <= 3n comparisons (Prop. 2) and keeps
    size(U)+size(L) <= w+1 (Prop. 4)."""
    f = _facts()
    for n in range(1, 8):
        for perm in itertools.permutations(range(n)):
            a = np.array(perm, dtype=np.float64)
            for w in range(1, n + 1):
                bmx, bmn = oracle.bf1d(a, w)
                wmx, wmn, st = oracle.wedge(a, w)
                assert np.array_equal(bmx, wmx) and np.array_equal(bmn, wmn), (perm, w)
                assert st["ncmp"] <= f["prop2_max_comparisons_per_element"] * n
                assert st["max_size"] <= w + f["prop4_wedge_size_excess_over_w"]
                assert st["stale_fronts"] == 0


def test_exhaustive_ternary_with_ties():
    """All {0,1,2}^n for n <= 8 (many ties): same three facts, plus the
    characterisation of each output."""
    f = _facts()
    for n in range(1, 9):
        for tup in itertools.product(range(3), repeat=n):
            a = np.array(tup, dtype=np.int16)
            for w in range(1, n + 1):
                bmx, bmn = oracle.bf1d(a, w)
                wmx, wmn, st = oracle.wedge(a, w)
                assert np.array_equal(bmx, wmx) and np.array_equal(bmn, wmn)
                assert st["ncmp"] <= f["prop2_max_comparisons_per_element"] * n
                assert st["max_size"] <= w + f["prop4_wedge_size_excess_over_w"]
                assert st["stale_fronts"] == 0
            _characterises(a, 2 if n >= 2 else 1, *oracle.bf1d(a, 2 if n >= 2 else 1))


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("decreasing", [False, True])
def test_monotone_closed_form(dtype, decreasing):
    """On non-decreasing input the window max is its last element and the min
    its first (reversed on non-increasing input).  With ties, Algorithm 1
    stays within the general 3n bound of Prop. 2."""
    n = 5000
    a = synth.monotone(n, seed=7, dtype=dtype, decreasing=decreasing)
    for w in (1, 2, 3, 17, 101, n):
        mx, mn = oracle.bf1d(a, w)
        first, last = a[: n - w + 1], a[w - 1:]
        if decreasing:
            assert np.array_equal(mx, first) and np.array_equal(mn, last)
        else:
            assert np.array_equal(mx, last) and np.array_equal(mn, first)
        wmx, wmn, st = oracle.wedge(a, w)
        assert np.array_equal(wmx, mx) and np.array_equal(wmn, mn)
        assert st["ncmp"] <= 3 * n


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("decreasing", [False, True])
def test_prop3_strictly_monotone_two_comparisons(dtype, decreasing):
    """Prop. 3: on monotonic data the while-loop conditions are never true,
    so at most 2 comparisons per element.  The proof's claim holds for
    strictly monotone input (reading: ties are excluded, see next test)."""
    f = _facts()
    n = 250 if dtype == np.uint8 else 5000
    a = np.arange(n, dtype=np.float64)
    a = (a[::-1] if decreasing else a).astype(dtype)
    for w in (1, 2, 3, 17, 101, n):
        _, _, st = oracle.wedge(a, w)
        assert st["ncmp"] <= f["prop3_max_comparisons_per_element_monotone"] * n


def test_prop3_ties_can_exceed_two_comparisons():
    """Non-decreasing input with long runs of ties: each tie keeps its index
    in U, and the next strict rise pops them with true while-comparisons,
    so the count exceeds 2n (still <= 3n by Prop. 2)."""
    a = np.repeat(np.arange(50, dtype=np.float64), 40)
    _, _, st = oracle.wedge(a, 101)
    assert 2 * a.size < st["ncmp"] <= 3 * a.size


@pytest.mark.parametrize("dtype", DTYPES)
def test_degenerate_windows_against_library(dtype):
    a = synth.random_walk(3001, 11, dtype)
    mx, mn = oracle.bf1d(a, 1)
    assert np.array_equal(mx, a) and np.array_equal(mn, a)           # w = 1
    mx, mn = oracle.bf1d(a, a.size)
    assert mx.tolist() == [a.max()] and mn.tolist() == [a.min()]     # w = n
    mx, mn = oracle.bf1d(a, a.size + 1)
    assert mx.size == 0 and mn.size == 0                             # w > n
    c = np.full(257, a[5], dtype)
    for w in (1, 4, 257):
        mx, mn = oracle.bf1d(c, w)
        assert (mx == a[5]).all() and (mn == a[5]).all()


def test_empty_and_invalid():
    e = np.empty(0, np.float32)
    mx, mn = oracle.bf1d(e, 3)
    assert mx.size == 0
    mx, mn, st = oracle.wedge(e, 3)
    assert mx.size == 0 and st["ncmp"] == 0
    with pytest.raises(ValueError):
        oracle.bf1d(np.zeros(4, np.float32), 0)


# ------------------------------------------------- characterisation & identities

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dist", synth.DISTS)
def test_characterisation_random(dtype, dist):
    a = synth.by_name(dist, 4000, 5, dtype)
    for w in (2, 3, 31, 257, 1001):
        mx, mn = oracle.bf1d(a, w)
        _characterises(a, w, mx, mn)
        wmx, wmn, st = oracle.wedge(a, w)
        assert np.array_equal(wmx, mx) and np.array_equal(wmn, mn)
        assert st["ncmp"] <= 3 * a.size and st["max_size"] <= w + 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_negation_symmetry(dtype):
    """max-filter(a) = -min-filter(-a), bitwise (negation is exact)."""
    a = synth.random_walk(5000, 13, dtype)
    for w in (3, 64, 999):
        mx, mn = oracle.bf1d(a, w)
        nmx, nmn = oracle.bf1d(-a, w)
        assert np.array_equal(mx, -nmn) and np.array_equal(mn, -nmx)


@pytest.mark.parametrize("dtype", DTYPES)
def test_semigroup_composition(dtype):
    """Sliding max over w2 of sliding max over w1 = sliding max over w1+w2-1."""
    a = synth.uniform(6000, 17, dtype)
    for w1, w2 in ((3, 5), (16, 17), (100, 901), (1, 7)):
        m1, n1 = oracle.bf1d(a, w1)
        m12, _ = oracle.bf1d(m1, w2)
        _, n12 = oracle.bf1d(n1, w2)
        m, n = oracle.bf1d(a, w1 + w2 - 1)
        assert np.array_equal(m12, m) and np.array_equal(n12, n)


@pytest.mark.parametrize("dtype", DTYPES)
def test_chunk_invariance(dtype):
    """Filtering any chunk with a w-1 halo gives the same outputs (each
    output depends only on its own window)."""
    a = synth.piecewise_monotone(20000, 19, dtype)
    w = 333
    mx, mn = oracle.bf1d(a, w)
    cuts = [0, 1, 500, 4096, 7777, 19000, a.size - w + 1]
    for s, e in zip(cuts[:-1], cuts[1:]):
        cmx, cmn, _ = oracle.wedge(a[s:e + w - 1], w)
        assert np.array_equal(cmx, mx[s:e]) and np.array_equal(cmn, mn[s:e])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("threads", [1, 2, 3, 7, 64])
def test_wedge_mt_equals_definition(dtype, threads):
    """The threaded chunk+halo wedge (the timed CPU baseline) against the
    definition, with thread counts that leave ragged and empty ranges."""
    for n, w in ((20011, 1), (20011, 2), (20011, 101), (300, 250), (50, 50), (10, 20)):
        a = synth.random_walk(n, n + w, dtype)
        mx, mn = oracle.bf1d(a, w)
        tmx, tmn, used = oracle.wedge_mt(a, w, threads)
        assert used >= 1
        assert np.array_equal(tmx, mx) and np.array_equal(tmn, mn)


@pytest.mark.parametrize("dtype", DTYPES)
def test_sampled_equals_full(dtype):
    a = synth.random_walk(10000, 23, dtype)
    w = 777
    mx, mn = oracle.bf1d(a, w)
    starts = np.random.default_rng(1).integers(0, a.size - w + 1, size=500)
    smx, smn = oracle.bf1d_at(a, w, starts)
    assert np.array_equal(smx, mx[starts]) and np.array_equal(smn, mn[starts])


def test_sine_wave_is_cheap_for_the_wedge():
    """The paper's sine input (period 10 000) is piecewise monotone, so the
    wedge makes close to 2 comparisons per element (Section 5 explains its
    2x speed-up there by Prop. 3)."""
    a = synth.sine(200000)
    _, _, st = oracle.wedge(a, 1000)
    assert st["ncmp"] <= 2.01 * a.size
    r = synth.uniform(200000, 1, np.float64)
    _, _, st_r = oracle.wedge(r, 1000)
    assert st_r["ncmp"] > st["ncmp"]


# ----------------------------------------------------------------- envelope

@pytest.mark.parametrize("dtype", DTYPES)
def test_envelope_pins(dtype):
    a = synth.random_walk(3000, 29, dtype)
    n = a.size
    for r in (0, 1, 51, 400):
        up, lo = oracle.envelope(a, r)
        if r == 0:
            assert np.array_equal(up, a) and np.array_equal(lo, a)
            continue
        mx, mn = oracle.bf1d(a, 2 * r + 1)
        # interior: centred window = the valid window starting at i - r
        assert np.array_equal(up[r:n - r], mx) and np.array_equal(lo[r:n - r], mn)
        # left end: clipped window [0, i + r] is a prefix -> running max
        assert np.array_equal(up[:r], np.maximum.accumulate(a)[r:2 * r])
        assert np.array_equal(lo[:r], np.minimum.accumulate(a)[r:2 * r])
        # right end: suffix maxima
        sfx_max = np.maximum.accumulate(a[::-1])[::-1]
        sfx_min = np.minimum.accumulate(a[::-1])[::-1]
        assert np.array_equal(up[n - r:], sfx_max[n - 2 * r:n - r])
        assert np.array_equal(lo[n - r:], sfx_min[n - 2 * r:n - r])
    up, lo = oracle.envelope(a, n + 5)
    assert (up == a.max()).all() and (lo == a.min()).all()


# ----------------------------------------------------------------------- 2D

@pytest.mark.parametrize("dtype", [np.float32, np.uint8])
def test_2d_separable_and_reductions(dtype):
    """Section 1: the 2D filter is the 1D filter on rows then on columns.
    The oracle's literal rectangle must equal both orders of separation,
    and reduce to the 1D filter for 1-wide windows."""
    img = synth.blobs2d(1, 57, 71, 41, dtype, nblobs=12)[0]
    for wy, wx in ((3, 3), (5, 9), (1, 7), (6, 1), (57, 71)):
        mx, mn = oracle.bf2d(img, wy, wx)
        rmx = np.stack([oracle.bf1d(row, wx)[0] for row in img])
        rmn = np.stack([oracle.bf1d(row, wx)[1] for row in img])
        cmx = np.stack([oracle.bf1d(col, wy)[0] for col in rmx.T]).T
        cmn = np.stack([oracle.bf1d(col, wy)[1] for col in rmn.T]).T
        assert np.array_equal(mx, cmx) and np.array_equal(mn, cmn)
        c2mx = np.stack([oracle.bf1d(col, wy)[0] for col in img.T]).T
        r2mx = np.stack([oracle.bf1d(row, wx)[0] for row in c2mx])
        assert np.array_equal(mx, r2mx)
        if (wy, wx) == (57, 71):
            assert mx.item() == img.max() and mn.item() == img.min()
        ys = np.random.default_rng(2).integers(0, img.shape[0] - wy + 1, 50)
        xs = np.random.default_rng(3).integers(0, img.shape[1] - wx + 1, 50)
        smx, smn = oracle.bf2d_at(img, wy, wx, ys, xs)
        assert np.array_equal(smx, mx[ys, xs]) and np.array_equal(smn, mn[ys, xs])


def test_stream_reference_is_concatenation():
    a = synth.random_walk(5000, 31)
    chunks = np.split(a, [3, 100, 2500, 2501])
    mx, mn = oracle.stream_reference(chunks, 64)
    bmx, bmn = oracle.bf1d(a, 64)
    assert np.array_equal(mx, bmx) and np.array_equal(mn, bmn)


# ------------------------------------------------ envelope lower bound (DTW)

def test_lb_keogh_worked_example():
    """Hand-computed: series c = (1, 1, 1), query q = (0, 5, 0), r = 1.  The
    envelope of c is U = L = (1, 1, 1); q leaves it by 1, 4 and 1, so the
    bound is sqrt(1 + 16 + 1).  With the roles swapped (the envelope of q,
    U = (5, 5, 5), L = (0, 0, 0)) every c_i lies inside and the bound is 0:
    the envelope belongs to the series, the excursions to the query."""
    c = np.array([1, 1, 1], np.float64)
    q = np.array([0, 5, 0], np.float64)
    assert oracle.lb_keogh(c, q, 1) == np.sqrt(18.0)
    assert oracle.lb_keogh(q, c, 1) == 0.0


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
def test_lb_keogh_radius_zero_is_euclidean(dtype):
    """r = 0: the envelope is the series itself, so the bound is the plain
    Euclidean distance (a textbook formula, computed here with numpy)."""
    for n in (1, 2, 17, 300):
        c = synth.uniform(n, seed=n, dtype=dtype)
        q = synth.uniform(n, seed=n + 1, dtype=dtype)
        e = np.sqrt(((q.astype(np.float64) - c.astype(np.float64)) ** 2).sum())
        assert abs(oracle.lb_keogh(c, q, 0) - e) <= 1e-12 * max(1.0, e)
        assert abs(oracle.dtw_band(q, c, 0) - e) <= 1e-12 * max(1.0, e)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16])
def test_lb_keogh_below_banded_dtw(dtype):
    """The bound never exceeds the time-warping distance with the same band
    (brute-force dynamic programming on small series), for any radius; the
    banded distance only falls as the band widens, and a query inside the
    envelope (the series itself, or halfway between U and L) gives 0."""
    for seed in range(12):
        n = 5 + 7 * seed
        c = synth.random_walk(n, seed=seed, dtype=dtype)
        q = synth.random_walk(n, seed=100 + seed, dtype=dtype)
        prev = None
        for r in (0, 1, 2, 4, n):
            lb = oracle.lb_keogh(c, q, r)
            d = oracle.dtw_band(q, c, r)
            assert lb <= d * (1 + 1e-12) + 1e-12
            if prev is not None:
                assert d <= prev * (1 + 1e-12) + 1e-12
            prev = d
            assert oracle.lb_keogh(c, c, r) == 0.0
            up, lo = oracle.envelope(c, r)
            mid = ((up.astype(np.float64) + lo.astype(np.float64)) / 2).astype(dtype)
            assert oracle.lb_keogh(c, mid, r) == 0.0


def test_lb_keogh_is_monotone_in_radius():
    """A wider radius widens the envelope, so the bound can only fall."""
    c = synth.random_walk(400, seed=5, dtype=np.float64)
    q = synth.random_walk(400, seed=6, dtype=np.float64)
    vals = [oracle.lb_keogh(c, q, r) for r in (0, 1, 3, 10, 50, 399)]
    assert all(b <= a for a, b in zip(vals, vals[1:]))
    assert vals[0] > vals[-1] >= 0.0


# ------------------------------------------------ window 3, 2 comparisons

@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
def test_w3_two_comparisons_per_element(dtype):
    """The proposition after Section 3's lower bound: w = 3 needs at most 2
    comparisons per element with zero latency.  The oracle's version agrees
    with the definition on every input (uint8 data is full of ties, and the
    exhaustive part covers every order of up to 6 elements over 3 values),
    and its count is exactly 2n - 3 <= 2n."""
    for n in (0, 1, 2, 3, 4, 17, 10_000):
        a = synth.uniform(n, seed=n, dtype=dtype) if n else np.zeros(0, dtype)
        mx, mn, c = oracle.w3(a)
        emx, emn = oracle.bf1d(a, 3)
        assert np.array_equal(mx, emx) and np.array_equal(mn, emn)
        assert c == (2 * n - 3 if n >= 3 else 0) and c <= 2 * n
    for n in range(3, 7):
        for t in itertools.product(range(3), repeat=n):
            a = np.array(t, dtype)
            mx, mn, _ = oracle.w3(a)
            emx, emn = oracle.bf1d(a, 3)
            assert np.array_equal(mx, emx) and np.array_equal(mn, emn)


# --------------------------------------------------- arg-max / arg-min

@pytest.mark.parametrize("dtype", [np.float32, np.int16, np.uint8])
def test_argbf1d_leftmost_extreme(dtype):
    """Every location holds the window's extreme value (the definition's max
    and min), lies inside the window, and no earlier position of the window
    holds the same value (leftmost rule), checked with numpy independently
    of the oracle's loop; a constant array gives the window starts."""
    a = synth.uniform(3000, seed=8, dtype=dtype)
    if dtype == np.uint8:
        a = (a // 16).astype(np.uint8)  # long runs of ties
    for w in (1, 2, 3, 7, 64):
        imx, imn = oracle.argbf1d(a, w)
        mx, mn = oracle.bf1d(a, w)
        j = np.arange(imx.size)
        assert ((imx >= j) & (imx < j + w)).all() and ((imn >= j) & (imn < j + w)).all()
        assert np.array_equal(a[imx], mx) and np.array_equal(a[imn], mn)
        for k in range(0, imx.size, 97):
            win = a[k:k + w]
            assert imx[k] == k + int(np.argmax(win)) and imn[k] == k + int(np.argmin(win))
    c = np.full(50, 7, dtype)
    imx, imn = oracle.argbf1d(c, 5)
    assert np.array_equal(imx, np.arange(46)) and np.array_equal(imn, np.arange(46))


EXHAUSTIVE_C = r"""
#include <stdint.h>
#include <stdio.h>
#include <string.h>
typedef struct { int64_t ncmp, max_size, stale_fronts, steps; } orc_wedge_stats;
int oracle_bf1d_f64(const double *, int64_t, int64_t, double *, double *);
int oracle_wedge_f64(const double *, int64_t, int64_t, double *, double *, orc_wedge_stats *);
int oracle_argbf1d_f64(const double *, int64_t, int64_t, int64_t *, int64_t *);
int oracle_w3_f64(const double *, int64_t, double *, double *, int64_t *);

static long checked = 0;
static int check(const double *a, int n) {
    double bm[16], bn[16], wm[16], wn[16], tm[16], tn[16];
    int64_t im[16], in[16], c;
    for (int w = 1; w <= n; ++w) {
        orc_wedge_stats st;
        if (oracle_bf1d_f64(a, n, w, bm, bn) || oracle_wedge_f64(a, n, w, wm, wn, &st) ||
            oracle_argbf1d_f64(a, n, w, im, in)) return 1;
        for (int j = 0; j + w <= n; ++j) {
            if (wm[j] != bm[j] || wn[j] != bn[j]) return 2;
            if (im[j] < j || im[j] >= j + w || a[im[j]] != bm[j]) return 3;
            if (in[j] < j || in[j] >= j + w || a[in[j]] != bn[j]) return 3;
            for (int k = j; k < im[j]; ++k) if (a[k] == bm[j]) return 4;  /* leftmost */
            for (int k = j; k < in[j]; ++k) if (a[k] == bn[j]) return 4;
        }
        if (st.ncmp > 3 * n || st.max_size > w + 1 || st.stale_fronts != 0) return 5;
        ++checked;
    }
    if (n >= 3) {
        if (oracle_w3_f64(a, n, tm, tn, &c) || c != 2 * n - 3) return 6;
        oracle_bf1d_f64(a, n, 3, bm, bn);
        for (int j = 0; j + 3 <= n; ++j) if (tm[j] != bm[j] || tn[j] != bn[j]) return 7;
    }
    return 0;
}

int main(void) {
    double a[16];
    for (int n = 1; n <= 8; ++n) {       /* every permutation of 0..n-1 */
        int p[16];
        for (int i = 0; i < n; ++i) p[i] = i;
        for (;;) {
            for (int i = 0; i < n; ++i) a[i] = p[i];
            int r = check(a, n);
            if (r) { printf("perm fail %d n=%d\n", r, n); return r; }
            int i = n - 2;
            while (i >= 0 && p[i] > p[i + 1]) --i;
            if (i < 0) break;
            int j = n - 1;
            while (p[j] < p[i]) --j;
            int t = p[i]; p[i] = p[j]; p[j] = t;
            for (int l = i + 1, h = n - 1; l < h; ++l, --h) { t = p[l]; p[l] = p[h]; p[h] = t; }
        }
    }
    for (int n = 1; n <= 10; ++n) {      /* every array over {0, 1, 2} */
        long total = 1;
        for (int i = 0; i < n; ++i) total *= 3;
        for (long c = 0; c < total; ++c) {
            long v = c;
            for (int i = 0; i < n; ++i) { a[i] = (double)(v % 3); v /= 3; }
            int r = check(a, n);
            if (r) { printf("ternary fail %d n=%d\n", r, n); return r; }
        }
    }
    printf("ok %ld\n", checked);
    return 0;
}
"""


def test_exhaustive_permutations_8_and_ternary_10_in_c(tmp_path):
    """Every permutation of up to 8 elements and every array of up to 10
    elements over {0, 1, 2}, every window: Algorithm 1 equals the definition
    with <= 3n comparisons (Prop. 2), size(U)+size(L) <= w+1 (Prop. 4) and no
    step with both fronts stale; the arg filter's positions hold the extremes
    and are the leftmost; the window-3 scheme equals the definition in
    exactly 2n-3 comparisons.  Run as a C program over the oracle's source
    (the sizes are too many calls for Python)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    drv = tmp_path / "exhaustive.c"
    drv.write_text(EXHAUSTIVE_C)
    exe = tmp_path / "exhaustive"
    src = os.path.join(os.path.dirname(oracle.__file__), "mmf_oracle.c")
    subprocess.run(["gcc", "-O2", "-std=c99", str(drv), src, "-lm", "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
