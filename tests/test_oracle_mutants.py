"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/mmf_oracle.c``, plants one plausible mistake (a
short window, a flipped comparison, a wrong deque end, an off-by-one expiry,
a clipped envelope, a short rectangle; for the arg filter a rightmost tie
rule or a short window; for the window-3 scheme swapped branches, a stale
order or a wrong count; for the envelope bound a missing side, the wrong
envelope side or a missing square root; for the banded warping distance a
missing diagonal step or a band one too wide), compiles the copy with gcc
into a temporary library, and runs pin checks against it: a compact set
here and, for the later functions, the pins of ``test_oracle`` themselves.
At least one pin must fail for every mutant.  The real oracle is untouched.
"""
import contextlib
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "mmf_oracle.c")

MUTANTS = {
    "bf1d_short_window": ("for (int64_t i = j + 1; i < j + w; ++i) {",
                          "for (int64_t i = j + 1; i < j + w - 1; ++i) {"),
    "bf1d_flipped_max": ("if (a[i] > hi) hi = a[i];", "if (a[i] < hi) hi = a[i];"),
    "wedge_back_not_front": ("if (mx) mx[i - w] = a[dq_front(&U)];",
                             "if (mx) mx[i - w] = a[dq_back(&U)];"),
    "wedge_late_expiry": ("int u_stale = dq_front(&U) == i - w;",
                          "int u_stale = dq_front(&U) == i - w - 1;"),
    "wedge_wrong_side": ("if (a[i] > a[i - 1]) {", "if (a[i] < a[i - 1]) {"),
    "envelope_short_right": ("int64_t e = i + r > n - 1 ? n - 1 : i + r;",
                             "int64_t e = i + r > n - 1 ? n - 1 : i + r - 1;"),
    "bf2d_short_rows": ("for (int64_t dy = 0; dy < wy; ++dy)",
                        "for (int64_t dy = 0; dy < wy - 1; ++dy)"),
    "argbf1d_rightmost": ("if (a[k] > a[bx]) bx = k;", "if (a[k] >= a[bx]) bx = k;"),
    "argbf1d_short_window": ("for (int64_t k = j + 1; k < j + w; ++k) {",
                             "for (int64_t k = j + 1; k < j + w - 1; ++k) {"),
    "w3_branches_swapped": ("if (older_greater) {", "if (!older_greater) {"),
    "w3_stale_order": ("older_greater = prev_gt;", "older_greater = older_gt;"),
    "w3_count": ("c += 2;", "c += 3;"),
    "lb_no_lower_side": ("else if (qi < (double)lw)", "else if (0 && qi < (double)lw)"),
    "lb_wrong_envelope_side": ("if (qi > (double)hi) sum += (qi - (double)hi) * (qi - (double)hi);",
                               "if (qi > (double)lw) sum += (qi - (double)lw) * (qi - (double)lw);"),
    "lb_no_sqrt": ("*out = sqrt(sum);", "*out = sum;"),
    "dtw_no_diagonal": ("if (i > 0 && j > 0 && D[(i - 1) * n + j - 1] < best)",
                        "if (0 && i > 0 && j > 0 && D[(i - 1) * n + j - 1] < best)"),
    "dtw_band_too_wide": ("if (i - j > r || j - i > r)", "if (i - j > r + 1 || j - i > r + 1)"),
}

FUNCS = ("bf1d", "bf1d_at", "wedge", "envelope", "bf2d", "bf2d_at", "argbf1d", "w3", "lb_keogh", "dtw_band")


@contextlib.contextmanager
def _mutant_lib(find, repl):
    src = open(SRC).read()
    assert find in src, find
    mutated = src.replace(find, repl, 1)  # the first occurrence
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "m.so")
        open(c, "w").write(mutated)
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-w", "-o", so, c, "-lm"])
        real = oracle._load()
        lib = ctypes.CDLL(so)
        for suf in ("f32", "f64", "i16", "u8"):
            for fn in FUNCS:
                f = getattr(lib, f"oracle_{fn}_{suf}")
                g = getattr(real, f"oracle_{fn}_{suf}")
                f.argtypes, f.restype = g.argtypes, g.restype
        oracle._lib = lib
        try:
            yield
        finally:
            oracle._lib = real


def _pins_hold() -> bool:
    """A compact run of the oracle pins; False as soon as one fails."""
    try:
        a = synth.monotone(600, 7, np.float32)
        for w in (3, 17):
            mx, mn = oracle.bf1d(a, w)
            if not (np.array_equal(mx, a[w - 1:]) and np.array_equal(mn, a[: a.size - w + 1])):
                return False
        r = synth.random_walk(700, 5, np.float64)
        for w in (2, 5, 31):
            mx, mn = oracle.bf1d(r, w)
            win = np.lib.stride_tricks.sliding_window_view(r, w)
            if not ((win <= mx[:, None]).all() and (win == mx[:, None]).any(1).all()
                    and (win >= mn[:, None]).all() and (win == mn[:, None]).any(1).all()):
                return False
            wmx, wmn, st = oracle.wedge(r, w)
            if not (np.array_equal(wmx, mx) and np.array_equal(wmn, mn)):
                return False
            if st["ncmp"] > 3 * r.size or st["max_size"] > w + 1:
                return False
        for rr in (1, 7):
            up, lo = oracle.envelope(r, rr)
            mx, mn = oracle.bf1d(r, 2 * rr + 1)
            n = r.size
            if not (np.array_equal(up[rr:n - rr], mx) and
                    np.array_equal(up[n - rr:], np.maximum.accumulate(r[::-1])[::-1][n - 2 * rr:n - rr])):
                return False
        img = synth.blobs2d(1, 20, 23, 1, np.float32, nblobs=4)[0]
        mx, _ = oracle.bf2d(img, 3, 4)
        rows = np.stack([oracle.bf1d(row, 4)[0] for row in img])
        sep = np.stack([oracle.bf1d(col, 3)[0] for col in rows.T]).T
        if not np.array_equal(mx, sep):
            return False
    except (ValueError, AssertionError):
        return False
    return True


def _paper_pins_hold() -> bool:
    """The pins of test_oracle for the arg filter, the window-3 scheme, the
    envelope bound and the banded warping distance."""
    import test_oracle as t
    try:
        for dt in (np.float32, np.uint8):
            t.test_argbf1d_leftmost_extreme(dt)
            t.test_w3_two_comparisons_per_element(dt)
        t.test_lb_keogh_worked_example()
        t.test_lb_keogh_radius_zero_is_euclidean(np.float64)
        t.test_lb_keogh_below_banded_dtw(np.float64)
        t.test_lb_keogh_is_monotone_in_radius()
    except (ValueError, AssertionError):
        return False
    return True


def test_real_oracle_passes_compact_pins():
    assert _pins_hold()
    assert _paper_pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    find, repl = MUTANTS[name]
    with _mutant_lib(find, repl):
        assert not (_pins_hold() and _paper_pins_hold()), f"planted mistake {name} went unnoticed"
