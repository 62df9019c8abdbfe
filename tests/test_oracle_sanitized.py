"""The oracle's C source built with AddressSanitizer and UndefinedBehavior-
Sanitizer and driven over exhaustive small inputs: every function, every
window, every element type, empty and degenerate sizes.  A buffer overrun, a
use of uninitialised deque slots through a bad index, a signed overflow or a
leak ends the run with a sanitizer report (non-zero exit).  The driver also
checks the relations that hold exactly at these sizes (Algorithm 1 and the
window-3 scheme equal the definition, the positions hold the extremes, the
centred envelope at radius 0 is the input), so a sanitized build that
computed something else would fail as well."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int64_t ncmp, max_size, stale_fronts, steps; } orc_wedge_stats;

#define DECL(SUF, T)                                                                          \
int oracle_bf1d_##SUF(const T *, int64_t, int64_t, T *, T *);                                 \
int oracle_bf1d_at_##SUF(const T *, int64_t, int64_t, const int64_t *, int64_t, T *, T *);    \
int oracle_wedge_##SUF(const T *, int64_t, int64_t, T *, T *, orc_wedge_stats *);             \
int oracle_envelope_##SUF(const T *, int64_t, int64_t, T *, T *);                             \
int oracle_bf2d_##SUF(const T *, int64_t, int64_t, int64_t, int64_t, int64_t, T *, T *);      \
int oracle_argbf1d_##SUF(const T *, int64_t, int64_t, int64_t *, int64_t *);                  \
int oracle_w3_##SUF(const T *, int64_t, T *, T *, int64_t *);                                 \
int oracle_lb_keogh_##SUF(const T *, const T *, int64_t, int64_t, double *);                  \
int oracle_dtw_band_##SUF(const T *, const T *, int64_t, int64_t, double *);

DECL(f32, float)
DECL(f64, double)
DECL(i16, int16_t)
DECL(u8, uint8_t)

static int fails = 0;
#define CHECK(c) do { if (!(c)) { fprintf(stderr, "check failed line %d\n", __LINE__); fails++; } } while (0)

/* Every array of length n over {0, 1, 2}, every window 1..n+1 (heap buffers
 * of exactly the needed size so that any overrun is caught). */
#define RUN(SUF, T)                                                                           \
static void run_##SUF(void) {                                                                 \
    for (int64_t n = 0; n <= 7; ++n) {                                                        \
        int64_t combos = 1;                                                                   \
        for (int64_t k = 0; k < n; ++k) combos *= 3;                                          \
        for (int64_t c = 0; c < combos; ++c) {                                                \
            T *a = (T *)malloc((size_t)(n ? n : 1) * sizeof(T));                              \
            int64_t v = c;                                                                    \
            for (int64_t k = 0; k < n; ++k) { a[k] = (T)(v % 3); v /= 3; }                    \
            for (int64_t w = 1; w <= n + 1; ++w) {                                            \
                int64_t m = n >= w ? n - w + 1 : 0;                                           \
                size_t mb = (size_t)(m ? m : 1);                                              \
                T *mx = (T *)malloc(mb * sizeof(T)), *mn = (T *)malloc(mb * sizeof(T));       \
                T *wx = (T *)malloc(mb * sizeof(T)), *wn = (T *)malloc(mb * sizeof(T));       \
                int64_t *ix = (int64_t *)malloc(mb * 8), *in = (int64_t *)malloc(mb * 8);     \
                orc_wedge_stats st;                                                           \
                CHECK(oracle_bf1d_##SUF(a, n, w, mx, mn) == 0);                               \
                CHECK(oracle_wedge_##SUF(a, n, w, wx, wn, &st) == 0);                         \
                CHECK(oracle_argbf1d_##SUF(a, n, w, ix, in) == 0);                            \
                for (int64_t j = 0; j < m; ++j) {                                             \
                    CHECK(wx[j] == mx[j] && wn[j] == mn[j]);                                  \
                    CHECK(ix[j] >= j && ix[j] < j + w && a[ix[j]] == mx[j]);                  \
                    CHECK(in[j] >= j && in[j] < j + w && a[in[j]] == mn[j]);                  \
                }                                                                             \
                CHECK(st.ncmp <= 3 * n && st.max_size <= w + 1 && st.stale_fronts == 0);      \
                if (m > 0) {                                                                  \
                    int64_t *starts = (int64_t *)malloc((size_t)m * 8);                       \
                    T *sx = (T *)malloc((size_t)m * sizeof(T)), *sn = (T *)malloc((size_t)m * sizeof(T)); \
                    for (int64_t j = 0; j < m; ++j) starts[j] = m - 1 - j;                    \
                    CHECK(oracle_bf1d_at_##SUF(a, n, w, starts, m, sx, sn) == 0);             \
                    for (int64_t j = 0; j < m; ++j) CHECK(sx[j] == mx[m - 1 - j] && sn[j] == mn[m - 1 - j]); \
                    free(starts); free(sx); free(sn);                                         \
                }                                                                             \
                if (w == 3) {                                                                 \
                    int64_t nc = 0;                                                           \
                    CHECK(oracle_w3_##SUF(a, n, wx, wn, &nc) == 0);                           \
                    for (int64_t j = 0; j < m; ++j) CHECK(wx[j] == mx[j] && wn[j] == mn[j]);  \
                    CHECK(n < 3 || nc == 2 * n - 3);                                          \
                }                                                                             \
                free(mx); free(mn); free(wx); free(wn); free(ix); free(in);                   \
            }                                                                                 \
            if (n > 0) {                                                                      \
                T *up = (T *)malloc((size_t)n * sizeof(T)), *lo = (T *)malloc((size_t)n * sizeof(T)); \
                for (int64_t r = 0; r <= n + 1; ++r) {                                        \
                    CHECK(oracle_envelope_##SUF(a, n, r, up, lo) == 0);                       \
                    for (int64_t i = 0; i < n; ++i) {                                         \
                        CHECK(lo[i] <= a[i] && a[i] <= up[i]);                                \
                        if (r == 0) CHECK(up[i] == a[i] && lo[i] == a[i]);                    \
                    }                                                                         \
                    double lb = -1.0, d = -1.0;                                               \
                    CHECK(oracle_lb_keogh_##SUF(a, a, n, r, &lb) == 0 && lb == 0.0);          \
                    CHECK(oracle_dtw_band_##SUF(a, a, n, r, &d) == 0 && d == 0.0);            \
                }                                                                             \
                free(up); free(lo);                                                           \
                /* the array as a 1 x n image and as an n x 1 image */                        \
                for (int64_t wv = 1; wv <= n; ++wv) {                                         \
                    int64_t m = n - wv + 1;                                                   \
                    T *px = (T *)malloc((size_t)m * sizeof(T)), *pn = (T *)malloc((size_t)m * sizeof(T)); \
                    T *qx = (T *)malloc((size_t)m * sizeof(T)), *qn = (T *)malloc((size_t)m * sizeof(T)); \
                    T *ex = (T *)malloc((size_t)m * sizeof(T)), *en = (T *)malloc((size_t)m * sizeof(T)); \
                    CHECK(oracle_bf2d_##SUF(a, 1, n, n, 1, wv, px, pn) == 0);                 \
                    CHECK(oracle_bf2d_##SUF(a, n, 1, 1, wv, 1, qx, qn) == 0);                 \
                    CHECK(oracle_bf1d_##SUF(a, n, wv, ex, en) == 0);                          \
                    for (int64_t j = 0; j < m; ++j)                                           \
                        CHECK(px[j] == ex[j] && pn[j] == en[j] && qx[j] == ex[j] && qn[j] == en[j]); \
                    free(px); free(pn); free(qx); free(qn); free(ex); free(en);               \
                }                                                                             \
            }                                                                                 \
            free(a);                                                                          \
        }                                                                                     \
    }                                                                                         \
    /* empty inputs and rejected arguments touch nothing */                                   \
    T dummy = 0;                                                                              \
    orc_wedge_stats st;                                                                       \
    CHECK(oracle_bf1d_##SUF(NULL, 0, 3, NULL, NULL) == 0);                                    \
    CHECK(oracle_wedge_##SUF(NULL, 0, 3, NULL, NULL, &st) == 0);                              \
    CHECK(oracle_bf1d_##SUF(&dummy, 1, 0, NULL, NULL) != 0);                                  \
    CHECK(oracle_wedge_##SUF(&dummy, -1, 3, NULL, NULL, &st) != 0);                           \
    CHECK(oracle_envelope_##SUF(&dummy, 1, -1, NULL, NULL) != 0);                             \
    CHECK(oracle_bf2d_##SUF(&dummy, 1, 1, 0, 1, 1, NULL, NULL) != 0);                         \
}

RUN(f32, float)
RUN(f64, double)
RUN(i16, int16_t)
RUN(u8, uint8_t)

int main(void) {
    run_f32();
    run_f64();
    run_i16();
    run_u8();
    if (fails) { fprintf(stderr, "%d checks failed\n", fails); return 1; }
    printf("ok\n");
    return 0;
}
"""


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    drv = tmp_path / "drive_oracle.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "drive_oracle"
    cmd = ["gcc", "-std=c99", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", str(drv), os.path.join(ROOT, "oracle", "mmf_oracle.c"), "-lm",
           "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr.lower() or "ubsan" in r.stderr.lower()):
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    out = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stderr[-4000:])
