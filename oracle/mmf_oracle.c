/*
 * CPU oracle for the running maximum-minimum filter.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it computes (Lemire, "Streaming Maximum-Minimum Filter Using No More
 * than Three Comparisons per Element"):
 *
 *   bf1d      the definition of Section 1: for every window [j, j+w) of
 *             a_0..a_{n-1} (0-based), the maximum and the minimum, for
 *             j = 0..n-w (n-w+1 outputs; none when w > n).  This is the
 *             "naive" row of Table 1: 2w-2 comparisons per window.
 *   bf1d_at   the same definition evaluated at caller-chosen window starts.
 *   wedge     Algorithm 1 (Section 4), the streaming monotonic-wedge
 *             algorithm, with U and L kept as fixed-capacity rings, a count
 *             of value comparisons (the cost model of Section 1: one count
 *             per a<b or b<a) and the wedge size size(U)+size(L) checked at
 *             the end of every step (Proposition 4).  The last window, which
 *             the pseudocode leaves implicit, is emitted after the loop, as
 *             the appendix does.
 *   envelope  centred, end-clipped windows: U_i = max a[max(0,i-r) ..
 *             min(n-1,i+r)] and L_i likewise (the envelope use of the filter
 *             cited in Section 1), n outputs.
 *   bf2d      the two-dimensional filter of Section 1 ("rows then columns")
 *             written as the literal maximum/minimum over each wy x wx
 *             rectangle (valid mode), with no separation.
 *   bf2d_at   the same at caller-chosen output pixels.
 *   lb_keogh  the lower bound of the dynamic-time-warping distance built on a
 *             precomputed max-min envelope (the application cited in
 *             Section 1): with U, L the centred, end-clipped envelope of
 *             radius r of a series c (as in `envelope`) and a query q of
 *             the same length, sqrt of the sum over i of (q_i - U_i)^2 where
 *             q_i > U_i and (L_i - q_i)^2 where q_i < L_i, in double.
 *   argbf1d   the locations of the maximum and the minimum of every window
 *             [j, j+w) (the arg-max/arg-min filter that stored locations give
 *             at no cost, Section 5): the leftmost position among equal
 *             extremes, found by scanning the window left to right and
 *             replacing the candidate only on a strictly larger (smaller)
 *             value.
 *   w3        the window-3 filter of the proposition after the lower
 *             bound in Section 3 (at most 2 comparisons per element, zero
 *             latency): the order of the last two elements is known from
 *             the previous step, so comparing the new element with each of
 *             them fixes the maximum, the minimum and the next order.  One
 *             comparison starts the first pair; 2 per later element.
 *   dtw_band  the dynamic-time-warping distance of q and c with warping
 *             restricted to |i - j| <= r: sqrt of the least sum of
 *             (q_i - c_j)^2 along a monotone path from (0,0) to (n-1,n-1)
 *             with unit steps, by dynamic programming, in double.  It is the
 *             quantity lb_keogh bounds from below (used to pin lb_keogh).
 *
 * Every result is one of the input elements, so there is no rounding: all
 * comparisons are the plain C operators on the element type.
 *
 * Readings where the paper is silent (listed in the design notes):
 *   - 0-based window starts j = 0..n-w; w > n gives zero outputs; any w >= 1
 *     is accepted (Algorithm 1 states w > 2 but nothing in it needs that).
 *   - Algorithm 1's while loops stop without a comparison when the deque is
 *     empty; such a non-comparison is not counted.
 *   - The two front checks are an if / else-if, as printed: at most one
 *     front leaves per step (the proof of Proposition 2 shows that every
 *     older index is in exactly one of U, L).  The oracle counts the steps
 *     where both fronts were stale and reports it; it must stay zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Status codes of the oracle (its own, unrelated to the library's). */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
    int64_t ncmp;          /* value comparisons made (Section 1 cost model) */
    int64_t max_size;      /* max over steps of size(U)+size(L), Prop. 4 */
    int64_t stale_fronts;  /* steps where both fronts had left: must be 0 */
    int64_t steps;         /* loop iterations run */
} orc_wedge_stats;

/* A double-ended queue of indices with a fixed power-of-two capacity.  Its
 * size never exceeds w+2 in Algorithm 1 (the w window elements plus the new
 * index before the expired front is dropped), so capacity >= w+2 suffices. */
typedef struct {
    int64_t *buf;
    int64_t mask;
    int64_t head; /* index of the front slot */
    int64_t size;
} orc_deque;

static int dq_init(orc_deque *d, int64_t min_cap) {
    int64_t cap = 1;
    while (cap < min_cap) cap <<= 1;
    d->buf = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!d->buf) return ORC_ENOMEM;
    d->mask = cap - 1;
    d->head = 0;
    d->size = 0;
    return ORC_OK;
}
static void dq_free(orc_deque *d) { free(d->buf); d->buf = NULL; }
static int64_t dq_front(const orc_deque *d) { return d->buf[d->head & d->mask]; }
static int64_t dq_back(const orc_deque *d) { return d->buf[(d->head + d->size - 1) & d->mask]; }
static void dq_push_back(orc_deque *d, int64_t v) { d->buf[(d->head + d->size) & d->mask] = v; d->size++; }
static void dq_pop_back(orc_deque *d) { d->size--; }
static void dq_pop_front(orc_deque *d) { d->head++; d->size--; }

#define ORC_DEFINE(SUF, T)                                                        \
                                                                                  \
/* Definition of Section 1: max/min over [j, j+w) for every j = 0..n-w. */        \
int oracle_bf1d_##SUF(const T *a, int64_t n, int64_t w, T *mx, T *mn) {          \
    if (n < 0 || w < 1 || (n > 0 && !a)) return ORC_EINVAL;                       \
    for (int64_t j = 0; j + w <= n; ++j) {                                        \
        T hi = a[j], lo = a[j];                                                   \
        for (int64_t i = j + 1; i < j + w; ++i) {                                 \
            if (a[i] > hi) hi = a[i];                                             \
            if (a[i] < lo) lo = a[i];                                             \
        }                                                                         \
        if (mx) mx[j] = hi;                                                       \
        if (mn) mn[j] = lo;                                                       \
    }                                                                             \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
/* The same definition at m chosen window starts (each 0 <= s <= n-w). */         \
int oracle_bf1d_at_##SUF(const T *a, int64_t n, int64_t w, const int64_t *starts, \
                         int64_t m, T *mx, T *mn) {                               \
    if (n < 0 || w < 1 || m < 0) return ORC_EINVAL;                               \
    for (int64_t t = 0; t < m; ++t) {                                             \
        int64_t j = starts[t];                                                    \
        if (j < 0 || j + w > n) return ORC_EINVAL;                                \
        T hi = a[j], lo = a[j];                                                   \
        for (int64_t i = j + 1; i < j + w; ++i) {                                 \
            if (a[i] > hi) hi = a[i];                                             \
            if (a[i] < lo) lo = a[i];                                             \
        }                                                                         \
        if (mx) mx[t] = hi;                                                       \
        if (mn) mn[t] = lo;                                                       \
    }                                                                             \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
/* Algorithm 1, restated with 0-based indices: the paper's step i (1-based,     \
 * i = 2..n) is step i = 1..n-1 here, and its window [i-w, i) becomes the      \
 * 0-based start i-w.  cmp counts every evaluated value comparison. */           \
int oracle_wedge_##SUF(const T *a, int64_t n, int64_t w, T *mx, T *mn,            \
                       orc_wedge_stats *st) {                                     \
    orc_wedge_stats s = {0, 0, 0, 0};                                             \
    if (n < 0 || w < 1 || (n > 0 && !a)) return ORC_EINVAL;                       \
    if (n == 0) { if (st) *st = s; return ORC_OK; }                               \
    orc_deque U, L;                                                               \
    if (dq_init(&U, w + 2) != ORC_OK) return ORC_ENOMEM;                          \
    if (dq_init(&L, w + 2) != ORC_OK) { dq_free(&U); return ORC_ENOMEM; }         \
    /* "append 1 to U and L" */                                                   \
    dq_push_back(&U, 0);                                                          \
    dq_push_back(&L, 0);                                                          \
    s.max_size = 2;                                                               \
    for (int64_t i = 1; i < n; ++i) {                                             \
        s.steps++;                                                                \
        /* Emit the window that ended at i-1: fronts of U and L. */               \
        if (i >= w) {                                                             \
            if (mx) mx[i - w] = a[dq_front(&U)];                                  \
            if (mn) mn[i - w] = a[dq_front(&L)];                                  \
        }                                                                         \
        /* One comparison against the previous element picks the side. */        \
        s.ncmp++;                                                                 \
        if (a[i] > a[i - 1]) {                                                    \
            dq_pop_back(&U); /* removes i-1 from U */                             \
            while (U.size > 0) {                                                  \
                s.ncmp++;                                                         \
                if (!(a[i] > a[dq_back(&U)])) break;                              \
                dq_pop_back(&U);                                                  \
            }                                                                     \
        } else {                                                                  \
            dq_pop_back(&L); /* removes i-1 from L */                             \
            while (L.size > 0) {                                                  \
                s.ncmp++;                                                         \
                if (!(a[i] < a[dq_back(&L)])) break;                              \
                dq_pop_back(&L);                                                  \
            }                                                                     \
        }                                                                         \
        dq_push_back(&U, i);                                                      \
        dq_push_back(&L, i);                                                      \
        /* Drop the index that left the window [i-w+1, i]. */                     \
        {                                                                         \
            int u_stale = dq_front(&U) == i - w;                                  \
            int l_stale = dq_front(&L) == i - w;                                  \
            if (u_stale) dq_pop_front(&U);                                        \
            else if (l_stale) dq_pop_front(&L);                                   \
            if (u_stale && l_stale) s.stale_fronts++;                             \
        }                                                                         \
        if (U.size + L.size > s.max_size) s.max_size = U.size + L.size;           \
    }                                                                             \
    /* The final window [n-w, n), emitted after the loop. */                      \
    if (n >= w) {                                                                 \
        if (mx) mx[n - w] = a[dq_front(&U)];                                      \
        if (mn) mn[n - w] = a[dq_front(&L)];                                      \
    }                                                                             \
    dq_free(&U);                                                                  \
    dq_free(&L);                                                                  \
    if (st) *st = s;                                                              \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
/* Centred, end-clipped windows of radius r: n outputs. */                        \
int oracle_envelope_##SUF(const T *a, int64_t n, int64_t r, T *up, T *lo) {       \
    if (n < 0 || r < 0 || (n > 0 && !a)) return ORC_EINVAL;                       \
    for (int64_t i = 0; i < n; ++i) {                                             \
        int64_t b = i - r < 0 ? 0 : i - r;                                        \
        int64_t e = i + r > n - 1 ? n - 1 : i + r;                                \
        T hi = a[b], lw = a[b];                                                   \
        for (int64_t k = b + 1; k <= e; ++k) {                                    \
            if (a[k] > hi) hi = a[k];                                             \
            if (a[k] < lw) lw = a[k];                                             \
        }                                                                         \
        if (up) up[i] = hi;                                                       \
        if (lo) lo[i] = lw;                                                       \
    }                                                                             \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
/* Literal rectangle max/min, valid mode: out is (H-wy+1) x (W-wx+1), packed. */ \
int oracle_bf2d_##SUF(const T *img, int64_t H, int64_t W, int64_t pitch,          \
                      int64_t wy, int64_t wx, T *mx, T *mn) {                     \
    if (H < 0 || W < 0 || wy < 1 || wx < 1 || pitch < W) return ORC_EINVAL;      \
    int64_t Ho = H - wy + 1, Wo = W - wx + 1;                                     \
    if (Ho <= 0 || Wo <= 0) return ORC_OK;                                        \
    for (int64_t y = 0; y < Ho; ++y)                                              \
        for (int64_t x = 0; x < Wo; ++x) {                                        \
            T hi = img[y * pitch + x], lw = hi;                                   \
            for (int64_t dy = 0; dy < wy; ++dy)                                   \
                for (int64_t dx = 0; dx < wx; ++dx) {                             \
                    T v = img[(y + dy) * pitch + (x + dx)];                       \
                    if (v > hi) hi = v;                                           \
                    if (v < lw) lw = v;                                           \
                }                                                                 \
            if (mx) mx[y * Wo + x] = hi;                                          \
            if (mn) mn[y * Wo + x] = lw;                                          \
        }                                                                         \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
/* Literal rectangle max/min at m chosen output pixels (ys[t], xs[t]). */         \
int oracle_bf2d_at_##SUF(const T *img, int64_t H, int64_t W, int64_t pitch,       \
                         int64_t wy, int64_t wx, const int64_t *ys,               \
                         const int64_t *xs, int64_t m, T *mx, T *mn) {            \
    if (H < 0 || W < 0 || wy < 1 || wx < 1 || pitch < W || m < 0)                 \
        return ORC_EINVAL;                                                        \
    for (int64_t t = 0; t < m; ++t) {                                             \
        int64_t y = ys[t], x = xs[t];                                             \
        if (y < 0 || x < 0 || y + wy > H || x + wx > W) return ORC_EINVAL;        \
        T hi = img[y * pitch + x], lw = hi;                                       \
        for (int64_t dy = 0; dy < wy; ++dy)                                       \
            for (int64_t dx = 0; dx < wx; ++dx) {                                 \
                T v = img[(y + dy) * pitch + (x + dx)];                           \
                if (v > hi) hi = v;                                               \
                if (v < lw) lw = v;                                               \
            }                                                                     \
        if (mx) mx[t] = hi;                                                       \
        if (mn) mn[t] = lw;                                                       \
    }                                                                             \
    return ORC_OK;                                                                \
}

ORC_DEFINE(f32, float)
ORC_DEFINE(f64, double)
ORC_DEFINE(i16, int16_t)
ORC_DEFINE(u8, uint8_t)

/* The envelope bound and the banded warping distance, in double. */
#define ORC_DEFINE_LB(SUF, T)                                                     \
int oracle_lb_keogh_##SUF(const T *c, const T *q, int64_t n, int64_t r,           \
                          double *out) {                                          \
    if (n < 0 || r < 0 || !out || (n > 0 && (!c || !q))) return ORC_EINVAL;       \
    double sum = 0.0;                                                             \
    for (int64_t i = 0; i < n; ++i) {                                             \
        int64_t b = i - r < 0 ? 0 : i - r;                                        \
        int64_t e = i + r > n - 1 ? n - 1 : i + r;                                \
        T hi = c[b], lw = c[b];                                                   \
        for (int64_t k = b + 1; k <= e; ++k) {                                    \
            if (c[k] > hi) hi = c[k];                                             \
            if (c[k] < lw) lw = c[k];                                             \
        }                                                                         \
        double qi = (double)q[i];                                                 \
        if (qi > (double)hi) sum += (qi - (double)hi) * (qi - (double)hi);        \
        else if (qi < (double)lw) sum += ((double)lw - qi) * ((double)lw - qi);   \
    }                                                                             \
    *out = sqrt(sum);                                                             \
    return ORC_OK;                                                                \
}                                                                                 \
                                                                                  \
int oracle_dtw_band_##SUF(const T *q, const T *c, int64_t n, int64_t r,           \
                          double *out) {                                          \
    if (n < 1 || r < 0 || !out || !q || !c) return ORC_EINVAL;                    \
    double *D = (double *)malloc((size_t)(n * n) * sizeof(double));               \
    if (!D) return ORC_ENOMEM;                                                    \
    for (int64_t i = 0; i < n; ++i)                                               \
        for (int64_t j = 0; j < n; ++j) {                                         \
            if (i - j > r || j - i > r) { D[i * n + j] = INFINITY; continue; }    \
            double d = (double)q[i] - (double)c[j];                               \
            double best;                                                          \
            if (i == 0 && j == 0) best = 0.0;                                     \
            else {                                                                \
                best = INFINITY;                                                  \
                if (i > 0 && D[(i - 1) * n + j] < best) best = D[(i - 1) * n + j];\
                if (j > 0 && D[i * n + j - 1] < best) best = D[i * n + j - 1];    \
                if (i > 0 && j > 0 && D[(i - 1) * n + j - 1] < best)              \
                    best = D[(i - 1) * n + j - 1];                                \
            }                                                                     \
            D[i * n + j] = best + d * d;                                          \
        }                                                                         \
    *out = sqrt(D[n * n - 1]);                                                    \
    free(D);                                                                      \
    return ORC_OK;                                                                \
}

/* Leftmost arg-max / arg-min of every window [j, j+w), by scanning it. */
#define ORC_DEFINE_ARG(SUF, T)                                                    \
int oracle_argbf1d_##SUF(const T *a, int64_t n, int64_t w, int64_t *imx,          \
                         int64_t *imn) {                                          \
    if (n < 0 || w < 1 || (n > 0 && !a)) return ORC_EINVAL;                       \
    for (int64_t j = 0; j + w <= n; ++j) {                                        \
        int64_t bx = j, bn = j;                                                   \
        for (int64_t k = j + 1; k < j + w; ++k) {                                 \
            if (a[k] > a[bx]) bx = k;                                             \
            if (a[k] < a[bn]) bn = k;                                             \
        }                                                                         \
        if (imx) imx[j] = bx;                                                     \
        if (imn) imn[j] = bn;                                                     \
    }                                                                             \
    return ORC_OK;                                                                \
}

ORC_DEFINE_ARG(f32, float)
ORC_DEFINE_ARG(f64, double)
ORC_DEFINE_ARG(i16, int16_t)
ORC_DEFINE_ARG(u8, uint8_t)

/* Window 3 in two comparisons per element; *ncmp counts them. */
#define ORC_DEFINE_W3(SUF, T)                                                     \
int oracle_w3_##SUF(const T *a, int64_t n, T *mx, T *mn, int64_t *ncmp) {         \
    if (n < 0 || (n > 0 && !a)) return ORC_EINVAL;                                \
    int64_t c = 0;                                                                \
    if (n >= 3) {                                                                 \
        int older_greater = a[0] > a[1]; /* order of the last two */             \
        c = 1;                                                                    \
        for (int64_t i = 2; i < n; ++i) {                                         \
            int prev_gt = a[i - 1] > a[i];   /* comparison 1 */                   \
            int older_gt = a[i - 2] > a[i];  /* comparison 2 */                   \
            c += 2;                                                               \
            T hi, lw;                                                             \
            if (older_greater) {   /* a[i-2] > a[i-1] */                          \
                hi = older_gt ? a[i - 2] : a[i];                                  \
                lw = prev_gt ? a[i] : a[i - 1];                                   \
            } else {               /* a[i-1] >= a[i-2] */                         \
                hi = prev_gt ? a[i - 1] : a[i];                                   \
                lw = older_gt ? a[i] : a[i - 2];                                  \
            }                                                                     \
            mx[i - 2] = hi;                                                       \
            mn[i - 2] = lw;                                                       \
            older_greater = prev_gt;                                              \
        }                                                                         \
    }                                                                             \
    if (ncmp) *ncmp = c;                                                          \
    return ORC_OK;                                                                \
}

ORC_DEFINE_W3(f32, float)
ORC_DEFINE_W3(f64, double)
ORC_DEFINE_W3(i16, int16_t)
ORC_DEFINE_W3(u8, uint8_t)

ORC_DEFINE_LB(f32, float)
ORC_DEFINE_LB(f64, double)
ORC_DEFINE_LB(i16, int16_t)
ORC_DEFINE_LB(u8, uint8_t)
