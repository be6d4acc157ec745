/*
 * oracle.c -- plain, slow CPU reference for the Mandelbrot dwell map.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the package's smoke check and the
 * benchmark's CPU-baseline leg are the only callers. The GPU library does not
 * link, load or include anything from this directory, and this file includes
 * nothing from the GPU library.
 *
 * What it computes (paper: "Modeling GPU Dynamic Parallelism for Self Similar
 * Density Workloads"):
 *   - the dwell of one point c: iterate z <- z^2 + c from z = 0 and count the
 *     updates made while |z| < 2, up to MAX_DWELL (Sec. 6, first paragraph);
 *   - the exhaustive map: that dwell at every pixel of the n x n grid
 *     (Sec. 4.1, Eq. 1-2; implementation "Ex" of Sec. 6.1);
 *   - the Mariani-Silver map: an initial g x g grid of regions; each region's
 *     perimeter dwells are computed; a region whose perimeter is uniform is
 *     filled with that dwell, otherwise it is split into r x r sub-regions,
 *     and once sub-regions would fall below side B the region's pixels are
 *     computed one by one (Sec. 4.2.1 assumption iii, the Mandelbrot
 *     instantiation of Q, T and S in Sec. 4.2.1, and Sec. 5.1's final
 *     terminal pass). ASK (Sec. 5) and DP (Sec. 3) are two schedules of this
 *     same recursion; the oracle runs it serially, depth first.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - escape test: keep iterating while |z|^2 < 4 (strict), checked before
 *     each update, so the dwell is the number of updates performed; the flag
 *     ORACLE_ESCAPE_LE switches to |z|^2 <= 4 to show the difference;
 *   - single precision with this exact rounding sequence per iteration:
 *       zi2 = zi*zi; m = fmaf(zr, zr, zi2);            -- |z|^2
 *       t = fmaf(-zi, zi, cr); zr' = fmaf(zr, zr, t);   -- zr^2 - zi^2 + cr
 *       zi' = fmaf(zr + zr, zi, ci);                    -- 2 zr zi + ci
 *     and, for deep zooms where single precision cannot separate
 *     neighbouring pixels, the same sequence with every operation rounded
 *     once to double (the *64 functions, window given in double), or in
 *     float-float arithmetic (ORACLE_FLOAT_FLOAT, see oracle_dwell_ff);
 *   - pixel (px, py) samples c at its corner:
 *       dx = (re_max - re_min) / n, dy = (im_max - im_min) / n  (float)
 *       cr = fmaf(px, dx, re_min), ci = fmaf(py, dy, im_min)
 *     and the map is row-major, out[py * n + px];
 *   - region sides: s0 = ceil(n / g), a child of a side-s region has side
 *     ceil(s / r); every region is clipped to its parent (and the image), and
 *     empty children are dropped;
 *   - a non-uniform region is split when ceil(s / r) >= B, otherwise it is a
 *     leaf whose pixels are all computed (so leaves have side in [B, rB) once
 *     s0 >= B); a region of side 1 has no sub-regions and is always a leaf;
 *   - the perimeter is the region's own outermost rows and columns;
 *   - a fill writes the whole region, perimeter included.
 *
 * Build: cc -std=c11 -O2 -ffp-contract=off (no -ffast-math), see build.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------ */
/* Per-point dwell (Sec. 6: z_{i+1} = z_i^2 + c, z_0 = 0; the dwell is the
 * number of passes made before |z| < 2 stops holding).                  */
/* ------------------------------------------------------------------ */
uint32_t oracle_dwell(float cr, float ci, uint32_t max_dwell, uint32_t flags)
{
    float zr = 0.0f, zi = 0.0f;
    uint32_t d = 0;
    while (d < max_dwell) {
        float zi2 = zi * zi;
        float m = fmaf(zr, zr, zi2);
        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m < 4.0f);
        if (!bounded)
            break;
        float t = fmaf(-zi, zi, cr);
        float nzr = fmaf(zr, zr, t);
        float nzi = fmaf(zr + zr, zi, ci);
        zr = nzr;
        zi = nzi;
        d++;
    }
    return d;
}

/* The same iteration in double precision (deep zooms, where neighbouring
 * pixels are closer than single precision can tell apart). */
uint32_t oracle_dwell64(double cr, double ci, uint32_t max_dwell, uint32_t flags)
{
    double zr = 0.0, zi = 0.0;
    uint32_t d = 0;
    while (d < max_dwell) {
        double zi2 = zi * zi;
        double m = fma(zr, zr, zi2);
        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0) : (m < 4.0);
        if (!bounded)
            break;
        double t = fma(-zi, zi, cr);
        double nzr = fma(zr, zr, t);
        double nzi = fma(zr + zr, zi, ci);
        zr = nzr;
        zi = nzi;
        d++;
    }
    return d;
}

/* The same iteration in float-float ("double-single") arithmetic, a value
 * being the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2.
 * It carries about 48 significant bits using single-precision operations
 * only, for GPUs whose single-precision rate is many times their
 * double-precision rate.  Building blocks, each float operation rounded once:
 *   TwoSum(a, b) (Knuth): s = a + b and the exact error of that sum;
 *   Fast2Sum(a, b) (Dekker): the same in 3 operations when |a| >= |b|;
 *   the exact error of a product a*b, as fma(a, b, -a*b).
 * On them (Dekker's products; the "sloppy" sum, whose error is bounded
 * relative to the operands rather than to the result, which suffices here
 * since |z| and |c| stay near 2 while the orbit is tested):
 *   add(x, y):  (s, e) = TwoSum(xh, yh); w = e + (xl + yl); Fast2Sum(s, w)
 *   mul(x, y):  p = xh*yh; e = fma(xh, yh, -p); e = fma(xh, yl, e);
 *               e = fma(xl, yh, e); Fast2Sum(p, e)
 *   sqr(x):     p = xh*xh; e = fma(xh, xh, -p); e = fma(xh + xh, xl, e);
 *               Fast2Sum(p, e)
 * One iteration: zr2 = sqr(zr), zi2 = sqr(zi); continue while
 * zr2.hi + zi2.hi < 4; zr' = add(zr2, add(cr, -zi2)); zi' = add(2 mul(zr, zi), ci)
 * (negation and doubling are exact on both halves). */
typedef struct {
    float hi, lo;
} ff_t;

static ff_t ff_fast_two_sum(float a, float b)
{
    ff_t r;
    r.hi = a + b;
    r.lo = b - (r.hi - a);
    return r;
}

static ff_t ff_add(ff_t x, ff_t y)
{
    float s = x.hi + y.hi;
    float bb = s - x.hi;
    float e = (x.hi - (s - bb)) + (y.hi - bb);
    float w = e + (x.lo + y.lo);
    return ff_fast_two_sum(s, w);
}

static ff_t ff_mul(ff_t x, ff_t y)
{
    float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return ff_fast_two_sum(p, e);
}

static ff_t ff_sqr(ff_t x)
{
    float p = x.hi * x.hi;
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(x.hi + x.hi, x.lo, e);
    return ff_fast_two_sum(p, e);
}

static ff_t ff_from_double(double v)
{
    ff_t r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

uint32_t oracle_dwell_ff(double cr_d, double ci_d, uint32_t max_dwell, uint32_t flags)
{
    const ff_t cr = ff_from_double(cr_d), ci = ff_from_double(ci_d);
    ff_t zr = {0.0f, 0.0f}, zi = {0.0f, 0.0f};
    uint32_t d = 0;
    while (d < max_dwell) {
        ff_t zr2 = ff_sqr(zr), zi2 = ff_sqr(zi);
        float m = zr2.hi + zi2.hi;
        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m < 4.0f);
        if (!bounded)
            break;
        ff_t neg_zi2 = {-zi2.hi, -zi2.lo};
        ff_t nzr = ff_add(zr2, ff_add(cr, neg_zi2));
        ff_t p = ff_mul(zr, zi);
        ff_t p2 = {p.hi + p.hi, p.lo + p.lo};
        ff_t nzi = ff_add(p2, ci);
        zr = nzr;
        zi = nzi;
        d++;
    }
    return d;
}

/* Pixel -> point of the complex plane (corner sampling, see header). */
void oracle_pixel_to_c(const oracle_window *win, uint32_t n, uint32_t px,
                       uint32_t py, float *cr, float *ci)
{
    float dx = (win->re_max - win->re_min) / (float)n;
    float dy = (win->im_max - win->im_min) / (float)n;
    *cr = fmaf((float)px, dx, win->re_min);
    *ci = fmaf((float)py, dy, win->im_min);
}

void oracle_pixel_to_c64(const oracle_window64 *win, uint32_t n, uint32_t px,
                         uint32_t py, double *cr, double *ci)
{
    double dx = (win->re_max - win->re_min) / (double)n;
    double dy = (win->im_max - win->im_min) / (double)n;
    *cr = fma((double)px, dx, win->re_min);
    *ci = fma((double)py, dy, win->im_min);
}

/* The window of a map in either precision: exactly one pointer is set. */
typedef struct {
    const oracle_window *w32;
    const oracle_window64 *w64;
} any_window;

static uint32_t pixel_dwell(const any_window *win, uint32_t n,
                            uint32_t max_dwell, uint32_t flags, uint32_t px,
                            uint32_t py)
{
    if (win->w64) {
        double cr, ci;
        oracle_pixel_to_c64(win->w64, n, px, py, &cr, &ci);
        if (flags & ORACLE_FLOAT_FLOAT)
            return oracle_dwell_ff(cr, ci, max_dwell, flags);
        return oracle_dwell64(cr, ci, max_dwell, flags);
    }
    float cr, ci;
    oracle_pixel_to_c(win->w32, n, px, py, &cr, &ci);
    return oracle_dwell(cr, ci, max_dwell, flags);
}

static int window_ok(const oracle_window *w)
{
    return w && isfinite(w->re_min) && isfinite(w->re_max) && isfinite(w->im_min) &&
           isfinite(w->im_max) && w->re_max > w->re_min && w->im_max > w->im_min;
}

static int window64_ok(const oracle_window64 *w)
{
    return w && isfinite(w->re_min) && isfinite(w->re_max) && isfinite(w->im_min) &&
           isfinite(w->im_max) && w->re_max > w->re_min && w->im_max > w->im_min;
}

static int any_window_ok(const any_window *w)
{
    return w->w64 ? window64_ok(w->w64) : window_ok(w->w32);
}

/* ------------------------------------------------------------------ */
/* Exhaustive map (Sec. 4.1, Eq. 1-2): one dwell per pixel.             */
/* ------------------------------------------------------------------ */
typedef struct {
    const any_window *win;
    uint32_t n, max_dwell, flags;
    uint32_t row_begin, row_end;
    uint32_t *out;
    uint64_t iterations;
} ex_job;

static void *ex_rows(void *arg)
{
    ex_job *j = (ex_job *)arg;
    uint64_t it = 0;
    for (uint32_t py = j->row_begin; py < j->row_end; py++)
        for (uint32_t px = 0; px < j->n; px++) {
            uint32_t d = pixel_dwell(j->win, j->n, j->max_dwell, j->flags, px, py);
            j->out[(size_t)py * j->n + px] = d;
            it += d;
        }
    j->iterations = it;
    return NULL;
}

static int render_exhaustive(const any_window *win, uint32_t n,
                             uint32_t max_dwell, uint32_t flags, uint32_t *out,
                             int nthreads, uint64_t *iterations)
{
    if (!out || n == 0 || max_dwell == 0 || !any_window_ok(win))
        return -1;
    if (nthreads < 1)
        nthreads = 1;
    if ((uint32_t)nthreads > n)
        nthreads = (int)n;
    ex_job *jobs = (ex_job *)calloc((size_t)nthreads, sizeof(ex_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -2;
    }
    for (int t = 0; t < nthreads; t++) {
        jobs[t].win = win;
        jobs[t].n = n;
        jobs[t].max_dwell = max_dwell;
        jobs[t].flags = flags;
        jobs[t].row_begin = (uint32_t)(((uint64_t)n * (uint64_t)t) / (uint64_t)nthreads);
        jobs[t].row_end = (uint32_t)(((uint64_t)n * (uint64_t)(t + 1)) / (uint64_t)nthreads);
        jobs[t].out = out;
    }
    for (int t = 1; t < nthreads; t++)
        pthread_create(&tid[t], NULL, ex_rows, &jobs[t]);
    ex_rows(&jobs[0]);
    uint64_t total = jobs[0].iterations;
    for (int t = 1; t < nthreads; t++) {
        pthread_join(tid[t], NULL);
        total += jobs[t].iterations;
    }
    if (iterations)
        *iterations = total;
    free(jobs);
    free(tid);
    return 0;
}

int oracle_render_exhaustive(const oracle_window *win, uint32_t n,
                             uint32_t max_dwell, uint32_t flags, uint32_t *out,
                             int nthreads, uint64_t *iterations)
{
    any_window w = {win, NULL};
    return render_exhaustive(&w, n, max_dwell, flags, out, nthreads, iterations);
}

int oracle_render_exhaustive64(const oracle_window64 *win, uint32_t n,
                               uint32_t max_dwell, uint32_t flags, uint32_t *out,
                               int nthreads, uint64_t *iterations)
{
    any_window w = {NULL, win};
    return render_exhaustive(&w, n, max_dwell, flags, out, nthreads, iterations);
}

/* ------------------------------------------------------------------ */
/* Mariani-Silver subdivision (Sec. 4.2.1 and Sec. 6), serial and       */
/* depth first.                                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    const any_window *win;
    uint32_t n, max_dwell, g, r, B, flags;
    /* output: the full map (out_stride == n, origin 0,0) or one initial
     * region's tile (origin ox,oy, row stride out_stride) */
    uint32_t *out;
    uint32_t ox, oy;
    size_t out_stride;
    oracle_ms_stats st;
    oracle_region *log;
    uint64_t log_cap, log_len;
} ms_job;

static uint32_t ceil_div(uint32_t a, uint32_t b) { return a / b + (a % b != 0); }

static void put(ms_job *j, uint32_t x, uint32_t y, uint32_t d)
{
    j->out[(size_t)(y - j->oy) * j->out_stride + (x - j->ox)] = d;
}

static void log_region(ms_job *j, uint32_t level, uint32_t x0, uint32_t y0,
                       uint32_t w, uint32_t h, uint32_t s, uint32_t kind,
                       uint32_t d)
{
    if (j->log && j->log_len < j->log_cap) {
        oracle_region *e = &j->log[j->log_len];
        e->level = level;
        e->x0 = x0;
        e->y0 = y0;
        e->w = w;
        e->h = h;
        e->s = s;
        e->kind = kind;
        e->dwell = d;
    }
    j->log_len++;
}

/* One region: origin (x0, y0), clipped extent w x h, nominal side s. */
static void ms_region(ms_job *j, uint32_t level, uint32_t x0, uint32_t y0,
                      uint32_t w, uint32_t h, uint32_t s)
{
    if (level < ORACLE_MAX_LEVELS)
        j->st.regions_per_level[level]++;
    if (level + 1 > j->st.levels)
        j->st.levels = level + 1;

    /* Exploration query Q: dwell on the perimeter, i.e. the top row, the
     * bottom row, and the left and right columns between them. */
    uint32_t first = 0;
    int have_first = 0, uniform = 1;
    for (uint32_t y = y0; y < y0 + h; y++) {
        int edge_row = (y == y0) || (y == y0 + h - 1);
        uint32_t step = edge_row ? 1u : (w > 1 ? w - 1 : 1u);
        for (uint32_t x = x0; x < x0 + w; x += step) {
            uint32_t d = pixel_dwell(j->win, j->n, j->max_dwell, j->flags, x, y);
            j->st.border_pixels++;
            j->st.iterations += d;
            if (!have_first) {
                first = d;
                have_first = 1;
            } else if (d != first) {
                uniform = 0;
            }
        }
    }

    if (uniform && !(j->flags & ORACLE_NO_FILL)) {
        /* Terminal work T: write the common dwell on every pixel. */
        for (uint32_t y = y0; y < y0 + h; y++)
            for (uint32_t x = x0; x < x0 + w; x++)
                put(j, x, y, first);
        if (level < ORACLE_MAX_LEVELS)
            j->st.fills_per_level[level]++;
        j->st.fill_pixels += (uint64_t)w * h;
        log_region(j, level, x0, y0, w, h, s, ORACLE_REGION_FILL, first);
        return;
    }

    uint32_t sc = ceil_div(s, j->r); /* side of the children */
    if (s > 1 && sc >= j->B) {
        /* Subdivision S: r x r children, clipped to this region. */
        if (level < ORACLE_MAX_LEVELS)
            j->st.subdivisions_per_level[level]++;
        log_region(j, level, x0, y0, w, h, s, ORACLE_REGION_SUBDIVIDE, 0);
        for (uint32_t b = 0; b < j->r; b++) {
            for (uint32_t a = 0; a < j->r; a++) {
                uint64_t cx = (uint64_t)x0 + (uint64_t)a * sc;
                uint64_t cy = (uint64_t)y0 + (uint64_t)b * sc;
                if (cx >= (uint64_t)x0 + w || cy >= (uint64_t)y0 + h)
                    continue; /* empty child */
                uint32_t cw = (uint32_t)((uint64_t)x0 + w - cx);
                uint32_t ch = (uint32_t)((uint64_t)y0 + h - cy);
                if (cw > sc)
                    cw = sc;
                if (ch > sc)
                    ch = sc;
                ms_region(j, level + 1, (uint32_t)cx, (uint32_t)cy, cw, ch, sc);
            }
        }
        return;
    }

    /* Last level L: per-pixel dwell on every pixel of the region. */
    for (uint32_t y = y0; y < y0 + h; y++)
        for (uint32_t x = x0; x < x0 + w; x++) {
            uint32_t d = pixel_dwell(j->win, j->n, j->max_dwell, j->flags, x, y);
            put(j, x, y, d);
            j->st.iterations += d;
        }
    j->st.leaves++;
    j->st.leaf_pixels += (uint64_t)w * h;
    log_region(j, level, x0, y0, w, h, s, ORACLE_REGION_LEAF, 0);
}

/* Initial region (gx, gy) of the g x g grid; returns 0 if it is empty. */
static int initial_region(uint32_t n, uint32_t g, uint32_t gx, uint32_t gy,
                          uint32_t *x0, uint32_t *y0, uint32_t *w, uint32_t *h,
                          uint32_t *s)
{
    uint32_t s0 = ceil_div(n, g);
    uint64_t X = (uint64_t)gx * s0, Y = (uint64_t)gy * s0;
    if (X >= n || Y >= n)
        return 0;
    *x0 = (uint32_t)X;
    *y0 = (uint32_t)Y;
    *w = (uint32_t)((uint64_t)n - X < s0 ? (uint64_t)n - X : s0);
    *h = (uint32_t)((uint64_t)n - Y < s0 ? (uint64_t)n - Y : s0);
    *s = s0;
    return 1;
}

static int ms_args_ok(const any_window *win, uint32_t n, uint32_t max_dwell,
                      uint32_t g, uint32_t r, uint32_t B)
{
    return any_window_ok(win) && n > 0 && max_dwell > 0 && g > 0 && r >= 2 && B > 0;
}

typedef struct {
    ms_job job;
    uint32_t first_region, stride, nregions;
} ms_thread;

static void *ms_worker(void *arg)
{
    ms_thread *t = (ms_thread *)arg;
    ms_job *j = &t->job;
    for (uint32_t k = t->first_region; k < t->nregions; k += t->stride) {
        uint32_t x0, y0, w, h, s;
        if (initial_region(j->n, j->g, k % j->g, k / j->g, &x0, &y0, &w, &h, &s))
            ms_region(j, 0, x0, y0, w, h, s);
    }
    return NULL;
}

static void add_stats(oracle_ms_stats *a, const oracle_ms_stats *b)
{
    if (b->levels > a->levels)
        a->levels = b->levels;
    for (int i = 0; i < ORACLE_MAX_LEVELS; i++) {
        a->regions_per_level[i] += b->regions_per_level[i];
        a->fills_per_level[i] += b->fills_per_level[i];
        a->subdivisions_per_level[i] += b->subdivisions_per_level[i];
    }
    a->leaves += b->leaves;
    a->fill_pixels += b->fill_pixels;
    a->leaf_pixels += b->leaf_pixels;
    a->border_pixels += b->border_pixels;
    a->iterations += b->iterations;
}

static int render_ms(const any_window *win, uint32_t n, uint32_t max_dwell,
                     uint32_t g, uint32_t r, uint32_t B, uint32_t flags,
                     uint32_t *out, int nthreads, oracle_ms_stats *stats,
                     oracle_region *log, uint64_t log_cap, uint64_t *log_len)
{
    if (!out || !ms_args_ok(win, n, max_dwell, g, r, B))
        return -1;
    if (nthreads < 1 || log)
        nthreads = 1; /* the region log is kept in visiting order */
    uint64_t nreg64 = (uint64_t)g * g;
    if (nreg64 > 0xffffffffull)
        return -1;
    uint32_t nregions = (uint32_t)nreg64;
    if ((uint32_t)nthreads > nregions)
        nthreads = (int)nregions;

    ms_thread *th = (ms_thread *)calloc((size_t)nthreads, sizeof(ms_thread));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th || !tid) {
        free(th);
        free(tid);
        return -2;
    }
    for (int t = 0; t < nthreads; t++) {
        ms_job *j = &th[t].job;
        j->win = win;
        j->n = n;
        j->max_dwell = max_dwell;
        j->g = g;
        j->r = r;
        j->B = B;
        j->flags = flags;
        j->out = out;
        j->ox = 0;
        j->oy = 0;
        j->out_stride = n;
        j->log = (t == 0) ? log : NULL;
        j->log_cap = (t == 0) ? log_cap : 0;
        th[t].first_region = (uint32_t)t;
        th[t].stride = (uint32_t)nthreads;
        th[t].nregions = nregions;
    }
    for (int t = 1; t < nthreads; t++)
        pthread_create(&tid[t], NULL, ms_worker, &th[t]);
    ms_worker(&th[0]);
    oracle_ms_stats total;
    memset(&total, 0, sizeof(total));
    add_stats(&total, &th[0].job.st);
    for (int t = 1; t < nthreads; t++) {
        pthread_join(tid[t], NULL);
        add_stats(&total, &th[t].job.st);
    }
    if (stats)
        *stats = total;
    if (log_len)
        *log_len = th[0].job.log_len;
    free(th);
    free(tid);
    return 0;
}

int oracle_render_ms(const oracle_window *win, uint32_t n, uint32_t max_dwell,
                     uint32_t g, uint32_t r, uint32_t B, uint32_t flags,
                     uint32_t *out, int nthreads, oracle_ms_stats *stats,
                     oracle_region *log, uint64_t log_cap, uint64_t *log_len)
{
    any_window w = {win, NULL};
    return render_ms(&w, n, max_dwell, g, r, B, flags, out, nthreads, stats, log, log_cap,
                     log_len);
}

int oracle_render_ms64(const oracle_window64 *win, uint32_t n, uint32_t max_dwell,
                       uint32_t g, uint32_t r, uint32_t B, uint32_t flags,
                       uint32_t *out, int nthreads, oracle_ms_stats *stats,
                       oracle_region *log, uint64_t log_cap, uint64_t *log_len)
{
    any_window w = {NULL, win};
    return render_ms(&w, n, max_dwell, g, r, B, flags, out, nthreads, stats, log, log_cap,
                     log_len);
}

int oracle_initial_region(uint32_t n, uint32_t g, uint32_t gx, uint32_t gy,
                          uint32_t *x0, uint32_t *y0, uint32_t *w, uint32_t *h)
{
    uint32_t s;
    if (n == 0 || g == 0 || gx >= g || gy >= g)
        return 0;
    return initial_region(n, g, gx, gy, x0, y0, w, h, &s);
}

static int render_ms_region(const any_window *win, uint32_t n,
                            uint32_t max_dwell, uint32_t g, uint32_t r,
                            uint32_t B, uint32_t flags, uint32_t gx,
                            uint32_t gy, uint32_t *tile, size_t tile_stride,
                            oracle_ms_stats *stats);

int oracle_render_ms_region(const oracle_window *win, uint32_t n,
                            uint32_t max_dwell, uint32_t g, uint32_t r,
                            uint32_t B, uint32_t flags, uint32_t gx,
                            uint32_t gy, uint32_t *tile, size_t tile_stride,
                            oracle_ms_stats *stats)
{
    any_window aw = {win, NULL};
    return render_ms_region(&aw, n, max_dwell, g, r, B, flags, gx, gy, tile, tile_stride, stats);
}

int oracle_render_ms_region64(const oracle_window64 *win, uint32_t n,
                              uint32_t max_dwell, uint32_t g, uint32_t r,
                              uint32_t B, uint32_t flags, uint32_t gx,
                              uint32_t gy, uint32_t *tile, size_t tile_stride,
                              oracle_ms_stats *stats)
{
    any_window aw = {NULL, win};
    return render_ms_region(&aw, n, max_dwell, g, r, B, flags, gx, gy, tile, tile_stride, stats);
}

static int render_ms_region(const any_window *win, uint32_t n,
                            uint32_t max_dwell, uint32_t g, uint32_t r,
                            uint32_t B, uint32_t flags, uint32_t gx,
                            uint32_t gy, uint32_t *tile, size_t tile_stride,
                            oracle_ms_stats *stats)
{
    const any_window aw = *win;
    if (!tile || !ms_args_ok(&aw, n, max_dwell, g, r, B) || gx >= g || gy >= g)
        return -1;
    ms_job j;
    memset(&j, 0, sizeof(j));
    j.win = &aw;
    j.n = n;
    j.max_dwell = max_dwell;
    j.g = g;
    j.r = r;
    j.B = B;
    j.flags = flags;
    j.out = tile;
    uint32_t x0, y0, w, h, s;
    if (!initial_region(n, g, gx, gy, &x0, &y0, &w, &h, &s))
        return 1; /* empty region: nothing to render */
    if (tile_stride < w)
        return -1;
    j.ox = x0;
    j.oy = y0;
    j.out_stride = tile_stride;
    ms_region(&j, 0, x0, y0, w, h, s);
    if (stats)
        *stats = j.st;
    return 0;
}
