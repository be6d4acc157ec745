/*
 * oracle.h -- interface of the CPU reference (test infrastructure only).
 * Nothing outside the tests, the smoke check and the benchmark's CPU
 * baseline includes or loads this; the GPU library has its own header.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_MAX_LEVELS 32

/* flags */
#define ORACLE_ESCAPE_LE 1u /* continue while |z|^2 <= 4 instead of < 4 */
#define ORACLE_NO_FILL 2u   /* never fill: every region ends as a leaf */
/* Double-precision windows only: iterate in float-float arithmetic
 * (oracle_dwell_ff) instead of binary64. */
#define ORACLE_FLOAT_FLOAT 4u

/* region kinds in the log */
#define ORACLE_REGION_FILL 0u
#define ORACLE_REGION_SUBDIVIDE 1u
#define ORACLE_REGION_LEAF 2u

typedef struct {
    float re_min, re_max, im_min, im_max;
} oracle_window;

/* Double-precision window, for the FP64 (deep-zoom) maps. */
typedef struct {
    double re_min, re_max, im_min, im_max;
} oracle_window64;

typedef struct {
    uint32_t levels;
    uint32_t pad_;
    uint64_t regions_per_level[ORACLE_MAX_LEVELS];
    uint64_t fills_per_level[ORACLE_MAX_LEVELS];
    uint64_t subdivisions_per_level[ORACLE_MAX_LEVELS];
    uint64_t leaves;
    uint64_t fill_pixels;
    uint64_t leaf_pixels;
    uint64_t border_pixels;
    uint64_t iterations; /* z-updates over every dwell evaluated */
} oracle_ms_stats;

typedef struct {
    uint32_t level, x0, y0, w, h, s, kind, dwell;
} oracle_region;

uint32_t oracle_dwell(float cr, float ci, uint32_t max_dwell, uint32_t flags);
void oracle_pixel_to_c(const oracle_window *win, uint32_t n, uint32_t px,
                       uint32_t py, float *cr, float *ci);
int oracle_render_exhaustive(const oracle_window *win, uint32_t n,
                             uint32_t max_dwell, uint32_t flags, uint32_t *out,
                             int nthreads, uint64_t *iterations);
int oracle_render_ms(const oracle_window *win, uint32_t n, uint32_t max_dwell,
                     uint32_t g, uint32_t r, uint32_t B, uint32_t flags,
                     uint32_t *out, int nthreads, oracle_ms_stats *stats,
                     oracle_region *log, uint64_t log_cap, uint64_t *log_len);
int oracle_initial_region(uint32_t n, uint32_t g, uint32_t gx, uint32_t gy,
                          uint32_t *x0, uint32_t *y0, uint32_t *w, uint32_t *h);
/* The same dwell, pixel mapping and maps in double precision, with the same
 * operation sequence (each operation rounded once to double):
 *   zi2 = zi*zi; m = fma(zr, zr, zi2); t = fma(-zi, zi, cr);
 *   zr' = fma(zr, zr, t); zi' = fma(zr + zr, zi, ci);
 *   dx = (re_max - re_min) / n; cr = fma(px, dx, re_min) (likewise ci). */
uint32_t oracle_dwell64(double cr, double ci, uint32_t max_dwell, uint32_t flags);
void oracle_pixel_to_c64(const oracle_window64 *win, uint32_t n, uint32_t px,
                         uint32_t py, double *cr, double *ci);
/* Dwell in float-float arithmetic: each value is an unevaluated sum hi + lo
 * of two floats (about 48 significant bits), every float operation rounded
 * once; c = (cr, ci) is split as hi = (float)c, lo = (float)(c - hi). */
uint32_t oracle_dwell_ff(double cr, double ci, uint32_t max_dwell, uint32_t flags);
int oracle_render_exhaustive64(const oracle_window64 *win, uint32_t n,
                               uint32_t max_dwell, uint32_t flags, uint32_t *out,
                               int nthreads, uint64_t *iterations);
int oracle_render_ms64(const oracle_window64 *win, uint32_t n, uint32_t max_dwell,
                       uint32_t g, uint32_t r, uint32_t B, uint32_t flags,
                       uint32_t *out, int nthreads, oracle_ms_stats *stats,
                       oracle_region *log, uint64_t log_cap, uint64_t *log_len);

int oracle_render_ms_region(const oracle_window *win, uint32_t n,
                            uint32_t max_dwell, uint32_t g, uint32_t r,
                            uint32_t B, uint32_t flags, uint32_t gx,
                            uint32_t gy, uint32_t *tile, size_t tile_stride,
                            oracle_ms_stats *stats);
/* The same for a double-precision window (binary64, or float-float with
 * ORACLE_FLOAT_FLOAT in flags). */
int oracle_render_ms_region64(const oracle_window64 *win, uint32_t n,
                              uint32_t max_dwell, uint32_t g, uint32_t r,
                              uint32_t B, uint32_t flags, uint32_t gx,
                              uint32_t gy, uint32_t *tile, size_t tile_stride,
                              oracle_ms_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
