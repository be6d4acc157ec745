/*
 * ask.h -- C ABI of the GB300 (sm_103a) Mandelbrot dwell-map library.
 *
 * The library computes the escape-time ("dwell") map of the Mandelbrot set
 * over an n x n pixel window of the complex plane, three ways:
 *
 *   ASK_METHOD_EXHAUSTIVE  one flat kernel, one dwell per pixel
 *                          (paper Sec. 4.1, Eq. 1-2; implementation "Ex" of
 *                          Sec. 6.1);
 *   ASK_METHOD_ASK         Mariani-Silver subdivision scheduled as Adaptive
 *                          Serial Kernels: one kernel per subdivision level
 *                          reading a device-resident offset lookup table of
 *                          active regions and appending sub-regions to the
 *                          next one, then one kernel for the leaf regions
 *                          (Sec. 5, Sec. 5.2-5.3; subdivision rule Sec. 4.2.1);
 *   ASK_METHOD_CDP2        the same subdivision with device-side child
 *                          launches, one r x r child grid per subdividing
 *                          region, in CUDA Dynamic Parallelism's tail-launch
 *                          stream (the DP scheme of Sec. 3, SBR mapping of
 *                          Sec. 4.3.1).
 *
 * Arithmetic (all methods, identical bits): single precision, each
 * iteration computes zi2 = zi*zi, m = fma(zr, zr, zi2), and while m < 4
 * updates zr' = fma(zr, zr, fma(-zi, zi, cr)), zi' = fma(zr + zr, zi, ci);
 * the dwell is the number of updates, capped at max_dwell.  Pixel (px, py)
 * samples c = (fma(px, dx, re_min), fma(py, dy, im_min)) with
 * dx = (re_max - re_min) / n and dy = (im_max - im_min) / n in float.
 *
 * ask_render64 renders the exhaustive and ASK maps with the same sequence in
 * double precision, for deep zooms, or in float-float arithmetic
 * (ASK_FLAG_FLOAT_FLOAT).
 *
 * Output layout: uint32 dwell[py * n + px], row-major, py = 0 <-> im_min.
 *
 * Subdivision (ASK and CDP2): initial regions of side s0 = ceil(n / g);
 * a region's perimeter (outermost rows and columns) is evaluated; a uniform
 * perimeter fills the whole region with that dwell; otherwise, if the
 * region's side s > 1 and ceil(s / r) >= B it splits into r x r children of
 * side ceil(s / r), clipped to the parent, empty children dropped; else it is
 * a leaf and every pixel is evaluated.  ASK and CDP2 produce identical maps.
 *
 * Errors: every entry point returns an ask_status.  Argument errors are
 * detected before anything is launched and leave the output untouched.
 * Errors that only the device can see (an overflowing region table, a
 * failed device-side launch) are latched in the context and reported by the
 * next call that synchronises: ask_render with a non-NULL stats pointer,
 * ask_render_host, or ask_check.
 *
 * Threading: a context may be used by one host thread at a time; calls on
 * one context are ordered by the stream they are given.
 */
#ifndef ASK_H
#define ASK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASK_MAX_LEVELS 32
#define ASK_MAX_N 65536u

typedef enum {
    ASK_OK = 0,
    ASK_EINVAL = 1,        /* invalid argument (nothing launched) */
    ASK_ENOMEM = 2,        /* device or host allocation failed */
    ASK_ECUDA = 3,         /* a CUDA runtime call failed; see ask_last_error */
    ASK_EOVERFLOW = 4,     /* a device-side capacity check failed */
    ASK_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    ASK_EUNSUPPORTED = 6,  /* the device is not sm_103 or lacks a feature */
    ASK_ECAPACITY = 7      /* ask_render_noalloc: request exceeds its fixed scratch */
} ask_status;

typedef enum {
    ASK_METHOD_EXHAUSTIVE = 0,
    ASK_METHOD_ASK = 1,
    ASK_METHOD_CDP2 = 2
} ask_method;

/* flags of ask_params */
#define ASK_FLAG_COUNT 1u   /* count dwell iterations and pixels per kind (slower) */
#define ASK_FLAG_TIMING 2u  /* record per-kernel device times (read with ask_timing_read) */
#define ASK_FLAG_CDP2_FIRE_AND_FORGET 4u /* CDP2: launch children into the fire-and-forget
                                          * stream (concurrent) instead of the tail-launch
                                          * stream (children of one grid run in order) */
#define ASK_FLAG_EXACT_BORDERS 8u /* ASK: at the last level evaluate every perimeter dwell
                                   * (staged in shared memory, written to the map) and let
                                   * the leaf kernel skip perimeters; by default the last
                                   * level stops at the first two differing dwells and the
                                   * leaf kernel computes whole leaves */
#define ASK_FLAG_LEAF_TILED 16u   /* ASK: leaf kernel with one thread per pixel in
                                   * block_x x block_y tiles instead of the lane-refill
                                   * kernel (same map) */
/* The paper's block-to-region mappings (Sec. 4.3), as comparison variants
 * with the same map.  ASK_METHOD_ASK: one CTA of block_x * block_y threads
 * per region for the perimeter query and the split; with ASK_FLAG_SBR
 * (Sec. 4.3.1) that CTA also fills a uniform region and one CTA computes
 * each leaf region; with ASK_FLAG_MBR (Sec. 4.3.2) fills and leaf pixels are
 * spread over many blocks per region (fill list, tiled leaf kernel).
 * ASK_METHOD_CDP2: ASK_FLAG_MBR makes uniform and leaf regions launch a
 * multi-block child grid (DP-MBR); ASK_FLAG_SBR is the default DP mapping.
 * The two flags exclude each other and ASK_FLAG_EXACT_BORDERS and
 * ASK_FLAG_LEAF_TILED (ASK_EINVAL); the exhaustive method ignores them. */
#define ASK_FLAG_SBR 32u
#define ASK_FLAG_MBR 64u
/* ask_render_host: render the whole map, then copy it (no banded pipeline). */
#define ASK_FLAG_STAGED_COPY 128u
/* ASK: write the deferred fills (uniform regions of more than 16384 pixels)
 * with the fill kernel alone, on the render stream before the leaf kernel,
 * over every SM; by default the leaf kernel's fill warps write them beside
 * its FP32 work.  The same map.  With ASK_FLAG_TIMING this times the fill
 * kernel by itself. */
#define ASK_FLAG_SERIAL_FILL 256u
/* ASK, fault injection for tests of error reporting: the kernels see region
 * tables of capacity 1 (the allocations keep their size, nothing is written
 * out of bounds), so a render that needs more latches a capacity overflow:
 * the next synchronising call returns ASK_EOVERFLOW and clears it.  The map
 * of such a render is incomplete. */
#define ASK_FLAG_INJECT_OVERFLOW 512u
/* ask_render64 only: iterate in float-float arithmetic on the FP32 pipe
 * instead of binary64 (see ask_render64). */
#define ASK_FLAG_FLOAT_FLOAT 1024u
/* ask_render_batch / ask_graph_create_batch: render the batch with one
 * persistent kernel fed from a device work queue (after an init kernel that
 * writes every frame's initial regions), instead of one level kernel per
 * subdivision depth.  The queue holds the regions of every frame and every
 * depth, each region's perimeter query possibly cut into chunk items;
 * deciding a region pushes its children (or fill bands) back onto the queue
 * or appends it to a leaf list that the same kernel's warps work through
 * whenever they have no region item ready, so depths and leaves overlap with
 * no grid-wide step (Sec. 5's region tables kept on the device, without the
 * per-depth launches).  Same maps.  Every device-side wait is bounded: a
 * render in which no warp finds work for a long time (about a minute of
 * back-off polls, counted afresh whenever the queue or the leaf list moves)
 * latches a timeout, reported as ASK_ETIMEOUT by the next synchronising
 * call.  Combines with ASK_FLAG_COUNT, not with ASK_FLAG_EXACT_BORDERS. */
#define ASK_FLAG_PERSISTENT 2048u
/* Tests of the timeout path only (with ASK_FLAG_PERSISTENT): a warp gives
 * up at its first idle poll, so a render where some warp ever waits latches
 * the timeout and returns ASK_ETIMEOUT; its map is incomplete. */
#define ASK_FLAG_WAIT_TEST 4096u

typedef struct {
    float re_min, re_max, im_min, im_max;
} ask_window;

typedef struct {
    uint32_t g;        /* initial grid g x g (Sec. 4.2, G = g^2) */
    uint32_t r;        /* subdivision r x r per split (Sec. 4.2, R = r^2), >= 2 */
    uint32_t B;        /* stop splitting below side B (Sec. 4.2.1 assumption iii) */
    uint32_t block_x;  /* CTA shape of the per-pixel kernels; block_x * block_y */
    uint32_t block_y;  /*   must be a multiple of 32 in [32, 1024] */
    uint32_t flags;    /* ASK_FLAG_* */
} ask_params;

typedef struct {
    uint32_t levels;                           /* subdivision levels run */
    uint32_t pad_;
    uint64_t regions_per_level[ASK_MAX_LEVELS];      /* regions evaluated at level i */
    uint64_t fills_per_level[ASK_MAX_LEVELS];        /* uniform regions filled at level i */
    uint64_t subdivisions_per_level[ASK_MAX_LEVELS]; /* regions split at level i */
    uint64_t leaves;                           /* regions computed per pixel */
    uint64_t fill_pixels;                      /* ASK_FLAG_COUNT only */
    uint64_t leaf_pixels;                      /* ASK_FLAG_COUNT only */
    uint64_t border_pixels;                    /* ASK_FLAG_COUNT only */
    uint64_t iterations;                       /* ASK_FLAG_COUNT only: z-updates executed */
    uint64_t iterations_per_level[ASK_MAX_LEVELS]; /* ASK_FLAG_COUNT, ASK: z-updates of level i */
    uint64_t leaf_iterations;                  /* ASK_FLAG_COUNT, ASK: z-updates of the leaf kernel */
    float ms_total;                            /* device time of the render */
    float ms_per_level[ASK_MAX_LEVELS];        /* ASK: device time of level kernel i */
    float ms_leaf;                             /* ASK: leaf kernel (by default with the
                                                * deferred fills), after the fill kernel when
                                                * that runs (ASK_FLAG_SERIAL_FILL, tiled leaf,
                                                * MBR) */
    float ms_fill;                             /* ASK: the fill kernel when it runs, else ~0 */
    uint32_t kernel_launches;                  /* kernels this render launched from the host */
    uint32_t pad2_;
    uint64_t deferred_fill_pixels;             /* ASK_FLAG_COUNT, ASK: pixels of the uniform
                                                * regions left to the deferred fills */
} ask_stats;

/* Per-kernel device time summed over the renders made with ASK_FLAG_TIMING
 * since the previous ask_timing_read (at most the last 64 of them). */
typedef struct {
    uint32_t renders;                          /* renders summed */
    uint32_t dropped;                          /* renders recorded but overwritten */
    uint32_t levels;                           /* ASK: levels of the most recent render */
    uint32_t method;                           /* method of the most recent render */
    float ms_total;                            /* whole renders */
    float ms_init;                             /* ASK: init kernel */
    float ms_per_level[ASK_MAX_LEVELS];        /* ASK: level kernel i */
    float ms_leaf;                             /* ASK: leaf kernel (as in ask_stats) */
    float ms_fill;                             /* ASK: deferred-fill kernel (as in ask_stats) */
} ask_timing;

typedef struct ask_ctx ask_ctx;

/* Create a context on CUDA device `device` (which becomes current).  The
 * context owns all scratch memory (region tables, counters, and for
 * ask_render_host a device copy of the map).  Returns ASK_EUNSUPPORTED on a
 * device other than compute capability 10.3. */
ask_status ask_ctx_create(ask_ctx **out, int device);

/* Free everything the context owns.  NULL is ignored. */
void ask_ctx_destroy(ask_ctx *ctx);

/* Allocate the scratch that renders of size n with these parameters need,
 * so that later ask_render calls with them allocate nothing (and may be
 * captured into a CUDA graph).  ask_render calls this itself when needed. */
ask_status ask_reserve(ask_ctx *ctx, ask_method method, uint32_t n,
                       const ask_params *params);

/* Render the n x n dwell map of `window` into the caller-owned device
 * buffer d_dwell (n*n uint32, 16-byte aligned) on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  Asynchronous when stats == NULL; with a
 * non-NULL stats pointer it synchronises the stream, fills *stats and
 * reports latched device-side errors.  1 <= n <= 65536, max_dwell >= 1;
 * params may be NULL for the exhaustive method (default 16 x 16 blocks). */
ask_status ask_render(ask_ctx *ctx, ask_method method, const ask_window *window,
                      uint32_t n, uint32_t max_dwell, const ask_params *params,
                      uint32_t *d_dwell, void *stream, ask_stats *stats);

/* Same as ask_render but the map lands in host memory h_dwell (n*n uint32,
 * pageable or pinned; pinned is faster), and the call synchronises `stream`
 * before returning.  The context renders into its own device buffer.  For
 * ASK without stats (and without ASK_FLAG_STAGED_COPY) a map of 192 MiB or
 * more is rendered in bands of initial-region rows -- independent
 * subtrees that cover contiguous map rows -- and each band is copied to the
 * host on a second stream while the next band renders; otherwise the whole
 * map is rendered and then copied on `stream`.  The map is the same. */
ask_status ask_render_host(ask_ctx *ctx, ask_method method, const ask_window *window,
                           uint32_t n, uint32_t max_dwell, const ask_params *params,
                           uint32_t *h_dwell, void *stream, ask_stats *stats);

/* One frame of a batch: its own window, size, dwell cap, subdivision
 * parameters and caller-owned device output (n*n uint32, 16-byte aligned). */
typedef struct {
    ask_window window;
    uint32_t n, max_dwell;
    uint32_t g, r, B;
    uint32_t pad_;
    uint32_t *d_dwell;
} ask_frame;

/* Render `nframes` frames of different sizes, windows and dwell caps with
 * one chain of launches for the whole batch: an init kernel, one persistent
 * level kernel per subdivision depth whose work queue holds the regions of
 * every frame at that depth, the deferred-fill kernel and one leaf kernel
 * over the leaves of every frame (ASK, Sec. 5, with region records that name
 * their frame); with ASK_FLAG_PERSISTENT, one persistent kernel over a device
 * work queue instead (see the flag).  flags: ASK_FLAG_COUNT,
 * ASK_FLAG_EXACT_BORDERS (not with ASK_FLAG_PERSISTENT), ASK_FLAG_PERSISTENT,
 * ASK_FLAG_WAIT_TEST.  Maps are
 * identical to rendering each frame alone with ask_render.  Asynchronous on
 * `stream` unless stats != NULL (then it synchronises and sums counts over
 * the frames).  The context's batch scratch grows as needed. */
ask_status ask_render_batch(ask_ctx *ctx, const ask_frame *frames, uint32_t nframes,
                            uint32_t flags, void *stream, ask_stats *stats);

/* A batch render captured as a CUDA graph with its own scratch: replaying it
 * renders the same frames into the same buffers with one graph launch.
 * flags: ASK_FLAG_EXACT_BORDERS or ASK_FLAG_PERSISTENT.  Creation allocates
 * and synchronises `stream`; launches do neither. */
typedef struct ask_graph ask_graph;
ask_status ask_graph_create_batch(ask_ctx *ctx, const ask_frame *frames, uint32_t nframes,
                                  uint32_t flags, void *stream, ask_graph **out);
ask_status ask_graph_launch(ask_graph *graph, void *stream);
void ask_graph_destroy(ask_graph *graph);

/* Synchronise `stream`, then sum the device times recorded by renders made
 * with ASK_FLAG_TIMING since the previous call into *out and forget them.
 * The renders must all have been issued on `stream` (or be complete). */
ask_status ask_timing_read(ask_ctx *ctx, void *stream, ask_timing *out);

/* Synchronise `stream` and return (and clear) any latched device error. */
ask_status ask_check(ask_ctx *ctx, void *stream);

/* Host-side plan of the subdivision levels for (n, g, r, B): writes the
 * region side of each level into sides[0..*levels-1] (up to cap entries)
 * and the maximum number of regions a level can hold into max_regions
 * (may be NULL).  No device work. */
ask_status ask_plan_levels(uint32_t n, uint32_t g, uint32_t r, uint32_t B,
                           uint32_t *sides, uint64_t *max_regions, uint32_t cap,
                           uint32_t *levels);

/* ASK render that allocates nothing (the paper has no counterpart: this is a
 * service for callers).  For callers that may not call cudaMalloc -- a frame
 * loop or host callback where an allocation and the synchronisation it may
 * cause are not allowed, a plug-in whose host application owns all device
 * memory, a service held to a fixed memory budget.  The scratch comes from
 * arrays with static storage on the device, shared by every call: at most
 * 2^20 regions per subdivision level and 2^20 leaves (about 24 MiB on every
 * device that loads the library, held until the process exits).  The rule is
 * exact: every level's bound (intervals per axis)^2, as ask_plan_levels
 * reports it in max_regions, must be at most 2^20.  For g a power of two that
 * divides n this holds for n up to 16384 with B >= 16 or n up to 4096 with
 * B >= 4; a g that leaves remainder intervals can exceed it at those sizes
 * (n = 16384, g = 17, r = 2, B = 16 does).  A larger plan returns
 * ASK_ECAPACITY before anything is launched; other argument errors return
 * ASK_EINVAL.  params->flags must be 0.  The call is asynchronous on `stream`
 * and renders into the caller's d_dwell (n*n uint32, 16-byte aligned) on the
 * current device.  The first call on a device looks up the scratch addresses
 * (cudaGetSymbolAddress); make it before any stream capture.  Calls whose
 * work overlaps on the GPU share the scratch and race: order them on one
 * stream.  Each call clears the counters it needs on its stream first. */
ask_status ask_render_noalloc(const ask_window *window, uint32_t n, uint32_t max_dwell,
                              const ask_params *params, uint32_t *d_dwell, void *stream);

/* Window of a double-precision render. */
typedef struct {
    double re_min, re_max, im_min, im_max;
} ask_window64;

/* Render in double precision, for deep zooms: past a zoom of about 1e4 over
 * the paper's 2 x 2 window (Sec. 6.1) the pixels of a large map are closer
 * together than single precision separates, and neighbouring columns would
 * share one c.  The same arithmetic sequence as the single-precision methods
 * with every operation rounded once to binary64 (zi2 = zi*zi,
 * m = fma(zr, zr, zi2), while m < 4: zr' = fma(zr, zr, fma(-zi, zi, cr)),
 * zi' = fma(zr + zr, zi, ci)); pixel (px, py) samples
 * c = (fma(px, dx, re_min), fma(py, dy, im_min)) with
 * dx = (re_max - re_min) / n and dy = (im_max - im_min) / n in double.
 * Methods ASK_METHOD_EXHAUSTIVE and ASK_METHOD_ASK (same subdivision rule,
 * Sec. 4.2.1 and Sec. 5; one warp per region, so g should give a few
 * thousand initial regions); ASK_METHOD_CDP2 returns ASK_EINVAL.
 * params->flags: ASK_FLAG_COUNT and ASK_FLAG_FLOAT_FLOAT.  With
 * ASK_FLAG_FLOAT_FLOAT every value is the unevaluated sum hi + lo of two
 * floats (about 48 significant bits) and the iteration runs on the FP32
 * pipe, which GB300 runs 64 times faster than FP64: c from the double pixel
 * map split as hi = (float)c, lo = (float)(c - hi); sums by TwoSum of the
 * hi parts, plus the lo parts, then Fast2Sum; products and squares by
 * Dekker's scheme with fma; the test zr^2.hi + zi^2.hi < 4.  Its maps
 * differ from the binary64 maps only where the orbit is chaotic.  Output, ownership, stream, stats and
 * error behaviour as ask_render (ms_fill is 0: uniform regions are filled
 * by the level kernels). */
ask_status ask_render64(ask_ctx *ctx, ask_method method, const ask_window64 *window,
                        uint32_t n, uint32_t max_dwell, const ask_params *params,
                        uint32_t *d_dwell, void *stream, ask_stats *stats);

/* Human-readable name of a status code (static storage). */
const char *ask_status_str(ask_status status);

/* Text of the last CUDA error seen by this context ("" if none). */
const char *ask_last_error(const ask_ctx *ctx);

/* Library version string (static storage). */
const char *ask_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ASK_H */
