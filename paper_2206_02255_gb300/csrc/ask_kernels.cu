// ask_kernels.cu -- exhaustive kernel and the Adaptive Serial Kernels (ASK)
// pipeline: init, one level kernel per subdivision depth, leaf kernel (which
// also writes the deferred fills), and the fill kernel of the variants that
// fill in a pass of their own.
//
// ASK (paper Sec. 5): the active regions of depth i sit in a device-resident
// offset lookup table (read-OLT, Sec. 5.2).  One kernel per depth evaluates
// every region's perimeter (the exploration query Q of Sec. 4.2.1), fills
// uniform regions (terminal work T), and appends the r x r sub-regions of the
// others to the write-OLT with atomic adds on a global counter (Sec. 5.3.1);
// the counter's final value is the next depth's region count.  The tables are
// swapped between depths (Sec. 5.3.2).  Regions that may not split further
// go to a leaf list, evaluated pixel by pixel by the last kernel (the final
// terminal pass of Sec. 5.1, L(n, tau) of Sec. 4.2).
//
// GB300 layout of that scheme:
//  * level kernels are persistent (a grid sized to the SM count), read the
//    region count from device memory and hand out work with an atomic
//    counter, so no depth needs a host round trip;
//  * a work item is one region's perimeter, or one chunk of kChunkPx
//    (kChunkPxBatch in a batch) perimeter pixels of a large region (several
//    warps per region: the MBR mapping of Sec. 4.3.2 applied to the query),
//    one warp per item;
//  * a query stops at the first two perimeter dwells known to differ; warps
//    of one region share that verdict through a per-region state word, and
//    the warp that finishes the region's last chunk takes the decision;
//  * decisions are compacted per warp: each lane keeps the outcome of one
//    region, then one atomicAdd per list serves up to 32 regions (the
//    block-scan + single atomic alternative of Sec. 5.3.1, at warp scope);
//  * small uniform regions are filled in place by their warp; large ones go
//    to a fill list as bands of rows, written with 128-bit stores by the
//    leaf kernel's fill warps beside its FP32 work (or by the fill kernel);
//  * the OLTs are preallocated for the worst case, so nothing is resized
//    between depths (Sec. 5.3.2 reallocates instead).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_internal.h"

namespace ask {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kWarpStage = 512;  // staged perimeter pixels per warp (exact last level)
constexpr uint32_t kNone = 0xffffffffu;

enum : uint32_t { KIND_NONE = 0, KIND_FILL = 1, KIND_SPLIT = 2, KIND_LEAF = 3, KIND_FILL_LATER = 4 };

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Exhaustive: one thread per pixel over a flat grid of block_x x block_y
// tiles (paper Sec. 4.1: |G_E| = n^2 threads, work n^2 A).
// ---------------------------------------------------------------------------
template <bool COUNT>
__global__ void __launch_bounds__(1024) exhaustive_kernel(uint32_t *__restrict__ map, uint32_t n,
                                                          PixelMap pm, uint32_t max_dwell,
                                                          uint32_t tiles_x, DevCounters *ctr)
{
    const uint32_t tile = blockIdx.x;
    const uint32_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const uint32_t px = tx * blockDim.x + threadIdx.x;
    const uint32_t py = ty * blockDim.y + threadIdx.y;
    uint32_t d = 0;
    if (px < n && py < n) {
        const float2 c = pixel_c(pm, px, py);
        d = dwell(c.x, c.y, max_dwell);
        map[(size_t)py * n + px] = d;
    }
    if (COUNT) {
        const unsigned long long s = warp_sum_u64(d);
        if ((threadIdx.x + threadIdx.y * blockDim.x) % 32u == 0u && s)
            atomicAdd(&ctr->iterations, s);
    }
}

// Zero the per-render counters (the latched error word is kept), write the
// level-0 OLT (the axis0 x axis0 non-empty initial regions of side s0) and,
// when level 0 is queried in chunks, its per-region state.
__global__ void init_kernel(uint2 *__restrict__ olt0, uint4 *__restrict__ rst0, DevCounters *ctr,
                            uint32_t n, uint32_t s0, uint32_t axis0, uint32_t row0, uint32_t rows)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t total = axis0 * rows;
    if (ctr != nullptr) {
        uint32_t *w = reinterpret_cast<uint32_t *>(ctr);
        const uint32_t words = (uint32_t)(sizeof(DevCounters) / sizeof(uint32_t));
        const uint32_t err_word = (uint32_t)(offsetof(DevCounters, error) / sizeof(uint32_t));
        for (uint32_t k = tid; k < words; k += stride)
            if (k != err_word)
                w[k] = (k == 0u) ? total : 0u;  // word 0 is count[0]
    }
    if (olt0 == nullptr)
        return;
    for (uint32_t k = tid; k < total; k += stride) {
        const uint32_t gx = k % axis0, gy = row0 + k / axis0;
        const uint32_t x0 = gx * s0, y0 = gy * s0;
        olt0[k] = pack_region(x0, y0, min(s0, n - x0), min(s0, n - y0));
        if (rst0 != nullptr)
            rst0[k] = make_uint4(kNone, 0u, 0u, 0u);
    }
}

// ---------------------------------------------------------------------------
// Region records: uint2 for one frame, uint4 (with the frame id) for a batch.
// ---------------------------------------------------------------------------
template <bool BATCH>
struct Rec;
template <>
struct Rec<false> {
    using T = uint2;
    static __device__ __forceinline__ Region region(T e) { return unpack_region(e); }
    static __device__ __forceinline__ uint32_t frame(T) { return 0u; }
    static __device__ __forceinline__ T child(T, uint2 c) { return c; }
};
template <>
struct Rec<true> {
    using T = uint4;
    static __device__ __forceinline__ Region region(T e) { return unpack_region(make_uint2(e.x, e.y)); }
    static __device__ __forceinline__ uint32_t frame(T e) { return e.z; }
    static __device__ __forceinline__ T child(T p, uint2 c) { return make_uint4(c.x, c.y, p.z, 0u); }
};

// The parameters of the frame a region belongs to, at one level.
struct FView {
    uint32_t *map;
    PixelMap pm;
    uint32_t n, max_dwell, side, child_side, r;
    bool split;
};

__device__ __forceinline__ FView view_single(const LevelArgs &a)
{
    FView v;
    v.map = a.map;
    v.pm = a.pm;
    v.n = a.n;
    v.max_dwell = a.max_dwell;
    v.side = a.side;
    v.child_side = a.child_side;
    v.r = a.r;
    v.split = a.split != 0u;
    return v;
}

__device__ __forceinline__ FView view_frame(const FrameDesc *frames, uint32_t f, uint32_t level)
{
    const FrameDesc &d = frames[f];
    FView v;
    v.map = d.map;
    v.pm = d.pm;
    v.n = d.n;
    v.max_dwell = d.max_dwell;
    v.r = d.r;
    v.side = d.side[level];
    v.child_side = ceil_div_u32(v.side, v.r);
    v.split = level + 1u < d.levels;
    return v;
}

// ---------------------------------------------------------------------------
// Per-warp record of decided regions, flushed with one atomic per list.
// ---------------------------------------------------------------------------
template <bool BATCH>
struct WarpBatch {
    typename Rec<BATCH>::T rec;  // lane j: record of the j-th region decided
    uint32_t kind;   // KIND_*
    uint32_t nchild; // children of a splitting region
    uint32_t dwell;  // dwell of a uniform region filled later
    uint32_t sc, r;  // child side and split factor of its frame
};

template <bool BATCH>
__device__ __forceinline__ void flush_batch(const LevelArgs &a, WarpBatch<BATCH> &b, uint32_t lane)
{
    using R = Rec<BATCH>;
    using T = typename R::T;
    T *leaves = static_cast<T *>(a.leaves);
    T *olt_out = static_cast<T *>(a.olt_out);
    DevCounters *ctr = a.ctr;
    const unsigned lt = (1u << lane) - 1u;
    // leaves: ballot + popc gives each leaf its slot
    const unsigned leaf_mask = __ballot_sync(kFull, b.kind == KIND_LEAF);
    if (leaf_mask) {
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(&ctr->leaf_count, (uint32_t)__popc(leaf_mask));
        base = __shfl_sync(kFull, base, 0);
        if (b.kind == KIND_LEAF) {
            const uint32_t slot = base + (uint32_t)__popc(leaf_mask & lt);
            if (slot < a.leaf_cap)
                leaves[slot] = b.rec;
            else
                atomicOr(&ctr->error, ERR_LEAF_OVERFLOW);
        }
    }
    // large uniform regions for the fill list, as bands of rows: a warp
    // scan of the band counts, one atomicAdd, then each lane writes the
    // bands of its region
    const unsigned later_mask = __ballot_sync(kFull, b.kind == KIND_FILL_LATER);
    if (later_mask) {
        const Region g = R::region(b.rec);
        const uint32_t nb = (b.kind == KIND_FILL_LATER) ? fill_band_count(g.w, g.h) : 0u;
        uint32_t incl = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o)
                incl += v;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(&ctr->fill_count, total);
        base = __shfl_sync(kFull, base, 0) + incl - nb;
        const uint32_t rows = fill_band_rows(g.w);
        for (uint32_t j = 0; j < nb; ++j) {
            const uint2 band = pack_region(g.x0, g.y0 + j * rows, g.w, min(rows, g.h - j * rows));
            if (base + j < a.fill_cap)
                a.fills[base + j] = make_uint4(band.x, band.y, b.dwell, R::frame(b.rec));
            else
                atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
        }
    }
    // children: warp inclusive scan of child counts, one atomicAdd
    uint32_t incl = b.nchild;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o)
            incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total) {
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(&ctr->count[a.level + 1], total);
        base = __shfl_sync(kFull, base, 0);
        if (b.nchild) {
            const Region g = R::region(b.rec);
            const uint32_t first = base + incl - b.nchild;
            for (uint32_t j = 0; j < b.nchild; ++j) {
                const uint32_t slot = first + j;
                if (slot < a.olt_cap) {
                    olt_out[slot] = R::child(b.rec, child_region(g, b.sc, b.r, j));
                    if (a.next_chunks > 1u)
                        a.rst_out[slot] = make_uint4(kNone, 0u, 0u, 0u);
                } else {
                    atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
                }
            }
        }
    }
    const unsigned fill_mask = __ballot_sync(kFull, b.kind == KIND_FILL || b.kind == KIND_FILL_LATER);
    const unsigned split_mask = __ballot_sync(kFull, b.kind == KIND_SPLIT);
    if (lane == 0) {
        if (fill_mask)
            atomicAdd(&ctr->fills[a.level], (uint32_t)__popc(fill_mask));
        if (split_mask)
            atomicAdd(&ctr->subdivs[a.level], (uint32_t)__popc(split_mask));
    }
    b.kind = KIND_NONE;
    b.nchild = 0;
}

// Rounds between issuing a state load and using it, for one frame.  A
// batch keeps enough warps resident to hide the load, and there a late
// stop costs more than the wait, so it uses the value one round later.
constexpr uint32_t kPollLag = 8;

// One chunk [k0, k1) of a large region's perimeter, queried by one warp.  The
// region's state st: x = common dwell found so far (kNone: none yet),
// y = 1 once two dwells are known to differ, z = chunks finished.  Chunks of
// the same region run on other warps at the same time and stop as soon as
// one of them has set y.
template <bool BATCH>
__device__ __forceinline__ void chunk_query(const FView &a, const Region &g, uint32_t k0,
                                            uint32_t k1, uint4 *st, uint32_t lane,
                                            unsigned long long &it)
{
    const volatile uint32_t *ps = reinterpret_cast<const volatile uint32_t *>(st);
    for (uint32_t base = k0; base < k1; base += 32u) {
        // the state load is issued first; the group's set-up hides its latency
        uint32_t sx = 0, sy = 0;
        if (lane == 0) {
            sx = ps[0];
            sy = ps[1];
        }
        const uint32_t k = base + lane;
        const bool active = k < k1;
        const unsigned amask = __ballot_sync(kFull, active);
        uint32_t px = g.x0, py = g.y0;
        if (active)
            perimeter_pixel(g, k, px, py);
        Orbit o = orbit_start(pixel_c(a.pm, px, py));
        uint32_t stt = active ? ORBIT_RUN : ORBIT_DONE;
        bool differ = false, stop = false;
        uint2 v = make_uint2(__shfl_sync(kFull, sx, 0), __shfl_sync(kFull, sy, 0));
        if (v.y)
            return;
        // A state load is issued every kPollLag rounds (every round in a
        // batch) and consumed that many rounds later, so its L2 latency
        // hides behind the updates of those rounds; a stale value is
        // harmless (the common dwell is set once, the flag only rises).
        uint32_t nx = v.x, ny = v.y, lag = 0;
        for (;;) {
            if (lag == 0 && lane == 0) {
                nx = ps[0];
                ny = ps[1];
            }
            const uint32_t limit = (v.x != kNone) ? min(a.max_dwell, v.x + 1u) : a.max_dwell;
            if (stt == ORBIT_RUN)
                stt = orbit_step<kQueryRoundLarge>(o, limit);
            const unsigned dm = __ballot_sync(kFull, stt != ORBIT_RUN) & amask;
            if (dm == amask)
                break;
            if (dm) {
                differ = true;
                break;
            }
            if (++lag == (BATCH ? 1u : kPollLag)) {
                lag = 0;
                v.x = __shfl_sync(kFull, nx, 0);
                v.y = __shfl_sync(kFull, ny, 0);
                if (v.y) {
                    stop = true;
                    break;
                }
            }
        }
        if (!stop && !differ && stt == ORBIT_PEND)
            orbit_resolve<kQueryRoundLarge>(o);
        if (active)
            it += o.d;
        if (stop)
            return;
        if (differ) {
            if (lane == 0)
                atomicExch(&st->y, 1u);
            return;
        }
        const uint32_t vmin = __reduce_min_sync(kFull, active ? o.d : kNone);
        const uint32_t vmax = __reduce_max_sync(kFull, active ? o.d : 0u);
        if (lane == 0) {
            if (vmin != vmax) {
                atomicExch(&st->y, 1u);
            } else {
                const uint32_t old = atomicCAS(&st->x, kNone, vmin);
                if (old != kNone && old != vmin)
                    atomicExch(&st->y, 1u);
            }
        }
        __syncwarp();
    }
}

// One chunk [k0, k1) of a large last-level region with exact perimeters:
// every dwell is computed and written; st.x / st.y collect min / max.
__device__ __forceinline__ void chunk_exact(const FView &a, const Region &g, uint32_t k0,
                                            uint32_t k1, uint4 *st, uint32_t lane,
                                            unsigned long long &it)
{
    uint32_t dmin = kNone, dmax = 0u;
    for (uint32_t k = k0 + lane; k < k1; k += 32u) {
        uint32_t px, py;
        perimeter_pixel(g, k, px, py);
        const float2 c = pixel_c(a.pm, px, py);
        const uint32_t d = dwell(c.x, c.y, a.max_dwell);
        a.map[(size_t)py * a.n + px] = d;
        dmin = min(dmin, d);
        dmax = max(dmax, d);
        it += d;
    }
    dmin = __reduce_min_sync(kFull, dmin);
    dmax = __reduce_max_sync(kFull, dmax);
    if (lane == 0) {
        atomicMin(&st->x, dmin);
        atomicMax(&st->y, dmax);
    }
}

// ---------------------------------------------------------------------------
// Level kernel: one warp per work item (a region, or a perimeter chunk of a
// large region).
// ---------------------------------------------------------------------------
template <bool COUNT, bool BATCH>
__global__ void __launch_bounds__(256) level_kernel(LevelArgs a)
{
    using R = Rec<BATCH>;
    using T = typename R::T;
    extern __shared__ uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *stage = smem + (threadIdx.x >> 5) * kWarpStage;
    const T *olt_in = static_cast<const T *>(a.olt_in);
    const uint32_t count = min(a.ctr->count[a.level], a.olt_cap);
    const uint32_t chunks = a.chunks;
    const uint32_t items = count * chunks;  // the host keeps this below 2^32

    WarpBatch<BATCH> b;
    b.rec = T();
    b.kind = KIND_NONE;
    b.nchild = 0;
    b.dwell = 0;
    b.sc = b.r = 1u;
    uint32_t j = 0;
    unsigned long long it = 0, bpx = 0, fpx = 0, dpx = 0;

    for (;;) {
        // items are handed out one at a time: their costs differ by orders
        // of magnitude (a uniform perimeter inside the set runs to max_dwell)
        uint32_t t = 0;
        if (lane == 0)
            t = atomicAdd(&a.ctr->work[a.level], 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= items)
            break;
        const uint32_t region = (chunks == 1u) ? t : t / chunks;
        const T e = olt_in[region];
        const Region g = R::region(e);
        const FView f = BATCH ? view_frame(a.frames, R::frame(e), a.level) : view_single(a);
        const bool query = f.split || !a.exact_last;
        const uint32_t P = perimeter_size(g.w, g.h);
        bool decided = false, uniform = false;
        uint32_t wv = 0;

        if (chunks == 1u) {
            decided = true;
            if (COUNT && lane == 0)
                bpx += P;
            if (query) {
                uniform = warp_perimeter_uniform(f.pm, f.max_dwell, g, lane, &wv, it);
            } else {
                // last level, exact perimeters staged in shared memory: a leaf
                // keeps them and the leaf kernel skips them
                uint32_t dmin = kNone, dmax = 0u;
                for (uint32_t k = lane; k < P; k += 32u) {
                    uint32_t px, py;
                    perimeter_pixel(g, k, px, py);
                    const float2 c = pixel_c(f.pm, px, py);
                    const uint32_t d = dwell(c.x, c.y, f.max_dwell);
                    dmin = min(dmin, d);
                    dmax = max(dmax, d);
                    if (k < kWarpStage)
                        stage[k] = d;
                    else
                        f.map[(size_t)py * f.n + px] = d;  // beyond the stage: write through
                    if (COUNT)
                        it += d;
                }
                dmin = __reduce_min_sync(kFull, dmin);
                dmax = __reduce_max_sync(kFull, dmax);
                uniform = (dmin == dmax);
                wv = dmin;
                if (!uniform) {
                    const uint32_t staged = min(P, kWarpStage);
                    for (uint32_t k = lane; k < staged; k += 32u) {
                        uint32_t px, py;
                        perimeter_pixel(g, k, px, py);
                        f.map[(size_t)py * f.n + px] = stage[k];
                    }
                }
            }
        } else {
            const uint32_t c = t - region * chunks;
            uint4 *st = a.rst_in + region;
            // one frame: chunks cover the level's largest perimeter; a batch
            // caps the chunk count, so a large region takes longer chunks
            const uint32_t CP = BATCH ? max(kChunkPxBatch, ceil_div_u32(P, chunks)) : kChunkPx;
            const uint32_t k0 = min(P, c * CP), k1 = min(P, k0 + CP);
            if (COUNT && lane == 0)
                bpx += k1 - k0;
            if (k0 < k1) {
                if (query)
                    chunk_query<BATCH>(f, g, k0, k1, st, lane, it);
                else
                    chunk_exact(f, g, k0, k1, st, lane, it);
            }
            // the warp that finishes the region's last chunk decides
            uint32_t last = 0;
            if (lane == 0) {
                __threadfence();
                last = (atomicAdd(&st->z, 1u) == chunks - 1u) ? 1u : 0u;
                if (last)
                    __threadfence();
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                uint32_t sx = 0, sy = 0;
                if (lane == 0) {
                    sx = atomicAdd(&st->x, 0u);
                    sy = atomicAdd(&st->y, 0u);
                }
                sx = __shfl_sync(kFull, sx, 0);
                sy = __shfl_sync(kFull, sy, 0);
                uniform = query ? (sy == 0u && sx != kNone) : (sx == sy);
                wv = sx;
                decided = true;
            }
        }

        if (decided) {
            uint32_t kind;
            if (uniform) {
                const uint32_t area = g.w * g.h;
                if (a.fills != nullptr && area > kInPlaceFillArea) {
                    kind = KIND_FILL_LATER;
                } else {
                    fill_rect(f.map, f.n, g, wv, lane, 32u);
                    kind = KIND_FILL;
                }
                if (COUNT && lane == 0) {
                    fpx += area;
                    if (kind == KIND_FILL_LATER)
                        dpx += area;
                }
            } else {
                kind = f.split ? KIND_SPLIT : KIND_LEAF;
            }
            if (lane == j) {
                b.rec = e;
                b.kind = kind;
                b.dwell = wv;
                b.sc = f.child_side;
                b.r = f.r;
                b.nchild = (kind == KIND_SPLIT) ? child_count(g, f.child_side, f.r) : 0u;
            }
            __syncwarp();
            if (++j == 32u) {
                flush_batch<BATCH>(a, b, lane);
                j = 0;
            }
        }
    }
    if (j)
        flush_batch<BATCH>(a, b, lane);
    if (COUNT) {
        it = warp_sum_u64(it);
        bpx = warp_sum_u64(bpx);
        fpx = warp_sum_u64(fpx);
        dpx = warp_sum_u64(dpx);
        if (lane == 0) {
            if (it) {
                atomicAdd(&a.ctr->iterations, it);
                atomicAdd(&a.ctr->level_iters[a.level], it);
            }
            if (bpx)
                atomicAdd(&a.ctr->border_pixels, bpx);
            if (fpx)
                atomicAdd(&a.ctr->fill_pixels, fpx);
            if (dpx)
                atomicAdd(&a.ctr->deferred_fill_pixels, dpx);
        }
    }
}

// ---------------------------------------------------------------------------
// Fill kernel: the bands of the large uniform regions (at most kFillBandPx
// pixels each), one band per warp item, 128-bit stores; pure HBM writes.
// ---------------------------------------------------------------------------
template <bool BATCH>
__global__ void __launch_bounds__(256) fill_kernel(FillArgs f)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nfill = min(f.ctr->fill_count, f.fill_cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t fi = warp; fi < nfill; fi += nwarps) {
        const uint4 e = f.fills[fi];
        const Region g = unpack_region(make_uint2(e.x, e.y));
        if (BATCH) {
            const FrameDesc &d = f.frames[e.w];
            fill_band_warp(d.map, d.n, g, e.z, lane);
        } else {
            fill_band_warp(f.map, f.n, g, e.z, lane);
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled leaf kernel (ASK_FLAG_LEAF_TILED): (leaf, tile) items with block_x x
// block_y tiles, one thread per pixel; persistent grid, warps walk the item
// sequence on their own.
// ---------------------------------------------------------------------------
template <bool COUNT>
__global__ void __launch_bounds__(1024) leaf_kernel(LeafArgs a, uint32_t leaf_cap, uint32_t tiles_x,
                                                    uint32_t tiles_per_leaf)
{
    const uint32_t nleaves = min(a.ctr->leaf_count, leaf_cap);
    const unsigned long long total = (unsigned long long)nleaves * tiles_per_leaf;
    unsigned long long it = 0, lpx = 0;
    for (unsigned long long item = blockIdx.x; item < total; item += gridDim.x) {
        const uint32_t leaf = (uint32_t)(item / tiles_per_leaf);
        const uint32_t t = (uint32_t)(item - (unsigned long long)leaf * tiles_per_leaf);
        const Region g = unpack_region(static_cast<const uint2 *>(a.leaves)[leaf]);
        const uint32_t ty = t / tiles_x, tx = t - ty * tiles_x;
        const uint32_t px = g.x0 + tx * blockDim.x + threadIdx.x;
        const uint32_t py = g.y0 + ty * blockDim.y + threadIdx.y;
        if (px < g.x0 + g.w && py < g.y0 + g.h && !(a.skip_perimeter && on_perimeter(g, px, py))) {
            const float2 c = pixel_c(a.pm, px, py);
            const uint32_t d = dwell(c.x, c.y, a.max_dwell);
            a.map[(size_t)py * a.n + px] = d;
            if (COUNT) {
                it += d;
                ++lpx;
            }
        }
    }
    if (COUNT) {
        it = warp_sum_u64(it);
        lpx = warp_sum_u64(lpx);
        if ((threadIdx.x + threadIdx.y * blockDim.x) % 32u == 0u) {
            if (it) {
                atomicAdd(&a.ctr->iterations, it);
                atomicAdd(&a.ctr->leaf_iters, it);
            }
            if (lpx)
                atomicAdd(&a.ctr->leaf_pixels, lpx);
        }
    }
}

// ---------------------------------------------------------------------------
// Leaf kernel with lane refill (default).  Leaf pixels near the set's
// boundary have dwells from a handful of updates to max_dwell side by side,
// so a warp that owned 32 fixed pixels would idle most lanes while one orbit
// runs on.  Here each warp takes leaves from a device counter and feeds their
// pixels to its lanes one at a time:
//  * every round, each busy lane advances its orbit by one unchecked block
//    (see dwell()); a lane whose block ends escaped, or that has fewer than a
//    block's worth of updates left, parks (saved state, count, pixel) in the
//    warp's buffer in shared memory and takes a new pixel at once;
//  * when 32 orbits are parked, the warp finishes them together, one per
//    lane: a binary search over the parked block finds the exact escape
//    (the block's midpoint state is parked too, so the first halving costs
//    one test; then unchecked quarter, eighth, ... blocks and one test
//    each, the same number of steps on every lane), and the dwells are
//    written.
// ---------------------------------------------------------------------------
constexpr int kRefillWarps = 8;    // warps per CTA
// Resident CTAs per SM: 5 for one frame (48 registers a thread; at 6 CTAs,
// 40 registers, the refill loop spills once the fill warp's code is in the
// kernel, and it measured slower), 4 for a batch (its per-frame lookups need
// up to 64 registers).
constexpr int kRefillMinBlocks = 5;
constexpr int kRefillMinBlocksBatch = 4;
constexpr uint32_t kParkCap = 128; // parked orbits per warp (< 32 + 2 * 32)
constexpr int kLeafUnroll = 32;    // updates per unchecked block (a power of two)

// The output and pixel mapping of the frame a leaf belongs to.
struct LView {
    uint32_t *map;
    PixelMap pm;
    uint32_t n, max_dwell;
};

template <bool BATCH>
__device__ __forceinline__ LView leaf_view(const LeafArgs &a, uint32_t frame)
{
    LView v;
    if (BATCH) {
        const FrameDesc &d = a.frames[frame];
        v.map = d.map;
        v.pm = d.pm;
        v.n = d.n;
        v.max_dwell = d.max_dwell;
    } else {
        v.map = a.map;
        v.pm = a.pm;
        v.n = a.n;
        v.max_dwell = a.max_dwell;
    }
    return v;
}

// Exact dwell of a parked orbit: s.xy = state after d updates, known to
// pass the test, s.zw = the state kLeafUnroll / 2 updates later (the block's
// midpoint), and "escaped, or d >= max_dwell" known to hold kLeafUnroll
// updates later.  Points where escape is not absorbing take the tested loop
// instead.  u = (count, py << 16 | px, frame).
template <bool COUNT, bool BATCH>
__device__ __forceinline__ void finish_parked(const LeafArgs &a, float4 s, uint4 u,
                                              unsigned long long &it)
{
    const LView v = leaf_view<BATCH>(a, u.z);
    const uint32_t px = u.y & 0xffffu, py = u.y >> 16;
    const float2 c = pixel_c(v.pm, px, py);
    uint32_t d = u.x;
    float x = s.x, y = s.y;
    if (!escape_absorbing(c.x, c.y)) {
        while (d < v.max_dwell && z_bounded(x, y)) {
            z_update(x, y, c.x, c.y);
            ++d;
        }
    } else if (d < v.max_dwell) {
        // invariant: count d passes (d < max_dwell) and the predicate holds
        // at d + 2h; halve h until the first count where it holds is d + 1.
        // The first halving uses the block's saved midpoint state.
        {
            const uint32_t h = (uint32_t)kLeafUnroll / 2u;
            const bool hit = (v.max_dwell - d <= h) || !z_bounded(s.z, s.w);
            if (!hit) {
                x = s.z;
                y = s.w;
                d += h;
            }
        }
#pragma unroll
        for (uint32_t h = (uint32_t)kLeafUnroll / 4u; h >= 1u; h >>= 1) {
            float tx = x, ty = y;
#pragma unroll
            for (uint32_t k = 0; k < h; ++k)
                z_update(tx, ty, c.x, c.y);
            const bool hit = (v.max_dwell - d <= h) || !z_bounded(tx, ty);
            if (!hit) {
                x = tx;
                y = ty;
                d += h;
            }
        }
        d += 1u;
    }
    v.map[(size_t)py * v.n + px] = d;
    if (COUNT)
        it += d;
}

// Deferred fills ride along the leaf pass.  The last warp of every CTA
// starts as a fill warp: it takes bands of the fill list (at most
// kFillBandPx pixels each, 128-bit stores) from a counter until none are
// left, then joins the leaf work; every warp that runs out of leaves helps
// with the bands still left.  The HBM writes so proceed beside the FP32 work
// of the other warps instead of in a kernel of their own (the bands and the
// leaves are disjoint pixels), and the fill code sits outside the refill
// loop, adding nothing to its registers.
template <bool BATCH>
__device__ __forceinline__ void drain_fills(const LeafArgs &a, uint32_t lane)
{
    const uint32_t nfill = min(a.ctr->fill_count, a.fill_cap);
    for (;;) {
        uint32_t fi = 0;
        if (lane == 0)
            fi = atomicAdd(&a.ctr->fill_work, 1u);
        fi = __shfl_sync(kFull, fi, 0);
        if (fi >= nfill)
            return;
        const uint4 e = a.fills[fi];
        const Region g = unpack_region(make_uint2(e.x, e.y));
        if (BATCH) {
            const FrameDesc &d = a.frames[e.w];
            fill_band_warp(d.map, d.n, g, e.z, lane);
        } else {
            fill_band_warp(a.map, a.n, g, e.z, lane);
        }
    }
}

// floor(q / w) for q < 2^22 given inv_w = 1/w rounded to float: (q + 1/2)/w
// lies at least 1/(2w) away from an integer, far more than the rounding of
// the two float operations, so truncation gives the exact quotient.
__device__ __forceinline__ uint32_t rows_in(uint32_t q, float inv_w)
{
    return __float2uint_rz(__fmul_rz(__uint2float_rn(q) + 0.5f, inv_w));
}

// One orbit slot of a lane.
struct Slot {
    float x, y, cr, ci;
    uint32_t d, pix;  // count, pixel (py << 16 | px)
    uint32_t lim;     // a whole unchecked block may run while d < lim
    bool busy;
};

// lim = max_dwell - kLeafUnroll + 1 where escape is absorbing (the block
// stays within max_dwell), else 0 (such points go straight to the tested
// loop of finish_parked).
__device__ __forceinline__ void slot_start(Slot &o, const PixelMap &pm, uint32_t md, uint32_t px,
                                           uint32_t py)
{
    const float2 c = pixel_c(pm, px, py);
    o.cr = c.x;
    o.ci = c.y;
    o.x = 0.0f;
    o.y = 0.0f;
    o.d = 0;
    o.pix = (py << 16) | px;
    o.lim = (escape_absorbing(c.x, c.y) && md >= (uint32_t)kLeafUnroll) ? md - (uint32_t)kLeafUnroll + 1u
                                                                         : 0u;
    o.busy = true;
}

// Each lane carries two independent orbits, so one round's bookkeeping
// (votes, refills, parking) serves two blocks of updates, and the two update
// chains interleave.  All lanes of a warp work on the same leaf (the same
// frame) at a time; parked orbits remember their frame.
template <bool COUNT, bool BATCH>
__global__ void __launch_bounds__(kRefillWarps * 32, BATCH ? kRefillMinBlocksBatch : kRefillMinBlocks)
    leaf_refill_kernel(LeafArgs a)
{
    using R = Rec<BATCH>;
    using T = typename R::T;
    __shared__ float4 park_s[kRefillWarps][kParkCap];  // saved state at the block's start and midpoint
    __shared__ uint4 park_u[kRefillWarps][kParkCap];   // count, pixel, frame
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    if (a.fills != nullptr && wib == kRefillWarps - 1u)
        drain_fills<BATCH>(a, lane);  // the CTA's fill warp
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *qs = park_s[wib];
    uint4 *qu = park_u[wib];
    uint32_t parked = 0;  // warp-uniform

    const T *leaves = static_cast<const T *>(a.leaves);
    const uint32_t nleaves = min(a.ctr->leaf_count, a.leaf_cap);
    const uint32_t K = (uint32_t)kLeafUnroll;
    // the warp's current leaf: the part still to hand out, as a row-major cursor
    uint32_t rem = 0, row0 = 0, col0 = 0, ox = 0, oy = 0, cw = 1, frame = 0;
    float inv_cw = 1.0f;
    LView lv = leaf_view<BATCH>(a, 0u);
    bool more = true;
    Slot s0, s1;
    s0.busy = s1.busy = false;
    s0.x = s0.y = s0.cr = s0.ci = s1.x = s1.y = s1.cr = s1.ci = 0.0f;
    s0.d = s1.d = s0.pix = s1.pix = 0;
    s0.lim = s1.lim = 0;
    uint32_t f0 = 0, f1 = 0;  // frames of the slots' orbits
    unsigned long long it = 0, lpx = 0;

    for (;;) {
        // ---- refill idle slots: slot 0 of the idle lanes, then slot 1
        unsigned i0 = __ballot_sync(kFull, !s0.busy), i1 = __ballot_sync(kFull, !s1.busy);
        while ((i0 | i1) && more) {
            if (rem == 0) {
                uint32_t li = 0;
                if (lane == 0)
                    li = atomicAdd(&a.ctr->leaf_work, 1u);
                li = __shfl_sync(kFull, li, 0);
                if (li >= nleaves) {
                    more = false;
                    break;
                }
                const T e = leaves[li];
                const Region g = R::region(e);
                frame = R::frame(e);
                if (BATCH)
                    lv = leaf_view<BATCH>(a, frame);
                if (a.skip_perimeter) {
                    // only the interior; a leaf of side <= 2 is all perimeter
                    cw = g.w > 2u ? g.w - 2u : 1u;
                    rem = (g.w > 2u && g.h > 2u) ? (g.w - 2u) * (g.h - 2u) : 0u;
                    ox = g.x0 + 1u;
                    oy = g.y0 + 1u;
                } else {
                    cw = g.w;
                    rem = g.w * g.h;
                    ox = g.x0;
                    oy = g.y0;
                }
                row0 = col0 = 0;
                inv_cw = 1.0f / (float)cw;
                continue;
            }
            const uint32_t n0 = (uint32_t)__popc(i0);
            const uint32_t idle = n0 + (uint32_t)__popc(i1);
            const uint32_t take = min(idle, rem);
            const uint32_t r0 = (uint32_t)__popc(i0 & lt_mask);
            const uint32_t r1 = n0 + (uint32_t)__popc(i1 & lt_mask);
            if (!s0.busy && r0 < take) {
                const uint32_t q = col0 + r0, dr = rows_in(q, inv_cw);
                slot_start(s0, lv.pm, lv.max_dwell, ox + q - dr * cw, oy + row0 + dr);
                f0 = frame;
            }
            if (!s1.busy && r1 < take) {
                const uint32_t q = col0 + r1, dr = rows_in(q, inv_cw);
                slot_start(s1, lv.pm, lv.max_dwell, ox + q - dr * cw, oy + row0 + dr);
                f1 = frame;
            }
            {
                const uint32_t q = col0 + take, dr = rows_in(q, inv_cw);
                col0 = q - dr * cw;
                row0 += dr;
            }
            rem -= take;
            if (take == idle)
                break;  // every slot busy
            i0 = __ballot_sync(kFull, !s0.busy);
            i1 = __ballot_sync(kFull, !s1.busy);
        }
        // slots stay idle only once the leaves have run out
        if (!more && !__any_sync(kFull, s0.busy || s1.busy))
            break;

        // ---- one unchecked block on both slots (results of a slot that is
        //      idle or parks this round are not used)
        const float sx0 = s0.x, sy0 = s0.y, sx1 = s1.x, sy1 = s1.y;
#pragma unroll
        for (int k = 0; k < kLeafUnroll / 2; ++k) {
            z_update(s0.x, s0.y, s0.cr, s0.ci);
            z_update(s1.x, s1.y, s1.cr, s1.ci);
        }
        const float mx0 = s0.x, my0 = s0.y, mx1 = s1.x, my1 = s1.y;  // midpoint states
#pragma unroll
        for (int k = 0; k < kLeafUnroll / 2; ++k) {
            z_update(s0.x, s0.y, s0.cr, s0.ci);
            z_update(s1.x, s1.y, s1.cr, s1.ci);
        }
        bool park0 = false, park1 = false;
        if (s0.busy) {
            if (s0.d < s0.lim && z_bounded(s0.x, s0.y))
                s0.d += K;
            else
                park0 = true;  // escaped in this block, tail below max_dwell, or |c| near 2
        }
        if (s1.busy) {
            if (s1.d < s1.lim && z_bounded(s1.x, s1.y))
                s1.d += K;
            else
                park1 = true;
        }

        // ---- park finished orbits (state before this block); finish the
        //      top 32 parked orbits whenever there are 32
        const unsigned p0 = __ballot_sync(kFull, park0), p1 = __ballot_sync(kFull, park1);
        if (p0 | p1) {
            const uint32_t n0 = (uint32_t)__popc(p0);
            if (park0) {
                const uint32_t slot = parked + (uint32_t)__popc(p0 & lt_mask);
                qs[slot] = make_float4(sx0, sy0, mx0, my0);
                qu[slot] = make_uint4(s0.d, s0.pix, f0, 0u);
                s0.busy = false;
            }
            if (park1) {
                const uint32_t slot = parked + n0 + (uint32_t)__popc(p1 & lt_mask);
                qs[slot] = make_float4(sx1, sy1, mx1, my1);
                qu[slot] = make_uint4(s1.d, s1.pix, f1, 0u);
                s1.busy = false;
            }
            parked += n0 + (uint32_t)__popc(p1);
            __syncwarp();
            while (parked >= 32u) {
                parked -= 32u;
                const float4 sv = qs[parked + lane];
                const uint4 uv = qu[parked + lane];
                __syncwarp();
                finish_parked<COUNT, BATCH>(a, sv, uv, it);
                if (COUNT)
                    ++lpx;
            }
        }
    }
    if (a.fills != nullptr)
        drain_fills<BATCH>(a, lane);
    // ---- the orbits still parked
    if (lane < parked) {
        finish_parked<COUNT, BATCH>(a, qs[lane], qu[lane], it);
        if (COUNT)
            ++lpx;
    }
    if (COUNT) {
        it = warp_sum_u64(it);
        lpx = warp_sum_u64(lpx);
        if (lane == 0) {
            if (it) {
                atomicAdd(&a.ctr->iterations, it);
                atomicAdd(&a.ctr->leaf_iters, it);
            }
            if (lpx)
                atomicAdd(&a.ctr->leaf_pixels, lpx);
        }
    }
}

// Level-0 records and counters of a batch: block f writes frame f's
// axis0 x axis0 initial regions at its offset; block 0 zeroes the counters.
__global__ void init_batch_kernel(uint4 *__restrict__ olt0, uint4 *__restrict__ rst0,
                                  DevCounters *ctr, const FrameDesc *frames, uint32_t total0)
{
    const uint32_t f = blockIdx.x;
    if (f == 0) {
        uint32_t *w = reinterpret_cast<uint32_t *>(ctr);
        const uint32_t words = (uint32_t)(sizeof(DevCounters) / sizeof(uint32_t));
        const uint32_t err_word = (uint32_t)(offsetof(DevCounters, error) / sizeof(uint32_t));
        for (uint32_t k = threadIdx.x; k < words; k += blockDim.x)
            if (k != err_word)
                w[k] = (k == 0u) ? total0 : 0u;  // word 0 is count[0]
    }
    const FrameDesc &d = frames[f];
    const uint32_t per = d.axis0 * d.axis0;
    for (uint32_t k = threadIdx.x; k < per; k += blockDim.x) {
        const uint32_t gx = k % d.axis0, gy = k / d.axis0;
        const uint32_t x0 = gx * d.s0, y0 = gy * d.s0;
        const uint2 rec = pack_region(x0, y0, min(d.s0, d.n - x0), min(d.s0, d.n - y0));
        olt0[d.olt0_offset + k] = make_uint4(rec.x, rec.y, f, 0u);
        if (rst0 != nullptr)
            rst0[d.olt0_offset + k] = make_uint4(kNone, 0u, 0u, 0u);
    }
}

template <typename K>
int persistent_grid(K kernel, int threads, size_t smem, int sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

}  // namespace

cudaError_t launch_exhaustive(uint32_t *map, uint32_t n, PixelMap pm, uint32_t max_dwell,
                              uint32_t bx, uint32_t by, bool count, DevCounters *ctr,
                              cudaStream_t s)
{
    const uint32_t tiles_x = (n + bx - 1) / bx, tiles_y = (n + by - 1) / by;
    const dim3 block(bx, by);
    const unsigned long long tiles = (unsigned long long)tiles_x * tiles_y;
    if (tiles > 0x7fffffffull)
        return cudaErrorInvalidConfiguration;
    if (count)
        exhaustive_kernel<true><<<(unsigned)tiles, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
    else
        exhaustive_kernel<false><<<(unsigned)tiles, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
    return cudaGetLastError();
}

cudaError_t launch_init(uint2 *olt0, uint4 *rst0, DevCounters *ctr, uint32_t n, uint32_t s0,
                        uint32_t axis0, uint32_t row0, uint32_t rows, cudaStream_t s)
{
    const uint32_t total = axis0 * rows;
    uint32_t blocks = (total + 255u) / 256u;
    if (blocks < 1)
        blocks = 1;
    if (blocks > 4096)
        blocks = 4096;
    init_kernel<<<blocks, 256, 0, s>>>(olt0, rst0, ctr, n, s0, axis0, row0, rows);
    return cudaGetLastError();
}

template <bool COUNT, bool BATCH>
static void level_launch(const LevelArgs &a, int sms, cudaStream_t s)
{
    const size_t smem = (size_t)(256 / 32) * kWarpStage * sizeof(uint32_t);
    const int grid = persistent_grid(level_kernel<COUNT, BATCH>, 256, smem, sms);
    level_kernel<COUNT, BATCH><<<grid, 256, smem, s>>>(a);
}

cudaError_t launch_level(const LevelArgs &a, bool count, bool batch, int sms, cudaStream_t s)
{
    if (batch) {
        if (count)
            level_launch<true, true>(a, sms, s);
        else
            level_launch<false, true>(a, sms, s);
    } else {
        if (count)
            level_launch<true, false>(a, sms, s);
        else
            level_launch<false, false>(a, sms, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_fill(const FillArgs &f, bool batch, int sms, cudaStream_t s)
{
    if (batch) {
        const int grid = persistent_grid(fill_kernel<true>, 256, 0, sms);
        fill_kernel<true><<<grid, 256, 0, s>>>(f);
    } else {
        const int grid = persistent_grid(fill_kernel<false>, 256, 0, sms);
        fill_kernel<false><<<grid, 256, 0, s>>>(f);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_batch(uint4 *olt0, uint4 *rst0, DevCounters *ctr, const FrameDesc *frames,
                              uint32_t nframes, uint32_t total0, cudaStream_t s)
{
    init_batch_kernel<<<nframes, 256, 0, s>>>(olt0, rst0, ctr, frames, total0);
    return cudaGetLastError();
}

template <bool COUNT, bool BATCH>
static void refill_launch(const LeafArgs &a, int sms, cudaStream_t s)
{
    const int threads = kRefillWarps * 32;
    const int grid = persistent_grid(leaf_refill_kernel<COUNT, BATCH>, threads, 0, sms);
    leaf_refill_kernel<COUNT, BATCH><<<grid, threads, 0, s>>>(a);
}

cudaError_t launch_leaf(const LeafArgs &a, uint32_t bx, uint32_t by, bool count, bool tiled,
                        bool batch, int sms, cudaStream_t s)
{
    if (batch) {
        if (tiled)
            return cudaErrorInvalidValue;
        if (count)
            refill_launch<true, true>(a, sms, s);
        else
            refill_launch<false, true>(a, sms, s);
        return cudaGetLastError();
    }
    if (!tiled) {
        if (count)
            refill_launch<true, false>(a, sms, s);
        else
            refill_launch<false, false>(a, sms, s);
        return cudaGetLastError();
    }
    const uint32_t tiles_x = (a.side + bx - 1) / bx, tiles_y = (a.side + by - 1) / by;
    const dim3 block(bx, by);
    const int threads = (int)(bx * by);
    if (count) {
        const int grid = persistent_grid(leaf_kernel<true>, threads, 0, sms);
        leaf_kernel<true><<<grid, block, 0, s>>>(a, a.leaf_cap, tiles_x, tiles_x * tiles_y);
    } else {
        const int grid = persistent_grid(leaf_kernel<false>, threads, 0, sms);
        leaf_kernel<false><<<grid, block, 0, s>>>(a, a.leaf_cap, tiles_x, tiles_x * tiles_y);
    }
    return cudaGetLastError();
}

}  // namespace ask
