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
//    (kChunkPxBatch in a batch; half of kChunkPx at a level with few items)
//    perimeter pixels of a large region (several warps per region: the MBR
//    mapping of Sec. 4.3.2 applied to the query), one warp per item;
//  * each region table is filled from both ends (regions whose centre orbit
//    stays bounded for a short probe from the front), so a level kernel
//    takes its longest regions first; the leaf list likewise;
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
#include "ask_work.cuh"

namespace ask {

namespace {

constexpr uint32_t kWarpStage = 512;  // staged perimeter pixels per warp (exact last level)
constexpr int kOrderProbe = 64;       // updates of the order probe (region_probe)

enum : uint32_t { KIND_NONE = 0, KIND_FILL = 1, KIND_SPLIT = 2, KIND_LEAF = 3, KIND_FILL_LATER = 4 };

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

// Order probe of a region (the order in which the region tables and the
// leaf list are taken): does the orbit of the region's centre pixel stay
// bounded for kOrderProbe updates?  Regions inside the set, whose perimeter
// orbits all run to max_dwell, and leaves holding such orbits answer yes;
// taking them first lets a kernel's warps run out of work together instead
// of ending on a wave of its longest items.  Only the order of the work
// depends on it, never a dwell.  Unchecked updates: an escaped orbit runs to
// inf or NaN and fails the test; where escape is not absorbing the answer is
// no.
__device__ __forceinline__ bool region_probe(const PixelMap &pm, const Region &g)
{
    const float2 c = pixel_c(pm, g.x0 + g.w / 2u, g.y0 + g.h / 2u);
    if (!escape_absorbing(c.x, c.y))
        return false;
    float x = 0.0f, y = 0.0f;
#pragma unroll 8
    for (int k = 0; k < kOrderProbe; ++k)
        z_update(x, y, c.x, c.y);
    return z_bounded(x, y);
}

// Zero the per-render counters (the latched error word is kept), write the
// level-0 OLT (the axis0 x axis0 non-empty initial regions of side s0) and,
// when level 0 is queried in chunks, its per-region state.  `order` (one
// block only): regions whose probe stays bounded from slot 0 up (count[0]),
// the others from slot total - 1 down (back[0]); else in grid order.
__global__ void init_kernel(uint2 *__restrict__ olt0, uint4 *__restrict__ rst0, DevCounters *ctr,
                            uint32_t n, uint32_t s0, uint32_t axis0, uint32_t row0, uint32_t rows,
                            PixelMap pm, uint32_t order)
{
    __shared__ uint32_t s_front, s_back;
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
    if (order) {
        if (threadIdx.x == 0) {
            s_front = 0;
            s_back = 0;
        }
        __syncthreads();  // also orders the counter words above before the totals below
    }
    for (uint32_t k = tid; k < total; k += stride) {
        const uint32_t gx = k % axis0, gy = row0 + k / axis0;
        const uint32_t x0 = gx * s0, y0 = gy * s0;
        const uint2 rec = pack_region(x0, y0, min(s0, n - x0), min(s0, n - y0));
        uint32_t slot = k;
        if (order)
            slot = region_probe(pm, unpack_region(rec)) ? atomicAdd(&s_front, 1u)
                                                        : total - 1u - atomicAdd(&s_back, 1u);
        olt0[slot] = rec;
        if (rst0 != nullptr)
            rst0[slot] = make_uint4(kNone, 0u, 0u, 0u);
    }
    if (order) {
        __syncthreads();
        if (threadIdx.x == 0 && ctr != nullptr) {
            ctr->count[0] = s_front;
            ctr->back[0] = s_back;
        }
    }
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

// Pixel map of a region record's frame.
template <bool BATCH>
__device__ __forceinline__ PixelMap record_pm(const LevelArgs &a, const typename Rec<BATCH>::T &e)
{
    return BATCH ? a.frames[Rec<BATCH>::frame(e)].pm : a.pm;
}

template <bool BATCH>
__device__ __forceinline__ void flush_batch(const LevelArgs &a, WarpBatch<BATCH> &b, uint32_t lane)
{
    using R = Rec<BATCH>;
    using T = typename R::T;
    T *leaves = static_cast<T *>(a.leaves);
    T *olt_out = static_cast<T *>(a.olt_out);
    DevCounters *ctr = a.ctr;
    const unsigned lt = (1u << lane) - 1u;
    // leaves: ballot + popc gives each leaf its slot, from the front of the
    // list for the leaves whose probe stayed bounded, from the back for the
    // others
    const unsigned leaf_mask = __ballot_sync(kFull, b.kind == KIND_LEAF);
    if (leaf_mask) {
        const bool is_leaf = b.kind == KIND_LEAF;
        const bool heavy = is_leaf && region_probe(record_pm<BATCH>(a, b.rec), R::region(b.rec));
        const unsigned hm = __ballot_sync(kFull, heavy), lm = leaf_mask & ~hm;
        uint32_t hb = 0, lb = 0;
        if (lane == 0) {
            if (hm)
                hb = atomicAdd(&ctr->leaf_count, (uint32_t)__popc(hm));
            if (lm)
                lb = atomicAdd(&ctr->leaf_light, (uint32_t)__popc(lm));
        }
        hb = __shfl_sync(kFull, hb, 0);
        lb = __shfl_sync(kFull, lb, 0);
        if (is_leaf) {
            const uint32_t k = heavy ? hb + (uint32_t)__popc(hm & lt) : lb + (uint32_t)__popc(lm & lt);
            if (k < a.leaf_cap)
                leaves[heavy ? k : a.leaf_cap - 1u - k] = b.rec;
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
    // children: each lane probes its region's children (at most 64; a region
    // with more sends them all to the front); warp inclusive scans of the
    // counts going to the front and to the back of the next level's table,
    // one atomicAdd for each
    const unsigned split_any = __ballot_sync(kFull, b.nchild != 0u);
    if (split_any) {
        const Region g = R::region(b.rec);
        unsigned long long heavy = ~0ull;  // bit j: child j goes to the front
        uint32_t nh = b.nchild;
        if (b.nchild != 0u && b.nchild <= 64u) {
            const PixelMap pm = record_pm<BATCH>(a, b.rec);
            heavy = 0ull;
            nh = 0;
            for (uint32_t j = 0; j < b.nchild; ++j)
                if (region_probe(pm, unpack_region(child_region(g, b.sc, b.r, j)))) {
                    heavy |= 1ull << j;
                    ++nh;
                }
        }
        const uint32_t nl = b.nchild - nh;
        uint32_t ih = nh, il = nl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t vh = __shfl_up_sync(kFull, ih, o), vl = __shfl_up_sync(kFull, il, o);
            if (lane >= (uint32_t)o) {
                ih += vh;
                il += vl;
            }
        }
        const uint32_t th = __shfl_sync(kFull, ih, 31), tl = __shfl_sync(kFull, il, 31);
        uint32_t hb = 0, lb = 0;
        if (lane == 0) {
            if (th)
                hb = atomicAdd(&ctr->count[a.level + 1], th);
            if (tl)
                lb = atomicAdd(&ctr->back[a.level + 1], tl);
        }
        hb = __shfl_sync(kFull, hb, 0) + ih - nh;  // this lane's first front index
        lb = __shfl_sync(kFull, lb, 0) + il - nl;  // and first back index
        for (uint32_t j = 0; j < b.nchild; ++j) {
            const bool front = (heavy >> (j & 63u)) & 1ull;
            const uint32_t k = front ? hb++ : lb++;
            if (k < a.out_cap) {
                const uint32_t slot = front ? k : a.out_cap - 1u - k;
                olt_out[slot] = R::child(b.rec, child_region(g, b.sc, b.r, j));
                if (a.next_chunks > 1u)
                    a.rst_out[slot] = make_uint4(kNone, 0u, 0u, 0u);
            } else {
                atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
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
    // regions from the front of the table first, then those from the back
    const uint32_t front = min(a.ctr->count[a.level], a.in_cap);
    const uint32_t count = front + min(a.ctr->back[a.level], a.in_cap - front);
    if (blockIdx.x == 0 && threadIdx.x == 0 &&
        (unsigned long long)a.ctr->count[a.level] + a.ctr->back[a.level] > a.in_cap)
        atomicOr(&a.ctr->error, ERR_OLT_OVERFLOW);
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
        const uint32_t li = (chunks == 1u) ? t : t / chunks;  // in the order taken
        const uint32_t region = table_slot(li, front, a.in_cap);  // its slot
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
                uniform = warp_perimeter_uniform<BATCH ? kQueryRoundBatch : kQueryRound, !BATCH || kBatchShortWhole>(
                    f.pm, f.max_dwell, g, lane, &wv, it);
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
            const uint32_t c = t - li * chunks;
            uint4 *st = a.rst_in + region;
            // one frame: chunks cover the level's largest perimeter; a batch
            // caps the chunk count, so a large region takes longer chunks
            const uint32_t CP = BATCH ? max(kChunkPxBatch, ceil_div_u32(P, chunks)) : a.chunk_px;
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
    uint32_t front, nleaves;
    leaf_extent(a.ctr, leaf_cap, front, nleaves);
    const unsigned long long total = (unsigned long long)nleaves * tiles_per_leaf;
    unsigned long long it = 0, lpx = 0;
    for (unsigned long long item = blockIdx.x; item < total; item += gridDim.x) {
        const uint32_t leaf = (uint32_t)(item / tiles_per_leaf);
        const uint32_t t = (uint32_t)(item - (unsigned long long)leaf * tiles_per_leaf);
        const Region g = unpack_region(static_cast<const uint2 *>(a.leaves)[table_slot(leaf, front, leaf_cap)]);
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
// Leaf kernel (default): a coherent first pass over fresh pixels, then lane
// refill for the orbits that survive it.
//
// Leaf pixels lie near the set's boundary: their dwells run from a handful
// of updates to max_dwell side by side (at n = 16384 the median leaf pixel
// escapes after 19 updates, 71% within 32, while the 5% that reach max_dwell
// hold two thirds of the updates).  A warp that owned 32 fixed pixels would
// idle most lanes while one orbit runs on, so each warp takes leaves from a
// device counter and works in two stages:
//  * pre-pass: 32 fresh pixels at a time, one per lane, all lanes in
//    lockstep, run their first kPrePass updates in unchecked blocks of
//    kPreBlock with one test per block (see dwell()).  An orbit that escapes
//    there is resolved on the spot by a binary search over its last block
//    and written; the others are pushed, with their state, onto the warp's
//    ring of survivors in shared memory.  Most pixels end here, with no
//    per-pixel bookkeeping beyond the lane they run on;
//  * refill loop over the survivors: each lane carries two orbits; every
//    round each orbit runs one unchecked block of kLeafUnroll updates; an
//    orbit that escaped (or has less than a block left) parks its saved
//    state in the warp's park buffer and its slot takes the next survivor
//    from the ring at once (the pre-pass tops the ring up when it runs
//    short);
//  * when 32 orbits are parked, the warp finishes them together, one per
//    lane: a binary search over the parked block finds the exact escape (the
//    block's midpoint state is parked too, so the first halving costs one
//    test; then unchecked quarter, eighth, ... blocks and one test each, the
//    same number of steps on every lane), and the dwells are written;
//  * the leaves are taken in the order of the list, whose front holds the
//    leaves whose centre orbit the level kernel's probe found bounded (most
//    long orbits), so the warps end on short orbits; once the list has run
//    out and a warp's orbits fit in one slot per lane, slot 1 folds into
//    slot 0 and the last rounds update one orbit per lane.
// ---------------------------------------------------------------------------
// The leaf kernel over the leaf list of a launch chain.  Each lane of the
// refill loop carries two independent orbits, so one round's bookkeeping
// (votes, refills, parking) serves two blocks of updates, and the two update
// chains interleave.  Parked orbits and ring entries remember their frame.
template <bool COUNT, bool BATCH>
__global__ void __launch_bounds__(kRefillWarps * 32, BATCH ? kRefillMinBlocksBatch : kRefillMinBlocks)
    leaf_refill_kernel(LeafArgs a)
{
    __shared__ float4 park_s[kRefillWarps][kParkCap];  // saved state at the block's start and midpoint
    __shared__ uint4 park_u[kRefillWarps][kParkCap];   // count, pixel, frame
    __shared__ float4 ring_s[kRefillWarps][kRingCap];  // survivor state and c
    __shared__ uint4 ring_u[kRefillWarps][kRingCap];   // count, pixel, frame, block limit
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    if (a.fills != nullptr && wib == kRefillWarps - 1u)
        drain_fills<BATCH>(a, lane);  // the CTA's fill warp
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *qs = park_s[wib];
    uint4 *qu = park_u[wib];
    float4 *rs = ring_s[wib];
    uint4 *ru = ring_u[wib];
    uint32_t parked = 0;             // warp-uniform
    uint32_t ring_h = 0, ring_n = 0;  // warp-uniform: first entry, entries

    LeafList<BATCH> src;
    src.leaves = static_cast<const typename Rec<BATCH>::T *>(a.leaves);
    src.cap = a.leaf_cap;
    leaf_extent(a.ctr, a.leaf_cap, src.front, src.total);
    uint32_t srcst = SRC_MORE;
    LeafCursor lc;
    lc.rem = lc.row0 = lc.col0 = lc.ox = lc.oy = lc.frame = 0;
    lc.cw = 1;
    lc.inv_cw = 1.0f;
    Slot s0, s1;
    s0.busy = s1.busy = false;
    s0.x = s0.y = s0.cr = s0.ci = s1.x = s1.y = s1.cr = s1.ci = 0.0f;
    s0.d = s1.d = s0.pix = s1.pix = 0;
    s0.lim = s1.lim = 0;
    uint32_t f0 = 0, f1 = 0;  // frames of the slots' orbits
    unsigned long long it = 0, lpx = 0;

    for (;;) {
        // refill idle slots from the ring, topping it up with pre-passes
        // while it holds fewer survivors than idle slots (at most 32)
        const unsigned i0 = __ballot_sync(kFull, !s0.busy), i1 = __ballot_sync(kFull, !s1.busy);
        if (i0 | i1) {
            const uint32_t want = min((uint32_t)(__popc(i0) + __popc(i1)), 32u);
            while (ring_n < want && srcst == SRC_MORE)
                pre_pass<COUNT, BATCH>(a, src, lc, srcst, rs, ru, ring_h, ring_n, lane, lt_mask, it,
                                       lpx);
            refill_from_ring(s0, s1, f0, f1, rs, ru, ring_h, ring_n, i0, i1, lane, lt_mask);
        }
        // once the leaves have run out and the orbits left fit in one slot
        // per lane, the tail runs on slot 0 alone
        if (srcst != SRC_MORE &&
            ring_n + (uint32_t)__popc(__ballot_sync(kFull, s0.busy)) +
                    (uint32_t)__popc(__ballot_sync(kFull, s1.busy)) <= 32u)
            break;
        refill_round<COUNT, BATCH>(a, s0, s1, f0, f1, qs, qu, parked, lane, lt_mask, it, lpx);
    }
    fold_slot1(s1, f1, rs, ru, ring_h, ring_n, lt_mask);
    refill_from_ring(s0, s1, f0, f1, rs, ru, ring_h, ring_n, __ballot_sync(kFull, !s0.busy), 0u, lane,
                     lt_mask);
    while (__any_sync(kFull, s0.busy))
        refill_round<COUNT, BATCH, false>(a, s0, s1, f0, f1, qs, qu, parked, lane, lt_mask, it, lpx);
    if (a.fills != nullptr)
        drain_fills<BATCH>(a, lane);
    // the orbits still parked
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
                        uint32_t axis0, uint32_t row0, uint32_t rows, cudaStream_t s,
                        const PixelMap *order)
{
    const uint32_t total = axis0 * rows;
    if (order != nullptr && olt0 != nullptr && total <= kInitOrderMax) {
        init_kernel<<<1, 1024, 0, s>>>(olt0, rst0, ctr, n, s0, axis0, row0, rows, *order, 1u);
        return cudaGetLastError();
    }
    uint32_t blocks = (total + 255u) / 256u;
    if (blocks < 1)
        blocks = 1;
    if (blocks > 4096)
        blocks = 4096;
    init_kernel<<<blocks, 256, 0, s>>>(olt0, rst0, ctr, n, s0, axis0, row0, rows, PixelMap{}, 0u);
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
