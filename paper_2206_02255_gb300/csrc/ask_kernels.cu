// ask_kernels.cu -- exhaustive kernel and the Adaptive Serial Kernels (ASK)
// pipeline: init, one level kernel per subdivision depth, leaf kernel.
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
//  * level kernels are persistent (a grid sized to the SM count) and read the
//    region count from device memory, so no depth needs a host round trip
//    and the whole sequence is a fixed chain of launches;
//  * perimeter dwells are staged in shared memory; a uniform perimeter is
//    detected with warp min/max reductions (__reduce_min/max_sync);
//  * deep levels run one warp per region and compact their appends per warp:
//    each lane keeps the outcome of one region the warp processed, then one
//    atomicAdd per list reserves space for up to 32 regions at once (the
//    block-scan + single atomic alternative of Sec. 5.3.1, at warp scope);
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
constexpr uint32_t kWarpStage = 512;     // staged perimeter pixels per warp
constexpr uint32_t kCtaStageMax = 16384; // staged perimeter pixels per CTA

enum : uint32_t { KIND_NONE = 0, KIND_FILL = 1, KIND_SPLIT = 2, KIND_LEAF = 3 };

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

// Zero the per-render counters (the latched error word is kept) and write
// the level-0 OLT: the axis0 x axis0 non-empty initial regions of side s0.
__global__ void init_kernel(uint2 *__restrict__ olt0, DevCounters *ctr, uint32_t n, uint32_t s0,
                            uint32_t axis0)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t total = axis0 * axis0;
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
        const uint32_t gx = k % axis0, gy = k / axis0;
        const uint32_t x0 = gx * s0, y0 = gy * s0;
        olt0[k] = pack_region(x0, y0, min(s0, n - x0), min(s0, n - y0));
    }
}

// ---------------------------------------------------------------------------
// Level kernel, one warp per region.
// ---------------------------------------------------------------------------
struct WarpBatch {
    uint2 rec;       // lane j: OLT record of the j-th region of the batch
    uint32_t kind;   // KIND_*
    uint32_t nchild; // children of a splitting region
};

// Reserve list space for the batch with one atomicAdd per list and write the
// leaf records and child records.  Called by all 32 lanes.
__device__ __forceinline__ void flush_batch(const LevelArgs &a, WarpBatch &b, uint32_t lane)
{
    DevCounters *ctr = a.ctr;
    // leaves: ballot + popc gives each leaf its slot
    const unsigned leaf_mask = __ballot_sync(kFull, b.kind == KIND_LEAF);
    if (leaf_mask) {
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(&ctr->leaf_count, (uint32_t)__popc(leaf_mask));
        base = __shfl_sync(kFull, base, 0);
        if (b.kind == KIND_LEAF) {
            const uint32_t slot = base + (uint32_t)__popc(leaf_mask & ((1u << lane) - 1u));
            if (slot < a.leaf_cap)
                a.leaves[slot] = b.rec;
            else
                atomicOr(&ctr->error, ERR_LEAF_OVERFLOW);
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
            const Region g = unpack_region(b.rec);
            const uint32_t first = base + incl - b.nchild;
            for (uint32_t j = 0; j < b.nchild; ++j) {
                const uint32_t slot = first + j;
                if (slot < a.olt_cap)
                    a.olt_out[slot] = child_region(g, a.child_side, a.r, j);
                else
                    atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
            }
        }
    }
    const unsigned fill_mask = __ballot_sync(kFull, b.kind == KIND_FILL);
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

template <bool COUNT>
__global__ void __launch_bounds__(256) level_warp_kernel(LevelArgs a, uint32_t olt_in_cap)
{
    extern __shared__ uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *stage = smem + (threadIdx.x >> 5) * kWarpStage;
    const uint32_t count = min(a.ctr->count[a.level], olt_in_cap);

    WarpBatch b;
    b.rec = make_uint2(0, 0);
    b.kind = KIND_NONE;
    b.nchild = 0;
    uint32_t j = 0;
    unsigned long long it = 0, bpx = 0, fpx = 0;

    for (;;) {
        // regions are handed out one at a time: their costs differ by orders
        // of magnitude (a uniform perimeter inside the set runs to max_dwell)
        uint32_t idx = 0;
        if (lane == 0)
            idx = atomicAdd(&a.ctr->work[a.level], 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= count)
            break;
        const uint2 e = a.olt_in[idx];
        const Region g = unpack_region(e);
        uint32_t kind;
        if (a.split || !a.exact_last) {
            // only "uniform, and to what" matters: stop at the first difference
            // (a leaf's pixels, perimeter included, are then all computed by
            // the leaf kernel)
            uint32_t wv = 0;
            if (warp_perimeter_uniform(a.pm, a.max_dwell, g, lane, &wv, it)) {
                fill_rect(a.map, a.n, g, wv, lane, 32u);
                kind = KIND_FILL;
                if (COUNT && lane == 0)
                    fpx += (unsigned long long)g.w * g.h;
            } else {
                kind = a.split ? KIND_SPLIT : KIND_LEAF;
            }
            if (COUNT && lane == 0)
                bpx += perimeter_size(g.w, g.h);
        } else {
            // last level, exact perimeters: every perimeter dwell is final (a
            // leaf keeps them and the leaf kernel skips them)
            const uint32_t P = perimeter_size(g.w, g.h);
            uint32_t dmin = 0xffffffffu, dmax = 0u;
            for (uint32_t k = lane; k < P; k += 32u) {
                uint32_t px, py;
                perimeter_pixel(g, k, px, py);
                const float2 c = pixel_c(a.pm, px, py);
                const uint32_t d = dwell(c.x, c.y, a.max_dwell);
                dmin = min(dmin, d);
                dmax = max(dmax, d);
                if (k < kWarpStage)
                    stage[k] = d;
                else
                    a.map[(size_t)py * a.n + px] = d;  // beyond the stage: write through
                if (COUNT) {
                    it += d;
                    ++bpx;
                }
            }
            dmin = __reduce_min_sync(kFull, dmin);
            dmax = __reduce_max_sync(kFull, dmax);
            if (dmin == dmax) {
                fill_rect(a.map, a.n, g, dmin, lane, 32u);
                kind = KIND_FILL;
                if (COUNT && lane == 0)
                    fpx += (unsigned long long)g.w * g.h;
            } else {
                // leaf: its perimeter is final, the leaf kernel skips it
                const uint32_t staged = min(P, kWarpStage);
                for (uint32_t k = lane; k < staged; k += 32u) {
                    uint32_t px, py;
                    perimeter_pixel(g, k, px, py);
                    a.map[(size_t)py * a.n + px] = stage[k];
                }
                kind = KIND_LEAF;
            }
        }
        if (lane == j) {
            b.rec = e;
            b.kind = kind;
            b.nchild = (kind == KIND_SPLIT) ? child_count(g, a.child_side, a.r) : 0u;
        }
        __syncwarp();
        if (++j == 32u) {
            flush_batch(a, b, lane);
            j = 0;
        }
    }
    if (j)
        flush_batch(a, b, lane);
    if (COUNT) {
        it = warp_sum_u64(it);
        bpx = warp_sum_u64(bpx);
        fpx = warp_sum_u64(fpx);
        if (lane == 0) {
            if (it) {
                atomicAdd(&a.ctr->iterations, it);
                atomicAdd(&a.ctr->level_iters[a.level], it);
            }
            if (bpx)
                atomicAdd(&a.ctr->border_pixels, bpx);
            if (fpx)
                atomicAdd(&a.ctr->fill_pixels, fpx);
        }
    }
}

// ---------------------------------------------------------------------------
// Level kernel, one CTA per region (large regions, few of them).
// ---------------------------------------------------------------------------
template <bool COUNT>
__global__ void __launch_bounds__(1024) level_cta_kernel(LevelArgs a, uint32_t olt_in_cap,
                                                         uint32_t stage_cap)
{
    extern __shared__ uint32_t stage[];
    __shared__ uint32_t red_min[32], red_max[32];
    __shared__ uint32_t s_min, s_max, s_base, s_flag, s_w, s_idx;
    const uint32_t tid = threadIdx.x, T = blockDim.x, lane = tid & 31u, wid = tid >> 5;
    const uint32_t nw = T >> 5;
    const uint32_t count = min(a.ctr->count[a.level], olt_in_cap);
    unsigned long long it = 0, bpx = 0, fpx = 0;
    const bool query = a.split || !a.exact_last;

    for (;;) {
        if (tid == 0)
            s_idx = atomicAdd(&a.ctr->work[a.level], 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= count)
            break;  // uniform over the CTA
        const uint2 e = a.olt_in[idx];
        const Region g = unpack_region(e);
        const uint32_t P = perimeter_size(g.w, g.h);
        uint32_t dmin, dmax;
        if (query) {
            if (tid == 0) {
                s_flag = 0u;
                s_w = 0xffffffffu;
            }
            __syncthreads();
            uint32_t wv = 0;
            const bool uni = cta_perimeter_uniform(a.pm, a.max_dwell, g, tid, T, &s_flag, &s_w, &wv, it);
            dmin = wv;
            dmax = uni ? wv : wv + 1u;
            if (COUNT && tid == 0)
                bpx += P;
        } else {
            dmin = 0xffffffffu;
            dmax = 0u;
            for (uint32_t k = tid; k < P; k += T) {
                uint32_t px, py;
                perimeter_pixel(g, k, px, py);
                const float2 c = pixel_c(a.pm, px, py);
                const uint32_t d = dwell(c.x, c.y, a.max_dwell);
                dmin = min(dmin, d);
                dmax = max(dmax, d);
                if (k < stage_cap)
                    stage[k] = d;
                else
                    a.map[(size_t)py * a.n + px] = d;
                if (COUNT) {
                    it += d;
                    ++bpx;
                }
            }
            dmin = __reduce_min_sync(kFull, dmin);
            dmax = __reduce_max_sync(kFull, dmax);
            if (lane == 0) {
                red_min[wid] = dmin;
                red_max[wid] = dmax;
            }
            __syncthreads();
            if (wid == 0) {
                uint32_t m0 = lane < nw ? red_min[lane] : 0xffffffffu;
                uint32_t m1 = lane < nw ? red_max[lane] : 0u;
                m0 = __reduce_min_sync(kFull, m0);
                m1 = __reduce_max_sync(kFull, m1);
                if (lane == 0) {
                    s_min = m0;
                    s_max = m1;
                }
            }
            __syncthreads();
            dmin = s_min;
            dmax = s_max;
        }
        if (dmin == dmax) {
            fill_rect(a.map, a.n, g, dmin, tid, T);
            if (tid == 0) {
                atomicAdd(&a.ctr->fills[a.level], 1u);
                if (COUNT)
                    fpx += (unsigned long long)g.w * g.h;
            }
        } else if (a.split) {
            const uint32_t nc = child_count(g, a.child_side, a.r);
            if (tid == 0) {
                s_base = atomicAdd(&a.ctr->count[a.level + 1], nc);
                atomicAdd(&a.ctr->subdivs[a.level], 1u);
            }
            __syncthreads();
            for (uint32_t j = tid; j < nc; j += T) {
                const uint32_t slot = s_base + j;
                if (slot < a.olt_cap)
                    a.olt_out[slot] = child_region(g, a.child_side, a.r, j);
                else
                    atomicOr(&a.ctr->error, ERR_OLT_OVERFLOW);
            }
        } else {
            if (!query) {
                const uint32_t staged = min(P, stage_cap);
                for (uint32_t k = tid; k < staged; k += T) {
                    uint32_t px, py;
                    perimeter_pixel(g, k, px, py);
                    a.map[(size_t)py * a.n + px] = stage[k];
                }
            }
            if (tid == 0) {
                const uint32_t slot = atomicAdd(&a.ctr->leaf_count, 1u);
                if (slot < a.leaf_cap)
                    a.leaves[slot] = e;
                else
                    atomicOr(&a.ctr->error, ERR_LEAF_OVERFLOW);
            }
        }
        __syncthreads();  // the stage and s_* are reused by the next region
    }
    __syncthreads();
    if (COUNT) {
        it = warp_sum_u64(it);
        bpx = warp_sum_u64(bpx);
        fpx = warp_sum_u64(fpx);
        if (lane == 0) {
            if (it) {
                atomicAdd(&a.ctr->iterations, it);
                atomicAdd(&a.ctr->level_iters[a.level], it);
            }
            if (bpx)
                atomicAdd(&a.ctr->border_pixels, bpx);
            if (fpx)
                atomicAdd(&a.ctr->fill_pixels, fpx);
        }
    }
}

// ---------------------------------------------------------------------------
// Leaf kernel: every interior pixel of every leaf region.  Work items are
// (leaf, tile) pairs with block_x x block_y tiles; the grid is persistent and
// each warp walks the item sequence on its own (no CTA barrier).
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
        const Region g = unpack_region(a.leaves[leaf]);
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
// Leaf kernel with lane refill.  Leaf pixels near the set's boundary have
// dwells from a handful of updates to max_dwell side by side, so a warp that
// owned 32 fixed pixels would idle most lanes while one orbit runs on.  Here
// each warp takes leaves from a device counter and feeds their pixels to its
// lanes one at a time:
//  * every round, each busy lane advances its orbit by one unchecked block
//    (see dwell()); a lane whose block ends escaped, or that has fewer than a
//    block's worth of updates left, parks (saved state, count, pixel) in the
//    warp's replay buffer in shared memory and takes a new pixel at once;
//  * when 32 orbits are parked, the warp replays them together, one per
//    lane, with a tested update per step (at most one block each), and
//    writes their dwells.
// Lanes stay busy until the warp runs out of leaves.
// ---------------------------------------------------------------------------
constexpr int kRefillWarps = 8;   // warps per CTA
constexpr uint32_t kParkCap = 64; // parked orbits per warp (< 32 + 32)

template <bool COUNT>
__device__ __forceinline__ void replay_parked(const LeafArgs &a, float4 f, uint2 u,
                                              unsigned long long &it)
{
    float x = f.x, y = f.y;
    const float cr = f.z, ci = f.w;
    uint32_t d = u.x;
    while (d < a.max_dwell && z_bounded(x, y)) {
        z_update(x, y, cr, ci);
        ++d;
    }
    const uint32_t px = u.y & 0xffffu, py = u.y >> 16;
    a.map[(size_t)py * a.n + px] = d;
    if (COUNT)
        it += d;
}

template <bool COUNT>
__global__ void __launch_bounds__(kRefillWarps * 32) leaf_refill_kernel(LeafArgs a)
{
    __shared__ float4 park_f[kRefillWarps][kParkCap];  // saved x, y and c
    __shared__ uint2 park_u[kRefillWarps][kParkCap];   // count, pixel (py << 16 | px)
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *qf = park_f[wib];
    uint2 *qu = park_u[wib];
    uint32_t parked = 0;  // warp-uniform

    const uint32_t nleaves = min(a.ctr->leaf_count, a.leaf_cap);
    const uint32_t K = (uint32_t)kUnroll;
    // the warp's current leaf: the part still to hand out, as a row-major cursor
    Region g;
    g.x0 = g.y0 = 0;
    g.w = g.h = 1;
    uint32_t rem = 0, row0 = 0, col0 = 0, ox = 0, oy = 0, cw = 1;
    bool more = true;
    // this lane's orbit
    bool busy = false, fast = false;
    float x = 0.0f, y = 0.0f, cr = 0.0f, ci = 0.0f;
    uint32_t d = 0, pix = 0;
    unsigned long long it = 0, lpx = 0;

    for (;;) {
        // ---- refill idle lanes
        unsigned idle = __ballot_sync(kFull, !busy);
        while (idle && more) {
            if (rem == 0) {
                uint32_t li = 0;
                if (lane == 0)
                    li = atomicAdd(&a.ctr->leaf_work, 1u);
                li = __shfl_sync(kFull, li, 0);
                if (li >= nleaves) {
                    more = false;
                    break;
                }
                g = unpack_region(a.leaves[li]);
                if (a.skip_perimeter) {
                    // only the interior; a leaf of side <= 2 is all perimeter
                    cw = g.w > 2u ? g.w - 2u : 0u;
                    rem = (g.w > 2u && g.h > 2u) ? cw * (g.h - 2u) : 0u;
                    ox = g.x0 + 1u;
                    oy = g.y0 + 1u;
                } else {
                    cw = g.w;
                    rem = g.w * g.h;
                    ox = g.x0;
                    oy = g.y0;
                }
                row0 = col0 = 0;
                continue;
            }
            const uint32_t nidle = (uint32_t)__popc(idle);
            const uint32_t take = min(nidle, rem);
            const uint32_t rank = (uint32_t)__popc(idle & lt_mask);
            if (!busy && rank < take) {
                uint32_t col = col0 + rank, row = row0;
                while (col >= cw) {
                    col -= cw;
                    ++row;
                }
                const uint32_t px = ox + col, py = oy + row;
                const float2 c = pixel_c(a.pm, px, py);
                cr = c.x;
                ci = c.y;
                x = 0.0f;
                y = 0.0f;
                d = 0;
                pix = (py << 16) | px;
                fast = escape_absorbing(cr, ci);
                busy = true;
            }
            col0 += take;
            while (col0 >= cw) {
                col0 -= cw;
                ++row0;
            }
            rem -= take;
            idle = __ballot_sync(kFull, !busy);
        }
        if (!__any_sync(kFull, busy))
            break;

        // ---- one unchecked block per busy lane
        bool park = false;
        float sx = x, sy = y;
        if (busy) {
            if (fast && a.max_dwell - d >= K) {
#pragma unroll
                for (int k = 0; k < kUnroll; ++k)
                    z_update(x, y, cr, ci);
                if (z_bounded(x, y)) {
                    d += K;
                } else {
                    park = true;  // escaped inside this block: replay it
                }
            } else {
                park = true;      // tail below max_dwell, or |c| near 2
            }
        }

        // ---- park finished orbits; replay 32 at a time
        const unsigned pmask = __ballot_sync(kFull, park);
        if (pmask) {
            if (park) {
                const uint32_t slot = parked + (uint32_t)__popc(pmask & lt_mask);
                qf[slot] = make_float4(sx, sy, cr, ci);
                qu[slot] = make_uint2(d, pix);
                busy = false;
            }
            parked += (uint32_t)__popc(pmask);
            __syncwarp();
            if (parked >= 32u) {
                const float4 f = qf[lane];
                const uint2 u = qu[lane];
                float4 f2 = make_float4(0.f, 0.f, 0.f, 0.f);
                uint2 u2 = make_uint2(0u, 0u);
                if (lane < parked - 32u) {
                    f2 = qf[32u + lane];
                    u2 = qu[32u + lane];
                }
                __syncwarp();
                if (lane < parked - 32u) {
                    qf[lane] = f2;
                    qu[lane] = u2;
                }
                parked -= 32u;
                __syncwarp();
                replay_parked<COUNT>(a, f, u, it);
                if (COUNT)
                    ++lpx;
            }
        }
    }
    // ---- the orbits still parked
    if (lane < parked) {
        replay_parked<COUNT>(a, qf[lane], qu[lane], it);
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

cudaError_t launch_init(uint2 *olt0, DevCounters *ctr, uint32_t n, uint32_t s0, uint32_t axis0,
                        cudaStream_t s)
{
    const uint32_t total = axis0 * axis0;
    uint32_t blocks = (total + 255u) / 256u;
    if (blocks < 1)
        blocks = 1;
    if (blocks > 4096)
        blocks = 4096;
    init_kernel<<<blocks, 256, 0, s>>>(olt0, ctr, n, s0, axis0);
    return cudaGetLastError();
}

cudaError_t launch_level(const LevelArgs &a, int mode, uint32_t threads, bool count, int sms,
                         cudaStream_t s)
{
    // both tables have the same capacity; a count past it (an overflow that
    // the previous level latched) is clamped so nothing reads out of bounds
    const uint32_t in_cap = a.olt_cap;
    if (mode == 0) {
        const size_t smem = (size_t)(256 / 32) * kWarpStage * sizeof(uint32_t);
        if (count) {
            const int grid = persistent_grid(level_warp_kernel<true>, 256, smem, sms);
            level_warp_kernel<true><<<grid, 256, smem, s>>>(a, in_cap);
        } else {
            const int grid = persistent_grid(level_warp_kernel<false>, 256, smem, sms);
            level_warp_kernel<false><<<grid, 256, smem, s>>>(a, in_cap);
        }
    } else {
        const uint32_t P = 4u * a.side;
        const uint32_t stage_cap = P < kCtaStageMax ? P : kCtaStageMax;
        const size_t smem = (size_t)stage_cap * sizeof(uint32_t);
        if (smem > 48 * 1024) {
            cudaFuncSetAttribute(level_cta_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kCtaStageMax * sizeof(uint32_t)));
            cudaFuncSetAttribute(level_cta_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kCtaStageMax * sizeof(uint32_t)));
        }
        if (count) {
            const int grid = persistent_grid(level_cta_kernel<true>, (int)threads, smem, sms);
            level_cta_kernel<true><<<grid, threads, smem, s>>>(a, in_cap, stage_cap);
        } else {
            const int grid = persistent_grid(level_cta_kernel<false>, (int)threads, smem, sms);
            level_cta_kernel<false><<<grid, threads, smem, s>>>(a, in_cap, stage_cap);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_leaf(const LeafArgs &a, uint32_t bx, uint32_t by, bool count, bool tiled,
                        int sms, cudaStream_t s)
{
    if (!tiled) {
        const int threads = kRefillWarps * 32;
        if (count) {
            const int grid = persistent_grid(leaf_refill_kernel<true>, threads, 0, sms);
            leaf_refill_kernel<true><<<grid, threads, 0, s>>>(a);
        } else {
            const int grid = persistent_grid(leaf_refill_kernel<false>, threads, 0, sms);
            leaf_refill_kernel<false><<<grid, threads, 0, s>>>(a);
        }
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
