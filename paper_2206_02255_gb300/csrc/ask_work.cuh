// ask_work.cuh -- device building blocks shared by the ASK launch chain
// (ask_kernels.cu: one level kernel per depth, then the leaf kernel) and the
// persistent batch kernel fed from a device work queue (ask_queue.cu):
// region records, the chunked perimeter query, and the leaf machinery (the
// coherent pre-pass over fresh pixels, the ring of survivors, the two-orbit
// refill round, parking and the batched finish of parked orbits).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_internal.h"

namespace ask {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
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

// Rounds between issuing a state load and using it, for one frame.  A
// batch keeps enough warps resident to hide the load, and there a late
// stop costs more than the wait, so it uses the value one round later.
constexpr uint32_t kPollLag = 8;
// Chunked queries of regions with longer perimeters skip the short first
// rounds of query_step (at n = 16384 they slowed levels 0 and 1, whose
// regions of side 1024 and 256 are seldom uniform outside the set, and sped
// up level 2, side 64).
constexpr uint32_t kShortRoundsMaxPerimeter = 512;

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
        // short first rounds for small regions only: large ones are mostly
        // inside the set or on its boundary, rarely uniform outside it
        uint32_t nx = v.x, ny = v.y, lag = 0;
        constexpr bool kShort = !BATCH || kBatchShortChunks;
        uint32_t rnd = (kShort && perimeter_size(g.w, g.h) <= kShortRoundsMaxPerimeter) ? 0u : 3u;
        for (;; ++rnd) {
            if (lag == 0 && lane == 0) {
                nx = ps[0];
                ny = ps[1];
            }
            const uint32_t limit = (v.x != kNone) ? min(a.max_dwell, v.x + 1u) : a.max_dwell;
            if (kShort)
                query_step<kQueryRoundLarge>(o, stt, limit, rnd);
            else if (stt == ORBIT_RUN)
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
        // every orbit finished in round rnd (else they would differ)
        if (!stop && !differ && stt == ORBIT_PEND) {
            if (kShort)
                query_resolve<kQueryRoundLarge>(o, rnd);
            else
                orbit_resolve<kQueryRoundLarge>(o);
        }
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

// ---------------------------------------------------------------------------
// Leaf machinery (see the leaf kernel in ask_kernels.cu)
// ---------------------------------------------------------------------------
constexpr int kRefillWarps = 8;    // warps per CTA
// Resident CTAs per SM: the park buffer and the ring take 5 KB of shared
// memory a warp, so 5 CTAs of 8 warps fit an SM (200 KB) with up to 48
// registers a thread (one frame); a batch's per-frame lookups need more
// registers, 4 CTAs.
constexpr int kRefillMinBlocks = 5;
constexpr int kRefillMinBlocksBatch = 4;
constexpr uint32_t kParkCap = 96;  // parked orbits per warp (< 32 + 2 * 32)
constexpr uint32_t kRingCap = 64;  // survivors per warp (< 32 + 32: topped up while below 32)
constexpr int kLeafUnroll = 64;    // updates per unchecked block of the refill loop (a power of two)
constexpr int kPreBlock = 8;       // updates per unchecked block of the pre-pass (a power of two)
constexpr int kPrePass = 64;       // updates of the pre-pass (a multiple of kPreBlock)

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


// One orbit slot of a lane in the refill loop.
struct Slot {
    float x, y, cr, ci;
    uint32_t d, pix;  // count, pixel (py << 16 | px)
    uint32_t lim;     // a whole unchecked block may run while d < lim
    bool busy;
};

// The warp's current leaf, handed out as a row-major cursor.
struct LeafCursor {
    uint32_t rem, row0, col0, ox, oy, cw, frame;
    float inv_cw;
};

// Where the pre-pass takes its leaves from.
enum : uint32_t {
    SRC_MORE = 0,  // a leaf was given, or more may be asked for
    SRC_WAIT = 1,  // none is ready now, more may come (persistent batch kernel)
    SRC_DONE = 2,  // the leaves have run out
};

// Point the cursor at leaf region g of `frame`: its interior only when the
// perimeters are already in the map (a leaf of side <= 2 is all perimeter).
__device__ __forceinline__ void cursor_at(LeafCursor &lc, const Region &g, uint32_t frame,
                                          bool skip_perimeter)
{
    lc.frame = frame;
    if (skip_perimeter) {
        lc.cw = g.w > 2u ? g.w - 2u : 1u;
        lc.rem = (g.w > 2u && g.h > 2u) ? (g.w - 2u) * (g.h - 2u) : 0u;
        lc.ox = g.x0 + 1u;
        lc.oy = g.y0 + 1u;
    } else {
        lc.cw = g.w;
        lc.rem = g.w * g.h;
        lc.ox = g.x0;
        lc.oy = g.y0;
    }
    lc.row0 = lc.col0 = 0;
    lc.inv_cw = 1.0f / (float)lc.cw;
}

// Region tables and leaf lists are filled from both ends: `front` entries
// from slot 0 up (the regions or leaves likely to hold long orbits, or every
// entry where the producer does not order them) and the rest from slot
// cap - 1 down.  Entry t of the order in which they are taken (the front
// first, then the back in append order) sits at this slot.
__device__ __forceinline__ uint32_t table_slot(uint32_t t, uint32_t front, uint32_t cap)
{
    return t < front ? t : cap - 1u - (t - front);
}

// Entries of the front and of the whole list, within `cap`.  More leaves
// than `cap` (front and back met) latch the overflow error; block 0 reports.
__device__ __forceinline__ void leaf_extent(DevCounters *ctr, uint32_t cap, uint32_t &front,
                                            uint32_t &total)
{
    const uint32_t h = ctr->leaf_count, l = ctr->leaf_light;
    front = min(h, cap);
    total = front + min(l, cap - front);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (unsigned long long)h + l > cap)
        atomicOr(&ctr->error, ERR_LEAF_OVERFLOW);
}

// The leaf list of a launch chain: complete when the leaf kernel starts, its
// leaves handed out one at a time by a device counter.
template <bool BATCH>
struct LeafList {
    const typename Rec<BATCH>::T *leaves;
    uint32_t front, total, cap;

    __device__ __forceinline__ uint32_t next(const LeafArgs &a, LeafCursor &lc, uint32_t lane)
    {
        using R = Rec<BATCH>;
        uint32_t li = 0;
        if (lane == 0)
            li = atomicAdd(&a.ctr->leaf_work, 1u);
        li = __shfl_sync(kFull, li, 0);
        if (li >= total)
            return SRC_DONE;
        const typename R::T e = leaves[table_slot(li, front, cap)];
        cursor_at(lc, R::region(e), R::frame(e), a.skip_perimeter != 0u);
        return SRC_MORE;
    }
};

// Pre-pass: up to 32 fresh pixels from the leaf cursor, the j-th on lane j,
// run their first kPrePass updates in lockstep (unchecked blocks of
// kPreBlock, one test each, only while a whole block stays within
// max_dwell).  An orbit whose block ends escaped has its dwell in that block:
// a binary search over the block (kPreBlock - 1 updates and log2(kPreBlock)
// tests, the same on every lane) finds it, and the dwell is written.  Every
// other pixel is pushed onto the ring with its state: survivors of the whole
// pass, orbits stopped by max_dwell, and points where escape is not
// absorbing (d = 0; the refill loop parks them at once and finish_parked
// runs the tested loop).  Leaves come from `src` (see LeafList); `srcst`
// becomes SRC_WAIT or SRC_DONE when it has none to give.  Returns the number
// of pixels taken.
template <bool COUNT, bool BATCH, typename Src>
__device__ __forceinline__ uint32_t pre_pass(const LeafArgs &a, Src &src, LeafCursor &lc,
                                             uint32_t &srcst, float4 *rs, uint4 *ru, uint32_t ring_h,
                                             uint32_t &ring_n, uint32_t lane, unsigned lt_mask,
                                             unsigned long long &it, unsigned long long &lpx)
{
    uint32_t pix = 0, frame = 0;
    bool have = false;
    uint32_t base = 0;
    while (base < 32u && srcst == SRC_MORE) {
        if (lc.rem == 0) {
            srcst = src.next(a, lc, lane);
            continue;
        }
        const uint32_t take = min(32u - base, lc.rem);
        if (lane >= base && lane < base + take) {
            const uint32_t q = lc.col0 + (lane - base), dr = rows_in(q, lc.inv_cw);
            pix = ((lc.oy + lc.row0 + dr) << 16) | (lc.ox + q - dr * lc.cw);
            frame = lc.frame;
            have = true;
        }
        const uint32_t q = lc.col0 + take, dr = rows_in(q, lc.inv_cw);
        lc.col0 = q - dr * lc.cw;
        lc.row0 += dr;
        lc.rem -= take;
        base += take;
    }
    if (base == 0)
        return 0;
    const LView v = leaf_view<BATCH>(a, frame);
    const uint32_t px = pix & 0xffffu, py = pix >> 16;
    const float2 c = pixel_c(v.pm, px, py);
    const bool absorbing = escape_absorbing(c.x, c.y);
    // A lane runs while its orbit passes every block's test; (ex, ey) keeps
    // the state a stopped lane stopped at (the start of its escaping block,
    // or, in a batch, the state its own max_dwell left no room beyond), so
    // a stopped lane's (x, y) may run on to garbage with no rollback.  d
    // counts only the blocks a lane ran.
    float x = 0.0f, y = 0.0f, ex = 0.0f, ey = 0.0f;
    uint32_t d = 0;
    bool run = have && absorbing, esc = false;
    // one frame: the blocks that fit below max_dwell, the same for every lane
    const uint32_t nb = BATCH ? (uint32_t)(kPrePass / kPreBlock)
                              : min((uint32_t)(kPrePass / kPreBlock), v.max_dwell / (uint32_t)kPreBlock);
#pragma unroll
    for (int b = 0; b < kPrePass / kPreBlock; ++b) {
        if (!BATCH && (uint32_t)b >= nb)
            break;
        if (BATCH) {
            const bool fits = v.max_dwell - d >= (uint32_t)kPreBlock;  // a whole block fits
            if (run && !fits) {
                ex = x;
                ey = y;
            }
            run = run && fits;
        }
        if (!__any_sync(kFull, run))
            break;
        const float sx = x, sy = y;
#pragma unroll
        for (int k = 0; k < kPreBlock; ++k)
            z_update(x, y, c.x, c.y);
        const bool ok = z_bounded(x, y);
        if (run && !ok) {
            esc = true;  // the dwell lies in (d, d + kPreBlock]
            ex = sx;
            ey = sy;
        }
        if (run && ok)
            d += (uint32_t)kPreBlock;
        run = run && ok;
    }
    if (run) {
        ex = x;
        ey = y;
    }
    if (__any_sync(kFull, esc)) {
        // invariant: the state at count d passes the test and the state at
        // d + 2h fails; halve h until the first failing count is d + 1
        float rx = ex, ry = ey;
        uint32_t rd = d;
#pragma unroll
        for (uint32_t h = (uint32_t)kPreBlock / 2u; h >= 1u; h >>= 1) {
            float tx = rx, ty = ry;
#pragma unroll
            for (uint32_t k = 0; k < h; ++k)
                z_update(tx, ty, c.x, c.y);
            if (z_bounded(tx, ty)) {
                rx = tx;
                ry = ty;
                rd += h;
            }
        }
        if (esc) {
            v.map[(size_t)py * v.n + px] = rd + 1u;
            if (COUNT) {
                it += rd + 1u;
                ++lpx;
            }
        }
    }
    const bool push = have && !esc;
    const unsigned pm = __ballot_sync(kFull, push);
    if (push) {
        uint32_t slot = ring_h + ring_n + (uint32_t)__popc(pm & lt_mask);
        if (slot >= kRingCap)
            slot -= kRingCap;
        const uint32_t K = (uint32_t)kLeafUnroll;
        const uint32_t lim = (absorbing && v.max_dwell >= K) ? v.max_dwell - K + 1u : 0u;
        rs[slot] = make_float4(ex, ey, c.x, c.y);
        ru[slot] = make_uint4(d, pix, frame, lim);
    }
    ring_n += (uint32_t)__popc(pm);
    __syncwarp();
    return base;
}


// Refill the idle slots of the refill loop from the ring of survivors: slot 0
// of the idle lanes first, then slot 1 (i0, i1: ballots of the idle slots).
__device__ __forceinline__ void refill_from_ring(Slot &s0, Slot &s1, uint32_t &f0, uint32_t &f1,
                                                 const float4 *rs, const uint4 *ru, uint32_t &ring_h,
                                                 uint32_t &ring_n, unsigned i0, unsigned i1,
                                                 uint32_t lane, unsigned lt_mask)
{
    const uint32_t n0 = (uint32_t)__popc(i0);
    const uint32_t take = min(n0 + (uint32_t)__popc(i1), ring_n);
    const uint32_t r0 = (uint32_t)__popc(i0 & lt_mask);
    const uint32_t r1 = n0 + (uint32_t)__popc(i1 & lt_mask);
    if (!s0.busy && r0 < take) {
        uint32_t k = ring_h + r0;
        if (k >= kRingCap)
            k -= kRingCap;
        const float4 sv = rs[k];
        const uint4 uv = ru[k];
        s0.x = sv.x;
        s0.y = sv.y;
        s0.cr = sv.z;
        s0.ci = sv.w;
        s0.d = uv.x;
        s0.pix = uv.y;
        f0 = uv.z;
        s0.lim = uv.w;
        s0.busy = true;
    }
    if (!s1.busy && r1 < take) {
        uint32_t k = ring_h + r1;
        if (k >= kRingCap)
            k -= kRingCap;
        const float4 sv = rs[k];
        const uint4 uv = ru[k];
        s1.x = sv.x;
        s1.y = sv.y;
        s1.cr = sv.z;
        s1.ci = sv.w;
        s1.d = uv.x;
        s1.pix = uv.y;
        f1 = uv.z;
        s1.lim = uv.w;
        s1.busy = true;
    }
    ring_h += take;
    if (ring_h >= kRingCap)
        ring_h -= kRingCap;
    ring_n -= take;
    __syncwarp();
}

// Move the orbits of slot 1 onto the ring (the ring and both slots hold at
// most 32 orbits between them when this is called), so the refill that
// follows puts every orbit in slot 0 and the rounds after it update one
// orbit per lane: once the leaves have run out and few orbits are left, a
// round then costs half the instructions.
__device__ __forceinline__ void fold_slot1(Slot &s1, uint32_t f1, float4 *rs, uint4 *ru,
                                           uint32_t ring_h, uint32_t &ring_n, unsigned lt_mask)
{
    const unsigned b1 = __ballot_sync(kFull, s1.busy);
    if (s1.busy) {
        uint32_t slot = ring_h + ring_n + (uint32_t)__popc(b1 & lt_mask);
        if (slot >= kRingCap)
            slot -= kRingCap;
        rs[slot] = make_float4(s1.x, s1.y, s1.cr, s1.ci);
        ru[slot] = make_uint4(s1.d, s1.pix, f1, s1.lim);
        s1.busy = false;
    }
    ring_n += (uint32_t)__popc(b1);
    __syncwarp();
}

// One round of the refill loop: an unchecked block of kLeafUnroll updates on
// both slots (TWO) or on slot 0 alone (the results of a slot that is idle or
// parks are not used); an orbit that escaped in the block, has less than a
// block left below max_dwell or has |c| near 2 parks its state before the
// block (and the block's midpoint state) in the park buffer; whenever 32
// orbits are parked the warp finishes them together.
template <bool COUNT, bool BATCH, bool TWO = true>
__device__ __forceinline__ void refill_round(const LeafArgs &a, Slot &s0, Slot &s1, uint32_t f0,
                                             uint32_t f1, float4 *qs, uint4 *qu, uint32_t &parked,
                                             uint32_t lane, unsigned lt_mask, unsigned long long &it,
                                             unsigned long long &lpx)
{
    const uint32_t K = (uint32_t)kLeafUnroll;
    const float sx0 = s0.x, sy0 = s0.y, sx1 = s1.x, sy1 = s1.y;
#pragma unroll
    for (int k = 0; k < kLeafUnroll / 2; ++k) {
        z_update(s0.x, s0.y, s0.cr, s0.ci);
        if (TWO)
            z_update(s1.x, s1.y, s1.cr, s1.ci);
    }
    const float mx0 = s0.x, my0 = s0.y, mx1 = s1.x, my1 = s1.y;  // midpoint states
#pragma unroll
    for (int k = 0; k < kLeafUnroll / 2; ++k) {
        z_update(s0.x, s0.y, s0.cr, s0.ci);
        if (TWO)
            z_update(s1.x, s1.y, s1.cr, s1.ci);
    }
    bool park0 = false, park1 = false;
    if (s0.busy) {
        if (s0.d < s0.lim && z_bounded(s0.x, s0.y))
            s0.d += K;
        else
            park0 = true;
    }
    if (TWO && s1.busy) {
        if (s1.d < s1.lim && z_bounded(s1.x, s1.y))
            s1.d += K;
        else
            park1 = true;
    }
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

}  // namespace ask
