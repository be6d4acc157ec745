// ask_queue.cu -- a batch of frames rendered by one persistent kernel fed
// from a device work queue.
//
// The launch chain of ask_kernels.cu renders a batch depth by depth: one
// level kernel per subdivision depth, each a grid-wide step, so the tail of
// the slowest frame's level idles the GPU before the next depth can start,
// and the leaf pass waits for the last depth.  Here the region tables of the
// ASK scheme (paper Sec. 5.2-5.3) become one device work queue holding the
// regions of every frame and every depth:
//
//  * the queue is a linear array of items {origin, extent, tag, epoch}
//    (tag = frame | depth | kind | perimeter chunk), one more word of aux
//    (the chunk's query-state index, or a fill band's dwell);
//  * a warp takes a ticket (atomicAdd on `head`) and processes the item in
//    that slot once it is published: the perimeter query Q (Sec. 4.2.1) of a
//    region or of one chunk of a large region's perimeter, then the decision:
//    fill the region (small ones in place, large ones pushed back as bands of
//    rows), push its r x r children (Sec. 5.3.1) or append it to the leaf
//    list;
//  * pushes reserve slots with one atomicAdd on `tail`, write the items, and
//    publish each by a release store of the render's epoch (takers read it
//    with an acquire load), so a slot is valid exactly when it carries the
//    current epoch (no clearing between renders);
//  * `pending` counts pushed items not yet finished; a warp that finishes an
//    item adds (items it pushed - 1) before publishing them, so the count
//    reaches 0 exactly when the last item is done; that warp marks the
//    render's regions done, and tickets beyond the final tail are void;
//  * leaves go to a second published list, taken by tickets on `leaf_head`;
//    a warp runs the leaf machinery of ask_work.cuh (pre-pass, ring of
//    survivors, two-orbit refill rounds, parked finishes) on leaves while it
//    has no ready region item, and takes a ready region item as soon as it
//    has one: the depths and the leaf pass overlap, with no grid-wide step.
//
// Every wait is bounded: a warp that has found nothing to do for
// wait_limit polls in a row (backing off with __nanosleep; the count starts
// again whenever the queue or the leaf list moves) sets ERR_TIMEOUT and
// leaves, and the host reports ASK_ETIMEOUT.  No warp waits for a warp that
// has not started, so the kernel needs no co-residency guarantee.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_internal.h"
#include "ask_work.cuh"

namespace ask {

namespace {

enum : uint32_t { QITEM_REGION = 0, QITEM_FILL = 1 };

// Leaf rounds between polls of the held region ticket while a warp is busy.
constexpr uint32_t kQueuePollRounds = 8;

__device__ __forceinline__ uint32_t qtag(uint32_t frame, uint32_t level, uint32_t kind, uint32_t chunk)
{
    return frame | (level << 20) | (kind << 25) | (chunk << 26);
}

__device__ __forceinline__ uint32_t load_volatile(const uint32_t *p)
{
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

__device__ __forceinline__ void store_volatile(uint32_t *p, uint32_t v)
{
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// Acquire / release at GPU scope: a slot is published by a release store of
// its epoch word, and taken after an acquire load of it, so its contents
// need no full fence on either side.  Writes of other lanes of the warp are
// ordered before a lane's release by a __syncwarp between them, and reads of
// other lanes after a lane's acquire the same way.
__device__ __forceinline__ uint32_t load_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t *p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// A ticket of the warp: lane 0 takes it, every lane gets it.
__device__ __forceinline__ uint32_t warp_ticket(uint32_t *counter, uint32_t lane)
{
    uint32_t t = 0;
    if (lane == 0)
        t = atomicAdd(counter, 1u);
    return __shfl_sync(kFull, t, 0);
}

// Finish an item that pushed nothing: the warp's earlier writes first, then
// the count (an acquire-release add, so the counts form one chain of
// releases); the warp that takes it to 0 marks the render's regions done.
__device__ __forceinline__ void finish_item(const QueueArgs &q, uint32_t epoch, uint32_t lane)
{
    __syncwarp();
    if (lane == 0 && atomic_add_acq_rel(&q.qs->pending, 0xffffffffu) == 1u)
        store_release(&q.qs->done, epoch);
    __syncwarp();
}

// Reserve n queue slots (lane 0; every lane gets the base), or kNone and a
// latched overflow when the queue is full.
__device__ __forceinline__ uint32_t reserve_items(const QueueArgs &q, uint32_t n, uint32_t lane)
{
    uint32_t base = 0;
    if (lane == 0) {
        base = atomicAdd(&q.qs->tail, n);
        if ((uint64_t)base + n > q.item_cap) {
            atomicOr(&q.ctr->error, ERR_OLT_OVERFLOW);
            base = kNone;
        }
    }
    return __shfl_sync(kFull, base, 0);
}

// Publish the n items written at base (each lane its own, written by it):
// the count of pending items first grows by n - 1 (the finishing item
// replaced by its n), then each item gets the epoch by a release store.
__device__ __forceinline__ void publish_items(const QueueArgs &q, uint32_t base, uint32_t n,
                                              uint32_t epoch, uint32_t lane)
{
    __syncwarp();
    if (lane == 0)
        atomic_add_acq_rel(&q.qs->pending, n - 1u);
    __syncwarp();
    for (uint32_t k = lane; k < n; k += 32u)
        store_release(&q.items[base + k].w, epoch);
    __syncwarp();
}

// Whether the item in slot t is ready: 1 published, -1 never will be (the
// render's regions are done and t is past the final tail), 0 not yet (or
// not known: `final` = false skips the second load that tells "never").
__device__ __forceinline__ int poll_item(const QueueArgs &q, uint32_t t, uint32_t epoch, bool final,
                                         uint32_t lane)
{
    int r = 0;
    if (lane == 0) {
        if (t < q.item_cap && load_acquire(&q.items[t].w) == epoch) {
            r = 1;
        } else if (final && load_acquire(&q.qs->done) == epoch) {
            r = (t < q.item_cap && load_acquire(&q.items[t].w) == epoch) ? 1 : -1;
        }
    }
    return __shfl_sync(kFull, r, 0);
}

// The published leaf list of the queue, taken by tickets: a ticket's leaf
// may not be appended yet (SRC_WAIT); once the regions are done, a ticket
// past the final count means the leaves have run out.
struct QueueLeaves {
    const QueueArgs *q;
    uint32_t epoch;
    uint32_t ticket;  // held ticket, kNone if none

    __device__ __forceinline__ uint32_t next(const LeafArgs &a, LeafCursor &lc, uint32_t lane)
    {
        if (ticket == kNone)
            ticket = warp_ticket(&q->qs->leaf_head, lane);
        const uint32_t t = ticket;
        int r = 0;
        uint4 e = make_uint4(0u, 0u, 0u, 0u);
        if (lane == 0) {
            if (t < q->leaf_cap && load_acquire(&q->leaves[t].w) == epoch) {
                r = 1;
            } else if (load_acquire(&q->qs->done) == epoch) {
                r = (t < q->leaf_cap && load_acquire(&q->leaves[t].w) == epoch) ? 1 : -1;
            }
            if (r > 0)
                e = __ldcg(&q->leaves[t]);  // after the acquire
        }
        r = __shfl_sync(kFull, r, 0);
        if (r == 0)
            return SRC_WAIT;
        ticket = kNone;
        if (r < 0)
            return SRC_DONE;
        e.x = __shfl_sync(kFull, e.x, 0);
        e.y = __shfl_sync(kFull, e.y, 0);
        e.z = __shfl_sync(kFull, e.z, 0);
        cursor_at(lc, unpack_region(make_uint2(e.x, e.y)), e.z, false);
        return SRC_MORE;
    }
};

// One published region or fill item, processed by the whole warp (the
// warp's leaf orbits wait in their registers meanwhile).
template <bool COUNT>
__device__ __forceinline__ void process_item(const QueueArgs &q, uint32_t t, uint32_t epoch,
                                             uint32_t lane)
{
    // lane 0 takes the slot (an acquire of its epoch word, which the poll
    // saw published) and hands its contents to the warp
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    uint32_t aux = 0;
    if (lane == 0) {
        (void)load_acquire(&q.items[t].w);
        e = __ldcg(&q.items[t]);
        aux = __ldcg(&q.aux[t]);
    }
    e.x = __shfl_sync(kFull, e.x, 0);
    e.y = __shfl_sync(kFull, e.y, 0);
    e.z = __shfl_sync(kFull, e.z, 0);
    aux = __shfl_sync(kFull, aux, 0);
    const uint32_t frame = e.z & 0xfffffu, level = (e.z >> 20) & 31u;
    const uint32_t kind = (e.z >> 25) & 1u, c = e.z >> 26;
    const Region g = unpack_region(make_uint2(e.x, e.y));
    const FrameDesc &fd = q.frames[frame];
    if (kind == QITEM_FILL) {
        fill_band_warp(fd.map, fd.n, g, aux, lane);
        finish_item(q, epoch, lane);
        return;
    }
    const FView f = view_frame(q.frames, frame, level);
    const uint32_t C = fd.chunks[level];
    const uint32_t P = perimeter_size(g.w, g.h);
    unsigned long long it = 0;
    bool decided = false, uniform = false;
    uint32_t wv = 0;
    if (C <= 1u) {
        decided = true;
        uniform = warp_perimeter_uniform<kQueryRoundBatch, kBatchShortWhole>(f.pm, f.max_dwell, g, lane, &wv, it);
    } else {
        uint4 *st = q.rst + aux;
        const uint32_t CP = max(q.chunk_px, ceil_div_u32(P, C));
        const uint32_t k0 = min(P, c * CP), k1 = min(P, k0 + CP);
        if (k0 < k1)
            chunk_query<true>(f, g, k0, k1, st, lane, it);
        // the warp that finishes the region's last chunk decides
        uint32_t last = 0;
        if (lane == 0)
            last = (atomic_add_acq_rel(&st->z, 1u) == C - 1u) ? 1u : 0u;
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            uint32_t sx = 0, sy = 0;
            if (lane == 0) {
                sx = atomicAdd(&st->x, 0u);
                sy = atomicAdd(&st->y, 0u);
            }
            sx = __shfl_sync(kFull, sx, 0);
            sy = __shfl_sync(kFull, sy, 0);
            uniform = (sy == 0u && sx != kNone);
            wv = sx;
            decided = true;
        }
    }
    if (COUNT) {
        it = warp_sum_u64(it);
        if (lane == 0 && it) {
            atomicAdd(&q.ctr->iterations, it);
            atomicAdd(&q.ctr->level_iters[level], it);
        }
    }
    if (!decided) {
        finish_item(q, epoch, lane);
        return;
    }
    if (uniform) {
        if (lane == 0)
            atomicAdd(&q.ctr->fills[level], 1u);
        const uint32_t area = g.w * g.h;
        if (area <= kInPlaceFillArea) {
            fill_rect(f.map, f.n, g, wv, lane, 32u);
            finish_item(q, epoch, lane);
            return;
        }
        // a large region: bands of whole rows, pushed back as fill items
        const uint32_t nb = fill_band_count(g.w, g.h), rows = fill_band_rows(g.w);
        const uint32_t base = reserve_items(q, nb, lane);
        if (base == kNone) {
            finish_item(q, epoch, lane);
            return;
        }
        for (uint32_t k = lane; k < nb; k += 32u) {
            const uint2 band = pack_region(g.x0, g.y0 + k * rows, g.w, min(rows, g.h - k * rows));
            uint4 *it4 = &q.items[base + k];
            it4->x = band.x;
            it4->y = band.y;
            it4->z = qtag(frame, level, QITEM_FILL, 0u);
            q.aux[base + k] = wv;
        }
        publish_items(q, base, nb, epoch, lane);
        return;
    }
    if (!f.split) {
        // a leaf: appended to the published leaf list
        if (lane == 0) {
            const uint32_t slot = atomicAdd(&q.ctr->leaf_count, 1u);
            if (slot < q.leaf_cap) {
                uint4 *l = &q.leaves[slot];
                l->x = e.x;
                l->y = e.y;
                l->z = frame;
                store_release(&l->w, epoch);
            } else {
                atomicOr(&q.ctr->error, ERR_LEAF_OVERFLOW);
            }
        }
        finish_item(q, epoch, lane);
        return;
    }
    // split: r x r children (clipped, empty ones dropped), each as the
    // chunk items of its depth
    const uint32_t nchild = child_count(g, f.child_side, f.r);
    const uint32_t C1 = fd.chunks[level + 1u];
    const uint32_t n = nchild * C1;
    if (lane == 0) {
        atomicAdd(&q.ctr->subdivs[level], 1u);
        atomicAdd(&q.ctr->count[level + 1u], nchild);
    }
    uint32_t sbase = 0;
    if (C1 > 1u) {
        if (lane == 0) {
            sbase = atomicAdd(&q.qs->states, nchild);
            if ((uint64_t)sbase + nchild > q.rst_cap) {
                atomicOr(&q.ctr->error, ERR_OLT_OVERFLOW);
                sbase = kNone;
            }
        }
        sbase = __shfl_sync(kFull, sbase, 0);
        if (sbase == kNone) {
            finish_item(q, epoch, lane);
            return;
        }
    }
    const uint32_t base = reserve_items(q, n, lane);
    if (base == kNone) {
        finish_item(q, epoch, lane);
        return;
    }
    for (uint32_t k = lane; k < n; k += 32u) {
        const uint32_t j = k / C1, cc = k - j * C1;
        const uint2 rec = child_region(g, f.child_side, f.r, j);
        uint4 *it4 = &q.items[base + k];
        it4->x = rec.x;
        it4->y = rec.y;
        it4->z = qtag(frame, level + 1u, QITEM_REGION, cc);
        q.aux[base + k] = (C1 > 1u) ? sbase + j : 0u;
        if (C1 > 1u && cc == 0u)
            q.rst[sbase + j] = make_uint4(kNone, 0u, 0u, 0u);
    }
    publish_items(q, base, n, epoch, lane);
}

// Counters and the level-0 items of every frame: block f writes frame f's
// initial regions (each as its perimeter chunks) with the render's epoch;
// block 0 also resets the counters and the queue state.  The epoch of a
// render is the stored epoch + 1 (the persistent kernel stores it when its
// last warp leaves).
__global__ void queue_init_kernel(QueueArgs q)
{
    const uint32_t epoch = load_volatile(&q.qs->epoch) + 1u;
    const uint32_t f = blockIdx.x;
    if (f == 0) {
        uint32_t *w = reinterpret_cast<uint32_t *>(q.ctr);
        const uint32_t words = (uint32_t)(sizeof(DevCounters) / sizeof(uint32_t));
        const uint32_t err_word = (uint32_t)(offsetof(DevCounters, error) / sizeof(uint32_t));
        for (uint32_t k = threadIdx.x; k < words; k += blockDim.x)
            if (k != err_word)
                w[k] = (k == 0u) ? q.regions0 : 0u;  // word 0 is count[0]
        if (threadIdx.x == 0) {
            q.qs->head = 0;
            q.qs->tail = q.total0;
            q.qs->pending = q.total0;
            q.qs->done = 0;
            q.qs->states = q.states0;
            q.qs->leaf_head = 0;
            q.qs->exited = 0;
        }
    }
    const FrameDesc &d = q.frames[f];
    const uint32_t C0 = d.chunks[0] > 0u ? d.chunks[0] : 1u;
    const uint32_t per = d.axis0 * d.axis0;
    for (uint32_t k = threadIdx.x; k < per * C0; k += blockDim.x) {
        const uint32_t region = k / C0, c = k - region * C0;
        const uint32_t gx = region % d.axis0, gy = region / d.axis0;
        const uint32_t x0 = gx * d.s0, y0 = gy * d.s0;
        const uint2 rec = pack_region(x0, y0, min(d.s0, d.n - x0), min(d.s0, d.n - y0));
        q.items[d.item0 + k] = make_uint4(rec.x, rec.y, qtag(f, 0u, QITEM_REGION, c), epoch);
        q.aux[d.item0 + k] = (C0 > 1u) ? d.state0 + region : 0u;
        if (C0 > 1u && c == 0u)
            q.rst[d.state0 + region] = make_uint4(kNone, 0u, 0u, 0u);
    }
}

// The persistent kernel: every warp alternates between region items (taken
// first, as soon as the held ticket's slot is published) and leaf work.
template <bool COUNT>
__global__ void __launch_bounds__(kRefillWarps * 32, kRefillMinBlocksBatch) queue_kernel(QueueArgs q, LeafArgs a)
{
    __shared__ float4 park_s[kRefillWarps][kParkCap];
    __shared__ uint4 park_u[kRefillWarps][kParkCap];
    __shared__ float4 ring_s[kRefillWarps][kRingCap];
    __shared__ uint4 ring_u[kRefillWarps][kRingCap];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    float4 *qs = park_s[wib];
    uint4 *qu = park_u[wib];
    float4 *rs = ring_s[wib];
    uint4 *ru = ring_u[wib];
    uint32_t parked = 0, ring_h = 0, ring_n = 0;  // warp-uniform

    uint32_t epoch = 0;
    if (lane == 0)
        epoch = load_volatile(&q.qs->epoch) + 1u;
    epoch = __shfl_sync(kFull, epoch, 0);

    QueueLeaves src;
    src.q = &q;
    src.epoch = epoch;
    src.ticket = kNone;
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
    uint32_t f0 = 0, f1 = 0;
    unsigned long long it = 0, lpx = 0;

    uint32_t rt = kNone;      // region ticket held
    bool rclosed = false;     // no region item will come any more
    uint32_t polls = 0;       // idle polls in a row
    uint32_t seen_p = 0, seen_l = 0;
    uint32_t rounds = 0;      // leaf rounds since the held ticket's slot was loaded
    uint32_t seen_w = 0;      // lane 0: that load (the slot's epoch word)
    bool idle = true;         // the last pass found no leaf work

    for (;;) {
        // The held ticket: an idle warp polls it at once (with the check
        // that tells a ticket past the final tail).  A busy warp loads the
        // slot's epoch word, carries on with its leaf rounds, and reads the
        // loaded value kQueuePollRounds rounds later, so the L2 round trip
        // never stalls it.
        if (!rclosed) {
            if (rt == kNone) {
                rt = warp_ticket(&q.qs->head, lane);
                rounds = kQueuePollRounds;  // nothing loaded yet
                seen_w = 0;
            }
            int r = 0;
            if (idle) {
                r = poll_item(q, rt, epoch, true, lane);
                rounds = kQueuePollRounds;
            } else if (rounds >= kQueuePollRounds) {
                r = __shfl_sync(kFull, seen_w == epoch ? 1 : 0, 0);
                if (lane == 0 && rt < q.item_cap)
                    seen_w = load_volatile(&q.items[rt].w);
                rounds = 0;
            }
            if (r > 0) {
                process_item<COUNT>(q, rt, epoch, lane);
                rt = kNone;
                polls = 0;
                continue;
            }
            if (r < 0)
                rclosed = true;
        }
        if (srcst == SRC_WAIT)
            srcst = SRC_MORE;  // ask again
        bool worked = false;
        const unsigned i0 = __ballot_sync(kFull, !s0.busy), i1 = __ballot_sync(kFull, !s1.busy);
        if (i0 | i1) {
            const uint32_t want = min((uint32_t)(__popc(i0) + __popc(i1)), 32u);
            while (ring_n < want && srcst == SRC_MORE)
                if (pre_pass<COUNT, true>(a, src, lc, srcst, rs, ru, ring_h, ring_n, lane, lt_mask, it,
                                          lpx))
                    worked = true;
            refill_from_ring(s0, s1, f0, f1, rs, ru, ring_h, ring_n, i0, i1, lane, lt_mask);
        }
        if (__any_sync(kFull, s0.busy || s1.busy)) {
            refill_round<COUNT, true>(a, s0, s1, f0, f1, qs, qu, parked, lane, lt_mask, it, lpx);
            worked = true;
            ++rounds;
        }
        idle = !worked;
        if (worked) {
            polls = 0;
            continue;
        }
        if (rclosed && srcst == SRC_DONE && ring_n == 0)
            break;
        // nothing to do now: back off; the count starts again whenever the
        // queue or the leaf list moves
        uint32_t p = 0, l = 0;
        if (lane == 0) {
            p = load_volatile(&q.qs->pending);
            l = load_volatile(&q.ctr->leaf_count);
        }
        p = __shfl_sync(kFull, p, 0);
        l = __shfl_sync(kFull, l, 0);
        if (p != seen_p || l != seen_l) {
            seen_p = p;
            seen_l = l;
            polls = 0;
        }
        if (++polls > q.wait_limit) {
            if (lane == 0)
                atomicOr(&q.ctr->error, ERR_TIMEOUT);
            break;
        }
        __nanosleep(polls < 32u ? 32u : 256u);
    }
    // the orbits still parked
    if (lane < parked) {
        finish_parked<COUNT, true>(a, qs[lane], qu[lane], it);
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
    // the last warp to leave stores the epoch, so the next render's items
    // are told apart from this render's
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&q.qs->exited, 1u) == gridDim.x * (uint32_t)kRefillWarps - 1u)
            store_volatile(&q.qs->epoch, epoch);
    }
}

template <typename K>
int resident_grid(K kernel, int threads, int sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

}  // namespace

cudaError_t launch_queue(const QueueArgs &q, uint32_t nframes, bool count, int sms, cudaStream_t s)
{
    queue_init_kernel<<<nframes, 256, 0, s>>>(q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    LeafArgs a;
    a.map = nullptr;
    a.n = 0;
    a.pm = PixelMap{0.0f, 0.0f, 0.0f, 0.0f};
    a.max_dwell = 0;
    a.side = 0;
    a.leaves = q.leaves;
    a.leaf_cap = q.leaf_cap;
    a.skip_perimeter = 0;
    a.fills = nullptr;
    a.fill_cap = 0;
    a.frames = q.frames;
    a.ctr = q.ctr;
    const int threads = kRefillWarps * 32;
    if (count)
        queue_kernel<true><<<resident_grid(queue_kernel<true>, threads, sms), threads, 0, s>>>(q, a);
    else
        queue_kernel<false><<<resident_grid(queue_kernel<false>, threads, sms), threads, 0, s>>>(q, a);
    return cudaGetLastError();
}

}  // namespace ask
