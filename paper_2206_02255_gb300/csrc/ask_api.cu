// ask_api.cu -- host side of the C ABI declared in include/ask.h: argument
// checks, the subdivision plan, scratch ownership, and the launch sequence
// of each method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ask_fp64.h"
#include "ask_internal.h"

// Device scratch of a batch render (owned by a context, or by a graph).
struct BatchBuffers {
    uint4 *olt[2] = {nullptr, nullptr};  // region records with frame ids
    uint64_t olt_cap = 0;
    uint4 *leaves = nullptr;
    uint64_t leaf_cap = 0;
    uint4 *rst[2] = {nullptr, nullptr};
    uint64_t rst_cap = 0;
    uint4 *fills = nullptr;
    uint64_t fill_cap = 0;
    ask::FrameDesc *frames = nullptr;    // device frame table
    uint64_t frames_cap = 0;
    ask::DevCounters *ctr = nullptr;     // not owned when it is the context's
};

// Device scratch of a batch rendered by the persistent kernel (owned by a
// context, or by a graph): the work queue, chunk-query states, leaf list,
// frame table and queue state.  Queue and leaf slots are zeroed when
// allocated, so no stale word can carry a render's epoch.
struct QueueBuffers {
    uint4 *items = nullptr;
    uint32_t *aux = nullptr;
    uint64_t item_cap = 0;
    uint4 *rst = nullptr;
    uint64_t rst_cap = 0;
    uint4 *leaves = nullptr;
    uint64_t leaf_cap = 0;
    ask::FrameDesc *frames = nullptr;
    uint64_t frames_cap = 0;
    ask::QueueState *qs = nullptr;
    ask::DevCounters *ctr = nullptr;     // not owned when it is the context's
};

struct ask_ctx {
    ask::DeviceInfo dev;
    BatchBuffers batch;
    QueueBuffers queue;
    ask::FrameDesc *h_frames = nullptr;  // pinned staging of the frame table
    uint64_t h_frames_cap = 0;
    cudaEvent_t frames_copied = nullptr; // the staging buffer may be rewritten after it
    // region tables (double buffered), leaf list, counters
    uint2 *olt[2] = {nullptr, nullptr};
    uint64_t olt_cap = 0;
    uint2 *leaves = nullptr;
    uint64_t leaf_cap = 0;
    uint4 *rst[2] = {nullptr, nullptr};  // per-region state of chunked queries
    uint64_t rst_cap = 0;
    uint4 *fills = nullptr;              // deferred fills
    uint64_t fill_cap = 0;
    ask::DevCounters *ctr = nullptr;
    ask::DevCounters *h_ctr = nullptr;  // pinned mirror for stats
    // device map for ask_render_host (when the host buffer is not pinned)
    uint32_t *dmap = nullptr;
    size_t dmap_elems = 0;
    // banded ask_render_host: copy stream and one event per band
    static constexpr uint32_t kMaxBands = 64;
    cudaStream_t cpy = nullptr;
    cudaEvent_t band_ev[kMaxBands] = {};
    // events of the synchronous stats path: 0 = start, 1 = after init,
    // 2 + i = after level i, levels + 2 = after the leaf kernel
    cudaEvent_t ev[ASK_MAX_LEVELS + 4];
    bool events = false;
    // ASK_FLAG_TIMING: a ring of per-render event sets, read by ask_timing_read
    struct TimingSlot {
        cudaEvent_t ev[ASK_MAX_LEVELS + 4];
        uint32_t levels;
        uint32_t method;
    };
    static constexpr uint32_t kRing = 64;
    TimingSlot *ring = nullptr;
    uint64_t ring_head = 0, ring_tail = 0;
    uint32_t ring_dropped = 0;
    size_t cdp_pending = 0;
    char err[256];
};

struct ask_graph {
    int device = 0;
    BatchBuffers buf;
    QueueBuffers qbuf;
    bool persistent = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace ask {

static uint32_t ceil_div(uint32_t a, uint32_t b) { return a / b + (a % b != 0u); }

// Target bytes of map per band of the banded ask_render_host pipeline.  At
// n = 16384 (1 GiB) 8 bands of 128 MiB took 6.2 ms per call, 4 of 256 MiB
// 6.45 ms, and 16 of 64 MiB 8.4 ms: a band's render must stay shorter than
// its copy, and small bands leave the level kernels too few regions.
constexpr uint64_t kBandBytes = 128ull << 20;

bool make_plan(uint32_t n, uint32_t g, uint32_t r, uint32_t B, LevelPlan *plan, uint32_t chunk_px,
               uint64_t few_items)
{
    if (n == 0 || g == 0 || r < 2 || B == 0 || !plan)
        return false;
    std::memset(plan, 0, sizeof(*plan));
    // (levels are capped below ASK_MAX_LEVELS so event arrays have room)
    uint32_t s = ceil_div(n, g);
    // multiset of interval lengths along one axis: (length, how many)
    std::vector<std::pair<uint32_t, uint64_t>> lens;
    const uint32_t full = n / s, rem = n % s;
    if (full)
        lens.push_back({s, full});
    if (rem)
        lens.push_back({rem, 1});
    plan->axis0 = full + (rem ? 1u : 0u);
    for (uint32_t i = 0;; ++i) {
        if (i >= ASK_MAX_LEVELS - 2)
            return false;
        uint64_t axis = 0;
        for (auto &p : lens)
            axis += p.second;
        plan->side[i] = s;
        plan->max_regions[i] = axis * axis;
        if (plan->max_regions[i] >= 0xffffffffull)
            return false;
        const uint64_t per = (s <= 2u) ? (uint64_t)s * s : 4ull * s - 4ull;
        uint32_t cp = chunk_px;
        if (few_items && cp >= 64u && plan->max_regions[i] * ((per + cp - 1) / cp) < few_items)
            cp /= 2u;
        plan->chunk_px[i] = cp;
        plan->chunks[i] = (uint32_t)((per + cp - 1) / cp);
        if (plan->max_regions[i] * plan->chunks[i] >= 0xffffffffull)
            return false;
        const uint32_t sc = ceil_div(s, r);
        plan->split[i] = (s > 1u && sc >= B) ? 1u : 0u;
        plan->levels = i + 1;
        if (!plan->split[i])
            break;
        std::vector<std::pair<uint32_t, uint64_t>> next;
        auto add = [&next](uint32_t len, uint64_t cnt) {
            for (auto &q : next)
                if (q.first == len) {
                    q.second += cnt;
                    return;
                }
            next.push_back({len, cnt});
        };
        for (auto &p : lens) {
            if (p.first / sc)
                add(sc, (uint64_t)(p.first / sc) * p.second);
            if (p.first % sc)
                add(p.first % sc, p.second);
        }
        lens.swap(next);
        s = sc;
    }
    return true;
}

}  // namespace ask

using namespace ask;

namespace {

ask_status set_err(ask_ctx *ctx, ask_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

ask_status cuda_err(ask_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess)
        return ASK_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_err(ctx, ASK_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_err(ctx, ASK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool window_ok(const ask_window *w)
{
    return w && std::isfinite(w->re_min) && std::isfinite(w->re_max) && std::isfinite(w->im_min) &&
           std::isfinite(w->im_max) && w->re_max > w->re_min && w->im_max > w->im_min;
}

bool block_ok(uint32_t bx, uint32_t by)
{
    const uint64_t t = (uint64_t)bx * by;
    return bx >= 1 && by >= 1 && bx <= 1024 && by <= 1024 && t >= 32 && t <= 1024 && t % 32 == 0;
}

ask_status check_args(ask_ctx *ctx, ask_method method, const ask_window *window, uint32_t n,
                      uint32_t max_dwell, const ask_params *p, ask_params *eff)
{
    if (!ctx)
        return ASK_EINVAL;
    if (method != ASK_METHOD_EXHAUSTIVE && method != ASK_METHOD_ASK && method != ASK_METHOD_CDP2)
        return set_err(ctx, ASK_EINVAL, "unknown method %d", (int)method);
    if (!window_ok(window))
        return set_err(ctx, ASK_EINVAL, "window must be finite with min < max");
    if (n == 0 || n > ASK_MAX_N)
        return set_err(ctx, ASK_EINVAL, "n must be in [1, 65536]");
    if (max_dwell == 0 || max_dwell == 0xffffffffu)
        return set_err(ctx, ASK_EINVAL, "max_dwell must be in [1, 2^32 - 2]");
    ask_params d{};
    d.g = 16;
    d.r = 2;
    d.B = 32;
    d.block_x = 16;
    d.block_y = 16;
    d.flags = 0;
    if (p)
        d = *p;
    else if (method != ASK_METHOD_EXHAUSTIVE)
        return set_err(ctx, ASK_EINVAL, "params are required for subdivision methods");
    if (!block_ok(d.block_x, d.block_y))
        return set_err(ctx, ASK_EINVAL, "block_x * block_y must be a multiple of 32 in [32, 1024]");
    if (d.flags & ~(ASK_FLAG_COUNT | ASK_FLAG_TIMING | ASK_FLAG_CDP2_FIRE_AND_FORGET |
                    ASK_FLAG_EXACT_BORDERS | ASK_FLAG_LEAF_TILED | ASK_FLAG_SBR | ASK_FLAG_MBR |
                    ASK_FLAG_STAGED_COPY | ASK_FLAG_SERIAL_FILL | ASK_FLAG_INJECT_OVERFLOW))
        return set_err(ctx, ASK_EINVAL, "unknown flags 0x%x", d.flags);
    if ((d.flags & ASK_FLAG_SBR) && (d.flags & ASK_FLAG_MBR))
        return set_err(ctx, ASK_EINVAL, "ASK_FLAG_SBR and ASK_FLAG_MBR exclude each other");
    if ((d.flags & (ASK_FLAG_SBR | ASK_FLAG_MBR)) && (d.flags & (ASK_FLAG_EXACT_BORDERS | ASK_FLAG_LEAF_TILED)))
        return set_err(ctx, ASK_EINVAL,
                       "ASK_FLAG_SBR / ASK_FLAG_MBR do not combine with EXACT_BORDERS or LEAF_TILED");
    if (method != ASK_METHOD_EXHAUSTIVE) {
        if (d.g == 0 || d.g > n)
            return set_err(ctx, ASK_EINVAL, "g must be in [1, n]");
        if (d.r < 2 || d.r > 64)
            return set_err(ctx, ASK_EINVAL, "r must be in [2, 64]");
        if (d.B == 0)
            return set_err(ctx, ASK_EINVAL, "B must be >= 1");
    }
    *eff = d;
    return ASK_OK;
}

PixelMap pixel_map(const ask_window *w, uint32_t n)
{
    PixelMap pm;
    pm.re_min = w->re_min;
    pm.im_min = w->im_min;
    // float subtraction and division, each rounded once (no contraction is
    // possible in these expressions)
    const float wr = w->re_max - w->re_min;
    const float wi = w->im_max - w->im_min;
    pm.dx = wr / (float)n;
    pm.dy = wi / (float)n;
    return pm;
}

ask_status ensure_counters(ask_ctx *ctx)
{
    if (ctx->ctr)
        return ASK_OK;
    cudaError_t e = cudaMalloc(&ctx->ctr, sizeof(DevCounters));
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "cudaMalloc(counters)");
    e = cudaMemset(ctx->ctr, 0, sizeof(DevCounters));
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "cudaMemset(counters)");
    e = cudaMallocHost(&ctx->h_ctr, sizeof(DevCounters));
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "cudaMallocHost(counters)");
    return ASK_OK;
}

template <typename T>
ask_status grow(ask_ctx *ctx, T **buf, uint64_t *cap, uint64_t need, const char *what)
{
    if (need <= *cap)
        return ASK_OK;
    if (*buf)
        cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, need * sizeof(T));
    if (e != cudaSuccess)
        return cuda_err(ctx, e, what);
    *cap = need;
    return ASK_OK;
}

// Deferred fills can come from levels whose regions exceed the in-place size.
// Fill-list entries a render can append: the bands of the regions larger
// than the in-place limit, or (MBR) of every region of every level.  A
// clipped region has no more bands than a full one of its level.
uint64_t fill_need(const LevelPlan &plan, bool all = false)
{
    uint64_t need = 0;
    for (uint32_t i = 0; i < plan.levels; ++i)
        if (all || (uint64_t)plan.side[i] * plan.side[i] > kInPlaceFillArea)
            need += plan.max_regions[i] * fill_band_count(plan.side[i], plan.side[i]);
    return need;
}

ask_status reserve_ask(ask_ctx *ctx, const LevelPlan &plan, bool fill_all = false)
{
    uint64_t olt_need = 0, rst_need = 0;
    for (uint32_t i = 0; i < plan.levels; ++i) {
        if (plan.max_regions[i] > olt_need)
            olt_need = plan.max_regions[i];
        if (plan.chunks[i] > 1u && plan.max_regions[i] > rst_need)
            rst_need = plan.max_regions[i];
    }
    const uint64_t leaf_need = plan.max_regions[plan.levels - 1];
    ask_status st;
    if (olt_need > ctx->olt_cap) {
        uint64_t c0 = ctx->olt_cap, c1 = ctx->olt_cap;
        if ((st = grow(ctx, &ctx->olt[0], &c0, olt_need, "cudaMalloc(region table)")) != ASK_OK ||
            (st = grow(ctx, &ctx->olt[1], &c1, olt_need, "cudaMalloc(region table)")) != ASK_OK) {
            ctx->olt_cap = 0;
            return st;
        }
        ctx->olt_cap = olt_need;
    }
    if (rst_need > ctx->rst_cap) {
        uint64_t c0 = ctx->rst_cap, c1 = ctx->rst_cap;
        if ((st = grow(ctx, &ctx->rst[0], &c0, rst_need, "cudaMalloc(query state)")) != ASK_OK ||
            (st = grow(ctx, &ctx->rst[1], &c1, rst_need, "cudaMalloc(query state)")) != ASK_OK) {
            ctx->rst_cap = 0;
            return st;
        }
        ctx->rst_cap = rst_need;
    }
    if ((st = grow(ctx, &ctx->leaves, &ctx->leaf_cap, leaf_need, "cudaMalloc(leaf list)")) != ASK_OK)
        return st;
    if ((st = grow(ctx, &ctx->fills, &ctx->fill_cap, fill_need(plan, fill_all), "cudaMalloc(fill list)")) !=
        ASK_OK)
        return st;
    return ensure_counters(ctx);
}

ask_status ensure_events(ask_ctx *ctx)
{
    if (ctx->events)
        return ASK_OK;
    for (int i = 0; i < ASK_MAX_LEVELS + 4; ++i) {
        cudaError_t e = cudaEventCreate(&ctx->ev[i]);
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaEventCreate");
    }
    ctx->events = true;
    return ASK_OK;
}

ask_status latched_error(ask_ctx *ctx, uint32_t err)
{
    if (err & ERR_DEVICE_LAUNCH)
        return set_err(ctx, ASK_ECUDA, "a device-side child launch failed (pending-launch limit?)");
    if (err & (ERR_OLT_OVERFLOW | ERR_LEAF_OVERFLOW))
        return set_err(ctx, ASK_EOVERFLOW, "a region table overflowed its capacity");
    if (err & ERR_TIMEOUT)
        return set_err(ctx, ASK_ETIMEOUT, "a bounded wait of the persistent batch kernel gave up");
    if (err)
        return set_err(ctx, ASK_EOVERFLOW, "device error bits 0x%x", err);
    return ASK_OK;
}

// Copy counters back (the stream is synchronised), clear the latched error.
ask_status read_counters(ask_ctx *ctx, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(ctx->h_ctr, ctx->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "reading device counters");
    const uint32_t err = ctx->h_ctr->error;
    if (err) {
        e = cudaMemsetAsync(&ctx->ctr->error, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "clearing the device error word");
    }
    return latched_error(ctx, err);
}

ask_status ensure_bands(ask_ctx *ctx)
{
    if (ctx->cpy)
        return ASK_OK;
    for (uint32_t b = 0; b < ask_ctx::kMaxBands; ++b) {
        cudaError_t e = cudaEventCreateWithFlags(&ctx->band_ev[b], cudaEventDisableTiming);
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaEventCreate");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->cpy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        ctx->cpy = nullptr;
        return cuda_err(ctx, e, "copy stream");
    }
    return ASK_OK;
}

ask_status ensure_ring(ask_ctx *ctx)
{
    if (ctx->ring)
        return ASK_OK;
    ask_ctx::TimingSlot *ring = new (std::nothrow) ask_ctx::TimingSlot[ask_ctx::kRing];
    if (!ring)
        return set_err(ctx, ASK_ENOMEM, "timing ring");
    for (uint32_t k = 0; k < ask_ctx::kRing; ++k) {
        ring[k].levels = 0;
        ring[k].method = 0;
        for (int i = 0; i < ASK_MAX_LEVELS + 4; ++i) {
            cudaError_t e = cudaEventCreate(&ring[k].ev[i]);
            if (e != cudaSuccess) {
                delete[] ring;
                return cuda_err(ctx, e, "cudaEventCreate");
            }
        }
    }
    ctx->ring = ring;
    return ASK_OK;
}

// Event marks of one render: the stats events and/or a timing-ring slot.
struct Marks {
    cudaEvent_t *st = nullptr;
    cudaEvent_t *tm = nullptr;
    void at(int k, cudaStream_t s) const
    {
        if (st)
            cudaEventRecord(st[k], s);
        if (tm)
            cudaEventRecord(tm[k], s);
    }
};

// ASK renders only the initial-region rows [row0, row0 + rows) when rows is
// given (the banded host pipeline); every other method renders the frame.
ask_status render_impl(ask_ctx *ctx, ask_method method, const ask_window *window, uint32_t n,
                       uint32_t max_dwell, const ask_params &p, uint32_t *d_dwell, cudaStream_t s,
                       ask_stats *stats, uint32_t row0 = 0, uint32_t rows = 0xffffffffu)
{
    const bool count = (p.flags & ASK_FLAG_COUNT) != 0;
    const bool timing = (p.flags & ASK_FLAG_TIMING) != 0;
    const PixelMap pm = pixel_map(window, n);
    ask_status st;
    cudaError_t e;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        if ((st = ensure_events(ctx)) != ASK_OK)
            return st;
    }
    if (timing && (st = ensure_ring(ctx)) != ASK_OK)
        return st;
    if ((st = ensure_counters(ctx)) != ASK_OK)
        return st;
    Marks mk;
    if (stats)
        mk.st = ctx->ev;
    ask_ctx::TimingSlot *slot = nullptr;
    if (timing) {
        if (ctx->ring_head - ctx->ring_tail == ask_ctx::kRing) {
            ++ctx->ring_tail;  // the oldest unread render is overwritten
            ++ctx->ring_dropped;
        }
        slot = &ctx->ring[ctx->ring_head % ask_ctx::kRing];
        slot->method = (uint32_t)method;
        slot->levels = 0;
        mk.tm = slot->ev;
    }
    uint32_t launches = 0;

    if (method == ASK_METHOD_EXHAUSTIVE) {
        mk.at(0, s);
        if (count) {
            if ((e = launch_init(nullptr, nullptr, ctx->ctr, n, 1, 0, 0, 0, s)) != cudaSuccess)
                return cuda_err(ctx, e, "init kernel");
            ++launches;
        }
        if ((e = launch_exhaustive(d_dwell, n, pm, max_dwell, p.block_x, p.block_y, count, ctx->ctr, s)) !=
            cudaSuccess)
            return cuda_err(ctx, e, "exhaustive kernel");
        ++launches;
        mk.at(1, s);
        if (timing)
            ++ctx->ring_head;
        if (stats) {
            if ((st = read_counters(ctx, s)) != ASK_OK)
                return st;
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[1]);
            stats->iterations = count ? ctx->h_ctr->iterations : 0;
            stats->kernel_launches = launches;
        }
        return ASK_OK;
    }

    LevelPlan plan;
    if (!make_plan(n, p.g, p.r, p.B, &plan))
        return set_err(ctx, ASK_EINVAL, "no valid subdivision plan for n=%u g=%u r=%u B=%u", n, p.g, p.r, p.B);

    if (method == ASK_METHOD_CDP2) {
        if (plan.levels > 23)
            return set_err(ctx, ASK_EINVAL, "CDP2 nesting would exceed the device runtime's depth limit");
        // At most one pending launch per subdividing region of a level.  The
        // limit is set generously on first use; raising it later may be
        // refused once device-runtime kernels have run, in which case the old
        // limit stays and a device launch that exceeds it is latched as an
        // error (never a hang or a fault).
        // DP-MBR: every region may launch one child, so bound by the sum.
        const bool mbr = (p.flags & ASK_FLAG_MBR) != 0;
        uint64_t need = 1u << 18, sum = 0;
        for (uint32_t i = 0; i < plan.levels; ++i) {
            if (plan.split[i] && plan.max_regions[i] > need)
                need = plan.max_regions[i];
            sum += plan.max_regions[i];
        }
        if (mbr && sum > need)
            need = sum;
        if (need > (1u << 22))
            need = 1u << 22;
        if (need > ctx->cdp_pending) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
                return cuda_err(ctx, e, "cudaStreamSynchronize");
            if (cdp2_set_pending_limit((size_t)need) == cudaSuccess)
                ctx->cdp_pending = (size_t)need;
            else if (ctx->cdp_pending == 0)
                return set_err(ctx, ASK_EUNSUPPORTED, "cannot set the device runtime's pending-launch limit");
            cudaGetLastError();  // a refused raise is not sticky
        }
        // tail launches without MBR: one device-launched grid per depth over
        // a list of that depth's regions (the region tables hold the lists)
        const bool fnf = (p.flags & ASK_FLAG_CDP2_FIRE_AND_FORGET) != 0;
        if (!fnf && !mbr && (st = reserve_ask(ctx, plan)) != ASK_OK)
            return st;
        mk.at(0, s);
        if ((e = launch_init(nullptr, nullptr, ctx->ctr, n, 1, 0, 0, 0, s)) != cudaSuccess)
            return cuda_err(ctx, e, "init kernel");
        CdpArgs a;
        a.map = d_dwell;
        a.n = n;
        a.pm = pm;
        a.max_dwell = max_dwell;
        a.r = p.r;
        a.B = p.B;
        a.count = count ? 1u : 0u;
        a.fire_and_forget = (p.flags & ASK_FLAG_CDP2_FIRE_AND_FORGET) ? 1u : 0u;
        a.mbr = mbr ? 1u : 0u;
        a.list[0] = (!fnf && !mbr) ? ctx->olt[0] : nullptr;
        a.list[1] = (!fnf && !mbr) ? ctx->olt[1] : nullptr;
        a.list_cap = (!fnf && !mbr) ? (uint32_t)ctx->olt_cap : 0u;
        a.ctr = ctx->ctr;
        if ((e = launch_cdp2(a, p.g, plan.side[0], p.block_x, p.block_y, s)) != cudaSuccess)
            return cuda_err(ctx, e, "CDP2 root kernel");
        launches = 2;
        mk.at(1, s);
        if (timing)
            ++ctx->ring_head;
        if (stats) {
            if ((st = read_counters(ctx, s)) != ASK_OK)
                return st;
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[1]);
            const DevCounters &c = *ctx->h_ctr;
            stats->levels = plan.levels;
            for (uint32_t i = 0; i < plan.levels; ++i) {
                stats->fills_per_level[i] = c.fills[i];
                stats->subdivisions_per_level[i] = c.subdivs[i];
            }
            stats->leaves = c.leaf_count + c.leaf_light;
            stats->iterations = c.iterations;
            stats->kernel_launches = launches;
        }
        return ASK_OK;
    }

    // ---- ASK: init, one level kernel per depth, fills, leaf kernel --------
    // The SBR / MBR mappings take whole regions per CTA: no chunked queries.
    const bool sbr = (p.flags & ASK_FLAG_SBR) != 0, mbr = (p.flags & ASK_FLAG_MBR) != 0;
    if (sbr || mbr)
        for (uint32_t i = 0; i < plan.levels; ++i)
            plan.chunks[i] = 1u;
    if ((st = reserve_ask(ctx, plan, mbr)) != ASK_OK)
        return st;
    const int sms = ctx->dev.sms;
    const uint32_t L = plan.levels;
    const bool exact = (p.flags & ASK_FLAG_EXACT_BORDERS) != 0;
    // ASK_FLAG_INJECT_OVERFLOW: the kernels see region tables of capacity 1
    // (the allocations keep their full size, so nothing is written out of
    // bounds) and latch the overflow, as a real one would be.
    const bool inject = (p.flags & ASK_FLAG_INJECT_OVERFLOW) != 0;
    const uint32_t olt_cap = inject ? 1u : (uint32_t)ctx->olt_cap;
    const uint32_t leaf_cap = inject ? 1u : (uint32_t)ctx->leaf_cap;
    mk.at(0, s);
    if (row0 >= plan.axis0)
        return set_err(ctx, ASK_EINVAL, "band starts past the last initial-region row");
    const uint32_t rows0 = std::min(rows, plan.axis0 - row0);
    if ((e = launch_init(ctx->olt[0], plan.chunks[0] > 1u ? ctx->rst[0] : nullptr, ctx->ctr, n,
                         plan.side[0], plan.axis0, row0, rows0, s, (sbr || mbr) ? nullptr : &pm)) !=
        cudaSuccess)
        return cuda_err(ctx, e, "init kernel");
    // the bound on level i's regions, which its table fills from both ends:
    // the initial regions written, then (intervals per axis)^2
    auto level_cap = [&](uint32_t i) -> uint32_t {
        const uint64_t c = (i == 0) ? (uint64_t)plan.axis0 * rows0 : plan.max_regions[i];
        return (uint32_t)std::min<uint64_t>(c, olt_cap);
    };
    ++launches;
    mk.at(1, s);
    for (uint32_t i = 0; i < L; ++i) {
        LevelArgs a;
        a.map = d_dwell;
        a.n = n;
        a.pm = pm;
        a.max_dwell = max_dwell;
        a.level = i;
        a.side = plan.side[i];
        a.split = plan.split[i];
        a.child_side = ceil_div(plan.side[i], p.r);
        a.r = p.r;
        a.olt_in = ctx->olt[i & 1];
        a.olt_out = ctx->olt[(i + 1) & 1];
        a.olt_cap = olt_cap;
        a.in_cap = level_cap(i);
        a.out_cap = (i + 1 < L) ? level_cap(i + 1) : 0u;
        a.chunks = plan.chunks[i];
        a.chunk_px = plan.chunk_px[i];
        a.next_chunks = (i + 1 < L) ? plan.chunks[i + 1] : 1u;
        a.rst_in = ctx->rst[i & 1];
        a.rst_out = ctx->rst[(i + 1) & 1];
        a.leaves = ctx->leaves;
        a.leaf_cap = leaf_cap;
        a.fills = ctx->fill_cap ? ctx->fills : nullptr;
        a.fill_cap = (uint32_t)ctx->fill_cap;
        a.exact_last = exact ? 1u : 0u;
        a.ctr = ctx->ctr;
        if (sbr || mbr)
            e = launch_level_region(a, mbr, count, p.block_x * p.block_y, sms, s);
        else
            e = launch_level(a, count, false, sms, s);
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "level kernel");
        ++launches;
        mk.at(2 + (int)i, s);
    }
    // Marks: L + 1 = levels done (fill and leaf start), L + 2 = fill done,
    // L + 3 = leaf done, L + 4 = render done.  With the default mapping the
    // deferred fills (HBM writes) ride along the lane-refill leaf kernel
    // (FP32 work): its warps write one band of the fill list every few
    // rounds.  The tiled leaf kernel, the MBR mapping and
    // ASK_FLAG_SERIAL_FILL run the fill kernel alone first.
    const bool tiled = mbr || (p.flags & ASK_FLAG_LEAF_TILED) != 0;
    const bool fills = !sbr && fill_need(plan, mbr) > 0;
    const bool fused = fills && !tiled && !(p.flags & ASK_FLAG_SERIAL_FILL);
    if (fills && !fused) {
        FillArgs f;
        f.map = d_dwell;
        f.n = n;
        f.fills = ctx->fills;
        f.fill_cap = (uint32_t)ctx->fill_cap;
        f.ctr = ctx->ctr;
        if ((e = launch_fill(f, false, sms, s)) != cudaSuccess)
            return cuda_err(ctx, e, "fill kernel");
        ++launches;
    }
    mk.at(2 + (int)L, s);
    LeafArgs la;
    la.map = d_dwell;
    la.n = n;
    la.pm = pm;
    la.max_dwell = max_dwell;
    la.side = plan.side[L - 1];
    la.leaves = ctx->leaves;
    la.leaf_cap = leaf_cap;
    la.skip_perimeter = exact ? 1u : 0u;
    la.fills = fused ? ctx->fills : nullptr;
    la.fill_cap = fused ? (uint32_t)ctx->fill_cap : 0u;
    la.ctr = ctx->ctr;
    if (sbr)
        e = launch_leaf_region(la, p.block_x, p.block_y, count, sms, s);
    else
        e = launch_leaf(la, p.block_x, p.block_y, count, tiled, false, sms, s);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "leaf kernel");
    ++launches;
    mk.at(3 + (int)L, s);
    mk.at(4 + (int)L, s);
    if (timing) {
        slot->levels = L;
        ++ctx->ring_head;
    }
    if (stats) {
        if ((st = read_counters(ctx, s)) != ASK_OK)
            return st;
        cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[L + 4]);
        for (uint32_t i = 0; i < L; ++i)
            cudaEventElapsedTime(&stats->ms_per_level[i], ctx->ev[i + 1], ctx->ev[i + 2]);
        cudaEventElapsedTime(&stats->ms_fill, ctx->ev[L + 1], ctx->ev[L + 2]);
        cudaEventElapsedTime(&stats->ms_leaf, ctx->ev[L + 2], ctx->ev[L + 3]);
        const DevCounters &c = *ctx->h_ctr;
        stats->levels = L;
        for (uint32_t i = 0; i < L; ++i) {
            stats->regions_per_level[i] = c.count[i] + c.back[i];
            stats->fills_per_level[i] = c.fills[i];
            stats->subdivisions_per_level[i] = c.subdivs[i];
            stats->iterations_per_level[i] = c.level_iters[i];
        }
        stats->leaves = c.leaf_count + c.leaf_light;
        stats->fill_pixels = c.fill_pixels;
        stats->deferred_fill_pixels = c.deferred_fill_pixels;
        stats->leaf_pixels = c.leaf_pixels;
        stats->border_pixels = c.border_pixels;
        stats->iterations = c.iterations;
        stats->leaf_iterations = c.leaf_iters;
        stats->kernel_launches = launches;
    }
    return ASK_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
struct BatchPlan {
    std::vector<FrameDesc> desc;
    uint32_t L = 0;                       // deepest level over the frames
    uint32_t chunks[ASK_MAX_LEVELS] = {};  // chunks per region at each level (max over frames)
    uint64_t olt_need = 0, leaf_need = 0, rst_need = 0, fill_need = 0;
    uint64_t level_cap[ASK_MAX_LEVELS] = {};  // bound on each level's regions over the frames
    uint32_t total0 = 0;
    // the persistent batch kernel: queue items (every level's chunk items and
    // fill bands of every frame), chunk states, level-0 items and states
    uint64_t q_items = 0, q_states = 0, q_total0 = 0, q_states0 = 0;
};

// Chunk items per region of a level of side s in the persistent batch
// kernel: kChunkPxQueue perimeter pixels each, at most kMaxChunksQueue.
uint32_t queue_chunks(uint32_t s)
{
    const uint64_t per = (s <= 2u) ? (uint64_t)s * s : 4ull * s - 4ull;
    const uint64_t c = (per + kChunkPxQueue - 1) / kChunkPxQueue;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(c, kMaxChunksQueue));
}

ask_status plan_batch(ask_ctx *ctx, const ask_frame *frames, uint32_t nframes, uint32_t flags,
                      uint32_t allowed_flags, BatchPlan &bp)
{
    if (!frames || nframes == 0 || nframes > (1u << 20))
        return set_err(ctx, ASK_EINVAL, "a batch needs 1 to 2^20 frames");
    if (flags & ~allowed_flags)
        return set_err(ctx, ASK_EINVAL, "unsupported flags 0x%x for a batch", flags);
    bp.desc.resize(nframes);
    uint64_t level_regions[ASK_MAX_LEVELS] = {};
    uint64_t total0 = 0;
    for (uint32_t f = 0; f < nframes; ++f) {
        const ask_frame &fr = frames[f];
        ask_params p{};
        p.g = fr.g;
        p.r = fr.r;
        p.B = fr.B;
        p.block_x = 16;
        p.block_y = 16;
        ask_params eff;
        ask_status st = check_args(ctx, ASK_METHOD_ASK, &fr.window, fr.n, fr.max_dwell, &p, &eff);
        if (st != ASK_OK) {
            char why[sizeof(ctx->err)];
            std::memcpy(why, ctx->err, sizeof(why));
            return set_err(ctx, st, "frame %u: %s", f, why);
        }
        if (!fr.d_dwell || ((uintptr_t)fr.d_dwell & 15u))
            return set_err(ctx, ASK_EINVAL, "frame %u: d_dwell must be 16-byte aligned", f);
        LevelPlan plan;
        if (!make_plan(fr.n, fr.g, fr.r, fr.B, &plan, kChunkPxBatch, 0))
            return set_err(ctx, ASK_EINVAL, "frame %u: no valid subdivision plan", f);
        FrameDesc &d = bp.desc[f];
        std::memset(&d, 0, sizeof(d));
        d.map = fr.d_dwell;
        d.pm = pixel_map(&fr.window, fr.n);
        d.n = fr.n;
        d.max_dwell = fr.max_dwell;
        d.r = fr.r;
        d.levels = plan.levels;
        d.s0 = plan.side[0];
        d.axis0 = plan.axis0;
        d.olt0_offset = (uint32_t)total0;
        d.item0 = (uint32_t)std::min<uint64_t>(bp.q_total0, 0xffffffffull);
        d.state0 = (uint32_t)std::min<uint64_t>(bp.q_states0, 0xffffffffull);
        for (uint32_t i = 0; i < plan.levels; ++i) {
            d.side[i] = plan.side[i];
            d.chunks[i] = queue_chunks(plan.side[i]);
            level_regions[i] += plan.max_regions[i];
            if (plan.chunks[i] > bp.chunks[i])
                bp.chunks[i] = plan.chunks[i];
            bp.q_items += plan.max_regions[i] * d.chunks[i];
            if (d.chunks[i] > 1u)
                bp.q_states += plan.max_regions[i];
            if ((uint64_t)plan.side[i] * plan.side[i] > kInPlaceFillArea) {
                const uint64_t bands = plan.max_regions[i] * fill_band_count(plan.side[i], plan.side[i]);
                bp.fill_need += bands;
                bp.q_items += bands;
            }
        }
        const uint64_t regions0 = (uint64_t)plan.axis0 * plan.axis0;
        bp.q_total0 += regions0 * d.chunks[0];
        if (d.chunks[0] > 1u)
            bp.q_states0 += regions0;
        bp.leaf_need += plan.max_regions[plan.levels - 1];
        total0 += (uint64_t)plan.axis0 * plan.axis0;
        if (plan.levels > bp.L)
            bp.L = plan.levels;
    }
    for (uint32_t i = 0; i < bp.L; ++i) {
        bp.chunks[i] = std::min(bp.chunks[i], kMaxChunksBatch);
        if (level_regions[i] * bp.chunks[i] >= 0xffffffffull)
            return set_err(ctx, ASK_EINVAL, "batch too large: level %u holds too many work items", i);
        bp.level_cap[i] = level_regions[i];
        if (level_regions[i] > bp.olt_need)
            bp.olt_need = level_regions[i];
        if (bp.chunks[i] > 1u && level_regions[i] > bp.rst_need)
            bp.rst_need = level_regions[i];
    }
    if (bp.leaf_need >= 0xffffffffull || bp.fill_need >= 0xffffffffull)
        return set_err(ctx, ASK_EINVAL, "batch too large");
    if ((flags & ASK_FLAG_PERSISTENT) && (bp.q_items >= 0xffffffffull || bp.q_states >= 0xffffffffull))
        return set_err(ctx, ASK_EINVAL, "batch too large for the persistent kernel's work queue");
    bp.total0 = (uint32_t)total0;
    return ASK_OK;
}

ask_status reserve_batch(ask_ctx *ctx, BatchBuffers &b, const BatchPlan &bp, bool own_counters)
{
    ask_status st;
    if (bp.olt_need > b.olt_cap) {
        uint64_t c0 = b.olt_cap, c1 = b.olt_cap;
        if ((st = grow(ctx, &b.olt[0], &c0, bp.olt_need, "cudaMalloc(batch regions)")) != ASK_OK ||
            (st = grow(ctx, &b.olt[1], &c1, bp.olt_need, "cudaMalloc(batch regions)")) != ASK_OK) {
            b.olt_cap = 0;
            return st;
        }
        b.olt_cap = bp.olt_need;
    }
    if (bp.rst_need > b.rst_cap) {
        uint64_t c0 = b.rst_cap, c1 = b.rst_cap;
        if ((st = grow(ctx, &b.rst[0], &c0, bp.rst_need, "cudaMalloc(batch query state)")) != ASK_OK ||
            (st = grow(ctx, &b.rst[1], &c1, bp.rst_need, "cudaMalloc(batch query state)")) != ASK_OK) {
            b.rst_cap = 0;
            return st;
        }
        b.rst_cap = bp.rst_need;
    }
    if ((st = grow(ctx, &b.leaves, &b.leaf_cap, bp.leaf_need, "cudaMalloc(batch leaves)")) != ASK_OK)
        return st;
    if ((st = grow(ctx, &b.fills, &b.fill_cap, bp.fill_need, "cudaMalloc(batch fills)")) != ASK_OK)
        return st;
    if ((st = grow(ctx, &b.frames, &b.frames_cap, (uint64_t)bp.desc.size(), "cudaMalloc(frame table)")) !=
        ASK_OK)
        return st;
    if (own_counters && !b.ctr) {
        cudaError_t e = cudaMalloc(&b.ctr, sizeof(DevCounters));
        if (e == cudaSuccess)
            e = cudaMemset(b.ctr, 0, sizeof(DevCounters));
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaMalloc(batch counters)");
    }
    return ASK_OK;
}

void free_batch(BatchBuffers &b, bool own_counters)
{
    for (int k = 0; k < 2; ++k) {
        if (b.olt[k])
            cudaFree(b.olt[k]);
        if (b.rst[k])
            cudaFree(b.rst[k]);
    }
    if (b.leaves)
        cudaFree(b.leaves);
    if (b.fills)
        cudaFree(b.fills);
    if (b.frames)
        cudaFree(b.frames);
    if (own_counters && b.ctr)
        cudaFree(b.ctr);
    b = BatchBuffers();
}

// The launch chain of a batch; the frame table must already be on the device.
ask_status enqueue_batch(ask_ctx *ctx, const BatchBuffers &b, const BatchPlan &bp, uint32_t flags,
                         cudaStream_t s, uint32_t *launches)
{
    const int sms = ctx->dev.sms;
    const bool count = (flags & ASK_FLAG_COUNT) != 0;
    const bool exact = (flags & ASK_FLAG_EXACT_BORDERS) != 0;
    const uint32_t nframes = (uint32_t)bp.desc.size();
    cudaError_t e;
    if ((e = launch_init_batch(b.olt[0], bp.chunks[0] > 1u ? b.rst[0] : nullptr, b.ctr, b.frames, nframes,
                               bp.total0, s)) != cudaSuccess)
        return cuda_err(ctx, e, "batch init kernel");
    uint32_t n_launch = 1;
    for (uint32_t i = 0; i < bp.L; ++i) {
        LevelArgs a;
        std::memset(&a, 0, sizeof(a));
        a.level = i;
        a.olt_in = b.olt[i & 1];
        a.olt_out = b.olt[(i + 1) & 1];
        a.olt_cap = (uint32_t)b.olt_cap;
        a.in_cap = (i == 0) ? bp.total0 : (uint32_t)bp.level_cap[i];
        a.out_cap = (i + 1 < bp.L) ? (uint32_t)bp.level_cap[i + 1] : 0u;
        a.chunks = bp.chunks[i];
        a.next_chunks = (i + 1 < bp.L) ? bp.chunks[i + 1] : 1u;
        a.rst_in = b.rst[i & 1];
        a.rst_out = b.rst[(i + 1) & 1];
        a.leaves = b.leaves;
        a.leaf_cap = (uint32_t)b.leaf_cap;
        a.fills = bp.fill_need ? b.fills : nullptr;
        a.fill_cap = (uint32_t)b.fill_cap;
        a.exact_last = exact ? 1u : 0u;
        a.frames = b.frames;
        a.ctr = b.ctr;
        if ((e = launch_level(a, count, true, sms, s)) != cudaSuccess)
            return cuda_err(ctx, e, "batch level kernel");
        ++n_launch;
    }
    // the deferred fills ride along the leaf kernel
    LeafArgs la;
    std::memset(&la, 0, sizeof(la));
    la.fills = bp.fill_need ? b.fills : nullptr;
    la.fill_cap = bp.fill_need ? (uint32_t)b.fill_cap : 0u;
    la.leaves = b.leaves;
    la.leaf_cap = (uint32_t)b.leaf_cap;
    la.skip_perimeter = exact ? 1u : 0u;
    la.frames = b.frames;
    la.ctr = b.ctr;
    if ((e = launch_leaf(la, 16, 16, count, false, true, sms, s)) != cudaSuccess)
        return cuda_err(ctx, e, "batch leaf kernel");
    ++n_launch;
    if (launches)
        *launches = n_launch;
    return ASK_OK;
}

// Copy the frame table through the context's pinned staging buffer.
ask_status upload_frames(ask_ctx *ctx, FrameDesc *dst, const BatchPlan &bp, cudaStream_t s)
{
    const uint64_t nf = bp.desc.size();
    cudaError_t e;
    if (ctx->frames_copied && (e = cudaEventSynchronize(ctx->frames_copied)) != cudaSuccess)
        return cuda_err(ctx, e, "waiting for the previous frame-table copy");
    if (nf > ctx->h_frames_cap) {
        if (ctx->h_frames)
            cudaFreeHost(ctx->h_frames);
        ctx->h_frames = nullptr;
        ctx->h_frames_cap = 0;
        if ((e = cudaMallocHost(&ctx->h_frames, nf * sizeof(FrameDesc))) != cudaSuccess)
            return cuda_err(ctx, e, "cudaMallocHost(frame table)");
        ctx->h_frames_cap = nf;
    }
    if (!ctx->frames_copied && (e = cudaEventCreateWithFlags(&ctx->frames_copied, cudaEventDisableTiming)) !=
                                   cudaSuccess)
        return cuda_err(ctx, e, "cudaEventCreate");
    std::memcpy(ctx->h_frames, bp.desc.data(), nf * sizeof(FrameDesc));
    if ((e = cudaMemcpyAsync(dst, ctx->h_frames, nf * sizeof(FrameDesc), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_err(ctx, e, "copying the frame table");
    if ((e = cudaEventRecord(ctx->frames_copied, s)) != cudaSuccess)
        return cuda_err(ctx, e, "cudaEventRecord");
    return ASK_OK;
}

// ---------------------------------------------------------------------------
// Batches rendered by the persistent kernel over a device work queue
// ---------------------------------------------------------------------------

// Grow a queue array, zeroing new memory so that no word in it can carry a
// render's epoch.
template <typename T>
ask_status grow_zeroed(ask_ctx *ctx, T **buf, uint64_t *cap, uint64_t need, const char *what)
{
    if (need <= *cap)
        return ASK_OK;
    ask_status st = grow(ctx, buf, cap, need, what);
    if (st != ASK_OK)
        return st;
    cudaError_t e = cudaMemset(*buf, 0, need * sizeof(T));
    return e == cudaSuccess ? ASK_OK : cuda_err(ctx, e, what);
}

ask_status reserve_queue(ask_ctx *ctx, QueueBuffers &b, const BatchPlan &bp, bool own_counters)
{
    ask_status st;
    if (bp.q_items > b.item_cap) {
        uint64_t c = b.item_cap;
        if ((st = grow_zeroed(ctx, &b.items, &c, bp.q_items, "cudaMalloc(work queue)")) != ASK_OK ||
            (st = grow(ctx, &b.aux, &b.item_cap, bp.q_items, "cudaMalloc(work queue)")) != ASK_OK) {
            b.item_cap = 0;
            return st;
        }
    }
    if ((st = grow(ctx, &b.rst, &b.rst_cap, std::max<uint64_t>(bp.q_states, 1), "cudaMalloc(query states)")) !=
        ASK_OK)
        return st;
    if ((st = grow_zeroed(ctx, &b.leaves, &b.leaf_cap, bp.leaf_need, "cudaMalloc(leaf list)")) != ASK_OK)
        return st;
    if ((st = grow(ctx, &b.frames, &b.frames_cap, (uint64_t)bp.desc.size(), "cudaMalloc(frame table)")) != ASK_OK)
        return st;
    if (!b.qs) {
        cudaError_t e = cudaMalloc(&b.qs, sizeof(QueueState));
        if (e == cudaSuccess)
            e = cudaMemset(b.qs, 0, sizeof(QueueState));
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaMalloc(queue state)");
    }
    if (own_counters && !b.ctr) {
        cudaError_t e = cudaMalloc(&b.ctr, sizeof(DevCounters));
        if (e == cudaSuccess)
            e = cudaMemset(b.ctr, 0, sizeof(DevCounters));
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaMalloc(batch counters)");
    }
    return ASK_OK;
}

void free_queue(QueueBuffers &b, bool own_counters)
{
    void *bufs[] = {b.items, b.aux, b.rst, b.leaves, b.frames, b.qs};
    for (void *p : bufs)
        if (p)
            cudaFree(p);
    if (own_counters && b.ctr)
        cudaFree(b.ctr);
    b = QueueBuffers();
}

// The two launches of a persistent batch: the init kernel and the
// persistent kernel; the frame table must already be on the device.
ask_status enqueue_queue(ask_ctx *ctx, const QueueBuffers &b, const BatchPlan &bp, uint32_t flags,
                         cudaStream_t s, uint32_t *launches)
{
    QueueArgs q;
    q.items = b.items;
    q.aux = b.aux;
    q.item_cap = (uint32_t)b.item_cap;
    q.rst = b.rst;
    q.rst_cap = (uint32_t)b.rst_cap;
    q.leaves = b.leaves;
    q.leaf_cap = (uint32_t)b.leaf_cap;
    q.frames = b.frames;
    q.ctr = b.ctr;
    q.qs = b.qs;
    q.regions0 = bp.total0;
    q.total0 = (uint32_t)bp.q_total0;
    q.states0 = (uint32_t)bp.q_states0;
    q.chunk_px = kChunkPxQueue;
    q.wait_limit = (flags & ASK_FLAG_WAIT_TEST) ? 0u : kQueueWaitLimit;
    cudaError_t e = launch_queue(q, (uint32_t)bp.desc.size(), (flags & ASK_FLAG_COUNT) != 0, ctx->dev.sms, s);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "persistent batch kernel");
    if (launches)
        *launches = 2;
    return ASK_OK;
}

}  // namespace

extern "C" {

const char *ask_version(void) { return "ask-gb300 0.1 (sm_103a)"; }

const char *ask_status_str(ask_status s)
{
    switch (s) {
    case ASK_OK: return "ok";
    case ASK_EINVAL: return "invalid argument";
    case ASK_ENOMEM: return "out of memory";
    case ASK_ECUDA: return "CUDA error";
    case ASK_EOVERFLOW: return "device capacity overflow";
    case ASK_ETIMEOUT: return "device wait timed out";
    case ASK_EUNSUPPORTED: return "unsupported device";
    case ASK_ECAPACITY: return "request exceeds the fixed scratch of ask_render_noalloc";
    }
    return "unknown status";
}

const char *ask_last_error(const ask_ctx *ctx) { return ctx ? ctx->err : ""; }

ask_status ask_ctx_create(ask_ctx **out, int device)
{
    if (!out)
        return ASK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0 || device < 0 || device >= ndev)
        return ASK_EUNSUPPORTED;
    if (cudaSetDevice(device) != cudaSuccess)
        return ASK_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return ASK_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3))
        return ASK_EUNSUPPORTED;  // the library is built for sm_103a only
    ask_ctx *ctx = new (std::nothrow) ask_ctx();
    if (!ctx)
        return ASK_ENOMEM;
    ctx->err[0] = 0;
    ctx->dev.device = device;
    ctx->dev.sms = prop.multiProcessorCount;
    ctx->dev.cc_major = prop.major;
    ctx->dev.cc_minor = prop.minor;
    *out = ctx;
    return ASK_OK;
}

void ask_ctx_destroy(ask_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->dev.device);
    for (int b = 0; b < 2; ++b)
        if (ctx->olt[b])
            cudaFree(ctx->olt[b]);
    if (ctx->leaves)
        cudaFree(ctx->leaves);
    for (int b = 0; b < 2; ++b)
        if (ctx->rst[b])
            cudaFree(ctx->rst[b]);
    if (ctx->fills)
        cudaFree(ctx->fills);
    free_batch(ctx->batch, false);
    free_queue(ctx->queue, false);
    if (ctx->h_frames)
        cudaFreeHost(ctx->h_frames);
    if (ctx->frames_copied)
        cudaEventDestroy(ctx->frames_copied);
    if (ctx->ctr)
        cudaFree(ctx->ctr);
    if (ctx->h_ctr)
        cudaFreeHost(ctx->h_ctr);
    if (ctx->dmap)
        cudaFree(ctx->dmap);
    if (ctx->cpy)
        cudaStreamDestroy(ctx->cpy);
    for (uint32_t b = 0; b < ask_ctx::kMaxBands; ++b)
        if (ctx->band_ev[b])
            cudaEventDestroy(ctx->band_ev[b]);
    if (ctx->events)
        for (int i = 0; i < ASK_MAX_LEVELS + 4; ++i)
            cudaEventDestroy(ctx->ev[i]);
    if (ctx->ring) {
        for (uint32_t k = 0; k < ask_ctx::kRing; ++k)
            for (int i = 0; i < ASK_MAX_LEVELS + 4; ++i)
                cudaEventDestroy(ctx->ring[k].ev[i]);
        delete[] ctx->ring;
    }
    delete ctx;
}

ask_status ask_plan_levels(uint32_t n, uint32_t g, uint32_t r, uint32_t B, uint32_t *sides,
                           uint64_t *max_regions, uint32_t cap, uint32_t *levels)
{
    if (!levels || n == 0 || n > ASK_MAX_N || g == 0 || g > n || r < 2 || r > 64 || B == 0)
        return ASK_EINVAL;
    LevelPlan plan;
    if (!make_plan(n, g, r, B, &plan))
        return ASK_EINVAL;
    *levels = plan.levels;
    for (uint32_t i = 0; i < plan.levels && i < cap; ++i) {
        if (sides)
            sides[i] = plan.side[i];
        if (max_regions)
            max_regions[i] = plan.max_regions[i];
    }
    return ASK_OK;
}

ask_status ask_reserve(ask_ctx *ctx, ask_method method, uint32_t n, const ask_params *params)
{
    if (!ctx)
        return ASK_EINVAL;
    const ask_window w = {-2.0f, 1.0f, -1.5f, 1.5f};
    ask_params eff;
    ask_status st = check_args(ctx, method, &w, n, 1, params, &eff);
    if (st != ASK_OK)
        return st;
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    if (method != ASK_METHOD_ASK)
        return ensure_counters(ctx);
    LevelPlan plan;
    if (!make_plan(n, eff.g, eff.r, eff.B, &plan))
        return set_err(ctx, ASK_EINVAL, "no valid subdivision plan");
    return reserve_ask(ctx, plan);
}

ask_status ask_render(ask_ctx *ctx, ask_method method, const ask_window *window, uint32_t n,
                      uint32_t max_dwell, const ask_params *params, uint32_t *d_dwell, void *stream,
                      ask_stats *stats)
{
    ask_params eff;
    ask_status st = check_args(ctx, method, window, n, max_dwell, params, &eff);
    if (st != ASK_OK)
        return st;
    if (!d_dwell || ((uintptr_t)d_dwell & 15u))
        return set_err(ctx, ASK_EINVAL, "d_dwell must be a non-NULL 16-byte aligned device pointer");
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    return render_impl(ctx, method, window, n, max_dwell, eff, d_dwell, (cudaStream_t)stream, stats);
}

ask_status ask_render_host(ask_ctx *ctx, ask_method method, const ask_window *window, uint32_t n,
                           uint32_t max_dwell, const ask_params *params, uint32_t *h_dwell,
                           void *stream, ask_stats *stats)
{
    ask_params eff;
    ask_status st = check_args(ctx, method, window, n, max_dwell, params, &eff);
    if (st != ASK_OK)
        return st;
    if (!h_dwell)
        return set_err(ctx, ASK_EINVAL, "h_dwell must be non-NULL");
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    const size_t elems = (size_t)n * n;
    cudaStream_t s = (cudaStream_t)stream;
    if (elems > ctx->dmap_elems) {
        if (ctx->dmap) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->dmap);
        }
        ctx->dmap = nullptr;
        ctx->dmap_elems = 0;
        cudaError_t e = cudaMalloc(&ctx->dmap, elems * sizeof(uint32_t));
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "cudaMalloc(device map)");
        ctx->dmap_elems = elems;
    }
    // ASK without stats: the frame is rendered in bands of initial-region
    // rows (independent subtrees, contiguous map rows); each band's rows go
    // to the host on a copy stream while the next band renders.
    LevelPlan plan;
    uint32_t bands = 1;
    if (method == ASK_METHOD_ASK && !stats && !(eff.flags & ASK_FLAG_STAGED_COPY) &&
        make_plan(n, eff.g, eff.r, eff.B, &plan)) {
        const uint64_t want = (elems * sizeof(uint32_t) + kBandBytes / 2) / kBandBytes;
        bands = (uint32_t)std::min<uint64_t>(std::min<uint64_t>(want, plan.axis0), ask_ctx::kMaxBands);
        if (bands < 1)
            bands = 1;
    }
    if (bands > 1) {
        if ((st = ensure_bands(ctx)) != ASK_OK)
            return st;
        const uint32_t per = (plan.axis0 + bands - 1) / bands;  // initial-region rows per band
        bands = (plan.axis0 + per - 1) / per;
        auto copy_band = [&](uint32_t b) -> ask_status {
            const size_t y0 = (size_t)b * per * plan.side[0];
            const size_t y1 = std::min<size_t>(n, (size_t)(b + 1) * per * plan.side[0]);
            cudaError_t e = cudaStreamWaitEvent(ctx->cpy, ctx->band_ev[b], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_dwell + y0 * n, ctx->dmap + y0 * n, (y1 - y0) * n * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, ctx->cpy);
            return e == cudaSuccess ? ASK_OK : cuda_err(ctx, e, "copying a band of the map to the host");
        };
        // A copy into pinned memory is asynchronous, so band b - 1's copy is
        // queued right after band b's render; a copy into pageable memory
        // blocks the host, so every render is queued before the first copy.
        cudaPointerAttributes pa;
        const bool pinned = cudaPointerGetAttributes(&pa, h_dwell) == cudaSuccess && pa.type == cudaMemoryTypeHost;
        cudaGetLastError();
        for (uint32_t b = 0; b < bands; ++b) {
            st = render_impl(ctx, method, window, n, max_dwell, eff, ctx->dmap, s, nullptr, b * per, per);
            if (st != ASK_OK)
                return st;
            cudaError_t e = cudaEventRecord(ctx->band_ev[b], s);
            if (e != cudaSuccess)
                return cuda_err(ctx, e, "cudaEventRecord");
            if (pinned && b > 0 && (st = copy_band(b - 1)) != ASK_OK)
                return st;
        }
        for (uint32_t b = pinned ? bands - 1 : 0; b < bands; ++b)
            if ((st = copy_band(b)) != ASK_OK)
                return st;
        cudaError_t e = cudaStreamSynchronize(ctx->cpy);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "copying the map to the host");
        return read_counters(ctx, s);  // report latched device errors
    }
    st = render_impl(ctx, method, window, n, max_dwell, eff, ctx->dmap, s, stats);
    if (st != ASK_OK)
        return st;
    cudaError_t e = cudaMemcpyAsync(h_dwell, ctx->dmap, elems * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "copying the map to the host");
    if (!stats)
        return read_counters(ctx, s);  // report latched device errors
    return ASK_OK;
}

ask_status ask_timing_read(ask_ctx *ctx, void *stream, ask_timing *out)
{
    if (!ctx || !out)
        return ASK_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "cudaStreamSynchronize");
    out->dropped = ctx->ring_dropped;
    for (uint64_t k = ctx->ring_tail; k < ctx->ring_head; ++k) {
        const ask_ctx::TimingSlot &sl = ctx->ring[k % ask_ctx::kRing];
        const uint32_t L = sl.levels;
        const int last = (sl.method == ASK_METHOD_ASK) ? (int)L + 4 : 1;
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, sl.ev[0], sl.ev[last])) != cudaSuccess)
            return cuda_err(ctx, e, "cudaEventElapsedTime");
        out->ms_total += ms;
        if (sl.method == ASK_METHOD_ASK) {
            cudaEventElapsedTime(&ms, sl.ev[0], sl.ev[1]);
            out->ms_init += ms;
            for (uint32_t i = 0; i < L; ++i) {
                cudaEventElapsedTime(&ms, sl.ev[i + 1], sl.ev[i + 2]);
                out->ms_per_level[i] += ms;
            }
            cudaEventElapsedTime(&ms, sl.ev[L + 1], sl.ev[L + 2]);
            out->ms_fill += ms;
            cudaEventElapsedTime(&ms, sl.ev[L + 2], sl.ev[L + 3]);
            out->ms_leaf += ms;
        }
        out->levels = L;
        out->method = sl.method;
        ++out->renders;
    }
    ctx->ring_tail = ctx->ring_head;
    ctx->ring_dropped = 0;
    return ASK_OK;
}

ask_status ask_render_batch(ask_ctx *ctx, const ask_frame *frames, uint32_t nframes, uint32_t flags,
                            void *stream, ask_stats *stats)
{
    if (!ctx)
        return ASK_EINVAL;
    const bool persistent = (flags & ASK_FLAG_PERSISTENT) != 0;
    if ((flags & ASK_FLAG_WAIT_TEST) && !persistent)
        return set_err(ctx, ASK_EINVAL, "ASK_FLAG_WAIT_TEST needs ASK_FLAG_PERSISTENT");
    BatchPlan bp;
    ask_status st = plan_batch(ctx, frames, nframes, flags,
                               persistent ? (ASK_FLAG_COUNT | ASK_FLAG_PERSISTENT | ASK_FLAG_WAIT_TEST)
                                          : (ASK_FLAG_COUNT | ASK_FLAG_EXACT_BORDERS),
                               bp);
    if (st != ASK_OK)
        return st;
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    if ((st = ensure_counters(ctx)) != ASK_OK)
        return st;
    if (persistent) {
        ctx->queue.ctr = ctx->ctr;
        st = reserve_queue(ctx, ctx->queue, bp, false);
    } else {
        ctx->batch.ctr = ctx->ctr;
        st = reserve_batch(ctx, ctx->batch, bp, false);
    }
    if (st != ASK_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        if ((st = ensure_events(ctx)) != ASK_OK)
            return st;
    }
    if ((st = upload_frames(ctx, persistent ? ctx->queue.frames : ctx->batch.frames, bp, s)) != ASK_OK)
        return st;
    if (stats)
        cudaEventRecord(ctx->ev[0], s);
    uint32_t launches = 0;
    if (persistent)
        st = enqueue_queue(ctx, ctx->queue, bp, flags, s, &launches);
    else
        st = enqueue_batch(ctx, ctx->batch, bp, flags, s, &launches);
    if (st != ASK_OK)
        return st;
    if (stats) {
        cudaEventRecord(ctx->ev[1], s);
        if ((st = read_counters(ctx, s)) != ASK_OK)
            return st;
        cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[1]);
        const DevCounters &c = *ctx->h_ctr;
        stats->levels = bp.L;
        for (uint32_t i = 0; i < bp.L; ++i) {
            stats->regions_per_level[i] = c.count[i] + c.back[i];
            stats->fills_per_level[i] = c.fills[i];
            stats->subdivisions_per_level[i] = c.subdivs[i];
            stats->iterations_per_level[i] = c.level_iters[i];
        }
        stats->leaves = c.leaf_count + c.leaf_light;
        stats->fill_pixels = c.fill_pixels;
        stats->deferred_fill_pixels = c.deferred_fill_pixels;
        stats->leaf_pixels = c.leaf_pixels;
        stats->border_pixels = c.border_pixels;
        stats->iterations = c.iterations;
        stats->leaf_iterations = c.leaf_iters;
        stats->kernel_launches = launches;
    }
    return ASK_OK;
}

ask_status ask_graph_create_batch(ask_ctx *ctx, const ask_frame *frames, uint32_t nframes,
                                  uint32_t flags, void *stream, ask_graph **out)
{
    if (!ctx || !out)
        return ASK_EINVAL;
    *out = nullptr;
    const bool persistent = (flags & ASK_FLAG_PERSISTENT) != 0;
    BatchPlan bp;
    ask_status st = plan_batch(ctx, frames, nframes, flags,
                               persistent ? ASK_FLAG_PERSISTENT : ASK_FLAG_EXACT_BORDERS, bp);
    if (st != ASK_OK)
        return st;
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    ask_graph *g = new (std::nothrow) ask_graph();
    if (!g)
        return ASK_ENOMEM;
    g->device = ctx->dev.device;
    g->persistent = persistent;
    auto release = [](ask_graph *gr) {
        if (gr->exec)
            cudaGraphExecDestroy(gr->exec);
        if (gr->graph)
            cudaGraphDestroy(gr->graph);
        free_batch(gr->buf, true);
        free_queue(gr->qbuf, true);
        delete gr;
    };
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (persistent)
        st = reserve_queue(ctx, g->qbuf, bp, true);
    else
        st = reserve_batch(ctx, g->buf, bp, true);
    if (st == ASK_OK)
        st = upload_frames(ctx, persistent ? g->qbuf.frames : g->buf.frames, bp, s);
    if (st != ASK_OK) {
        release(g);
        return st;
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        release(g);
        return cuda_err(ctx, e, "cudaStreamSynchronize");
    }
    // capture on a private stream so the caller's stream is never in capture mode
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
        release(g);
        return cuda_err(ctx, e, "cudaStreamCreate");
    }
    st = ASK_OK;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        st = cuda_err(ctx, e, "cudaStreamBeginCapture");
    } else {
        const ask_status est = persistent ? enqueue_queue(ctx, g->qbuf, bp, flags, cs, nullptr)
                                          : enqueue_batch(ctx, g->buf, bp, flags, cs, nullptr);
        e = cudaStreamEndCapture(cs, &g->graph);
        if (est != ASK_OK)
            st = est;
        else if (e != cudaSuccess)
            st = cuda_err(ctx, e, "cudaStreamEndCapture");
        else if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
            st = cuda_err(ctx, e, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cs);
    if (st != ASK_OK) {
        release(g);
        return st;
    }
    *out = g;
    return ASK_OK;
}

ask_status ask_graph_launch(ask_graph *g, void *stream)
{
    if (!g || !g->exec)
        return ASK_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess)
        return ASK_ECUDA;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? ASK_OK : ASK_ECUDA;
}

void ask_graph_destroy(ask_graph *g)
{
    if (!g)
        return;
    cudaSetDevice(g->device);
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->graph)
        cudaGraphDestroy(g->graph);
    free_batch(g->buf, true);
    free_queue(g->qbuf, true);
    delete g;
}

ask_status ask_check(ask_ctx *ctx, void *stream)
{
    if (!ctx)
        return ASK_EINVAL;
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    ask_status st = ensure_counters(ctx);
    if (st != ASK_OK)
        return st;
    return read_counters(ctx, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Double precision (deep zooms): the exhaustive method and ASK with the
// arithmetic of ask_fp64.cu, on the context's region tables and counters.
// ---------------------------------------------------------------------------
namespace {

bool window64_ok(const ask_window64 *w)
{
    return w && std::isfinite(w->re_min) && std::isfinite(w->re_max) && std::isfinite(w->im_min) &&
           std::isfinite(w->im_max) && w->re_max > w->re_min && w->im_max > w->im_min;
}

PixelMap64 pixel_map64(const ask_window64 *w, uint32_t n)
{
    PixelMap64 pm;
    pm.re_min = w->re_min;
    pm.im_min = w->im_min;
    // double subtraction and division, each rounded once
    const double wr = w->re_max - w->re_min;
    const double wi = w->im_max - w->im_min;
    pm.dx = wr / (double)n;
    pm.dy = wi / (double)n;
    return pm;
}

ask_status render64_impl(ask_ctx *ctx, ask_method method, const ask_window64 *window, uint32_t n,
                         uint32_t max_dwell, const ask_params &p, uint32_t *d_dwell, cudaStream_t s,
                         ask_stats *stats)
{
    const bool count = (p.flags & ASK_FLAG_COUNT) != 0;
    const bool ff = (p.flags & ASK_FLAG_FLOAT_FLOAT) != 0;
    const PixelMap64 pm = pixel_map64(window, n);
    ask_status st;
    cudaError_t e;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        if ((st = ensure_events(ctx)) != ASK_OK)
            return st;
    }
    if ((st = ensure_counters(ctx)) != ASK_OK)
        return st;
    uint32_t launches = 0;
    if (stats)
        cudaEventRecord(ctx->ev[0], s);

    if (method == ASK_METHOD_EXHAUSTIVE) {
        if (count) {
            if ((e = launch_init(nullptr, nullptr, ctx->ctr, n, 1, 0, 0, 0, s)) != cudaSuccess)
                return cuda_err(ctx, e, "init kernel");
            ++launches;
        }
        if ((e = launch_exhaustive64(d_dwell, n, pm, max_dwell, p.block_x, p.block_y, count, ff,
                                     ctx->ctr, s)) != cudaSuccess)
            return cuda_err(ctx, e, "double-precision exhaustive kernel");
        ++launches;
        if (stats) {
            cudaEventRecord(ctx->ev[1], s);
            if ((st = read_counters(ctx, s)) != ASK_OK)
                return st;
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[1]);
            stats->iterations = count ? ctx->h_ctr->iterations : 0;
            stats->kernel_launches = launches;
        }
        return ASK_OK;
    }

    LevelPlan plan;
    if (!make_plan(n, p.g, p.r, p.B, &plan))
        return set_err(ctx, ASK_EINVAL, "no valid subdivision plan for n=%u g=%u r=%u B=%u", n, p.g, p.r, p.B);
    for (uint32_t i = 0; i < plan.levels; ++i)
        plan.chunks[i] = 1u;  // one warp per region: no chunked-query state
    if ((st = reserve_ask(ctx, plan)) != ASK_OK)
        return st;
    const uint32_t L = plan.levels;
    if ((e = launch_init(ctx->olt[0], nullptr, ctx->ctr, n, plan.side[0], plan.axis0, 0, plan.axis0, s)) !=
        cudaSuccess)
        return cuda_err(ctx, e, "init kernel");
    ++launches;
    if (stats)
        cudaEventRecord(ctx->ev[1], s);
    for (uint32_t i = 0; i < L; ++i) {
        Level64Args a;
        a.map = d_dwell;
        a.n = n;
        a.pm = pm;
        a.max_dwell = max_dwell;
        a.level = i;
        a.split = plan.split[i];
        a.child_side = ceil_div(plan.side[i], p.r);
        a.r = p.r;
        a.olt_in = ctx->olt[i & 1];
        a.olt_out = ctx->olt[(i + 1) & 1];
        a.olt_cap = (uint32_t)ctx->olt_cap;
        a.leaves = ctx->leaves;
        a.leaf_cap = (uint32_t)ctx->leaf_cap;
        a.ctr = ctx->ctr;
        if ((e = launch_level64(a, count, ff, ctx->dev.sms, s)) != cudaSuccess)
            return cuda_err(ctx, e, "double-precision level kernel");
        ++launches;
        if (stats)
            cudaEventRecord(ctx->ev[2 + i], s);
    }
    Leaf64Args la;
    la.map = d_dwell;
    la.n = n;
    la.pm = pm;
    la.max_dwell = max_dwell;
    la.leaves = ctx->leaves;
    la.leaf_cap = (uint32_t)ctx->leaf_cap;
    la.ctr = ctx->ctr;
    if ((e = launch_leaf64(la, count, ff, ctx->dev.sms, s)) != cudaSuccess)
        return cuda_err(ctx, e, "double-precision leaf kernel");
    ++launches;
    if (stats) {
        cudaEventRecord(ctx->ev[2 + L], s);
        if ((st = read_counters(ctx, s)) != ASK_OK)
            return st;
        cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[2 + L]);
        for (uint32_t i = 0; i < L; ++i)
            cudaEventElapsedTime(&stats->ms_per_level[i], ctx->ev[1 + i], ctx->ev[2 + i]);
        cudaEventElapsedTime(&stats->ms_leaf, ctx->ev[1 + L], ctx->ev[2 + L]);
        const DevCounters &c = *ctx->h_ctr;
        stats->levels = L;
        for (uint32_t i = 0; i < L; ++i) {
            stats->regions_per_level[i] = c.count[i] + c.back[i];
            stats->fills_per_level[i] = c.fills[i];
            stats->subdivisions_per_level[i] = c.subdivs[i];
            stats->iterations_per_level[i] = c.level_iters[i];
        }
        stats->leaves = c.leaf_count + c.leaf_light;
        stats->fill_pixels = c.fill_pixels;
        stats->leaf_pixels = c.leaf_pixels;
        stats->iterations = c.iterations;
        stats->leaf_iterations = c.leaf_iters;
        stats->kernel_launches = launches;
    }
    return ASK_OK;
}

}  // namespace

extern "C" ask_status ask_render64(ask_ctx *ctx, ask_method method, const ask_window64 *window,
                                   uint32_t n, uint32_t max_dwell, const ask_params *params,
                                   uint32_t *d_dwell, void *stream, ask_stats *stats)
{
    if (!ctx)
        return ASK_EINVAL;
    if (!window64_ok(window))
        return set_err(ctx, ASK_EINVAL, "window must be finite with min < max");
    if (method == ASK_METHOD_CDP2)
        return set_err(ctx, ASK_EINVAL, "ask_render64: CDP2 has no double-precision variant");
    // the float window only stands in for the argument checks of the rest
    const ask_window unit = {0.0f, 1.0f, 0.0f, 1.0f};
    ask_params eff, plain;
    if (params) {
        plain = *params;
        plain.flags &= ~ASK_FLAG_FLOAT_FLOAT;  // a flag of this entry point only
    }
    ask_status st = check_args(ctx, method, &unit, n, max_dwell, params ? &plain : nullptr, &eff);
    if (st != ASK_OK)
        return st;
    if (params)
        eff.flags = params->flags;
    if (eff.flags & ~(ASK_FLAG_COUNT | ASK_FLAG_FLOAT_FLOAT))
        return set_err(ctx, ASK_EINVAL,
                       "ask_render64 accepts ASK_FLAG_COUNT and ASK_FLAG_FLOAT_FLOAT only (flags 0x%x)",
                       eff.flags);
    if (!d_dwell || ((uintptr_t)d_dwell & 15u))
        return set_err(ctx, ASK_EINVAL, "d_dwell must be a non-NULL 16-byte aligned device pointer");
    if (cudaSetDevice(ctx->dev.device) != cudaSuccess)
        return set_err(ctx, ASK_ECUDA, "cudaSetDevice");
    return render64_impl(ctx, method, window, n, max_dwell, eff, d_dwell, (cudaStream_t)stream, stats);
}
