// ask_noalloc.cu -- ask_render_noalloc: an ASK render that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs inside a frame loop or
// a host callback where an allocation (and the device synchronisation that
// cudaMalloc/cudaFree may imply) is not allowed, plug-ins hosted by an
// application that owns all device memory through its own pool, or services
// held to a fixed memory budget.  For them this entry point takes its
// scratch (two region tables, the leaf list and the counters) from arrays
// with static storage on the device, sized once for all calls:
// kNoAllocRegions entries per table, about 24 MiB per device, held by every
// GPU that loads the library until the process exits.  The caller still
// passes the window and owns the output buffer.
//
// The arrays are shared by every call: two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on them.  Each
// call clears what must start at zero (counters, error word) on its stream
// before its first kernel, so the previous call's leftovers do no harm.
#include <cuda_runtime.h>

#include <mutex>

#include "ask_internal.h"

namespace {

// Entries per region table and in the leaf list.
constexpr uint32_t kNoAllocRegions = 1u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint2 g_olt_a[kNoAllocRegions];
static __device__ __align__(256) uint2 g_olt_b[kNoAllocRegions];
static __device__ __align__(256) uint2 g_leaves[kNoAllocRegions];
static __device__ __align__(256) ask::DevCounters g_counters;

// Device addresses of the arrays above, looked up once per device.  In host
// code the array names are host-side stand-ins, not device addresses, so
// kernels only ever receive these looked-up pointers.
struct DeviceScratch {
    uint2 *olt[2];
    uint2 *leaves;
    ask::DevCounters *ctr;
    int sms;
    bool ready;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

ask_status setup_device(int dev, const DeviceScratch **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return ASK_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DeviceScratch &s = g_scratch[dev];
    if (!s.ready) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ASK_ECUDA;
        if (!(major == 10 && minor == 3))
            return ASK_EUNSUPPORTED;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_olt_a) != cudaSuccess || !p)
            return ASK_ECUDA;
        s.olt[0] = static_cast<uint2 *>(p);
        if (cudaGetSymbolAddress(&p, g_olt_b) != cudaSuccess || !p)
            return ASK_ECUDA;
        s.olt[1] = static_cast<uint2 *>(p);
        if (cudaGetSymbolAddress(&p, g_leaves) != cudaSuccess || !p)
            return ASK_ECUDA;
        s.leaves = static_cast<uint2 *>(p);
        if (cudaGetSymbolAddress(&p, g_counters) != cudaSuccess || !p)
            return ASK_ECUDA;
        s.ctr = static_cast<ask::DevCounters *>(p);
        s.sms = sms;
        s.ready = true;
    }
    *out = &s;
    return ASK_OK;
}

uint32_t ceil_div(uint32_t a, uint32_t b) { return a / b + (a % b != 0u); }

// The level plan of the subdivision, computed without touching the heap:
// per level the region side, whether non-uniform regions split, and the
// bound A_i^2 on its region count (A_i = intervals per axis).
struct NoAllocPlan {
    uint32_t levels, axis0;
    uint32_t side[ASK_MAX_LEVELS], split[ASK_MAX_LEVELS];
    uint64_t max_regions[ASK_MAX_LEVELS];
};

bool plan_without_heap(uint32_t n, uint32_t g, uint32_t r, uint32_t B, NoAllocPlan *p)
{
    constexpr int kLens = 2 * ASK_MAX_LEVELS + 2;
    uint32_t len[kLens];
    uint64_t cnt[kLens];
    int nl = 0;
    uint32_t s = ceil_div(n, g);
    if (n / s) {
        len[nl] = s;
        cnt[nl++] = n / s;
    }
    if (n % s) {
        len[nl] = n % s;
        cnt[nl++] = 1;
    }
    p->axis0 = n / s + (n % s ? 1u : 0u);
    for (uint32_t i = 0;; ++i) {
        if (i >= ASK_MAX_LEVELS)
            return false;
        uint64_t axis = 0;
        for (int k = 0; k < nl; ++k)
            axis += cnt[k];
        p->side[i] = s;
        p->max_regions[i] = axis * axis;
        const uint32_t sc = ceil_div(s, r);
        p->split[i] = (s > 1u && sc >= B) ? 1u : 0u;
        p->levels = i + 1;
        if (!p->split[i])
            return true;
        uint32_t nlen[kLens];
        uint64_t ncnt[kLens];
        int nn = 0;
        auto add = [&](uint32_t l, uint64_t c) {
            for (int k = 0; k < nn; ++k)
                if (nlen[k] == l) {
                    ncnt[k] += c;
                    return true;
                }
            if (nn == kLens)
                return false;
            nlen[nn] = l;
            ncnt[nn++] = c;
            return true;
        };
        for (int k = 0; k < nl; ++k) {
            if (len[k] / sc && !add(sc, (uint64_t)(len[k] / sc) * cnt[k]))
                return false;
            if (len[k] % sc && !add(len[k] % sc, cnt[k]))
                return false;
        }
        for (int k = 0; k < nn; ++k) {
            len[k] = nlen[k];
            cnt[k] = ncnt[k];
        }
        nl = nn;
        s = sc;
    }
}

bool finite_window(const ask_window *w)
{
    return w && w->re_min == w->re_min && w->re_max == w->re_max && w->im_min == w->im_min &&
           w->im_max == w->im_max && w->re_min > -3.4e38f && w->re_max < 3.4e38f &&
           w->im_min > -3.4e38f && w->im_max < 3.4e38f && w->re_max > w->re_min &&
           w->im_max > w->im_min;
}

}  // namespace

extern "C" ask_status ask_render_noalloc(const ask_window *window, uint32_t n, uint32_t max_dwell,
                                         const ask_params *params, uint32_t *d_dwell, void *stream)
{
    using namespace ask;
    if (!finite_window(window) || n == 0 || n > ASK_MAX_N || max_dwell == 0 ||
        max_dwell == 0xffffffffu || !params || !d_dwell || ((uintptr_t)d_dwell & 15u))
        return ASK_EINVAL;
    const ask_params &p = *params;
    const uint64_t threads_per_block = (uint64_t)p.block_x * p.block_y;
    if (p.g == 0 || p.g > n || p.r < 2 || p.r > 64 || p.B == 0 || p.flags != 0 ||
        p.block_x == 0 || p.block_y == 0 || threads_per_block < 32 || threads_per_block > 1024 ||
        threads_per_block % 32 != 0)
        return ASK_EINVAL;
    NoAllocPlan plan;
    if (!plan_without_heap(n, p.g, p.r, p.B, &plan))
        return ASK_EINVAL;
    for (uint32_t i = 0; i < plan.levels; ++i)
        if (plan.max_regions[i] > kNoAllocRegions)
            return ASK_ECAPACITY;  // the fixed scratch is too small for this request

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return ASK_ECUDA;
    const DeviceScratch *sc = nullptr;
    ask_status st = setup_device(dev, &sc);
    if (st != ASK_OK)
        return st;

    cudaStream_t s = (cudaStream_t)stream;
    const float wr = window->re_max - window->re_min;
    const float wi = window->im_max - window->im_min;
    PixelMap pm;
    pm.re_min = window->re_min;
    pm.im_min = window->im_min;
    pm.dx = wr / (float)n;
    pm.dy = wi / (float)n;

    // the shared counters keep the previous call's values: clear the latched
    // error word here; the init kernel zeroes the rest and writes OLT 0
    if (cudaMemsetAsync(&sc->ctr->error, 0, sizeof(uint32_t), s) != cudaSuccess)
        return ASK_ECUDA;
    if (launch_init(sc->olt[0], nullptr, sc->ctr, n, plan.side[0], plan.axis0, 0u, plan.axis0, s) != cudaSuccess)
        return ASK_ECUDA;
    const uint32_t L = plan.levels;
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
        a.olt_in = sc->olt[i & 1];
        a.olt_out = sc->olt[(i + 1) & 1];
        a.olt_cap = kNoAllocRegions;
        a.in_cap = kNoAllocRegions;  // the tables fill from both ends of the whole array
        a.out_cap = kNoAllocRegions;
        // one warp per region and fills in place: no per-region query state
        // or fill list, so the fixed scratch stays at three tables
        a.chunks = 1u;
        a.chunk_px = kChunkPx;
        a.next_chunks = 1u;
        a.rst_in = nullptr;
        a.rst_out = nullptr;
        a.leaves = sc->leaves;
        a.leaf_cap = kNoAllocRegions;
        a.fills = nullptr;
        a.fill_cap = 0u;
        a.exact_last = 0u;
        a.ctr = sc->ctr;
        if (launch_level(a, false, false, sc->sms, s) != cudaSuccess)
            return ASK_ECUDA;
    }
    LeafArgs la;
    la.map = d_dwell;
    la.n = n;
    la.pm = pm;
    la.max_dwell = max_dwell;
    la.side = plan.side[L - 1];
    la.leaves = sc->leaves;
    la.leaf_cap = kNoAllocRegions;
    la.skip_perimeter = 0u;
    la.fills = nullptr;
    la.fill_cap = 0u;
    la.frames = nullptr;
    la.ctr = sc->ctr;
    if (launch_leaf(la, p.block_x, p.block_y, false, false, false, sc->sms, s) != cudaSuccess)
        return ASK_ECUDA;
    return ASK_OK;
}
