// ask_device.cuh -- device helpers shared by the exhaustive, ASK and CDP2
// kernels: the per-pixel dwell, the pixel -> c mapping, region records,
// perimeter enumeration and vectorised fills.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_internal.h"

namespace ask {

// Updates per unchecked block in the dwell loops (see dwell()).
constexpr int kUnroll = 16;

// |c|^2 bound below which escape is absorbing in float arithmetic (see dwell()).
constexpr float kAbsorbR2 = 3.999f;

__device__ __forceinline__ float2 pixel_c(const PixelMap &pm, uint32_t px, uint32_t py)
{
    return make_float2(__fmaf_rn(__uint2float_rn(px), pm.dx, pm.re_min),
                       __fmaf_rn(__uint2float_rn(py), pm.dy, pm.im_min));
}

// One update z <- z^2 + c, each operation rounded once (the _rn intrinsics
// are never fused or reassociated by the compiler):
//   zr' = fma(zr, zr, fma(-zi, zi, cr)),  zi' = fma(zr + zr, zi, ci).
__device__ __forceinline__ void z_update(float &x, float &y, float cr, float ci)
{
    const float t = __fmaf_rn(-y, y, cr);
    const float nx = __fmaf_rn(x, x, t);
    const float ny = __fmaf_rn(__fadd_rn(x, x), y, ci);
    x = nx;
    y = ny;
}

// The escape test of the current state: |z|^2 = fma(zr, zr, zi*zi) < 4.
__device__ __forceinline__ bool z_bounded(float x, float y)
{
    return __fmaf_rn(x, x, __fmul_rn(y, y)) < 4.0f;
}

// Escape is absorbing when |c| < 2 - 2.4e-4, i.e. fma(cr, cr, ci*ci) < 3.999:
// if the rounded |z_j|^2 >= 4 then the exact |z_j|^2 > 4 - 4e-7, so the exact
// |z_j^2 + c| > 2 + 2.3e-4, and the rounding of one update (a few ulps of
// |z|^2) cannot take it back below 2; by induction |z| keeps growing until it
// overflows, and an inf or NaN state also fails the test "|z|^2 < 4".  So for
// such c, a state that passes the test proves that every earlier state passed.
__device__ __forceinline__ bool escape_absorbing(float cr, float ci)
{
    return __fmaf_rn(cr, cr, __fmul_rn(ci, ci)) < kAbsorbR2;
}

// Dwell of c (paper Sec. 6): the number of updates z <- z^2 + c, from z = 0,
// made while |z|^2 < 4, at most max_dwell.
//
// Where escape is absorbing, updates run in blocks of kUnroll with a single
// test on the block's last state: 3 FFMA + 1 FADD per update, the test
// amortised over the block.  A block whose last state fails the test is
// rolled back and replayed one tested update at a time, so the count is
// exactly the stepwise one.  Other points, and the tail below max_dwell, take
// the tested loop.
__device__ __forceinline__ uint32_t dwell(float cr, float ci, uint32_t max_dwell)
{
    float x = 0.0f, y = 0.0f;
    uint32_t d = 0;
    if (escape_absorbing(cr, ci)) {
        while (max_dwell - d >= (uint32_t)kUnroll) {
            const float sx = x, sy = y;
#pragma unroll
            for (int k = 0; k < kUnroll; ++k)
                z_update(x, y, cr, ci);
            if (!z_bounded(x, y)) {
                x = sx;
                y = sy;
                break;
            }
            d += (uint32_t)kUnroll;
        }
    }
    while (d < max_dwell && z_bounded(x, y)) {
        z_update(x, y, cr, ci);
        ++d;
    }
    return d;
}

// Resumable orbit of one point, for perimeter queries that stop early.
struct Orbit {
    float x, y, cr, ci;
    uint32_t d;     // updates made; every state before z_d passed the test
    bool fast;      // escape is absorbing for this c
};

__device__ __forceinline__ Orbit orbit_start(float2 c)
{
    Orbit o;
    o.x = 0.0f;
    o.y = 0.0f;
    o.cr = c.x;
    o.ci = c.y;
    o.d = 0;
    o.fast = escape_absorbing(c.x, c.y);
    return o;
}

// Outcome of one round of an orbit.
enum : uint32_t {
    ORBIT_RUN = 0,   // every state so far passed; more rounds to go
    ORBIT_DONE = 1,  // finished with o.d exact: escaped, or made `limit` updates
    ORBIT_PEND = 2,  // escaped within the round's unchecked block: the dwell is in
                     // (o.d, o.d + K], o keeps the block's starting state
};

// Updates per unchecked block of a perimeter-query round after the short
// first rounds of query_step, for a large region's chunks and for a small
// region's whole perimeter.  The short rounds take the orbits that escape
// early, so the long ones serve orbits that run long (at n = 16384 whole
// perimeters of 16 x 16 regions ran faster with 64 than with 32; chunks ran
// slower with 128).
constexpr uint32_t kQueryRoundLarge = 64;
constexpr uint32_t kQueryRound = 64;
// The CTA-wide query of the paper's SBR / MBR mappings: blocks of 32 from
// the first round.
constexpr uint32_t kQueryRoundCta = 32;
// Batches (zoomed frames, higher dwell caps, regions of many sizes): whole
// perimeters in blocks of kQueryRoundBatch, short first rounds where the
// flags say (a batch's chunk queries read their region's state every round,
// and a short round cannot hide that load).
constexpr uint32_t kQueryRoundBatch = 32;
constexpr bool kBatchShortWhole = false;
constexpr bool kBatchShortChunks = false;

// Advance an orbit by up to K updates (a power of two) without passing
// `limit`.  An orbit still running after a round has made more updates than
// any orbit that finished (or became pending) in it: its dwell is strictly
// larger.  A pending orbit needs orbit_resolve only if its exact dwell is
// wanted.
template <uint32_t K>
__device__ __forceinline__ uint32_t orbit_step(Orbit &o, uint32_t limit)
{
    if (o.d >= limit)
        return ORBIT_DONE;
    if (o.fast && limit - o.d >= K) {
        float x = o.x, y = o.y;
#pragma unroll
        for (uint32_t k = 0; k < K; ++k)
            z_update(x, y, o.cr, o.ci);
        if (!z_bounded(x, y))
            return ORBIT_PEND;
        o.x = x;
        o.y = y;
        o.d += K;
        return o.d >= limit ? ORBIT_DONE : ORBIT_RUN;
    }
    for (uint32_t k = 0; k < K; ++k) {
        if (o.d >= limit || !z_bounded(o.x, o.y))
            return ORBIT_DONE;
        z_update(o.x, o.y, o.cr, o.ci);
        ++o.d;
    }
    return o.d >= limit ? ORBIT_DONE : ORBIT_RUN;
}

// Exact dwell of an orbit left pending by orbit_step<K>: its starting state
// z_d passed the test and z_{d + K} failed; halving the gap finds the first
// failing state (K - 1 updates, log2(K) tests, no branches that differ by
// lane).
template <uint32_t K>
__device__ __forceinline__ void orbit_resolve(Orbit &o)
{
    float x = o.x, y = o.y;
    uint32_t d = o.d;
#pragma unroll
    for (uint32_t h = K / 2u; h >= 1u; h >>= 1) {
        float tx = x, ty = y;
#pragma unroll
        for (uint32_t k = 0; k < h; ++k)
            z_update(tx, ty, o.cr, o.ci);
        if (z_bounded(tx, ty)) {
            x = tx;
            y = ty;
            d += h;
        }
    }
    o.x = x;
    o.y = y;
    o.d = d + 1u;
}

// Rounds of a perimeter query: unchecked blocks of 8, 8 and 16 updates, then
// K.  Most perimeter orbits outside the set escape within a few updates; a
// short first block and the short binary search after it cost them about 15
// updates where a K-update block and its search cost 2K - 1, while an orbit
// that runs long pays three short rounds.  Every lane of a group runs the
// same block in a round, so a running orbit still outlives every orbit that
// finished in that round.
template <uint32_t K>
__device__ __forceinline__ void query_step(Orbit &o, uint32_t &stt, uint32_t limit, uint32_t rnd)
{
    if (stt != ORBIT_RUN)
        return;
    if (rnd < 2u)
        stt = orbit_step<8>(o, limit);
    else if (rnd == 2u)
        stt = orbit_step<16>(o, limit);
    else
        stt = orbit_step<K>(o, limit);
}

// Exact dwell of an orbit left pending by query_step<K> in round `rnd`.
template <uint32_t K>
__device__ __forceinline__ void query_resolve(Orbit &o, uint32_t rnd)
{
    if (rnd < 2u)
        orbit_resolve<8>(o);
    else if (rnd == 2u)
        orbit_resolve<16>(o);
    else
        orbit_resolve<K>(o);
}

// Region record of the offset lookup tables (Sec. 5.2): origin and clipped
// extent, 16 bits each (n <= 65536 so x0, y0, w-1, h-1 < 65536).
struct Region {
    uint32_t x0, y0, w, h;
};

__device__ __forceinline__ uint2 pack_region(uint32_t x0, uint32_t y0, uint32_t w, uint32_t h)
{
    return make_uint2(x0 | (y0 << 16), (w - 1u) | ((h - 1u) << 16));
}

__device__ __forceinline__ Region unpack_region(uint2 e)
{
    Region g;
    g.x0 = e.x & 0xffffu;
    g.y0 = e.x >> 16;
    g.w = (e.y & 0xffffu) + 1u;
    g.h = (e.y >> 16) + 1u;
    return g;
}

// Number of perimeter pixels of a w x h region (outermost rows and columns).
__device__ __forceinline__ uint32_t perimeter_size(uint32_t w, uint32_t h)
{
    return (w <= 2u || h <= 2u) ? w * h : 2u * w + 2u * (h - 2u);
}

// k-th perimeter pixel: top row, bottom row, left column, right column
// (columns without the corners), so neighbouring k are neighbouring pixels.
__device__ __forceinline__ void perimeter_pixel(const Region &g, uint32_t k, uint32_t &px,
                                                uint32_t &py)
{
    if (g.w <= 2u || g.h <= 2u) {
        px = g.x0 + k % g.w;
        py = g.y0 + k / g.w;
        return;
    }
    if (k < g.w) {
        px = g.x0 + k;
        py = g.y0;
    } else if (k < 2u * g.w) {
        px = g.x0 + (k - g.w);
        py = g.y0 + g.h - 1u;
    } else {
        const uint32_t j = k - 2u * g.w, hh = g.h - 2u;
        px = (j < hh) ? g.x0 : g.x0 + g.w - 1u;
        py = g.y0 + 1u + ((j < hh) ? j : j - hh);
    }
}

__device__ __forceinline__ bool on_perimeter(const Region &g, uint32_t px, uint32_t py)
{
    return px == g.x0 || py == g.y0 || px == g.x0 + g.w - 1u || py == g.y0 + g.h - 1u;
}

// Cooperative fill of the rectangle g with value v by `nthr` threads
// (thread index `t`).  Each row is cut at 16-byte boundaries of the map; full
// 16-byte chunks take one 128-bit store, the partial chunks at the row ends
// take scalar stores.  The map base must be 16-byte aligned.
__device__ __forceinline__ void fill_rect(uint32_t *__restrict__ map, uint32_t n, const Region &g,
                                          uint32_t v, uint32_t t, uint32_t nthr)
{
    const uint32_t cpr = (g.w + 3u) / 4u + 1u;  // chunks per row, an upper bound for any alignment
    const uint4 v4 = make_uint4(v, v, v, v);
    uint32_t row = t / cpr, c = t - row * cpr;   // then advanced without dividing
    while (row < g.h) {
        const size_t start = (size_t)(g.y0 + row) * n + g.x0;
        const size_t end = start + g.w;
        const size_t e0 = ((start >> 2) + c) << 2;
        if (e0 < end) {
            if (e0 >= start && e0 + 4u <= end) {
                *reinterpret_cast<uint4 *>(map + e0) = v4;
            } else {
#pragma unroll
                for (uint32_t k = 0; k < 4u; ++k)
                    if (e0 + k >= start && e0 + k < end)
                        map[e0 + k] = v;
            }
        }
        c += nthr;
        while (c >= cpr) {
            c -= cpr;
            ++row;
        }
    }
}

// Warp fill of a band of the deferred-fill list.  Rows of at least 128
// pixels go one at a time, the lanes striding over the row's whole 16-byte
// chunks (one 128-bit store, a pointer step and a compare each), with the at
// most 3 + 3 pixels outside them stored singly; narrower bands use fill_rect.
__device__ __forceinline__ void fill_band_warp(uint32_t *__restrict__ map, uint32_t n,
                                               const Region &g, uint32_t v, uint32_t lane)
{
    if (g.w < 128u) {
        fill_rect(map, n, g, v, lane, 32u);
        return;
    }
    const uint4 v4 = make_uint4(v, v, v, v);
    for (uint32_t row = 0; row < g.h; ++row) {
        const size_t start = (size_t)(g.y0 + row) * n + g.x0;
        const size_t end = start + g.w;
        const size_t a4 = (start + 3u) >> 2, b4 = end >> 2;  // whole chunks [a4, b4)
        uint4 *q = reinterpret_cast<uint4 *>(map) + a4 + lane;
        uint4 *const qe = reinterpret_cast<uint4 *>(map) + b4;
        for (; q < qe; q += 32)
            *q = v4;
        if (lane < 3u && start + lane < (a4 << 2))
            map[start + lane] = v;
        if (lane >= 3u && lane < 6u && (b4 << 2) + (lane - 3u) < end)
            map[(b4 << 2) + (lane - 3u)] = v;
    }
}

// ---------------------------------------------------------------------------
// Perimeter uniformity queries for regions that split when not uniform.
//
// Such a region needs only the answer "all perimeter dwells equal, and to
// what", not the dwells themselves (its children evaluate their own
// perimeters).  The orbits of a group of 32 perimeter pixels advance in
// rounds; running orbits stay in lockstep, so as soon as one orbit has
// finished while another still runs, their dwells differ and the query
// stops.  Once one group has finished with a common dwell w, later groups
// stop at w + 1 updates: more updates than w already means a different dwell.
// ---------------------------------------------------------------------------
constexpr unsigned kLaneMask = 0xffffffffu;

// One warp queries the whole perimeter of g.  Returns true and the common
// dwell in *w_out if the perimeter is uniform; `it` gains the updates made.
template <uint32_t K, bool SHORT>
__device__ __forceinline__ bool warp_perimeter_uniform(const PixelMap &pm, uint32_t max_dwell,
                                                       const Region &g, uint32_t lane,
                                                       uint32_t *w_out, unsigned long long &it)
{
    const uint32_t P = perimeter_size(g.w, g.h);
    bool have = false;
    uint32_t w = 0;
    for (uint32_t base = 0; base < P; base += 32u) {
        const uint32_t k = base + lane;
        const bool active = k < P;
        const unsigned amask = __ballot_sync(kLaneMask, active);
        uint32_t px = g.x0, py = g.y0;
        if (active)
            perimeter_pixel(g, k, px, py);
        Orbit o = orbit_start(pixel_c(pm, px, py));
        uint32_t stt = active ? ORBIT_RUN : ORBIT_DONE;
        const uint32_t limit = have ? min(max_dwell, w + 1u) : max_dwell;
        bool differ = false;
        uint32_t rnd = 0;
        for (;; ++rnd) {
            if (SHORT)
                query_step<K>(o, stt, limit, rnd);
            else if (stt == ORBIT_RUN)
                stt = orbit_step<K>(o, limit);
            const unsigned dm = __ballot_sync(kLaneMask, stt != ORBIT_RUN) & amask;
            if (dm == amask)
                break;
            if (dm) {
                differ = true;
                break;
            }
        }
        // every orbit finished in round rnd (else they would differ)
        if (!differ && stt == ORBIT_PEND) {
            if (SHORT)
                query_resolve<K>(o, rnd);
            else
                orbit_resolve<K>(o);
        }
        if (active)
            it += o.d;
        if (differ)
            return false;
        const uint32_t vmin = __reduce_min_sync(kLaneMask, active ? o.d : 0xffffffffu);
        const uint32_t vmax = __reduce_max_sync(kLaneMask, active ? o.d : 0u);
        if (vmin != vmax || (have && vmin != w))
            return false;
        have = true;
        w = vmin;
    }
    *w_out = w;
    return true;
}

// All warps of a CTA query the perimeter of g together; warps share the
// verdict through s_flag (1 = not uniform) and the common dwell through s_w
// (0xffffffff = none yet).  The caller sets *s_flag = 0 and *s_w = 0xffffffff
// and synchronises the CTA before the call; the call ends with a CTA barrier.
__device__ __forceinline__ bool cta_perimeter_uniform(const PixelMap &pm, uint32_t max_dwell,
                                                      const Region &g, uint32_t tid, uint32_t T,
                                                      uint32_t *s_flag, uint32_t *s_w,
                                                      uint32_t *w_out, unsigned long long &it)
{
    const uint32_t P = perimeter_size(g.w, g.h);
    const uint32_t lane = tid & 31u;
    volatile uint32_t *vflag = s_flag;
    volatile uint32_t *vw = s_w;
    for (uint32_t base = (tid & ~31u); base < P; base += T) {
        if (__shfl_sync(kLaneMask, *vflag, 0))
            break;
        const uint32_t k = base + lane;
        const bool active = k < P;
        const unsigned amask = __ballot_sync(kLaneMask, active);
        uint32_t px = g.x0, py = g.y0;
        if (active)
            perimeter_pixel(g, k, px, py);
        Orbit o = orbit_start(pixel_c(pm, px, py));
        uint32_t stt = active ? ORBIT_RUN : ORBIT_DONE;
        bool differ = false, stop = false;
        for (;;) {
            // one value per warp, so every lane uses the same limit
            const uint32_t wv = __shfl_sync(kLaneMask, *vw, 0);
            const uint32_t limit = (wv != 0xffffffffu) ? min(max_dwell, wv + 1u) : max_dwell;
            if (stt == ORBIT_RUN)
                stt = orbit_step<kQueryRoundCta>(o, limit);
            const unsigned dm = __ballot_sync(kLaneMask, stt != ORBIT_RUN) & amask;
            if (dm == amask)
                break;
            if (dm) {
                differ = true;
                break;
            }
            if (__shfl_sync(kLaneMask, *vflag, 0)) {
                stop = true;
                break;
            }
        }
        if (!stop && !differ && stt == ORBIT_PEND)
            orbit_resolve<kQueryRoundCta>(o);
        if (active)
            it += o.d;
        if (stop)
            break;
        if (differ) {
            if (lane == 0)
                *vflag = 1u;
            break;
        }
        const uint32_t vmin = __reduce_min_sync(kLaneMask, active ? o.d : 0xffffffffu);
        const uint32_t vmax = __reduce_max_sync(kLaneMask, active ? o.d : 0u);
        if (lane == 0) {
            if (vmin != vmax) {
                *vflag = 1u;
            } else {
                const uint32_t old = atomicCAS(s_w, 0xffffffffu, vmin);
                if (old != 0xffffffffu && old != vmin)
                    *vflag = 1u;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    const bool uniform = (*vflag == 0u);
    *w_out = *vw;
    __syncthreads();
    return uniform;
}

__device__ __forceinline__ uint32_t ceil_div_u32(uint32_t a, uint32_t b)
{
    return a / b + (a % b != 0u);
}

// Number of non-empty children of a region (r x r split into side sc,
// clipped to the region).
__device__ __forceinline__ uint32_t child_count(const Region &g, uint32_t sc, uint32_t r)
{
    const uint32_t cx = min(r, ceil_div_u32(g.w, sc));
    const uint32_t cy = min(r, ceil_div_u32(g.h, sc));
    return cx * cy;
}

// j-th non-empty child (row-major over the cx x cy children).
__device__ __forceinline__ uint2 child_region(const Region &g, uint32_t sc, uint32_t r, uint32_t j)
{
    const uint32_t cx = min(r, ceil_div_u32(g.w, sc));
    const uint32_t a = j % cx, b = j / cx;
    const uint32_t x = g.x0 + a * sc, y = g.y0 + b * sc;
    const uint32_t w = min(sc, g.x0 + g.w - x), h = min(sc, g.y0 + g.h - y);
    return pack_region(x, y, w, h);
}

}  // namespace ask
