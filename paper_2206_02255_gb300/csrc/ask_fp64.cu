// ask_fp64.cu -- dwell maps for deep zooms: the exhaustive kernel and the
// ASK pipeline (one level kernel per depth, one leaf kernel) in double
// precision (every operation of the iteration rounded once to binary64) or,
// with ASK_FLAG_FLOAT_FLOAT, in float-float arithmetic on the FP32 pipe.
//
// Past a zoom of about 1e4 over the paper's 2 x 2 window (Sec. 6.1), the
// pixels of a large map lie closer together than single precision can tell
// apart near |c| ~ 1, so neighbouring columns share one c.  Such frames are
// rendered in wider arithmetic.  The subdivision is the single-precision
// path's (Sec. 4.2.1, Sec. 5): the same plan, region tables, counters and
// decisions; only the arithmetic of the dwell differs.  Binary64:
//   zi2 = zi*zi; m = fma(zr, zr, zi2); continue while m < 4;
//   zr' = fma(zr, zr, fma(-zi, zi, cr)); zi' = fma(zr + zr, zi, ci);
//   cr = fma(px, dx, re_min), ci = fma(py, dy, im_min), dx and dy in double.
// Float-float: see ArithFF.
//
// GB300 issues double-precision instructions at 1/64 of its single-precision
// rate, so the binary64 kernels are bound by the FP64 pipe, and votes,
// shared-memory parking and address arithmetic hide behind it; float-float
// spends about 14x more instructions per update on a pipe 64x faster.  In
// both, what matters is that lanes spend their arithmetic on useful updates:
//  * level kernel: persistent, one warp per region from an atomic counter;
//    the perimeter is queried 32 pixels at a time with the orbits in
//    lockstep rounds, so the query stops as soon as one orbit has finished
//    while another still runs; uniform regions are filled in place;
//  * leaf kernel: persistent; a lane whose orbit ends takes the next pixel
//    of its warp's current leaf (then of the next leaf) at once; an orbit
//    that escapes inside an unchecked block is parked in shared memory and
//    32 parked orbits are resolved together, so no lane replays alone.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_fp64.h"

namespace ask {

namespace {

constexpr unsigned kAll = 0xffffffffu;
// Updates per unchecked block of the exhaustive kernel's dwell loop, and per
// lockstep round of the perimeter queries and of the leaf kernel's orbits.
constexpr uint32_t kBlock64 = 16;
constexpr uint32_t kRound64 = 8;
// |c|^2 bounds below which escape is absorbing (see the policies' absorbing()).
constexpr double kAbsorbR2_F64 = 3.999;
constexpr float kAbsorbR2_FF = 3.999f;
// Leaf kernel: warps per CTA and parked orbits per warp (fewer than 32 wait
// between resolves, and one round parks at most 32 more).
constexpr uint32_t kLeaf64Warps = 4;
constexpr uint32_t kPark64 = 64;

__device__ __forceinline__ double2 pixel_c64(const PixelMap64 &pm, uint32_t px, uint32_t py)
{
    return make_double2(__fma_rn(__uint2double_rn(px), pm.dx, pm.re_min),
                        __fma_rn(__uint2double_rn(py), pm.dy, pm.im_min));
}

// Binary64: one update z <- z^2 + c, each operation rounded once to double.
struct ArithF64 {
    using T = double;
    static __device__ __forceinline__ T from_double(double v) { return v; }
    static __device__ __forceinline__ void update(T &x, T &y, T cr, T ci)
    {
        const double t = __fma_rn(-y, y, cr);
        const double nx = __fma_rn(x, x, t);
        const double ny = __fma_rn(__dadd_rn(x, x), y, ci);
        x = nx;
        y = ny;
    }
    static __device__ __forceinline__ bool bounded(T x, T y)
    {
        return __fma_rn(x, x, __dmul_rn(y, y)) < 4.0;
    }
    // The single-precision argument carries over with a wider margin: for
    // |c|^2 < 3.999, a rounded |z_j|^2 >= 4 means the exact |z_j|^2 exceeds
    // 4 - 1e-15, so |z_j^2 + c| > 2 + 2.3e-4, far beyond what the rounding
    // of one update (a few ulps) can undo; |z| then grows until it overflows
    // to inf and NaN, which also fail the test.  So a state that passes the
    // test proves that every earlier state passed.
    static __device__ __forceinline__ bool absorbing(T cr, T ci)
    {
        return __fma_rn(cr, cr, __dmul_rn(ci, ci)) < kAbsorbR2_F64;
    }
};

// Float-float ("double-single"): a value is the unevaluated sum hi + lo of
// two floats (x = hi, y = lo), about 48 significant bits on the FP32 pipe.
// Building blocks, each float operation rounded once: TwoSum (Knuth),
// Fast2Sum (Dekker) and the exact error of a product, fma(a, b, -a*b).
//   add(x, y): (s, e) = TwoSum(xh, yh); Fast2Sum(s, e + (xl + yl))
//     (the "sloppy" sum: its error is bounded relative to the operands,
//     which suffices while |z| and |c| stay near 2);
//   mul(x, y): p = xh*yh; e = fma(xh, yh, -p); e = fma(xh, yl, e);
//     e = fma(xl, yh, e); Fast2Sum(p, e); sqr likewise with one 2*xh*xl term.
// One update: zr2 = sqr(zr), zi2 = sqr(zi); zr' = add(zr2, add(cr, -zi2));
// zi' = add(2 mul(zr, zi), ci).  The test: zr2.hi + zi2.hi < 4.  c comes
// from the double-precision pixel map, split as hi = (float)c,
// lo = (float)(c - hi).  About 60 FP32 instructions per update.
struct ArithFF {
    using T = float2;
    static __device__ __forceinline__ float2 fast_two_sum(float a, float b)
    {
        const float s = __fadd_rn(a, b);
        return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
    }
    static __device__ __forceinline__ float2 add(float2 x, float2 y)
    {
        const float s = __fadd_rn(x.x, y.x);
        const float bb = __fsub_rn(s, x.x);
        const float e = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bb)), __fsub_rn(y.x, bb));
        return fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.y, y.y)));
    }
    static __device__ __forceinline__ float2 mul(float2 x, float2 y)
    {
        const float p = __fmul_rn(x.x, y.x);
        float e = __fmaf_rn(x.x, y.x, -p);
        e = __fmaf_rn(x.x, y.y, e);
        e = __fmaf_rn(x.y, y.x, e);
        return fast_two_sum(p, e);
    }
    static __device__ __forceinline__ float2 sqr(float2 x)
    {
        const float p = __fmul_rn(x.x, x.x);
        float e = __fmaf_rn(x.x, x.x, -p);
        e = __fmaf_rn(__fadd_rn(x.x, x.x), x.y, e);
        return fast_two_sum(p, e);
    }
    static __device__ __forceinline__ T from_double(double v)
    {
        const float hi = __double2float_rn(v);
        return make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
    }
    static __device__ __forceinline__ void update(T &x, T &y, T cr, T ci)
    {
        const float2 zr2 = sqr(x), zi2 = sqr(y);
        const float2 nx = add(zr2, add(cr, make_float2(-zi2.x, -zi2.y)));
        const float2 p = mul(x, y);
        const float2 ny = add(make_float2(__fadd_rn(p.x, p.x), __fadd_rn(p.y, p.y)), ci);
        x = nx;
        y = ny;
    }
    static __device__ __forceinline__ bool bounded(T x, T y)
    {
        return __fadd_rn(sqr(x).x, sqr(y).x) < 4.0f;
    }
    // As in single precision: if zr2.hi + zi2.hi rounds to >= 4 the exact
    // |z_j|^2 exceeds 4 - 1e-6, so for |c|^2 < 3.999 (tested on the hi parts)
    // |z_j^2 + c| > 2 + 2e-4, which no rounding of an update undoes; |z|
    // grows until the float parts overflow, and inf and NaN fail the test.
    static __device__ __forceinline__ bool absorbing(T cr, T ci)
    {
        return __fmaf_rn(cr.x, cr.x, __fmul_rn(ci.x, ci.x)) < kAbsorbR2_FF;
    }
};

// Dwell of one point: blocks of kBlock64 unchecked updates where escape is
// absorbing, the failing block replayed one tested update at a time.
template <class A>
__device__ __forceinline__ uint32_t dwell_w(double2 c, uint32_t max_dwell)
{
    using T = typename A::T;
    const T cr = A::from_double(c.x), ci = A::from_double(c.y);
    T x = A::from_double(0.0), y = A::from_double(0.0);
    uint32_t d = 0;
    if (A::absorbing(cr, ci)) {
        while (max_dwell - d >= kBlock64) {
            const T sx = x, sy = y;
#pragma unroll
            for (uint32_t k = 0; k < kBlock64; ++k)
                A::update(x, y, cr, ci);
            if (!A::bounded(x, y)) {
                x = sx;
                y = sy;
                break;
            }
            d += kBlock64;
        }
    }
    while (d < max_dwell && A::bounded(x, y)) {
        A::update(x, y, cr, ci);
        ++d;
    }
    return d;
}

// Resumable orbit (the wide twin of the single-precision perimeter
// queries' orbit): every state before z_d passed the test.
template <class A>
struct OrbitW {
    typename A::T x, y, cr, ci;
    uint32_t d;
    bool fast;
};

template <class A>
__device__ __forceinline__ OrbitW<A> orbit_w_start(double2 c)
{
    OrbitW<A> o;
    o.x = A::from_double(0.0);
    o.y = A::from_double(0.0);
    o.cr = A::from_double(c.x);
    o.ci = A::from_double(c.y);
    o.d = 0;
    o.fast = A::absorbing(o.cr, o.ci);
    return o;
}

// Up to K more updates without passing `limit` (ORBIT_RUN / ORBIT_DONE /
// ORBIT_PEND as for the single-precision orbits): a pending orbit escaped
// inside the unchecked block and keeps the block's starting state.
template <class A, uint32_t K>
__device__ __forceinline__ uint32_t orbit_w_step(OrbitW<A> &o, uint32_t limit)
{
    if (o.d >= limit)
        return ORBIT_DONE;
    if (o.fast && limit - o.d >= K) {
        typename A::T x = o.x, y = o.y;
#pragma unroll
        for (uint32_t k = 0; k < K; ++k)
            A::update(x, y, o.cr, o.ci);
        if (!A::bounded(x, y))
            return ORBIT_PEND;
        o.x = x;
        o.y = y;
        o.d += K;
        return o.d >= limit ? ORBIT_DONE : ORBIT_RUN;
    }
    for (uint32_t k = 0; k < K; ++k) {
        if (o.d >= limit || !A::bounded(o.x, o.y))
            return ORBIT_DONE;
        A::update(o.x, o.y, o.cr, o.ci);
        ++o.d;
    }
    return o.d >= limit ? ORBIT_DONE : ORBIT_RUN;
}

// Exact dwell of a pending orbit: z_d passed, z_{d+K} failed, and failing is
// absorbing, so halving the gap finds the first failing state (K - 1
// updates, log2(K) tests, the same instruction stream on every lane).
template <class A, uint32_t K>
__device__ __forceinline__ void orbit_w_resolve(OrbitW<A> &o)
{
    typename A::T x = o.x, y = o.y;
    uint32_t d = o.d;
#pragma unroll
    for (uint32_t h = K / 2u; h >= 1u; h >>= 1) {
        typename A::T tx = x, ty = y;
#pragma unroll
        for (uint32_t k = 0; k < h; ++k)
            A::update(tx, ty, o.cr, o.ci);
        if (A::bounded(tx, ty)) {
            x = tx;
            y = ty;
            d += h;
        }
    }
    o.d = d + 1u;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kAll, v, o);
    return v;
}

// One warp queries the whole perimeter of g (Q of Sec. 4.2.1): 32 perimeter
// pixels at a time, their orbits in lockstep rounds.  An orbit still running
// after a round has made more updates than any that finished in it, so one
// finished and one running orbit prove the perimeter non-uniform.  Once a
// group ends with a common dwell w, later groups stop at w + 1 updates.
// Returns true with the common dwell in *w_out; `it` gains the updates made.
template <class A>
__device__ __forceinline__ bool warp_uniform_w(const PixelMap64 &pm, uint32_t max_dwell,
                                               const Region &g, uint32_t lane, uint32_t *w_out,
                                               unsigned long long &it)
{
    const uint32_t P = perimeter_size(g.w, g.h);
    bool have = false;
    uint32_t w = 0;
    for (uint32_t base = 0; base < P; base += 32u) {
        const uint32_t k = base + lane;
        const bool active = k < P;
        const unsigned amask = __ballot_sync(kAll, active);
        uint32_t px = g.x0, py = g.y0;
        if (active)
            perimeter_pixel(g, k, px, py);
        OrbitW<A> o = orbit_w_start<A>(pixel_c64(pm, px, py));
        uint32_t stt = active ? ORBIT_RUN : ORBIT_DONE;
        const uint32_t limit = have ? min(max_dwell, w + 1u) : max_dwell;
        bool differ = false;
        for (;;) {
            if (stt == ORBIT_RUN)
                stt = orbit_w_step<A, kRound64>(o, limit);
            const unsigned dm = __ballot_sync(kAll, stt != ORBIT_RUN) & amask;
            if (dm == amask)
                break;
            if (dm) {
                differ = true;
                break;
            }
        }
        if (!differ && stt == ORBIT_PEND)
            orbit_w_resolve<A, kRound64>(o);
        if (active)
            it += o.d;
        if (differ)
            return false;
        const uint32_t vmin = __reduce_min_sync(kAll, active ? o.d : 0xffffffffu);
        const uint32_t vmax = __reduce_max_sync(kAll, active ? o.d : 0u);
        if (vmin != vmax || (have && vmin != w))
            return false;
        have = true;
        w = vmin;
    }
    *w_out = w;
    return true;
}

// ---------------------------------------------------------------------------
// Exhaustive: one thread per pixel in block_x x block_y tiles (Sec. 4.1).
// ---------------------------------------------------------------------------
template <class A, bool COUNT>
__global__ void __launch_bounds__(1024) exhaustive64_kernel(uint32_t *__restrict__ map, uint32_t n,
                                                            PixelMap64 pm, uint32_t max_dwell,
                                                            uint32_t tiles_x, DevCounters *ctr)
{
    const uint32_t tile = blockIdx.x;
    const uint32_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const uint32_t px = tx * blockDim.x + threadIdx.x;
    const uint32_t py = ty * blockDim.y + threadIdx.y;
    uint32_t d = 0;
    if (px < n && py < n) {
        d = dwell_w<A>(pixel_c64(pm, px, py), max_dwell);
        map[(size_t)py * n + px] = d;
    }
    if (COUNT) {
        const unsigned long long s = warp_sum64(d);
        if ((threadIdx.x + threadIdx.y * blockDim.x) % 32u == 0u && s)
            atomicAdd(&ctr->iterations, s);
    }
}

// ---------------------------------------------------------------------------
// Level kernel of depth a.level: query, fill (T, in place), split (S, appended
// to the write-OLT with one atomicAdd for the region's r x r children,
// Sec. 5.3.1) or leaf.
// ---------------------------------------------------------------------------
template <class A, bool COUNT>
__global__ void __launch_bounds__(256) level64_kernel(Level64Args a)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t total = min(a.ctr->count[a.level], a.olt_cap);
    unsigned long long it = 0, fill_px = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0u)
            i = atomicAdd(&a.ctr->work[a.level], 1u);
        i = __shfl_sync(kAll, i, 0);
        if (i >= total)
            break;
        const uint2 rec = a.olt_in[i];
        const Region g = unpack_region(rec);
        uint32_t w = 0;
        if (warp_uniform_w<A>(a.pm, a.max_dwell, g, lane, &w, it)) {
            fill_rect(a.map, a.n, g, w, lane, 32u);
            if (lane == 0u) {
                atomicAdd(&a.ctr->fills[a.level], 1u);
                fill_px += (unsigned long long)g.w * g.h;
            }
        } else if (a.split) {
            const uint32_t nc = child_count(g, a.child_side, a.r);
            uint32_t base = 0;
            if (lane == 0u) {
                base = atomicAdd(&a.ctr->count[a.level + 1u], nc);
                atomicAdd(&a.ctr->subdivs[a.level], 1u);
            }
            base = __shfl_sync(kAll, base, 0);
            if ((unsigned long long)base + nc > a.olt_cap) {
                if (lane == 0u)
                    atomicOr(&a.ctr->error, ERR_OLT_OVERFLOW);
            } else {
                for (uint32_t j = lane; j < nc; j += 32u)
                    a.olt_out[base + j] = child_region(g, a.child_side, a.r, j);
            }
        } else if (lane == 0u) {
            const uint32_t slot = atomicAdd(&a.ctr->leaf_count, 1u);
            if (slot < a.leaf_cap)
                a.leaves[slot] = rec;
            else
                atomicOr(&a.ctr->error, ERR_LEAF_OVERFLOW);
        }
    }
    if (COUNT) {
        it = warp_sum64(it);
        if (lane == 0u) {
            atomicAdd(&a.ctr->level_iters[a.level], it);
            atomicAdd(&a.ctr->iterations, it);
            if (fill_px)
                atomicAdd(&a.ctr->fill_pixels, fill_px);
        }
    }
}

// ---------------------------------------------------------------------------
// Leaf kernel: every pixel of every leaf region (the final terminal pass of
// Sec. 5.1).
// ---------------------------------------------------------------------------
template <class A>
struct ParkW {
    typename A::T x[kLeaf64Warps][kPark64], y[kLeaf64Warps][kPark64];
    typename A::T cr[kLeaf64Warps][kPark64], ci[kLeaf64Warps][kPark64];
    uint32_t d[kLeaf64Warps][kPark64], pix[kLeaf64Warps][kPark64];
};

template <class A, bool COUNT>
__device__ __forceinline__ void resolve_parked_w(const Leaf64Args &a, ParkW<A> &pk, uint32_t wid,
                                                 uint32_t e, unsigned long long &it,
                                                 unsigned long long &npx)
{
    OrbitW<A> q;
    q.x = pk.x[wid][e];
    q.y = pk.y[wid][e];
    q.cr = pk.cr[wid][e];
    q.ci = pk.ci[wid][e];
    q.d = pk.d[wid][e];
    q.fast = true;
    const uint32_t pix = pk.pix[wid][e];
    orbit_w_resolve<A, kRound64>(q);
    a.map[(size_t)(pix >> 16) * a.n + (pix & 0xffffu)] = q.d;
    if (COUNT) {
        it += q.d;
        ++npx;
    }
}

template <class A, bool COUNT>
__global__ void __launch_bounds__(kLeaf64Warps * 32) leaf64_kernel(Leaf64Args a)
{
    __shared__ ParkW<A> pk;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const uint32_t nleaves = min(a.ctr->leaf_count, a.leaf_cap);
    // warp-uniform: the leaf being handed out and how many of its pixels are
    Region cur;
    cur.x0 = cur.y0 = 0;
    cur.w = cur.h = 1;
    unsigned long long next = 0, npix = 0;  // a leaf may hold up to 2^32 pixels
    bool have = false, exhausted = false;
    uint32_t parked = 0;
    // per lane: its orbit and pixel (x | y << 16; n <= 65536)
    OrbitW<A> o = orbit_w_start<A>(make_double2(0.0, 0.0));
    uint32_t pix = 0;
    bool busy = false;
    unsigned long long it = 0, npx = 0;
    for (;;) {
        unsigned need = __ballot_sync(kAll, !busy);
        while (need != 0u && !exhausted) {
            if (!have) {
                uint32_t li = 0;
                if (lane == 0u)
                    li = atomicAdd(&a.ctr->leaf_work, 1u);
                li = __shfl_sync(kAll, li, 0);
                if (li >= nleaves) {
                    exhausted = true;
                    break;
                }
                cur = unpack_region(a.leaves[li]);
                next = 0;
                npix = (unsigned long long)cur.w * cur.h;
                have = true;
            }
            const unsigned long long avail = npix - next;
            const uint32_t rank = (uint32_t)__popc(need & below);
            if (!busy && rank < avail) {
                const unsigned long long k = next + rank;
                const uint32_t ry = (uint32_t)(k / cur.w);
                const uint32_t px = cur.x0 + (uint32_t)(k - (unsigned long long)ry * cur.w);
                const uint32_t py = cur.y0 + ry;
                o = orbit_w_start<A>(pixel_c64(a.pm, px, py));
                pix = px | (py << 16);
                busy = true;
            }
            next += min((unsigned long long)__popc(need), avail);
            if (next >= npix)
                have = false;
            need = __ballot_sync(kAll, !busy);
        }
        if (__ballot_sync(kAll, busy) == 0u)
            break;
        uint32_t st = ORBIT_RUN;
        if (busy) {
            st = orbit_w_step<A, kRound64>(o, a.max_dwell);
            if (st == ORBIT_DONE) {
                a.map[(size_t)(pix >> 16) * a.n + (pix & 0xffffu)] = o.d;
                if (COUNT) {
                    it += o.d;
                    ++npx;
                }
                busy = false;
            }
        }
        const unsigned pend = __ballot_sync(kAll, busy && st == ORBIT_PEND);
        if (pend != 0u) {
            if (busy && st == ORBIT_PEND) {
                const uint32_t e = parked + (uint32_t)__popc(pend & below);
                pk.x[wid][e] = o.x;
                pk.y[wid][e] = o.y;
                pk.cr[wid][e] = o.cr;
                pk.ci[wid][e] = o.ci;
                pk.d[wid][e] = o.d;
                pk.pix[wid][e] = pix;
                busy = false;
            }
            parked += (uint32_t)__popc(pend);
            __syncwarp();
            if (parked >= 32u) {
                parked -= 32u;
                resolve_parked_w<A, COUNT>(a, pk, wid, parked + lane, it, npx);
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (lane < parked)
        resolve_parked_w<A, COUNT>(a, pk, wid, lane, it, npx);
    if (COUNT) {
        it = warp_sum64(it);
        npx = warp_sum64(npx);
        if (lane == 0u) {
            atomicAdd(&a.ctr->leaf_iters, it);
            atomicAdd(&a.ctr->iterations, it);
            atomicAdd(&a.ctr->leaf_pixels, npx);
        }
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

cudaError_t launch_exhaustive64(uint32_t *map, uint32_t n, PixelMap64 pm, uint32_t max_dwell,
                                uint32_t bx, uint32_t by, bool count, bool ff, DevCounters *ctr,
                                cudaStream_t s)
{
    const uint32_t tiles_x = (n + bx - 1) / bx, tiles_y = (n + by - 1) / by;
    const unsigned long long tiles = (unsigned long long)tiles_x * tiles_y;
    if (tiles > 0x7fffffffull)
        return cudaErrorInvalidConfiguration;
    const dim3 block(bx, by);
    const unsigned grid = (unsigned)tiles;
    if (ff) {
        if (count)
            exhaustive64_kernel<ArithFF, true><<<grid, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
        else
            exhaustive64_kernel<ArithFF, false><<<grid, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
    } else {
        if (count)
            exhaustive64_kernel<ArithF64, true><<<grid, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
        else
            exhaustive64_kernel<ArithF64, false><<<grid, block, 0, s>>>(map, n, pm, max_dwell, tiles_x, ctr);
    }
    return cudaGetLastError();
}

template <class A, bool COUNT>
static void level_w_launch(const Level64Args &a, int sms, cudaStream_t s)
{
    level64_kernel<A, COUNT><<<resident_grid(level64_kernel<A, COUNT>, 256, sms), 256, 0, s>>>(a);
}

cudaError_t launch_level64(const Level64Args &a, bool count, bool ff, int sms, cudaStream_t s)
{
    if (ff)
        count ? level_w_launch<ArithFF, true>(a, sms, s) : level_w_launch<ArithFF, false>(a, sms, s);
    else
        count ? level_w_launch<ArithF64, true>(a, sms, s) : level_w_launch<ArithF64, false>(a, sms, s);
    return cudaGetLastError();
}

template <class A, bool COUNT>
static void leaf_w_launch(const Leaf64Args &a, int sms, cudaStream_t s)
{
    const int threads = (int)kLeaf64Warps * 32;
    leaf64_kernel<A, COUNT><<<resident_grid(leaf64_kernel<A, COUNT>, threads, sms), threads, 0, s>>>(a);
}

cudaError_t launch_leaf64(const Leaf64Args &a, bool count, bool ff, int sms, cudaStream_t s)
{
    if (ff)
        count ? leaf_w_launch<ArithFF, true>(a, sms, s) : leaf_w_launch<ArithFF, false>(a, sms, s);
    else
        count ? leaf_w_launch<ArithF64, true>(a, sms, s) : leaf_w_launch<ArithF64, false>(a, sms, s);
    return cudaGetLastError();
}

}  // namespace ask
