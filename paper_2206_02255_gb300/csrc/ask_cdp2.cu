// ask_cdp2.cu -- Mariani-Silver subdivision driven by CUDA Dynamic
// Parallelism (paper Sec. 3; the DP implementations compared in Sec. 6),
// written for the CDP2 device runtime of CUDA 12+: a subdividing region
// launches one child grid, r x r CTAs (one per non-empty sub-region, the SBR
// mapping of Sec. 4.3.1), so no parent ever waits on a child.  By default the
// child goes into the tail-launch stream: it starts once the parent grid has
// finished, and the tail launches of one grid run in launch order.  With
// ASK_FLAG_CDP2_FIRE_AND_FORGET it goes into the fire-and-forget stream and
// runs concurrently with its parent and siblings.  The host sees the render
// complete when the whole tree of grids has completed.
//
// With ASK_FLAG_MBR (the DP-MBR scheme, Sec. 4.3.2) a region's fill and a
// leaf region's pixels are not done by its own CTA either: it launches a
// child grid of many blocks for them, into the same stream as its splits.
//
// This translation unit is compiled with relocatable device code and linked
// against the device runtime; the rest of the library is not.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_internal.h"

namespace ask {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kStageMax = 16384;  // staged perimeter pixels per CTA

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// DP-MBR fill: block b writes rows [b * rows, b * rows + rows) of g.
__global__ void __launch_bounds__(1024) cdp2_fill_kernel(uint32_t *map, uint32_t n, Region g,
                                                         uint32_t v, uint32_t rows)
{
    Region band = g;
    band.y0 = g.y0 + blockIdx.x * rows;
    if (band.y0 >= g.y0 + g.h)
        return;
    band.h = min(rows, g.y0 + g.h - band.y0);
    fill_rect(map, n, band, v, threadIdx.x, blockDim.x);
}

// DP-MBR leaf: one thread per interior pixel of g (its perimeter is already
// written), block (blockIdx.x, blockIdx.y) covers one blockDim tile.
__global__ void __launch_bounds__(1024) cdp2_pixel_kernel(CdpArgs a, Region g)
{
    const uint32_t px = g.x0 + blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t py = g.y0 + blockIdx.y * blockDim.y + threadIdx.y;
    unsigned long long it = 0;
    if (px < g.x0 + g.w && py < g.y0 + g.h && !on_perimeter(g, px, py)) {
        const float2 c = pixel_c(a.pm, px, py);
        const uint32_t d = dwell(c.x, c.y, a.max_dwell);
        a.map[(size_t)py * a.n + px] = d;
        it = d;
    }
    if (a.count) {
        it = warp_sum_u64(it);
        if (((threadIdx.x + threadIdx.y * blockDim.x) & 31u) == 0u && it)
            atomicAdd(&a.ctr->iterations, it);
    }
}

// Shared memory of a region's CTA besides the perimeter stage.
struct CdpShared {
    uint32_t red_min[32], red_max[32];
    uint32_t s_min, s_max, s_flag, s_w, s_base;
};

// Tail launches without MBR take the per-depth lists.
__device__ __forceinline__ bool list_mode(const CdpArgs &a) { return !a.fire_and_forget && !a.mbr; }

__global__ void __launch_bounds__(1024) cdp2_region_kernel(CdpArgs a, uint32_t px0, uint32_t py0,
                                                           uint32_t pw, uint32_t ph, uint32_t side,
                                                           uint32_t level);

// The work of one region g of nominal side `side` at depth `level`, by one
// CTA: the exploration query, then a fill, a split (a child grid, or the
// next depth's list) or the leaf's pixels.
__device__ __forceinline__ void cdp2_region(const CdpArgs &a, const Region &g, uint32_t side,
                                            uint32_t level, uint32_t *stage, CdpShared &sh)
{
    const uint32_t T = blockDim.x * blockDim.y;
    const uint32_t tid = threadIdx.x + threadIdx.y * blockDim.x;
    const uint32_t lane = tid & 31u, wid = tid >> 5, nw = T >> 5;
    const uint32_t stage_cap = min(4u * side, kStageMax);
    const uint32_t sc = ceil_div_u32(side, a.r);
    const bool split = side > 1u && sc >= a.B;
    unsigned long long it = 0;
    const uint32_t P = perimeter_size(g.w, g.h);
    uint32_t dmin, dmax;

    if (split) {
        // exploration query that stops at the first difference
        if (tid == 0) {
            sh.s_flag = 0u;
            sh.s_w = 0xffffffffu;
        }
        __syncthreads();
        uint32_t wv = 0;
        const bool uni = cta_perimeter_uniform(a.pm, a.max_dwell, g, tid, T, &sh.s_flag, &sh.s_w, &wv, it);
        dmin = wv;
        dmax = uni ? wv : wv + 1u;
    } else {
        // exploration query of a region that would be a leaf: perimeter
        // dwells staged in shared memory
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
            it += d;
        }
        dmin = __reduce_min_sync(kFull, dmin);
        dmax = __reduce_max_sync(kFull, dmax);
        if (lane == 0) {
            sh.red_min[wid] = dmin;
            sh.red_max[wid] = dmax;
        }
        __syncthreads();
        if (wid == 0) {
            uint32_t m0 = lane < nw ? sh.red_min[lane] : 0xffffffffu;
            uint32_t m1 = lane < nw ? sh.red_max[lane] : 0u;
            m0 = __reduce_min_sync(kFull, m0);
            m1 = __reduce_max_sync(kFull, m1);
            if (lane == 0) {
                sh.s_min = m0;
                sh.s_max = m1;
            }
        }
        __syncthreads();
        dmin = sh.s_min;
        dmax = sh.s_max;
    }

    if (dmin == dmax) {
        if (a.mbr) {
            if (tid == 0) {
                // about four pixels per thread of a block
                const uint32_t rows = max(1u, (4u * T) / g.w);
                const uint32_t nb = ceil_div_u32(g.h, rows);
                if (a.fire_and_forget)
                    cdp2_fill_kernel<<<nb, T, 0, cudaStreamFireAndForget>>>(a.map, a.n, g, dmin, rows);
                else
                    cdp2_fill_kernel<<<nb, T, 0, cudaStreamTailLaunch>>>(a.map, a.n, g, dmin, rows);
                if (cudaGetLastError() != cudaSuccess)
                    atomicOr(&a.ctr->error, ERR_DEVICE_LAUNCH);
            }
        } else {
            fill_rect(a.map, a.n, g, dmin, tid, T);
        }
        if (tid == 0)
            atomicAdd(&a.ctr->fills[min(level, (uint32_t)ASK_MAX_LEVELS - 1u)], 1u);
    } else {
        if (split && list_mode(a)) {
            // append the children to the next depth's list
            const uint32_t cx = min(a.r, ceil_div_u32(g.w, sc));
            const uint32_t cy = min(a.r, ceil_div_u32(g.h, sc));
            if (tid == 0) {
                atomicAdd(&a.ctr->subdivs[min(level, (uint32_t)ASK_MAX_LEVELS - 1u)], 1u);
                sh.s_base = atomicAdd(&a.ctr->count[level + 1u], cx * cy);
            }
            __syncthreads();
            for (uint32_t j = tid; j < cx * cy; j += T) {
                const uint32_t slot = sh.s_base + j;
                if (slot < a.list_cap)
                    a.list[(level + 1u) & 1u][slot] = child_region(g, sc, a.r, j);
                else
                    atomicOr(&a.ctr->error, ERR_OLT_OVERFLOW);
            }
        } else if (split) {
            if (tid == 0) {
                atomicAdd(&a.ctr->subdivs[min(level, (uint32_t)ASK_MAX_LEVELS - 1u)], 1u);
                const uint32_t cx = min(a.r, ceil_div_u32(g.w, sc));
                const uint32_t cy = min(a.r, ceil_div_u32(g.h, sc));
                const size_t smem = (size_t)min(4u * sc, kStageMax) * sizeof(uint32_t);
                if (a.fire_and_forget)
                    cdp2_region_kernel<<<dim3(cx, cy), dim3(blockDim.x, blockDim.y), smem,
                                         cudaStreamFireAndForget>>>(a, g.x0, g.y0, g.w, g.h, sc,
                                                                    level + 1u);
                else
                    cdp2_region_kernel<<<dim3(cx, cy), dim3(blockDim.x, blockDim.y), smem,
                                         cudaStreamTailLaunch>>>(a, g.x0, g.y0, g.w, g.h, sc,
                                                                 level + 1u);
                if (cudaGetLastError() != cudaSuccess)
                    atomicOr(&a.ctr->error, ERR_DEVICE_LAUNCH);
            }
        } else {
            // leaf: perimeter from the stage, interior pixel by pixel
            const uint32_t staged = min(P, stage_cap);
            for (uint32_t k = tid; k < staged; k += T) {
                uint32_t px, py;
                perimeter_pixel(g, k, px, py);
                a.map[(size_t)py * a.n + px] = stage[k];
            }
            if (a.mbr) {
                if (tid == 0) {
                    if (g.w > 2u && g.h > 2u) {
                        const dim3 grid(ceil_div_u32(g.w, blockDim.x), ceil_div_u32(g.h, blockDim.y));
                        const dim3 block(blockDim.x, blockDim.y);
                        if (a.fire_and_forget)
                            cdp2_pixel_kernel<<<grid, block, 0, cudaStreamFireAndForget>>>(a, g);
                        else
                            cdp2_pixel_kernel<<<grid, block, 0, cudaStreamTailLaunch>>>(a, g);
                        if (cudaGetLastError() != cudaSuccess)
                            atomicOr(&a.ctr->error, ERR_DEVICE_LAUNCH);
                    }
                    atomicAdd(&a.ctr->leaf_count, 1u);
                }
            } else {
                for (uint32_t ty0 = 0; ty0 < g.h; ty0 += blockDim.y) {
                    for (uint32_t tx0 = 0; tx0 < g.w; tx0 += blockDim.x) {
                        const uint32_t px = g.x0 + tx0 + threadIdx.x, py = g.y0 + ty0 + threadIdx.y;
                        if (px < g.x0 + g.w && py < g.y0 + g.h && !on_perimeter(g, px, py)) {
                            const float2 c = pixel_c(a.pm, px, py);
                            const uint32_t d = dwell(c.x, c.y, a.max_dwell);
                            a.map[(size_t)py * a.n + px] = d;
                            it += d;
                        }
                    }
                }
                if (tid == 0)
                    atomicAdd(&a.ctr->leaf_count, 1u);
            }
        }
    }
    if (a.count) {
        it = warp_sum_u64(it);
        if (lane == 0 && it)
            atomicAdd(&a.ctr->iterations, it);
    }
}

__global__ void __launch_bounds__(1024) cdp2_list_kernel(CdpArgs a, uint32_t side, uint32_t level);

// The last CTA of a depth's grid to finish tail-launches one grid over the
// next depth's list (list mode only); `nblocks` CTAs count.
__device__ __forceinline__ void cdp2_grid_done(const CdpArgs &a, uint32_t side, uint32_t level,
                                               uint32_t nblocks)
{
    __syncthreads();  // every append of this CTA is issued
    if (threadIdx.x + threadIdx.y * blockDim.x != 0u)
        return;
    __threadfence();
    if (atomicAdd(&a.ctr->work[level], 1u) != nblocks - 1u)
        return;
    __threadfence();
    const uint32_t cnt = min(atomicAdd(&a.ctr->count[level + 1u], 0u), a.list_cap);
    if (cnt == 0u)
        return;
    const uint32_t sc = ceil_div_u32(side, a.r);
    const size_t smem = (size_t)min(4u * sc, kStageMax) * sizeof(uint32_t);
    cdp2_list_kernel<<<cnt, dim3(blockDim.x, blockDim.y), smem, cudaStreamTailLaunch>>>(a, sc, level + 1u);
    if (cudaGetLastError() != cudaSuccess)
        atomicOr(&a.ctr->error, ERR_DEVICE_LAUNCH);
}

// One CTA = one region: child (blockIdx.x, blockIdx.y) of side `side` inside
// the parent rectangle (px0, py0, pw, ph).  The root grid's "parent" is the
// whole image and its children are the g x g initial regions.
__global__ void __launch_bounds__(1024) cdp2_region_kernel(CdpArgs a, uint32_t px0, uint32_t py0,
                                                           uint32_t pw, uint32_t ph, uint32_t side,
                                                           uint32_t level)
{
    extern __shared__ uint32_t stage[];
    __shared__ CdpShared sh;
    const uint32_t x0 = px0 + blockIdx.x * side, y0 = py0 + blockIdx.y * side;
    if (x0 < px0 + pw && y0 < py0 + ph) {  // else an empty child (uniform over the CTA)
        Region g;
        g.x0 = x0;
        g.y0 = y0;
        g.w = min(side, px0 + pw - x0);
        g.h = min(side, py0 + ph - y0);
        cdp2_region(a, g, side, level, stage, sh);
    }
    if (list_mode(a))
        cdp2_grid_done(a, side, level, gridDim.x * gridDim.y);
}

// One CTA per region of depth `level`'s list (list mode).
__global__ void __launch_bounds__(1024) cdp2_list_kernel(CdpArgs a, uint32_t side, uint32_t level)
{
    extern __shared__ uint32_t stage[];
    __shared__ CdpShared sh;
    const Region g = unpack_region(a.list[level & 1u][blockIdx.x]);
    cdp2_region(a, g, side, level, stage, sh);
    cdp2_grid_done(a, side, level, gridDim.x);
}

bool list_mode_host(const CdpArgs &a) { return !a.fire_and_forget && !a.mbr; }

}  // namespace

cudaError_t launch_cdp2(const CdpArgs &a, uint32_t g, uint32_t s0, uint32_t bx, uint32_t by,
                        cudaStream_t s)
{
    const uint32_t axis0 = (a.n + s0 - 1) / s0;  // non-empty initial regions per axis
    (void)g;
    const size_t smem = (size_t)min(4u * s0, kStageMax) * sizeof(uint32_t);
    if (smem > 48 * 1024 || list_mode_host(a)) {
        cudaFuncSetAttribute(cdp2_region_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kStageMax * sizeof(uint32_t)));
        cudaFuncSetAttribute(cdp2_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kStageMax * sizeof(uint32_t)));
    }
    cdp2_region_kernel<<<dim3(axis0, axis0), dim3(bx, by), smem, s>>>(a, 0u, 0u, a.n, a.n, s0, 0u);
    return cudaGetLastError();
}

cudaError_t cdp2_set_pending_limit(size_t launches)
{
    return cudaDeviceSetLimit(cudaLimitDevRuntimePendingLaunchCount, launches);
}

}  // namespace ask
