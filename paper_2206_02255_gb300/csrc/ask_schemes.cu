// ask_schemes.cu -- the paper's two block-to-region mappings for ASK
// (Sec. 4.3): single block per region (SBR, Sec. 4.3.1) and multiple blocks
// per region (MBR, Sec. 4.3.2), as comparison variants of the default
// mapping in ask_kernels.cu.
//
//  * Both: one CTA of block_x * block_y threads takes a region, evaluates
//    its perimeter (Q) with every thread and decides fill, split (S) or
//    leaf.  CTAs are persistent and take regions from a device counter, so
//    every region is still handled by exactly one block without the host
//    reading the region count back.
//  * SBR: the same CTA writes a uniform region's fill (T); the last-level
//    pass gives each leaf region to one CTA, which computes all its pixels.
//  * MBR: a uniform region is appended to the fill list and written by the
//    fill kernel, whose blocks each take 8-row bands, so one region spreads
//    over many blocks; each leaf region is cut into block_x x block_y tiles
//    and the tiles go to different blocks (the tiled leaf kernel).
//
// Every variant writes the same map as the default mapping.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_device.cuh"
#include "ask_internal.h"

namespace ask {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoneW = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// One CTA per region: query, then fill in place (SBR) or defer the fill
// (MBR), append children or the leaf.  blockDim.x is a multiple of 32.
template <bool COUNT, bool MBR>
__global__ void __launch_bounds__(1024) region_level_kernel(LevelArgs a)
{
    __shared__ uint32_t s_item, s_flag, s_w, s_base;
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u;
    const uint2 *olt_in = static_cast<const uint2 *>(a.olt_in);
    uint2 *olt_out = static_cast<uint2 *>(a.olt_out);
    uint2 *leaves = static_cast<uint2 *>(a.leaves);
    DevCounters *ctr = a.ctr;
    const uint32_t count = min(ctr->count[a.level], a.olt_cap);
    unsigned long long it = 0, bpx = 0, fpx = 0;

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(&ctr->work[a.level], 1u);
            s_flag = 0u;
            s_w = kNoneW;
        }
        __syncthreads();
        const uint32_t t = s_item;
        if (t >= count)
            break;
        const uint2 e = olt_in[t];
        const Region g = unpack_region(e);
        uint32_t wv = 0;
        const bool uniform =
            cta_perimeter_uniform(a.pm, a.max_dwell, g, tid, T, &s_flag, &s_w, &wv, it);
        if (COUNT && tid == 0)
            bpx += perimeter_size(g.w, g.h);
        if (uniform) {
            if (MBR) {
                // the region's bands of rows go to the fill list
                const uint32_t nb = fill_band_count(g.w, g.h), rows = fill_band_rows(g.w);
                if (tid == 0)
                    s_base = atomicAdd(&ctr->fill_count, nb);
                __syncthreads();
                const uint32_t base = s_base;
                for (uint32_t j = tid; j < nb; j += T) {
                    const uint2 band = pack_region(g.x0, g.y0 + j * rows, g.w, min(rows, g.h - j * rows));
                    if (base + j < a.fill_cap)
                        a.fills[base + j] = make_uint4(band.x, band.y, wv, 0u);
                    else
                        atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
                }
                __syncthreads();
            } else {
                fill_rect(a.map, a.n, g, wv, tid, T);
            }
            if (tid == 0) {
                atomicAdd(&ctr->fills[a.level], 1u);
                if (COUNT)
                    fpx += (unsigned long long)g.w * g.h;
            }
        } else if (a.split) {
            const uint32_t nchild = child_count(g, a.child_side, a.r);
            if (tid == 0) {
                s_base = atomicAdd(&ctr->count[a.level + 1], nchild);
                atomicAdd(&ctr->subdivs[a.level], 1u);
            }
            __syncthreads();
            const uint32_t base = s_base;
            for (uint32_t j = tid; j < nchild; j += T) {
                if (base + j < a.olt_cap)
                    olt_out[base + j] = child_region(g, a.child_side, a.r, j);
                else
                    atomicOr(&ctr->error, ERR_OLT_OVERFLOW);
            }
        } else if (tid == 0) {
            const uint32_t slot = atomicAdd(&ctr->leaf_count, 1u);
            if (slot < a.leaf_cap)
                leaves[slot] = e;
            else
                atomicOr(&ctr->error, ERR_LEAF_OVERFLOW);
        }
        __syncthreads();  // s_* are rewritten by the next item
    }
    if (COUNT) {
        it = warp_sum_u64(it);
        if (lane == 0 && it) {
            atomicAdd(&ctr->iterations, it);
            atomicAdd(&ctr->level_iters[a.level], it);
        }
        if (tid == 0) {
            if (bpx)
                atomicAdd(&ctr->border_pixels, bpx);
            if (fpx)
                atomicAdd(&ctr->fill_pixels, fpx);
        }
    }
}

// SBR last level: one CTA per leaf region computes every pixel of it in
// block_x x block_y tiles.
template <bool COUNT>
__global__ void __launch_bounds__(1024) region_leaf_kernel(LeafArgs a)
{
    __shared__ uint32_t s_item;
    const uint32_t tid = threadIdx.x + threadIdx.y * blockDim.x;
    const uint2 *leaves = static_cast<const uint2 *>(a.leaves);
    const uint32_t nleaves = min(a.ctr->leaf_count, a.leaf_cap);
    unsigned long long it = 0, lpx = 0;
    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(&a.ctr->leaf_work, 1u);
        __syncthreads();
        const uint32_t li = s_item;
        __syncthreads();
        if (li >= nleaves)
            break;
        const Region g = unpack_region(leaves[li]);
        for (uint32_t ty0 = 0; ty0 < g.h; ty0 += blockDim.y) {
            for (uint32_t tx0 = 0; tx0 < g.w; tx0 += blockDim.x) {
                const uint32_t px = g.x0 + tx0 + threadIdx.x, py = g.y0 + ty0 + threadIdx.y;
                if (px < g.x0 + g.w && py < g.y0 + g.h) {
                    const float2 c = pixel_c(a.pm, px, py);
                    const uint32_t d = dwell(c.x, c.y, a.max_dwell);
                    a.map[(size_t)py * a.n + px] = d;
                    if (COUNT) {
                        it += d;
                        ++lpx;
                    }
                }
            }
        }
    }
    if (COUNT) {
        it = warp_sum_u64(it);
        lpx = warp_sum_u64(lpx);
        if ((tid & 31u) == 0u) {
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
int resident_grid(K kernel, int threads, int sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

template <bool COUNT, bool MBR>
void region_level_launch(const LevelArgs &a, uint32_t threads, int sms, cudaStream_t s)
{
    const int grid = resident_grid(region_level_kernel<COUNT, MBR>, (int)threads, sms);
    region_level_kernel<COUNT, MBR><<<grid, threads, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_level_region(const LevelArgs &a, bool mbr, bool count, uint32_t threads, int sms,
                                cudaStream_t s)
{
    if (threads < 32u || threads > 1024u || threads % 32u != 0u)
        return cudaErrorInvalidValue;
    if (mbr) {
        if (count)
            region_level_launch<true, true>(a, threads, sms, s);
        else
            region_level_launch<false, true>(a, threads, sms, s);
    } else {
        if (count)
            region_level_launch<true, false>(a, threads, sms, s);
        else
            region_level_launch<false, false>(a, threads, sms, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_leaf_region(const LeafArgs &a, uint32_t bx, uint32_t by, bool count, int sms,
                               cudaStream_t s)
{
    const dim3 block(bx, by);
    const int threads = (int)(bx * by);
    if (count) {
        const int grid = resident_grid(region_leaf_kernel<true>, threads, sms);
        region_leaf_kernel<true><<<grid, block, 0, s>>>(a);
    } else {
        const int grid = resident_grid(region_leaf_kernel<false>, threads, sms);
        region_leaf_kernel<false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ask
