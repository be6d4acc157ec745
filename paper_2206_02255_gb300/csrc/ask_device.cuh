// ask_device.cuh -- device helpers shared by the exhaustive, ASK and CDP2
// kernels: the per-pixel dwell, the pixel -> c mapping, region records,
// perimeter enumeration and vectorised fills.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_internal.h"

namespace ask {

// Iterations per escape check block in dwell(); see the comment there.
constexpr int kUnroll = 16;

__device__ __forceinline__ float2 pixel_c(const PixelMap &pm, uint32_t px, uint32_t py)
{
    return make_float2(__fmaf_rn(__uint2float_rn(px), pm.dx, pm.re_min),
                       __fmaf_rn(__uint2float_rn(py), pm.dy, pm.im_min));
}

// Dwell of c (paper Sec. 6): the number of updates z <- z^2 + c, from z = 0,
// made while |z|^2 < 4, at most max_dwell.  One iteration is
//   zi2 = zi*zi; m = fma(zr, zr, zi2)          (the escape test on m)
//   zr' = fma(zr, zr, fma(-zi, zi, cr)); zi' = fma(zr + zr, zi, ci)
// with every operation rounded once (the _rn intrinsics are never fused or
// reassociated by the compiler).
//
// To keep the FP32 pipe busy, iterations run in blocks of kUnroll with the
// escape tests OR-ed into one predicate and a single branch per block; a
// block whose predicate fired is rolled back to its saved start and replayed
// one checked step at a time, so the result is exactly the stepwise count.
__device__ __forceinline__ uint32_t dwell(float cr, float ci, uint32_t max_dwell)
{
    float x = 0.0f, y = 0.0f;
    uint32_t d = 0;
    while (max_dwell - d >= (uint32_t)kUnroll) {
        const float sx = x, sy = y;
        bool out = false;
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const float y2 = __fmul_rn(y, y);
            const float m = __fmaf_rn(x, x, y2);
            out |= !(m < 4.0f);
            const float t = __fmaf_rn(-y, y, cr);
            const float nx = __fmaf_rn(x, x, t);
            const float ny = __fmaf_rn(__fadd_rn(x, x), y, ci);
            x = nx;
            y = ny;
        }
        if (out) {
            x = sx;
            y = sy;
            break;
        }
        d += (uint32_t)kUnroll;
    }
    while (d < max_dwell) {
        const float y2 = __fmul_rn(y, y);
        const float m = __fmaf_rn(x, x, y2);
        if (!(m < 4.0f))
            break;
        const float t = __fmaf_rn(-y, y, cr);
        const float nx = __fmaf_rn(x, x, t);
        const float ny = __fmaf_rn(__fadd_rn(x, x), y, ci);
        x = nx;
        y = ny;
        ++d;
    }
    return d;
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
    const uint32_t chunks_per_row = (g.w + 3u) / 4u + 1u;  // upper bound for any alignment
    const uint32_t items = chunks_per_row * g.h;
    const uint4 v4 = make_uint4(v, v, v, v);
    for (uint32_t it = t; it < items; it += nthr) {
        const uint32_t row = it / chunks_per_row, c = it - row * chunks_per_row;
        const size_t start = (size_t)(g.y0 + row) * n + g.x0;
        const size_t end = start + g.w;
        const size_t e0 = ((start >> 2) + c) << 2;
        if (e0 >= end)
            continue;
        if (e0 >= start && e0 + 4u <= end) {
            *reinterpret_cast<uint4 *>(map + e0) = v4;
        } else {
#pragma unroll
            for (uint32_t k = 0; k < 4u; ++k)
                if (e0 + k >= start && e0 + k < end)
                    map[e0 + k] = v;
        }
    }
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
