// ask_fp64.h -- declarations of the deep-zoom kernels of ask_fp64.cu
// (binary64 or float-float), used by the host driver.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ask_internal.h"

namespace ask {

// Pixel -> c mapping in double: cr = fma(px, dx, re_min), ci = fma(py, dy,
// im_min) with dx = (re_max - re_min) / n computed in double on the host.
struct PixelMap64 {
    double re_min, im_min, dx, dy;
};

// One level of the double-precision ASK pipeline (one frame, whole-region
// work items: one warp per region).
struct Level64Args {
    uint32_t *map;
    uint32_t n;
    PixelMap64 pm;
    uint32_t max_dwell;
    uint32_t level;
    uint32_t split;       // non-uniform regions split (else become leaves)
    uint32_t child_side;  // ceil(side / r)
    uint32_t r;
    const uint2 *olt_in;
    uint2 *olt_out;
    uint32_t olt_cap;
    uint2 *leaves;
    uint32_t leaf_cap;
    DevCounters *ctr;
};

struct Leaf64Args {
    uint32_t *map;
    uint32_t n;
    PixelMap64 pm;
    uint32_t max_dwell;
    const uint2 *leaves;
    uint32_t leaf_cap;
    DevCounters *ctr;
};

// count: accumulate z-updates (and pixel counts) in the counters, as
// ASK_FLAG_COUNT does for the single-precision kernels.  ff: float-float
// arithmetic instead of binary64.
cudaError_t launch_exhaustive64(uint32_t *map, uint32_t n, PixelMap64 pm, uint32_t max_dwell,
                                uint32_t bx, uint32_t by, bool count, bool ff, DevCounters *ctr,
                                cudaStream_t s);
cudaError_t launch_level64(const Level64Args &a, bool count, bool ff, int sms, cudaStream_t s);
cudaError_t launch_leaf64(const Leaf64Args &a, bool count, bool ff, int sms, cudaStream_t s);

}  // namespace ask
