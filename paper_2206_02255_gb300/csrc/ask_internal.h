// ask_internal.h -- declarations shared by the library's translation units
// (host driver, ASK/exhaustive kernels, CDP2 kernels).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ask.h"

namespace ask {

// Pixel -> c mapping, computed on the host once per render:
// cr = fma(px, dx, re_min), ci = fma(py, dy, im_min).
struct PixelMap {
    float re_min, im_min, dx, dy;
};

// Device-resident counters of one render.  Zeroed by the init kernel.
struct DevCounters {
    uint32_t count[ASK_MAX_LEVELS + 1];     // entries in the region table of level i
    uint32_t fills[ASK_MAX_LEVELS];         // uniform regions filled at level i
    uint32_t subdivs[ASK_MAX_LEVELS];       // regions split at level i
    uint32_t leaf_count;                    // leaf-list entries from the front (all of them,
                                            // where the producer does not order its leaves)
    uint32_t error;                         // ERR_* bits, latched
    unsigned long long iterations;          // COUNT mode: z-updates
    unsigned long long fill_pixels;         // COUNT mode
    unsigned long long leaf_pixels;         // COUNT mode
    unsigned long long border_pixels;       // COUNT mode
    unsigned long long level_iters[ASK_MAX_LEVELS];  // COUNT mode: z-updates of level i
    unsigned long long leaf_iters;          // COUNT mode: z-updates of the leaf kernel
    unsigned long long deferred_fill_pixels; // COUNT mode: pixels of the deferred-fill list
    uint32_t work[ASK_MAX_LEVELS];          // next work item a level kernel hands out
    uint32_t leaf_work;                     // next leaf the leaf kernel hands out
    uint32_t fill_count;                    // bands in the deferred-fill list
    uint32_t fill_work;                     // next band the leaf kernel's fill warps take
    uint32_t leaf_light;                    // leaf-list entries from the back (level kernels:
                                            // leaves whose probe escaped, taken last)
    uint32_t back[ASK_MAX_LEVELS + 1];      // region-table entries of level i written from the
                                            // back (count[i] holds those from the front)
};

enum : uint32_t {
    ERR_OLT_OVERFLOW = 1u,
    ERR_LEAF_OVERFLOW = 2u,
    ERR_DEVICE_LAUNCH = 4u,
    ERR_DEPTH = 8u,
    ERR_TIMEOUT = 16u,  // a bounded wait of the persistent batch kernel gave up
};

// One level of the subdivision plan.
struct LevelPlan {
    uint32_t levels;                        // number of level kernels
    uint32_t side[ASK_MAX_LEVELS];          // nominal region side at level i
    uint32_t split[ASK_MAX_LEVELS];         // 1 if non-uniform regions of level i split
    uint64_t max_regions[ASK_MAX_LEVELS];   // upper bound on regions at level i
    uint32_t chunks[ASK_MAX_LEVELS];        // perimeter chunks per region (work items)
    uint32_t chunk_px[ASK_MAX_LEVELS];      // perimeter pixels per chunk
    uint32_t axis0;                         // non-empty initial regions per axis
};

// A level with fewer work items than this at chunk_px pixels a chunk takes
// chunks of half that size: its items are too few to keep every warp busy,
// and the kernel's time is set by its longest items (chunks of a region
// inside the set run max_dwell updates per pixel, one pixel per lane after
// another).
constexpr uint64_t kFewLevelItems = 32768;

// Fills `plan`; returns false if the parameters are invalid or a level could
// hold 2^32 regions or more.
// chunk_px: perimeter pixels per work item of the level kernels (chunks[i]);
// few_items: levels with fewer items take chunks of chunk_px / 2 (0: never).
bool make_plan(uint32_t n, uint32_t g, uint32_t r, uint32_t B, LevelPlan *plan, uint32_t chunk_px = 64,
               uint64_t few_items = kFewLevelItems);

// Launch configuration chosen per device at context creation.
struct DeviceInfo {
    int device;
    int sms;
    int cc_major, cc_minor;
};

// ---- kernels of ask_kernels.cu -------------------------------------------
cudaError_t launch_exhaustive(uint32_t *map, uint32_t n, PixelMap pm, uint32_t max_dwell,
                              uint32_t bx, uint32_t by, bool count, DevCounters *ctr,
                              cudaStream_t s);
// Zero the counters (except the latched error word) and, if olt0 is set,
// write the initial regions of initial-region rows [row0, row0 + rows) of the
// axis0 x axis0 grid of side s0 (count[0] = axis0 * rows).  With `order`
// (the frame's pixel map) and at most kInitOrderMax regions, the regions
// whose centre orbit stays bounded for a probe's updates fill the table from
// the front (count[0]) and the others from the back (back[0]), so the level
// kernel takes the long ones first.
constexpr uint32_t kInitOrderMax = 4096;
cudaError_t launch_init(uint2 *olt0, uint4 *rst0, DevCounters *ctr, uint32_t n, uint32_t s0,
                        uint32_t axis0, uint32_t row0, uint32_t rows, cudaStream_t s,
                        const PixelMap *order = nullptr);

// One frame of a batch, resident on the device.  Region records of a batch
// are uint4 {x0 | y0 << 16, (w-1) | (h-1) << 16, frame, 0}.
struct FrameDesc {
    uint32_t *map;        // the frame's output map
    PixelMap pm;
    uint32_t n, max_dwell, r, levels;
    uint32_t s0, axis0;   // level-0 side and non-empty regions per axis
    uint32_t olt0_offset; // first level-0 record of this frame
    uint32_t pad_;
    uint32_t side[ASK_MAX_LEVELS];  // region side at each level
    // persistent batch kernel (ask_queue.cu) only
    uint32_t item0;       // first level-0 queue item of this frame
    uint32_t state0;      // first level-0 chunk state of this frame
    uint32_t chunks[ASK_MAX_LEVELS];  // perimeter chunks (queue items) per region at each level
};

struct LevelArgs {
    // single frame (ignored by batch launches, which read the frame table)
    uint32_t *map;
    uint32_t n;
    PixelMap pm;
    uint32_t max_dwell;
    uint32_t side;        // nominal side of this level's regions
    uint32_t split;       // non-uniform regions split (else become leaves)
    uint32_t child_side;  // ceil(side / r)
    uint32_t r;
    // both
    uint32_t level;
    const void *olt_in;   // uint2 records (single frame) or uint4 records (batch)
    void *olt_out;
    uint32_t olt_cap;     // capacity of both region tables
    uint32_t in_cap;      // bound on this level's regions (<= olt_cap): olt_in holds
                          //   count[level] entries from slot 0 up and back[level] from
                          //   slot in_cap - 1 down
    uint32_t out_cap;     // the same bound for the next level's table (olt_out, rst_out)
    uint32_t chunks;      // perimeter chunks per region at this level (1 = one warp per region)
    uint32_t chunk_px;    // perimeter pixels per chunk (one frame; a batch derives its own)
    uint32_t next_chunks; // chunks per region at the next level
    uint4 *rst_in;        // per-region query state of this level (chunks > 1)
    uint4 *rst_out;       // state of the next level's regions, set when they are appended
    void *leaves;         // leaf records, same type as the region records
    uint32_t leaf_cap;
    uint4 *fills;         // deferred fills (region, dwell, frame); NULL = fill in place
    uint32_t fill_cap;
    uint32_t exact_last;  // last level: evaluate whole perimeters and write them
    const FrameDesc *frames;  // batch: the frame table
    DevCounters *ctr;
};
// Perimeter pixels per work item of a level kernel: one frame's top levels
// have few regions and need the parallelism of small chunks; a batch has
// regions enough, and there a chunk's fixed cost weighs more.
constexpr uint32_t kChunkPx = 64;
constexpr uint32_t kChunkPxBatch = 128;
// A batch splits every region of a level into the same number of chunks (the
// work items are region x chunk), at most kMaxChunksBatch; a region whose
// perimeter exceeds that many kChunkPxBatch chunks takes longer chunks.  The
// cap keeps one frame with huge regions from multiplying the work items of
// every other frame.
constexpr uint32_t kMaxChunksBatch = 8;
// Uniform regions larger than this are filled by the fill kernel.
constexpr uint32_t kInPlaceFillArea = 16384;
// The fill kernel's list holds bands of whole rows of a uniform region, at
// most kFillBandPx pixels each (one row if the region is wider), so its work
// items are of near-equal size whatever the regions' sizes.
constexpr uint32_t kFillBandPx = 16384;
__host__ __device__ inline uint32_t fill_band_rows(uint32_t w)
{
    return w >= kFillBandPx ? 1u : kFillBandPx / w;
}
__host__ __device__ inline uint32_t fill_band_count(uint32_t w, uint32_t h)
{
    const uint32_t rows = fill_band_rows(w);
    return h / rows + (h % rows != 0u);
}
cudaError_t launch_level(const LevelArgs &a, bool count, bool batch, int sms, cudaStream_t s);

struct FillArgs {
    uint32_t *map;        // single frame (batch entries name their frame)
    uint32_t n;
    const uint4 *fills;   // bands (origin, extent, dwell, frame)
    uint32_t fill_cap;
    const FrameDesc *frames;
    DevCounters *ctr;
};
// One resident wave of 256-thread CTAs over all SMs.
cudaError_t launch_fill(const FillArgs &f, bool batch, int sms, cudaStream_t s);
cudaError_t launch_init_batch(uint4 *olt0, uint4 *rst0, DevCounters *ctr, const FrameDesc *frames,
                              uint32_t nframes, uint32_t total0, cudaStream_t s);

struct LeafArgs {
    // single frame (ignored by batch launches)
    uint32_t *map;
    uint32_t n;
    PixelMap pm;
    uint32_t max_dwell;
    uint32_t side;        // nominal side of the leaf regions
    // both
    const void *leaves;   // uint2 (single frame) or uint4 (batch) records
    uint32_t leaf_cap;    // capacity of the leaf list
    uint32_t skip_perimeter;  // leaf perimeters are already in the map
    const uint4 *fills;   // lane-refill kernel: deferred-fill bands to write
    uint32_t fill_cap;    //   along the way (NULL: none)
    const FrameDesc *frames;
    DevCounters *ctr;
};
// tiled = false: lane-refill kernel (default); true: one thread per pixel in
// block_x x block_y tiles (single frame only)
cudaError_t launch_leaf(const LeafArgs &a, uint32_t bx, uint32_t by, bool count, bool tiled,
                        bool batch, int sms, cudaStream_t s);

// ---- the persistent batch kernel of ask_queue.cu -------------------------
// Queue state of one render, next to its items.  `epoch` survives between
// renders (the render's items carry epoch + 1); the init kernel resets the
// rest.
struct QueueState {
    uint32_t epoch;      // epoch of the last finished render
    uint32_t head;       // next region ticket
    uint32_t tail;       // queue slots reserved
    uint32_t pending;    // items pushed and not yet finished
    uint32_t done;       // = the render's epoch once pending reached 0
    uint32_t states;     // chunk-query states handed out
    uint32_t leaf_head;  // next leaf ticket
    uint32_t exited;     // warps that have left the persistent kernel
};

struct QueueArgs {
    uint4 *items;         // {origin, extent, tag, epoch}: tag = frame | level << 20 | kind << 25 | chunk << 26
    uint32_t *aux;        // per item: chunk-state index (region) or dwell (fill band)
    uint32_t item_cap;
    uint4 *rst;           // chunk-query states {common dwell, differs, chunks done, -}
    uint32_t rst_cap;
    uint4 *leaves;        // leaf list {origin, extent, frame, epoch}
    uint32_t leaf_cap;
    const FrameDesc *frames;
    DevCounters *ctr;
    QueueState *qs;
    uint32_t regions0;    // level-0 regions of all frames
    uint32_t total0;      // level-0 items of all frames
    uint32_t states0;     // level-0 chunk states of all frames
    uint32_t chunk_px;    // perimeter pixels per chunk item (a region's last chunks may be longer)
    uint32_t wait_limit;  // idle polls in a row before a warp reports ERR_TIMEOUT
};
// Perimeter pixels per chunk item and the most chunk items per region of the
// persistent batch kernel (a region whose perimeter needs more takes longer
// chunks; the tag has 6 bits for the chunk).
constexpr uint32_t kChunkPxQueue = 128;
constexpr uint32_t kMaxChunksQueue = 16;
// Idle polls in a row (with __nanosleep back-off of up to 256 ns, reset
// whenever the queue or the leaf list moves) before a warp gives up.
constexpr uint32_t kQueueWaitLimit = 1u << 26;
// Init kernel (one block per frame) and the persistent kernel, on `s`.
cudaError_t launch_queue(const QueueArgs &q, uint32_t nframes, bool count, int sms, cudaStream_t s);

// ---- kernels of ask_cdp2.cu ----------------------------------------------
struct CdpArgs {
    uint32_t *map;
    uint32_t n;
    PixelMap pm;
    uint32_t max_dwell;
    uint32_t r, B;
    uint32_t count;       // ASK_FLAG_COUNT
    uint32_t fire_and_forget;  // children into cudaStreamFireAndForget, not the tail stream
    uint32_t mbr;              // DP-MBR: fills and leaf pixels by child grids
    // tail launches without MBR: the regions a grid splits into are appended
    // to list[(level + 1) & 1] and the grid's last CTA tail-launches one grid
    // over all of them
    uint2 *list[2];
    uint32_t list_cap;
    DevCounters *ctr;
};
cudaError_t launch_cdp2(const CdpArgs &a, uint32_t g, uint32_t s0, uint32_t bx, uint32_t by,
                        cudaStream_t s);
cudaError_t cdp2_set_pending_limit(size_t launches);

// The paper's SBR / MBR mappings of ASK (Sec. 4.3.1-4.3.2), ask_schemes.cu.
// One CTA of `threads` threads per region for the query and the split;
// mbr = 0 fills in place, mbr = 1 appends uniform regions to the fill list.
cudaError_t launch_level_region(const LevelArgs &a, bool mbr, bool count, uint32_t threads, int sms,
                                cudaStream_t s);
// SBR last level: one CTA (bx x by threads) per leaf region.
cudaError_t launch_leaf_region(const LeafArgs &a, uint32_t bx, uint32_t by, bool count, int sms,
                               cudaStream_t s);

}  // namespace ask
