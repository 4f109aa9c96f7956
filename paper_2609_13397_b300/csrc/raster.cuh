// Arguments of the tile rasteriser and its adjoint, and per-pixel ray loads.
#pragma once
#include "pair.cuh"

namespace conegs {

struct RasterArgs {
    int W, H, tiles_x;
    const uint2 *ranges;
    const uint32_t *gids;
    const float4 *rec;
    const float *d, *dx, *dy;
    const uint8_t *valid;
    float *out_rgb, *out_T, *keep_T;   // keep_T: copy of the final T kept for the adjoint (may be NULL)
    uint32_t *last;        // per pixel: list entries up to and including the last contributor
    unsigned long long *evaluated;   // optional (profiling): [0] list entries walked, [1] full evaluations
    int additive;
};

__device__ __forceinline__ void load_pixel(const RasterArgs &a, int64_t pix, int64_t P, PixelRays &px) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        px.d[k] = a.d[k * P + pix];
        px.dx[k] = a.dx[k * P + pix];
        px.dy[k] = a.dy[k * P + pix];
    }
    px.d_dx = dot3(px.d, px.dx);
    px.d_dy = dot3(px.d, px.dy);
    px.dxdx = dot3(px.dx, px.dx);
    px.dxdy = dot3(px.dx, px.dy);
    px.dydy = dot3(px.dy, px.dy);
}

// ---------------------------------------------------------------- long-list split (forward and adjoint)

constexpr uint32_t SEG_MIN = 256;
constexpr uint32_t CTA_SLOTS = 148 * 16;   // resident 64-thread raster CTAs on a B300
constexpr uint32_t NO_STOP = 0xffffffffu;

struct SegArgs {
    const unsigned long long *stat;   // [0] non-empty tiles, [1] total list length -> segment length
    const uint32_t *nseg, *seg_off;   // per tile: segment count, first item
    const uint2 *work;      // (tile, segment >= 1)
    const uint32_t *total;  // number of such items
    float4 *seg_c;          // [item][TILE_PX]: pass A: C0, C1, C2, T_seg of the local walk;
                            //   after the merge and replay: the segment's share of C and T after it;
                            //   after the suffix pass: colour composited behind the segment, T after it
    uint32_t *seg_l;        // [item][TILE_PX]: last contributor (local, 1-based; 0 none) | stopped << 31
    uint32_t *seg_all;      // [item]: 1 if every pixel of the tile stopped inside this segment
    uint32_t *need_item;    // [item]: 1 if some pixel's walk stops inside this segment (replay it)
    float4 *rp_c;           // [tile][TILE_PX]: C0, C1, C2, T_in entering the stop segment
    uint32_t *rp_need;      // [tile][TILE_PX]: the stop segment to replay (NO_STOP: none)
    uint32_t *rp_last;      // [tile][TILE_PX]: last contributor before it (1-based in the tile list)
    uint32_t *rp_end;       // [tile][TILE_PX]: last segment the pixel's walk reaches (NO_STOP: not rendered)
};

// Segment length L: with fewer non-empty tiles than two per resident CTA,
// about two segments per resident CTA (at least 256 entries); otherwise 4x the
// mean non-empty list (rounded up), so that only tail lists split.  Either way
// the segment count stays below ntiles + max(2 CTA_SLOTS, ntiles / 4) + 1.
static __device__ __forceinline__ uint32_t seg_length_dev(const unsigned long long *stat) {
    const unsigned long long ne = stat[0] > 0 ? stat[0] : 1, tot = stat[1];
    unsigned long long s;
    if (ne < 2ull * CTA_SLOTS) {
        s = (tot + 2ull * CTA_SLOTS - 1) / (2ull * CTA_SLOTS);
        s = (s + TILE_PX - 1) / TILE_PX * TILE_PX;
    } else {
        s = (4ull * tot + ne - 1) / ne;
    }
    if (s < SEG_MIN) s = SEG_MIN;
    return (uint32_t)(s < 0x7fffffffull ? s : 0x7fffffffull);
}

// The split state of a view with ntiles tiles inside its scratch buffer
// (split_scratch_words(ntiles) words); *items: the item bound (grid size).
SegArgs split_args(uint32_t *scratch, int ntiles, int64_t *items);
int64_t split_scratch_words(int ntiles);

}  // namespace conegs
