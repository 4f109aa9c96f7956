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
    unsigned long long *evaluated;   // optional (profiling): [0] list entries walked, [1] full evaluations,
                                     // [2] of those, flat (FP64) evaluations
    // flat Gaussians (records marked flat, see pair.cuh): their pairs' responses, in
    // FP64, come from flat_pairs_kernel: list entry k -> slot flat_slot[k], response
    // flat_T[slot * TILE_PX + pixel in tile] (-1: t* <= T_NEAR, skipped); with the
    // adjoint state, flat_G[(slot * 13 + j) * TILE_PX + pixel] = dT / d(record j)
    // (W_eff 9, o_u 3, sigma_eff).  NULL when the view has no flat Gaussian.
    const uint32_t *flat_slot;
    const float *flat_T, *flat_G;
    int additive;
    int pixtest;           // 1: the records hold the pinhole (pixel-space) pre-test
    int footprint;         // 0: the pixel's own differentials; 1: isotropic reduction; 2: z/f sizing
    float zax[3];          // z/f: optical axis (world); zf_scale = 1 / (2 f_x)
    float zf_scale;
};

constexpr int FOOTPRINT_OWN = 0, FOOTPRINT_ISO = 1, FOOTPRINT_ZF = 2;

// Isotropic footprint variants: the half-edge differentials become a b1, a b2
// with (b1, b2) orthonormal across d (b1 from the coordinate axis least aligned
// with d), a^2 = (|dx_perp|^2 + |dy_perp|^2) / 2 (ISO) or a = |<d, z_cam>| / (2 f_x) (ZF).
__device__ __forceinline__ void isotropic_differentials(const RasterArgs &a, PixelRays &px) {
    const float *d = px.d;
    float s2;
    if (a.footprint == FOOTPRINT_ISO) {
        const float sx = dot3(d, px.dx), sy = dot3(d, px.dy);
        float n2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float ux = px.dx[k] - sx * d[k], uy = px.dy[k] - sy * d[k];
            n2 += ux * ux + uy * uy;
        }
        s2 = 0.5f * n2;
    } else {
        const float z = d[0] * a.zax[0] + d[1] * a.zax[1] + d[2] * a.zax[2];
        s2 = (z * a.zf_scale) * (z * a.zf_scale);
    }
    const float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    float b1[3] = {0.f, 0.f, 0.f};
    if (ax <= ay && ax <= az) b1[0] = 1.f; else if (ay <= az) b1[1] = 1.f; else b1[2] = 1.f;
    const float s = dot3(b1, d);
#pragma unroll
    for (int k = 0; k < 3; ++k) b1[k] -= s * d[k];
    const float rn = rsqrtf(dot3(b1, b1));
    const float am = sqrtf(s2);
#pragma unroll
    for (int k = 0; k < 3; ++k) b1[k] *= rn;
    px.dx[0] = am * b1[0]; px.dx[1] = am * b1[1]; px.dx[2] = am * b1[2];
    px.dy[0] = am * (d[1] * b1[2] - d[2] * b1[1]);
    px.dy[1] = am * (d[2] * b1[0] - d[0] * b1[2]);
    px.dy[2] = am * (d[0] * b1[1] - d[1] * b1[0]);
}

__device__ __forceinline__ void load_pixel(const RasterArgs &a, int64_t pix, int64_t P, PixelRays &px) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        px.d[k] = a.d[k * P + pix];
        px.dx[k] = a.dx[k * P + pix];
        px.dy[k] = a.dy[k * P + pix];
    }
    if (a.footprint != FOOTPRINT_OWN) isotropic_differentials(a, px);
    px.d_dx = dot3(px.d, px.dx);
    px.d_dy = dot3(px.d, px.dy);
    px.dxdx = dot3(px.dx, px.dx);
    px.dxdy = dot3(px.dx, px.dy);
    px.dydy = dot3(px.dy, px.dy);
    const uint32_t p32 = (uint32_t)pix, w32 = (uint32_t)a.W;
    px.pc[0] = (float)(p32 % w32) + 0.5f;
    px.pc[1] = (float)(p32 / w32) + 0.5f;
}

// ---------------------------------------------------------------- long-list split (forward and adjoint)

constexpr uint32_t SEG_MIN = 256;
constexpr uint32_t NO_STOP = 0xffffffffu;

// Resident raster CTAs on the device (SMs x CTAs per SM of the forward raster
// kernel), the unit of the long-list split; queried once per device.
uint32_t raster_slots();

struct SegArgs {
    uint32_t slots;                   // raster_slots() of the device
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
// the segment count stays below ntiles + max(2 slots, ntiles / 4) + 1, the
// bound split_items_max sizes the split state with: a shorter L (more segments
// per resident CTA) must raise that bound with it, or the passes write past
// the state.
static __device__ __forceinline__ uint32_t seg_length_dev(const unsigned long long *stat, uint32_t slots) {
    const unsigned long long ne = stat[0] > 0 ? stat[0] : 1, tot = stat[1];
    unsigned long long s;
    if (ne < 2ull * slots) {
        s = (tot + 2ull * slots - 1) / (2ull * slots);
        s = (s + TILE_PX - 1) / TILE_PX * TILE_PX;
    } else {
        s = (4ull * tot + ne - 1) / ne;
    }
    if (s < SEG_MIN) s = SEG_MIN;
    return (uint32_t)(s < 0x7fffffffull ? s : 0x7fffffffull);
}
static __device__ __forceinline__ uint32_t seg_length_dev(const SegArgs &g) { return seg_length_dev(g.stat, g.slots); }

// The split state of a view with ntiles tiles inside its scratch buffer
// (split_scratch_words(ntiles) words); *items: the item bound (grid size).
SegArgs split_args(uint32_t *scratch, int ntiles, int64_t *items);
int64_t split_scratch_words(int ntiles);

}  // namespace conegs
