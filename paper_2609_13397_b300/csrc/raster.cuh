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

}  // namespace conegs
