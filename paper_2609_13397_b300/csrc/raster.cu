// K5: tile rasteriser, forward (Sec. 3 Eq. 4 compositing over Eq. 9 responses).
//
// One CTA of 64 threads per 8x8 tile, one thread per pixel.  The tile's
// depth-sorted Gaussian list is walked in batches of 64: each thread loads
// one Gaussian's 80-byte record (5 x float4, coalesced gather) into shared
// memory, then every thread evaluates the whole batch against its pixel's
// rays from registers.  Compositing follows the 3DGS conventions: a =
// min(0.99, T); pairs with a < 1/255 are skipped; a pixel stops before the
// pair that would take its transmittance below 1e-4; the CTA leaves the
// list as soon as all its pixels have stopped (__syncthreads_count).
// Per pixel the kernel writes rgb, the final transmittance and the number of
// list entries walked up to the last contributing pair (for the adjoint).
#include "raster.cuh"

namespace conegs {

template <bool FILTER>
__global__ void __launch_bounds__(TILE_PX) raster_fwd_kernel(const RasterArgs a) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const bool inside = i < a.W && j < a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    PixelRays px;
    bool done = true;
    if (inside && a.valid[pix]) {
        load_pixel(a, pix, P, px);
        done = false;
    }
    const uint2 range = a.ranges[tile];
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tacc = 1.0f;
    uint32_t last = 0, walked = 0, full = 0;
    for (uint32_t start = range.x; start < range.y; start += TILE_PX) {
        if (__syncthreads_count(done) == TILE_PX) break;
        const uint32_t idx = start + threadIdx.x;
        if (idx < range.y) {
            const float4 *r = a.rec + (size_t)REC_F4 * a.gids[idx];
#pragma unroll
            for (int k = 0; k < REC_F4; ++k) s_rec[k][threadIdx.x] = r[k];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)TILE_PX, range.y - start);
        // phase 1: cone pre-test of every staged entry against this pixel (the
        // shared-memory reads are broadcasts: all lanes read the same entry)
        unsigned long long mask = 0ull;
        if (!done) {
            walked += (uint32_t)nb;
            for (int b = 0; b < nb; ++b) {
                const float4 r4 = s_rec[4][b], r5 = s_rec[5][b], r6 = s_rec[6][b];
                const float e0 = px.d[0] - r4.x, e1 = px.d[1] - r4.y, e2 = px.d[2] - r4.z;
                const float qa = r5.z * e0 + r6.y * e1 + r6.z * e2;
                const float qb = r5.w * e1 + r6.w * e2;
                const float cone = -1.0f + r4.w * e0 + r5.x * e1 + r5.y * e2 + qa * e0 + qb * e1 + r6.x * e2 * e2;
                if (!(cone > 1e-3f)) mask |= 1ull << b;
            }
        }
        // phase 2: each lane walks its own passing entries in depth order, so
        // the warp's lanes evaluate different entries in lockstep
        while (__any_sync(0xffffffffu, mask != 0ull)) {
            if (mask != 0ull) {
                const int b = __ffsll((long long)mask) - 1;
                mask &= mask - 1ull;
                ++full;
                const float4 r3 = s_rec[3][b];
                float T;
                if (pair_response<FILTER>(s_rec[0][b], s_rec[1][b], s_rec[2][b], r3.w, s_rec[7][b].x,
                                          a.additive != 0, px, T)) {
                    const float alpha = fminf(ALPHA_MAX, T);
                    if (!(alpha < ALPHA_MIN)) {
                        const float test = Tacc * (1.0f - alpha);
                        if (test < T_STOP) {
                            done = true;
                            mask = 0ull;
                        } else {
                            const float w = alpha * Tacc;
                            C0 += r3.x * w;
                            C1 += r3.y * w;
                            C2 += r3.z * w;
                            Tacc = test;
                            last = start - range.x + (uint32_t)b + 1u;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (a.evaluated) {
        unsigned long long w = walked, f = full;
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, o);
            f += __shfl_xor_sync(0xffffffffu, f, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.evaluated, w);
            atomicAdd(a.evaluated + 1, f);
        }
    }
    if (inside) {
        a.out_rgb[pix] = C0;
        a.out_rgb[P + pix] = C1;
        a.out_rgb[2 * P + pix] = C2;
        if (a.out_T) a.out_T[pix] = Tacc;
        if (a.keep_T) a.keep_T[pix] = Tacc;
        if (a.last) a.last[pix] = last;
    }
}

cudaError_t launch_raster_fwd(const RasterArgs &a, int ntiles, bool filter, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    if (filter)
        raster_fwd_kernel<true><<<ntiles, TILE_PX, 0, s>>>(a);
    else
        raster_fwd_kernel<false><<<ntiles, TILE_PX, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
