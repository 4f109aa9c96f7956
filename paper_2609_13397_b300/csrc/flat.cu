// FP64 responses of the pairs of near-degenerate flat Gaussians (pair.cuh:
// effective scale ratio above FLAT_RATIO), precomputed for the rasteriser and
// its adjoint.
//
// The FP32 raster kernels stay as they are for every other pair: the FP64
// evaluation needs about twice their registers, and a few flat Gaussians in a
// view would otherwise halve the occupancy of the whole render.  Here each
// tile-list entry whose Gaussian is flat gets a slot; one CTA per slot
// evaluates Eq. 2-12 and Eq. 9 in FP64 (pair_response<.., double>) for the 64
// pixels of the entry's tile, and, when the adjoint will run, the derivatives
// dT/d(W_eff, o_u, sigma_eff) at dL/dT = 1 (pair_adjoint<.., double>; every
// term of the adjoint is linear in dL/dT, so the adjoint walk scales them).
// The raster kernels read the response where they would have computed it, in
// list order, so compositing and its thresholds see the FP64 value.
#include "adjoint.cuh"
#include "raster.cuh"

namespace conegs {

// One slot per list entry whose Gaussian is flat (any order).
__global__ void assign_flat_slots_kernel(const uint32_t *__restrict__ gids, int64_t npairs,
                                         const uint8_t *__restrict__ gflat, uint32_t *__restrict__ slot_of,
                                         uint32_t *__restrict__ slot_pair, unsigned long long *__restrict__ counter) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs || gflat[gids[p]] == 0) return;
    const uint32_t s = (uint32_t)atomicAdd(counter, 1ull);
    slot_of[p] = s;
    slot_pair[s] = (uint32_t)p;
}

// One CTA per slot, one thread per pixel of the entry's tile.
template <bool FILTER, bool ADJ>
__global__ void __launch_bounds__(TILE_PX) flat_pairs_kernel(const RasterArgs a, const uint32_t *__restrict__ tiles,
                                                             const uint32_t *__restrict__ slot_pair,
                                                             float *__restrict__ flat_T, float *__restrict__ flat_G) {
    const size_t slot = blockIdx.x;
    const uint32_t p = slot_pair[slot];
    const int tile = (int)tiles[p];
    const float4 *r = a.rec + (size_t)REC_F4 * a.gids[p];
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    float T = -1.0f;
    float gW[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gou[3] = {0.f, 0.f, 0.f}, gsig = 0.f;
    if (i < a.W && j < a.H && a.valid[pix]) {
        PixelRays px32;
        load_pixel(a, pix, P, px32);
        const PixelRaysT<double> px = widen(px32);
        const GaussRec<double> g = rec_f64(r[0], r[1], r[2], r[3].w, r[7]);
        if (ADJ) {
            PairFwdT<double> f;
            float Tp;
            if (pair_response<FILTER, true, double>(g, a.additive != 0, px, Tp, &f)) {
                T = Tp;
                gsig = pair_adjoint<FILTER, double>(f, g, px, 1.0f, gW, gou);
            }
        } else {
            float Tp;
            if (pair_response<FILTER, false, double>(g, a.additive != 0, px, Tp)) T = Tp;
        }
    }
    flat_T[slot * TILE_PX + threadIdx.x] = T;
    if (ADJ) {
        float *gd = flat_G + slot * 13 * TILE_PX + threadIdx.x;
#pragma unroll
        for (int k = 0; k < 9; ++k) gd[k * TILE_PX] = gW[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) gd[(9 + k) * TILE_PX] = gou[k];
        gd[12 * TILE_PX] = gsig;
    }
}

// nslots: the number of list entries whose Gaussian is flat (known on the host
// from the count pass); counter: one zeroed word of scratch.
cudaError_t launch_flat_pairs(const RasterArgs &a, const uint32_t *tiles, int64_t npairs, const uint8_t *gflat,
                              uint32_t *slot_of, uint32_t *slot_pair, unsigned long long *counter, int64_t nslots,
                              float *flat_T, float *flat_G, bool filter, cudaStream_t s) {
    if (nslots == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    assign_flat_slots_kernel<<<(unsigned)div_up(npairs, 256), 256, 0, s>>>(a.gids, npairs, gflat, slot_of, slot_pair,
                                                                         counter);
    const unsigned grid = (unsigned)nslots;
    if (filter) {
        if (flat_G)
            flat_pairs_kernel<true, true><<<grid, TILE_PX, 0, s>>>(a, tiles, slot_pair, flat_T, flat_G);
        else
            flat_pairs_kernel<true, false><<<grid, TILE_PX, 0, s>>>(a, tiles, slot_pair, flat_T, flat_G);
    } else {
        if (flat_G)
            flat_pairs_kernel<false, true><<<grid, TILE_PX, 0, s>>>(a, tiles, slot_pair, flat_T, flat_G);
        else
            flat_pairs_kernel<false, false><<<grid, TILE_PX, 0, s>>>(a, tiles, slot_pair, flat_T, flat_G);
    }
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace conegs
