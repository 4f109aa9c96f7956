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
#include <algorithm>

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

// ---------------------------------------------------------------- long lists split across CTAs
//
// A tile list longer than the view's segment length is cut into segments processed by
// separate CTAs (pass A), each walking its entries for the tile's 64 pixels
// from a local transmittance of 1 and keeping (C_seg, T_seg, last
// contributor).  A segment may stop early once T_local (1 - a) < 1e-4:
// the transmittance entering it is at most 1, so the true walk stops there or
// earlier.  Pass B composites the segments of each pixel front to back,
//   C += T_in C_seg,  T_in *= T_seg,
// while T_in T_seg >= 1e-4 and no local stop happened; T_local after each
// contributing pair only decreases, so the true stop lies in the first
// segment where that fails, and only that segment is walked again, exactly
// (sequential rules from T_in).  Tiles with one segment run the single-pass
// walk directly.

constexpr uint32_t SEG_MIN = 1024;
constexpr uint32_t CTA_SLOTS = 148 * 16;   // resident 64-thread raster CTAs on a B300

uint32_t segment_length(int, int64_t) { return SEG_MIN; }   // the smallest segment (sizes scratch)

// Non-empty tile count and total list length (stat[0], stat[1]).
__global__ void seg_stat_kernel(const uint2 *__restrict__ ranges, int nt, unsigned long long *__restrict__ stat) {
    unsigned long long ne = 0, len = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint32_t l = ranges[t].y - ranges[t].x;
        ne += l > 0;
        len += l;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
        len += __shfl_xor_sync(0xffffffffu, len, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stat, ne);
        atomicAdd(stat + 1, len);
    }
}

// Segment length: 1024 entries when the view has too few non-empty tiles to fill
// the GPU; otherwise 4x the mean non-empty list, so that only tail lists split.
__device__ __forceinline__ uint32_t seg_length_dev(const unsigned long long *stat) {
    const unsigned long long ne = stat[0] > 0 ? stat[0] : 1;
    if (ne < 2 * CTA_SLOTS) return SEG_MIN;
    const unsigned long long s = 4ull * (stat[1] / ne);
    return (uint32_t)(s > SEG_MIN ? (s < 0x7fffffffull ? s : 0x7fffffffull) : SEG_MIN);
}

__global__ void seg_count_kernel(const uint2 *__restrict__ ranges, int nt, const unsigned long long *__restrict__ stat,
                                 uint32_t *__restrict__ nseg) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const uint32_t seg = seg_length_dev(stat);
    const uint32_t len = ranges[t].y - ranges[t].x;
    nseg[t] = len > seg ? (len + seg - 1) / seg : 1u;
}

// Work items of the second and later segments, tile-major (the first segments
// of all tiles run as one launch before them).
__global__ void seg_map_kernel(const uint32_t *__restrict__ nseg, const uint32_t *__restrict__ off, int nt,
                               uint2 *__restrict__ work, uint32_t *__restrict__ total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    for (uint32_t k = 1; k < nseg[t]; ++k) work[off[t] - t + k - 1] = make_uint2((uint32_t)t, k);
    if (t == nt - 1) *total = off[t] + nseg[t] - (uint32_t)nt;
}

struct SegArgs {
    const unsigned long long *stat;   // -> segment length (seg_length_dev)
    const uint32_t *nseg, *seg_off;
    const uint2 *work;      // (tile, segment >= 1)
    const uint32_t *total;  // number of such items
    float4 *seg_c;          // [item][TILE_PX]: C0, C1, C2, T_seg   (item = seg_off[tile] + segment)
    uint32_t *seg_l;        // [item][TILE_PX]: last contributor (local, 1-based; 0 none) | stopped << 31
    uint32_t *seg_all;      // [item]: 1 if every pixel of the tile stopped inside this segment
};

// FIRST: one CTA per tile for its first segment; else one per later segment.
template <bool FILTER, bool FIRST>
__global__ void __launch_bounds__(TILE_PX) raster_seg_kernel(const RasterArgs a, const SegArgs g) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    uint2 tw;
    if (FIRST) {
        tw = make_uint2(blockIdx.x, 0u);
    } else {
        if (blockIdx.x >= *g.total) return;
        tw = g.work[blockIdx.x];
    }
    const int tile = (int)tw.x;
    const uint32_t nseg = g.nseg[tile];
    const uint32_t w = g.seg_off[tile] + tw.y;
    if (!FIRST) {
        // an earlier segment already stopped every pixel of the tile: this one is never read
        bool skip = false;
        for (uint32_t k = g.seg_off[tile]; k < w && !skip; ++k) skip = ((volatile uint32_t *)g.seg_all)[k] != 0u;
        if (skip) return;
    }
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
    const uint32_t seg = seg_length_dev(g.stat);
    const uint32_t b0 = range.x + tw.y * seg;
    const uint32_t b1 = nseg == 1 ? range.y : min(range.y, b0 + seg);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tacc = 1.0f;
    uint32_t last = 0, walked = 0, full = 0;
    bool stopped = false;
    for (uint32_t start = b0; start < b1; start += TILE_PX) {
        if (__syncthreads_count(done) == TILE_PX) break;
        const uint32_t idx = start + threadIdx.x;
        if (idx < b1) {
            const float4 *r = a.rec + (size_t)REC_F4 * a.gids[idx];
#pragma unroll
            for (int k = 0; k < REC_F4; ++k) s_rec[k][threadIdx.x] = r[k];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)TILE_PX, b1 - start);
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
                            stopped = true;
                            mask = 0ull;
                        } else {
                            const float wgt = alpha * Tacc;
                            C0 += r3.x * wgt;
                            C1 += r3.y * wgt;
                            C2 += r3.z * wgt;
                            Tacc = test;
                            last = start - b0 + (uint32_t)b + 1u;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (a.evaluated) {
        unsigned long long wk = walked, f = full;
        for (int o = 16; o > 0; o >>= 1) {
            wk += __shfl_xor_sync(0xffffffffu, wk, o);
            f += __shfl_xor_sync(0xffffffffu, f, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.evaluated, wk);
            atomicAdd(a.evaluated + 1, f);
        }
    }
    if (nseg == 1) {                       // the whole list: final result
        if (inside) {
            a.out_rgb[pix] = C0;
            a.out_rgb[P + pix] = C1;
            a.out_rgb[2 * P + pix] = C2;
            if (a.out_T) a.out_T[pix] = Tacc;
            if (a.keep_T) a.keep_T[pix] = Tacc;
            if (a.last) a.last[pix] = last;
        }
        return;
    }
    g.seg_c[(size_t)w * TILE_PX + threadIdx.x] = make_float4(C0, C1, C2, Tacc);
    g.seg_l[(size_t)w * TILE_PX + threadIdx.x] = last | (stopped ? 0x80000000u : 0u);
    const int all = __syncthreads_and(stopped || !(inside && a.valid[pix]));
    if (threadIdx.x == 0) g.seg_all[w] = all ? 1u : 0u;
}

template <bool FILTER>
__global__ void __launch_bounds__(TILE_PX) raster_merge_kernel(const RasterArgs a, const SegArgs g) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    __shared__ uint32_t s_need[TILE_PX];          // stop segment per pixel (0xffffffff: none)
    const int tile = blockIdx.x;
    const uint32_t nseg = g.nseg[tile];
    if (nseg == 1) return;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const bool inside = i < a.W && j < a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    const uint2 range = a.ranges[tile];
    const uint32_t seg = seg_length_dev(g.stat);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tin = 1.0f;
    uint32_t last = 0, need = 0xffffffffu;
    const bool live = inside && a.valid[pix];
    if (live) {
        const uint32_t w0 = g.seg_off[tile];
        for (uint32_t sgm = 0; sgm < nseg; ++sgm) {
            const float4 c = g.seg_c[(size_t)(w0 + sgm) * TILE_PX + threadIdx.x];
            const uint32_t l = g.seg_l[(size_t)(w0 + sgm) * TILE_PX + threadIdx.x];
            const bool stopped = (l & 0x80000000u) != 0u;
            if (sgm == 0 && stopped) {
                // the first segment starts from T = 1: its walk is the exact one
                C0 = c.x; C1 = c.y; C2 = c.z; Tin = c.w;
                last = l & 0x7fffffffu;
                break;
            }
            if (!stopped && Tin * c.w >= T_STOP) {
                C0 += Tin * c.x;
                C1 += Tin * c.y;
                C2 += Tin * c.z;
                Tin *= c.w;
                if (l & 0x7fffffffu) last = sgm * seg + (l & 0x7fffffffu);
                continue;
            }
            need = sgm;                              // the walk stops inside this segment
            break;
        }
    }
    s_need[threadIdx.x] = need;
    __syncthreads();
    // replay each distinct stop segment once, staged through shared memory, for
    // the pixels that stop in it (exact sequential rules from their T_in)
    PixelRays px;
    if (need != 0xffffffffu) load_pixel(a, pix, P, px);
    uint32_t cur = 0;
    while (true) {
        // smallest stop segment >= cur among the tile's pixels
        uint32_t nxt = 0xffffffffu;
        for (int k = 0; k < TILE_PX; ++k) {
            const uint32_t v = s_need[k];
            if (v >= cur && v < nxt) nxt = v;
        }
        if (nxt == 0xffffffffu) break;
        cur = nxt + 1;
        const uint32_t b0 = range.x + nxt * seg, b1 = min(range.y, b0 + seg);
        bool active = need == nxt;
        for (uint32_t start = b0; start < b1; start += TILE_PX) {
            if (__syncthreads_count(active) == 0) break;
            const uint32_t idx = start + threadIdx.x;
            if (idx < b1) {
                const float4 *r = a.rec + (size_t)REC_F4 * a.gids[idx];
#pragma unroll
                for (int k = 0; k < REC_F4; ++k) s_rec[k][threadIdx.x] = r[k];
            }
            __syncthreads();
            const int nb = (int)min((uint32_t)TILE_PX, b1 - start);
            unsigned long long mask = 0ull;
            if (active) {
                for (int b = 0; b < nb; ++b) {
                    const float4 r4 = s_rec[4][b], r5 = s_rec[5][b], r6 = s_rec[6][b];
                    const float e0 = px.d[0] - r4.x, e1 = px.d[1] - r4.y, e2 = px.d[2] - r4.z;
                    const float qa = r5.z * e0 + r6.y * e1 + r6.z * e2;
                    const float qb = r5.w * e1 + r6.w * e2;
                    const float cone =
                        -1.0f + r4.w * e0 + r5.x * e1 + r5.y * e2 + qa * e0 + qb * e1 + r6.x * e2 * e2;
                    if (!(cone > 1e-3f)) mask |= 1ull << b;
                }
            }
            while (__any_sync(0xffffffffu, mask != 0ull)) {
                if (mask != 0ull) {
                    const int b = __ffsll((long long)mask) - 1;
                    mask &= mask - 1ull;
                    const float4 r3 = s_rec[3][b];
                    float T;
                    if (pair_response<FILTER>(s_rec[0][b], s_rec[1][b], s_rec[2][b], r3.w, s_rec[7][b].x,
                                              a.additive != 0, px, T)) {
                        const float alpha = fminf(ALPHA_MAX, T);
                        if (!(alpha < ALPHA_MIN)) {
                            const float test = Tin * (1.0f - alpha);
                            if (test < T_STOP) {
                                active = false;
                                mask = 0ull;
                            } else {
                                const float wgt = alpha * Tin;
                                C0 += r3.x * wgt;
                                C1 += r3.y * wgt;
                                C2 += r3.z * wgt;
                                Tin = test;
                                last = start - range.x + (uint32_t)b + 1u;
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (!inside) return;
    a.out_rgb[pix] = C0;
    a.out_rgb[P + pix] = C1;
    a.out_rgb[2 * P + pix] = C2;
    if (a.out_T) a.out_T[pix] = Tin;
    if (a.keep_T) a.keep_T[pix] = Tin;
    if (a.last) a.last[pix] = last;
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, int pred,
                           cudaStream_t s);

// Scratch words (uint32) of the split path for ntiles tiles and n_pairs pairs.
int64_t split_scratch_words(int ntiles, int64_t n_pairs) {
    const int64_t wmax = ntiles + n_pairs / segment_length(ntiles, n_pairs) + 1;
    return 2LL * ntiles + 2 * wmax + 4 + 5 * wmax * TILE_PX + wmax + 64 + 4;
}

cudaError_t launch_raster_split(const RasterArgs &a, int ntiles, int64_t n_pairs, bool filter, uint32_t *scratch,
                                uint32_t *scan_scratch, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const int64_t wmax = ntiles + n_pairs / SEG_MIN + 1;
    SegArgs g;
    uint32_t *nseg = scratch, *off = scratch + ntiles;
    uint2 *work = reinterpret_cast<uint2 *>(scratch + 2 * (int64_t)ntiles + 2);   // 8-byte aligned
    uint32_t *total = scratch + 2 * (int64_t)ntiles;
    float4 *seg_c = reinterpret_cast<float4 *>(scratch + ((2 * (int64_t)ntiles + 2 + 2 * wmax + 3) & ~3LL));
    uint32_t *seg_l = reinterpret_cast<uint32_t *>(seg_c + wmax * TILE_PX);
    uint32_t *seg_all = seg_l + wmax * TILE_PX;
    unsigned long long *stat = reinterpret_cast<unsigned long long *>(seg_all + ((wmax + 1) & ~1LL));
    g.nseg = nseg; g.seg_off = off; g.work = work; g.total = total; g.seg_c = seg_c; g.seg_l = seg_l;
    g.seg_all = seg_all;
    g.stat = stat;
    cudaError_t e0 = cudaMemsetAsync(stat, 0, 2 * sizeof(unsigned long long), s);
    if (e0 != cudaSuccess) return e0;
    seg_stat_kernel<<<(unsigned)std::min<int64_t>(div_up(ntiles, 256), 148), 256, 0, s>>>(a.ranges, ntiles, stat);
    note_launches(1);
    seg_count_kernel<<<(unsigned)div_up(ntiles, 256), 256, 0, s>>>(a.ranges, ntiles, stat, nseg);
    note_launches(1);
    cudaError_t e = exclusive_scan(nseg, off, ntiles, scan_scratch, 0, s);
    if (e != cudaSuccess) return e;
    seg_map_kernel<<<(unsigned)div_up(ntiles, 256), 256, 0, s>>>(nseg, off, ntiles, work, total);
    note_launches(1);
    // flags must start at 0 every render: a stale 1 would skip a live segment
    cudaError_t ez = cudaMemsetAsync(seg_all, 0, sizeof(uint32_t) * (size_t)wmax, s);
    if (ez != cudaSuccess) return ez;
    const unsigned later = (unsigned)std::max<int64_t>(1, wmax - ntiles);
    if (filter) {
        raster_seg_kernel<true, true><<<ntiles, TILE_PX, 0, s>>>(a, g);
        raster_seg_kernel<true, false><<<later, TILE_PX, 0, s>>>(a, g);
        raster_merge_kernel<true><<<ntiles, TILE_PX, 0, s>>>(a, g);
    } else {
        raster_seg_kernel<false, true><<<ntiles, TILE_PX, 0, s>>>(a, g);
        raster_seg_kernel<false, false><<<later, TILE_PX, 0, s>>>(a, g);
        raster_merge_kernel<false><<<ntiles, TILE_PX, 0, s>>>(a, g);
    }
    note_launches(3);
    return cudaGetLastError();
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
