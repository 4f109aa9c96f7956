// K5: tile rasteriser, forward (Sec. 3 Eq. 4 compositing over Eq. 9 responses).
//
// One CTA of 64 threads per 8x8 tile (per list segment, for long lists), one
// thread per pixel.  The tile's depth-sorted Gaussian list is walked in
// batches of 64: each thread loads one Gaussian's 128-byte view record (8 x
// float4, coalesced gather) into shared memory; every thread then pre-tests
// the batch against its pixel's ray (a broadcast read per entry) and
// evaluates its passing entries in depth order, the warp's lanes on different
// entries in lockstep.  Compositing follows the 3DGS conventions: a =
// min(0.99, T); pairs with a < 1/255 are skipped; a pixel stops before the
// pair that would take its transmittance below 1e-4; the CTA leaves the list
// as soon as all its pixels have stopped (__syncthreads_count).  Per pixel the
// kernels write rgb, the final transmittance and the number of list entries
// walked up to the last contributing pair (for the adjoint, which recomputes
// the same pre-test and responses bit for bit).
#include <algorithm>

#include "raster.cuh"

namespace conegs {

// ---------------------------------------------------------------- long lists split across CTAs
//
// A tile list longer than the view's segment length L (seg_length_dev) is cut
// into segments processed by separate CTAs (pass A), each walking its entries
// for the tile's 64 pixels from a local transmittance of 1 and keeping (C_seg,
// T_seg, last contributor).  A segment may stop early once T_local (1 - a) <
// 1e-4: the transmittance entering it is at most 1, so the true walk stops
// there or earlier.  The merge composites the segments of each pixel front to
// back,
//   C += T_in C_seg,  T_in *= T_seg,
// while T_in T_seg >= 1e-4 and no local stop happened; T_local after each
// contributing pair only decreases, so the true stop lies in the first segment
// where that fails.  That segment is walked again with the sequential rules
// from the pixel's T_in by the replay pass, one CTA per (tile, segment) that
// some pixel stops in.  Tiles with one segment finish in pass A.  When the
// adjoint will run, a suffix pass leaves per (segment, pixel) the colour
// composited behind the segment and the transmittance after it: the state
// from which the adjoint walks each segment back to front on its own.

int64_t split_items_max(int ntiles) {
    return (int64_t)ntiles + std::max<int64_t>(2 * (int64_t)raster_slots(), ntiles / 4 + 1) + 1;
}

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

__global__ void seg_count_kernel(const uint2 *__restrict__ ranges, int nt, const unsigned long long *__restrict__ stat,
                                 uint32_t slots, uint32_t *__restrict__ nseg) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const uint32_t seg = seg_length_dev(stat, slots);
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

// Walks list entries [b0, b1) for the tile's pixels from (C, Tacc), with the
// sequential compositing rules.  `live` pixels take part; a pixel leaves at its
// stop (sets stopped) or at b1.  last is 1-based relative to `base`.  PIX: the
// records hold the pinhole (pixel-space) form of the pre-test.
template <bool FILTER, bool PIX>
__device__ __forceinline__ void walk_entries(const RasterArgs &a, float4 (*s_rec)[TILE_PX], uint32_t b0, uint32_t b1,
                                             uint32_t base, bool live, const PixelRays &px, float &C0, float &C1,
                                             float &C2, float &Tacc, uint32_t &last, bool &stopped,
                                             uint32_t &walked, uint32_t &full, uint32_t &nflat) {
    bool done = !live;
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
        // phase 1: cone pre-test of every staged entry against this pixel (the
        // shared-memory reads are broadcasts: all lanes read the same entry)
        unsigned long long mask = 0ull;
        if (!done) {
            walked += (uint32_t)nb;
            for (int b = 0; b < nb; ++b)
                if (staged_pretest<PIX>(s_rec, b, px)) mask |= 1ull << b;
        }
        // phase 2: each lane walks its own passing entries in depth order, so
        // the warp's lanes evaluate different entries in lockstep
        while (__any_sync(0xffffffffu, mask != 0ull)) {
            if (mask != 0ull) {
                const int b = __ffsll((long long)mask) - 1;
                mask &= mask - 1ull;
                ++full;
                const float4 r3 = s_rec[3][b];
                const float r7x = s_rec[7][b].x;          // rho^2 (sign bit: flat)
                float T;
                bool hit;
                if (!rec_is_flat(r7x)) {
                    hit = pair_response<FILTER>(rec_f32(s_rec[0][b], s_rec[1][b], s_rec[2][b], r3.w, r7x),
                                                a.additive != 0, px, T);
                } else {                          // FP64 response, precomputed
                    ++nflat;
                    T = a.flat_T[(size_t)a.flat_slot[start + b] * TILE_PX + threadIdx.x];
                    hit = T >= 0.0f;
                }
                if (hit) {
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
                            last = start - base + (uint32_t)b + 1u;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void count_walk(const RasterArgs &a, uint32_t walked, uint32_t full, uint32_t nflat) {
    if (!a.evaluated) return;
    unsigned long long wk = walked, f = full, fl = nflat;
    for (int o = 16; o > 0; o >>= 1) {
        wk += __shfl_xor_sync(0xffffffffu, wk, o);
        f += __shfl_xor_sync(0xffffffffu, f, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.evaluated, wk);
        atomicAdd(a.evaluated + 1, f);
        if (fl) atomicAdd(a.evaluated + 2, fl);
    }
}

__device__ __forceinline__ void write_pixel(const RasterArgs &a, int64_t pix, int64_t P, float C0, float C1, float C2,
                                            float T, uint32_t last) {
    a.out_rgb[pix] = C0;
    a.out_rgb[P + pix] = C1;
    a.out_rgb[2 * P + pix] = C2;
    if (a.out_T) a.out_T[pix] = T;
    if (a.keep_T) a.keep_T[pix] = T;
    if (a.last) a.last[pix] = last;
}

// Pass A.  FIRST: one CTA per tile for its first segment; else one per later segment.
template <bool FILTER, bool FIRST, bool PIX>
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
    const bool live = inside && a.valid[pix];
    PixelRays px;
    if (live) load_pixel(a, pix, P, px);
    const uint2 range = a.ranges[tile];
    const uint32_t seg = seg_length_dev(g);
    const uint32_t b0 = range.x + tw.y * seg;
    const uint32_t b1 = nseg == 1 ? range.y : min(range.y, b0 + seg);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tacc = 1.0f;
    uint32_t last = 0, walked = 0, full = 0, nflat = 0;
    bool stopped = false;
    walk_entries<FILTER, PIX>(a, s_rec, b0, b1, b0, live, px, C0, C1, C2, Tacc, last, stopped, walked, full, nflat);
    count_walk(a, walked, full, nflat);
    if (nseg == 1) {                       // the whole list: final result
        if (inside) write_pixel(a, pix, P, C0, C1, C2, Tacc, last);
        return;
    }
    g.seg_c[(size_t)w * TILE_PX + threadIdx.x] = make_float4(C0, C1, C2, Tacc);
    g.seg_l[(size_t)w * TILE_PX + threadIdx.x] = last | (stopped ? 0x80000000u : 0u);
    const int all = __syncthreads_and(stopped || !live);
    if (threadIdx.x == 0) g.seg_all[w] = all ? 1u : 0u;
}

// Merge: per pixel, composite the segments front to back up to the stop
// segment; pixels that never stop are final, the others hand (C, T_in, last)
// to the replay pass and mark their stop segment.  Each segment before the
// stop is rewritten in place as (T_in C_seg, T after it).
__global__ void __launch_bounds__(TILE_PX) raster_merge_kernel(const RasterArgs a, const SegArgs g) {
    const int tile = blockIdx.x;
    const uint32_t nseg = g.nseg[tile];
    if (nseg == 1) return;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const bool inside = i < a.W && j < a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    const uint32_t seg = seg_length_dev(g);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tin = 1.0f;
    uint32_t last = 0, need = NO_STOP, reach = NO_STOP;
    const uint32_t w0 = g.seg_off[tile];
    if (inside && a.valid[pix]) {
        reach = nseg - 1;
        for (uint32_t sgm = 0; sgm < nseg; ++sgm) {
            float4 *cp = g.seg_c + (size_t)(w0 + sgm) * TILE_PX + threadIdx.x;
            const float4 c = *cp;
            const uint32_t l = g.seg_l[(size_t)(w0 + sgm) * TILE_PX + threadIdx.x];
            const bool stopped = (l & 0x80000000u) != 0u;
            if (sgm == 0 && stopped) {
                // the first segment starts from T = 1: its walk is the exact one
                C0 = c.x; C1 = c.y; C2 = c.z; Tin = c.w;
                last = l & 0x7fffffffu;
                reach = 0;
                break;
            }
            if (!stopped && Tin * c.w >= T_STOP) {
                const float4 share = make_float4(Tin * c.x, Tin * c.y, Tin * c.z, Tin * c.w);
                C0 += share.x;
                C1 += share.y;
                C2 += share.z;
                Tin = share.w;
                *cp = share;
                if (l & 0x7fffffffu) last = sgm * seg + (l & 0x7fffffffu);
                continue;
            }
            need = reach = sgm;                      // the walk stops inside this segment
            break;
        }
    }
    const size_t q = (size_t)tile * TILE_PX + threadIdx.x;
    g.rp_need[q] = need;
    g.rp_end[q] = reach;
    if (need != NO_STOP) {
        g.rp_c[q] = make_float4(C0, C1, C2, Tin);
        g.rp_last[q] = last;
        g.need_item[w0 + need] = 1u;                 // every writer stores 1
    } else if (inside) {
        write_pixel(a, pix, P, C0, C1, C2, Tin, last);
    }
}

// Replay: one CTA per segment item; walks the segment again for the pixels
// whose walk stops in it, from their T_in, and writes their final result; the
// segment's share of C and the final T replace its pass-A entry.
template <bool FILTER, bool PIX>
__global__ void __launch_bounds__(TILE_PX) raster_replay_kernel(const RasterArgs a, const SegArgs g, int ntiles) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    uint2 tw;
    if ((int)blockIdx.x < ntiles) {
        tw = make_uint2(blockIdx.x, 0u);
    } else {
        const uint32_t k = blockIdx.x - (uint32_t)ntiles;
        if (k >= *g.total) return;
        tw = g.work[k];
    }
    const int tile = (int)tw.x;
    if (g.nseg[tile] == 1) return;
    const uint32_t w = g.seg_off[tile] + tw.y;
    if (g.need_item[w] == 0u) return;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const bool inside = i < a.W && j < a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    const size_t q = (size_t)tile * TILE_PX + threadIdx.x;
    const bool mine = g.rp_need[q] == tw.y;
    float4 cin = make_float4(0.f, 0.f, 0.f, 1.0f);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.0f;      // C: this segment's share
    uint32_t last = 0, walked = 0, full = 0, nflat = 0;
    PixelRays px;
    if (mine) {
        cin = g.rp_c[q];
        T = cin.w;
        last = g.rp_last[q];
        load_pixel(a, pix, P, px);
    }
    const uint2 range = a.ranges[tile];
    const uint32_t seg = seg_length_dev(g);
    const uint32_t b0 = range.x + tw.y * seg, b1 = min(range.y, b0 + seg);
    bool stopped = false;
    walk_entries<FILTER, PIX>(a, s_rec, b0, b1, range.x, mine, px, C0, C1, C2, T, last, stopped, walked, full,
                              nflat);
    if (mine) {
        g.seg_c[(size_t)w * TILE_PX + threadIdx.x] = make_float4(C0, C1, C2, T);
        if (inside) write_pixel(a, pix, P, cin.x + C0, cin.y + C1, cin.z + C2, T, last);
    }
}

// Suffix (adjoint state): per pixel, from its last segment back to the first,
// (share of C, T after) -> (colour composited behind the segment, T after).
__global__ void __launch_bounds__(TILE_PX) raster_suffix_kernel(const SegArgs g) {
    const int tile = blockIdx.x;
    if (g.nseg[tile] == 1) return;
    const size_t q = (size_t)tile * TILE_PX + threadIdx.x;
    const uint32_t reach = g.rp_end[q];
    if (reach == NO_STOP) return;
    const uint32_t w0 = g.seg_off[tile];
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;
    for (uint32_t sgm = reach + 1; sgm-- > 0;) {
        float4 *cp = g.seg_c + (size_t)(w0 + sgm) * TILE_PX + threadIdx.x;
        const float4 c = *cp;
        *cp = make_float4(S0, S1, S2, c.w);
        S0 += c.x;
        S1 += c.y;
        S2 += c.z;
    }
}

uint32_t raster_slots() {
    static uint32_t slots[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!slots[dev]) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_seg_kernel<true, true, false>, TILE_PX, 0) !=
                cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 16;
        }
        slots[dev] = (uint32_t)(per_sm * num_sms());
    }
    return slots[dev];
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, int pred,
                           cudaStream_t s);

namespace {
struct SplitLayout {
    int64_t wmax, words;
    int64_t o_nseg, o_off, o_total, o_work, o_seg_c, o_seg_l, o_seg_all, o_stat, o_need, o_rp_c, o_rp_need, o_rp_last,
        o_rp_end;
};
SplitLayout split_layout(int ntiles) {
    SplitLayout L;
    const int64_t nt = ntiles, wmax = split_items_max(ntiles);
    auto up4 = [](int64_t x) { return (x + 3) & ~3LL; };
    L.wmax = wmax;
    L.o_nseg = 0;
    L.o_off = nt;
    L.o_total = 2 * nt;                       // 2 words (keeps work 8-byte aligned)
    L.o_work = 2 * nt + 2;                    // 2 words per item
    L.o_seg_c = up4(L.o_work + 2 * wmax);     // 16-byte aligned
    L.o_seg_l = L.o_seg_c + 4 * wmax * TILE_PX;
    L.o_seg_all = L.o_seg_l + wmax * TILE_PX;
    L.o_stat = L.o_seg_all + ((wmax + 1) & ~1LL);   // 8-byte aligned
    L.o_need = L.o_stat + 4;
    L.o_rp_c = up4(L.o_need + wmax);
    L.o_rp_need = L.o_rp_c + 4 * nt * TILE_PX;
    L.o_rp_last = L.o_rp_need + nt * TILE_PX;
    L.o_rp_end = L.o_rp_last + nt * TILE_PX;
    L.words = L.o_rp_end + nt * TILE_PX;
    return L;
}
}  // namespace

int64_t split_scratch_words(int ntiles) { return split_layout(ntiles).words; }

SegArgs split_args(uint32_t *scratch, int ntiles, int64_t *items) {
    const SplitLayout L = split_layout(ntiles);
    SegArgs g;
    g.slots = raster_slots();
    g.nseg = scratch + L.o_nseg;
    g.seg_off = scratch + L.o_off;
    g.total = scratch + L.o_total;
    g.work = reinterpret_cast<const uint2 *>(scratch + L.o_work);
    g.seg_c = reinterpret_cast<float4 *>(scratch + L.o_seg_c);
    g.seg_l = scratch + L.o_seg_l;
    g.seg_all = scratch + L.o_seg_all;
    g.stat = reinterpret_cast<const unsigned long long *>(scratch + L.o_stat);
    g.need_item = scratch + L.o_need;
    g.rp_c = reinterpret_cast<float4 *>(scratch + L.o_rp_c);
    g.rp_need = scratch + L.o_rp_need;
    g.rp_last = scratch + L.o_rp_last;
    g.rp_end = scratch + L.o_rp_end;
    if (items) *items = L.wmax;
    return g;
}

template <bool FILTER, bool PIX>
static void launch_raster_passes(const RasterArgs &a, const SegArgs &g, int ntiles, unsigned later, int64_t wmax,
                                 cudaStream_t s, cudaEvent_t main0, cudaEvent_t main1) {
    if (main0) cudaEventRecord(main0, s);
    raster_seg_kernel<FILTER, true, PIX><<<ntiles, TILE_PX, 0, s>>>(a, g);
    if (main1) cudaEventRecord(main1, s);
    raster_seg_kernel<FILTER, false, PIX><<<later, TILE_PX, 0, s>>>(a, g);
    raster_merge_kernel<<<ntiles, TILE_PX, 0, s>>>(a, g);
    raster_replay_kernel<FILTER, PIX><<<(unsigned)wmax, TILE_PX, 0, s>>>(a, g, ntiles);
    note_launches(4);
}

// main0/main1 (may be NULL): events recorded around the first-segment launch.
cudaError_t launch_raster_split(const RasterArgs &a, int ntiles, bool filter, uint32_t *scratch,
                                uint32_t *scan_scratch, cudaStream_t s, cudaEvent_t main0, cudaEvent_t main1) {
    if (ntiles == 0) {
        if (main0) cudaEventRecord(main0, s);
        if (main1) cudaEventRecord(main1, s);
        return cudaGetLastError();
    }
    int64_t wmax = 0;
    const SegArgs g = split_args(scratch, ntiles, &wmax);
    uint32_t *nseg = const_cast<uint32_t *>(g.nseg), *off = const_cast<uint32_t *>(g.seg_off);
    uint2 *work = const_cast<uint2 *>(g.work);
    unsigned long long *stat = const_cast<unsigned long long *>(g.stat);
    cudaError_t e0 = cudaMemsetAsync(stat, 0, 2 * sizeof(unsigned long long), s);
    if (e0 != cudaSuccess) return e0;
    seg_stat_kernel<<<(unsigned)std::min<int64_t>(div_up(ntiles, 256), num_sms()), 256, 0, s>>>(a.ranges, ntiles,
                                                                                              stat);
    seg_count_kernel<<<(unsigned)div_up(ntiles, 256), 256, 0, s>>>(a.ranges, ntiles, stat, g.slots, nseg);
    note_launches(2);
    cudaError_t e = exclusive_scan(nseg, off, ntiles, scan_scratch, 0, s);
    if (e != cudaSuccess) return e;
    seg_map_kernel<<<(unsigned)div_up(ntiles, 256), 256, 0, s>>>(nseg, off, ntiles, work,
                                                                 const_cast<uint32_t *>(g.total));
    note_launches(1);
    // flags must start at 0 every render: a stale 1 would skip a live segment or replay a dead one
    cudaError_t ez = cudaMemsetAsync(g.seg_all, 0, sizeof(uint32_t) * (size_t)wmax, s);
    if (ez != cudaSuccess) return ez;
    ez = cudaMemsetAsync(g.need_item, 0, sizeof(uint32_t) * (size_t)wmax, s);
    if (ez != cudaSuccess) return ez;
    const unsigned later = (unsigned)(wmax - ntiles);
    if (filter && a.pixtest)
        launch_raster_passes<true, true>(a, g, ntiles, later, wmax, s, main0, main1);
    else if (filter)
        launch_raster_passes<true, false>(a, g, ntiles, later, wmax, s, main0, main1);
    else if (a.pixtest)
        launch_raster_passes<false, true>(a, g, ntiles, later, wmax, s, main0, main1);
    else
        launch_raster_passes<false, false>(a, g, ntiles, later, wmax, s, main0, main1);
    if (a.keep_T) {
        raster_suffix_kernel<<<ntiles, TILE_PX, 0, s>>>(g);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace conegs
