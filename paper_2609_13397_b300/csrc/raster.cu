// K5: tile rasteriser, forward (Sec. 3 Eq. 4 compositing over Eq. 9 responses).
//
// One warp per 8x8 tile (per list segment, for long lists), each lane two
// horizontally adjacent pixels whose responses it evaluates together in
// packed FP32 (f32x2 instructions, pair_eval<float2>).  The tile's
// depth-sorted Gaussian list is walked in batches of 32: each lane stages one
// Gaussian's view record into shared memory, every value the packed
// evaluation reads stored twice; every lane then pre-tests the batch against
// its two pixels' rays (broadcast reads) and walks the entries either pixel
// passed in depth order, the warp's lanes on different entries in lockstep.
// Compositing follows the 3DGS conventions: a = min(0.99, T); pairs with
// a < 1/255 are skipped; a pixel stops before the pair that would take its
// transmittance below 1e-4; the warp leaves the list as soon as all 64 pixels
// have stopped.  Per pixel the kernels write rgb, the final transmittance and
// the number of list entries walked up to the last contributing pair (for the
// adjoint, which recomputes the same responses bit for bit in scalar form).
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
    return (int64_t)ntiles + std::max<int64_t>(2 * (int64_t)CTA_SLOTS, ntiles / 4 + 1) + 1;
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

// ---------------------------------------------------------------- the walk
//
// One warp per tile (or list segment): lane l owns the horizontally adjacent
// pixels (2 (l mod 4), l / 4) and (2 (l mod 4) + 1, l / 4) of the 8x8 tile,
// and evaluates both against each Gaussian in packed FP32 (pair_eval<float2>).
// The list is staged BATCH entries at a time in shared memory, every value the
// packed evaluation reads stored twice (a float2 per scalar), so that it loads
// ready for the f32x2 instructions.  Phase 1 pre-tests every staged entry
// against both pixels (broadcast reads); phase 2 walks, in depth order, the
// entries either pixel passed, each lane on its own entries, and composites
// each pixel with the entries it passed itself.

constexpr int RASTER_THREADS = 32;
constexpr int BATCH = 32;

struct StagedBatch {
    float2 w[14][BATCH];   // W_eff rows (9), o_u (3), sigma_eff, rho^2 (sign bit: flat)
    float2 t[12][BATCH];   // pre-test: u (3), g (3), C00, C11, C22, 2 C01, 2 C02, 2 C12
    float4 c[BATCH];       // rgb
};

struct PixState {
    float C0, C1, C2, T;
    uint32_t last;         // list entries up to and including the last contributor (1-based)
    bool stopped;
};

__device__ __forceinline__ void stage_entry(StagedBatch &sb, int k, const float4 *r) {
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5], r6 = r[6];
    const float r7x = r[7].x;
    const float w[14] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z, r0.w, r1.w, r2.w, r3.w, r7x};
    const float t[12] = {r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w, r6.x, r6.y, r6.z, r6.w};
#pragma unroll
    for (int j = 0; j < 14; ++j) sb.w[j][k] = make_float2(w[j], w[j]);
#pragma unroll
    for (int j = 0; j < 12; ++j) sb.t[j][k] = make_float2(t[j], t[j]);
    sb.c[k] = r3;
}

// One compositing step (Eq. 4 with the 3DGS conventions): a = min(0.99, T);
// a < 1/255 is skipped; the pixel stops before the pair that would take its
// transmittance below 1e-4 (returns true); else the pair's colour is added.
__device__ __forceinline__ bool composite_step(PixState &s, float T, const float4 rgb, uint32_t walk1) {
    const float alpha = fminf(ALPHA_MAX, T);
    if (alpha < ALPHA_MIN) return false;
    const float test = s.T * (1.0f - alpha);
    if (test < T_STOP) return true;
    const float wgt = alpha * s.T;
    s.C0 += rgb.x * wgt;
    s.C1 += rgb.y * wgt;
    s.C2 += rgb.z * wgt;
    s.T = test;
    s.last = walk1;
    return false;
}

// Walks list entries [b0, b1) for the lane's two pixels (tile pixel indices qa,
// qa + 1) from their states, with the sequential compositing rules.  Live
// pixels take part; a pixel leaves at its stop (sets stopped) or at b1.  last is
// 1-based relative to `base`.  Counters: list entries walked and evaluations
// past the pre-test, per pixel; of those, FP64 (flat) ones.
template <bool FILTER>
__device__ __forceinline__ void walk2(const RasterArgs &a, StagedBatch &sb, uint32_t b0, uint32_t b1, uint32_t base,
                                      bool liveA, bool liveB, const PixelRaysT<float2> &px, int qa, PixState &A,
                                      PixState &B, uint32_t &walked, uint32_t &full, uint32_t &nflat) {
    using O = Ops<float2>;
    bool doneA = !liveA, doneB = !liveB;
    for (uint32_t start = b0; start < b1; start += BATCH) {
        if (__all_sync(0xffffffffu, doneA && doneB)) break;
        const uint32_t idx = start + threadIdx.x;
        __syncwarp();
        if (idx < b1) stage_entry(sb, threadIdx.x, a.rec + (size_t)REC_F4 * a.gids[idx]);
        __syncwarp();
        const int nb = (int)min((uint32_t)BATCH, b1 - start);
        // phase 1: pre-test of every staged entry against both pixels
        uint32_t mA = 0u, mB = 0u;
        if (!(doneA && doneB)) {
            walked += (uint32_t)nb * ((doneA ? 0u : 1u) + (doneB ? 0u : 1u));
            for (int b = 0; b < nb; ++b) {
                const Bool2 pass = pretest<float2>(sb.t[0][b], sb.t[1][b], sb.t[2][b], sb.t[3][b], sb.t[4][b],
                                                   sb.t[5][b], sb.t[6][b], sb.t[7][b], sb.t[8][b], sb.t[9][b],
                                                   sb.t[10][b], sb.t[11][b], px.d);
                mA |= (pass.x ? 1u : 0u) << b;
                mB |= (pass.y ? 1u : 0u) << b;
            }
            if (doneA) mA = 0u;
            if (doneB) mB = 0u;
        }
        // phase 2: the entries either pixel passed, in depth order
        uint32_t m = mA | mB;
        while (__any_sync(0xffffffffu, m != 0u)) {
            if (m == 0u) continue;
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const bool inA = (mA >> b) & 1u, inB = (mB >> b) & 1u;
            full += (inA ? 1u : 0u) + (inB ? 1u : 0u);
            const float2 r7 = sb.w[13][b];
            float2 T;
            Bool2 hit;
            if (!rec_is_flat(r7.x)) {
                const GaussRec<float2> g{{sb.w[0][b], sb.w[1][b], sb.w[2][b], sb.w[3][b], sb.w[4][b], sb.w[5][b],
                                          sb.w[6][b], sb.w[7][b], sb.w[8][b]},
                                         {sb.w[9][b], sb.w[10][b], sb.w[11][b]},
                                         sb.w[12][b],
                                         r7};
                pair_eval<FILTER, false, float2>(g, a.additive != 0, px, T, hit);
            } else {                                  // FP64 responses, precomputed
                const float *ft = a.flat_T + (size_t)a.flat_slot[start + b] * TILE_PX + qa;
                T = make_float2(ft[0], ft[1]);
                hit = Bool2{T.x >= 0.0f, T.y >= 0.0f};
                nflat += (inA ? 1u : 0u) + (inB ? 1u : 0u);
            }
            const float4 rgb = sb.c[b];
            const uint32_t walk1 = start - base + (uint32_t)b + 1u;
            if (inA && hit.x && composite_step(A, T.x, rgb, walk1)) {
                A.stopped = doneA = true;
                mA = 0u;
                m &= mB;
            }
            if (inB && hit.y && composite_step(B, T.y, rgb, walk1)) {
                B.stopped = doneB = true;
                mB = 0u;
                m &= mA;
            }
        }
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

// The lane's two pixels: tile pixel indices q, q + 1; image coordinates; rays.
struct LanePixels {
    int q;
    int64_t pixA, pixB;
    bool insideA, insideB, liveA, liveB;
};

__device__ __forceinline__ LanePixels lane_pixels(const RasterArgs &a, int tile) {
    LanePixels L;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int row = threadIdx.x >> 2, col = (threadIdx.x & 3) * 2;
    L.q = row * TILE + col;
    const int i = tx * TILE + col, j = ty * TILE + row;
    L.pixA = (int64_t)j * a.W + i;
    L.pixB = L.pixA + 1;
    L.insideA = i < a.W && j < a.H;
    L.insideB = i + 1 < a.W && j < a.H;
    L.liveA = L.insideA && a.valid[L.pixA];
    L.liveB = L.insideB && a.valid[L.pixB];
    return L;
}

__device__ __forceinline__ PixelRaysT<float2> lane_rays(const RasterArgs &a, const LanePixels &L, int64_t P,
                                                        bool useA, bool useB) {
    PixelRays ra{}, rb{};
    if (useA) load_pixel(a, L.pixA, P, ra);
    if (useB) load_pixel(a, L.pixB, P, rb);
    return pack_pixels(ra, rb);
}

// Pass A.  FIRST: one warp per tile for its first segment; else one per later segment.
template <bool FILTER, bool FIRST>
__global__ void __launch_bounds__(RASTER_THREADS) raster_seg_kernel(const RasterArgs a, const SegArgs g) {
    __shared__ StagedBatch sb;
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
    const LanePixels L = lane_pixels(a, tile);
    const int64_t P = (int64_t)a.W * a.H;
    const PixelRaysT<float2> px = lane_rays(a, L, P, L.liveA, L.liveB);
    const uint2 range = a.ranges[tile];
    const uint32_t seg = seg_length_dev(g.stat);
    const uint32_t b0 = range.x + tw.y * seg;
    const uint32_t b1 = nseg == 1 ? range.y : min(range.y, b0 + seg);
    PixState A{0.f, 0.f, 0.f, 1.0f, 0u, false}, B{0.f, 0.f, 0.f, 1.0f, 0u, false};
    uint32_t walked = 0, full = 0, nflat = 0;
    walk2<FILTER>(a, sb, b0, b1, b0, L.liveA, L.liveB, px, L.q, A, B, walked, full, nflat);
    count_walk(a, walked, full, nflat);
    if (nseg == 1) {                       // the whole list: final result
        if (L.insideA) write_pixel(a, L.pixA, P, A.C0, A.C1, A.C2, A.T, A.last);
        if (L.insideB) write_pixel(a, L.pixB, P, B.C0, B.C1, B.C2, B.T, B.last);
        return;
    }
    const size_t o = (size_t)w * TILE_PX + L.q;
    g.seg_c[o] = make_float4(A.C0, A.C1, A.C2, A.T);
    g.seg_c[o + 1] = make_float4(B.C0, B.C1, B.C2, B.T);
    g.seg_l[o] = A.last | (A.stopped ? 0x80000000u : 0u);
    g.seg_l[o + 1] = B.last | (B.stopped ? 0x80000000u : 0u);
    const bool all = __all_sync(0xffffffffu, (A.stopped || !L.liveA) && (B.stopped || !L.liveB));
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
    const uint32_t seg = seg_length_dev(g.stat);
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

// Replay: one warp per segment item; walks the segment again for the pixels
// whose walk stops in it, from their T_in, and writes their final result; the
// segment's share of C and the final T replace its pass-A entry.
template <bool FILTER>
__global__ void __launch_bounds__(RASTER_THREADS) raster_replay_kernel(const RasterArgs a, const SegArgs g,
                                                                       int ntiles) {
    __shared__ StagedBatch sb;
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
    const LanePixels L = lane_pixels(a, tile);
    const int64_t P = (int64_t)a.W * a.H;
    const size_t q = (size_t)tile * TILE_PX + L.q;
    const bool mineA = g.rp_need[q] == tw.y, mineB = g.rp_need[q + 1] == tw.y;
    float4 cinA = make_float4(0.f, 0.f, 0.f, 1.0f), cinB = cinA;
    PixState A{0.f, 0.f, 0.f, 1.0f, 0u, false}, B{0.f, 0.f, 0.f, 1.0f, 0u, false};   // C: this segment's share
    if (mineA) {
        cinA = g.rp_c[q];
        A.T = cinA.w;
        A.last = g.rp_last[q];
    }
    if (mineB) {
        cinB = g.rp_c[q + 1];
        B.T = cinB.w;
        B.last = g.rp_last[q + 1];
    }
    const PixelRaysT<float2> px = lane_rays(a, L, P, mineA, mineB);
    const uint2 range = a.ranges[tile];
    const uint32_t seg = seg_length_dev(g.stat);
    const uint32_t b0 = range.x + tw.y * seg, b1 = min(range.y, b0 + seg);
    uint32_t walked = 0, full = 0, nflat = 0;
    walk2<FILTER>(a, sb, b0, b1, range.x, mineA, mineB, px, L.q, A, B, walked, full, nflat);
    if (mineA) {
        g.seg_c[(size_t)w * TILE_PX + L.q] = make_float4(A.C0, A.C1, A.C2, A.T);
        if (L.insideA) write_pixel(a, L.pixA, P, cinA.x + A.C0, cinA.y + A.C1, cinA.z + A.C2, A.T, A.last);
    }
    if (mineB) {
        g.seg_c[(size_t)w * TILE_PX + L.q + 1] = make_float4(B.C0, B.C1, B.C2, B.T);
        if (L.insideB) write_pixel(a, L.pixB, P, cinB.x + B.C0, cinB.y + B.C1, cinB.z + B.C2, B.T, B.last);
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

template <bool FILTER>
static void launch_raster_passes(const RasterArgs &a, const SegArgs &g, int ntiles, unsigned later, int64_t wmax,
                                 cudaStream_t s, cudaEvent_t main0, cudaEvent_t main1) {
    if (main0) cudaEventRecord(main0, s);
    raster_seg_kernel<FILTER, true><<<ntiles, RASTER_THREADS, 0, s>>>(a, g);
    if (main1) cudaEventRecord(main1, s);
    raster_seg_kernel<FILTER, false><<<later, RASTER_THREADS, 0, s>>>(a, g);
    raster_merge_kernel<<<ntiles, TILE_PX, 0, s>>>(a, g);
    raster_replay_kernel<FILTER><<<(unsigned)wmax, RASTER_THREADS, 0, s>>>(a, g, ntiles);
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
    seg_stat_kernel<<<(unsigned)std::min<int64_t>(div_up(ntiles, 256), 148), 256, 0, s>>>(a.ranges, ntiles, stat);
    seg_count_kernel<<<(unsigned)div_up(ntiles, 256), 256, 0, s>>>(a.ranges, ntiles, stat, nseg);
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
    if (filter)
        launch_raster_passes<true>(a, g, ntiles, later, wmax, s, main0, main1);
    else
        launch_raster_passes<false>(a, g, ntiles, later, wmax, s, main0, main1);
    if (a.keep_T) {
        raster_suffix_kernel<<<ntiles, TILE_PX, 0, s>>>(g);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace conegs
