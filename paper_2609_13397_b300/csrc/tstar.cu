// Per-ray compositing order (flag CONEGS_ORDER_TSTAR): the pairs of a pixel are
// composited by their own max-response depth t* on the pixel's ray (Sec. 3:
// the composite is sorted by t*_k), instead of by the tile list's per-Gaussian
// key |mu - o|.
//
// The tile list stays sorted by the key; each pixel re-orders the pairs that
// reach it through a k-buffer of TS_K entries (t*, alpha, Gaussian), kept
// sorted in shared memory.  A pair arriving at a full buffer first releases the
// smallest t* of the buffer and itself, and the released pair is composited
// with the rules of Eq. 4 (a = min(0.99, T), a < 1/255 skipped, stop before
// T_acc (1 - a) < 1e-4).  At the end of the list the buffer is composited in
// order.  Ties in t* go to the earlier list entry, i.e. to the smaller key and
// then the smaller index, as in the exact per-pixel sort.
//
// Exactness: the order is the exact per-pixel t* order whenever no pair is
// released before a later-arriving pair of smaller t*; in particular whenever a
// pixel has at most TS_K pairs with a >= 1/255 before its stop (nothing is
// released before the final, fully sorted flush).  Beyond that the buffer
// corrects any displacement of fewer than TS_K contributing pairs between the
// key order and the t* order.
//
// One CTA of 64 threads per 8x8 tile walks the whole list (no segment split:
// the segments' merge assumes the key order across segments).  Forward only:
// the adjoint walk replays the key order.
#include "raster.cuh"

namespace conegs {

constexpr int TS_K = 32;

namespace {

// Composites one released pair; false once the pixel stops.
__device__ __forceinline__ bool ts_emit(const RasterArgs &a, float alpha, uint32_t gid, float &C0, float &C1, float &C2,
                                        float &Tacc) {
    const float test = Tacc * (1.0f - alpha);
    if (test < T_STOP) return false;
    const float4 c = a.rec[(size_t)REC_F4 * gid + 3];
    const float wgt = alpha * Tacc;
    C0 += c.x * wgt;
    C1 += c.y * wgt;
    C2 += c.z * wgt;
    Tacc = test;
    return true;
}

}  // namespace

template <bool FILTER, bool PIX>
__global__ void __launch_bounds__(TILE_PX) raster_tstar_kernel(const RasterArgs a) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    __shared__ uint32_t s_gid[TILE_PX];
    __shared__ float s_ts[TS_K][TILE_PX];
    __shared__ float s_al[TS_K][TILE_PX];
    __shared__ uint32_t s_bg[TS_K][TILE_PX];
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    const bool inside = i < a.W && j < a.H;
    const bool live = inside && a.valid[pix];
    PixelRays px;
    if (live) load_pixel(a, pix, P, px);
    const uint2 range = a.ranges[tile];
    const int t = threadIdx.x;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tacc = 1.0f;
    int nbuf = 0;                       // entries s_*[0 .. nbuf), t* descending (the next to release last)
    bool done = !live;
    uint32_t walked = 0, full = 0, nflat = 0;
    for (uint32_t start = range.x; start < range.y; start += TILE_PX) {
        if (__syncthreads_count(done) == TILE_PX) break;
        const uint32_t idx = start + t;
        if (idx < range.y) {
            const uint32_t gid = a.gids[idx];
            const float4 *r = a.rec + (size_t)REC_F4 * gid;
#pragma unroll
            for (int k = 0; k < REC_F4; ++k) s_rec[k][t] = r[k];
            s_gid[t] = gid;
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)TILE_PX, range.y - start);
        if (!done) walked += (uint32_t)nb;
        for (int b = 0; b < nb && !done; ++b) {
            if (!staged_pretest<PIX>(s_rec, b, px)) continue;
            ++full;
            const float r7x = s_rec[7][b].x;
            const GaussRec<float> g = rec_f32(s_rec[0][b], s_rec[1][b], s_rec[2][b], s_rec[3][b].w, r7x);
            // t* of the pair on this ray (Eq. 2): the ordering key
            // (the response's own operations, so the compiler shares them)
            const float du0 = dot3v(g.W[0], g.W[1], g.W[2], px.d[0], px.d[1], px.d[2]);
            const float du1 = dot3v(g.W[3], g.W[4], g.W[5], px.d[0], px.d[1], px.d[2]);
            const float du2 = dot3v(g.W[6], g.W[7], g.W[8], px.d[0], px.d[1], px.d[2]);
            const float ts = -(dot3v(g.ou[0], g.ou[1], g.ou[2], du0, du1, du2) *
                               Ops<float>::rcp(dot3v(du0, du1, du2, du0, du1, du2)));
            float T;
            bool hit;
            if (!rec_is_flat(r7x)) {
                hit = pair_response<FILTER>(g, a.additive != 0, px, T);
            } else {                              // FP64 response, precomputed
                ++nflat;
                T = a.flat_T[(size_t)a.flat_slot[start + b] * TILE_PX + t];
                hit = T >= 0.0f;
            }
            if (!hit) continue;
            const float alpha = fminf(ALPHA_MAX, T);
            if (alpha < ALPHA_MIN) continue;
            const uint32_t gid = s_gid[b];
            if (nbuf == TS_K) {
                if (ts < s_ts[TS_K - 1][t]) {     // the new pair comes first
                    if (!ts_emit(a, alpha, gid, C0, C1, C2, Tacc)) done = true;
                    continue;
                }
                const bool ok = ts_emit(a, s_al[TS_K - 1][t], s_bg[TS_K - 1][t], C0, C1, C2, Tacc);
                --nbuf;
                if (!ok) {
                    done = true;
                    continue;
                }
            }
            // stable insertion: the new pair goes before (is released after) equal t*
            int k = nbuf;
            while (k > 0 && s_ts[k - 1][t] <= ts) {
                s_ts[k][t] = s_ts[k - 1][t];
                s_al[k][t] = s_al[k - 1][t];
                s_bg[k][t] = s_bg[k - 1][t];
                --k;
            }
            s_ts[k][t] = ts;
            s_al[k][t] = alpha;
            s_bg[k][t] = gid;
            ++nbuf;
        }
        __syncthreads();
    }
    for (int k = nbuf - 1; k >= 0 && !done; --k)
        if (!ts_emit(a, s_al[k][t], s_bg[k][t], C0, C1, C2, Tacc)) done = true;
    if (a.evaluated) {
        unsigned long long wk = walked, f = full, fl = nflat;
        for (int o = 16; o > 0; o >>= 1) {
            wk += __shfl_xor_sync(0xffffffffu, wk, o);
            f += __shfl_xor_sync(0xffffffffu, f, o);
            fl += __shfl_xor_sync(0xffffffffu, fl, o);
        }
        if ((t & 31) == 0) {
            atomicAdd(a.evaluated, wk);
            atomicAdd(a.evaluated + 1, f);
            if (fl) atomicAdd(a.evaluated + 2, fl);
        }
    }
    if (!inside) return;
    a.out_rgb[pix] = C0;
    a.out_rgb[P + pix] = C1;
    a.out_rgb[2 * P + pix] = C2;
    if (a.out_T) a.out_T[pix] = Tacc;
}

cudaError_t launch_raster_tstar(const RasterArgs &a, int ntiles, bool filter, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (filter && a.pixtest)
        raster_tstar_kernel<true, true><<<ntiles, TILE_PX, 0, s>>>(a);
    else if (filter)
        raster_tstar_kernel<true, false><<<ntiles, TILE_PX, 0, s>>>(a);
    else if (a.pixtest)
        raster_tstar_kernel<false, true><<<ntiles, TILE_PX, 0, s>>>(a);
    else
        raster_tstar_kernel<false, false><<<ntiles, TILE_PX, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
