// K4: device scan, compaction and stable LSD radix sort of (key, value) pairs.
//
// Radix sort: 8-bit digits, reduce-then-scan.  A fixed grid of G blocks
// each owns one contiguous chunk (a multiple of its tile size); per pass
//   upsweep   per-block digit histogram             -> counts[digit][block]
//   scan      exclusive scan of the 256*G counters (digit-major)
//   downsweep per tile (3072 items; 1024 for sorts of up to 2^20 items, so that
//             small sorts still spread over the SMs): each warp ranks its items in lane order
//             with bit-sliced ballots (stable), warps are offset by a per-digit
//             scan across warps; the tile is rearranged in shared memory in
//             digit order and written out so that runs of one digit land on
//             consecutive addresses (coalesced stores).
// Stability of every pass makes the whole sort stable, so equal keys keep
// their input order (the binning stage relies on it: Gaussians are emitted
// in depth order and the per-tile lists must keep that order).
#include "common.cuh"

namespace conegs {

// ---------------------------------------------------------------- scan

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &total) {
    __shared__ uint32_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    total = warp_sums[SCAN_THREADS / 32 - 1];
    const uint32_t before = wid > 0 ? warp_sums[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

// out[i] = sum_{j<i} in[i] (per tile), block_sums[b] = tile total.
// If pred != 0 the input is (in[i] > 0) instead of in[i].
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_kernel(const uint32_t *__restrict__ in, int64_t n,
                                                                  uint32_t *__restrict__ out,
                                                                  uint32_t *__restrict__ block_sums, int pred) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        uint32_t x = i < n ? in[i] : 0u;
        if (pred) x = x > 0u ? 1u : 0u;
        v[k] = s;
        s += x;
    }
    uint32_t total;
    const uint32_t off = block_exclusive_scan(s, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = off + v[k];
    }
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

__global__ void add_offsets_kernel(uint32_t *__restrict__ out, int64_t n, const uint32_t *__restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / SCAN_TILE];
}

// One CTA per scan tile: adds the sum of the preceding tiles' totals (read
// directly from block_sums, at most SCAN_TILE of them) to the tile's outputs,
// so a scan of up to SCAN_TILE^2 items needs two launches.
__global__ void __launch_bounds__(SCAN_THREADS) add_tile_prefix_kernel(uint32_t *__restrict__ out, int64_t n,
                                                                       const uint32_t *__restrict__ block_sums) {
    const int b = (int)blockIdx.x;
    uint32_t v = 0u;
    for (int j = threadIdx.x; j < b; j += SCAN_THREADS) v += block_sums[j];
    uint32_t total;
    block_exclusive_scan(v, total);
    const int64_t base = (int64_t)b * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] += total;
    }
}

// Scratch words needed by exclusive_scan for n items.
int64_t scan_scratch_words(int64_t n) {
    int64_t w = 0;
    while (n > SCAN_TILE) {
        n = div_up(n, SCAN_TILE);
        w += n;
    }
    return w + 1;
}

// Exclusive scan of n uint32 (or of in[i] > 0 when pred) into out; scratch of
// scan_scratch_words(n) words.
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, int pred,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = div_up(n, SCAN_TILE);
    uint32_t *bs = nb > 1 ? scratch : nullptr;
    scan_tiles_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, out, bs, pred);
    note_launches(1);
    if (nb > 1 && nb <= SCAN_TILE) {
        add_tile_prefix_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, bs);
        note_launches(1);
    } else if (nb > 1) {
        cudaError_t e = exclusive_scan(bs, bs, nb, scratch + nb, 0, s);
        if (e != cudaSuccess) return e;
        add_offsets_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(out, n, bs);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions, compaction, gathers

// Sum and number of non-zero entries of in[n]; with flag (may be NULL), also the
// sum over the entries whose flag is set.
__global__ void __launch_bounds__(256) sum_u64_kernel(const uint32_t *__restrict__ in, int64_t n,
                                                      unsigned long long *__restrict__ total,
                                                      unsigned long long *__restrict__ nonzero,
                                                      const uint8_t *__restrict__ flag,
                                                      unsigned long long *__restrict__ flagged) {
    unsigned long long s = 0, z = 0, f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = in[i];
        s += v;
        z += v > 0u;
        if (flag && flag[i]) f += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
        f += __shfl_xor_sync(0xffffffffu, f, o);
    }
    // one set of atomics per block (per-warp atomics on the same addresses serialise)
    __shared__ unsigned long long ss[8], sz[8], sf[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ss[w] = s;
        sz[w] = z;
        sf[w] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            s += ss[k];
            z += sz[k];
            f += sf[k];
        }
        atomicAdd(total, s);
        atomicAdd(nonzero, z);
        if (flag && f) atomicAdd(flagged, f);
    }
}

cudaError_t sum_counts(const uint32_t *in, int64_t n, unsigned long long *d_two, const uint8_t *flag,
                       unsigned long long *d_flagged, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_two, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && flag) e = cudaMemsetAsync(d_flagged, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    int grid = (int)std::min<int64_t>(div_up(n, 256), 8 * (int64_t)num_sms());
    sum_u64_kernel<<<grid, 256, 0, s>>>(in, n, d_two, d_two + 1, flag, d_flagged);
    note_launches(1);
    return cudaGetLastError();
}

// Visible Gaussians (count > 0) -> (depth key, id) at their compacted position.
__global__ void compact_kernel(const uint32_t *__restrict__ counts, const uint32_t *__restrict__ pos, int64_t n,
                               const float4 *__restrict__ gview, uint32_t *__restrict__ keys,
                               uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || counts[i] == 0u) return;
    const uint32_t p = pos[i];
    keys[p] = __float_as_uint(gview[i].w);   // L >= 0: its bits sort like the value
    vals[p] = (uint32_t)i;
}

cudaError_t launch_compact(const uint32_t *counts, const uint32_t *pos, int64_t n, const float4 *gview,
                           uint32_t *keys, uint32_t *vals, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    compact_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(counts, pos, n, gview, keys, vals);
    note_launches(1);
    return cudaGetLastError();
}

__global__ void gather_u32_kernel(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                                  uint32_t *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

cudaError_t launch_gather(const uint32_t *src, const uint32_t *idx, int64_t n, uint32_t *dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    gather_u32_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(src, idx, n, dst);
    note_launches(1);
    return cudaGetLastError();
}

// Per-tile [begin, end) ranges from the tile-sorted key array: a tile's range
// starts where its key differs from the one before and ends where it differs
// from the one after.  Each thread takes four consecutive keys with one 16-byte
// load (keys 16-byte aligned) and reads the two neighbours once.
__global__ void ranges_kernel(const uint32_t *__restrict__ keys, int64_t n, uint2 *__restrict__ ranges) {
    const int64_t p0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (p0 >= n) return;
    uint32_t k[4];
    if (p0 + 4 <= n) {
        const uint4 v = *reinterpret_cast<const uint4 *>(keys + p0);
        k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) k[j] = p0 + j < n ? keys[p0 + j] : 0u;
    }
    uint32_t prev = p0 > 0 ? keys[p0 - 1] : ~k[0];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t p = p0 + j;
        if (p >= n) break;
        const uint32_t t = k[j];
        const uint32_t next = p + 1 >= n ? ~t : (j < 3 ? k[j + 1] : keys[p + 1]);
        if (prev != t) ranges[t].x = (uint32_t)p;
        if (next != t) ranges[t].y = (uint32_t)(p + 1);
        prev = t;
    }
}

cudaError_t launch_ranges(const uint32_t *keys, int64_t n, uint2 *ranges, int ntiles, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (e != cudaSuccess || n == 0) return e;
    if (reinterpret_cast<uintptr_t>(keys) % 16 != 0) return cudaErrorMisalignedAddress;
    ranges_kernel<<<(unsigned)div_up(div_up(n, 4), 256), 256, 0, s>>>(keys, n, ranges);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort

// Lanes of the warp holding the same digit as this lane (bit-sliced: one ballot
// per digit bit); lanes without an item (ok false) match only themselves.
__device__ __forceinline__ uint32_t digit_peers(uint32_t dig, int nbits, bool ok) {
    const uint32_t okm = __ballot_sync(0xffffffffu, ok);
    uint32_t peers = okm;
    for (int b = 0; b < nbits; ++b) {
        const bool on = (dig >> b) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, on);
        peers &= on ? v : ~v;
    }
    return ok ? peers : (1u << (threadIdx.x & 31));
}

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS_LARGE = 12;                 // 32-item rounds per warp per tile: 3072-item tiles
constexpr int RS_ROUNDS_SMALL = 4;                  // 1024-item tiles for sorts of up to RS_SMALL_N items
constexpr int64_t RS_SMALL_N = 1 << 20;             // (their 3072-item tiles would not fill the SMs)

// Resident scatter CTAs per SM of the tile size (queried once per device): the
// grid is one wave of them, each CTA walking its own contiguous chunk.
int rs_blocks_per_sm(bool small);

struct RsPlan {
    int64_t n;
    int blocks;
    int64_t chunk;
    int rounds;
};

RsPlan rs_plan(int64_t n) {
    RsPlan p;
    p.n = n;
    p.rounds = n <= RS_SMALL_N ? RS_ROUNDS_SMALL : RS_ROUNDS_LARGE;
    const int64_t tile = (int64_t)RS_THREADS * p.rounds;
    int64_t tiles = div_up(n, tile);
    int64_t blocks = std::min<int64_t>(tiles, (int64_t)rs_blocks_per_sm(p.rounds == RS_ROUNDS_SMALL) * num_sms());
    if (blocks < 1) blocks = 1;
    int64_t tiles_per = div_up(tiles, blocks);
    p.chunk = tiles_per * tile;
    p.blocks = (int)std::max<int64_t>(1, div_up(n, p.chunk));
    return p;
}

int64_t radix_scratch_words(int64_t n) {
    RsPlan p = rs_plan(n);
    int64_t cnt = 256LL * p.blocks;
    return cnt * 2 + scan_scratch_words(cnt);
}

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys, int64_t n, int64_t chunk,
                                                         int shift, uint32_t mask, uint32_t *__restrict__ counts) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = std::min<int64_t>(n, beg + chunk);
    for (int64_t i = beg + threadIdx.x; i < end; i += RS_THREADS) atomicAdd(&hist[(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    counts[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = hist[threadIdx.x];
}

template <int RS_ROUNDS>
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                                                           uint32_t *__restrict__ vout, int64_t n, int64_t chunk,
                                                           int shift, uint32_t mask,
                                                           const uint32_t *__restrict__ offsets) {
    __shared__ uint32_t running[256];               // global position of the next item of each digit
    __shared__ uint32_t wcount[RS_WARPS][256];      // per-warp digit counts, then per-warp local bases
    __shared__ uint32_t gofs[256];                  // global position minus local position, per digit
    __shared__ uint32_t wsum[RS_WARPS];
    constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
    __shared__ uint32_t s_k[RS_TILE], s_v[RS_TILE];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    running[threadIdx.x] = offsets[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) wcount[w][threadIdx.x] = 0u;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = std::min<int64_t>(n, beg + chunk);
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t t0 = beg; t0 < end; t0 += RS_TILE) {
        const int tn = (int)std::min<int64_t>(RS_TILE, end - t0);
        uint32_t k[RS_ROUNDS], v[RS_ROUNDS], rank[RS_ROUNDS];
        // 0. every load of the tile issued before any is used (all in flight at once)
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int li = wid * (RS_ROUNDS * 32) + r * 32 + lane;
            const bool ok = li < tn;
            k[r] = ok ? kin[t0 + li] : 0u;
            v[r] = ok ? vin[t0 + li] : 0u;
        }
        // 1. stable rank of each item among the earlier items of its warp with the same digit
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int li = wid * (RS_ROUNDS * 32) + r * 32 + lane;
            const bool ok = li < tn;
            const uint32_t dig = ok ? ((k[r] >> shift) & mask) : (256u + (uint32_t)lane);
            const uint32_t peers = digit_peers(dig, __popc(mask), ok);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0u;
            if (ok && lane == leader) {
                old = wcount[wid][dig];
                wcount[wid][dig] = old + (uint32_t)__popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[r] = ok ? old + (uint32_t)__popc(peers & lt) : 0xffffffffu;
            __syncwarp();
        }
        __syncthreads();
        // 2. digit d (thread d): tile total, exclusive scan over digits -> local bases
        const int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) tot += wcount[w][d];
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) before += w < wid ? wsum[w] : 0u;
        const uint32_t dbase = before + x - tot;          // first local slot of digit d in this tile
        {
            uint32_t b = dbase;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = wcount[w][d];
                wcount[w][d] = b;                          // now the warp's local base of digit d
                b += c;
            }
        }
        gofs[d] = running[d] - dbase;
        running[d] += tot;
        __syncthreads();
        // 3. items to their digit-sorted slot of the tile in shared memory
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            if (rank[r] != 0xffffffffu) {
                const uint32_t slot = wcount[wid][(k[r] >> shift) & mask] + rank[r];
                s_k[slot] = k[r];
                s_v[slot] = v[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wcount[w][threadIdx.x] = 0u;   // counts of the next tile
        // 4. write out in slot order: runs of one digit go to consecutive addresses
        for (int j = threadIdx.x; j < tn; j += RS_THREADS) {
            const uint32_t kk = s_k[j];
            const uint32_t dst = gofs[(kk >> shift) & mask] + (uint32_t)j;
            kout[dst] = kk;
            vout[dst] = s_v[j];
        }
        __syncthreads();
    }
}

// Sorts of at most RS_ONE_MAX items: one CTA does every pass in shared memory
// (one launch instead of an upsweep, a scan and a scatter per pass), with the
// same stable ranking as rs_downsweep: each warp ranks its items in lane order
// (digit_peers), the warps in order, the digits by an exclusive scan.
constexpr int RS_ONE_THREADS = 256;
constexpr int RS_ONE_WARPS = RS_ONE_THREADS / 32;
constexpr int RS_ONE_ROUNDS = 8;
constexpr int RS_ONE_MAX = RS_ONE_THREADS * RS_ONE_ROUNDS;   // 2048 items

__global__ void __launch_bounds__(RS_ONE_THREADS) rs_one_cta_kernel(uint32_t *__restrict__ keys,
                                                                    uint32_t *__restrict__ vals, int n, int begin_bit,
                                                                    int end_bit) {
    __shared__ uint32_t sk[2][RS_ONE_MAX], sv[2][RS_ONE_MAX];
    __shared__ uint32_t wcount[RS_ONE_WARPS][256];
    __shared__ uint32_t wsum[RS_ONE_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < n; i += RS_ONE_THREADS) {
        sk[0][i] = keys[i];
        sv[0][i] = vals[i];
    }
    int cur = 0;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const uint32_t mask = (1u << min(8, end_bit - shift)) - 1u;
#pragma unroll
        for (int w = 0; w < RS_ONE_WARPS; ++w) wcount[w][threadIdx.x] = 0u;
        __syncthreads();
        uint32_t k[RS_ONE_ROUNDS], v[RS_ONE_ROUNDS], rank[RS_ONE_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS_ONE_ROUNDS; ++r) {
            const int li = wid * (RS_ONE_ROUNDS * 32) + r * 32 + lane;
            const bool ok = li < n;
            k[r] = ok ? sk[cur][li] : 0u;
            v[r] = ok ? sv[cur][li] : 0u;
            const uint32_t dig = ok ? ((k[r] >> shift) & mask) : (256u + (uint32_t)lane);
            const uint32_t peers = digit_peers(dig, __popc(mask), ok);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0u;
            if (ok && lane == leader) {
                old = wcount[wid][dig];
                wcount[wid][dig] = old + (uint32_t)__popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[r] = ok ? old + (uint32_t)__popc(peers & lt) : 0xffffffffu;
            __syncwarp();
        }
        __syncthreads();
        // digit d (thread d): total, exclusive scan over digits, per-warp bases
        const int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < RS_ONE_WARPS; ++w) tot += wcount[w][d];
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < RS_ONE_WARPS; ++w) before += w < wid ? wsum[w] : 0u;
        uint32_t b = before + x - tot;
#pragma unroll
        for (int w = 0; w < RS_ONE_WARPS; ++w) {
            const uint32_t c = wcount[w][d];
            wcount[w][d] = b;
            b += c;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ONE_ROUNDS; ++r) {
            if (rank[r] != 0xffffffffu) {
                const uint32_t slot = wcount[wid][(k[r] >> shift) & mask] + rank[r];
                sk[cur ^ 1][slot] = k[r];
                sv[cur ^ 1][slot] = v[r];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int i = threadIdx.x; i < n; i += RS_ONE_THREADS) {
        keys[i] = sk[cur][i];
        vals[i] = sv[cur][i];
    }
}

int rs_blocks_per_sm(bool small) {
    static int cached[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int &c = cached[dev][small ? 1 : 0];
    if (!c) {
        int per_sm = 0;
        const cudaError_t e = small ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                          &per_sm, rs_downsweep<RS_ROUNDS_SMALL>, RS_THREADS, 0)
                                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                          &per_sm, rs_downsweep<RS_ROUNDS_LARGE>, RS_THREADS, 0);
        if (e != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 2;
        }
        c = std::min(per_sm, 8);
    }
    return c;
}

// Stable sort of (keys, vals) on bits [begin_bit, end_bit); result ends in
// (keys, vals) (alt_* are same-size scratch).  scratch: radix_scratch_words(n).
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *alt_keys, uint32_t *alt_vals, int64_t n,
                             int begin_bit, int end_bit, uint32_t *scratch, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return cudaSuccess;
    if (n <= RS_ONE_MAX) {
        rs_one_cta_kernel<<<1, RS_ONE_THREADS, 0, s>>>(keys, vals, (int)n, begin_bit, end_bit);
        note_launches(1);
        return cudaGetLastError();
    }
    const RsPlan p = rs_plan(n);
    const int64_t cnt = 256LL * p.blocks;
    uint32_t *counts = scratch, *offs = scratch + cnt, *scan_scr = scratch + 2 * cnt;
    uint32_t *ki = keys, *vi = vals, *ko = alt_keys, *vo = alt_vals;
    int passes = 0;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const int bits = std::min(8, end_bit - shift);
        const uint32_t mask = (1u << bits) - 1u;
        rs_upsweep<<<p.blocks, RS_THREADS, 0, s>>>(ki, n, p.chunk, shift, mask, counts);
        note_launches(1);
        cudaError_t e = exclusive_scan(counts, offs, cnt, scan_scr, 0, s);
        if (e != cudaSuccess) return e;
        if (p.rounds == RS_ROUNDS_SMALL)
            rs_downsweep<RS_ROUNDS_SMALL><<<p.blocks, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, p.chunk, shift, mask, offs);
        else
            rs_downsweep<RS_ROUNDS_LARGE><<<p.blocks, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, p.chunk, shift, mask, offs);
        note_launches(1);
        std::swap(ki, ko);
        std::swap(vi, vo);
        ++passes;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ki, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

}  // namespace conegs
