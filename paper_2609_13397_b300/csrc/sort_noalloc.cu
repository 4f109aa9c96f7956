// conegs_radix_sort_pairs_noalloc: the library's stable LSD radix sort with
// its scratch in a fixed device array instead of allocated memory.
//
// Why: some callers cannot allocate device memory when they sort.  Their
// device memory may be entirely reserved by another allocator (a framework's
// caching allocator), so a cudaMalloc would fail or fragment it; or they run
// in a latency-critical loop that must never block on, or fail in, an
// allocation.  This entry point lets them sort without touching any
// allocator: the caller passes the keys and values, and the scratch (the
// alternate key/value buffers and the digit counters) lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
//
// Limits and rules (also stated in include/conegs.h):
//   * at most NOALLOC_MAX_ITEMS pairs per call (262,144); larger calls are
//     rejected with CONEGS_ERR_ARG;
//   * the first call on a device looks up the array's device address on that
//     device (cudaGetSymbolAddress with that device current) and caches it;
//     make that first call before any stream capture;
//   * every call shares the one array and it keeps the last call's contents:
//     calls whose work overlaps on the GPU race with each other and must be
//     ordered by the caller (same stream, or events).  Nothing in the array
//     needs to start at zero: each pass writes every counter and buffer
//     entry it later reads.
#include <cstdio>
#include <mutex>

#include "../../include/conegs.h"
#include "common.cuh"

namespace conegs {
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *alt_keys, uint32_t *alt_vals, int64_t n,
                             int begin_bit, int end_bit, uint32_t *scratch, cudaStream_t s);
int64_t radix_scratch_words(int64_t n);
void set_error_message(const char *msg);
}  // namespace conegs

namespace {

constexpr int64_t NOALLOC_MAX_ITEMS = 1 << 18;
// digit counters + offsets of at most 256 sort blocks (2^18 items in 1024-item
// tiles), plus the scan scratch for them
constexpr int64_t NOALLOC_COUNTER_WORDS = 2 * 256 * 256 + 256;
constexpr int64_t NOALLOC_WORDS = 2 * NOALLOC_MAX_ITEMS + NOALLOC_COUNTER_WORDS;

static __device__ __align__(256) uint32_t g_sort_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
uint32_t *g_scratch_dev[MAX_DEVICES] = {nullptr};

conegs_status fail_msg(conegs_status st, const char *msg) {
    conegs::set_error_message(msg);
    return st;
}

}  // namespace

extern "C" conegs_status conegs_radix_sort_pairs_noalloc(uint32_t *keys, uint32_t *values, int64_t n,
                                                         int begin_bit, int end_bit, void *stream) {
    if (n < 0 || (n > 0 && (!keys || !values)))
        return fail_msg(CONEGS_ERR_ARG, "radix_sort_pairs_noalloc: bad argument");
    if (begin_bit < 0 || end_bit > 32 || begin_bit > end_bit)
        return fail_msg(CONEGS_ERR_ARG, "radix_sort_pairs_noalloc: bad bit range");
    if (n > NOALLOC_MAX_ITEMS)
        return fail_msg(CONEGS_ERR_ARG,
                        "radix_sort_pairs_noalloc: n exceeds the fixed scratch limit of 262144 pairs");
    if (n <= 1) return CONEGS_OK;
    if (conegs::radix_scratch_words(n) > NOALLOC_COUNTER_WORDS)
        return fail_msg(CONEGS_ERR_ARG, "radix_sort_pairs_noalloc: counter scratch too small for n");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail_msg(CONEGS_ERR_CUDA, "radix_sort_pairs_noalloc: no usable current device");
    uint32_t *base = nullptr;
    {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail_msg(CONEGS_ERR_CUDA, "radix_sort_pairs_noalloc: cudaGetSymbolAddress failed");
            }
            g_scratch_dev[dev] = static_cast<uint32_t *>(p);
        }
        base = g_scratch_dev[dev];
    }
    cudaError_t e = conegs::radix_sort_pairs(keys, values, base, base + NOALLOC_MAX_ITEMS, n, begin_bit, end_bit,
                                             base + 2 * NOALLOC_MAX_ITEMS, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        // the launch check can also surface an earlier, unrelated asynchronous fault: name the error
        char msg[192];
        snprintf(msg, sizeof msg, "radix_sort_pairs_noalloc: CUDA error after the sort launches: %s",
                 cudaGetErrorString(e));
        return fail_msg(CONEGS_ERR_CUDA, msg);
    }
    return CONEGS_OK;
}
