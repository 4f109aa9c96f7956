// C ABI of the library (include/conegs.h): contexts, views, scratch memory
// and the render pipeline
//   K1 ray table + tile cones (set_camera)
//   K2a scene cache (set_scene)
//   K2b view records -> K3 count -> scan/compact -> K4 depth sort ->
//   K3 emit -> K4 tile sort -> ranges -> K5 raster (render)
//   K6/K7 adjoint (render_backward)
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/conegs.h"
#include "raster.cuh"

namespace conegs {
// launchers defined in the other translation units
cudaError_t launch_ray_table(const CamParams &c, float *d, float *dx, float *dy, uint8_t *valid, cudaStream_t s);
cudaError_t launch_tile_tables(const CamParams &c, float *table, float *super, float *mcam, cudaStream_t s);
cudaError_t launch_footprint_min(const CamParams &c, const float *d, const float *dx, const float *dy,
                                 const uint8_t *valid, float *out, cudaStream_t s);
cudaError_t launch_gauss_scene_rule(const SceneParams &sp, float *binrec, cudaStream_t s);
cudaError_t launch_bin_count(const CamParams &c, const float *binrec, const float4 *gview, const float2 *gcone,
                             const uint8_t *gflag, const float *table, const float *super, const float *mcam,
                             float mzf, int64_t n, uint32_t *counts, uint4 *cache, uint32_t *blist,
                             unsigned long long *bcursor, unsigned long long bcap, const float4 *gell,
                             const float *ut_means, const float *ut_W, const float *ut_sig_eff, cudaStream_t s);
cudaError_t launch_bin_emit(const CamParams &c, const float *binrec, const float4 *gview, const float2 *gcone,
                            const uint8_t *gflag, const float *table, const float *super, const float *mcam,
                            float mzf, int64_t n_sorted, const uint32_t *order, const uint32_t *offsets,
                            const uint4 *cache, const uint32_t *blist, uint32_t *out_tile, uint32_t *out_gid,
                            const float4 *gell, bool ut, cudaStream_t s);
cudaError_t launch_scene_cache(const SceneParams &sp, float *W, float *sig_eff, cudaStream_t s);
cudaError_t launch_view_records(const CamParams &c, const SceneParams &sp, const float *mcam, float mzf,
                                int fov_cull, int pretest, int pixtest, int dilute, float4 *rec, float4 *gview,
                                float2 *gcone, uint8_t *gflag, float4 *gell, unsigned long long *nflat,
                                uint8_t *gflat, cudaStream_t s);
int64_t scan_scratch_words(int64_t n);
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, int pred,
                           cudaStream_t s);
cudaError_t sum_counts(const uint32_t *in, int64_t n, unsigned long long *d_two, const uint8_t *flag,
                       unsigned long long *d_flagged, cudaStream_t s);
cudaError_t launch_compact(const uint32_t *counts, const uint32_t *pos, int64_t n, const float4 *gview,
                           uint32_t *keys, uint32_t *vals, cudaStream_t s);
cudaError_t launch_gather(const uint32_t *src, const uint32_t *idx, int64_t n, uint32_t *dst, cudaStream_t s);
cudaError_t launch_ranges(const uint32_t *keys, int64_t n, uint2 *ranges, int ntiles, cudaStream_t s);
int64_t radix_scratch_words(int64_t n);
// Scratch words of a render's two radix sorts (M depth keys, Pn tile ids).
static int64_t sort_scratch_words(int64_t M, int64_t Pn) {
    return std::max(radix_scratch_words(std::max<int64_t>(M, 1)), radix_scratch_words(std::max<int64_t>(Pn, 1)));
}
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *alt_keys, uint32_t *alt_vals, int64_t n,
                             int begin_bit, int end_bit, uint32_t *scratch, cudaStream_t s);
cudaError_t launch_floor(const CamParams *cams_dev, int nv, const float *means, int64_t n, float *rho2,
                         cudaStream_t s);
cudaError_t launch_raster_split(const RasterArgs &a, int ntiles, bool filter, uint32_t *scratch,
                                uint32_t *scan_scratch, cudaStream_t s, cudaEvent_t main0, cudaEvent_t main1);
cudaError_t launch_raster_tstar(const RasterArgs &a, int ntiles, bool filter, cudaStream_t s);
cudaError_t launch_flat_pairs(const RasterArgs &a, const uint32_t *tiles, int64_t npairs, const uint8_t *gflat,
                              uint32_t *slot_of, uint32_t *slot_pair, unsigned long long *counter, int64_t nslots,
                              float *flat_T, float *flat_G, bool filter, cudaStream_t s);
cudaError_t launch_backward(const RasterArgs &a, int ntiles, bool filter, uint32_t *split_scratch,
                            const float *dL_drgb, const float *dL_dT, const float *final_T, float *g_rec,
                            cudaStream_t s);
cudaError_t launch_backward_params(const CamParams &c, const SceneParams &sp, const float *g_rec,
                                   const uint8_t *gflag, const float4 *gview, float *g_means, float *g_log_scales,
                                   float *g_quats, float *g_logits, float *g_sh, cudaStream_t s);
}  // namespace conegs

using namespace conegs;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace conegs {
// Lets other translation units of the library report a message through
// conegs_last_error().
void set_error_message(const char *msg) { g_last_error = msg; }
static std::atomic<long long> g_launches{0};
void note_launches(int k) { g_launches += k; }
long long launches_so_far() { return g_launches.load(); }
}  // namespace conegs

namespace {

}  // namespace

namespace conegs {
int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        sms[dev] = v;
    }
    return sms[dev];
}
}  // namespace conegs

namespace {

conegs_status fail(conegs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                                  \
    do {                                                                                                \
        cudaError_t _e = (expr);                                                                        \
        if (_e != cudaSuccess) return fail(CONEGS_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                                           __FILE__, __LINE__);                                         \
    } while (0)

#define TRY(expr)                              \
    do {                                       \
        conegs_status _s = (expr);             \
        if (_s != CONEGS_OK) return _s;        \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard() {
        if (prev_ != dev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0, dev_ = 0;
};

}  // namespace

struct conegs_ctx {
    int device = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    std::mutex mu;
    // scene
    SceneParams sp{};
    bool has_scene = false;
    uint64_t scene_gen = 0;
    DevBuf W, sig_eff, binrec;
    cudaEvent_t scene_ready = nullptr;
    std::vector<conegs_view *> views;
};

struct conegs_view {
    conegs_ctx *ctx = nullptr;
    CamParams cam{};
    bool has_cam = false;
    DevBuf d, dx, dy, valid, table, super, mcam, bincache, binlist;
    uint64_t list_want = 0;   // tile ids the last count pass wanted to keep in binlist
    long long launches0 = 0;  // launch counter at the start of the current render
    // per-render scratch
    DevBuf rec, gview, gcone, gflag, gell, counts, vispos, scan_scr, dkeys, dvals, dkeys_alt, dvals_alt, sorted_counts, offsets;
    DevBuf pair_tile, pair_gid, pair_tile_alt, pair_gid_alt, ranges, last, sums, rs_scr, tmp_rgb, tmp_T;
    DevBuf g_rec, keep_T, split, gflat, flat_slot, flat_pair, flat_T, flat_G;
    int64_t n_flat_pairs = 0;
    // a count pass run ahead of the render (conegs_render_count): its flags and scene
    bool counted = false;
    unsigned counted_flags = 0;
    uint64_t counted_gen = 0;
    unsigned long long *h_sums = nullptr;   // pinned
    int64_t n_visible = 0, n_pairs = 0, n_valid = 0, n_launches = 0, n_flat = 0;
    bool has_forward = false;
    unsigned last_flags = 0;
    uint64_t forward_gen = 0;
    cudaEvent_t done = nullptr;
    cudaEvent_t prof[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool profiled = false;
    DevBuf evaluated;
    cudaStream_t last_stream = nullptr;
    bool has_stream = false;
    // pipelined host renders: two device staging images used in turn, their copies
    // to the host on a stream of the view's own, each marked done by copied[k]
    DevBuf stage_rgb[2], stage_T[2];
    int stage = 0;
    bool stage_pending[2] = {false, false};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t rendered = nullptr;
};

namespace {

conegs_status ensure(conegs_ctx *ctx, DevBuf &b, size_t need, cudaStream_t s) {
    if (need <= b.bytes) return CONEGS_OK;
    size_t want = std::max<size_t>(need + need / 4, 256);
    if (ctx->budget) {
        size_t cur = ctx->used.load();
        if (cur - b.bytes + want > ctx->budget) {
            want = need;
            if (cur - b.bytes + want > ctx->budget)
                return fail(CONEGS_ERR_BUDGET, "memory budget exceeded: need %zu more bytes (budget %zu, in use %zu)",
                            want - b.bytes, ctx->budget, cur);
        }
    }
    if (b.p) {
        cudaError_t e = cudaFreeAsync(b.p, s);
        if (e != cudaSuccess) return fail(CONEGS_ERR_CUDA, "cudaFreeAsync: %s", cudaGetErrorString(e));
        ctx->used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, want, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CONEGS_ERR_OOM, "cudaMallocAsync(%zu bytes): %s", want, cudaGetErrorString(e));
    }
    b.p = p;
    b.bytes = want;
    ctx->used += want;
    return CONEGS_OK;
}

void release(conegs_ctx *ctx, DevBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        ctx->used -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

// Serialise a view's work across the streams it is used on.
conegs_status view_begin(conegs_view *v, cudaStream_t s) {
    if (v->has_stream && v->last_stream != s) CUDA_TRY(cudaStreamWaitEvent(s, v->done, 0));
    return CONEGS_OK;
}

conegs_status view_end(conegs_view *v, cudaStream_t s) {
    CUDA_TRY(cudaEventRecord(v->done, s));
    v->last_stream = s;
    v->has_stream = true;
    return CONEGS_OK;
}

int bits_for(int64_t n) {
    int b = 0;
    while ((1LL << b) < n) ++b;
    return std::max(b, 1);
}

float kb_P_host(const float k[4], float th) {
    // FP32 rule (no contraction: the host compiler runs with -ffp-contract=off)
    float t2 = th * th;
    float p = ((k[3] * t2 + k[2]) * t2 + k[1]) * t2 + k[0];
    return th * (1.0f + t2 * p);
}

// Stretch envelope of the KB projection on the sphere: the image moves by at most
// max(r'(theta), r(theta)/sin(theta)) per unit of arc (radial and tangential),
// so lip[j] bounds it on [0, theta_lim j/16] (dense sampling, 1% headroom).
void kb_lipschitz(const float k[4], float thlim, float lip[17]) {
    double env = 1.0;
    lip[0] = 1.01f;
    for (int j = 1; j <= 16; ++j) {
        const double a = (double)thlim * (j - 1) / 16, b = (double)thlim * j / 16;
        for (int i = 0; i <= 2000; ++i) {
            const double th = a + (b - a) * i / 2000, t2 = th * th;
            const double r = th * (1 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
            const double dr = 1 + t2 * (3 * k[0] + t2 * (5 * k[1] + t2 * (7 * k[2] + t2 * 9 * k[3])));
            const double tang = th > 1e-9 ? r / std::sin(th) : 1.0;
            env = std::max(env, std::max(std::fabs(dr), std::fabs(tang)));
        }
        lip[j] = (float)(env * 1.01);
    }
}

float derive_theta_lim(const float k[4]) {
    const double thmax = 95.0 * M_PI / 180.0;
    const int steps = 200000;
    double prev = 0.0;
    for (int i = 0; i <= steps; ++i) {
        double th = thmax * i / steps, t2 = th * th;
        double slope = 1 + 3 * k[0] * t2 + 5 * k[1] * t2 * t2 + 7 * k[2] * t2 * t2 * t2 + 9 * k[3] * t2 * t2 * t2 * t2;
        if (slope < 0.25) return (float)prev;
        prev = th;
    }
    return (float)thmax;
}

}  // namespace

extern "C" {

const char *conegs_last_error(void) { return g_last_error.c_str(); }

const char *conegs_version(void) { return "conegs 0.1 sm_103a"; }

conegs_status conegs_create(conegs_ctx **out, int device, size_t mem_budget_bytes) {
    if (!out) return fail(CONEGS_ERR_ARG, "conegs_create: out is NULL");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(CONEGS_ERR_ARG, "conegs_create: bad device %d", device);
    DeviceGuard g(device);
    auto *ctx = new conegs_ctx();
    ctx->device = device;
    ctx->budget = mem_budget_bytes;
    cudaError_t e = cudaEventCreateWithFlags(&ctx->scene_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(CONEGS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return CONEGS_OK;
}

void conegs_view_destroy(conegs_view *v);

void conegs_destroy(conegs_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    std::vector<conegs_view *> vs;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        vs = ctx->views;
    }
    for (auto *v : vs) conegs_view_destroy(v);
    release(ctx, ctx->W);
    release(ctx, ctx->sig_eff);
    release(ctx, ctx->binrec);
    if (ctx->scene_ready) cudaEventDestroy(ctx->scene_ready);
    delete ctx;
}

conegs_status conegs_set_scene(conegs_ctx *ctx, int64_t n, const float *means, const float *log_scales,
                               const float *quats, const void *opacity_logits, const void *sh, int sh_degree,
                               int storage, const float *rho2, void *stream) {
    if (!ctx) return fail(CONEGS_ERR_ARG, "set_scene: ctx is NULL");
    if (n < 0 || n > (1LL << 31) - 1) return fail(CONEGS_ERR_ARG, "set_scene: bad n %lld", (long long)n);
    if (sh_degree < 0 || sh_degree > 3) return fail(CONEGS_ERR_ARG, "set_scene: sh_degree %d not in 0..3", sh_degree);
    if (storage < 0 || storage > 2) return fail(CONEGS_ERR_ARG, "set_scene: bad storage dtype %d", storage);
    if (n > 0 && (!means || !log_scales || !quats || !opacity_logits || !sh))
        return fail(CONEGS_ERR_ARG, "set_scene: NULL parameter array");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TRY(ensure(ctx, ctx->W, sizeof(float) * 9 * (size_t)std::max<int64_t>(n, 1), s));
    TRY(ensure(ctx, ctx->sig_eff, sizeof(float) * (size_t)std::max<int64_t>(n, 1), s));
    TRY(ensure(ctx, ctx->binrec, sizeof(float) * BINREC * (size_t)std::max<int64_t>(n, 1), s));
    SceneParams sp{};
    sp.n = n;
    sp.sh_degree = sh_degree;
    sp.storage = storage;
    sp.means = means;
    sp.log_scales = log_scales;
    sp.quats = quats;
    sp.rho2 = rho2;
    sp.logits = opacity_logits;
    sp.sh = sh;
    sp.W = ctx->W.as<float>();
    sp.sig_eff = ctx->sig_eff.as<float>();
    sp.binrec = ctx->binrec.as<float>();
    CUDA_TRY(launch_scene_cache(sp, ctx->W.as<float>(), ctx->sig_eff.as<float>(), s));
    CUDA_TRY(launch_gauss_scene_rule(sp, ctx->binrec.as<float>(), s));
    CUDA_TRY(cudaEventRecord(ctx->scene_ready, s));
    ctx->sp = sp;
    ctx->has_scene = true;
    ctx->scene_gen++;
    return CONEGS_OK;
}

conegs_status conegs_view_create(conegs_ctx *ctx, conegs_view **out) {
    if (!ctx || !out) return fail(CONEGS_ERR_ARG, "view_create: NULL argument");
    DeviceGuard g(ctx->device);
    auto *v = new conegs_view();
    v->ctx = ctx;
    cudaError_t e = cudaEventCreateWithFlags(&v->done, cudaEventDisableTiming);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaEventCreate(&v->prof[k]);
    if (e == cudaSuccess) e = cudaMallocHost(&v->h_sums, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        if (v->done) cudaEventDestroy(v->done);
        delete v;
        return fail(CONEGS_ERR_CUDA, "view_create: %s", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->views.push_back(v);
    }
    *out = v;
    return CONEGS_OK;
}

void conegs_view_destroy(conegs_view *v) {
    if (!v) return;
    conegs_ctx *ctx = v->ctx;
    DeviceGuard g(ctx->device);
    if (v->done) {
        cudaEventSynchronize(v->done);
        cudaEventDestroy(v->done);
    }
    if (v->copy_stream) {
        cudaStreamSynchronize(v->copy_stream);
        cudaStreamDestroy(v->copy_stream);
    }
    for (cudaEvent_t e : {v->copied[0], v->copied[1], v->rendered})
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        release(ctx, v->stage_rgb[k]);
        release(ctx, v->stage_T[k]);
    }
    DevBuf *bufs[] = {&v->d, &v->dx, &v->dy, &v->valid, &v->table, &v->super, &v->mcam, &v->rec, &v->gview, &v->gcone, &v->gflag, &v->gell, &v->bincache, &v->binlist,
                      &v->counts, &v->vispos, &v->scan_scr, &v->dkeys, &v->dvals, &v->dkeys_alt, &v->dvals_alt,
                      &v->sorted_counts, &v->offsets, &v->pair_tile, &v->pair_gid, &v->pair_tile_alt,
                      &v->pair_gid_alt, &v->ranges, &v->last, &v->sums, &v->rs_scr, &v->tmp_rgb, &v->tmp_T,
                      &v->g_rec, &v->keep_T, &v->split, &v->gflat, &v->flat_slot, &v->flat_pair, &v->flat_T,
                      &v->flat_G};
    for (DevBuf *b : bufs) release(ctx, *b);
    if (v->h_sums) cudaFreeHost(v->h_sums);
    for (int k = 0; k < 6; ++k)
        if (v->prof[k]) cudaEventDestroy(v->prof[k]);
    release(ctx, v->evaluated);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->views.erase(std::remove(ctx->views.begin(), ctx->views.end(), v), ctx->views.end());
    }
    delete v;
}

conegs_status conegs_set_camera(conegs_view *v, int model, int width, int height, const float *intr,
                                const float *dist, const float *c2w, float theta_lim, void *stream) {
    if (!v) return fail(CONEGS_ERR_ARG, "set_camera: view is NULL");
    if (model != CONEGS_PINHOLE && model != CONEGS_KB_FISHEYE)
        return fail(CONEGS_ERR_ARG, "set_camera: unknown camera model %d", model);
    if (width <= 0 || height <= 0 || (int64_t)width * height > (1LL << 30))
        return fail(CONEGS_ERR_ARG, "set_camera: bad size %dx%d", width, height);
    if (!intr) return fail(CONEGS_ERR_ARG, "set_camera: intrinsics is NULL");
    if (!(intr[0] > 0.0f) || !(intr[1] > 0.0f) || !std::isfinite(intr[2]) || !std::isfinite(intr[3]))
        return fail(CONEGS_ERR_ARG, "set_camera: focal lengths must be positive and finite");
    conegs_ctx *ctx = v->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    CamParams c{};
    c.model = model;
    c.W = width;
    c.H = height;
    c.tiles_x = (width + TILE - 1) / TILE;
    c.tiles_y = (height + TILE - 1) / TILE;
    c.supers_x = (c.tiles_x + SUPER - 1) / SUPER;
    c.supers_y = (c.tiles_y + SUPER - 1) / SUPER;
    c.fx = intr[0]; c.fy = intr[1]; c.cx = intr[2]; c.cy = intr[3];
    for (int i = 0; i < 4; ++i) c.k[i] = (model == CONEGS_KB_FISHEYE && dist) ? dist[i] : 0.0f;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.R[3 * r + k] = c2w ? c2w[4 * r + k] : (r == k ? 1.0f : 0.0f);
        c.o[r] = c2w ? c2w[4 * r + 3] : 0.0f;
    }
    if (model == CONEGS_KB_FISHEYE) {
        float th = theta_lim > 0.0f ? theta_lim : derive_theta_lim(c.k);
        if (!(th > 0.0f) || th > 3.2f) return fail(CONEGS_ERR_ARG, "set_camera: bad theta_lim %g", th);
        // theta_d must increase on [0, theta_lim]
        for (int i = 1; i <= 1000; ++i) {
            double t = (double)th * i / 1000, t2 = t * t;
            double slope = 1 + 3 * c.k[0] * t2 + 5 * c.k[1] * t2 * t2 + 7 * c.k[2] * t2 * t2 * t2 +
                           9 * c.k[3] * t2 * t2 * t2 * t2;
            if (!(slope > 0.0)) return fail(CONEGS_ERR_NOCONVERGE, "set_camera: theta_d not monotone below theta_lim");
        }
        c.thlim = th;
        float rl = kb_P_host(c.k, th);
        c.rlim2 = rl * rl;
        kb_lipschitz(c.k, th, c.lip);
    }
    TRY(view_begin(v, s));
    const size_t P = (size_t)width * height;
    const size_t nt = (size_t)c.tiles_x * c.tiles_y, ns = (size_t)c.supers_x * c.supers_y;
    TRY(ensure(ctx, v->d, sizeof(float) * 3 * P, s));
    TRY(ensure(ctx, v->dx, sizeof(float) * 3 * P, s));
    TRY(ensure(ctx, v->dy, sizeof(float) * 3 * P, s));
    TRY(ensure(ctx, v->valid, P, s));
    TRY(ensure(ctx, v->table, sizeof(float) * 6 * nt, s));
    TRY(ensure(ctx, v->super, sizeof(float) * 6 * ns, s));
    TRY(ensure(ctx, v->mcam, MCAM_FLOATS * sizeof(float), s));
    TRY(ensure(ctx, v->ranges, sizeof(uint2) * nt, s));
    TRY(ensure(ctx, v->last, sizeof(uint32_t) * P, s));
    CUDA_TRY(launch_ray_table(c, v->d.as<float>(), v->dx.as<float>(), v->dy.as<float>(), v->valid.as<uint8_t>(), s));
    CUDA_TRY(launch_tile_tables(c, v->table.as<float>(), v->super.as<float>(), v->mcam.as<float>(), s));
    CUDA_TRY(launch_footprint_min(c, v->d.as<float>(), v->dx.as<float>(), v->dy.as<float>(), v->valid.as<uint8_t>(),
                                  v->mcam.as<float>() + FP_MIN, s));
    v->cam = c;
    v->has_cam = true;
    v->counted = false;
    v->has_forward = false;
    // count valid pixels once (host copy of the mask is small relative to the table)
    if (model == CONEGS_PINHOLE) {
        v->n_valid = (int64_t)P;
    } else {
        std::vector<uint8_t> mask(P);
        CUDA_TRY(cudaMemcpyAsync(mask.data(), v->valid.p, P, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        int64_t cnt = 0;
        for (uint8_t m : mask) cnt += m;
        v->n_valid = cnt;
    }
    return view_end(v, s);
}

// Footprint variant of a render (flags), and the z/f variant's FP32 bound 1/(6 f_x^2)
// on (|dx|^2 + |dy|^2)/3 (0 for the others); the same op sequence as the oracle.
static int footprint_mode(unsigned flags) {
    return (flags & CONEGS_FILTER_ISO) ? FOOTPRINT_ISO : (flags & CONEGS_FILTER_ZF) ? FOOTPRINT_ZF : FOOTPRINT_OWN;
}

static float zf_bound(const CamParams &c, unsigned flags) {
    if (!(flags & CONEGS_FILTER_ZF)) return 0.0f;
    const float f2 = c.fx * c.fx;
    const float d6 = 6.0f * f2;
    return 1.0f / d6;
}

// The records of a pinhole view hold the pixel-space form of the pre-test unless
// the render asks for the ray-direction form.
static int pixel_pretest(const CamParams &c, unsigned flags) {
    return c.model == 0 && !(flags & CONEGS_PRETEST_RAY) ? 1 : 0;
}

static void set_footprint(RasterArgs &a, const CamParams &c, unsigned flags) {
    a.footprint = footprint_mode(flags);
    a.zax[0] = c.R[2];
    a.zax[1] = c.R[5];
    a.zax[2] = c.R[8];
    a.zf_scale = 0.5f / c.fx;
}

// A render runs in two halves around the one host synchronisation it needs:
// render_front enqueues the view records, the bin count and the pair/visible
// totals (copied to pinned host memory); render_back, after the stream has
// reached that copy, sizes the pair buffers from the totals and enqueues the
// sorts, the emit and the rasteriser.
static conegs_status render_front(conegs_view *v, unsigned flags, cudaStream_t s) {
    {
        const unsigned fp = flags & (CONEGS_FILTER_NONE | CONEGS_FILTER_ISO | CONEGS_FILTER_ZF);
        if (fp & (fp - 1u)) return fail(CONEGS_ERR_ARG, "render: FILTER_NONE, FILTER_ISO and FILTER_ZF exclude each other");
        if ((flags & CONEGS_ORDER_TSTAR) && (flags & CONEGS_KEEP_FOR_BACKWARD))
            return fail(CONEGS_ERR_ARG, "render: ORDER_TSTAR is forward only (no KEEP_FOR_BACKWARD)");
    }
    conegs_ctx *ctx = v->ctx;
    const CamParams &c = v->cam;
    const int64_t n = ctx->sp.n;
    CUDA_TRY(cudaStreamWaitEvent(s, ctx->scene_ready, 0));
    v->launches0 = launches_so_far();
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    TRY(ensure(ctx, v->rec, sizeof(float4) * REC_F4 * nn, s));
    TRY(ensure(ctx, v->gview, sizeof(float4) * nn, s));
    TRY(ensure(ctx, v->gcone, sizeof(float2) * nn, s));
    TRY(ensure(ctx, v->gell, 3 * sizeof(float4) * nn, s));
    TRY(ensure(ctx, v->gflag, nn, s));
    TRY(ensure(ctx, v->bincache, 3 * sizeof(uint4) * nn, s));
    TRY(ensure(ctx, v->counts, sizeof(uint32_t) * nn, s));
    TRY(ensure(ctx, v->vispos, sizeof(uint32_t) * nn, s));
    TRY(ensure(ctx, v->scan_scr, sizeof(uint32_t) * (size_t)scan_scratch_words((int64_t)nn), s));
    TRY(ensure(ctx, v->sums, 6 * sizeof(unsigned long long), s));
    TRY(ensure(ctx, v->gflat, nn, s));
    // optional: without room (or over the memory budget) the emit pass evaluates the rule again
    if (v->list_want > 0 && ensure(ctx, v->binlist, sizeof(uint32_t) * (size_t)v->list_want, s) != CONEGS_OK)
        v->list_want = 0;
    SceneParams sp = ctx->sp;
    const bool prof = (flags & CONEGS_PROFILE) != 0;
    if (prof) {
        TRY(ensure(ctx, v->evaluated, 3 * sizeof(unsigned long long), s));
        CUDA_TRY(cudaMemsetAsync(v->evaluated.p, 0, 3 * sizeof(unsigned long long), s));
        CUDA_TRY(cudaEventRecord(v->prof[0], s));
    }
    // sums: [0] pairs, [1] visible Gaussians, [2] kept-tile list entries wanted, [3] flat Gaussians,
    // [4] pairs of flat Gaussians, [5] scratch (flat slot counter)
    CUDA_TRY(cudaMemsetAsync(v->sums.as<unsigned long long>() + 2, 0, 2 * sizeof(unsigned long long), s));
    CUDA_TRY(launch_view_records(c, sp, v->mcam.as<float>(), zf_bound(c, flags), (flags & CONEGS_BIN_UT) ? 0 : 1,
                                 (flags & CONEGS_PRETEST_OFF) ? 0 : 1, pixel_pretest(c, flags),
                                 (flags & (CONEGS_FILTER_NONE | CONEGS_FILTER_ZF)) ? 0 : 1,
                                 v->rec.as<float4>(), v->gview.as<float4>(),
                                 v->gcone.as<float2>(), v->gflag.as<uint8_t>(), v->gell.as<float4>(),
                                 v->sums.as<unsigned long long>() + 3, v->gflat.as<uint8_t>(), s));
    {
        const bool ut = (flags & CONEGS_BIN_UT) != 0;
        const unsigned long long cap = std::min<unsigned long long>(v->binlist.bytes / sizeof(uint32_t), 0xffffffffull);
        CUDA_TRY(launch_bin_count(c, sp.binrec, v->gview.as<float4>(), v->gcone.as<float2>(), v->gflag.as<uint8_t>(),
                                  v->table.as<float>(), v->super.as<float>(), v->mcam.as<float>(),
                                  zf_bound(c, flags), n, v->counts.as<uint32_t>(), v->bincache.as<uint4>(),
                                  v->binlist.as<uint32_t>(), v->sums.as<unsigned long long>() + 2, cap,
                                  v->gell.as<float4>(), ut ? sp.means : nullptr, ut ? sp.W : nullptr,
                                  ut ? sp.sig_eff : nullptr, s));
    }
    CUDA_TRY(sum_counts(v->counts.as<uint32_t>(), n, v->sums.as<unsigned long long>(), v->gflat.as<uint8_t>(),
                        v->sums.as<unsigned long long>() + 4, s));
    CUDA_TRY(exclusive_scan(v->counts.as<uint32_t>(), v->vispos.as<uint32_t>(), n, v->scan_scr.as<uint32_t>(), 1, s));
    if (prof) CUDA_TRY(cudaEventRecord(v->prof[1], s));
    CUDA_TRY(cudaMemcpyAsync(v->h_sums, v->sums.p, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    return CONEGS_OK;
}

static conegs_status render_back(conegs_view *v, float *out_rgb, float *out_T, unsigned flags, cudaStream_t s) {
    conegs_ctx *ctx = v->ctx;
    const CamParams &c = v->cam;
    const int64_t n = ctx->sp.n;
    const int64_t P = (int64_t)c.W * c.H;
    const int nt = c.tiles_x * c.tiles_y;
    const SceneParams sp = ctx->sp;
    const bool prof = (flags & CONEGS_PROFILE) != 0;
    const uint64_t total = v->h_sums[0];
    const int64_t M = (int64_t)v->h_sums[1];
    const int64_t nflat = (int64_t)v->h_sums[3];
    const int64_t nflat_pairs = (int64_t)v->h_sums[4];
    // room the count pass wanted for kept tile lists: grown (with headroom) before the next render
    if (v->h_sums[2] > v->binlist.bytes / sizeof(uint32_t))
        v->list_want = std::min<uint64_t>(v->h_sums[2] + v->h_sums[2] / 4, 1ull << 28);
    if (total >= (1ULL << 31)) return fail(CONEGS_ERR_OVERFLOW, "render: %llu tile/Gaussian pairs exceed 2^31",
                                           (unsigned long long)total);
    const int64_t Pn = (int64_t)total;
    const size_t mm = (size_t)std::max<int64_t>(M, 1), pp = (size_t)std::max<int64_t>(Pn, 1);
    TRY(ensure(ctx, v->dkeys, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->dvals, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->dkeys_alt, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->dvals_alt, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->sorted_counts, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->offsets, sizeof(uint32_t) * mm, s));
    TRY(ensure(ctx, v->pair_tile, sizeof(uint32_t) * pp, s));
    TRY(ensure(ctx, v->pair_gid, sizeof(uint32_t) * pp, s));
    TRY(ensure(ctx, v->pair_tile_alt, sizeof(uint32_t) * pp, s));
    TRY(ensure(ctx, v->pair_gid_alt, sizeof(uint32_t) * pp, s));
    // the two sorts (depth keys of M items, tile ids of Pn) plan their grids apart, and a
    // small sort may use more CTAs than a larger one: room for whichever needs more
    TRY(ensure(ctx, v->rs_scr, sizeof(uint32_t) * (size_t)sort_scratch_words(M, Pn), s));
    TRY(ensure(ctx, v->scan_scr, sizeof(uint32_t) * (size_t)scan_scratch_words(std::max<int64_t>(M, n)), s));
    CUDA_TRY(launch_compact(v->counts.as<uint32_t>(), v->vispos.as<uint32_t>(), n, v->gview.as<float4>(),
                            v->dkeys.as<uint32_t>(), v->dvals.as<uint32_t>(), s));
    CUDA_TRY(radix_sort_pairs(v->dkeys.as<uint32_t>(), v->dvals.as<uint32_t>(), v->dkeys_alt.as<uint32_t>(),
                              v->dvals_alt.as<uint32_t>(), M, 0, 32, v->rs_scr.as<uint32_t>(), s));
    CUDA_TRY(launch_gather(v->counts.as<uint32_t>(), v->dvals.as<uint32_t>(), M, v->sorted_counts.as<uint32_t>(), s));
    CUDA_TRY(exclusive_scan(v->sorted_counts.as<uint32_t>(), v->offsets.as<uint32_t>(), M, v->scan_scr.as<uint32_t>(),
                            0, s));
    CUDA_TRY(launch_bin_emit(c, sp.binrec, v->gview.as<float4>(), v->gcone.as<float2>(), v->gflag.as<uint8_t>(),
                             v->table.as<float>(), v->super.as<float>(), v->mcam.as<float>(), zf_bound(c, flags), M,
                             v->dvals.as<uint32_t>(), v->offsets.as<uint32_t>(), v->bincache.as<uint4>(),
                             v->binlist.as<uint32_t>(), v->pair_tile.as<uint32_t>(), v->pair_gid.as<uint32_t>(),
                             v->gell.as<float4>(), (flags & CONEGS_BIN_UT) != 0, s));
    CUDA_TRY(radix_sort_pairs(v->pair_tile.as<uint32_t>(), v->pair_gid.as<uint32_t>(), v->pair_tile_alt.as<uint32_t>(),
                              v->pair_gid_alt.as<uint32_t>(), Pn, 0, bits_for(nt), v->rs_scr.as<uint32_t>(), s));
    CUDA_TRY(launch_ranges(v->pair_tile.as<uint32_t>(), Pn, v->ranges.as<uint2>(), nt, s));
    if (prof) CUDA_TRY(cudaEventRecord(v->prof[2], s));
    RasterArgs a{};
    a.W = c.W;
    a.H = c.H;
    a.tiles_x = c.tiles_x;
    a.ranges = v->ranges.as<uint2>();
    a.gids = v->pair_gid.as<uint32_t>();
    a.rec = v->rec.as<float4>();
    a.d = v->d.as<float>();
    a.dx = v->dx.as<float>();
    a.dy = v->dy.as<float>();
    a.valid = v->valid.as<uint8_t>();
    a.out_rgb = out_rgb;
    a.out_T = out_T;
    a.last = v->last.as<uint32_t>();
    a.additive = (flags & CONEGS_COMP_ADDITIVE) ? 1 : 0;
    a.pixtest = pixel_pretest(c, flags);
    set_footprint(a, c, flags);
    if (nflat_pairs > 0) {
        // the pairs of flat Gaussians: responses (and their derivatives, for the adjoint) in FP64
        const bool adj = (flags & CONEGS_KEEP_FOR_BACKWARD) != 0;
        const size_t F = (size_t)nflat_pairs;
        TRY(ensure(ctx, v->flat_slot, sizeof(uint32_t) * pp, s));
        TRY(ensure(ctx, v->flat_pair, sizeof(uint32_t) * F, s));
        TRY(ensure(ctx, v->flat_T, sizeof(float) * TILE_PX * F, s));
        if (adj) TRY(ensure(ctx, v->flat_G, sizeof(float) * 13 * TILE_PX * F, s));
        CUDA_TRY(launch_flat_pairs(a, v->pair_tile.as<uint32_t>(), Pn, v->gflat.as<uint8_t>(),
                                   v->flat_slot.as<uint32_t>(), v->flat_pair.as<uint32_t>(),
                                   v->sums.as<unsigned long long>() + 5, nflat_pairs, v->flat_T.as<float>(),
                                   adj ? v->flat_G.as<float>() : nullptr, !(flags & CONEGS_FILTER_NONE), s));
        a.flat_slot = v->flat_slot.as<uint32_t>();
        a.flat_T = v->flat_T.as<float>();
        a.flat_G = adj ? v->flat_G.as<float>() : nullptr;
    }
    if (flags & CONEGS_KEEP_FOR_BACKWARD) {
        TRY(ensure(ctx, v->keep_T, sizeof(float) * (size_t)std::max<int64_t>(P, 1), s));
        a.keep_T = v->keep_T.as<float>();
    }
    a.evaluated = prof ? v->evaluated.as<unsigned long long>() : nullptr;
    TRY(ensure(ctx, v->split, sizeof(uint32_t) * (size_t)split_scratch_words(nt), s));
    TRY(ensure(ctx, v->scan_scr, sizeof(uint32_t) * (size_t)scan_scratch_words(std::max<int64_t>(std::max<int64_t>(M, n), nt)), s));
    if (flags & CONEGS_ORDER_TSTAR) {
        if (prof) CUDA_TRY(cudaEventRecord(v->prof[4], s));
        CUDA_TRY(launch_raster_tstar(a, nt, !(flags & CONEGS_FILTER_NONE), s));
        if (prof) CUDA_TRY(cudaEventRecord(v->prof[5], s));
    } else {
        CUDA_TRY(launch_raster_split(a, nt, !(flags & CONEGS_FILTER_NONE), v->split.as<uint32_t>(),
                                     v->scan_scr.as<uint32_t>(), s,
                                     prof ? v->prof[4] : nullptr, prof ? v->prof[5] : nullptr));
    }
    if (prof) {
        CUDA_TRY(cudaEventRecord(v->prof[3], s));
        CUDA_TRY(cudaMemcpyAsync(v->h_sums + 5, v->evaluated.p, 3 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
    }
    v->profiled = prof;
    v->n_launches = launches_so_far() - v->launches0;
    v->n_visible = M;
    v->n_pairs = Pn;
    v->n_flat = nflat;
    v->n_flat_pairs = nflat_pairs;
    v->last_flags = flags;
    v->has_forward = true;
    v->forward_gen = ctx->scene_gen;
    return CONEGS_OK;
}

static conegs_status render_impl(conegs_view *v, float *out_rgb, float *out_T, unsigned flags, cudaStream_t s) {
    const bool reuse = v->counted && v->counted_flags == flags && v->counted_gen == v->ctx->scene_gen;
    v->counted = false;
    if (!reuse) {
        TRY(render_front(v, flags, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return render_back(v, out_rgb, out_T, flags, s);
}

// Device bytes the back half of a render sizes from the counts: sort buffers of the
// visible Gaussians and of the pairs, tile ranges and split state, per-pixel state,
// and the FP64 responses of flat Gaussians' pairs.
static size_t back_bytes(const conegs_view *v, unsigned flags) {
    const int64_t n = v->ctx->sp.n;
    const int64_t M = (int64_t)v->h_sums[1], Pn = (int64_t)v->h_sums[0], F = (int64_t)v->h_sums[4];
    const int64_t nt = (int64_t)v->cam.tiles_x * v->cam.tiles_y, P = (int64_t)v->cam.W * v->cam.H;
    size_t b = sizeof(uint32_t) * (6 * (size_t)M + 4 * (size_t)Pn);
    b += sizeof(uint32_t) * (size_t)sort_scratch_words(M, Pn);
    b += sizeof(uint32_t) * (size_t)scan_scratch_words(std::max<int64_t>(std::max<int64_t>(M, n), nt));
    b += sizeof(uint32_t) * (size_t)split_scratch_words((int)nt) + sizeof(uint2) * (size_t)nt;
    b += sizeof(float) * 4 * (size_t)P + sizeof(uint32_t) * (size_t)P;
    if (flags & CONEGS_KEEP_FOR_BACKWARD) b += sizeof(float) * (size_t)P + sizeof(float) * 16 * (size_t)n;
    if (F > 0) {
        b += sizeof(uint32_t) * ((size_t)Pn + (size_t)F) + sizeof(float) * TILE_PX * (size_t)F;
        if (flags & CONEGS_KEEP_FOR_BACKWARD) b += sizeof(float) * 13 * TILE_PX * (size_t)F;
    }
    return b;
}

conegs_status conegs_render_count(conegs_view *v, unsigned flags, int64_t *pairs_host, size_t *bytes_host,
                                  void *stream) {
    if (!v) return fail(CONEGS_ERR_ARG, "render_count: NULL view");
    if (!v->has_cam) return fail(CONEGS_ERR_STATE, "render_count: set_camera was not called on this view");
    if (!v->ctx->has_scene) return fail(CONEGS_ERR_STATE, "render_count: set_scene was not called");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(view_begin(v, s));
    v->counted = false;
    conegs_status st = render_front(v, flags, s);
    if (st == CONEGS_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(CONEGS_ERR_CUDA, "render_count: %s", cudaGetErrorString(e));
    }
    if (st != CONEGS_OK) {
        view_end(v, s);
        return st;
    }
    v->counted = true;
    v->counted_flags = flags;
    v->counted_gen = v->ctx->scene_gen;
    if (pairs_host) *pairs_host = (int64_t)v->h_sums[0];
    if (bytes_host) *bytes_host = back_bytes(v, flags);
    return view_end(v, s);
}

conegs_status conegs_render(conegs_view *v, float *out_rgb, float *out_T, unsigned flags, void *stream) {
    if (!v || !out_rgb) return fail(CONEGS_ERR_ARG, "render: NULL argument");
    if (!v->has_cam) return fail(CONEGS_ERR_STATE, "render: set_camera was not called on this view");
    if (!v->ctx->has_scene) return fail(CONEGS_ERR_STATE, "render: set_scene was not called");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(view_begin(v, s));
    conegs_status st = render_impl(v, out_rgb, out_T, flags, s);
    if (st != CONEGS_OK) {
        v->has_forward = false;
        view_end(v, s);
        return st;
    }
    return view_end(v, s);
}

conegs_status conegs_render_batch(int n, conegs_view *const *views, float *const *out_rgb, float *const *out_T,
                                  unsigned flags, void *const *streams) {
    if (n < 0 || (n > 0 && (!views || !out_rgb))) return fail(CONEGS_ERR_ARG, "render_batch: bad argument");
    for (int i = 0; i < n; ++i) {
        if (!views[i] || !out_rgb[i]) return fail(CONEGS_ERR_ARG, "render_batch: NULL view or output %d", i);
        if (!views[i]->has_cam) return fail(CONEGS_ERR_STATE, "render_batch: view %d has no camera", i);
        if (views[i]->ctx != views[0]->ctx) return fail(CONEGS_ERR_ARG, "render_batch: views of different contexts");
        for (int j = 0; j < i; ++j)
            if (views[j] == views[i]) return fail(CONEGS_ERR_ARG, "render_batch: view %d repeated", i);
    }
    if (n == 0) return CONEGS_OK;
    if (!views[0]->ctx->has_scene) return fail(CONEGS_ERR_STATE, "render_batch: set_scene was not called");
    DeviceGuard g(views[0]->ctx->device);
    auto stream_of = [&](int i) { return streams ? (cudaStream_t)streams[i] : (cudaStream_t)0; };
    int started = 0;
    conegs_status st = CONEGS_OK;
    for (; started < n; ++started) {
        conegs_view *v = views[started];
        const cudaStream_t s = stream_of(started);
        v->has_forward = false;
        st = view_begin(v, s);
        if (st == CONEGS_OK) st = render_front(v, flags, s);
        if (st != CONEGS_OK) {
            view_end(v, s);
            break;
        }
    }
    // every started view must reach its back half or be closed, even after an error
    for (int i = 0; i < started; ++i) {
        conegs_view *v = views[i];
        const cudaStream_t s = stream_of(i);
        if (st == CONEGS_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = fail(CONEGS_ERR_CUDA, "render_batch: %s", cudaGetErrorString(e));
        }
        if (st == CONEGS_OK) {
            st = render_back(v, out_rgb[i], out_T ? out_T[i] : nullptr, flags, s);
            if (st != CONEGS_OK) v->has_forward = false;
        }
        view_end(v, s);
    }
    return st;
}

conegs_status conegs_render_host_batch(int n, conegs_view *const *views, float *const *out_rgb_host,
                                       float *const *out_T_host, unsigned flags, void *const *streams) {
    if (n < 0 || (n > 0 && (!views || !out_rgb_host))) return fail(CONEGS_ERR_ARG, "render_host_batch: bad argument");
    if (n == 0) return CONEGS_OK;
    std::vector<float *> drgb((size_t)n), dT((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!views[i] || !out_rgb_host[i]) return fail(CONEGS_ERR_ARG, "render_host_batch: NULL view or output %d", i);
        if (!views[i]->has_cam) return fail(CONEGS_ERR_STATE, "render_host_batch: view %d has no camera", i);
        conegs_view *v = views[i];
        DeviceGuard g(v->ctx->device);
        const cudaStream_t s = streams ? (cudaStream_t)streams[i] : (cudaStream_t)0;
        const size_t P = (size_t)v->cam.W * v->cam.H;
        TRY(view_begin(v, s));
        TRY(ensure(v->ctx, v->tmp_rgb, sizeof(float) * 3 * P, s));
        TRY(ensure(v->ctx, v->tmp_T, sizeof(float) * P, s));
        TRY(view_end(v, s));
        drgb[(size_t)i] = v->tmp_rgb.as<float>();
        dT[(size_t)i] = v->tmp_T.as<float>();
    }
    TRY(conegs_render_batch(n, views, drgb.data(), dT.data(), flags, streams));
    DeviceGuard g(views[0]->ctx->device);
    for (int i = 0; i < n; ++i) {
        conegs_view *v = views[i];
        const cudaStream_t s = streams ? (cudaStream_t)streams[i] : (cudaStream_t)0;
        const size_t P = (size_t)v->cam.W * v->cam.H;
        CUDA_TRY(cudaMemcpyAsync(out_rgb_host[i], v->tmp_rgb.p, sizeof(float) * 3 * P, cudaMemcpyDeviceToHost, s));
        if (out_T_host && out_T_host[i])
            CUDA_TRY(cudaMemcpyAsync(out_T_host[i], v->tmp_T.p, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
        TRY(view_end(v, s));
    }
    for (int i = 0; i < n; ++i) CUDA_TRY(cudaStreamSynchronize(streams ? (cudaStream_t)streams[i] : (cudaStream_t)0));
    return CONEGS_OK;
}

conegs_status conegs_render_host_batch_async(int n, conegs_view *const *views, float *const *out_rgb_host,
                                             float *const *out_T_host, unsigned flags, void *const *streams) {
    if (n < 0 || (n > 0 && (!views || !out_rgb_host)))
        return fail(CONEGS_ERR_ARG, "render_host_batch_async: bad argument");
    if (n == 0) return CONEGS_OK;
    std::vector<float *> drgb((size_t)n), dT((size_t)n);
    auto stream_of = [&](int i) { return streams ? (cudaStream_t)streams[i] : (cudaStream_t)0; };
    for (int i = 0; i < n; ++i) {
        if (!views[i] || !out_rgb_host[i])
            return fail(CONEGS_ERR_ARG, "render_host_batch_async: NULL view or output %d", i);
        if (!views[i]->has_cam) return fail(CONEGS_ERR_STATE, "render_host_batch_async: view %d has no camera", i);
        conegs_view *v = views[i];
        DeviceGuard g(v->ctx->device);
        if (!v->copy_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking);
            for (int k = 0; k < 2 && e == cudaSuccess; ++k)
                e = cudaEventCreateWithFlags(&v->copied[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->rendered, cudaEventDisableTiming);
            if (e != cudaSuccess) return fail(CONEGS_ERR_CUDA, "render_host_batch_async: %s", cudaGetErrorString(e));
        }
        const cudaStream_t s = stream_of(i);
        const int k = v->stage;
        const size_t P = (size_t)v->cam.W * v->cam.H;
        TRY(view_begin(v, s));
        // the staging image's previous copy (two calls back) must be done before it is
        // written again, or freed and grown
        if (v->stage_pending[k]) CUDA_TRY(cudaStreamWaitEvent(s, v->copied[k], 0));
        TRY(ensure(v->ctx, v->stage_rgb[k], sizeof(float) * 3 * P, s));
        TRY(ensure(v->ctx, v->stage_T[k], sizeof(float) * P, s));
        TRY(view_end(v, s));
        drgb[(size_t)i] = v->stage_rgb[k].as<float>();
        dT[(size_t)i] = v->stage_T[k].as<float>();
    }
    TRY(conegs_render_batch(n, views, drgb.data(), dT.data(), flags, streams));
    DeviceGuard g(views[0]->ctx->device);
    for (int i = 0; i < n; ++i) {
        conegs_view *v = views[i];
        const cudaStream_t s = stream_of(i);
        const int k = v->stage;
        const size_t P = (size_t)v->cam.W * v->cam.H;
        CUDA_TRY(cudaEventRecord(v->rendered, s));
        CUDA_TRY(cudaStreamWaitEvent(v->copy_stream, v->rendered, 0));
        CUDA_TRY(cudaMemcpyAsync(out_rgb_host[i], v->stage_rgb[k].p, sizeof(float) * 3 * P, cudaMemcpyDeviceToHost,
                                 v->copy_stream));
        if (out_T_host && out_T_host[i])
            CUDA_TRY(cudaMemcpyAsync(out_T_host[i], v->stage_T[k].p, sizeof(float) * P, cudaMemcpyDeviceToHost,
                                     v->copy_stream));
        CUDA_TRY(cudaEventRecord(v->copied[k], v->copy_stream));
        v->stage_pending[k] = true;
        v->stage ^= 1;
    }
    return CONEGS_OK;
}

conegs_status conegs_view_host_wait(conegs_view *v) {
    if (!v) return fail(CONEGS_ERR_ARG, "view_host_wait: NULL view");
    if (!v->copy_stream) return CONEGS_OK;
    DeviceGuard g(v->ctx->device);
    CUDA_TRY(cudaStreamSynchronize(v->copy_stream));
    return CONEGS_OK;
}

conegs_status conegs_render_host(conegs_view *v, float *out_rgb_host, float *out_T_host, unsigned flags,
                                 void *stream) {
    if (!v || !out_rgb_host) return fail(CONEGS_ERR_ARG, "render_host: NULL argument");
    if (!v->has_cam) return fail(CONEGS_ERR_STATE, "render_host: set_camera was not called on this view");
    if (!v->ctx->has_scene) return fail(CONEGS_ERR_STATE, "render_host: set_scene was not called");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(view_begin(v, s));
    const size_t P = (size_t)v->cam.W * v->cam.H;
    TRY(ensure(v->ctx, v->tmp_rgb, sizeof(float) * 3 * P, s));
    TRY(ensure(v->ctx, v->tmp_T, sizeof(float) * P, s));
    conegs_status st = render_impl(v, v->tmp_rgb.as<float>(), v->tmp_T.as<float>(), flags, s);
    if (st != CONEGS_OK) {
        view_end(v, s);
        return st;
    }
    CUDA_TRY(cudaMemcpyAsync(out_rgb_host, v->tmp_rgb.p, sizeof(float) * 3 * P, cudaMemcpyDeviceToHost, s));
    if (out_T_host) CUDA_TRY(cudaMemcpyAsync(out_T_host, v->tmp_T.p, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
    TRY(view_end(v, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return CONEGS_OK;
}

conegs_status conegs_render_backward(conegs_view *v, const float *dL_drgb, const float *dL_dT, float *g_means,
                                     float *g_log_scales, float *g_quats, float *g_opacity_logits, float *g_sh,
                                     void *stream) {
    if (!v || !dL_drgb) return fail(CONEGS_ERR_ARG, "render_backward: NULL argument");
    if (!v->has_forward || !(v->last_flags & CONEGS_KEEP_FOR_BACKWARD))
        return fail(CONEGS_ERR_STATE, "render_backward: no forward render with CONEGS_KEEP_FOR_BACKWARD on this view");
    conegs_ctx *ctx = v->ctx;
    if (v->forward_gen != ctx->scene_gen) return fail(CONEGS_ERR_STATE, "render_backward: scene changed since forward");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(view_begin(v, s));
    const CamParams &c = v->cam;
    const int64_t n = ctx->sp.n;
    const int nt = c.tiles_x * c.tiles_y;
    TRY(ensure(ctx, v->g_rec, sizeof(float) * 16 * (size_t)std::max<int64_t>(n, 1), s));
    CUDA_TRY(cudaMemsetAsync(v->g_rec.p, 0, sizeof(float) * 16 * (size_t)std::max<int64_t>(n, 1), s));
    RasterArgs a{};
    a.W = c.W;
    a.H = c.H;
    a.tiles_x = c.tiles_x;
    a.ranges = v->ranges.as<uint2>();
    a.gids = v->pair_gid.as<uint32_t>();
    a.rec = v->rec.as<float4>();
    a.d = v->d.as<float>();
    a.dx = v->dx.as<float>();
    a.dy = v->dy.as<float>();
    a.valid = v->valid.as<uint8_t>();
    a.last = v->last.as<uint32_t>();
    a.additive = (v->last_flags & CONEGS_COMP_ADDITIVE) ? 1 : 0;
    a.pixtest = pixel_pretest(c, v->last_flags);
    if (v->n_flat_pairs > 0) {
        a.flat_slot = v->flat_slot.as<uint32_t>();
        a.flat_T = v->flat_T.as<float>();
        a.flat_G = v->flat_G.as<float>();
    }
    set_footprint(a, c, v->last_flags);
    CUDA_TRY(launch_backward(a, nt, !(v->last_flags & CONEGS_FILTER_NONE), v->split.as<uint32_t>(), dL_drgb, dL_dT,
                             v->keep_T.as<float>(), v->g_rec.as<float>(), s));
    CUDA_TRY(launch_backward_params(c, ctx->sp, v->g_rec.as<float>(), v->gflag.as<uint8_t>(), v->gview.as<float4>(),
                                    g_means, g_log_scales, g_quats, g_opacity_logits, g_sh, s));
    return view_end(v, s);
}

conegs_status conegs_get_stats(const conegs_view *v, conegs_stats *out) {
    if (!v || !out) return fail(CONEGS_ERR_ARG, "get_stats: NULL argument");
    memset(out, 0, sizeof(*out));
    out->n_gaussians = v->ctx->has_scene ? v->ctx->sp.n : 0;
    out->n_visible = v->n_visible;
    out->n_flat = v->n_flat;
    out->n_pairs = v->n_pairs;
    out->width = v->cam.W;
    out->height = v->cam.H;
    out->tiles_x = v->cam.tiles_x;
    out->tiles_y = v->cam.tiles_y;
    out->n_valid_pixels = v->n_valid;
    out->n_launches = v->n_launches;
    const DevBuf *bufs[] = {&v->d, &v->dx, &v->dy, &v->valid, &v->table, &v->super, &v->mcam, &v->rec, &v->gview, &v->gcone, &v->gflag, &v->gell, &v->bincache, &v->binlist,
                            &v->counts, &v->vispos, &v->scan_scr, &v->dkeys, &v->dvals, &v->dkeys_alt, &v->dvals_alt,
                            &v->sorted_counts, &v->offsets, &v->pair_tile, &v->pair_gid, &v->pair_tile_alt,
                            &v->pair_gid_alt, &v->ranges, &v->last, &v->sums, &v->rs_scr, &v->tmp_rgb, &v->tmp_T,
                            &v->g_rec, &v->keep_T, &v->split, &v->gflat, &v->flat_slot, &v->flat_pair, &v->flat_T,
                      &v->flat_G};
    size_t tot = 0;
    for (const DevBuf *b : bufs) tot += b->bytes;
    out->device_bytes = tot;
    if (v->profiled && v->has_forward) {
        CUDA_TRY(cudaEventSynchronize(v->prof[3]));
        CUDA_TRY(cudaEventSynchronize(v->done));   // the counters are copied after prof[3]
        float t01 = 0, t12 = 0, t23 = 0, t03 = 0;
        CUDA_TRY(cudaEventElapsedTime(&t01, v->prof[0], v->prof[1]));
        CUDA_TRY(cudaEventElapsedTime(&t12, v->prof[1], v->prof[2]));
        CUDA_TRY(cudaEventElapsedTime(&t23, v->prof[2], v->prof[3]));
        CUDA_TRY(cudaEventElapsedTime(&t03, v->prof[0], v->prof[3]));
        out->ms_preprocess = t01;
        out->ms_sort = t12;
        out->ms_raster = t23;
        out->ms_total = t03;
        float t45 = 0;
        CUDA_TRY(cudaEventElapsedTime(&t45, v->prof[4], v->prof[5]));
        out->ms_raster_main = t45;
        out->n_walked = (int64_t)v->h_sums[5];
        out->n_evaluated = (int64_t)v->h_sums[6];
        out->n_evaluated_flat = (int64_t)v->h_sums[7];
    }
    return CONEGS_OK;
}

conegs_status conegs_compute_floor(conegs_ctx *ctx, int n_views, conegs_view *const *views, float *rho2_out,
                                   void *stream) {
    if (!ctx || !rho2_out || n_views < 0 || (n_views > 0 && !views))
        return fail(CONEGS_ERR_ARG, "compute_floor: bad argument");
    if (!ctx->has_scene) return fail(CONEGS_ERR_STATE, "compute_floor: set_scene was not called");
    std::vector<CamParams> cams;
    for (int i = 0; i < n_views; ++i) {
        if (!views[i] || !views[i]->has_cam) return fail(CONEGS_ERR_STATE, "compute_floor: view %d has no camera", i);
        cams.push_back(views[i]->cam);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    void *dcams = nullptr;
    if (n_views > 0) {
        CUDA_TRY(cudaMallocAsync(&dcams, sizeof(CamParams) * cams.size(), s));
        CUDA_TRY(cudaMemcpyAsync(dcams, cams.data(), sizeof(CamParams) * cams.size(), cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(cudaStreamWaitEvent(s, ctx->scene_ready, 0));
    CUDA_TRY(launch_floor(reinterpret_cast<const CamParams *>(dcams), n_views, ctx->sp.means, ctx->sp.n, rho2_out, s));
    if (dcams) CUDA_TRY(cudaFreeAsync(dcams, s));
    // the host vector must outlive the async copy
    CUDA_TRY(cudaStreamSynchronize(s));
    return CONEGS_OK;
}

conegs_status conegs_get_rays(const conegs_view *v, float *d, float *dx, float *dy, uint8_t *valid, void *stream) {
    if (!v || !v->has_cam) return fail(CONEGS_ERR_STATE, "get_rays: no camera");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = (size_t)v->cam.W * v->cam.H;
    CUDA_TRY(cudaStreamWaitEvent(s, v->done, 0));
    if (d) CUDA_TRY(cudaMemcpyAsync(d, v->d.p, sizeof(float) * 3 * P, cudaMemcpyDeviceToDevice, s));
    if (dx) CUDA_TRY(cudaMemcpyAsync(dx, v->dx.p, sizeof(float) * 3 * P, cudaMemcpyDeviceToDevice, s));
    if (dy) CUDA_TRY(cudaMemcpyAsync(dy, v->dy.p, sizeof(float) * 3 * P, cudaMemcpyDeviceToDevice, s));
    if (valid) CUDA_TRY(cudaMemcpyAsync(valid, v->valid.p, P, cudaMemcpyDeviceToDevice, s));
    return CONEGS_OK;
}

conegs_status conegs_get_tile_table(const conegs_view *v, float *table, void *stream) {
    if (!v || !v->has_cam || !table) return fail(CONEGS_ERR_STATE, "get_tile_table: no camera");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamWaitEvent(s, v->done, 0));
    const size_t nt = (size_t)v->cam.tiles_x * v->cam.tiles_y;
    CUDA_TRY(cudaMemcpyAsync(table, v->table.p, sizeof(float) * 6 * nt, cudaMemcpyDeviceToDevice, s));
    return CONEGS_OK;
}

}  // extern "C"

namespace {
__global__ void range_counts_kernel(const uint2 *ranges, int nt, int32_t *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) out[t] = (int32_t)(ranges[t].y - ranges[t].x);
}
__global__ void ranges_i32_kernel(const uint2 *ranges, int nt, int32_t *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) {
        out[2 * t] = (int32_t)ranges[t].x;
        out[2 * t + 1] = (int32_t)ranges[t].y;
    }
}
}  // namespace

extern "C" {

conegs_status conegs_get_bin_counts(const conegs_view *v, int32_t *per_gaussian, int32_t *per_tile, void *stream) {
    if (!v || !v->has_forward) return fail(CONEGS_ERR_STATE, "get_bin_counts: no render on this view");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamWaitEvent(s, v->done, 0));
    const int nt = v->cam.tiles_x * v->cam.tiles_y;
    if (per_gaussian && v->ctx->sp.n > 0)
        CUDA_TRY(cudaMemcpyAsync(per_gaussian, v->counts.p, sizeof(uint32_t) * (size_t)v->ctx->sp.n,
                                 cudaMemcpyDeviceToDevice, s));
    if (per_tile) {
        range_counts_kernel<<<(nt + 255) / 256, 256, 0, s>>>(v->ranges.as<uint2>(), nt, per_tile);
        CUDA_TRY(cudaGetLastError());
    }
    return CONEGS_OK;
}

conegs_status conegs_get_pairs(const conegs_view *v, int32_t *gaussian_ids, int32_t *tile_ranges, void *stream) {
    if (!v || !v->has_forward) return fail(CONEGS_ERR_STATE, "get_pairs: no render on this view");
    DeviceGuard g(v->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamWaitEvent(s, v->done, 0));
    const int nt = v->cam.tiles_x * v->cam.tiles_y;
    if (gaussian_ids && v->n_pairs > 0)
        CUDA_TRY(cudaMemcpyAsync(gaussian_ids, v->pair_gid.p, sizeof(uint32_t) * (size_t)v->n_pairs,
                                 cudaMemcpyDeviceToDevice, s));
    if (tile_ranges) {
        ranges_i32_kernel<<<(nt + 255) / 256, 256, 0, s>>>(v->ranges.as<uint2>(), nt, tile_ranges);
        CUDA_TRY(cudaGetLastError());
    }
    return CONEGS_OK;
}

conegs_status conegs_radix_sort_pairs(conegs_ctx *ctx, uint32_t *keys, uint32_t *values, int64_t n, int begin_bit,
                                      int end_bit, void *stream) {
    if (!ctx || n < 0 || (n > 0 && (!keys || !values))) return fail(CONEGS_ERR_ARG, "radix_sort_pairs: bad argument");
    if (begin_bit < 0 || end_bit > 32 || begin_bit > end_bit) return fail(CONEGS_ERR_ARG, "radix_sort_pairs: bad bits");
    if (n > (1LL << 31)) return fail(CONEGS_ERR_ARG, "radix_sort_pairs: n too large");
    if (n <= 1) return CONEGS_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    void *ak = nullptr, *av = nullptr, *scr = nullptr;
    CUDA_TRY(cudaMallocAsync(&ak, sizeof(uint32_t) * (size_t)n, s));
    CUDA_TRY(cudaMallocAsync(&av, sizeof(uint32_t) * (size_t)n, s));
    CUDA_TRY(cudaMallocAsync(&scr, sizeof(uint32_t) * (size_t)radix_scratch_words(n), s));
    cudaError_t e = radix_sort_pairs(keys, values, (uint32_t *)ak, (uint32_t *)av, n, begin_bit, end_bit,
                                     (uint32_t *)scr, s);
    cudaFreeAsync(ak, s);
    cudaFreeAsync(av, s);
    cudaFreeAsync(scr, s);
    if (e != cudaSuccess) return fail(CONEGS_ERR_CUDA, "radix_sort_pairs: %s", cudaGetErrorString(e));
    return CONEGS_OK;
}

}  // extern "C"
