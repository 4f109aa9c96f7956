/*
 * conegs.h -- C ABI of the B300 (sm_103a) ConeGaussian renderer.
 *
 * The library renders a 3D Gaussian scene through a calibrated central
 * camera (pinhole or Kannala-Brandt fisheye) with the anti-aliased,
 * ray-native pixel-footprint filter of ConeGaussian (arXiv 2609.13397):
 * per pixel, the half-pixel edge rays of the camera's own inverse mapping
 * (Sec. 4.1, Eq. 6) give an anisotropic footprint that is moment matched
 * (Eq. 8) and convolved in closed form with every Gaussian hit at its
 * maximum-response depth (Eq. 9), after the per-Gaussian training-frequency
 * floor (Eq. 10) and the marginal composition rule (Eq. 12); the responses
 * are alpha-composited front to back (Eq. 4).
 *
 * Conventions
 *   - Camera frame is OpenCV (x right, y down, z forward).  cam_to_world is
 *     a 3x4 row-major [R | o] (R: camera-frame directions -> world; o: the
 *     optical centre).  NULL means identity.
 *   - Pixel (i, j) is the square [i, i+1) x [j, j+1); its centre ray goes
 *     through (i + 1/2, j + 1/2).  Images are row-major, channel-planar:
 *     rgb[c * H * W + j * W + i].
 *   - Quaternions are (w, x, y, z), normalised inside.  Scales are given as
 *     log-scales, opacity as a logit (sigma = 1 / (1 + e^-logit)).
 *   - SH coefficients are [n][(deg+1)^2][3], real SH in (l, m = -l..l)
 *     order with positive normalisation constants; colour =
 *     max(0, sum_lm c_lm Y_lm(dir) + 1/2), dir = (mu - o)/|mu - o|.
 *
 * Ownership and memory
 *   - Every array argument is a DEVICE pointer owned by the caller unless
 *     its name ends in _host.  The library never frees caller memory.
 *   - set_scene keeps the caller's parameter arrays by reference (no copy):
 *     they must stay alive and unchanged until the next set_scene or
 *     conegs_destroy.  The library owns only derived state and scratch
 *     (per-Gaussian caches, ray tables, pair lists), allocated with
 *     cudaMalloc on the context's device and grown on demand.
 *
 * Streams and synchronisation
 *   - Every call enqueues its work on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) and returns without waiting, except
 *     conegs_render / conegs_render_host, which wait once for the
 *     4-byte pair count after binning in order to size the pair list.
 *   - A context may hold many views; different views may render
 *     concurrently from different host threads on different streams.
 *     Calls on the same view must not overlap.
 *
 * Errors
 *   - Every call returns a conegs_status; CONEGS_OK is 0.  A failed call
 *     leaves the previous state intact and records a message readable with
 *     conegs_last_error() (thread-local).  No call aborts the process.
 */
#ifndef CONEGS_H
#define CONEGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CONEGS_OK = 0,
    CONEGS_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, bad model) */
    CONEGS_ERR_OOM = 2,         /* device allocation failed */
    CONEGS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    CONEGS_ERR_NOCONVERGE = 4,  /* KB inverse mapping did not converge */
    CONEGS_ERR_OVERFLOW = 5,    /* pair list larger than 2^31 entries */
    CONEGS_ERR_STATE = 6,       /* call out of order (e.g. render before set_scene) */
    CONEGS_ERR_BUDGET = 7       /* request exceeds the context's memory budget */
} conegs_status;

typedef enum { CONEGS_PINHOLE = 0, CONEGS_KB_FISHEYE = 1 } conegs_model;

typedef enum { CONEGS_F32 = 0, CONEGS_BF16 = 1, CONEGS_F16 = 2 } conegs_dtype;

/* Render flags (bit set). */
enum {
    CONEGS_FILTER_NONE = 1u << 0,   /* centre-ray response sigma e^{-D^2/2} (no footprint, Eq. 3 with C=1) */
    CONEGS_COMP_ADDITIVE = 1u << 1, /* use Sigma_fp,eff directly instead of Eq. 12's marginal clamp */
    CONEGS_KEEP_FOR_BACKWARD = 1u << 2, /* keep pair lists and per-pixel state for render_backward */
    CONEGS_PROFILE = 1u << 3,  /* record per-stage CUDA events on the stream and count pair evaluations
                                  (read back by conegs_get_stats) */
    /* Isotropic footprint variants (the comparison axis of Sec. 5), at most one of
     * FILTER_NONE / FILTER_ISO / FILTER_ZF (else CONEGS_ERR_ARG).  Eq. 6-12 are kept;
     * the pixel's two half-edge differentials are replaced by a b1, a b2, (b1, b2) an
     * orthonormal basis across the pixel ray d, so the footprint is isotropic across
     * the ray with t^2 a^2 / 3 per axis (Eq. 8): */
    CONEGS_FILTER_ISO = 1u << 4, /* a^2 = (|dx_perp|^2 + |dy_perp|^2) / 2: half-trace of the true footprint */
    CONEGS_FILTER_ZF = 1u << 5,  /* a = |<d, z_cam>| / (2 f_x): paraxial z/f pixel size (VKRayGS-style sizing) */
    /* Unscented-transform binning (the 3DGUT-style backbone of Sec. 3) instead of the
     * conservative angular-tile rule; the response is unchanged.  Each Gaussian's seven
     * sigma points mu, mu +- sqrt(3) s_eff,i R_i go through the camera model (scaled UT,
     * alpha 1, beta 2, kappa 0); a tile is kept when its pixel-centre rectangle meets
     * the ellipse {y : (y - ybar)^T (Sigma_2 + I/12)^-1 (y - ybar) <= 2 ln(255 sigma_eff)}.
     * Approximate: a pair the ellipse misses is not evaluated.  Gaussians with a sigma
     * point outside the camera's domain (pinhole: p_z < 0.1 |p|; fisheye: beyond
     * theta_lim) keep the angular-tile rule. */
    CONEGS_BIN_UT = 1u << 6,
    /* Per-ray compositing order (Sec. 3: pairs composited by their max-response depth
     * t*_k): each pixel re-orders the pairs of its tile list by its own t* through a
     * k-buffer of 32 pairs (per pixel), instead of the tile list's per-Gaussian key
     * |mu - o|.  Exactly the per-pixel t* order (ties: key, then index) whenever a
     * pixel has at most 32 pairs with alpha >= 1/255 before it stops, and whenever no
     * contributing pair is displaced by 32 or more contributing pairs between the two
     * orders; otherwise an approximation of it.  Forward only: with
     * CONEGS_KEEP_FOR_BACKWARD the render fails with CONEGS_ERR_ARG. */
    CONEGS_ORDER_TSTAR = 1u << 7,
    /* The rasteriser's pre-test (which skips pairs that cannot reach alpha >= 1/255;
     * it changes no result) in its ray-direction form on pinhole views as well.  By
     * default a pinhole view tests each pixel centre against the ellipse that the
     * same visual cone cuts from the image plane, a cheaper test; fisheye views
     * always use the ray-direction form.  Both forms are conservative, so images are
     * the same either way; the flag exists to check exactly that. */
    CONEGS_PRETEST_RAY = 1u << 8,
    /* No pre-test: the rasteriser and its adjoint fully evaluate every pair of the
     * tile lists.  Slower, and bitwise the same images, transmittance and adjoint
     * state as with the pre-test (which only skips pairs that cannot reach
     * alpha >= 1/255); the flag exists to check that. */
    CONEGS_PRETEST_OFF = 1u << 9
};

typedef struct conegs_ctx conegs_ctx;
typedef struct conegs_view conegs_view;

typedef struct {
    int64_t n_gaussians;     /* scene size */
    int64_t n_visible;       /* Gaussians with at least one tile in the last render */
    int64_t n_pairs;         /* tile/Gaussian pairs of the last render */
    int32_t width, height;   /* camera */
    int32_t tiles_x, tiles_y;
    int64_t n_valid_pixels;  /* pixels inside the camera's valid domain */
    size_t device_bytes;     /* library-owned device memory of this view */
    int64_t n_launches;      /* CUDA kernels launched by the last render */
    /* filled when the last render used CONEGS_PROFILE (get_stats then waits for it): */
    int64_t n_walked;        /* tile-list entries walked by the rasteriser's pixels */
    int64_t n_evaluated;     /* of those, full pair responses evaluated (past the cone pre-test) */
    float ms_preprocess;     /* view records + bin count + scans */
    float ms_sort;           /* compaction + depth sort + emit + tile sort + ranges */
    float ms_raster;         /* tile rasteriser */
    float ms_total;          /* whole render on the device */
    float ms_raster_main;    /* of ms_raster: the launch that walks every tile's first list segment */
    int64_t n_evaluated_flat; /* (profiled) of n_evaluated: pairs of near-degenerate flat Gaussians,
                                 evaluated in FP64 (see n_flat) */
    int64_t n_flat;          /* visible near-degenerate flat Gaussians of the last render (effective
                                scale ratio s_max/s_min above 100, Eq. 10): their response and adjoint
                                are evaluated in FP64; a view with none runs the FP32-only kernels */
} conegs_stats;

/* Create a context on CUDA device `device` (its scene and views live there).
 * mem_budget_bytes bounds the library-owned memory of all views (0 = no bound);
 * a render that would exceed it fails with CONEGS_ERR_BUDGET. */
conegs_status conegs_create(conegs_ctx **out, int device, size_t mem_budget_bytes);

/* Release the context, its views and all library-owned memory.  Any work
 * still queued on streams that uses them must have completed. */
void conegs_destroy(conegs_ctx *ctx);

/* Human-readable message of the last failed call on this host thread. */
const char *conegs_last_error(void);

/* Library version string. */
const char *conegs_version(void);

/* Define the scene (Sec. 3 "Preliminaries": mean mu, covariance R S^2 R^T,
 * opacity sigma; Sec. 4.2 Eq. 10: per-Gaussian floor rho^2).
 *   means[n*3], log_scales[n*3], quats[n*4]   FP32
 *   opacity_logits[n], sh[n*(deg+1)^2*3]      in `storage` (F32, BF16 or F16);
 *                                             evaluated in FP32
 *   rho2[n]                                   FP32, or NULL for rho^2 = 0
 * Computes the camera-independent cache (W_eff = S_eff^-1 R^T, sigma_eff,
 * binning bounds) on `stream`.  n may be 0.  sh_degree in 0..3. */
conegs_status conegs_set_scene(conegs_ctx *ctx, int64_t n, const float *means, const float *log_scales,
                               const float *quats, const void *opacity_logits, const void *sh, int sh_degree,
                               int storage, const float *rho2, void *stream);

/* Create / destroy a view: one camera plus its ray table and render scratch. */
conegs_status conegs_view_create(conegs_ctx *ctx, conegs_view **out);
void conegs_view_destroy(conegs_view *view);

/* Set the view's camera (Sec. 3: rays r(t) = o + t d, d = Pi^-1(p) unit;
 * Sec. 4.1: edge rays Pi^-1(p + (1/2,0)), Pi^-1(p + (0,1/2)) of the same model).
 *   intrinsics_host[4] = fx, fy, cx, cy (pixels)
 *   distortion_host[4] = k1..k4 of theta_d = theta (1 + k1 th^2 + k2 th^4 + k3 th^6 + k4 th^8)
 *                        (KB only; ignored for pinhole; may be NULL = 0)
 *   cam_to_world_host[12] (may be NULL = identity)
 *   theta_lim (KB): valid half field of view in radians; a pixel is valid
 *     iff its normalised radius is at most theta_d(theta_lim); theta_d must be
 *     increasing on [0, theta_lim].  0 = the largest theta <= 95 deg below
 *     which d(theta_d)/d(theta) >= 1/4.
 * Builds the ray table (centre ray and the two half-pixel differentials per
 * pixel) and the per-tile cone table on `stream`.  Fails with CONEGS_ERR_ARG
 * for non-positive sizes/focal lengths or an unknown model. */
conegs_status conegs_set_camera(conegs_view *view, int model, int width, int height,
                                const float *intrinsics_host, const float *distortion_host,
                                const float *cam_to_world_host, float theta_lim, void *stream);

/* Forward render of the current scene through the view's camera.
 *   out_rgb[3*H*W] (channel-planar), out_T[H*W] (final transmittance; may be NULL)
 * Pixels outside the valid domain get rgb = 0, T = 1.  Background is 0.
 * flags: CONEGS_* render flags.  With CONEGS_KEEP_FOR_BACKWARD the view keeps
 * what render_backward needs (until the next render or set_camera on it). */
conegs_status conegs_render(conegs_view *view, float *out_rgb, float *out_T, unsigned flags, void *stream);

/* The same render for n views at once (a camera rig, or the views of one
 * step), each into its own output on its own stream.  A render needs one host
 * wait (for its pair count, to size the pair buffers); here the view records
 * and bin counts of all views are enqueued before the first wait, so the
 * views' work overlaps on the device.
 *   views[n]: distinct views of one context, each with a camera;
 *   out_rgb[n], out_T[n] (out_T may be NULL, or any entry of it), streams[n]
 *   (may be NULL: every view on the default stream).
 * flags apply to every view.  Returns the first error; views before the
 * failing one are rendered, the failing one and the rest are not (their
 * render_backward then fails with CONEGS_ERR_STATE). */
conegs_status conegs_render_batch(int n, conegs_view *const *views, float *const *out_rgb, float *const *out_T,
                                  unsigned flags, void *const *streams);

/* The count pass of a render, run ahead of it: the view records, the binning
 * count and the pair total (the host waits for them), so that a caller can
 * admit the render by the memory it will need.
 *   *pairs_host: tile/Gaussian pairs the render will walk (may be NULL);
 *   *bytes_host: device bytes the rest of the render sizes from the counts
 *                (pair lists and sort scratch, split state, per-pixel state;
 *                may be NULL).
 * The next conegs_render / conegs_render_host on this view with the same flags
 * and an unchanged scene and camera uses this count instead of counting again.
 * Errors as conegs_render. */
conegs_status conegs_render_count(conegs_view *view, unsigned flags, int64_t *pairs_host, size_t *bytes_host,
                                  void *stream);

/* conegs_render_batch into host memory: each view renders into its own device
 * scratch and its image is copied to out_rgb_host[i] (and out_T_host[i], when
 * out_T_host and that entry are non-NULL) on streams[i]; returns after every
 * copy has completed.  Host buffers should be pinned for asynchronous copies.
 * Errors as conegs_render_batch. */
conegs_status conegs_render_host_batch(int n, conegs_view *const *views, float *const *out_rgb_host,
                                       float *const *out_T_host, unsigned flags, void *const *streams);

/* Pipelined form of conegs_render_host_batch: renders the views and ENQUEUES
 * the copies of their images (rgb, and T where out_T_host and its entry are
 * non-NULL) to the host buffers, then returns without waiting for them.  Each
 * view renders into one of two view-owned device staging images in turn and
 * copies it back on a copy stream of its own, so the copy of one call overlaps
 * the next call's render of the same view (that render waits only for the copy
 * of two calls back, which used the same staging image).
 * Ownership: the host buffers must be pinned (the copies are asynchronous) and
 * stay valid, unread and unwritten until conegs_view_host_wait(view) returns.
 * Errors as conegs_render_batch; after an error no copy of that call is pending. */
conegs_status conegs_render_host_batch_async(int n, conegs_view *const *views, float *const *out_rgb_host,
                                             float *const *out_T_host, unsigned flags, void *const *streams);

/* Blocks until every image copy that conegs_render_host_batch_async enqueued for
 * this view has reached host memory.  CONEGS_ERR_CUDA if a copy failed. */
conegs_status conegs_view_host_wait(conegs_view *view);

/* Same as conegs_render, with HOST output buffers (pinned memory recommended):
 * renders into view-owned device memory and copies the result back on
 * `stream`; returns after the copy has completed. */
conegs_status conegs_render_host(conegs_view *view, float *out_rgb_host, float *out_T_host, unsigned flags,
                                 void *stream);

/* Adjoint of the last conegs_render on this view (which must have used
 * CONEGS_KEEP_FOR_BACKWARD): given dL/d rgb [3*H*W] (and optionally dL/dT
 * [H*W], may be NULL), ACCUMULATES (+=) the gradients w.r.t. the scene
 * parameters into caller buffers of the scene's shapes (FP32; any may be
 * NULL to skip): g_means[n*3], g_log_scales[n*3], g_quats[n*4],
 * g_opacity_logits[n], g_sh[n*(deg+1)^2*3].  rho^2 is not differentiated.
 * Transmittance is recomputed back to front from the final T (no per-pair
 * state is stored by the forward pass). */
conegs_status conegs_render_backward(conegs_view *view, const float *dL_drgb, const float *dL_dT, float *g_means,
                                     float *g_log_scales, float *g_quats, float *g_opacity_logits, float *g_sh,
                                     void *stream);

/* Statistics of the view's last render (host struct).  If that render used
 * CONEGS_PROFILE this call waits for it to finish. */
conegs_status conegs_get_stats(const conegs_view *view, conegs_stats *out_host);

/* Eq. 11 training-frequency floor: rho2_out[n] = min over the given views in
 * which mu is visible of tr(Sigma_fp)/2 at the pixel onto which mu projects,
 * evaluated in world space (before whitening); 0 if visible in none.
 * Visible: |mu - o| > 0.2 and the projection lies in the image and the
 * valid domain.  Reads the current scene's means. */
conegs_status conegs_compute_floor(conegs_ctx *ctx, int n_views, conegs_view *const *views_host, float *rho2_out,
                                   void *stream);

/* ---- inspection (tests and tools): copies of internal tables into caller
 * device buffers, enqueued on `stream` ---- */

/* Ray table: d, delta_x, delta_y as [3][H*W] each (world frame, FP32) and
 * valid[H*W] (1 inside the valid domain). */
conegs_status conegs_get_rays(const conegs_view *view, float *d, float *delta_x, float *delta_y, uint8_t *valid,
                              void *stream);

/* Per-tile cone table [tiles_y*tiles_x][6]: axis (3), sin(gamma/2), cos(gamma/2),
 * footprint bound m; sin(gamma/2) = -1 marks a tile without valid pixels. */
conegs_status conegs_get_tile_table(const conegs_view *view, float *table, void *stream);

/* Pair counts of the last render: per Gaussian [n] (tiles it was binned to)
 * and per tile [tiles_y*tiles_x] (Gaussians in its list). */
conegs_status conegs_get_bin_counts(const conegs_view *view, int32_t *per_gaussian, int32_t *per_tile,
                                    void *stream);

/* Sorted pair list of the last render: gaussian ids [n_pairs] in (tile, depth,
 * index) order, and per-tile [begin, end) ranges [tiles][2]. */
conegs_status conegs_get_pairs(const conegs_view *view, int32_t *gaussian_ids, int32_t *tile_ranges, void *stream);

/* Device radix sort used by the binning stage, exposed for testing:
 * stable LSD sort of (key, value) pairs on key bits [begin_bit, end_bit).
 * keys/values are sorted in place (device arrays of n entries). */
conegs_status conegs_radix_sort_pairs(conegs_ctx *ctx, uint32_t *keys, uint32_t *values, int64_t n, int begin_bit,
                                      int end_bit, void *stream);

/* Measured FP32 fused multiply-add throughput of device `device` (TFLOP/s, an
 * FMA counted as 2 flops): the denominator of the rasteriser's roofline, whose
 * pair response (Eq. 2-12) runs on the FP32 FMA pipe.  Runs independent FMA
 * chains (scalar and packed f32x2) on every SM for a few milliseconds and
 * reports the larger rate in *tflops_host and that launch's time in *ms_host
 * (may be NULL).  Allocates a small device buffer; synchronises the device's
 * legacy default stream.  The paper has no counterpart; this is a measurement
 * utility. */
conegs_status conegs_measure_fp32_peak(int device, double *tflops_host, double *ms_host);

/* The same stable radix sort, for callers that cannot allocate device memory
 * while they sort: their device memory may be fully reserved by another
 * allocator (a framework's caching allocator), or they run in a
 * latency-critical loop that must not block on or fail in an allocation.
 * The paper has no counterpart; this is a library service.
 * The scratch is a fixed array inside the library (about 2.6 MB on every GPU
 * that loads it, held until exit); the call allocates nothing.
 *   keys/values: device arrays of n entries, sorted in place on `stream`.
 *   n <= 262144; larger n fails with CONEGS_ERR_ARG.
 * The first call on a device looks up the array's address with that device
 * current; make it before any stream capture.  All calls share the one array
 * and it keeps the last call's contents (nothing in it must start at zero):
 * calls whose GPU work overlaps race, so order them (one stream, or events). */
conegs_status conegs_radix_sort_pairs_noalloc(uint32_t *keys, uint32_t *values, int64_t n, int begin_bit,
                                              int end_bit, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CONEGS_H */
