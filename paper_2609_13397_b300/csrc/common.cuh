// Shared device-side definitions of the ConeGaussian CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace conegs {

constexpr int TILE = 8;           // tile side in pixels (one CTA of TILE*TILE threads per tile)
constexpr int TILE_PX = TILE * TILE;
constexpr int SUPER = 8;          // tiles per super-tile side (coarse binning level)
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_STOP = 1e-4f;
constexpr float T_NEAR = 0.01f;
constexpr int REC_F4 = 8;         // float4 words per per-view raster record
constexpr int BINREC = 12;        // floats per Gaussian of the binning rule's scene record
// Per-view footprint extremes (per unit depth) for the rasteriser's pre-test,
// in the view's camera-bound block after the binning rule's words: the view-wide
// smallest eigenvalue, then FP_BANDS polar-angle bands of it (band j: the pixel
// rays at angle [j, j+1) pi / FP_BANDS from the optical axis), the view-wide
// largest eigenvalue, then its bands.
constexpr int FP_BANDS = 64;
constexpr int FP_MIN = 20;                        // offset of the smallest eigenvalue block
constexpr int FP_MAX = FP_MIN + 1 + FP_BANDS;     // offset of the largest eigenvalue block
constexpr int MCAM_MMIN = FP_MAX + 1 + FP_BANDS;   // the smallest footprint bound m over the valid tiles
constexpr int MCAM_FLOATS = MCAM_MMIN + 1;

// Camera passed by value to kernels.
struct CamParams {
    int model;        // 0 pinhole, 1 Kannala-Brandt
    int W, H, tiles_x, tiles_y, supers_x, supers_y;
    float fx, fy, cx, cy;
    float k[4];
    float R[9];       // camera -> world rotation, row-major
    float o[3];       // optical centre
    float thlim;      // KB valid half-FOV (rad)
    float rlim2;      // KB squared normalised radius limit (FP32 rule)
    float lip[17];    // KB: lip[j] >= max over theta in [0, theta_lim j/16] of max(r'(theta), r(theta)/sin(theta))
};

// Scene arrays (caller-owned parameters + library cache), passed by value.
struct SceneParams {
    int64_t n;
    int sh_degree;
    int storage;                  // 0 f32, 1 bf16, 2 f16
    const float *means, *log_scales, *quats, *rho2;
    const void *logits, *sh;
    // camera-independent cache
    const float *W;               // [n][9] W_eff = S_eff^-1 R^T
    const float *sig_eff;         // [n]
    const float *binrec;          // [n][BINREC] kap, ks, kr, r1sq, s2, flag, Sigma_eff (xx xy xz yy yz zz)
};

__device__ __forceinline__ float load_scalar(const void *p, int64_t i, int storage) {
    if (storage == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
    if (storage == 2) return __half2float(reinterpret_cast<const __half *>(p)[i]);
    return reinterpret_cast<const float *>(p)[i];
}

__host__ __device__ __forceinline__ int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Streaming multiprocessors of the current device (queried once per device).
int num_sms();

// Host-side count of kernel launches issued by the library (reported by
// conegs_get_stats for the last render).
void note_launches(int k);
long long launches_so_far();

}  // namespace conegs
