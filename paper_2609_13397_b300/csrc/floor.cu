// Eq. 11: per-Gaussian training-frequency floor
//   rho^2 = min over visible training views of tr(Sigma_fp^(v))/2,
// Sigma_fp^(v) built at the pixel onto which mu projects, before whitening:
// with p = Pi_v(mu) (continuous), d = (mu - o)/t, t = |mu - o| and the
// half-pixel differentials delta_i of the view's own inverse mapping at p,
// e_i = t (I - d d^T) delta_i and tr(Sigma_fp)/2 = (|e_x|^2 + |e_y|^2)/6.
// Visible: t > 0.2 and p inside the image and the valid domain.
// One thread per Gaussian, views read from a small device array.
#include "camera.cuh"

namespace conegs {

__global__ void __launch_bounds__(256) floor_kernel(const CamParams *__restrict__ cams, int nv,
                                                    const float *__restrict__ means, int64_t n,
                                                    float *__restrict__ rho2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float best = INFINITY;
    for (int v = 0; v < nv; ++v) {
        const CamParams &c = cams[v];
        const float w[3] = {mu[0] - c.o[0], mu[1] - c.o[1], mu[2] - c.o[2]};
        const float t = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (!(t > 0.2f)) continue;
        // world -> camera with R^T
        float xc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) xc[k] = c.R[k] * w[0] + c.R[3 + k] * w[1] + c.R[6 + k] * w[2];
        float px, py;
        if (c.model == 0) {
            if (!(xc[2] > 0.0f)) continue;
            px = c.fx * xc[0] / xc[2] + c.cx;
            py = c.fy * xc[1] / xc[2] + c.cy;
        } else {
            const float rho = sqrtf(xc[0] * xc[0] + xc[1] * xc[1]);
            const float th = atan2f(rho, xc[2]);
            if (th > c.thlim) continue;
            const float td = kb_P(c, th);
            px = rho > 0.0f ? c.fx * td * xc[0] / rho + c.cx : c.cx;
            py = rho > 0.0f ? c.fy * td * xc[1] / rho + c.cy : c.cy;
        }
        if (!(px >= 0.0f && px < (float)c.W && py >= 0.0f && py < (float)c.H)) continue;
        float vd[3], vx[3], vy[3];
        if (!point_rays(c, px, py, vd, vx, vy)) continue;
        float ex[3], ey[3];
        rotate(c, vx, ex);
        rotate(c, vy, ey);
        const float d[3] = {w[0] / t, w[1] / t, w[2] / t};
        const float ax = ex[0] * d[0] + ex[1] * d[1] + ex[2] * d[2];
        const float ay = ey[0] * d[0] + ey[1] * d[1] + ey[2] * d[2];
        float px2 = 0.f, py2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = ex[k] - ax * d[k], b = ey[k] - ay * d[k];
            px2 += a * a;
            py2 += b * b;
        }
        best = fminf(best, t * t * (px2 + py2) * (1.0f / 6.0f));
    }
    rho2[i] = isinf(best) ? 0.0f : best;
}

cudaError_t launch_floor(const CamParams *cams_dev, int nv, const float *means, int64_t n, float *rho2,
                         cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    floor_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(cams_dev, nv, means, n, rho2);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
