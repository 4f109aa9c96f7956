// K1: per-pixel ray table of a central camera (Sec. 3 and Sec. 4.1, Eq. 6).
//
// For every pixel centre p the table holds the unit centre ray d = Pi^-1(p)
// and the two half-pixel differentials delta_i = Pi^-1(p + Delta_i) - d,
// Delta_x = (1/2, 0), Delta_y = (0, 1/2), taken from the camera model itself
// (not a Jacobian).  |delta| is ~1/(2f), so a naive difference of two FP32
// unit vectors would lose ~4 digits; both models below form the difference
// without cancellation:
//   pinhole: delta = (v' - v)/|v'| + v (1/|v'| - 1/|v|), with |v|^2 - |v'|^2
//            formed exactly from the offset;
//   KB:      Newton on the increment Delta_theta of theta_d(theta) = r with
//            divided-difference polynomials, then sin/cos differences through
//            half-angle products.  Newton on theta runs in FP32 and is
//            polished in FP64 only near the edge of the field of view.
// Layout: SoA float d[3][P], dx[3][P], dy[3][P], uint8 valid[P] (P = W*H).
#include <algorithm>

#include "camera.cuh"

namespace conegs {

__global__ void __launch_bounds__(256) ray_table_kernel(CamParams c, float *__restrict__ d, float *__restrict__ dx,
                                                        float *__restrict__ dy, uint8_t *__restrict__ valid) {
    const int64_t P = (int64_t)c.W * c.H;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int i = (int)(p % c.W), j = (int)(p / c.W);
    const float x = (float)i + 0.5f, y = (float)j + 0.5f;
    float vd[3], vx[3], vy[3];
    const bool ok = point_rays(c, x, y, vd, vx, vy);
    float w[3];
    rotate(c, vd, w);
    d[p] = ok ? w[0] : 0.0f; d[P + p] = ok ? w[1] : 0.0f; d[2 * P + p] = ok ? w[2] : 0.0f;
    rotate(c, vx, w);
    dx[p] = ok ? w[0] : 0.0f; dx[P + p] = ok ? w[1] : 0.0f; dx[2 * P + p] = ok ? w[2] : 0.0f;
    rotate(c, vy, w);
    dy[p] = ok ? w[0] : 0.0f; dy[P + p] = ok ? w[1] : 0.0f; dy[2 * P + p] = ok ? w[2] : 0.0f;
    valid[p] = ok ? 1 : 0;
}

// Footprint extremes of the view, per unit depth, over its valid pixels, view
// wide and per polar-angle band (the angle of the pixel's centre ray from the
// optical axis z, band floor(angle / (pi / FP_BANDS))):
//   out[0], out[1 + j]: the smallest eigenvalue of [dp_i . dp_j] / 3, dp_i =
//           delta_i - (delta_i . d) d the half-edge differentials across the
//           centre ray.  At depth t a pixel's world footprint of Eq. 8 (its
//           half-edges f_i = t (delta_i - c_i d)) has both eigenvalues at least
//           t^2 times this.
//   out[1 + FP_BANDS], out[2 + FP_BANDS + j]: the largest eigenvalue of
//           [delta_i . delta_j] / 3 (the differentials themselves), so that
//           t^2 sum_i delta_i delta_i^T / 3 <= t^2 (this) I.
// Float bits of non-negative values, combined with unsigned min and max (which
// order them as the floats): the minima must hold 0xffffffff and the maxima
// zero before the launch; a band without valid pixels keeps them.
__global__ void __launch_bounds__(256) footprint_min_kernel(const float *__restrict__ d, const float *__restrict__ dx,
                                                            const float *__restrict__ dy,
                                                            const uint8_t *__restrict__ valid, int64_t P,
                                                            float z0, float z1, float z2,
                                                            unsigned int *__restrict__ out) {
    __shared__ unsigned int s_min[FP_BANDS], s_max[FP_BANDS];
    for (int j = threadIdx.x; j < FP_BANDS; j += blockDim.x) {
        s_min[j] = 0xffffffffu;
        s_max[j] = 0u;
    }
    __syncthreads();
    const float band_scale = (float)FP_BANDS / 3.14159265f;
    float best = 3.0e38f, top = 0.0f;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        if (!valid[p]) continue;
        const float d0 = d[p], d1 = d[P + p], d2 = d[2 * P + p];
        const float x0 = dx[p], x1 = dx[P + p], x2 = dx[2 * P + p];
        const float y0 = dy[p], y1 = dy[P + p], y2 = dy[2 * P + p];
        const float sx = x0 * d0 + x1 * d1 + x2 * d2, sy = y0 * d0 + y1 * d1 + y2 * d2;
        const float u0 = x0 - sx * d0, u1 = x1 - sx * d1, u2 = x2 - sx * d2;
        const float v0 = y0 - sy * d0, v1 = y1 - sy * d1, v2 = y2 - sy * d2;
        const float a = (u0 * u0 + u1 * u1 + u2 * u2) / 3.0f, b = (u0 * v0 + u1 * v1 + u2 * v2) / 3.0f,
                    c = (v0 * v0 + v1 * v1 + v2 * v2) / 3.0f;
        const float h = 0.5f * (a - c);
        const float lmax = 0.5f * (a + c) + sqrtf(h * h + b * b);
        const float lmin = lmax > 0.0f ? fmaxf(a * c - b * b, 0.0f) / lmax : 0.0f;   // det / lmax: no cancellation
        const float A = (x0 * x0 + x1 * x1 + x2 * x2) / 3.0f, B = (x0 * y0 + x1 * y1 + x2 * y2) / 3.0f,
                    C = (y0 * y0 + y1 * y1 + y2 * y2) / 3.0f;
        const float H = 0.5f * (A - C);
        const float top_p = 0.5f * (A + C) + sqrtf(H * H + B * B);
        best = fminf(best, lmin);
        top = fmaxf(top, top_p);
        const float ang = acosf(fminf(fmaxf(d0 * z0 + d1 * z1 + d2 * z2, -1.0f), 1.0f));
        const int j = min(FP_BANDS - 1, max(0, (int)(ang * band_scale)));
        atomicMin(&s_min[j], __float_as_uint(lmin));
        atomicMax(&s_max[j], __float_as_uint(top_p));
    }
    for (int o = 16; o > 0; o >>= 1) {
        best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        top = fmaxf(top, __shfl_xor_sync(0xffffffffu, top, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (best < 3.0e38f) atomicMin(out, __float_as_uint(best));
        atomicMax(out + 1 + FP_BANDS, __float_as_uint(top));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < FP_BANDS; j += blockDim.x) {
        if (s_min[j] != 0xffffffffu) atomicMin(out + 1 + j, s_min[j]);
        if (s_max[j] != 0u) atomicMax(out + 2 + FP_BANDS + j, s_max[j]);
    }
}

cudaError_t launch_footprint_min(const CamParams &c, const float *d, const float *dx, const float *dy,
                                 const uint8_t *valid, float *out, cudaStream_t s) {
    const int64_t P = (int64_t)c.W * c.H;
    cudaError_t e = cudaMemsetAsync(out, 0xff, sizeof(float) * (1 + FP_BANDS), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out + 1 + FP_BANDS, 0, sizeof(float) * (1 + FP_BANDS), s);
    if (e != cudaSuccess || P == 0) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(div_up(P, 256), 4 * (int64_t)num_sms());
    footprint_min_kernel<<<grid, 256, 0, s>>>(d, dx, dy, valid, P, c.R[2], c.R[5], c.R[8],
                                              reinterpret_cast<unsigned int *>(out));
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ray_table(const CamParams &c, float *d, float *dx, float *dy, uint8_t *valid, cudaStream_t s) {
    const int64_t P = (int64_t)c.W * c.H;
    if (P == 0) return cudaSuccess;
    ray_table_kernel<<<(unsigned)div_up(P, 256), 256, 0, s>>>(c, d, dx, dy, valid);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
