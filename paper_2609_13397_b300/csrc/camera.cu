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

cudaError_t launch_ray_table(const CamParams &c, float *d, float *dx, float *dy, uint8_t *valid, cudaStream_t s) {
    const int64_t P = (int64_t)c.W * c.H;
    if (P == 0) return cudaSuccess;
    ray_table_kernel<<<(unsigned)div_up(P, 256), 256, 0, s>>>(c, d, dx, dy, valid);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
