// Real spherical harmonics to degree 3 (positive constants, l-major order with
// m = -l..l), as used for the view-dependent colour rgb = max(0, SH(u) + 1/2)
// along u = (mu - o)/|mu - o|.
#pragma once
#include "common.cuh"

namespace conegs {

struct ShC {
    static constexpr float Y0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    static constexpr float C1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
    static constexpr float C2A = 1.0925484305920792f;   // sqrt(15/pi)/2
    static constexpr float C2B = 0.31539156525252005f;  // sqrt(5/pi)/4
    static constexpr float C2C = 0.54627421529603959f;  // sqrt(15/pi)/4
    static constexpr float C3A = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
    static constexpr float C3B = 2.8906114426405538f;   // sqrt(105/pi)/2
    static constexpr float C3C = 0.45704579946446572f;  // sqrt(21/(2 pi))/4
    static constexpr float C3D = 0.37317633259011540f;  // sqrt(7/pi)/4
    static constexpr float C3E = 1.4453057213202769f;   // sqrt(105/pi)/4
};

__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float Y[16]) {
    Y[0] = ShC::Y0;
    if (deg < 1) return;
    Y[1] = ShC::C1 * y; Y[2] = ShC::C1 * z; Y[3] = ShC::C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = ShC::C2A * x * y;
    Y[5] = ShC::C2A * y * z;
    Y[6] = ShC::C2B * (3.f * zz - 1.f);
    Y[7] = ShC::C2A * x * z;
    Y[8] = ShC::C2C * (xx - yy);
    if (deg < 3) return;
    Y[9] = ShC::C3A * y * (3.f * xx - yy);
    Y[10] = ShC::C3B * x * y * z;
    Y[11] = ShC::C3C * y * (5.f * zz - 1.f);
    Y[12] = ShC::C3D * z * (5.f * zz - 3.f);
    Y[13] = ShC::C3C * x * (5.f * zz - 1.f);
    Y[14] = ShC::C3E * z * (xx - yy);
    Y[15] = ShC::C3A * x * (xx - 3.f * yy);
}

// g += sum_j w_j dY_j/d(x, y, z) (the derivatives of the polynomials above).
__device__ __forceinline__ void sh_basis_grad_acc(float x, float y, float z, int deg, const float w[16], float g[3]) {
    if (deg < 1) return;
    g[0] += ShC::C1 * w[3];
    g[1] += ShC::C1 * w[1];
    g[2] += ShC::C1 * w[2];
    if (deg < 2) return;
    g[0] += ShC::C2A * (y * w[4] + z * w[7]) + 2.f * ShC::C2C * x * w[8];
    g[1] += ShC::C2A * (x * w[4] + z * w[5]) - 2.f * ShC::C2C * y * w[8];
    g[2] += ShC::C2A * (y * w[5] + x * w[7]) + 6.f * ShC::C2B * z * w[6];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += 6.f * ShC::C3A * x * y * w[9] + ShC::C3B * y * z * w[10] + ShC::C3C * (5.f * zz - 1.f) * w[13] +
            2.f * ShC::C3E * x * z * w[14] + ShC::C3A * (3.f * xx - 3.f * yy) * w[15];
    g[1] += ShC::C3A * (3.f * xx - 3.f * yy) * w[9] + ShC::C3B * x * z * w[10] + ShC::C3C * (5.f * zz - 1.f) * w[11] -
            2.f * ShC::C3E * y * z * w[14] - 6.f * ShC::C3A * x * y * w[15];
    g[2] += ShC::C3B * x * y * w[10] + 10.f * ShC::C3C * y * z * w[11] + ShC::C3D * (15.f * zz - 3.f) * w[12] +
            10.f * ShC::C3C * x * z * w[13] + ShC::C3E * (xx - yy) * w[14];
}

// rgb = max(0, sum_j c_j Y_j + 1/2) of Gaussian i, consuming the coefficients as
// they load (float4 loads for FP32 storage when 3K is a multiple of 4).
__device__ __forceinline__ void sh_colour(const void *sh, int64_t i, int deg, int storage, const float Y[16],
                                          float col[3]) {
    const int K = (deg + 1) * (deg + 1), n = 3 * K;
    float acc[3] = {0.5f, 0.5f, 0.5f};
    if (storage == 0 && (n & 3) == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(sh) + (size_t)n * i);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            if (4 * q < n) {
                const float4 v = p[q];
                acc[(4 * q) % 3] += v.x * Y[(4 * q) / 3];
                acc[(4 * q + 1) % 3] += v.y * Y[(4 * q + 1) / 3];
                acc[(4 * q + 2) % 3] += v.z * Y[(4 * q + 2) / 3];
                acc[(4 * q + 3) % 3] += v.w * Y[(4 * q + 3) / 3];
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 48; ++q)
            if (q < n) acc[q % 3] += load_scalar(sh, (int64_t)n * i + q, storage) * Y[q / 3];
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(acc[ch], 0.0f);
}

// The 3K colour coefficients of Gaussian i (c[3 j + channel]), K = (deg + 1)^2:
// float4 loads for FP32 storage when 3K is a multiple of 4 (degrees 1 and 3).
__device__ __forceinline__ void load_sh(const void *sh, int64_t i, int K, int storage, float c[48]) {
    const int n = 3 * K;
    if (storage == 0 && (n & 3) == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(sh) + (size_t)n * i);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            if (4 * q < n) {
                const float4 v = p[q];
                c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
            }
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 48; ++q)
        if (q < n) c[q] = load_scalar(sh, (int64_t)n * i + q, storage);
}

}  // namespace conegs
