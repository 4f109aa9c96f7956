// K2: per-Gaussian preprocess.
//
// K2a (camera independent, run by set_scene): R from the normalised
// quaternion, s = exp(log s), the footprint floor of Eq. 10
// (s_eff = sqrt(s^2 + rho^2), sigma_eff = sigma prod s/s_eff) and the
// whitening W_eff = S_eff^-1 R^T of Sec. 3.
// K2b (per view, run by render): o_u = W_eff (o - mu), the SH colour seen
// along (mu - o)/|mu - o|, and the binning rule's direction / depth key.
// The raster record is 5 float4 per Gaussian:
//   [W row 0 | o_u.x] [W row 1 | o_u.y] [W row 2 | o_u.z] [rgb | sigma_eff] [rho^2, 0, 0, 0]
#include "rule.cuh"

namespace conegs {

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9]) {
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

__global__ void __launch_bounds__(256) scene_cache_kernel(SceneParams sp, float *__restrict__ Wout,
                                                          float *__restrict__ sig_eff) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    float R[9];
    quat_to_rot(sp.quats[4 * i], sp.quats[4 * i + 1], sp.quats[4 * i + 2], sp.quats[4 * i + 3], R);
    const float rho2 = sp.rho2 ? sp.rho2[i] : 0.0f;
    const float logit = load_scalar(sp.logits, i, sp.storage);
    float sig = 1.0f / (1.0f + expf(-logit));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = expf(sp.log_scales[3 * i + a]);
        const float seff = sqrtf(s * s + rho2);
        sig *= s / seff;
        const float inv = 1.0f / seff;
#pragma unroll
        for (int b = 0; b < 3; ++b) Wout[9 * i + 3 * a + b] = R[3 * b + a] * inv;   // W_ab = R_ba / s_eff,a
    }
    sig_eff[i] = sig;
}

// Real SH basis to degree 3 (positive constants, l-major, m = -l..l).
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

// Per view: binning direction/depth (the FP32 rule) and the raster record.
__global__ void __launch_bounds__(256) view_records_kernel(CamParams c, SceneParams sp, float4 *__restrict__ rec,
                                                           float4 *__restrict__ gview,
                                                           uint8_t *__restrict__ gflag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    const float mu[3] = {sp.means[3 * i], sp.means[3 * i + 1], sp.means[3 * i + 2]};
    float flag = sp.binrec[6 * i + 5], u[3], L;
    rule_gauss_view(c, mu, flag, u, L);
    gview[i] = make_float4(u[0], u[1], u[2], L);
    gflag[i] = (uint8_t)flag;
    if (flag == 0.0f) return;
    float W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = sp.W[9 * i + k];
    const float w0 = c.o[0] - mu[0], w1 = c.o[1] - mu[1], w2 = c.o[2] - mu[2];
    float ou[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ou[a] = W[3 * a] * w0 + W[3 * a + 1] * w1 + W[3 * a + 2] * w2;
    // SH colour along (mu - o)/|mu - o|
    float dx = u[0], dy = u[1], dz = u[2];
    if (!(L > 0.0f)) { dx = 0.f; dy = 0.f; dz = 1.f; }
    float Y[16];
    sh_basis(dx, dy, dz, sp.sh_degree, Y);
    const int K = (sp.sh_degree + 1) * (sp.sh_degree + 1);
    float col[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
        for (int j = 0; j < K; ++j) acc += load_scalar(sp.sh, (i * K + j) * 3 + ch, sp.storage) * Y[j];
        col[ch] = fmaxf(acc + 0.5f, 0.0f);
    }
    float4 *r = rec + (size_t)REC_F4 * i;
    r[0] = make_float4(W[0], W[1], W[2], ou[0]);
    r[1] = make_float4(W[3], W[4], W[5], ou[1]);
    r[2] = make_float4(W[6], W[7], W[8], ou[2]);
    r[3] = make_float4(col[0], col[1], col[2], sp.sig_eff[i]);
    r[4] = make_float4(sp.rho2 ? sp.rho2[i] : 0.0f, 0.f, 0.f, 0.f);
}

cudaError_t launch_scene_cache(const SceneParams &sp, float *W, float *sig_eff, cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    scene_cache_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(sp, W, sig_eff);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_view_records(const CamParams &c, const SceneParams &sp, float4 *rec, float4 *gview,
                                uint8_t *gflag, cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    view_records_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(c, sp, rec, gview, gflag);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
