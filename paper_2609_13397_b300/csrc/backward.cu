// K6/K7 placeholder (filled in by the adjoint implementation).
#include "common.cuh"
namespace conegs {
struct RasterArgs;
cudaError_t launch_backward(const RasterArgs &, int, bool, const float *, const float *, const float *, float *,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_backward_params(const CamParams &, const SceneParams &, const float *, const uint8_t *,
                                   const float4 *, float *, float *, float *, float *, float *, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace conegs
