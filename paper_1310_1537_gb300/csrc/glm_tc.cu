// Tensor-core (tcgen05) batched pass: not built yet.
#include "glm_internal.cuh"

namespace glm {

bool tc_supported(const glm_ctx *) { return false; }

glm_status_t launch_tc(glm_ctx *, const void *, const float *, const uint8_t *, const float *, int,
                       double *, float *, cudaStream_t)
{
    return GLM_ERR_UNSUPPORTED;
}

}  // namespace glm
