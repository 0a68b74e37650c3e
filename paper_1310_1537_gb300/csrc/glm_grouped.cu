// Grouped (hierarchical) pass: not built yet.
#include "glm_internal.cuh"

namespace glm {

glm_status_t launch_grouped(glm_ctx *, const void *, const float *, const uint8_t *,
                            const int64_t *, int, const float *, const float *, double, double *,
                            float *, cudaStream_t)
{
    return GLM_ERR_UNSUPPORTED;
}

}  // namespace glm
