// Instantiations of the fused CUDA-core pass for one storage type of X.
#include "glm_fused.cuh"

namespace glm {

glm_status_t launch_fused_fp8(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s)
{
    return launch_fused_t<FP8Tag>(h, p, kc, s);
}

}  // namespace glm
