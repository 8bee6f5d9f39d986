// Tensor-core forward of the learned initialiser's 32 -> 32 channel layers.
#include "cnn_internal.h"

reg_status cnn_conv32_tc(const float *, int, const float *, float *, int, int, cudaStream_t)
{
    return reg_internal_fail(REG_EINVAL, "tensor-core convolution not available in this build");
}
