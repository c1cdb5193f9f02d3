// Tensor-core convolution path (placeholder until the tcgen05 kernel lands).
#include "interp.h"

namespace fvv {
int tc_prepare(fvv_interp *, const float *) {
    set_error("tensor-core path not built");
    return FVV_EINVAL;
}
int tc_conv(fvv_interp *, int, const void *, int, int, int, int, int, void *, int, int, bool, cudaStream_t) {
    set_error("tensor-core path not built");
    return FVV_EINVAL;
}
} // namespace fvv
