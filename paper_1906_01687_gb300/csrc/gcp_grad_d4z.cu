// Instantiations of the fused sampled-gradient kernel for 4 modes with
// the stratified zeros made in the launch (layout 3).
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d4z(int L, int NC, bool bf16)
{
    return bf16 ? grad_kernel_ptr_variant<4, true, 3>(L, NC) : grad_kernel_ptr_variant<4, false, 3>(L, NC);
}
}  // namespace gcpk
