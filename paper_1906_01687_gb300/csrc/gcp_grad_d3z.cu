// Instantiations of the fused sampled-gradient kernel for 3 modes with
// the stratified zeros made in the launch (layout 3).
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d3z(int L, int NC, bool bf16)
{
    return bf16 ? grad_kernel_ptr_variant<3, true, 3>(L, NC) : grad_kernel_ptr_variant<3, false, 3>(L, NC);
}
}  // namespace gcpk
