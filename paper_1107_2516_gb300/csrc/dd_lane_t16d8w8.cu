// Kernel 3 instantiation: 16 samples per lane, 8 DM trials per warp, 8 warps per block.
#include "dd_lane_impl.cuh"

namespace dd {

cudaError_t lane_launch_t16d8w8(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    return lane_launch_cfg<16, 8, 8>(t, a, s);
}

cudaError_t lane_prepare_t16d8w8(size_t optin) { return lane_prepare_cfg<16, 8, 8>(optin); }

}  // namespace dd
