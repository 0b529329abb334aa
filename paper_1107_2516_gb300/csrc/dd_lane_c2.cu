// Kernel 3 instantiation of tile configuration kLaneCfg[2].
#include "dd_lane_impl.cuh"

namespace dd {

cudaError_t lane_launch_c2(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    return lane_launch_cfg<kLaneCfg[2].ti, kLaneCfg[2].dr, kLaneCfg[2].nw, kLaneCfg[2].minb>(t, a, s);
}

cudaError_t lane_prepare_c2(size_t optin)
{
    return lane_prepare_cfg<kLaneCfg[2].ti, kLaneCfg[2].dr, kLaneCfg[2].nw, kLaneCfg[2].minb>(optin);
}

cudaError_t lane_batch_launch_c2(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    return lane_batch_launch_cfg<kLaneCfg[2].ti, kLaneCfg[2].dr, kLaneCfg[2].nw, kLaneCfg[2].minb>(b, sms, smem, s);
}

}  // namespace dd
