// Kernel 3 instantiation of tile configuration kLaneCfg[3].
#include "dd_lane_impl.cuh"

namespace dd {

cudaError_t lane_launch_c3(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    return lane_launch_cfg<kLaneCfg[3].ti, kLaneCfg[3].dr, kLaneCfg[3].nw, kLaneCfg[3].minb>(t, a, s);
}

cudaError_t lane_prepare_c3(size_t optin)
{
    return lane_prepare_cfg<kLaneCfg[3].ti, kLaneCfg[3].dr, kLaneCfg[3].nw, kLaneCfg[3].minb>(optin);
}

cudaError_t lane_batch_launch_c3(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    return lane_batch_launch_cfg<kLaneCfg[3].ti, kLaneCfg[3].dr, kLaneCfg[3].nw, kLaneCfg[3].minb>(b, sms, smem, s);
}

}  // namespace dd
