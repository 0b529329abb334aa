// Kernel 3 instantiation of tile configuration kLaneCfg[0].
#include "dd_lane_impl.cuh"

namespace dd {

cudaError_t lane_launch_c0(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    return lane_launch_cfg<kLaneCfg[0].ti, kLaneCfg[0].dr, kLaneCfg[0].nw, kLaneCfg[0].minb>(t, a, s);
}

cudaError_t lane_prepare_c0(size_t optin)
{
    return lane_prepare_cfg<kLaneCfg[0].ti, kLaneCfg[0].dr, kLaneCfg[0].nw, kLaneCfg[0].minb>(optin);
}

cudaError_t lane_batch_launch_c0(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    return lane_batch_launch_cfg<kLaneCfg[0].ti, kLaneCfg[0].dr, kLaneCfg[0].nw, kLaneCfg[0].minb>(b, sms, smem, s);
}

}  // namespace dd
