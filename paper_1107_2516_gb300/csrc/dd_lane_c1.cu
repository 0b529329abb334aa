// Kernel 3 instantiation of tile configuration kLaneCfg[1].
#include "dd_lane_impl.cuh"

namespace dd {

cudaError_t lane_launch_c1(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    return lane_launch_cfg<kLaneCfg[1].ti, kLaneCfg[1].dr, kLaneCfg[1].nw, kLaneCfg[1].minb>(t, a, s);
}

cudaError_t lane_prepare_c1(size_t optin)
{
    return lane_prepare_cfg<kLaneCfg[1].ti, kLaneCfg[1].dr, kLaneCfg[1].nw, kLaneCfg[1].minb>(optin);
}

cudaError_t lane_batch_launch_c1(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    return lane_batch_launch_cfg<kLaneCfg[1].ti, kLaneCfg[1].dr, kLaneCfg[1].nw, kLaneCfg[1].minb>(b, sms, smem, s);
}

}  // namespace dd
