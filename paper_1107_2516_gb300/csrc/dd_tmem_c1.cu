// Kernel 4 instantiation of tile configuration kTmemCfg[1].
#include "dd_tmem_impl.cuh"

namespace dd {

cudaError_t tmem_launch_c1(dd_dtype t, const TmemLaunch &a, cudaStream_t s)
{
    return tmem_launch_cfg<kTmemCfg[1].n, kTmemCfg[1].dbw, kTmemCfg[1].nw, kTmemCfg[1].tpw>(t, a, s);
}

cudaError_t tmem_prepare_c1(size_t optin)
{
    return tmem_prepare_cfg<kTmemCfg[1].n, kTmemCfg[1].dbw, kTmemCfg[1].nw, kTmemCfg[1].tpw>(optin);
}

}  // namespace dd
