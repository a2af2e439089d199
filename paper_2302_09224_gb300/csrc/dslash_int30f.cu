// Stencil kernels for the FIX32 gauge / INT30 spinor / float compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_int30f(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_FIX32, S_INT30, float>(long_recon, reduce, cfg, a, s);
}
bool launch_mee_int30f(int long_recon, int cfg, const MeeArgs &m, cudaStream_t s)
{
    return launch_mee_fused_t<G_FIX32, S_INT30, float>(long_recon, cfg, m, s);
}
}  // namespace hisq
