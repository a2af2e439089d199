// Stencil kernels for the FIX16 gauge / HALF spinor / float compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_half(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_FIX16, S_HALF, float>(long_recon, reduce, cfg, a, s);
}
bool launch_mee_half(int long_recon, int cfg, const MeeArgs &m, cudaStream_t s)
{
    return launch_mee_fused_t<G_FIX16, S_HALF, float>(long_recon, cfg, m, s);
}
}  // namespace hisq
