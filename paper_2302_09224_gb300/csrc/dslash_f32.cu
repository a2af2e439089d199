// Stencil kernels for the F32 gauge / F32 spinor / float compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_f32(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_F32, S_F32, float>(long_recon, reduce, cfg, a, s);
}
bool launch_mee_f32(int long_recon, int cfg, const MeeArgs &m, cudaStream_t s)
{
    return launch_mee_fused_t<G_F32, S_F32, float>(long_recon, cfg, m, s);
}
}  // namespace hisq
