// Batched-RHS stencil kernels for the F32 gauge / F32 spinor / float compute triplet.
#include "dslash_mrhs.cuh"

namespace hisq {
bool launch_mrhs_f32(int long_recon, bool reduce, int T, int variant, const DslashMArgs &a, cudaStream_t s)
{
    return launch_mrhs_t<G_F32, S_F32, float>(long_recon, reduce, T, variant, a, s);
}
}  // namespace hisq
