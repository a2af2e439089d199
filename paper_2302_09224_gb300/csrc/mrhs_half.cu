// Batched-RHS stencil kernels for the FIX16 gauge / HALF spinor / float compute triplet.
#include "dslash_mrhs.cuh"

namespace hisq {
bool launch_mrhs_half(int long_recon, bool reduce, int T, int variant, const DslashMArgs &a, cudaStream_t s)
{
    return launch_mrhs_t<G_FIX16, S_HALF, float>(long_recon, reduce, T, variant, a, s);
}
}  // namespace hisq
