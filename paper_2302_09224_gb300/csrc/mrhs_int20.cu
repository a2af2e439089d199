// Batched-RHS stencil kernels for the FIX16 gauge / INT20 spinor / float compute triplet.
#include "dslash_mrhs.cuh"

namespace hisq {
bool launch_mrhs_int20(int long_recon, bool reduce, int T, int variant, const DslashMArgs &a, cudaStream_t s)
{
    return launch_mrhs_t<G_FIX16, S_INT20, float>(long_recon, reduce, T, variant, a, s);
}
}  // namespace hisq
