// Stencil kernels for the FIX16 gauge / INT14 spinor / float compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_int14(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_FIX16, S_INT14, float>(long_recon, reduce, cfg, a, s);
}
}  // namespace hisq
