// Stencil kernels for the FIX32 gauge / INT30 spinor / double compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_int30d(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_FIX32, S_INT30, double>(long_recon, reduce, cfg, a, s);
}
}  // namespace hisq
