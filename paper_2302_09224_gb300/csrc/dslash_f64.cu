// Stencil kernels for the F64 gauge / F64 spinor / double compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_f64(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_F64, S_F64, double>(long_recon, reduce, cfg, a, s);
}
}  // namespace hisq
