// Stencil kernels for the SE15 gauge (15-bit, one exponent per link) / INT20 spinor / float compute triplet.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_int20se(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_SE15, S_INT20, float>(long_recon, reduce, cfg, a, s);
}
}  // namespace hisq
