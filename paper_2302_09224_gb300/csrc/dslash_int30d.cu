// Stencil kernels for the FIX32 gauge / INT30 spinor / FP64-class compute
// triplet: the compute precision is carried by FP32 pairs (ff.cuh) on GB300,
// whose FP64 pipe would make this triplet slower than plain FP64.
#include "dslash.cuh"

namespace hisq {
bool launch_dslash_int30d(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    return launch_dslash_t<G_FIX32, S_INT30, ff>(long_recon, reduce, cfg, a, s);
}
}  // namespace hisq
