// Dispatch from a runtime precision triplet to the compiled stencil kernels.
#include "internal.h"

namespace hisq {

bool launch_dslash_f64(int, bool, const DslashArgs &, cudaStream_t);
bool launch_dslash_f32(int, bool, const DslashArgs &, cudaStream_t);
bool launch_dslash_half(int, bool, const DslashArgs &, cudaStream_t);
bool launch_dslash_int20(int, bool, const DslashArgs &, cudaStream_t);
bool launch_dslash_int30d(int, bool, const DslashArgs &, cudaStream_t);
bool launch_dslash_int30f(int, bool, const DslashArgs &, cudaStream_t);

bool launch_dslash(int gf, int sf, int cf, int long_recon, bool reduce, const DslashArgs &a, cudaStream_t s)
{
    const bool f64 = cf == HISQ_COMPUTE_F64;
    if (gf == G_F64 && sf == S_F64 && f64) return launch_dslash_f64(long_recon, reduce, a, s);
    if (gf == G_F32 && sf == S_F32 && !f64) return launch_dslash_f32(long_recon, reduce, a, s);
    if (gf == G_FIX16 && sf == S_HALF && !f64) return launch_dslash_half(long_recon, reduce, a, s);
    if (gf == G_FIX16 && sf == S_INT20 && !f64) return launch_dslash_int20(long_recon, reduce, a, s);
    if (gf == G_FIX32 && sf == S_INT30) {
        if (f64) return launch_dslash_int30d(long_recon, reduce, a, s);
        return launch_dslash_int30f(long_recon, reduce, a, s);
    }
    return false;
}

}  // namespace hisq
