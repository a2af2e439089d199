// The summing launch after a reducing stencil pass, on its own: callers that
// time the stencil pass alone defer it (DslashArgs::defer_finish) and launch
// it here, with the block count of the launch shape the pass used.
#include "dslash.cuh"

namespace hisq {

unsigned dslash_partials(int gf, int sf, int cf, int long_recon, const Geom &g)
{
    const int cfg = stencil_config(gf, sf, cf, long_recon, true, g);
    return (unsigned)((g.vh + stencil_block(cfg) - 1) / stencil_block(cfg));
}

bool launch_dslash_finish(int gf, int sf, int cf, int long_recon, const DslashArgs &a, cudaStream_t s)
{
    const unsigned nb = dslash_partials(gf, sf, cf, long_recon, a.g);
    if (cf == HISQ_COMPUTE_F64 && sf == S_F64)
        launch_chained(stencil_finish_kernel<double>, dim3(1), dim3(1024), s, a.red, nb, a.fin, a.st, a.slot, a.active);
    else if (cf == HISQ_COMPUTE_F64)
        launch_chained(stencil_finish_kernel<ff>, dim3(1), dim3(1024), s, a.red, nb, a.fin, a.st, a.slot, a.active);
    else
        launch_chained(stencil_finish_kernel<float>, dim3(1), dim3(1024), s, a.red, nb, a.fin, a.st, a.slot, a.active);
    return true;
}

}  // namespace hisq
