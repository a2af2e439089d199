// blas.h -- argument block and launchers of the fused BLAS-1 kernels.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hisq {

struct BlasArgs {
    int n;                   // sites of the (half-lattice) fields
    char *v0;                // sloppy fields (meaning per kernel)
    char *v1;
    char *v2;
    double *x64;             // FP64 planar fields
    const double *b64;
    const double *ax64;
    double *r64;
    size_t slot_bytes;       // x_flush: bytes between ring slots
    int nslots;
    int clear_ring;          // p_update: zero the alpha ring (block 0)
    int slot;                // ring slot for finishers
    const int *active;       // skip when *active == 0 (null: always run)
    int *err;
    RedBuf red;
    CGState *st;
    int fin;                 // finisher override (0: the kernel's CG default)
    void *fst;               // state for the override finisher
    const double *alpha_src; // r_update: step size (null: st->alpha)
    int split;               // CG chain without one-block launches: r_update takes alpha from the
                             // reducing stencil pass's block partials, p_update beta from r_update's
    unsigned nparts;         // split: block partials left by the previous kernel
};

// Returns the number of block partials a split r_update leaves (0 otherwise).
unsigned launch_r_update(int sf, int cf, const BlasArgs &a, cudaStream_t s);
void launch_p_update(int sf, int cf, const BlasArgs &a, cudaStream_t s);
void launch_x_flush(int sf, int cf, const BlasArgs &a, cudaStream_t s);
void launch_true_residual(int sf, int cf, const BlasArgs &a, cudaStream_t s);
void launch_p_reliable(int sf, int cf, const BlasArgs &a, cudaStream_t s);
void launch_norm2(const BlasArgs &a, cudaStream_t s);  // |x64|^2 -> red.result[0]

}  // namespace hisq
