// reduce.cuh -- deterministic FP64 reductions fused into producing kernels.
//
// Each block reduces its threads' values with a fixed shuffle/shared-memory
// tree and writes one partial per value; the last block to finish (detected
// with a device-scope counter) sums the partials in a fixed order, so the
// result depends only on the grid shape, never on block scheduling.  The last
// block then runs a finisher that updates the solver's device-side scalars,
// which keeps a whole iteration on the device (and capturable in a graph).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hisq {

template <int NR>
__device__ __forceinline__ void warp_sum(double v[NR])
{
#pragma unroll
    for (int k = 0; k < NR; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Sum over the block; the result is valid in thread 0 only.
template <int NR>
__device__ __forceinline__ void block_sum(double v[NR], double (*sh)[NR])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    warp_sum<NR>(v);
    __syncthreads();  // sh may be reused from a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NR; k++) sh[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) v[k] = lane < nw ? sh[lane][k] : 0.0;
        warp_sum<NR>(v);
    }
}

// Returns true in every thread of the last block, with the grid totals in
// `tot` (shared memory).  All threads of every block must call it.  Grids may
// be two-dimensional (blocks are numbered x fastest).
template <int NR>
__device__ bool reduce_grid(double v[NR], const RedBuf &rb, double *tot)
{
    __shared__ double sh[32][NR];
    __shared__ int is_last;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    block_sum<NR>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) rb.partials[(size_t)bid * NR + k] = v[k];
        __threadfence();
        const unsigned prev = atomicAdd(rb.counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // every block's partials: coherent L2 loads (ld.cg), U rows per thread in
    // flight at once (one L2 round trip per U rows); the order is fixed
    constexpr int U = NR <= 4 ? 8 : NR <= 8 ? 4 : 1;
    double w[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) w[k] = 0.0;
    const unsigned step = blockDim.x;
    for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * step) {
        double tmp[U][NR];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned b = b0 + u * step;
#pragma unroll
            for (int k = 0; k < NR; k++) tmp[u][k] = b < nblocks ? __ldcg(rb.partials + (size_t)b * NR + k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int k = 0; k < NR; k++) w[k] += tmp[u][k];
    }
    block_sum<NR>(w, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) {
            tot[k] = w[k];
            rb.result[k] = w[k];
        }
        *rb.counter = 0u;
    }
    __syncthreads();
    return true;
}

}  // namespace hisq
