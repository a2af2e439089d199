// reduce.cuh -- deterministic reductions fused into producing kernels.
//
// Each block reduces its threads' values with a fixed shuffle/shared-memory
// tree and writes one partial per value; the last block to finish (detected
// with a device-scope counter) sums the partials in a fixed order, so the
// result depends only on the grid shape, never on block scheduling.  The last
// block then runs a finisher that updates the solver's device-side scalars,
// which keeps a whole iteration on the device (and capturable in a graph).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "ff.cuh"
#include "internal.h"

namespace hisq {

// Type of a thread's sums: the compute type (FP32 pairs stay pairs; their
// block sums run in pair arithmetic, see below).
template <typename real>
using red_t = real;

template <int NR, typename T>
__device__ __forceinline__ void warp_sum(T v[NR])
{
#pragma unroll
    for (int k = 0; k < NR; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Sum over the block in the values' own type; valid in thread 0 only.
template <int NR, typename T>
__device__ __forceinline__ void block_sum(T v[NR], T (*sh)[NR])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    warp_sum<NR, T>(v);
    __syncthreads();  // sh may be reused from a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NR; k++) sh[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) v[k] = lane < nw ? sh[lane][k] : T(0);
        warp_sum<NR, T>(v);
    }
}

// An unevaluated FP32 pair hi + lo (about 44 significant bits) and its sum by
// Knuth's error-free TwoSum: every step a plain FP32 add (no contraction), so
// the FP32 pipe carries the cross-block sum instead of the narrow FP64 pipe.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fadd_rn(s, -a.hi);
    float e = __fadd_rn(__fadd_rn(a.hi, -__fadd_rn(s, -bb)), __fadd_rn(b.hi, -bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return {hi, __fadd_rn(e, -__fadd_rn(hi, -s))};
}

// Type of the block partials: the compute type, an FP32 pair for pairs (the
// one block that sums them then stays on the FP32 pipe: FP64 adds of several
// thousand partials on one SM's narrow FP64 pipe took longer than the sum).
template <typename real>
using part_t = std::conditional_t<is_ff<real>::value, FF, real>;

template <int NR>
__device__ __forceinline__ void warp_sum_ff(FF v[NR])
{
#pragma unroll
    for (int k = 0; k < NR; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const FF o = {__shfl_down_sync(0xffffffffu, v[k].hi, off), __shfl_down_sync(0xffffffffu, v[k].lo, off)};
            v[k] = ff_add(v[k], o);
        }
}

// One block sums the partials of nblocks blocks (in a fixed order) into tot
// (shared memory), valid in thread 0: FP64 partials in FP64, FP32 partials and
// FP32-pair partials in the FP32 pair arithmetic.
template <int NR, typename T>
__device__ void sum_partials(const RedBuf &rb, unsigned nblocks, double *tot)
{
    __shared__ T sh[32][NR];
    const T *part = reinterpret_cast<const T *>(rb.partials);
    // every block's partials: coherent L2 loads (ld.cg), U rows per thread in
    // flight at once (one L2 round trip per U rows); the order is fixed
    constexpr int U = NR <= 4 ? 8 : NR <= 8 ? 4 : 1;
    const unsigned step = blockDim.x;
    if constexpr (std::is_same<T, FF>::value) {
        const float2 *pp = reinterpret_cast<const float2 *>(rb.partials);
        FF w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) w[k] = {0.0f, 0.0f};
        for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * step) {
            float2 tmp[U][NR];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const unsigned b = b0 + u * step;
#pragma unroll
                for (int k = 0; k < NR; k++)
                    tmp[u][k] = b < nblocks ? __ldcg(pp + (size_t)b * NR + k) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < NR; k++) w[k] = ff_add(w[k], FF{tmp[u][k].x, tmp[u][k].y});
        }
        __shared__ FF shp[32][NR];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int nw = (blockDim.x + 31) >> 5;
        warp_sum_ff<NR>(w);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NR; k++) shp[wid][k] = w[k];
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; k++) w[k] = lane < nw ? shp[lane][k] : FF{0.0f, 0.0f};
            warp_sum_ff<NR>(w);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < NR; k++) tot[k] = (double)w[k].hi + (double)w[k].lo;
        }
    } else if constexpr (sizeof(T) == 8) {
        double w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) w[k] = 0.0;
        for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * step) {
            double tmp[U][NR];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const unsigned b = b0 + u * step;
#pragma unroll
                for (int k = 0; k < NR; k++) tmp[u][k] = b < nblocks ? __ldcg(part + (size_t)b * NR + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < NR; k++) w[k] += tmp[u][k];
        }
        block_sum<NR, double>(w, sh);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NR; k++) tot[k] = w[k];
    } else {
        FF w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) w[k] = {0.0f, 0.0f};
        for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * step) {
            float tmp[U][NR];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const unsigned b = b0 + u * step;
#pragma unroll
                for (int k = 0; k < NR; k++) tmp[u][k] = b < nblocks ? __ldcg(part + (size_t)b * NR + k) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < NR; k++) w[k] = ff_add(w[k], FF{tmp[u][k], 0.0f});
        }
        __shared__ FF shf[32][NR];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int nw = (blockDim.x + 31) >> 5;
        warp_sum_ff<NR>(w);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NR; k++) shf[wid][k] = w[k];
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; k++) w[k] = lane < nw ? shf[lane][k] : FF{0.0f, 0.0f};
            warp_sum_ff<NR>(w);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < NR; k++) tot[k] = (double)w[k].hi + (double)w[k].lo;
        }
    }
}

// Warp 0 alone sums the partials of nblocks blocks (few: a wave of blocks) in
// the FP32 pair arithmetic (FP64 partials in FP64), in a fixed order (lane l
// takes rows l, l + 32, ..., then the warp's tree); the totals land in tot
// (shared memory), valid in thread 0.  The other warps do not take part (no
// block barrier).
template <int NR, typename T>
__device__ void warp0_sum_partials(const RedBuf &rb, unsigned nblocks, double *tot)
{
    if (threadIdx.x >= 32) return;
    constexpr int U = 4;
    if constexpr (std::is_same<T, double>::value) {  // FP64 partials, summed in FP64
        double w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) w[k] = 0.0;
        for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * 32) {
            double tmp[U][NR];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const unsigned b = b0 + u * 32;
#pragma unroll
                for (int k = 0; k < NR; k++)
                    tmp[u][k] = b < nblocks ? __ldcg(reinterpret_cast<const double *>(rb.partials) + (size_t)b * NR + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < NR; k++) w[k] += tmp[u][k];
        }
        warp_sum<NR, double>(w);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NR; k++) tot[k] = w[k];
    } else {
        static_assert(std::is_same<T, FF>::value || std::is_same<T, float>::value, "FP32 or FP32-pair partials");
        FF w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) w[k] = {0.0f, 0.0f};
        for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * 32) {
            FF tmp[U][NR];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const unsigned b = b0 + u * 32;
#pragma unroll
                for (int k = 0; k < NR; k++) {
                    if constexpr (std::is_same<T, FF>::value) {
                        const float2 v = b < nblocks
                                             ? __ldcg(reinterpret_cast<const float2 *>(rb.partials) + (size_t)b * NR + k)
                                             : make_float2(0.0f, 0.0f);
                        tmp[u][k] = FF{v.x, v.y};
                    } else {
                        tmp[u][k] = FF{b < nblocks ? __ldcg(reinterpret_cast<const float *>(rb.partials) + (size_t)b * NR + k)
                                                   : 0.0f,
                                       0.0f};
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < NR; k++) w[k] = ff_add(w[k], tmp[u][k]);
        }
        warp_sum_ff<NR>(w);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NR; k++) tot[k] = (double)w[k].hi + (double)w[k].lo;
    }
}

// Returns true in every thread of the last block, with the grid totals in
// `tot` (shared memory).  All threads of every block must call it.  Grids may
// be two-dimensional (blocks are numbered x fastest).
//
// FP64 values (FP64 compute) are summed in FP64 throughout.  FP32 values (one
// thread's sites formed in the FP32 compute precision) are summed in FP32 up
// to the block, each block storing one FP32 partial; the last block sums the
// partials in the FP32 pair arithmetic above and returns hi + lo in FP64.  On
// GB300 the FP64 pipe issues a small fraction of the FP32 rate, so FP64
// arithmetic in every block (or a long FP64 chain in the last one) dominated
// the short reducing kernels.
template <int NR, typename T>
__device__ bool reduce_grid(const T vin[NR], const RedBuf &rb, double *tot)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "float or double");
    __shared__ T sh[32][NR];
    __shared__ int is_last;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    T *part = reinterpret_cast<T *>(rb.partials);
    T v[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) v[k] = vin[k];
    block_sum<NR, T>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) part[(size_t)bid * NR + k] = v[k];
        __threadfence();
        const unsigned prev = atomicAdd(rb.counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    sum_partials<NR, T>(rb, nblocks, tot);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) rb.result[k] = tot[k];
        *rb.counter = 0u;
    }
    __syncthreads();
    return true;
}

// FP32-pair values (the FP64-class kernels): the block sums them in pair
// arithmetic (TwoSum at every level of the same fixed tree, nothing on the
// narrow FP64 pipe) and stores its pair; the last block sums the pairs in the
// same arithmetic and returns hi + lo in FP64.
template <int NR>
__device__ __forceinline__ void block_sum_pairs(const ff vin[NR], FF v[NR])
{
    __shared__ FF sh[32][NR];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NR; k++) v[k] = FF{vin[k].hi, vin[k].lo};
    warp_sum_ff<NR>(v);
    __syncthreads();  // sh may be reused from a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NR; k++) sh[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) v[k] = lane < nw ? sh[lane][k] : FF{0.0f, 0.0f};
        warp_sum_ff<NR>(v);
    }
}

template <int NR>
__device__ bool reduce_grid(const ff vin[NR], const RedBuf &rb, double *tot)
{
    __shared__ int is_last;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    FF v[NR];
    block_sum_pairs<NR>(vin, v);
    if (threadIdx.x == 0) {
        float2 *part = reinterpret_cast<float2 *>(rb.partials);
#pragma unroll
        for (int k = 0; k < NR; k++) part[(size_t)bid * NR + k] = make_float2(v[k].hi, v[k].lo);
        __threadfence();
        const unsigned prev = atomicAdd(rb.counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    sum_partials<NR, FF>(rb, nblocks, tot);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; k++) rb.result[k] = tot[k];
        *rb.counter = 0u;
    }
    __syncthreads();
    return true;
}

template <int NR>
__device__ void store_block_partial(const ff vin[NR], const RedBuf &rb)
{
    FF v[NR];
    block_sum_pairs<NR>(vin, v);
    if (threadIdx.x == 0) {
        float2 *part = reinterpret_cast<float2 *>(rb.partials);
        const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
        for (int k = 0; k < NR; k++) part[(size_t)bid * NR + k] = make_float2(v[k].hi, v[k].lo);
    }
}

// Blocks of one full wave of a kernel on the current device: the grid of a
// reducing kernel that loops over its sites, so that the end of a reducing
// block (block sum, partial store, fence, counter) is paid once per resident
// block rather than once per block of sites.
template <typename K>
int wave_blocks(K kernel, int block)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

// Only this block's share: its sums stored at its index of rb.partials, no
// completion counter (a separate one-block kernel sums them after the launch).
template <int NR, typename T>
__device__ void store_block_partial(const T vin[NR], const RedBuf &rb)
{
    __shared__ T sh[32][NR];
    T v[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) v[k] = vin[k];
    block_sum<NR, T>(v, sh);
    if (threadIdx.x == 0) {
        T *part = reinterpret_cast<T *>(rb.partials);
        const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
        for (int k = 0; k < NR; k++) part[(size_t)bid * NR + k] = v[k];
    }
}

}  // namespace hisq
