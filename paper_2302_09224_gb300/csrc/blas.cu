// blas.cu -- fused BLAS-1 kernels of the stabilised mixed-precision CG
// (Sec. 3.1), each a single pass over its vectors in the sloppy storage
// format with the reduction it needs fused in (deterministic; see reduce_grid
// for the precision of each stage):
//   r_update      r <- r - alpha Ap,     |r|^2 and Re<r_new, r_old>  (PR beta;
//                 for the 30-bit FP64-class triplet from the stored records)
//   p_update      p' <- r + beta p       (into the next ring slot)
//                 (both also in a split form for the CG, below: alpha and beta
//                 summed by every block from the previous kernel's partials)
//   x_flush       x_hi <- x_hi + sum_j alpha_j p_j   (buffered gradient vectors)
//   true_residual r_hi <- b - A x_hi (FP64), r <- r_hi (sloppy),
//                 |r_hi|^2 and <r_hi, p> for the re-projection of p
//   p_reliable    p' <- coef r_hi + beta p   (re-projected FR restart)
//   norm2         |v|^2 of an FP64 field
#include <cuda_runtime.h>

#include "blas.h"
#include "codecs.cuh"
#include "finish.cuh"
#include "launch.cuh"
#include "reduce.cuh"

namespace hisq {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool skip(const int *active)
{
    return active != nullptr && *(volatile const int *)active == 0;
}

__device__ __forceinline__ bool nonzero(float v) { return v != 0.0f; }
__device__ __forceinline__ bool nonzero(double v) { return v != 0.0; }
__device__ __forceinline__ bool nonzero(ff v) { return v.hi != 0.0f || v.lo != 0.0f; }

// A solver scalar (FP64 in the state) in the compute precision.  For FP32
// pairs the conversion runs on GB300's narrow FP64 pipe, so one thread of the
// block converts and the block reads the pair from shared memory.  Every
// thread of the block calls it, at most once per kernel.
template <typename real>
__device__ __forceinline__ real block_scalar(const double *src)
{
    if constexpr (is_ff<real>::value) {
        __shared__ ff sh;
        if (threadIdx.x == 0) sh = ff(*src);
        __syncthreads();
        return sh;
    } else {
        return (real)*src;
    }
}

// A float as a double, exactly, built from its bits on the integer pipe
// (zero and normal floats; subnormal, infinite and NaN ones take the
// conversion instruction).
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0u || e == 0xffu) return (double)f;
    return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}

// Sites per thread of the two per-iteration BLAS kernels: every load of a
// thread's sites is issued before any of them is used (memory-level
// parallelism for these short, latency-bound kernels).  Four sites a thread
// (one pass over 2^20 sites) and a grid over all sites instead of one wave
// measured the same within 2 % in the 32^3x64 solve.
constexpr int kRSites = 2;
constexpr int kPSites = 2;

// Loads of r (v0) and Ap (v1) at the U sites i0 + u * blockDim.x.
template <int SF, int U, int C>
__device__ __forceinline__ void r_load(const BlasArgs &a, int i0, uint4 (&cr)[U][C], uint4 (&ca)[U][C])
{
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int i = i0 + u * blockDim.x;
        if (i < a.n) {
            Spinor<SF>::gather(a.v0, a.n, i, cr[u]);
            Spinor<SF>::gather(a.v1, a.n, i, ca[u]);
        }
    }
}

// r <- r - alpha Ap at those sites, stored; |r_new|^2 and Re<r_new, r_old> added to v.
template <int SF, typename real, int U, int C>
__device__ __forceinline__ void r_group(const BlasArgs &a, int i0, const uint4 (&cr)[U][C], const uint4 (&ca)[U][C],
                                        real alpha, red_t<real> v[2])
{
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int i = i0 + u * blockDim.x;
        if (i >= a.n) continue;
        if constexpr (SF == S_INT30 && is_ff<real>::value) {
            // FP64-class: the update in FP32 pairs; |r|^2 and Re<r_new, r_old> exactly in integers
            // from the stored 30-bit records (products of 30-bit integers, sums below 2^62)
            int32_t qr[6];
            const uint32_t Er = Spinor<S_INT30>::raw(cr[u], qr);
            ff r[6], ap[6], rn[6];
            Spinor<S_INT30>::decode(cr[u], r);
            Spinor<S_INT30>::decode(ca[u], ap);
#pragma unroll
            for (int k = 0; k < 6; k++) rn[k] = r[k] - alpha * ap[k];
            uint32_t qn[6], En;
            if (!Spinor<S_INT30>::store_ff_q(a.v0, a.n, i, rn, qn, En)) atomicExch(a.err, 1);
            long long n2 = 0, d = 0;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                asm("mad.wide.s32 %0, %1, %1, %0;" : "+l"(n2) : "r"((int)qn[k]));
                asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(d) : "r"((int)qn[k]), "r"(qr[k]));
            }
            // a record's value is q 2^(E-127)
            v[0] += ff_ldexp(ff_from_ll(n2), 2 * (int)En - 254);
            v[1] += ff_ldexp(ff_from_ll(d), (int)En + (int)Er - 254);
        } else {
            real r[6], ap[6], rn[6];
            Spinor<SF>::decode(cr[u], r);
            Spinor<SF>::decode(ca[u], ap);
            real n2 = real(0), d = real(0);  // in the compute precision; the block sums the threads
#pragma unroll
            for (int k = 0; k < 6; k++) {
                rn[k] = r[k] - alpha * ap[k];
                n2 += rn[k] * rn[k];
                d += rn[k] * r[k];
            }
            v[0] += (red_t<real>)n2;
            v[1] += (red_t<real>)d;
            if (!Spinor<SF>::store(a.v0, a.n, i, rn)) atomicExch(a.err, 1);
        }
    }
}

template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) r_update_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kRSites, C = Spinor<SF>::chunks;
    red_t<real> v[2] = {0, 0};
    const real alpha = block_scalar<real>(a.alpha_src ? a.alpha_src : &a.st->alpha);
    // one wave of blocks loops over groups of U sites per thread (see wave_blocks)
    for (int i0 = blockIdx.x * blockDim.x * U + threadIdx.x; i0 < a.n; i0 += gridDim.x * blockDim.x * U) {
        uint4 cr[U][C], ca[U][C];
        r_load<SF>(a, i0, cr, ca);
        r_group<SF, real>(a, i0, cr, ca, alpha, v);
    }
    __shared__ double tot[2];
    if (reduce_grid<2>(v, a.red, tot) && threadIdx.x == 0) {
        if (a.fin)
            run_finisher(a.fin, tot, a.fst, a.slot);
        else if (a.st)
            run_finisher(FIN_CG_BETA, tot, a.st, a.slot);
    }
}

template <int SF, int U, int C>
__device__ __forceinline__ void p_load(const BlasArgs &a, int i0, uint4 (&cr)[U][C], uint4 (&cp)[U][C])
{
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int i = i0 + u * blockDim.x;
        if (i < a.n) {
            Spinor<SF>::gather(a.v0, a.n, i, cr[u]);
            Spinor<SF>::gather(a.v1, a.n, i, cp[u]);
        }
    }
}

// p' = r + beta p at those sites, stored into v2.
template <int SF, typename real, int U, int C>
__device__ __forceinline__ void p_group(const BlasArgs &a, int i0, const uint4 (&cr)[U][C], const uint4 (&cp)[U][C],
                                        real beta)
{
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int i = i0 + u * blockDim.x;
        if (i >= a.n) continue;
        real r[6], p[6];
        Spinor<SF>::decode(cr[u], r);
        Spinor<SF>::decode(cp[u], p);
#pragma unroll
        for (int k = 0; k < 6; k++) p[k] = r[k] + beta * p[k];
        if (!Spinor<SF>::store(a.v2, a.n, i, p)) atomicExch(a.err, 1);
    }
}

template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) p_update_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kPSites, C = Spinor<SF>::chunks;
    const int i0 = blockIdx.x * blockDim.x * U + threadIdx.x;
    if (a.clear_ring && i0 == 0)
        for (int j = 0; j < kMaxBuf; j++) a.st->alpha_ring[j] = 0.0;
    uint4 cr[U][C], cp[U][C];
    p_load<SF>(a, i0, cr, cp);
    const real beta = block_scalar<real>(&a.st->beta);
    p_group<SF, real>(a, i0, cr, cp, beta);
}

// The CG iteration's scalar steps without one-block launches or last-block
// tails (BlasArgs::split).  Every block of r_update sums the reducing stencil
// pass's block partials itself, in the one fixed order of sum_partials, and
// takes alpha = |r|^2 / Re<p, Ap> from them; block 0 also runs the alpha
// finisher (alpha ring, breakdown) and copies |r|^2 to rr_den.  r_update
// leaves its own block partials in the second half of the partials buffer;
// warp 0 of every block of p_update sums those and takes beta with rr_den as
// denominator, and block 0 runs the beta finisher (reliable-update and
// convergence decisions, the new |r|^2): no other block reads what it writes.
// A block that starts after block 0 has stopped the iteration skips its
// update, which is then partial; the solver never reads that ring slot before
// rewriting it (the slot's alpha is zero until then).  Each block's first
// loads are issued before its partial sums, so the sums overlap them.
inline __device__ RedBuf split_half(RedBuf rb)
{
    rb.partials += kSplitHalf;
    return rb;
}

template <int SF, typename real, int BS>
__global__ void __launch_bounds__(BS) r_update_split_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kRSites, C = Spinor<SF>::chunks;
    const int step = gridDim.x * BS * U;
    int i0 = blockIdx.x * BS * U + threadIdx.x;
    uint4 cr[U][C], ca[U][C];
    r_load<SF>(a, i0, cr, ca);
    __shared__ double tot[2];
    __shared__ real al_sh;
    __shared__ int ok_sh;
    sum_partials<2, part_t<real>>(a.red, a.nparts, tot);
    if (threadIdx.x == 0) {
        const double al = a.st->rr / tot[0];
        const bool ok = tot[0] > 0.0 && isfinite(al);  // else the finisher stops the iteration
        al_sh = ok ? real(al) : real(0);
        ok_sh = ok;
    }
    __syncthreads();
    const bool ok = ok_sh;
    if (ok) {
        const real alpha = al_sh;
        red_t<real> v[2] = {0, 0};
        for (; i0 < a.n; i0 += step) {
            r_group<SF, real>(a, i0, cr, ca, alpha, v);
            r_load<SF>(a, i0 + step, cr, ca);
        }
        store_block_partial<2>(v, split_half(a.red));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->rr_den = a.st->rr;
        run_finisher(FIN_CG_ALPHA, tot, a.st, a.slot);
    }
}

template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) p_update_split_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kPSites, C = Spinor<SF>::chunks;
    if (a.clear_ring && blockIdx.x == 0 && threadIdx.x == 0)
        for (int j = 0; j < kMaxBuf; j++) a.st->alpha_ring[j] = 0.0;
    const int i0 = blockIdx.x * kBlock * U + threadIdx.x;  // one group of U sites a thread (the grid covers all)
    uint4 cr[U][C], cp[U][C];
    p_load<SF>(a, i0, cr, cp);
    __shared__ double tot[2];
    __shared__ real be_sh;
    __shared__ int ok_sh;
    warp0_sum_partials<2, part_t<real>>(split_half(a.red), a.nparts, tot);
    if (threadIdx.x == 0) {
        // the beta finisher's arithmetic (Polak-Ribiere or Fletcher-Reeves)
        const double rr_new = tot[0];
        const double be = (a.st->pr ? rr_new - tot[1] : rr_new) / a.st->rr_den;
        const bool ok = isfinite(rr_new) && isfinite(be);  // else the finisher stops the iteration
        be_sh = ok ? real(be) : real(0);
        ok_sh = ok;
    }
    __syncthreads();
    if (ok_sh) p_group<SF, real>(a, i0, cr, cp, be_sh);
    // after the update: the finisher's registers are not live beside the loaded fields
    if (blockIdx.x == 0 && threadIdx.x == 0) run_finisher(FIN_CG_BETA, tot, a.st, a.slot);
}

// x_hi += sum_{j < nslots} alpha_j p_j; slots are consecutive fields of
// slot_bytes each starting at v0.  Unused slots carry alpha_j = 0.
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) x_flush_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ real al_s[kMaxBuf];  // the step sizes in the compute precision, converted once per block
    if (threadIdx.x < kMaxBuf) al_s[threadIdx.x] = threadIdx.x < a.nslots ? (real)a.st->alpha_ring[threadIdx.x] : real(0);
    __syncthreads();
    if (i >= a.n) return;
    constexpr int G = 4, C = Spinor<SF>::chunks;  // slots whose loads are in flight together
    uint4 cx[Spinor<S_F64>::chunks];
    Spinor<S_F64>::gather(reinterpret_cast<const char *>(a.x64), a.n, i, cx);
    // the increment sum_j alpha_j p_j carries the sloppy vectors' precision,
    // so it is formed in the compute precision and added to x in FP64
    real dx[6] = {0, 0, 0, 0, 0, 0};
    for (int j0 = 0; j0 < a.nslots; j0 += G) {
        uint4 cp[G][C];
        real al[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const int j = j0 + g;
            al[g] = j < a.nslots ? al_s[j] : real(0);
            if (nonzero(al[g])) Spinor<SF>::gather(a.v0 + (size_t)j * a.slot_bytes, a.n, i, cp[g]);
        }
#pragma unroll
        for (int g = 0; g < G; g++) {
            if (!nonzero(al[g])) continue;
            real p[6];
            Spinor<SF>::decode(cp[g], p);
#pragma unroll
            for (int k = 0; k < 6; k++) dx[k] += al[g] * p[k];
        }
    }
    double x[6];
    Spinor<S_F64>::decode(cx, x);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if constexpr (is_ff<real>::value)  // hi and lo widened on the integer pipe: two FP64 adds per real
            x[k] += f2d_bits(dx[k].hi) + f2d_bits(dx[k].lo);
        else
            x[k] += (double)dx[k];
    }
    Spinor<S_F64>::store(reinterpret_cast<char *>(a.x64), a.n, i, x);
}

// r_hi = b - Ax (FP64); r (sloppy) = r_hi; sums for FIN_CG_TRUE with p = v1.
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) true_residual_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (i < a.n) {
        double b[6], ax[6], r[6];
        Spinor<S_F64>::load(reinterpret_cast<const char *>(a.b64), a.n, i, b);
        if (a.ax64 != nullptr)
            Spinor<S_F64>::load(reinterpret_cast<const char *>(a.ax64), a.n, i, ax);
        else
#pragma unroll
            for (int k = 0; k < 6; k++) ax[k] = 0.0;
#pragma unroll
        for (int k = 0; k < 6; k++) r[k] = b[k] - ax[k];
        Spinor<S_F64>::store(reinterpret_cast<char *>(a.r64), a.n, i, r);
        if (!Spinor<SF>::store(a.v0, a.n, i, r)) atomicExch(a.err, 1);
        real p[6];
        Spinor<SF>::load(a.v1, a.n, i, p);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double rr = r[2 * c], ri = r[2 * c + 1], pr = p[2 * c], pi = p[2 * c + 1];
            v[0] += rr * rr + ri * ri;
            v[1] += rr * pr + ri * pi;  // Re conj(r) p
            v[2] += rr * pi - ri * pr;  // Im conj(r) p
        }
    }
    __shared__ double tot[3];
    if (reduce_grid<3>(v, a.red, tot) && threadIdx.x == 0) {
        if (a.fin)
            run_finisher(a.fin, tot, a.fst, a.slot);
        else if (a.st)
            run_finisher(FIN_CG_TRUE, tot, a.st, a.slot);
    }
}

// p' = coef r_hi + beta p (coef complex); clears the alpha ring.
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) p_reliable_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0)
        for (int j = 0; j < kMaxBuf; j++) a.st->alpha_ring[j] = 0.0;
    if (i >= a.n) return;
    double r[6];
    real p[6], o[6];
    Spinor<S_F64>::load(reinterpret_cast<const char *>(a.r64), a.n, i, r);
    Spinor<SF>::load(a.v1, a.n, i, p);
    const double cr = a.st->coef_re, ci = a.st->coef_im, beta = a.st->beta;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[2 * c] = (real)(cr * r[2 * c] - ci * r[2 * c + 1] + beta * (double)p[2 * c]);
        o[2 * c + 1] = (real)(cr * r[2 * c + 1] + ci * r[2 * c] + beta * (double)p[2 * c + 1]);
    }
    if (!Spinor<SF>::store(a.v2, a.n, i, o)) atomicExch(a.err, 1);
}

__global__ void __launch_bounds__(kBlock) norm2_kernel(BlasArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (i < a.n) {
        double x[6];
        Spinor<S_F64>::load(reinterpret_cast<const char *>(a.x64), a.n, i, x);
#pragma unroll
        for (int k = 0; k < 6; k++) v[0] += x[k] * x[k];
    }
    __shared__ double tot[1];
    reduce_grid<1>(v, a.red, tot);
}

int nblk(int n) { return (n + kBlock - 1) / kBlock; }

}  // namespace

#define HISQ_SF_DISPATCH(SF_, CF_, KERNEL, ...)                                              \
    do {                                                                                    \
        const bool f64_ = (CF_) == HISQ_COMPUTE_F64;                                        \
        switch (SF_) {                                                                      \
        case S_F64: launch_chained(KERNEL<S_F64, double>, __VA_ARGS__, a); break;           \
        case S_F32: launch_chained(KERNEL<S_F32, float>, __VA_ARGS__, a); break;            \
        case S_HALF: launch_chained(KERNEL<S_HALF, float>, __VA_ARGS__, a); break;          \
        case S_INT20: launch_chained(KERNEL<S_INT20, float>, __VA_ARGS__, a); break;        \
        case S_INT14: launch_chained(KERNEL<S_INT14, float>, __VA_ARGS__, a); break;        \
        case S_INT30:                                                                       \
            if (f64_) launch_chained(KERNEL<S_INT30, double>, __VA_ARGS__, a);              \
            else launch_chained(KERNEL<S_INT30, float>, __VA_ARGS__, a);                    \
            break;                                                                          \
        }                                                                                   \
    } while (0)

namespace {

// Block size of the split r_update: 1024 threads (each block sums the
// stencil pass's partials in one round of loads) where the kernel fits 64
// registers, 512 for the FP64 and FP32-pair kernels.  One wave of blocks, so
// p_update sums few partials.
template <typename real>
constexpr int split_block()
{
    return std::is_same<real, float>::value ? 1024 : 512;
}

template <int SF, typename real>
unsigned r_update_t(const BlasArgs &a, cudaStream_t s)
{
    if (a.split) {
        constexpr int BS = split_block<real>();
        static const int wave = wave_blocks(r_update_split_kernel<SF, real, BS>, BS);
        const int need = (a.n + BS * kRSites - 1) / (BS * kRSites);
        const int nb = need < wave ? need : wave;
        launch_chained(r_update_split_kernel<SF, real, BS>, dim3(nb), dim3(BS), s, a);
        return (unsigned)nb;
    }
    static const int wave = wave_blocks(r_update_kernel<SF, real>, kBlock);
    const int need = (a.n + kBlock * kRSites - 1) / (kBlock * kRSites);
    launch_chained(r_update_kernel<SF, real>, dim3(need < wave ? need : wave), dim3(kBlock), s, a);
    return 0;
}

template <int SF, typename real>
void p_update_t(const BlasArgs &a, cudaStream_t s)
{
    const int nb = (a.n + kBlock * kPSites - 1) / (kBlock * kPSites);
    if (a.split) {
        launch_chained(p_update_split_kernel<SF, real>, dim3(nb), dim3(kBlock), s, a);
        return;
    }
    launch_chained(p_update_kernel<SF, real>, dim3(nb), dim3(kBlock), s, a);
}

}  // namespace

unsigned launch_r_update(int sf, int cf, const BlasArgs &a, cudaStream_t s)
{
    switch (sf) {
    case S_F64: return r_update_t<S_F64, double>(a, s);
    case S_F32: return r_update_t<S_F32, float>(a, s);
    case S_HALF: return r_update_t<S_HALF, float>(a, s);
    case S_INT20: return r_update_t<S_INT20, float>(a, s);
    case S_INT14: return r_update_t<S_INT14, float>(a, s);
    case S_INT30:  // FP64-class compute in FP32 pairs (see ff.cuh)
        if (cf == HISQ_COMPUTE_F64) return r_update_t<S_INT30, ff>(a, s);
        return r_update_t<S_INT30, float>(a, s);
    }
    return 0;
}

void launch_p_update(int sf, int cf, const BlasArgs &a, cudaStream_t s)
{
    switch (sf) {
    case S_F64: p_update_t<S_F64, double>(a, s); break;
    case S_F32: p_update_t<S_F32, float>(a, s); break;
    case S_HALF: p_update_t<S_HALF, float>(a, s); break;
    case S_INT20: p_update_t<S_INT20, float>(a, s); break;
    case S_INT14: p_update_t<S_INT14, float>(a, s); break;
    case S_INT30:  // FP64-class compute in FP32 pairs (see ff.cuh)
        if (cf == HISQ_COMPUTE_F64)
            p_update_t<S_INT30, ff>(a, s);
        else
            p_update_t<S_INT30, float>(a, s);
        break;
    }
}

void launch_x_flush(int sf, int cf, const BlasArgs &a, cudaStream_t s)
{
    if (sf == S_INT30 && cf == HISQ_COMPUTE_F64) {  // the increment in FP32 pairs, not on the FP64 pipe
        launch_chained(x_flush_kernel<S_INT30, ff>, dim3(nblk(a.n)), dim3(kBlock), s, a);
        return;
    }
    HISQ_SF_DISPATCH(sf, cf, x_flush_kernel, dim3(nblk(a.n)), dim3(kBlock), s);
}

void launch_true_residual(int sf, int cf, const BlasArgs &a, cudaStream_t s)
{
    HISQ_SF_DISPATCH(sf, cf, true_residual_kernel, dim3(nblk(a.n)), dim3(kBlock), s);
}

void launch_p_reliable(int sf, int cf, const BlasArgs &a, cudaStream_t s)
{
    HISQ_SF_DISPATCH(sf, cf, p_reliable_kernel, dim3(nblk(a.n)), dim3(kBlock), s);
}

void launch_norm2(const BlasArgs &a, cudaStream_t s)
{
    launch_chained(norm2_kernel, dim3(nblk(a.n)), dim3(kBlock), s, a);
}

}  // namespace hisq
