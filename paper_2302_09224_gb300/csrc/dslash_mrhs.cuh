// dslash_mrhs.cuh -- the stencil applied to a tile of T right-hand sides at
// once (Sec. 1, block solvers: the link traffic is shared by the tile, which
// turns the matrix-vector stencil into a matrix-matrix one and raises its
// arithmetic intensity T-fold).
//
// One thread per output site and tile: each of the 16 links is loaded once
// (scaled to its true value, since that cost is now shared by T products) and
// applied to the T neighbour spinors.  Right-hand side t of the tile lives in
// the field at in + (t0 + t) * field_bytes.  Per right-hand side: its own xpay
// coefficient and, when reducing, Re<y_t, out_t> and |out_t|^2, whose totals
// drive the batched solver's per-RHS scalar recurrences.
#pragma once

#include <cuda_runtime.h>

#include "codecs.cuh"
#include "dslash.cuh"
#include "finish.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace hisq {

template <int GF, int RECON, typename real>
__device__ __forceinline__ void load_link_scaled(const char *base, size_t pstride, int li, real U[18], real scale,
                                                 real sign12)
{
    Link<GF, RECON>::load(base, pstride, li, U);
    if constexpr (LinkScaled<GF>::value) {
#pragma unroll
        for (int k = 0; k < RECON; k++) U[k] *= scale;
    }
    if constexpr (RECON == 12) rebuild_row2(U, sign12);
}

// Whether any right-hand side of the tile [t0, t0 + T) is still iterating
// (solver states present); a tile of stopped or empty slots is skipped.
template <int T>
__device__ __forceinline__ bool tile_active(const DslashMArgs &a)
{
    if (a.st == nullptr) return true;
    bool any = false;
#pragma unroll
    for (int j = 0; j < T; j++) any = any || *(volatile const int *)&a.st[a.t0 + j].active != 0;
    return any;
}

// U <- -U^+ (a backward term's matrix, so that every term is accumulated as
// acc += U s).
template <typename real>
__device__ __forceinline__ void neg_adjoint(real U[18])
{
    real V[18];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            V[2 * (3 * i + j)] = -U[2 * (3 * j + i)];
            V[2 * (3 * i + j) + 1] = U[2 * (3 * j + i) + 1];
        }
#pragma unroll
    for (int k = 0; k < 18; k++) U[k] = V[k];
}

// For tiles of 8 and 16 the loops over directions and over forward/backward
// hops stay rolled (only the loop over the tile's right-hand sides is
// unrolled): the kernel body then fits the instruction cache, which a fully
// unrolled body of 16 x T matrix-vector products did not.
template <int GF, int SF, typename real, int LREC, int T, bool RED>
__global__ void __launch_bounds__(kMrhsBlock) dslash_mrhs_kernel(const DslashMArgs a)
{
    if (a.active_any != nullptr && *(volatile const int *)a.active_any == 0) return;
    if (!tile_active<T>(a)) return;  // every system of this tile stopped or empty: uniform over the grid
    const Geom &g = a.g;
    const int vh = g.vh;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int po = a.out_parity, pi = 1 - po;
    const size_t pstride = (size_t)8 * vh * 16;
    constexpr bool kScaled = LinkScaled<GF>::value;
    const real fsc = kScaled ? (sizeof(real) == 8 ? (real)a.gv.fat_scale_d : (real)a.gv.fat_scale_f) : real(1);
    const real lsc = kScaled ? (sizeof(real) == 8 ? (real)a.gv.lng_scale_d : (real)a.gv.lng_scale_f) : real(1);
    real rv[2 * T];
#pragma unroll
    for (int k = 0; k < 2 * T; k++) rv[k] = 0;

    if (cb < vh) {
        int r = cb / g.xh;
        const int xh = cb - r * g.xh;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((y + z + t + po) & 1);
        const int lex = 2 * cb + (x & 1);
        // packed FP32 accumulators hold twice the registers: used up to 4 per thread
        using Acc = std::conditional_t<(T <= 4), SiteAcc<real>, SiteAccScalar<real>>;
        Acc acc[T];
#pragma unroll
        for (int j = 0; j < T; j++) acc[j].zero();
        // one term: link of hop k (1 fat, 3 long) in direction dir, applied to
        // the neighbour of every right-hand side of the tile
        auto term = [&](int mu, int cmu, int hop, int dir, int base, real eta) {
            const int L = g.L[mu], st = g.stride[mu];
            const int k = hop ? 3 : 1;
            const int cn = wrap_coord(dir ? cmu - k : cmu + k, L);
            const int nb = (base + cn * st) >> 1;
            const int li = ((dir ? pi : po) * 4 + mu) * vh + (dir ? nb : cb);
            real U[18];
            if (hop == 0) {
                load_link_scaled<GF, 18>(a.gv.fat, pstride, li, U, fsc, real(1));
            } else {
                // the boundary sign belongs to the link's own site: x for the
                // forward link, x - 3 mu for the backward one
                const bool flip = g.antiperiodic_t && mu == 3 && (dir ? cn : cmu) + 3 >= L;
                load_link_scaled<GF, LREC>(a.gv.lng, pstride, li, U, lsc, flip ? -eta : eta);
            }
            if (dir) neg_adjoint(U);
#pragma unroll
            for (int j = 0; j < T; j++) {
                real s[6];
                Spinor<SF>::load(a.in + (size_t)(a.t0 + j) * a.field_bytes, vh, nb, s);
                acc[j].add(U, s);
            }
        };
        const int c[4] = {x, y, z, t};
        int phase_sum = 0;
        if constexpr (T <= 4) {
            // small tiles: fully unrolled (index arithmetic folded at compile time)
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                const int base = lex - c[mu] * g.stride[mu];
                const real eta = (phase_sum & 1) ? real(-1) : real(1);
#pragma unroll
                for (int q = 0; q < 4; q++) term(mu, c[mu], q >> 1, q & 1, base, eta);
                phase_sum += c[mu];
            }
        } else {
            // large tiles: directions and hops rolled so that the body fits the
            // instruction cache
#pragma unroll 1
            for (int mu = 0; mu < 4; mu++) {
                const int cmu = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t;
                const int base = lex - cmu * g.stride[mu];
                const real eta = (phase_sum & 1) ? real(-1) : real(1);
#pragma unroll
                for (int hop = 0; hop < 2; hop++)
#pragma unroll 1
                    for (int dir = 0; dir < 2; dir++) term(mu, cmu, hop, dir, base, eta);
                phase_sum += cmu;
            }
        }

        const real sgn = (real)a.sign;
#pragma unroll
        for (int j = 0; j < T; j++) {
            real o[6];
#pragma unroll
            for (int k = 0; k < 6; k++) o[k] = sgn * acc[j].get(k);
            const size_t off = (size_t)(a.t0 + j) * a.field_bytes;
            if (a.xpay) {
                real yv[6];
                Spinor<SF>::load(a.y + off, vh, cb, yv);
                // a solver's per-system coefficient lives in its state (slots change hands)
                const real aa = a.st ? (real)a.st[a.t0 + j].diag : (real)a.a[a.t0 + j];
#pragma unroll
                for (int k = 0; k < 6; k++) o[k] = aa * yv[k] + o[k];
                if constexpr (RED) {
                    real d = 0;
#pragma unroll
                    for (int k = 0; k < 6; k++) d += yv[k] * o[k];
                    rv[2 * j] = d;
                }
            }
            if constexpr (RED) {
                real n2 = 0;
#pragma unroll
                for (int k = 0; k < 6; k++) n2 += o[k] * o[k];
                rv[2 * j + 1] = n2;
            }
            if (!Spinor<SF>::store(a.out + off, vh, cb, o)) atomicExch(a.err, 1);
        }
    }

    if constexpr (RED) {
        __shared__ double tot[2 * T];
        if (reduce_grid<2 * T>(rv, a.red, tot) && threadIdx.x == 0)
            run_batch_finisher(a.fin, tot, a.st, a.t0, T, a.slot);
    }
}

// ---------------------------------------------------------------------------
// Staged variant (16-byte spinor records: 16-bit and 20-bit formats).  For
// tiles of many right-hand sides the kernel above waits on one neighbour load
// at a time.  Here each thread copies the next term's link and its T
// neighbour records into its own slots of shared memory with cp.async (no
// registers held while in flight) and computes the current term meanwhile:
// double buffered, one copy group per term.  Each thread reads only the slots
// it wrote, so the copies need no block barrier, only the thread's own wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared slots per block: [stage][slot][thread] of 16 bytes, where the slots
// of a stage are the link's chunks (kLinkSlots) then one per right-hand side.
constexpr int kLinkSlots = 3;  // a fix16 r18 link: two 16-byte chunks and a 4-byte tail
__host__ __device__ constexpr int mrhs_staged_slots(int T) { return kLinkSlots + T; }
__host__ __device__ constexpr size_t mrhs_staged_smem(int T)
{
    return (size_t)2 * mrhs_staged_slots(T) * kMrhsBlock * 16;
}

template <int GF, int RECON>
__device__ __forceinline__ void stage_link(uint4 *slot0, int stride, const char *base, size_t pstride, int li)
{
    using LK = Link<GF, RECON>;
    static_assert(LK::chunks <= kLinkSlots, "link chunks exceed the staged slots");
#pragma unroll
    for (int k = 0; k < LK::n16; k++) cp_async_16(slot0 + k * stride, base + k * pstride + (size_t)li * 16);
    if constexpr (LK::tail == 4)
        cp_async_4(slot0 + LK::n16 * stride, base + LK::n16 * pstride + (size_t)li * 4);
    else if constexpr (LK::tail == 8)
        cp_async_8(slot0 + LK::n16 * stride, base + LK::n16 * pstride + (size_t)li * 8);
}

// Term q = 4 mu + 2 hop + dir of a site: neighbour (checkerboard) index and
// link index.
struct TermIdx {
    int nb, li, mu, hop, dir, cn;
};

__device__ __forceinline__ TermIdx term_index(const Geom &g, int q, const int c[4], int lex, int cb, int po)
{
    TermIdx r;
    r.mu = q >> 2;
    r.hop = (q >> 1) & 1;
    r.dir = q & 1;
    const int k = r.hop ? 3 : 1;
    const int L = g.L[r.mu], st = g.stride[r.mu];
    const int cmu = c[r.mu];
    r.cn = wrap_coord(r.dir ? cmu - k : cmu + k, L);
    r.nb = ((lex - cmu * st) + r.cn * st) >> 1;
    r.li = ((r.dir ? 1 - po : po) * 4 + r.mu) * g.vh + (r.dir ? r.nb : cb);
    return r;
}

template <int GF, int SF, typename real, int LREC, int T, bool RED>
__global__ void __launch_bounds__(kMrhsBlock) dslash_mrhs_staged_kernel(const DslashMArgs a)
{
    static_assert(Spinor<SF>::chunks == 1, "staged tiles take 16-byte spinor records");
    extern __shared__ __align__(16) uint4 stage_smem[];
    if (a.active_any != nullptr && *(volatile const int *)a.active_any == 0) return;
    if (!tile_active<T>(a)) return;  // every system of this tile stopped or empty: uniform over the grid
    const Geom &g = a.g;
    const int vh = g.vh;
    const int tid = threadIdx.x;
    const int cb = blockIdx.x * blockDim.x + tid;
    const int po = a.out_parity;
    const size_t pstride = (size_t)8 * vh * 16;
    constexpr bool kScaled = LinkScaled<GF>::value;
    const real fsc = kScaled ? (real)a.gv.fat_scale_f : real(1);
    const real lsc = kScaled ? (real)a.gv.lng_scale_f : real(1);
    constexpr int S = mrhs_staged_slots(T);
    auto slot = [&](int stage, int k) { return stage_smem + ((size_t)(stage * S + k) * kMrhsBlock + tid); };
    real rv[2 * T];
#pragma unroll
    for (int k = 0; k < 2 * T; k++) rv[k] = 0;

    if (cb < vh) {
        int r = cb / g.xh;
        const int xh = cb - r * g.xh;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((y + z + t + po) & 1);
        const int c[4] = {x, y, z, t};
        const int lex = 2 * cb + (x & 1);
        const int eta_bits = (0) | ((x & 1) << 1) | (((x + y) & 1) << 2) | (((x + y + z) & 1) << 3);  // eta_mu = -1 if bit mu

        // copies of term q into stage q & 1 (one group per term)
        auto issue = [&](const TermIdx &ti, int stage) {
            if (ti.hop == 0)
                stage_link<GF, 18>(slot(stage, 0), kMrhsBlock, a.gv.fat, pstride, ti.li);
            else
                stage_link<GF, LREC>(slot(stage, 0), kMrhsBlock, a.gv.lng, pstride, ti.li);
#pragma unroll
            for (int j = 0; j < T; j++)
                cp_async_16(slot(stage, kLinkSlots + j), a.in + (size_t)(a.t0 + j) * a.field_bytes + (size_t)ti.nb * 16);
        };

        using Acc = std::conditional_t<(T <= 4), SiteAcc<real>, SiteAccScalar<real>>;
        Acc acc[T];
#pragma unroll
        for (int j = 0; j < T; j++) acc[j].zero();

        TermIdx cur = term_index(g, 0, c, lex, cb, po);
        issue(cur, 0);
        cp_async_commit();
#pragma unroll 1
        for (int q = 0; q < 16; q++) {
            TermIdx nxt;
            if (q + 1 < 16) {
                nxt = term_index(g, q + 1, c, lex, cb, po);
                issue(nxt, (q + 1) & 1);
            }
            cp_async_commit();  // possibly empty: keeps one group per iteration
            cp_async_wait_1();  // term q's copies have landed (this thread's)
            const int stage = q & 1;
            real U[18];
            if (cur.hop == 0) {
                uint4 lc[Link<GF, 18>::chunks];
#pragma unroll
                for (int k = 0; k < Link<GF, 18>::chunks; k++) lc[k] = *slot(stage, k);
                Link<GF, 18>::decode(lc, U);
                if constexpr (kScaled)
#pragma unroll
                    for (int k = 0; k < 18; k++) U[k] *= fsc;
            } else {
                uint4 lc[Link<GF, LREC>::chunks];
#pragma unroll
                for (int k = 0; k < Link<GF, LREC>::chunks; k++) lc[k] = *slot(stage, k);
                Link<GF, LREC>::decode(lc, U);
                if constexpr (kScaled)
#pragma unroll
                    for (int k = 0; k < LREC; k++) U[k] *= lsc;
                if constexpr (LREC == 12) {
                    // the boundary sign belongs to the link's own site
                    const real eta = ((eta_bits >> cur.mu) & 1) ? real(-1) : real(1);
                    const bool flip = g.antiperiodic_t && cur.mu == 3 && (cur.dir ? cur.cn : c[3]) + 3 >= g.L[3];
                    rebuild_row2(U, flip ? -eta : eta);
                }
            }
            if (cur.dir) neg_adjoint(U);
#pragma unroll
            for (int j = 0; j < T; j++) {
                const uint4 sc[1] = {*slot(stage, kLinkSlots + j)};
                real sv[6];
                Spinor<SF>::decode(sc, sv);
                acc[j].add(U, sv);
            }
            if (q + 1 < 16) cur = nxt;
        }

        const real sgn = (real)a.sign;
#pragma unroll
        for (int j = 0; j < T; j++) {
            real o[6];
#pragma unroll
            for (int k = 0; k < 6; k++) o[k] = sgn * acc[j].get(k);
            const size_t off = (size_t)(a.t0 + j) * a.field_bytes;
            if (a.xpay) {
                real yv[6];
                Spinor<SF>::load(a.y + off, vh, cb, yv);
                const real aa = a.st ? (real)a.st[a.t0 + j].diag : (real)a.a[a.t0 + j];
#pragma unroll
                for (int k = 0; k < 6; k++) o[k] = aa * yv[k] + o[k];
                if constexpr (RED) {
                    real d = 0;
#pragma unroll
                    for (int k = 0; k < 6; k++) d += yv[k] * o[k];
                    rv[2 * j] = d;
                }
            }
            if constexpr (RED) {
                real n2 = 0;
#pragma unroll
                for (int k = 0; k < 6; k++) n2 += o[k] * o[k];
                rv[2 * j + 1] = n2;
            }
            if (!Spinor<SF>::store(a.out + off, vh, cb, o)) atomicExch(a.err, 1);
        }
    }

    if constexpr (RED) {
        __shared__ double tot[2 * T];
        if (reduce_grid<2 * T>(rv, a.red, tot) && threadIdx.x == 0)
            run_batch_finisher(a.fin, tot, a.st, a.t0, T, a.slot);
    }
}

template <int GF, int SF, typename real, int LREC, int T, bool RED>
bool launch_staged_tile(const DslashMArgs &a, cudaStream_t s)
{
    auto kern = dslash_mrhs_staged_kernel<GF, SF, real, LREC, T, RED>;
    constexpr size_t smem = mrhs_staged_smem(T);
    static const bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                           cudaSuccess;  // once per kernel
    if (!ok) return false;
    const int nb = (a.g.vh + kMrhsBlock - 1) / kMrhsBlock;
    kern<<<nb, kMrhsBlock, smem, s>>>(a);
    return true;
}

template <int GF, int SF, typename real, int LREC, bool RED>
void launch_mrhs_tile(int T, const DslashMArgs &a, cudaStream_t s)
{
    const int nb = (a.g.vh + kMrhsBlock - 1) / kMrhsBlock;
    switch (T) {
    case 16: dslash_mrhs_kernel<GF, SF, real, LREC, 16, RED><<<nb, kMrhsBlock, 0, s>>>(a); break;
    case 8: dslash_mrhs_kernel<GF, SF, real, LREC, 8, RED><<<nb, kMrhsBlock, 0, s>>>(a); break;
    case 4: dslash_mrhs_kernel<GF, SF, real, LREC, 4, RED><<<nb, kMrhsBlock, 0, s>>>(a); break;
    case 2: dslash_mrhs_kernel<GF, SF, real, LREC, 2, RED><<<nb, kMrhsBlock, 0, s>>>(a); break;
    default: dslash_mrhs_kernel<GF, SF, real, LREC, 1, RED><<<nb, kMrhsBlock, 0, s>>>(a); break;
    }
}

template <int GF, int SF, typename real, int LREC, bool RED>
bool launch_staged(int T, const DslashMArgs &a, cudaStream_t s)
{
    if constexpr (Spinor<SF>::chunks == 1 && std::is_same<real, float>::value) {
        switch (T) {
        case 16: return launch_staged_tile<GF, SF, real, LREC, 16, RED>(a, s);
        case 8: return launch_staged_tile<GF, SF, real, LREC, 8, RED>(a, s);
        case 4: return launch_staged_tile<GF, SF, real, LREC, 4, RED>(a, s);
        case 2: return launch_staged_tile<GF, SF, real, LREC, 2, RED>(a, s);
        default: return launch_staged_tile<GF, SF, real, LREC, 1, RED>(a, s);
        }
    }
    return false;
}

// All nrhs right-hand sides in tiles of T (T divides nrhs; one launch per
// tile); variant 0 the register kernel, 1 the staged one (16-byte records).
template <int GF, int SF, typename real>
bool launch_mrhs_t(int long_recon, bool reduce, int T, int variant, const DslashMArgs &args, cudaStream_t s)
{
    if (reduce && !red_fits(args.g.vh, kMrhsBlock, 2 * T)) return false;
    for (int t0 = 0; t0 < args.nrhs; t0 += T) {
        DslashMArgs a = args;
        a.t0 = t0;
        bool ok = true;
        if (variant == 1) {
            if (long_recon == 12)
                ok = reduce ? launch_staged<GF, SF, real, 12, true>(T, a, s) : launch_staged<GF, SF, real, 12, false>(T, a, s);
            else
                ok = reduce ? launch_staged<GF, SF, real, 18, true>(T, a, s) : launch_staged<GF, SF, real, 18, false>(T, a, s);
        } else if (long_recon == 12) {
            if (reduce)
                launch_mrhs_tile<GF, SF, real, 12, true>(T, a, s);
            else
                launch_mrhs_tile<GF, SF, real, 12, false>(T, a, s);
        } else {
            if (reduce)
                launch_mrhs_tile<GF, SF, real, 18, true>(T, a, s);
            else
                launch_mrhs_tile<GF, SF, real, 18, false>(T, a, s);
        }
        if (!ok) return false;
    }
    return true;
}

}  // namespace hisq
