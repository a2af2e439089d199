// dslash_mrhs.cuh -- the stencil applied to a tile of T right-hand sides at
// once (Sec. 1, block solvers: the link traffic is shared by the tile, which
// turns the matrix-vector stencil into a matrix-matrix one and raises its
// arithmetic intensity T-fold).
//
// One thread per output site and tile: each of the 16 links is loaded and
// decoded once and applied to the T neighbour spinors.  Right-hand side t of
// the tile lives in the field at in + (t0 + t) * field_bytes.  Per
// right-hand side: its own xpay coefficient and, when reducing, Re<y_t, out_t>
// and |out_t|^2, whose totals drive the batched solver's per-RHS scalar
// recurrences.
//
// Arithmetic.  The right-hand sides are processed in pairs on the packed
// FP32 pipe (float2 lanes, one __ffma2_rn per two products): each link
// element is broadcast to both lanes once per term and shared by every pair,
// and each spinor record is decoded straight into the operand pairs of the
// product (below).  Every lane runs exactly the operations a lone right-hand
// side would (a tile of one runs the same sequence in plain FP32), so a
// system's iterates do not depend on its tile or on its companions.
// Fixed-point links are applied unscaled: a long link's elements are
// multiplied by lsc/fsc (once per link, shared by the tile) and the sum is
// scaled by fsc once per output.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "codecs.cuh"
#include "dslash.cuh"
#include "finish.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace hisq {

// ---------------------------------------------------------------------------
// lanes: one right-hand side (float) or two (float2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <int NL>
using lanes_t = std::conditional_t<NL == 2, float2, float>;

template <typename V>
__device__ __forceinline__ V lanes(float x0, float x1);
template <>
__device__ __forceinline__ float lanes<float>(float x0, float) { return x0; }
template <>
__device__ __forceinline__ float2 lanes<float2>(float x0, float x1) { return make_float2(x0, x1); }

__device__ __forceinline__ float lane_of(float v, int) { return v; }
__device__ __forceinline__ float lane_of(float2 v, int l) { return l ? v.y : v.x; }

template <typename V>
constexpr int nlanes() { return sizeof(V) / sizeof(float); }

// ---------------------------------------------------------------------------
// Operands of one term for a group of right-hand sides, from their raw
// records (rec[l * chunks + k]: lane l, chunk k).  Per colour j, with v = s
// for a forward term (acc += U s) and v = -s for a backward one
// (acc += -U^+ s):
//   forward:  a = Re v, b = Im v, c = -Im v
//   backward: a = Re v, b = Im v, c = -Re v
// Every operand is the format's decoded value (exactly as Spinor<SF>::decode
// gives it) or its negation.
// ---------------------------------------------------------------------------
template <int SF>
struct TermOps;

template <>
struct TermOps<S_INT20> {
    // (m - M) up with m the magic float of the 20-bit field and M = 2^23 + 2^19
    // (the codec's decode), as one fma against the exact product M up; exact
    // for shared exponents E <= 231 (|values| below 2^123, far beyond any
    // field the FP32 stencil can apply without overflow).
    template <bool BWD, typename V>
    __device__ static void get(const uint4 *rec, V a[3], V b[3], V c[3])
    {
        constexpr int NL = nlanes<V>();
        float m[2][6], p[2], q[2];
#pragma unroll
        for (int l = 0; l < NL; l++) {
            const uint4 w = rec[l];
            const uint32_t u[6] = {w.x,
                                   ((w.x >> 20) << 8) | (w.y & 0xffu),
                                   w.y >> 8,
                                   ((w.y >> 28) << 16) | (w.z & 0xffffu),
                                   ((w.z >> 16) << 4) | (w.w & 0xfu),
                                   w.w >> 4};
#pragma unroll
            for (int k = 0; k < 6; k++) m[l][k] = __uint_as_float((u[k] & 0xfffffu) ^ 0x4B080000u);
            const float up = __uint_as_float(((w.w >> 24) << 23) | (BWD ? 0x80000000u : 0u));  // +-2^(E-127)
            p[l] = up;
            q[l] = fmul(-8912896.0f, up);
        }
        const V pv = lanes<V>(p[0], p[NL - 1]), qv = lanes<V>(q[0], q[NL - 1]);
        const V npv = lanes<V>(-p[0], -p[NL - 1]), nqv = lanes<V>(-q[0], -q[NL - 1]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const V mr = lanes<V>(m[0][2 * j], m[NL - 1][2 * j]);
            const V mi = lanes<V>(m[0][2 * j + 1], m[NL - 1][2 * j + 1]);
            a[j] = vfma(mr, pv, qv);
            b[j] = vfma(mi, pv, qv);
            c[j] = BWD ? vfma(mr, npv, nqv) : vfma(mi, npv, nqv);
        }
    }
};

template <>
struct TermOps<S_HALF> {
    template <bool BWD, typename V>
    __device__ static void get(const uint4 *rec, V a[3], V b[3], V c[3])
    {
        constexpr int NL = nlanes<V>();
        float qf[2][6], sc[2];
#pragma unroll
        for (int l = 0; l < NL; l++) {
            const uint4 r = rec[l];
            const float s = fmul(__uint_as_float(r.w), 1.0f / 32767.0f);
            sc[l] = BWD ? -s : s;
            qf[l][0] = i16lo_to_f(r.x); qf[l][1] = i16hi_to_f(r.x);
            qf[l][2] = i16lo_to_f(r.y); qf[l][3] = i16hi_to_f(r.y);
            qf[l][4] = i16lo_to_f(r.z); qf[l][5] = i16hi_to_f(r.z);
        }
        const V sv = lanes<V>(sc[0], sc[NL - 1]), nsv = lanes<V>(-sc[0], -sc[NL - 1]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const V qr = lanes<V>(qf[0][2 * j], qf[NL - 1][2 * j]);
            const V qi = lanes<V>(qf[0][2 * j + 1], qf[NL - 1][2 * j + 1]);
            a[j] = vmul(qr, sv);
            b[j] = vmul(qi, sv);
            c[j] = BWD ? vmul(qr, nsv) : vmul(qi, nsv);
        }
    }
};

template <>
struct TermOps<S_F32> {
    template <bool BWD, typename V>
    __device__ static void get(const uint4 *rec, V a[3], V b[3], V c[3])
    {
        constexpr int NL = nlanes<V>();
        float f[2][6];
#pragma unroll
        for (int l = 0; l < NL; l++) {
            float v[6];
            Spinor<S_F32>::decode(rec + 2 * l, v);
#pragma unroll
            for (int k = 0; k < 6; k++) f[l][k] = BWD ? -v[k] : v[k];
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            a[j] = lanes<V>(f[0][2 * j], f[NL - 1][2 * j]);
            b[j] = lanes<V>(f[0][2 * j + 1], f[NL - 1][2 * j + 1]);
            c[j] = BWD ? lanes<V>(-f[0][2 * j], -f[NL - 1][2 * j]) : lanes<V>(-f[0][2 * j + 1], -f[NL - 1][2 * j + 1]);
        }
    }
};

// acc += U v (forward, v = s) or acc += U^+ v (backward, v = -s) for one group, with the
// link's elements broadcast (ur[e], ui[e]: Re and Im of element e = 3 row +
// column):
//   forward:  Re acc_i += Re U_ij a_j + Im U_ij c_j,  Im acc_i += Re U_ij b_j + Im U_ij a_j
//   backward: Re acc_i += Re U_ji a_j + Im U_ji b_j,  Im acc_i += Re U_ji b_j + Im U_ji c_j
template <bool BWD, typename V>
__device__ __forceinline__ void term_mv(V re[3], V im[3], const V ur[9], const V ui[9], const V a[3], const V b[3],
                                        const V c[3])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int e = BWD ? 3 * j + i : 3 * i + j;
            re[i] = vfma(ur[e], a[j], re[i]);
            re[i] = vfma(ui[e], BWD ? b[j] : c[j], re[i]);
            im[i] = vfma(ur[e], b[j], im[i]);
            im[i] = vfma(ui[e], BWD ? c[j] : a[j], im[i]);
        }
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

// ---------------------------------------------------------------------------
// Staged loads (16-byte spinor records: 16-bit and 20-bit formats).  Each
// thread copies the next term's link and its T neighbour records into its own
// slots of shared memory with cp.async (no registers held while in flight)
// and computes the current term meanwhile: double buffered, one copy group
// per term.  Each thread reads only the slots it wrote, so the copies need no
// block barrier, only the thread's own wait.
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
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// Term k = 2 hop + dir of direction mu at a site: neighbour (checkerboard)
// index, link index and the neighbour's mu coordinate.
struct TermIdx {
    int nb, li, cn;
};

__device__ __forceinline__ TermIdx term_index(const Geom &g, int mu, int hop, int dir, int cmu, int base, int cb, int po)
{
    TermIdx r;
    const int k = hop ? 3 : 1;
    const int st = g.stride[mu];
    r.cn = wrap_coord(dir ? cmu - k : cmu + k, g.L[mu]);
    r.nb = (base + r.cn * st) >> 1;
    r.li = ((dir ? 1 - po : po) * 4 + mu) * g.vh + (dir ? r.nb : cb);
    return r;
}

// Resident blocks per SM asked of the register allocator: five for tiles of up
// to four (at most 96 registers: twenty warps keep the loads of neighbour
// records in flight), no cap for larger tiles (their accumulators need more).
__host__ __device__ constexpr int mrhs_min_blocks(int T) { return T <= 4 ? 5 : 1; }

// ---------------------------------------------------------------------------
// The kernel.  STAGED: neighbour records and links through shared memory
// (16-byte spinor records); otherwise loaded into registers term by term.
// Directions are a rolled loop; the four terms of a direction (forward and
// backward, one hop and three) are unrolled, so every term's link format and
// product are fixed at compile time.
// ---------------------------------------------------------------------------
template <int GF, int SF, int LREC, int T, bool RED, bool STAGED>
__global__ void __launch_bounds__(kMrhsBlock, mrhs_min_blocks(T)) dslash_mrhs_kernel(const __grid_constant__ DslashMArgs a)
{
    constexpr int NL = T >= 2 ? 2 : 1, NG = T / NL;  // lanes per group, groups
    using V = lanes_t<NL>;
    constexpr int SC = Spinor<SF>::chunks;
    static_assert(!STAGED || SC == 1, "staged tiles take 16-byte spinor records");
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
    const float fsc = kScaled ? a.gv.fat_scale_f : 1.0f;
    const float lsc = kScaled ? a.gv.lng_scale_f : 1.0f;
    const float ratio = lsc / fsc;
    constexpr int S = mrhs_staged_slots(T);
    auto slot = [&](int stage, int k) { return stage_smem + ((size_t)(stage * S + k) * kMrhsBlock + tid); };
    float rv[2 * T];
#pragma unroll
    for (int k = 0; k < 2 * T; k++) rv[k] = 0.0f;

    if (cb < vh) {
        int r = cb / g.xh;
        const int xh = cb - r * g.xh;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((y + z + t + po) & 1);
        const int lex = 2 * cb + (x & 1);
        const int eta_bits = ((x & 1) << 1) | (((x + y) & 1) << 2) | (((x + y + z) & 1) << 3);  // eta_mu = -1 if bit mu

        V re[NG][3], im[NG][3];
#pragma unroll
        for (int gi = 0; gi < NG; gi++)
#pragma unroll
            for (int i = 0; i < 3; i++) re[gi][i] = im[gi][i] = lanes<V>(0.0f, 0.0f);

        // copies of one term into a stage (one group per term)
        auto issue = [&](const TermIdx &ti, int hop, int stage) {
            if constexpr (STAGED) {
                if (hop == 0)
                    stage_link<GF, 18>(slot(stage, 0), kMrhsBlock, a.gv.fat, pstride, ti.li);
                else
                    stage_link<GF, LREC>(slot(stage, 0), kMrhsBlock, a.gv.lng, pstride, ti.li);
#pragma unroll
                for (int j = 0; j < T; j++)
                    cp_async_16(slot(stage, kLinkSlots + j),
                                a.in + (size_t)(a.t0 + j) * a.field_bytes + (size_t)ti.nb * 16);
            }
        };
        // staged: each term's indices are computed once, when its copies are
        // issued (one term ahead), and carried to the term itself
        TermIdx cur = term_index(g, 0, 0, 0, x, lex - x, cb, po);
        if constexpr (STAGED) {
            issue(cur, 0, 0);
            cp_async_commit();
        }

#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
            const int cmu = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t;
            const int base = lex - cmu * g.stride[mu];  // the site with coordinate mu set to 0
            const float eta = ((eta_bits >> mu) & 1) ? -1.0f : 1.0f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int hop = k >> 1, dir = k & 1;
                constexpr int LC = Link<GF, 18>::chunks > Link<GF, LREC>::chunks ? Link<GF, 18>::chunks
                                                                                  : Link<GF, LREC>::chunks;
                uint4 lc[LC];
                uint4 sc[T * SC];
                TermIdx nxt = cur;
                if constexpr (STAGED) {
                    const int q = 4 * mu + k;
                    if (k < 3) {
                        nxt = term_index(g, mu, (k + 1) >> 1, (k + 1) & 1, cmu, base, cb, po);
                        issue(nxt, (k + 1) >> 1, (q + 1) & 1);
                    } else if (mu < 3) {
                        const int m1 = mu + 1, c1 = m1 == 1 ? y : m1 == 2 ? z : t;
                        nxt = term_index(g, m1, 0, 0, c1, lex - c1 * g.stride[m1], cb, po);
                        issue(nxt, 0, (q + 1) & 1);
                    } else if (a.xpay) {
                        // the xpay records of every right-hand side, in flight during the last term
#pragma unroll
                        for (int j = 0; j < T; j++)
                            cp_async_16(slot(0, kLinkSlots + j), a.y + (size_t)(a.t0 + j) * a.field_bytes + (size_t)cb * 16);
                    }
                    cp_async_commit();  // possibly empty: keeps one group per term
                    cp_async_wait_1();  // this term's copies have landed (this thread's)
                    const int stage = q & 1;
#pragma unroll
                    for (int c = 0; c < LC; c++) lc[c] = *slot(stage, c);
#pragma unroll
                    for (int j = 0; j < T; j++) sc[j] = *slot(stage, kLinkSlots + j);
                } else {
                    cur = term_index(g, mu, hop, dir, cmu, base, cb, po);
                    if (hop == 0)
                        Link<GF, 18>::gather(a.gv.fat, pstride, cur.li, lc);
                    else
                        Link<GF, LREC>::gather(a.gv.lng, pstride, cur.li, lc);
#pragma unroll
                    for (int j = 0; j < T; j++)
                        Spinor<SF>::gather(a.in + (size_t)(a.t0 + j) * a.field_bytes, vh, cur.nb, sc + j * SC);
                }

                // the link, unscaled (fat) or in units of the fat scale (long)
                float U[18];
                if (hop == 0) {
                    Link<GF, 18>::decode(lc, U);
                } else {
                    Link<GF, LREC>::decode(lc, U);
                    if constexpr (kScaled)
#pragma unroll
                        for (int e = 0; e < LREC; e++) U[e] = fmul(U[e], ratio);
                    if constexpr (LREC == 12) {
                        // row 2 = eta * conj(row0 x row1) in true units; with rows 0, 1 in units
                        // of fsc the factor is eta * fsc.  The boundary sign belongs to the
                        // link's own site: x for the forward link, x - 3 mu for the backward one.
                        const bool flip = g.antiperiodic_t && mu == 3 && (dir ? cur.cn : cmu) + 3 >= g.L[3];
                        rebuild_row2(U, (flip ? -eta : eta) * fsc);
                    }
                }
                V ur[9], ui[9];
#pragma unroll
                for (int e = 0; e < 9; e++) {
                    ur[e] = lanes<V>(U[2 * e], U[2 * e]);
                    ui[e] = lanes<V>(U[2 * e + 1], U[2 * e + 1]);
                }
#pragma unroll
                for (int gi = 0; gi < NG; gi++) {
                    V oa[3], ob[3], oc[3];
                    if (dir) {
                        TermOps<SF>::template get<true, V>(sc + gi * NL * SC, oa, ob, oc);
                        term_mv<true, V>(re[gi], im[gi], ur, ui, oa, ob, oc);
                    } else {
                        TermOps<SF>::template get<false, V>(sc + gi * NL * SC, oa, ob, oc);
                        term_mv<false, V>(re[gi], im[gi], ur, ui, oa, ob, oc);
                    }
                }
                if constexpr (STAGED) cur = nxt;
            }
        }

        const float sf = (float)a.sign * fsc;
        if constexpr (STAGED) cp_async_wait_0();  // the xpay records
        // epilogue in groups of up to four right-hand sides: their xpay
        // records are loaded together (one round trip per group)
        constexpr int EG = T < 4 ? T : 4;
#pragma unroll
        for (int e0 = 0; e0 < T; e0 += EG) {
            uint4 yc[EG * SC];
            if (a.xpay) {
#pragma unroll
                for (int j = 0; j < EG; j++) {
                    if constexpr (STAGED)
                        yc[j] = *slot(0, kLinkSlots + e0 + j);
                    else
                        Spinor<SF>::gather(a.y + (size_t)(a.t0 + e0 + j) * a.field_bytes, vh, cb, yc + j * SC);
                }
            }
#pragma unroll
            for (int j = e0; j < e0 + EG; j++) {
                const int gi = j / NL, l = j % NL;
                float o[6];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    o[2 * i] = fmul(sf, lane_of(re[gi][i], l));
                    o[2 * i + 1] = fmul(sf, lane_of(im[gi][i], l));
                }
                const size_t off = (size_t)(a.t0 + j) * a.field_bytes;
                if (a.xpay) {
                    float yv[6];
                    Spinor<SF>::decode(yc + (j - e0) * SC, yv);
                    // a solver's per-system coefficient lives in its state (slots change hands)
                    const float aa = a.st ? (float)a.st[a.t0 + j].diag : (float)a.a[a.t0 + j];
#pragma unroll
                    for (int k = 0; k < 6; k++) o[k] = __fmaf_rn(aa, yv[k], o[k]);
                    if constexpr (RED) {
                        float d = 0.0f;
#pragma unroll
                        for (int k = 0; k < 6; k++) d = __fmaf_rn(yv[k], o[k], d);
                        rv[2 * j] = d;
                    }
                }
                if constexpr (RED) {
                    float n2 = 0.0f;
#pragma unroll
                    for (int k = 0; k < 6; k++) n2 = __fmaf_rn(o[k], o[k], n2);
                    rv[2 * j + 1] = n2;
                }
                if (!Spinor<SF>::store(a.out + off, vh, cb, o)) atomicExch(a.err, 1);
            }
        }
    }

    if constexpr (RED) store_block_partial<2 * T, float>(rv, a.red);  // summed by mrhs_finish_kernel
}

// After a reducing tile launch: one block sums the launch's block partials
// and runs the finisher of each active right-hand side of the tile.  The
// same thread count for every tile keeps each right-hand side's summation
// order, and so its iterates, independent of the tile.
constexpr int kMrhsFinishThreads = 1024;

template <int T>
__global__ void __launch_bounds__(kMrhsFinishThreads) mrhs_finish_kernel(const __grid_constant__ DslashMArgs a, unsigned nblocks)
{
    if (a.active_any != nullptr && *(volatile const int *)a.active_any == 0) return;
    if (!tile_active<T>(a)) return;
    __shared__ double tot[2 * T];
    sum_partials<2 * T, float>(a.red, nblocks, tot);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 2 * T; k++) a.red.result[k] = tot[k];
        run_batch_finisher(a.fin, tot, a.st, a.t0, T, a.slot);
    }
}

template <int GF, int SF, int LREC, int T, bool RED, bool STAGED>
bool launch_mrhs_kernel(const DslashMArgs &a, cudaStream_t s)
{
    auto kern = dslash_mrhs_kernel<GF, SF, LREC, T, RED, STAGED>;
    constexpr size_t smem = STAGED ? mrhs_staged_smem(T) : 0;
    if constexpr (STAGED) {
        static const bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                               cudaSuccess;  // once per kernel
        if (!ok) return false;
    }
    const int nb = (a.g.vh + kMrhsBlock - 1) / kMrhsBlock;
    kern<<<nb, kMrhsBlock, smem, s>>>(a);
    if constexpr (RED) mrhs_finish_kernel<T><<<1, kMrhsFinishThreads, 0, s>>>(a, (unsigned)nb);
    return true;
}

template <int GF, int SF, int LREC, bool RED, bool STAGED>
bool launch_mrhs_tile(int T, const DslashMArgs &a, cudaStream_t s)
{
    switch (T) {
    case 16: return launch_mrhs_kernel<GF, SF, LREC, 16, RED, STAGED>(a, s);
    case 8: return launch_mrhs_kernel<GF, SF, LREC, 8, RED, STAGED>(a, s);
    case 4: return launch_mrhs_kernel<GF, SF, LREC, 4, RED, STAGED>(a, s);
    case 2: return launch_mrhs_kernel<GF, SF, LREC, 2, RED, STAGED>(a, s);
    default: return launch_mrhs_kernel<GF, SF, LREC, 1, RED, STAGED>(a, s);
    }
}

template <int GF, int SF, int LREC, bool RED>
bool launch_mrhs_variant(int T, int variant, const DslashMArgs &a, cudaStream_t s)
{
    if (variant == 1) {
        if constexpr (Spinor<SF>::chunks == 1) return launch_mrhs_tile<GF, SF, LREC, RED, true>(T, a, s);
        return false;
    }
    return launch_mrhs_tile<GF, SF, LREC, RED, false>(T, a, s);
}

// All nrhs right-hand sides in tiles of T (T divides nrhs; one launch per
// tile); variant 0 the register kernel, 1 the staged one (16-byte records).
template <int GF, int SF, typename real>
bool launch_mrhs_t(int long_recon, bool reduce, int T, int variant, const DslashMArgs &args, cudaStream_t s)
{
    static_assert(std::is_same<real, float>::value, "the batched stencil computes in FP32");
    if (long_recon != 12 && long_recon != 18) return false;  // 18- and 12-real long links only
    if (reduce && !red_fits(args.g.vh, kMrhsBlock, 2 * T)) return false;
    for (int t0 = 0; t0 < args.nrhs; t0 += T) {
        if (args.tile_mask != 0u && !((args.tile_mask >> (t0 / T)) & 1u)) continue;  // no system of it iterates
        DslashMArgs a = args;
        a.t0 = t0;
        bool ok;
        if (long_recon == 12)
            ok = reduce ? launch_mrhs_variant<GF, SF, 12, true>(T, variant, a, s)
                        : launch_mrhs_variant<GF, SF, 12, false>(T, variant, a, s);
        else
            ok = reduce ? launch_mrhs_variant<GF, SF, 18, true>(T, variant, a, s)
                        : launch_mrhs_variant<GF, SF, 18, false>(T, variant, a, s);
        if (!ok) return false;
    }
    return true;
}

}  // namespace hisq
