// dslash.cuh -- the HISQ staggered stencil pass (the dominant kernel of every
// solver; Sec. 1 and Sec. 5.3), templated on the storage formats of the gauge
// and spinor fields and on the compute precision (Sec. 4: the triplet).
//
// One thread per output site x of parity p:
//   out(x) = a*y(x) + sign * sum_mu [ F_mu(x) in(x+mu) - F_mu(x-mu)^+ in(x-mu)
//                                    + L_mu(x) in(x+3mu) - L_mu(x-3mu)^+ in(x-3mu) ]
// Links are read exactly once per pass with evict-first loads (16 per site,
// each used once); neighbour spinors are read through the read-only path so
// the 16-fold reuse is served by L1/L2.  Coordinates come from the
// checkerboard index (no index tables), neighbours wrap periodically.
// Compressed long links (r12) rebuild row 2 in registers with the staggered
// phase times boundary sign of the link's site.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "codecs.cuh"
#include "finish.cuh"
#include "internal.h"
#include "launch.cuh"
#include "reduce.cuh"

namespace hisq {

__device__ __forceinline__ int wrap_coord(int c, int L)
{
    c += (c < 0) ? L : 0;
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    c -= (c >= L) ? L : 0;
    return c;
}

// acc += U s, every product accumulated by one fused multiply-add (four per
// complex product: on GB300's narrow FP64 pipe a separate multiply and add
// per pair of products would cost half as many instructions again)
template <typename real>
__device__ __forceinline__ void mv_add(real acc[6], const real U[18], const real s[6])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const real ur = U[2 * (3 * i + j)], ui = U[2 * (3 * i + j) + 1];
            acc[2 * i] = fma(ur, s[2 * j], acc[2 * i]);
            acc[2 * i] = fma(-ui, s[2 * j + 1], acc[2 * i]);
            acc[2 * i + 1] = fma(ur, s[2 * j + 1], acc[2 * i + 1]);
            acc[2 * i + 1] = fma(ui, s[2 * j], acc[2 * i + 1]);
        }
}

// acc -= U^+ s
template <typename real>
__device__ __forceinline__ void mv_adj_sub(real acc[6], const real U[18], const real s[6])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const real ur = U[2 * (3 * j + i)], ui = U[2 * (3 * j + i) + 1];  // conj(U_ji)
            acc[2 * i] = fma(-ur, s[2 * j], acc[2 * i]);
            acc[2 * i] = fma(-ui, s[2 * j + 1], acc[2 * i]);
            acc[2 * i + 1] = fma(-ur, s[2 * j + 1], acc[2 * i + 1]);
            acc[2 * i + 1] = fma(ui, s[2 * j], acc[2 * i + 1]);
        }
}

// Accumulator of one field's terms at a site.  The generic form keeps the
// six reals of the colour vector.  For FP32 compute it keeps, per colour row
// i, the pair sums P_i = sum (Re U, Im U) * (Re s, Re s) and Q_i = sum (Re U,
// Im U) * (Im s, Im s) on the packed FP32 pipe (one __ffma2_rn per two
// products, halving the issue slots of the complex matrix-vector products);
// the colour vector is then (P.x - Q.y, P.y + Q.x).  A subtracted adjoint term
// U^+ s uses the broadcasts (-Re s, Re s) and (-Im s, Im s) on the transposed
// element, which lands its real and imaginary parts in the same two sums.
template <typename real>
struct SiteAccScalar {
    real a[6];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 6; k++) a[k] = 0;
    }
    __device__ __forceinline__ void add(const real U[18], const real s[6]) { mv_add(a, U, s); }
    __device__ __forceinline__ void adj_sub(const real U[18], const real s[6]) { mv_adj_sub(a, U, s); }
    __device__ __forceinline__ real get(int k) const { return a[k]; }
};

struct SiteAccPacked {
    float2 P[3], Q[3];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 3; i++) P[i] = Q[i] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void add(const float U[18], const float s[6])
    {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float2 br = make_float2(s[2 * j], s[2 * j]), bi = make_float2(s[2 * j + 1], s[2 * j + 1]);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float2 u = make_float2(U[2 * (3 * i + j)], U[2 * (3 * i + j) + 1]);
                P[i] = __ffma2_rn(u, br, P[i]);
                Q[i] = __ffma2_rn(u, bi, Q[i]);
            }
        }
    }
    __device__ __forceinline__ void adj_sub(const float U[18], const float s[6])
    {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float2 br = make_float2(-s[2 * j], s[2 * j]), bi = make_float2(-s[2 * j + 1], s[2 * j + 1]);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float2 u = make_float2(U[2 * (3 * j + i)], U[2 * (3 * j + i) + 1]);  // element U_ji
                P[i] = __ffma2_rn(u, br, P[i]);
                Q[i] = __ffma2_rn(u, bi, Q[i]);
            }
        }
    }
    __device__ __forceinline__ float get(int k) const
    {
        const int i = k >> 1;
        return (k & 1) ? P[i].y + Q[i].x : P[i].x - Q[i].y;
    }
};

// (FP64-class compute, FP32 pairs, takes the integer-product path below.)
template <typename real>
using SiteAcc = std::conditional_t<std::is_same<real, float>::value, SiteAccPacked, SiteAccScalar<real>>;

// Launch shapes tried by the tuner: threads per block, the minimum number of
// resident blocks per SM asked of the register allocator (loads in flight per
// thread against warps per SM) and whether the direction loop is unrolled
// (more overlap across directions against a four times larger kernel body):
//   0: 128 threads, no cap, unrolled     1: 128, no cap, rolled
//   2: 128, <= 64 registers, rolled      3: 256, <= 64 registers, rolled
//   4: 128, <= 64 registers, unrolled
constexpr int kNumStencilConfigs = 5;
__host__ __device__ constexpr bool stencil_config_valid(int cfg, int gf) { return cfg >= 0 && cfg < kNumStencilConfigs && gf >= 0; }
__host__ __device__ constexpr int stencil_block(int cfg) { return cfg == 3 ? 256 : 128; }
__host__ __device__ constexpr int stencil_minb(int cfg) { return cfg == 2 ? 8 : cfg == 3 ? 4 : cfg == 4 ? 8 : 1; }
__host__ __device__ constexpr bool stencil_unrolled(int cfg) { return cfg == 0 || cfg == 4; }

// One direction mu of the stencil at site x (coordinates c, lex), accumulated
// into acc.  Fixed-point links are applied unscaled and the sum is kept in
// units of the fat scale: a long term's spinor is multiplied by lsc/fsc (one
// accumulator for both fields keeps registers for loads in flight).
template <typename real, int SF, bool COH>
__device__ __forceinline__ void load_neighbour(const char *b, int n, int i, real s[6])
{
    if constexpr (COH) {
        uint4 c[Spinor<SF>::chunks];
        gather_coherent<SF>(b, n, i, c);
        Spinor<SF>::decode(c, s);
    } else {
        Spinor<SF>::load(b, n, i, s);
    }
}

// Row 2 of a 13-real link whose phase t (as a fraction of pi) the loader left
// in U[12]: e^{i pi t} scale conj(row0 x row1), scale the long links'
// fixed-point scale (rows 0 and 1 are unscaled integers) or 1.
template <typename real>
__device__ __forceinline__ void rebuild_row2_r13(real U[18], real scale)
{
    static_assert(std::is_same<real, float>::value, "13-real links with FP32 compute");
    float sp, cp;
    sincospif(U[12], &sp, &cp);
    rebuild_row2_phase(U, scale * cp, scale * sp);
}

// An 8-real link (arg V00/pi, arg V20/pi, V01, V02, V10 of V = sign U, V in
// SU(3)) rebuilt in registers from unitarity and det V = 1: N = |V01|^2 +
// |V02|^2, V00 = sqrt(1 - N) e^{i pi t1}, V20 = sqrt(N - |V10|^2) e^{i pi t2},
// V11 = -(conj(V00) V01 V10 + conj(V02) conj(V20)) / N, V12 = (conj(V01)
// conj(V20) - conj(V00) V02 V10) / N, V21 = conj(V02 V10 - V00 V12), V22 =
// conj(V00 V11 - V01 V10).  U[0..7] holds the stored reals, es and as the
// element and angle scales (fixed point: the field's scale and 1/qmax); U
// receives V in true units.
__device__ __forceinline__ void rebuild_r8(float U[18], float es, float as)
{
    const float t1 = U[0] * as, t2 = U[1] * as;
    const float a2r = U[2] * es, a2i = U[3] * es, a3r = U[4] * es, a3i = U[5] * es, b1r = U[6] * es, b1i = U[7] * es;
    const float N = a2r * a2r + a2i * a2i + a3r * a3r + a3i * a3i;
    const float ra = sqrtf(fmaxf(1.0f - N, 0.0f)), rc = sqrtf(fmaxf(N - b1r * b1r - b1i * b1i, 0.0f));
    float s1, c1, s2, c2;
    sincospif(t1, &s1, &c1);
    sincospif(t2, &s2, &c2);
    const float inv = 1.0f / N;
    const float a1r = ra * c1, a1i = ra * s1, cr = rc * c2, ci = rc * s2;
    const float a1a2r = a1r * a2r + a1i * a2i, a1a2i = a1r * a2i - a1i * a2r;     // conj(a1) a2
    const float t3r = a1a2r * b1r - a1a2i * b1i, t3i = a1a2r * b1i + a1a2i * b1r;  // * b1
    const float t4r = a3r * cr - a3i * ci, t4i = -(a3r * ci + a3i * cr);            // conj(a3) conj(c1)
    const float b2r = -(t3r + t4r) * inv, b2i = -(t3i + t4i) * inv;
    const float t5r = a2r * cr - a2i * ci, t5i = -(a2r * ci + a2i * cr);            // conj(a2) conj(c1)
    const float a1a3r = a1r * a3r + a1i * a3i, a1a3i = a1r * a3i - a1i * a3r;       // conj(a1) a3
    const float t6r = a1a3r * b1r - a1a3i * b1i, t6i = a1a3r * b1i + a1a3i * b1r;   // * b1
    const float b3r = (t5r - t6r) * inv, b3i = (t5i - t6i) * inv;
    U[0] = a1r; U[1] = a1i; U[2] = a2r; U[3] = a2i; U[4] = a3r; U[5] = a3i;
    U[6] = b1r; U[7] = b1i; U[8] = b2r; U[9] = b2i; U[10] = b3r; U[11] = b3i;
    U[12] = cr; U[13] = ci;
    U[14] = (a3r * b1r - a3i * b1i) - (a1r * b3r - a1i * b3i);
    U[15] = -((a3r * b1i + a3i * b1r) - (a1r * b3i + a1i * b3r));
    U[16] = (a1r * b2r - a1i * b2i) - (a2r * b1r - a2i * b1i);
    U[17] = -((a1r * b2i + a1i * b2r) - (a2r * b1i + a2i * b1r));
}

template <int GF, int SF, typename real, int LREC, bool COH = false, bool KEEP = false>
__device__ __forceinline__ void stencil_direction(const DslashArgs &a, int mu, int cmu, int c3, int lex, int cb,
                                                  int po, size_t pstride, real lsc, real ratio, int phase_sum,
                                                  SiteAcc<real> &acc)
{
    constexpr bool kScaled = LinkScaled<GF>::value;
    const Geom &g = a.g;
    const int vh = g.vh, pi = 1 - po;
    const int L = g.L[mu], st = g.stride[mu];
    const int cp1 = wrap_coord(cmu + 1, L), cm1 = wrap_coord(cmu - 1, L);
    const int cp3 = wrap_coord(cmu + 3, L), cm3 = wrap_coord(cmu - 3, L);
    const int base = lex - cmu * st;
    const int np1 = (base + cp1 * st) >> 1, nm1 = (base + cm1 * st) >> 1;
    const int np3 = (base + cp3 * st) >> 1, nm3 = (base + cm3 * st) >> 1;
    real U[18], s[6];

    Link<GF, 18>::template load<real, KEEP>(a.gv.fat, pstride, (po * 4 + mu) * vh + cb, U);
    load_neighbour<real, SF, COH>(a.in, vh, np1, s);
    acc.add(U, s);

    Link<GF, 18>::template load<real, KEEP>(a.gv.fat, pstride, (pi * 4 + mu) * vh + nm1, U);
    load_neighbour<real, SF, COH>(a.in, vh, nm1, s);
    acc.adj_sub(U, s);

    // row 2 of an r12 link in the units of rows 0 and 1: sign * lsc * conj(row0 x row1)
    const real eta = (phase_sum & 1) ? -lsc : lsc;
    Link<GF, LREC>::template load<real, KEEP>(a.gv.lng, pstride, (po * 4 + mu) * vh + cb, U);
    if constexpr (LREC == 12) {
        const bool flip = g.antiperiodic_t && mu == 3 && c3 + 3 >= L;
        rebuild_row2(U, flip ? -eta : eta);
    } else if constexpr (LREC == 13) {
        rebuild_row2_r13(U, lsc);
    }
    // an 8-real link comes back in true units with its sign removed: the spinor takes the sign and 1/fsc
    if constexpr (LREC == 8) rebuild_r8(U, lsc, kScaled ? 1.0f / 32767.0f : 1.0f);
    load_neighbour<real, SF, COH>(a.in, vh, np3, s);
    if constexpr (LREC == 8) {
        const real r8s = kScaled ? ratio / lsc : real(1);
        const bool flip = g.antiperiodic_t && mu == 3 && c3 + 3 >= L;
        const real f = ((phase_sum & 1) != flip) ? -r8s : r8s;
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] *= f;
    } else if constexpr (kScaled) {
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] *= ratio;
    }
    acc.add(U, s);

    Link<GF, LREC>::template load<real, KEEP>(a.gv.lng, pstride, (pi * 4 + mu) * vh + nm3, U);
    if constexpr (LREC == 12) {
        const bool flip = g.antiperiodic_t && mu == 3 && cm3 + 3 >= L;
        rebuild_row2(U, flip ? -eta : eta);
    } else if constexpr (LREC == 13) {
        rebuild_row2_r13(U, lsc);
    }
    if constexpr (LREC == 8) rebuild_r8(U, lsc, kScaled ? 1.0f / 32767.0f : 1.0f);
    load_neighbour<real, SF, COH>(a.in, vh, nm3, s);
    if constexpr (LREC == 8) {
        const real r8s = kScaled ? ratio / lsc : real(1);
        const bool flip = g.antiperiodic_t && mu == 3 && cm3 + 3 >= L;
        const real f = ((phase_sum & 1) != flip) ? -r8s : r8s;
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] *= f;
    } else if constexpr (kScaled) {
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] *= ratio;
    }
    acc.adj_sub(U, s);
}

// ---------------------------------------------------------------------------
// The 30-bit triplet's FP64-class compute on exact integer products.  A
// 32-bit fixed-point link element u (|u| < 2^31) times a 30-bit field integer
// q (|q| < 2^29) is exact in 64 bits (mad.wide.s32, half the FP32 FMA rate on
// GB300), and one term's colour component, a sum of six such products, stays
// below 6 2^60 < 2^63.  So each term (one link, one neighbour) is formed
// exactly in integers, in units of the link field's scale times the
// neighbour's power of two 2^(E-127); it then enters an FP32-pair accumulator
// per link field: the 64-bit sum is cut into three pieces of at most 22 bits,
// each exact in FP32 and scaled by an exact power of two (one fma against the
// magic 2^23 each), the top piece added with an error-free TwoSum and the two
// lower pieces to the low word.  Instead of twelve FP32 operations per real
// multiply-add (a pair TwoProd and TwoSum), a term costs 36 integer
// multiply-adds and about 17 operations per colour component.
// ---------------------------------------------------------------------------
struct SiteAccI30 {
    float h[2][6], l[2][6];  // [fat, long][component]: unevaluated hi + lo

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int f = 0; f < 2; f++)
#pragma unroll
            for (int k = 0; k < 6; k++) h[f][k] = l[f][k] = 0.0f;
    }

    // acc[f][k] += P 2^e (P exact in 64 bits)
    __device__ __forceinline__ void add(int f, int k, long long P, float p0, float p21, float p42)
    {
        const unsigned lo = (unsigned)P, hi = (unsigned)((unsigned long long)P >> 32);
        const unsigned c0 = lo & 0x1FFFFFu;
        const unsigned c1 = __funnelshift_r(lo, hi, 21) & 0x1FFFFFu;
        const int c2 = (int)hi >> 10;  // bits 42..63 with the sign: |c2| < 2^21
        // 2^23 + c (or 2^23 + 2^22 + c2) is an exact float; one fma removes the offset and scales
        const float f0 = __fmaf_rn(__uint_as_float(0x4B000000u | c0), p0, -8388608.0f * p0);
        const float f1 = __fmaf_rn(__uint_as_float(0x4B000000u | c1), p21, -8388608.0f * p21);
        const float f2 = __fmaf_rn(__uint_as_float(0x4B000000u | (unsigned)(c2 + 0x400000)), p42, -12582912.0f * p42);
        const float s = __fadd_rn(h[f][k], f2);
        const float bb = __fsub_rn(s, h[f][k]);
        const float e = __fadd_rn(__fsub_rn(h[f][k], __fsub_rn(s, bb)), __fsub_rn(f2, bb));
        h[f][k] = s;
        l[f][k] = __fadd_rn(l[f][k], __fadd_rn(e, __fadd_rn(f1, f0)));
    }

    // one term: U s (BWD: -U^+ s) with u the link's 18 integers and q the
    // neighbour's 6 integers at the power of two 2^(E-127)
    template <bool BWD>
    __device__ __forceinline__ void term(int f, const int u[18], const int q[6], unsigned E)
    {
        // 2^(E-127), 2^(E-106), 2^(E-85) as exact floats (exponent fields clamped at 255: a term that
        // large overflows the FP32-range pairs anyway and the store reports it)
        const float p0 = __uint_as_float(E << 23);
        const float p21 = __uint_as_float(min(E + 21u, 255u) << 23);
        const float p42 = __uint_as_float(min(E + 42u, 255u) << 23);
        int sr[3], si[3], nsr[3], nsi[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            sr[j] = q[2 * j];
            si[j] = q[2 * j + 1];
            nsr[j] = -sr[j];
            nsi[j] = -si[j];
        }
#pragma unroll
        for (int i = 0; i < 3; i++) {
            long long re = 0, im = 0;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                // forward: Re += Ur sr - Ui si, Im += Ur si + Ui sr       (U_ij)
                // backward: Re += -Ur sr - Ui si, Im += -Ur si + Ui sr   (U_ji, conjugated, subtracted)
                const int e = BWD ? 3 * j + i : 3 * i + j;
                const int ur = u[2 * e], ui = u[2 * e + 1];
                asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(re) : "r"(ur), "r"(BWD ? nsr[j] : sr[j]));
                asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(re) : "r"(ui), "r"(nsi[j]));
                asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(im) : "r"(ur), "r"(BWD ? nsi[j] : si[j]));
                asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(im) : "r"(ui), "r"(sr[j]));
            }
            add(f, 2 * i, re, p0, p21, p42);
            add(f, 2 * i + 1, im, p0, p21, p42);
        }
    }

    // the total fsc * fat + lsc * long of component k
    __device__ __forceinline__ ff get(int k, ff fsc, ff lsc) const
    {
        const ff a = ff_fast_two_sum(h[0][k], l[0][k]) * fsc;
        const ff b = ff_fast_two_sum(h[1][k], l[1][k]) * lsc;
        return a + b;
    }
};

// A link of 18 32-bit fixed-point integers, raw.
template <bool KEEP>
__device__ __forceinline__ void load_link_ints(const char *base, size_t pstride, int li, int u[18])
{
    uint4 c[Link<G_FIX32, 18>::chunks];
    Link<G_FIX32, 18>::template gather<KEEP>(base, pstride, li, c);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        u[4 * k] = (int)c[k].x; u[4 * k + 1] = (int)c[k].y; u[4 * k + 2] = (int)c[k].z; u[4 * k + 3] = (int)c[k].w;
    }
    u[16] = (int)c[4].x;
    u[17] = (int)c[4].y;
}

// A 12-real long link in integers: rows 0 and 1 as stored (32-bit fixed
// point, scale s), row 2 = sgn * conj(row0 x row1) rebuilt exactly in 64-bit
// integers (row 1 halved with rounding first, so that each component, at most
// 1/(2 s^2) by unitarity, stays below 2^63 for any field whose largest element
// is at least 1/sqrt(3)) and brought back to the scale s in integers:
// q = round(P * 2s), 2s = mul * 2^-(32 + shift).  The rounding adds at most one
// unit of the 32-bit grid to row 2.
__device__ __forceinline__ int rescale_row2(long long P, int mul, int shift)
{
    const int ph = (int)(P >> 32);
    const unsigned pl = (unsigned)P;
    long long t = (long long)ph * mul + (long long)__umulhi(pl, (unsigned)mul);  // floor(P mul / 2^32)
    t = (t + (1LL << (shift - 1))) >> shift;
    t = t > 2147483647LL ? 2147483647LL : t < -2147483647LL ? -2147483647LL : t;
    return (int)t;
}

template <bool KEEP>
__device__ __forceinline__ void load_link_ints_r12(const char *base, size_t pstride, int li, int u[18], int sgn,
                                                   int mul, int shift)
{
    uint4 c[Link<G_FIX32, 12>::chunks];
    Link<G_FIX32, 12>::template gather<KEEP>(base, pstride, li, c);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        u[4 * k] = (int)c[k].x; u[4 * k + 1] = (int)c[k].y; u[4 * k + 2] = (int)c[k].z; u[4 * k + 3] = (int)c[k].w;
    }
    int b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = (u[6 + k] >> 1) + (u[6 + k] & 1);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;  // (row0 x row1)_j = a_k b_l - a_l b_k
        const int akr = u[2 * k], aki = u[2 * k + 1], alr = u[2 * l], ali = u[2 * l + 1];
        const int bkr = b[2 * k], bki = b[2 * k + 1], blr = b[2 * l], bli = b[2 * l + 1];
        long long pr = 0, pi = 0;
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pr) : "r"(akr), "r"(blr));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pr) : "r"(-aki), "r"(bli));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pr) : "r"(-alr), "r"(bkr));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pr) : "r"(ali), "r"(bki));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pi) : "r"(akr), "r"(bli));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pi) : "r"(aki), "r"(blr));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pi) : "r"(-alr), "r"(bki));
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pi) : "r"(-ali), "r"(bkr));
        u[12 + 2 * j] = sgn * rescale_row2(pr, mul, shift);
        u[13 + 2 * j] = -sgn * rescale_row2(pi, mul, shift);
    }
}

// A 30-bit record, raw: its six integers and its exponent field.
template <bool COH>
__device__ __forceinline__ unsigned load_int30_raw(const char *b, int n, int i, int q[6])
{
    uint4 c[2];
    if constexpr (COH)
        gather_coherent<S_INT30>(b, n, i, c);
    else
        Spinor<S_INT30>::gather(b, n, i, c);
    q[0] = sext_bits(c[0].x, 30); q[1] = sext_bits(c[0].y, 30);
    q[2] = sext_bits(c[0].z, 30); q[3] = sext_bits(c[0].w, 30);
    q[4] = sext_bits(c[1].x, 30); q[5] = sext_bits(c[1].y, 30);
    return (c[0].x >> 30) | ((c[0].y >> 30) << 2) | ((c[0].z >> 30) << 4) | ((c[0].w >> 30) << 6);
}

template <bool COH, bool KEEP, int LREC>
__device__ __forceinline__ void stencil_direction_i30(const DslashArgs &a, int mu, int cmu, int lex, int cb, int po,
                                                      size_t pstride, int phase_sum, SiteAccI30 &acc)
{
    const Geom &g = a.g;
    const int vh = g.vh, pi = 1 - po;
    const int L = g.L[mu], st = g.stride[mu];
    const int base = lex - cmu * st;
    const int np1 = (base + wrap_coord(cmu + 1, L) * st) >> 1, nm1 = (base + wrap_coord(cmu - 1, L) * st) >> 1;
    const int np3 = (base + wrap_coord(cmu + 3, L) * st) >> 1, nm3 = (base + wrap_coord(cmu - 3, L) * st) >> 1;
    int u[18], q[6];
    unsigned E;
    load_link_ints<KEEP>(a.gv.fat, pstride, (po * 4 + mu) * vh + cb, u);
    E = load_int30_raw<COH>(a.in, vh, np1, q);
    acc.term<false>(0, u, q, E);
    load_link_ints<KEEP>(a.gv.fat, pstride, (pi * 4 + mu) * vh + nm1, u);
    E = load_int30_raw<COH>(a.in, vh, nm1, q);
    acc.term<true>(0, u, q, E);
    if constexpr (LREC == 12) {
        // the sign of a long link: its staggered phase, flipped across an antiperiodic t boundary
        const int cm3 = wrap_coord(cmu - 3, L);
        const int eta = (phase_sum & 1) ? -1 : 1;
        const bool flipf = g.antiperiodic_t && mu == 3 && cmu + 3 >= L;
        const bool flipb = g.antiperiodic_t && mu == 3 && cm3 + 3 >= L;
        load_link_ints_r12<KEEP>(a.gv.lng, pstride, (po * 4 + mu) * vh + cb, u, flipf ? -eta : eta,
                                 a.gv.lng_r2_mul, a.gv.lng_r2_shift);
        E = load_int30_raw<COH>(a.in, vh, np3, q);
        acc.term<false>(1, u, q, E);
        load_link_ints_r12<KEEP>(a.gv.lng, pstride, (pi * 4 + mu) * vh + nm3, u, flipb ? -eta : eta,
                                 a.gv.lng_r2_mul, a.gv.lng_r2_shift);
    } else {
        load_link_ints<KEEP>(a.gv.lng, pstride, (po * 4 + mu) * vh + cb, u);
        E = load_int30_raw<COH>(a.in, vh, np3, q);
        acc.term<false>(1, u, q, E);
        load_link_ints<KEEP>(a.gv.lng, pstride, (pi * 4 + mu) * vh + nm3, u);
    }
    E = load_int30_raw<COH>(a.in, vh, nm3, q);
    acc.term<true>(1, u, q, E);
}

template <int GF, int SF, typename real, int LREC>
struct UsesIntPath {
    static constexpr bool value = GF == G_FIX32 && SF == S_INT30 && is_ff<real>::value && (LREC == 18 || LREC == 12);
};

// One output site cb: the stencil, the optional xpay, the store and, when
// reducing, this site's Re<y, out> and |out|^2 added to rv (in the compute
// precision; reduce_grid sums the threads).
template <int GF, int SF, typename real, int LREC, bool RED, int CFG, bool COH = false, bool KEEP = false>
__device__ __forceinline__ void stencil_site(const DslashArgs &a, int cb, size_t pstride, real fsc, real lsc,
                                             real ratio, real rv[2])
{
    const Geom &g = a.g;
    const int vh = g.vh;
    const int po = a.out_parity;
    int r = cb / g.xh;
    const int xh = cb - r * g.xh;
    const int y = r % g.L[1];
    r /= g.L[1];
    const int z = r % g.L[2];
    const int t = r / g.L[2];
    const int x = 2 * xh + ((y + z + t + po) & 1);
    const int c[4] = {x, y, z, t};
    const int lex = 2 * cb + (x & 1);
    real o[6];
    if constexpr (UsesIntPath<GF, SF, real, LREC>::value) {
        SiteAccI30 acc;
        acc.zero();
        if constexpr (stencil_unrolled(CFG)) {
            int phase_sum = 0;  // x + y + ... below mu: the staggered phase eta_mu(x)
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                stencil_direction_i30<COH, KEEP, LREC>(a, mu, c[mu], lex, cb, po, pstride, phase_sum, acc);
                phase_sum += c[mu];
            }
        } else {
            int phase_sum = 0;
#pragma unroll 1
            for (int mu = 0; mu < 4; mu++) {
                const int cmu = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t;
                stencil_direction_i30<COH, KEEP, LREC>(a, mu, cmu, lex, cb, po, pstride, phase_sum, acc);
                phase_sum += cmu;
            }
        }
        const ff sgn((float)a.sign);
#pragma unroll
        for (int k = 0; k < 6; k++) o[k] = acc.get(k, fsc, lsc) * sgn;
    } else {
    SiteAcc<real> acc;
    acc.zero();
    if constexpr (stencil_unrolled(CFG)) {
        int phase_sum = 0;  // x + y + ... below mu: the staggered phase eta_mu(x)
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            stencil_direction<GF, SF, real, LREC, COH, KEEP>(a, mu, c[mu], t, lex, cb, po, pstride, lsc, ratio,
                                                             phase_sum, acc);
            phase_sum += c[mu];
        }
    } else {
        int phase_sum = 0;
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
            const int cmu = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t;
            stencil_direction<GF, SF, real, LREC, COH, KEEP>(a, mu, cmu, t, lex, cb, po, pstride, lsc, ratio,
                                                             phase_sum, acc);
            phase_sum += cmu;
        }
    }

    const real sf = (real)a.sign * fsc;
#pragma unroll
    for (int k = 0; k < 6; k++) o[k] = sf * acc.get(k);
    }
    if constexpr (RED && UsesIntPath<GF, SF, real, LREC>::value) {
        // FP64-class: Re<y, out> and |out|^2 exactly in integers from the stored 30-bit records
        int32_t qy[6] = {0, 0, 0, 0, 0, 0};
        uint32_t Ey = 0;
        if (a.xpay) {
            uint4 cy[Spinor<S_INT30>::chunks];
            Spinor<S_INT30>::gather(a.y, vh, cb, cy);
            Ey = Spinor<S_INT30>::raw(cy, qy);
            real yv[6];
            Spinor<S_INT30>::decode(cy, yv);
            const real aa = (real)a.a;
#pragma unroll
            for (int k = 0; k < 6; k++) o[k] = aa * yv[k] + o[k];
        }
        uint32_t qo[6], Eo;
        if (!Spinor<S_INT30>::store_ff_q(a.out, vh, cb, o, qo, Eo)) atomicExch(a.err, 1);
        long long d = 0, n2 = 0;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(d) : "r"(qy[k]), "r"((int)qo[k]));
            asm("mad.wide.s32 %0, %1, %1, %0;" : "+l"(n2) : "r"((int)qo[k]));
        }
        if (a.xpay) rv[0] += ff_ldexp(ff_from_ll(d), (int)Ey + (int)Eo - 254);  // a record is q 2^(E-127)
        rv[1] += ff_ldexp(ff_from_ll(n2), 2 * (int)Eo - 254);
        return;
    }
    if (a.xpay) {
        real yv[6];
        Spinor<SF>::load(a.y, vh, cb, yv);
        const real aa = (real)a.a;
#pragma unroll
        for (int k = 0; k < 6; k++) o[k] = aa * yv[k] + o[k];
        if constexpr (RED) {
            real d = 0;
#pragma unroll
            for (int k = 0; k < 6; k++) d += yv[k] * o[k];
            rv[0] += d;
        }
    }
    if constexpr (RED) {
        real n2 = 0;
#pragma unroll
        for (int k = 0; k < 6; k++) n2 += o[k] * o[k];
        rv[1] += n2;
    }
    if (!Spinor<SF>::store(a.out, vh, cb, o)) atomicExch(a.err, 1);
}

// One thread per site.  A reducing pass ends each block with its block sum
// and a partial store; stencil_finish_kernel, launched after it, sums them
// (in the CG the residual update's blocks sum them instead: blas.cu).
template <int GF, int SF, typename real, int LREC, bool RED, int CFG>
__global__ void __launch_bounds__(stencil_block(CFG), stencil_minb(CFG))
    dslash_kernel(const __grid_constant__ DslashArgs a)
{
    pdl_wait();  // the input, xpay and state fields come from the previous kernel
    pdl_launch_dependents();
    if (a.active != nullptr && *(volatile const int *)a.active == 0) return;  // uniform over the grid
    const int vh = a.g.vh;
    const size_t pstride = (size_t)8 * vh * 16;
    constexpr bool kScaled = LinkScaled<GF>::value;
    // fixed-point links are applied unscaled, the sum kept in units of the fat scale
    const real fsc = kScaled ? (sizeof(real) == 8 ? (real)a.gv.fat_scale_d : (real)a.gv.fat_scale_f) : real(1);
    const real lsc = kScaled ? (sizeof(real) == 8 ? (real)a.gv.lng_scale_d : (real)a.gv.lng_scale_f) : real(1);
    const real ratio = lsc / fsc;
    real rv[2] = {real(0), real(0)};
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb < vh) stencil_site<GF, SF, real, LREC, RED, CFG>(a, cb, pstride, fsc, lsc, ratio, rv);
    if constexpr (RED) {  // summed by stencil_finish_kernel or by the CG's residual update
        const red_t<real> r2[2] = {(red_t<real>)rv[0], (red_t<real>)rv[1]};
        store_block_partial<2>(r2, a.red);
    }
}

// After a reducing pass: one block sums the pass's block partials and runs the
// solver's finisher (a separate launch instead of a completion counter in
// every block of the pass: no fence or atomic ends a stencil block).
template <typename real>
__global__ void __launch_bounds__(1024) stencil_finish_kernel(RedBuf red, unsigned nblocks, int fin, void *st,
                                                               int slot, const int *active)
{
    pdl_wait();
    pdl_launch_dependents();
    if (active != nullptr && *(volatile const int *)active == 0) return;
    __shared__ double tot[2];
    sum_partials<2, part_t<real>>(red, nblocks, tot);
    if (threadIdx.x == 0) {
        red.result[0] = tot[0];
        red.result[1] = tot[1];
        run_finisher(fin, tot, st, slot);
    }
}

template <int GF, int SF, typename real, int LREC, bool RED, int CFG>
void launch_cfg(const DslashArgs &a, cudaStream_t s)
{
    constexpr int B = stencil_block(CFG);
    const int nb = (a.g.vh + B - 1) / B;
    launch_chained(dslash_kernel<GF, SF, real, LREC, RED, CFG>, dim3(nb), dim3(B), s, a);
    if constexpr (RED)
        if (!a.defer_finish)
            launch_chained(stencil_finish_kernel<real>, dim3(1), dim3(1024), s, a.red, (unsigned)nb, a.fin, a.st,
                           a.slot, a.active);
}

template <int GF, int SF, typename real, int LREC, bool RED>
void launch_any(int cfg, const DslashArgs &a, cudaStream_t s)
{
    switch (cfg) {
    case 1: launch_cfg<GF, SF, real, LREC, RED, 1>(a, s); break;
    case 2: launch_cfg<GF, SF, real, LREC, RED, 2>(a, s); break;
    case 3: launch_cfg<GF, SF, real, LREC, RED, 3>(a, s); break;
    case 4: launch_cfg<GF, SF, real, LREC, RED, 4>(a, s); break;
    default: launch_cfg<GF, SF, real, LREC, RED, 0>(a, s); break;
    }
}

template <int GF, int SF, typename real>
bool launch_dslash_t(int long_recon, bool reduce, int cfg, const DslashArgs &a, cudaStream_t s)
{
    if (long_recon == 13 || long_recon == 8) {  // FP32 compute with 16-bit or FP32 links
        if constexpr (std::is_same<real, float>::value && (GF == G_FIX16 || GF == G_F32)) {
            if (long_recon == 13) {
                if (reduce)
                    launch_any<GF, SF, real, 13, true>(cfg, a, s);
                else
                    launch_any<GF, SF, real, 13, false>(cfg, a, s);
            } else {
                if (reduce)
                    launch_any<GF, SF, real, 8, true>(cfg, a, s);
                else
                    launch_any<GF, SF, real, 8, false>(cfg, a, s);
            }
            return true;
        }
        return false;
    }
    if (long_recon != 12 && long_recon != 18) return false;
    if (long_recon == 12) {
        if (reduce)
            launch_any<GF, SF, real, 12, true>(cfg, a, s);
        else
            launch_any<GF, SF, real, 12, false>(cfg, a, s);
    } else {
        if (reduce)
            launch_any<GF, SF, real, 18, true>(cfg, a, s);
        else
            launch_any<GF, SF, real, 18, false>(cfg, a, s);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Fused M_ee pass.  Both stencil passes of M_ee = diag - D_eo D_oe read every
// link of the lattice; run one after the other, the second reads them from
// HBM again.  Here one persistent kernel (one wave of blocks) sweeps the
// lattice in t-slices: D_oe of slice t into tmp, and D_eo of slice s as soon
// as D_oe is complete on slices s-3..s+3 (the reach of the three-hop term).
// The links D_eo(s) applies were read by D_oe a few slices earlier and are
// still in L2, so the pass reads them from HBM about once.
//
// Work items (slice task, chunk of one site per thread) are handed out in a
// fixed order by an atomic counter; a D_eo item only waits for D_oe items that
// come earlier in that order, and D_oe items never wait, so every wait ends.
// Each wait is also bounded: past the limit the kernel flags the error (bit 2
// of the error word) and goes on, so a fault can cost results, never a hang.
// The queue order puts D_eo(s) `lag` slices after the last D_oe slice it
// reads (so that, with a wave of blocks in flight, those D_oe items have
// mostly finished when it is taken), P = 6 + lag:
//   Lt >= 7 + lag:  D_oe 0..P-1, then (D_oe i, D_eo i-3-lag) for i = P..Lt-1,
//                   then D_eo 0, 1, 2, Lt-3-lag, ..., Lt-1;
//   otherwise:      every D_oe slice, then every D_eo slice.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mee_task(int k, int Lt, int lag, int &kind, int &slice)
{
    const int P = 6 + lag;  // leading D_oe-only tasks
    if (Lt < 7 + lag) {     // short lattice: every D_oe slice, then every D_eo slice
        kind = k >= Lt;
        slice = k - (kind ? Lt : 0);
        return;
    }
    if (k < P) {
        kind = 0;
        slice = k;
        return;
    }
    if (k < P + 2 * (Lt - P)) {  // pairs (D_oe i, D_eo i-3-lag), i = P..Lt-1
        const int j = k - P, i = P + (j >> 1);
        kind = j & 1;
        slice = kind ? i - 3 - lag : i;
        return;
    }
    const int m = k - P - 2 * (Lt - P);  // tail: D_eo 0, 1, 2 and Lt-3-lag..Lt-1
    kind = 1;
    slice = m < 3 ? m : Lt - 3 - lag + (m - 3);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr unsigned kMeeWaitPolls = 1u << 22;  // x >= 64 ns sleep: bounded well under a second

template <int GF, int SF, typename real, int LREC, int CFG>
__global__ void __launch_bounds__(stencil_block(CFG), stencil_minb(CFG))
    mee_fused_kernel(const __grid_constant__ MeeArgs m)
{
    const DslashArgs &a1 = m.d1, &a2 = m.d2;
    if (a2.active != nullptr && *(volatile const int *)a2.active == 0) return;  // uniform over the grid
    const Geom &g = a1.g;
    const int vh = g.vh, Lt = g.L[3];
    const size_t pstride = (size_t)8 * vh * 16;
    constexpr bool kScaled = LinkScaled<GF>::value;
    const real fsc = kScaled ? (sizeof(real) == 8 ? (real)a1.gv.fat_scale_d : (real)a1.gv.fat_scale_f) : real(1);
    const real lsc = kScaled ? (sizeof(real) == 8 ? (real)a1.gv.lng_scale_d : (real)a1.gv.lng_scale_f) : real(1);
    const real ratio = lsc / fsc;
    unsigned *work = a2.red.sync, *done = a2.red.sync + 32;
    const int B = blockDim.x;
    const int vs = vh / Lt;                // sites of one parity in a t-slice
    const int nch = (vs + B - 1) / B;      // chunks per slice
    const int nitems = 2 * Lt * nch;
    real rv[2] = {0, 0};
    __shared__ int item_sh;
    for (;;) {
        if (threadIdx.x == 0) item_sh = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int item = item_sh;
        __syncthreads();  // item_sh is rewritten by the next fetch
        if (item >= nitems) break;
        const int task = item / nch, chunk = item - task * nch;
        int kind, slice;
        mee_task(task, Lt, m.lag, kind, slice);
        const int off = chunk * B + (int)threadIdx.x;
        const int cb = slice * vs + off;
        if (kind == 0) {
            // links stay in L2 for D_eo a few slices later
            if (off < vs) stencil_site<GF, SF, real, LREC, false, CFG, false, true>(a1, cb, pstride, fsc, lsc, ratio, rv);
            __syncthreads();  // every thread's tmp stores precede the release below
            if (threadIdx.x == 0) red_release_add(done + slice, 1u);
        } else {
            if (threadIdx.x == 0) {
                for (int d = -3; d <= 3; d++) {
                    const int t = (slice + d + Lt) % Lt;
                    unsigned polls = 0;
                    while (ld_acquire(done + t) < (unsigned)nch + m.wait_extra) {
                        if (++polls > m.wait_polls) {
                            atomicOr(a2.err, 2);
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
            __syncthreads();
            // tmp is written by other blocks of this kernel: read through L2
            if (off < vs) stencil_site<GF, SF, real, LREC, true, CFG, true>(a2, cb, pstride, fsc, lsc, ratio, rv);
        }
    }
    __shared__ double tot[2];
    if (reduce_grid<2>(rv, a2.red, tot)) {  // the last block: every item is finished
        for (int t = threadIdx.x; t < Lt; t += B) done[t] = 0u;
        if (threadIdx.x == 0) {
            *work = 0u;
            run_finisher(a2.fin, tot, a2.st, a2.slot);
        }
    }
}

template <int GF, int SF, typename real, int LREC, int CFG>
void launch_mee_cfg(const MeeArgs &m, cudaStream_t s)
{
    constexpr int B = stencil_block(CFG);
    auto kern = mee_fused_kernel<GF, SF, real, LREC, CFG>;
    static const int wave = wave_blocks(kern, B);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = m.blocks_per_sm > 0 && m.blocks_per_sm * sms < wave ? m.blocks_per_sm * sms : wave;
    kern<<<grid, B, 0, s>>>(m);
}

template <int GF, int SF, typename real>
bool launch_mee_fused_t(int long_recon, int cfg, const MeeArgs &m, cudaStream_t s)
{
    // the unrolled 64-register shape only (the one the separate passes pick)
    (void)cfg;
    if (long_recon != 12 && long_recon != 18) return false;  // other long-link formats: two passes
    if (long_recon == 12)
        launch_mee_cfg<GF, SF, real, 12, 4>(m, s);
    else
        launch_mee_cfg<GF, SF, real, 18, 4>(m, s);
    return true;
}

}  // namespace hisq
