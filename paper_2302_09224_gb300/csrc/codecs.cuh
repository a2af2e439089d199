// codecs.cuh -- device-side storage formats: every kernel reads a site or link
// through these and converts to the compute precision in registers (Sec. 5.1:
// the format is a property of the accessor, not of the computation).
//
// Spinor formats (one half-lattice field of n sites; planar layout: 16-byte
// planes [plane][site] then a narrower tail plane):
//   F64    3 x 16 B        complex c in plane c
//   F32    16 + 8 B        (c0, c1) | (c2)
//   HALF   16 B            int16 q[6] | FP32 site max  (Sec. 2, Listing 1)
//   INT20  16 B            four words of the Appendix A bitfield layout
//   INT14  8 + 4 B         three words of 16-bit halves (q << 2 | exponent bits)
//   INT30  16 + 8 B        words 0..3 | words 4..5 (Sec. 4, Listing 3; our layout)
// Link formats ([plane][parity][mu][Vh]; reals row-major, first 12 for r12):
//   F64 16 B = 1 complex, F32 16 B = 2 complex, FIX16 16 B = 8 int16,
//   FIX32 16 B = 4 int32, SE15 16 B = 8 halves (15-bit q << 1 | one bit of
//   the link's exponent in halves 0..7); leftover reals go to a 4- or 8-byte
//   tail plane.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ff.cuh"
#include "internal.h"

namespace hisq {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// (gather_coherent, after the Spinor codecs, reads a record through L2 only.)
__device__ __forceinline__ int32_t sext_bits(uint32_t u, int bits)
{
    const uint32_t m = 1u << (bits - 1);
    u &= (1u << bits) - 1u;
    return (int32_t)((u ^ m) - m);
}

__device__ __forceinline__ uint32_t lo16(int v) { return (uint32_t)v & 0xffffu; }

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p)
{
    return __ldcs(p);  // read once: evict-first in L1 and L2
}

template <typename T>
__device__ __forceinline__ T ld_cached(const T *p)
{
    return __ldg(p);
}

// FP32 helpers that must not be contracted (codec arithmetic is specified
// step by step and is bit-exact with the CPU definition).
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// 16-bit fields: the hardware signed-halfword conversion (exact: |q| < 2^24).
// Measured on sm_103a it issues fewer instructions than any FP32-pipe
// emulation, which matters in the issue-bound stencil.
__device__ __forceinline__ float i16lo_to_f(uint32_t w)
{
    float f;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.rn.f32.s16 %0, lo; }" : "=f"(f) : "r"(w));
    return f;
}
__device__ __forceinline__ float i16hi_to_f(uint32_t w)
{
    float f;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.rn.f32.s16 %0, hi; }" : "=f"(f) : "r"(w));
    return f;
}

// 20-bit fields, exact on the FP32 and integer pipes: the two's-complement
// field u, offset by 2^19, is placed in the mantissa of 2^23 and the offset
// is subtracted; both operands are integers below 2^24, so the subtraction
// is exact and the result equals (float)q.
__device__ __forceinline__ float i20_to_f(uint32_t u)
{
    return __fsub_rn(__uint_as_float((u & 0xfffffu) ^ 0x4B080000u), 8912896.0f);  // 2^23 + 2^19
}

// ---------------------------------------------------------------------------
// spinor codecs
// ---------------------------------------------------------------------------
template <int SF>
struct Spinor;

template <>
struct Spinor<S_F64> {
    static constexpr int chunks = 3;  // 16-byte chunks per site (a tail chunk holds its bytes first)
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
#pragma unroll
        for (int k = 0; k < 3; k++) c[k] = ld_cached(reinterpret_cast<const uint4 *>(b) + (size_t)k * n + i);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            v[2 * k] = (real)__hiloint2double((int)c[k].y, (int)c[k].x);
            v[2 * k + 1] = (real)__hiloint2double((int)c[k].w, (int)c[k].z);
        }
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        double2 *p = reinterpret_cast<double2 *>(b);
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            p[(size_t)c * n + i] = make_double2((double)v[2 * c], (double)v[2 * c + 1]);
            ok = ok && isfinite((double)v[2 * c]) && isfinite((double)v[2 * c + 1]);
        }
        return ok;
    }
};

template <>
struct Spinor<S_F32> {
    static constexpr int chunks = 2;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
        c[0] = ld_cached(reinterpret_cast<const uint4 *>(b) + i);
        const uint2 t = ld_cached(reinterpret_cast<const uint2 *>(b + (size_t)16 * n) + i);
        c[1] = make_uint4(t.x, t.y, 0u, 0u);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
        v[0] = __uint_as_float(c[0].x); v[1] = __uint_as_float(c[0].y);
        v[2] = __uint_as_float(c[0].z); v[3] = __uint_as_float(c[0].w);
        v[4] = __uint_as_float(c[1].x); v[5] = __uint_as_float(c[1].y);
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        float f[6];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            f[k] = (float)v[k];
            ok = ok && isfinite(f[k]);
        }
        reinterpret_cast<float4 *>(b)[i] = make_float4(f[0], f[1], f[2], f[3]);
        reinterpret_cast<float2 *>(b + (size_t)16 * n)[i] = make_float2(f[4], f[5]);
        return ok;
    }
};

// 16-bit fixed point with a site-local FP32 norm.  Encode: inv = 32767/max
// (IEEE), q = rint(v*inv) clamped to +-32767; decode: v = q * (max*fl(1/32767)).
// Sites with max below 2^-110 (32767/max would overflow) are stored as zero.
template <>
struct Spinor<S_HALF> {
    static constexpr int chunks = 1;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
        (void)n;
        c[0] = ld_cached(reinterpret_cast<const uint4 *>(b) + i);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
        const uint4 r = c[0];
        const float scale = fmul(__uint_as_float(r.w), 1.0f / 32767.0f);
        const float q[6] = {i16lo_to_f(r.x), i16hi_to_f(r.x), i16lo_to_f(r.y),
                            i16hi_to_f(r.y), i16lo_to_f(r.z), i16hi_to_f(r.z)};
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = (real)fmul(q[k], scale);
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        (void)n;
        float f[6];
        float mx = 0.0f;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            f[k] = (float)v[k];
            ok = ok && isfinite(f[k]);
            mx = fmaxf(mx, fabsf(f[k]));
        }
        int q[6] = {0, 0, 0, 0, 0, 0};
        if (!ok || mx < 0x1p-110f) {  // non-finite, or too small for 32767/max in FP32
            mx = 0.0f;
        } else {
            const float inv = __fdiv_rn(32767.0f, mx);
#pragma unroll
            for (int k = 0; k < 6; k++) q[k] = max(-32767, min(32767, __float2int_rn(fmul(f[k], inv))));
        }
        int4 r;
        r.x = (int)(lo16(q[0]) | (lo16(q[1]) << 16));
        r.y = (int)(lo16(q[2]) | (lo16(q[3]) << 16));
        r.z = (int)(lo16(q[4]) | (lo16(q[5]) << 16));
        r.w = __float_as_int(mx);
        reinterpret_cast<int4 *>(b)[i] = r;
        return ok;
    }
};

// 20-bit shared exponent (Appendix A): E = exponent field of fl(max/(2^19-1))
// plus one, q = rint(v * 2^-(E-127)), bitfields least-significant first.
template <>
struct Spinor<S_INT20> {
    static constexpr int chunks = 1;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
        (void)n;
        c[0] = ld_cached(reinterpret_cast<const uint4 *>(b) + i);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
        const uint4 w = c[0];
        const float up = __uint_as_float((w.w >> 24) << 23);
        const uint32_t u[6] = {w.x,
                               ((w.x >> 20) << 8) | (w.y & 0xffu),
                               w.y >> 8,
                               ((w.y >> 28) << 16) | (w.z & 0xffffu),
                               ((w.z >> 16) << 4) | (w.w & 0xfu),
                               w.w >> 4};
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = (real)fmul(i20_to_f(u[k]), up);
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        (void)n;
        float f[6];
        float mx = 0.0f;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            f[k] = (float)v[k];
            ok = ok && isfinite(f[k]);
            mx = fmaxf(mx, fabsf(f[k]));
        }
        uint32_t u[6] = {0, 0, 0, 0, 0, 0};
        uint32_t E = 1;
        if (ok) {
            const float t = __fdiv_rn(mx, 524287.0f);
            E = ((__float_as_uint(t) >> 23) & 0xffu) + 1u;
            const float down = __uint_as_float((254u - E) << 23);
#pragma unroll
            for (int k = 0; k < 6; k++) u[k] = (uint32_t)__float2int_rn(fmul(f[k], down));
        }
        uint4 w;
        w.x = (u[0] & 0xfffffu) | (((u[1] >> 8) & 0xfffu) << 20);
        w.y = (u[1] & 0xffu) | ((u[2] & 0xfffffu) << 8) | (((u[3] >> 16) & 0xfu) << 28);
        w.z = (u[3] & 0xffffu) | (((u[4] >> 4) & 0xffffu) << 16);
        w.w = (u[4] & 0xfu) | ((u[5] & 0xfffffu) << 4) | (E << 24);
        reinterpret_cast<uint4 *>(b)[i] = w;
        return ok;
    }
};

// 14-bit shared exponent in 12 bytes (a third width of the Sec. 4 family):
// three words of two 16-bit halves, half k = q_k << 2 | e_k with e_k the
// exponent bits 2k..2k+1 (k < 4) and 0 for k = 4, 5; an 8-byte plane (words
// 0, 1) and a 4-byte plane (word 2).  Encode as the 20-bit format with scale
// 2^13 - 1.  Decode: masking the exponent bits leaves 4 q_k in each half, which
// the hardware halfword conversion turns into an exact float; the scale is
// then 2^(E-129) (a subnormal power of two for E < 3, still exact).
template <>
struct Spinor<S_INT14> {
    static constexpr int chunks = 1;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
        const uint2 a = ld_cached(reinterpret_cast<const uint2 *>(b) + i);
        const uint32_t w = ld_cached(reinterpret_cast<const uint32_t *>(b + (size_t)8 * n) + i);
        c[0] = make_uint4(a.x, a.y, w, 0u);
    }
    __device__ static uint32_t exponent(const uint4 &w)
    {
        return (w.x & 3u) | ((w.x >> 14) & 0xcu) | ((w.y & 3u) << 4) | ((w.y >> 10) & 0xc0u);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
        const uint4 w = c[0];
        const uint32_t E = exponent(w);
        const float up = __uint_as_float(E >= 3u ? (E - 2u) << 23 : E == 2u ? 0x00400000u : 0x00200000u);
        const uint32_t m0 = w.x & 0xfffcfffcu, m1 = w.y & 0xfffcfffcu, m2 = w.z & 0xfffcfffcu;
        const float q[6] = {i16lo_to_f(m0), i16hi_to_f(m0), i16lo_to_f(m1),
                            i16hi_to_f(m1), i16lo_to_f(m2), i16hi_to_f(m2)};
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = (real)fmul(q[k], up);
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        float f[6];
        float mx = 0.0f;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            f[k] = (float)v[k];
            ok = ok && isfinite(f[k]);
            mx = fmaxf(mx, fabsf(f[k]));
        }
        uint32_t h[6] = {0, 0, 0, 0, 0, 0};
        uint32_t E = 1;
        if (ok) {
            const float t = __fdiv_rn(mx, 8191.0f);
            E = ((__float_as_uint(t) >> 23) & 0xffu) + 1u;
            const float down = __uint_as_float((254u - E) << 23);
#pragma unroll
            for (int k = 0; k < 6; k++) h[k] = ((uint32_t)__float2int_rn(fmul(f[k], down)) & 0x3fffu) << 2;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) h[k] |= (E >> (2 * k)) & 3u;
        reinterpret_cast<uint2 *>(b)[i] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        reinterpret_cast<uint32_t *>(b + (size_t)8 * n)[i] = h[4] | (h[5] << 16);
        return ok;
    }
};

// 30-bit shared exponent (our layout of Listing 3): words k < 6 hold q_k in
// bits 0..29, bits 30..31 of words 0..3 hold exponent bits 2k..2k+1.  Encode
// in FP64: t = max/(2^29-1), 2^(E-127) the power of two just above t.
template <>
struct Spinor<S_INT30> {
    static constexpr int chunks = 2;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
        c[0] = ld_cached(reinterpret_cast<const uint4 *>(b) + i);
        const uint2 t = ld_cached(reinterpret_cast<const uint2 *>(b + (size_t)16 * n) + i);
        c[1] = make_uint4(t.x, t.y, 0u, 0u);
    }
    // the six integers and the exponent field of a gathered record
    __device__ static uint32_t raw(const uint4 c[chunks], int32_t q[6])
    {
        const uint4 a = c[0];
        q[0] = sext_bits(a.x, 30); q[1] = sext_bits(a.y, 30); q[2] = sext_bits(a.z, 30);
        q[3] = sext_bits(a.w, 30); q[4] = sext_bits(c[1].x, 30); q[5] = sext_bits(c[1].y, 30);
        return (a.x >> 30) | ((a.y >> 30) << 2) | ((a.z >> 30) << 4) | ((a.w >> 30) << 6);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
        int32_t q[6];
        const uint32_t E = raw(c, q);
        if constexpr (is_ff<real>::value) {  // exact: q as an FP32 pair, times a power of two
            const float up = __uint_as_float(E << 23);
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = ff_scale(ff_from_int(q[k]), up);
        } else if constexpr (sizeof(real) == 8) {
            const double up = __longlong_as_double((long long)(E + 896u) << 52);  // 2^(E-127)
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = __dmul_rn((double)q[k], up);
        } else {
            const float up = __uint_as_float(E << 23);
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = fmul(__int2float_rn(q[k]), up);
        }
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    // FP32 values, the same bits as the FP64 rule without FP64 arithmetic: for
    // a site maximum mx = m 2^(f-127) (f its exponent field, m < 2 - 2^-23)
    // the FP64 quotient mx/(2^29-1) = m (1 + 1/(2^29-1)) 2^(f-156) stays below
    // 2^(f-155) (m (1 + 2^-29) < 2 - 2^-53), so its exponent gives E = f - 28
    // (subnormal or small mx: E = 1); v 2^(127-E) is then exact in FP32 (a
    // power of two, magnitude below 2^29) and rounds to the same integer.
    __device__ static bool store_f32(char *b, int n, int i, const float v[6])
    {
        float mx = 0.0f;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ok = ok && isfinite(v[k]);
            mx = fmaxf(mx, fabsf(v[k]));
        }
        uint32_t E = 1;
        uint32_t u[6] = {0, 0, 0, 0, 0, 0};
        if (ok) {
            const int f = (int)((__float_as_uint(mx) >> 23) & 0xffu);
            E = (uint32_t)(f > 29 ? f - 28 : 1);
            // 2^(127-E), E in [1, 226]: a normal FP32 power of two
            const float down = __uint_as_float((254u - E) << 23);
#pragma unroll
            for (int k = 0; k < 6; k++) u[k] = (uint32_t)__float2int_rn(fmul(v[k], down));
        }
        pack(b, n, i, E, u);
        return ok;
    }

    // FP32-pair values (FP64-class compute), the 30-bit rule on the exact value
    // hi + lo without FP64 arithmetic.  Exponent: as store_f32 from hi's
    // exponent field f (E = f - 28), except that a power-of-two hi with an
    // opposite-sign lo larger than 2^(p-29) (p the exponent of hi) lies in
    // the binade below (E = f - 29).  Integer: round-to-nearest-even of the
    // scaled pair, exactly: r = rint(hi'), then the exact remainder
    // (hi' - r) + lo' (TwoSum) rounded the same way in a second stage.
    __device__ static bool store_ff(char *b, int n, int i, const ff v[6])
    {
        uint32_t u[6], E;
        return store_ff_q(b, n, i, v, u, E);
    }
    // the same, returning the stored integers (signed, in u) and exponent field
    __device__ static bool store_ff_q(char *b, int n, int i, const ff v[6], uint32_t u[6], uint32_t &E)
    {
        bool ok = true;
        int km = 0;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ok = ok && isfinite(v[k].hi) && isfinite(v[k].lo);
            // the larger magnitude: |hi|, then the lo with hi's sign
            const float a = fabsf(v[k].hi), am = fabsf(v[km].hi);
            const float l = copysignf(1.0f, v[k].hi) * v[k].lo, lm = copysignf(1.0f, v[km].hi) * v[km].lo;
            if (a > am || (a == am && l > lm)) km = k;
        }
        E = 1;
#pragma unroll
        for (int k = 0; k < 6; k++) u[k] = 0;
        if (ok) {
            const ff m = v[km];
            const uint32_t bits = __float_as_uint(fabsf(m.hi));
            const int f = (int)(bits >> 23);
            int e = f - 28;
            if ((bits & 0x7fffffu) == 0u && f > 0 && m.lo != 0.0f && ((m.lo < 0.0f) != (m.hi < 0.0f))) {
                const float thr = f >= 30 ? __uint_as_float((uint32_t)(f - 29) << 23) : 0.0f;  // 2^(p-29)
                if (fabsf(m.lo) > thr) e -= 1;
            }
            E = (uint32_t)(e > 1 ? e : 1);
            const float down = __uint_as_float((254u - E) << 23);  // 2^(127-E)
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float xh = fmul(v[k].hi, down), xl = fmul(v[k].lo, down);
                const float r = rintf(xh);
                const ff se = ff_two_sum(__fsub_rn(xh, r), xl);  // exact remainder
                const float kk = rintf(se.hi);
                const ff uw = ff_two_sum(__fsub_rn(se.hi, kk), se.lo);
                int q = __float2int_rn(r) + __float2int_rn(kk);
                if (uw.hi > 0.5f || (uw.hi == 0.5f && uw.lo > 0.0f))
                    q += 1;
                else if (uw.hi < -0.5f || (uw.hi == -0.5f && uw.lo < 0.0f))
                    q -= 1;
                else if (uw.lo == 0.0f && (uw.hi == 0.5f || uw.hi == -0.5f) && (q & 1))
                    q += uw.hi > 0.0f ? 1 : -1;  // a tie: to the even neighbour
                u[k] = (uint32_t)q;
            }
        }
        pack(b, n, i, E, u);
        return ok;
    }

    __device__ static void pack(char *b, int n, int i, uint32_t E, const uint32_t u[6])
    {
        uint4 a;
        a.x = (u[0] & 0x3fffffffu) | ((E & 3u) << 30);
        a.y = (u[1] & 0x3fffffffu) | (((E >> 2) & 3u) << 30);
        a.z = (u[2] & 0x3fffffffu) | (((E >> 4) & 3u) << 30);
        a.w = (u[3] & 0x3fffffffu) | (((E >> 6) & 3u) << 30);
        reinterpret_cast<uint4 *>(b)[i] = a;
        reinterpret_cast<uint2 *>(b + (size_t)16 * n)[i] = make_uint2(u[4] & 0x3fffffffu, u[5] & 0x3fffffffu);
    }

    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        if constexpr (std::is_same<real, float>::value) return store_f32(b, n, i, v);
        if constexpr (is_ff<real>::value) return store_ff(b, n, i, v);
        double d[6];
        double mx = 0.0;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            d[k] = (double)v[k];
            ok = ok && isfinite(d[k]);
            mx = fmax(mx, fabs(d[k]));
        }
        uint32_t E = 1;
        uint32_t u[6] = {0, 0, 0, 0, 0, 0};
        if (ok) {
            const double t = __ddiv_rn(mx, 536870911.0);
            const int biased = (int)((__double_as_longlong(t) >> 52) & 0x7ff);
            int e = (t > 0.0 && biased > 0) ? biased - 895 : 1;  // frexp exponent + 127
            if (e < 1) e = 1;
            if (e > 254) ok = false;
            if (ok) {
                E = (uint32_t)e;
                const double down = __longlong_as_double((long long)(1150 - e) << 52);  // 2^-(E-127)
#pragma unroll
                for (int k = 0; k < 6; k++) u[k] = (uint32_t)(int32_t)__double2ll_rn(__dmul_rn(d[k], down));
            }
        }
        pack(b, n, i, E, u);
        return ok;
    }
};

// ---------------------------------------------------------------------------
// link codecs (read-only in the stencil; written by the gauge loader)
// ---------------------------------------------------------------------------
// Row 2 of a compressed link: sign * conj(row0 x row1) (SU(3) up to a sign).
template <typename real>
__device__ __forceinline__ void rebuild_row2(real U[18], real sign)
{
    // U[2k], U[2k+1]: re, im of element k = 3*row + col
#define RE(k) U[2 * (k)]
#define IM(k) U[2 * (k) + 1]
    const real c0r = RE(1) * RE(5) - IM(1) * IM(5) - (RE(2) * RE(4) - IM(2) * IM(4));
    const real c0i = RE(1) * IM(5) + IM(1) * RE(5) - (RE(2) * IM(4) + IM(2) * RE(4));
    const real c1r = RE(2) * RE(3) - IM(2) * IM(3) - (RE(0) * RE(5) - IM(0) * IM(5));
    const real c1i = RE(2) * IM(3) + IM(2) * RE(3) - (RE(0) * IM(5) + IM(0) * RE(5));
    const real c2r = RE(0) * RE(4) - IM(0) * IM(4) - (RE(1) * RE(3) - IM(1) * IM(3));
    const real c2i = RE(0) * IM(4) + IM(0) * RE(4) - (RE(1) * IM(3) + IM(1) * RE(3));
    RE(6) = sign * c0r; IM(6) = -sign * c0i;
    RE(7) = sign * c1r; IM(7) = -sign * c1i;
    RE(8) = sign * c2r; IM(8) = -sign * c2i;
#undef RE
#undef IM
}

// Fixed-point links are returned unscaled: the integers q as exact reals.
// Their scale gmax/qmax is one number per field, so the stencil multiplies
// each field's accumulated sum by it once instead of every element.
template <int GF>
struct LinkScaled {
    static constexpr bool value = GF == G_FIX16 || GF == G_FIX32;
};

// FP32 pairs, three 16-byte planes of (hi, lo, hi, lo): the accumulators of
// FP64-class (pair) kernels, read and written without conversion.
template <>
struct Spinor<S_FF> {
    static constexpr int chunks = 3;
    __device__ static void gather(const char *b, int n, int i, uint4 c[chunks])
    {
#pragma unroll
        for (int k = 0; k < 3; k++) c[k] = ld_cached(reinterpret_cast<const uint4 *>(b) + (size_t)k * n + i);
    }
    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real v[6])
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const ff a(__uint_as_float(c[k].x), __uint_as_float(c[k].y));
            const ff b(__uint_as_float(c[k].z), __uint_as_float(c[k].w));
            if constexpr (is_ff<real>::value) {
                v[2 * k] = a;
                v[2 * k + 1] = b;
            } else {
                v[2 * k] = (real)(double)a;
                v[2 * k + 1] = (real)(double)b;
            }
        }
    }
    template <typename real>
    __device__ static void load(const char *b, int n, int i, real v[6])
    {
        uint4 c[chunks];
        gather(b, n, i, c);
        decode(c, v);
    }
    template <typename real>
    __device__ static bool store(char *b, int n, int i, const real v[6])
    {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            ff a, bb;
            if constexpr (is_ff<real>::value) {
                a = v[2 * k];
                bb = v[2 * k + 1];
            } else {
                a = ff((double)v[2 * k]);
                bb = ff((double)v[2 * k + 1]);
            }
            ok = ok && isfinite(a.hi) && isfinite(bb.hi);
            reinterpret_cast<uint4 *>(b)[(size_t)k * n + i] =
                make_uint4(__float_as_uint(a.hi), __float_as_uint(a.lo), __float_as_uint(bb.hi), __float_as_uint(bb.lo));
        }
        return ok;
    }
};

// A spinor record read through L2 only (ld.global.cg): for fields that other
// blocks of the same kernel write (the read-only path may not be used there).
// Same planar layout as Spinor<SF>::gather.
template <int SF>
__device__ __forceinline__ void gather_coherent(const char *b, int n, int i, uint4 c[Spinor<SF>::chunks])
{
    if constexpr (SF == S_INT14) {
        const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(b) + i);
        c[0] = make_uint4(a.x, a.y, __ldcg(reinterpret_cast<const uint32_t *>(b + (size_t)8 * n) + i), 0u);
        return;
    }
    constexpr int n16 = spinor_n16(SF), tail = spinor_tail(SF);
#pragma unroll
    for (int k = 0; k < n16; k++) c[k] = __ldcg(reinterpret_cast<const uint4 *>(b + (size_t)k * 16 * n) + i);
    if constexpr (tail == 8) {
        const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(b + (size_t)n16 * 16 * n) + i);
        c[n16] = make_uint4(t.x, t.y, 0u, 0u);
    }
}

// Row 2 of a 13-real link: f * conj(row0 x row1) with the complex factor
// f = (fr, fi) (the det phase e^{i pi t}, times the fixed-point scale).
template <typename real>
__device__ __forceinline__ void rebuild_row2_phase(real U[18], real fr, real fi)
{
#define RE(k) U[2 * (k)]
#define IM(k) U[2 * (k) + 1]
    const real c0r = RE(1) * RE(5) - IM(1) * IM(5) - (RE(2) * RE(4) - IM(2) * IM(4));
    const real c0i = RE(1) * IM(5) + IM(1) * RE(5) - (RE(2) * IM(4) + IM(2) * RE(4));
    const real c1r = RE(2) * RE(3) - IM(2) * IM(3) - (RE(0) * RE(5) - IM(0) * IM(5));
    const real c1i = RE(2) * IM(3) + IM(2) * RE(3) - (RE(0) * IM(5) + IM(0) * RE(5));
    const real c2r = RE(0) * RE(4) - IM(0) * IM(4) - (RE(1) * RE(3) - IM(1) * IM(3));
    const real c2i = RE(0) * IM(4) + IM(0) * RE(4) - (RE(1) * IM(3) + IM(1) * RE(3));
    RE(6) = fr * c0r + fi * c0i; IM(6) = fi * c0r - fr * c0i;
    RE(7) = fr * c1r + fi * c1i; IM(7) = fi * c1r - fr * c1i;
    RE(8) = fr * c2r + fi * c2i; IM(8) = fi * c2r - fr * c2i;
#undef RE
#undef IM
}

template <int GF, int RECON>
struct Link {
    static constexpr int n16 = link_n16(GF, RECON);
    static constexpr int tail = link_tail(GF, RECON);
    static constexpr int rows = link_rows_reals(RECON);  // reals in the row planes
    static constexpr bool kPhase = RECON == 13;           // a phase plane after the tail plane
    static constexpr int row_chunks = n16 + (tail ? 1 : 0);  // the tail chunk holds its 4 or 8 bytes first
    static constexpr int chunks = row_chunks + (kPhase ? 1 : 0);  // the phase chunk holds its real first

    // li = (parity*4 + mu)*Vh + cb; pstride = bytes of one plane (8*Vh*16).
    // Links are read once per pass: evict-first loads, unless KEEP (a link
    // that the same kernel applies again soon: normal priority in L2).
    template <bool KEEP = false>
    __device__ static void gather(const char *base, size_t pstride, int li, uint4 c[chunks])
    {
        auto ld = [](const auto *p) { return KEEP ? ld_cached(p) : ld_stream(p); };
#pragma unroll
        for (int k = 0; k < n16; k++) c[k] = ld(reinterpret_cast<const uint4 *>(base + k * pstride) + li);
        if constexpr (tail == 4) {
            c[n16] = make_uint4(ld(reinterpret_cast<const unsigned int *>(base + n16 * pstride) + li), 0u, 0u, 0u);
        } else if constexpr (tail == 8) {
            const uint2 t = ld(reinterpret_cast<const uint2 *>(base + n16 * pstride) + li);
            c[n16] = make_uint4(t.x, t.y, 0u, 0u);
        }
        if constexpr (kPhase) {
            // phase plane: after the tail plane (tail bytes per link), one real per link
            const char *pp = base + n16 * pstride + (size_t)tail * (pstride / 16);
            if constexpr (gauge_real_bytes(GF) == 2) {
                c[row_chunks] = make_uint4((unsigned)ld(reinterpret_cast<const unsigned short *>(pp) + li), 0u, 0u, 0u);
            } else if constexpr (gauge_real_bytes(GF) == 4) {
                c[row_chunks] = make_uint4(ld(reinterpret_cast<const unsigned int *>(pp) + li), 0u, 0u, 0u);
            } else {
                const uint2 t = ld(reinterpret_cast<const uint2 *>(pp) + li);
                c[row_chunks] = make_uint4(t.x, t.y, 0u, 0u);
            }
        }
    }

    // The stored phase of a 13-real link as a fraction t of pi (t in [-1, 1]).
    template <typename real>
    __device__ static real phase(const uint4 c[chunks])
    {
        static_assert(kPhase, "13-real links only");
        const uint4 w = c[row_chunks];
        if constexpr (GF == G_F64) {
            return (real)__hiloint2double((int)w.y, (int)w.x);
        } else if constexpr (GF == G_F32) {
            return (real)__uint_as_float(w.x);
        } else if constexpr (GF == G_FIX16) {
            return (real)__fmul_rn(__int2float_rn((int)(short)(w.x & 0xffffu)), 1.0f / 32767.0f);
        } else {
            return (real)((double)(int)w.x * (1.0 / 2147483647.0));
        }
    }

    template <typename real>
    __device__ static void decode(const uint4 c[chunks], real U[18])
    {
        if constexpr (GF == G_F64) {
#pragma unroll
            for (int k = 0; k < rows / 2; k++) {
                U[2 * k] = (real)__hiloint2double((int)c[k].y, (int)c[k].x);
                U[2 * k + 1] = (real)__hiloint2double((int)c[k].w, (int)c[k].z);
            }
        } else if constexpr (GF == G_F32) {
#pragma unroll
            for (int k = 0; k < n16; k++) {
                U[4 * k] = __uint_as_float(c[k].x); U[4 * k + 1] = __uint_as_float(c[k].y);
                U[4 * k + 2] = __uint_as_float(c[k].z); U[4 * k + 3] = __uint_as_float(c[k].w);
            }
            if constexpr (tail == 8) {
                U[4 * n16] = __uint_as_float(c[n16].x);
                U[4 * n16 + 1] = __uint_as_float(c[n16].y);
            }
        } else if constexpr (GF == G_FIX16 || GF == G_SE15) {
            uint32_t w[rows / 2];
#pragma unroll
            for (int k = 0; k < n16; k++) {
                w[4 * k] = c[k].x; w[4 * k + 1] = c[k].y; w[4 * k + 2] = c[k].z; w[4 * k + 3] = c[k].w;
            }
            if constexpr (tail == 4) {
                w[4 * n16] = c[n16].x;
            } else if constexpr (tail == 8) {
                w[4 * n16] = c[n16].x;
                w[4 * n16 + 1] = c[n16].y;
            }
            if constexpr (GF == G_SE15) {
                // exponent bit k in the low bit of half k (k < 8); masked, each half is 2 q_k, exact
                // in FP32, and the value q_k 2^(E-127) = (2 q_k) 2^(E-128) (subnormal scale for E = 1)
                const uint32_t E = (w[0] & 1u) | ((w[0] >> 15) & 2u) | ((w[1] & 1u) << 2) | ((w[1] >> 13) & 8u) |
                                   ((w[2] & 1u) << 4) | ((w[2] >> 11) & 32u) | ((w[3] & 1u) << 6) |
                                   ((w[3] >> 9) & 128u);
                const float sc = __uint_as_float(E >= 2u ? (E - 1u) << 23 : E == 1u ? 0x00400000u : 0u);
#pragma unroll
                for (int k = 0; k < rows / 2; k++) {
                    const uint32_t m = w[k] & 0xfffefffeu;
                    U[2 * k] = fmul(i16lo_to_f(m), sc);
                    U[2 * k + 1] = fmul(i16hi_to_f(m), sc);
                }
            } else {
#pragma unroll
                for (int k = 0; k < rows / 2; k++) {
                    if constexpr (sizeof(real) == 8) {
                        U[2 * k] = (double)(int)(short)(w[k] & 0xffffu);
                        U[2 * k + 1] = (double)((int)w[k] >> 16);
                    } else {
                        U[2 * k] = i16lo_to_f(w[k]);
                        U[2 * k + 1] = i16hi_to_f(w[k]);
                    }
                }
            }
        } else {  // G_FIX32
            int q[rows];
#pragma unroll
            for (int k = 0; k < n16; k++) {
                q[4 * k] = (int)c[k].x; q[4 * k + 1] = (int)c[k].y; q[4 * k + 2] = (int)c[k].z; q[4 * k + 3] = (int)c[k].w;
            }
            if constexpr (tail == 8) {
                q[4 * n16] = (int)c[n16].x;
                q[4 * n16 + 1] = (int)c[n16].y;
            }
#pragma unroll
            for (int k = 0; k < rows; k++) {
                if constexpr (is_ff<real>::value)
                    U[k] = ff_from_int(q[k]);
                else if constexpr (sizeof(real) == 8)
                    U[k] = (double)q[k];
                else
                    U[k] = __int2float_rn(q[k]);
            }
        }
    }

    // decoded rows; for the 13-real format U[12] receives the phase (the
    // caller rebuilds row 2 over it)
    template <typename real, bool KEEP = false>
    __device__ static void load(const char *base, size_t pstride, int li, real U[18])
    {
        uint4 c[chunks];
        gather<KEEP>(base, pstride, li, c);
        decode(c, U);
        if constexpr (kPhase) U[12] = phase<real>(c);
    }
};

}  // namespace hisq
