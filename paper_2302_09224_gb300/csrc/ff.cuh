// ff.cuh -- FP64-class arithmetic on the FP32 pipe: an unevaluated pair
// hi + lo of floats (|lo| <= ulp(hi)/2, about 48 significant bits), the
// "double-single" numbers of Dekker's and Knuth's error-free transformations:
//   TwoSum(a, b):      s = fl(a + b), e = (a - (s - bb)) + (b - bb), bb = s - a
//   FastTwoSum(a, b):  s = fl(a + b), e = b - (s - a)          (|a| >= |b|)
//   TwoProd(a, b):     p = fl(a b),   e = fma(a, b, -p)
// On GB300 the FP64 pipe issues a small fraction of the FP32 rate, so the
// compute precision of the 30-bit storage triplet (FP64 in the paper, Sec. 4)
// is carried by these pairs: their rounding (~2^-47 relative per operation)
// stays far below the 2^-29 of the 30-bit storage.
#pragma once

#include <cuda_runtime.h>

namespace hisq {

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(float x) : hi(x), lo(0.0f) {}
    __host__ __device__ constexpr ff(int x) : hi((float)x), lo(0.0f) {}  // small integers only (exact)
    __device__ explicit ff(double d)
    {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b)
{
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b)
{
    // two Newton-style quotient digits: q1 = a/b rounded, q2 = (a - q1 b)/b
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = a - b * ff(q1);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }
__device__ __forceinline__ ff &operator*=(ff &a, ff b) { return a = a * b; }

// An integer below 2^31 in magnitude as an exact pair: q = qh 2^16 + ql with
// qh and ql exact in FP32, summed error-free.
__device__ __forceinline__ ff ff_from_int(int q)
{
    const int qh = q >> 16;       // arithmetic shift: q = qh * 65536 + ql, 0 <= ql < 65536
    const int ql = q & 0xffff;
    return ff_two_sum(__fmul_rn(__int2float_rn(qh), 65536.0f), __int2float_rn(ql));
}

// Scale by a power of two given as a float (exact while the result is normal).
__device__ __forceinline__ ff ff_scale(ff a, float pow2) { return ff(__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)); }

// a 2^e for |e| <= 252, in two exact steps of at most 2^126 each
__device__ __forceinline__ ff ff_ldexp(ff a, int e)
{
    const int e1 = e >> 1, e2 = e - e1;
    return ff_scale(ff_scale(a, __uint_as_float((uint32_t)(e1 + 127) << 23)),
                    __uint_as_float((uint32_t)(e2 + 127) << 23));
}

// A 64-bit integer as a pair, on the FP32 and integer pipes only (the 64-bit
// conversion instructions run on GB300's narrow FP64 pipe): P = c2 2^42 +
// c1 2^21 + c0 with c2 the arithmetic top 22 bits and c1, c0 21-bit fields,
// each exact in FP32 (the field placed in the mantissa of 2^23, or of 2^23 +
// 2^22 for the signed one, and the offset subtracted), scaled by exact powers
// of two; the top two summed error-free, the low one added to the tail (about
// 45 significant bits or more, like any pair).
__device__ __forceinline__ ff ff_from_ll(long long P)
{
    const unsigned lo = (unsigned)P, hi = (unsigned)((unsigned long long)P >> 32);
    const unsigned c0 = lo & 0x1FFFFFu;
    const unsigned c1 = __funnelshift_r(lo, hi, 21) & 0x1FFFFFu;
    const int c2 = (int)hi >> 10;  // bits 42..63 with the sign: |c2| <= 2^21
    const float f0 = __fsub_rn(__uint_as_float(0x4B000000u | c0), 8388608.0f);
    const float f1 = __fmul_rn(__fsub_rn(__uint_as_float(0x4B000000u | c1), 8388608.0f), 2097152.0f);
    const float f2 = __fmul_rn(__fsub_rn(__uint_as_float(0x4B000000u | (unsigned)(c2 + 0x400000)), 12582912.0f),
                               4398046511104.0f);
    const ff s = ff_two_sum(f2, f1);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, f0));
}

template <typename T>
struct is_ff {
    static constexpr bool value = false;
};
template <>
struct is_ff<ff> {
    static constexpr bool value = true;
};

}  // namespace hisq
