// convert.cu -- format conversion kernels: spinor pack/unpack between the
// caller's FP64 [site][6] layout and the storage formats, and the gauge
// loader's scale, compression check and quantisation passes.
#include <cuda_runtime.h>

#include <cstdint>

#include "codecs.cuh"
#include "internal.h"

namespace hisq {

namespace {

constexpr int kBlock = 256;

template <int SF>
__global__ void pack_kernel(int64_t n, const double *in, char *out, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = in[6 * i + k];
    if (!Spinor<SF>::store(out, (int)n, (int)i, v)) atomicAdd(bad, 1);
}

// FP32 input through the FP32 store (the one FP32-compute kernels use)
template <int SF>
__global__ void pack32_kernel(int64_t n, const float *in, char *out, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = in[6 * i + k];
    if (!Spinor<SF>::store(out, (int)n, (int)i, v)) atomicAdd(bad, 1);
}

// FP32-pair input [n][6][hi, lo] through the pair store (FP64-class kernels)
__global__ void pack_pair_kernel(int64_t n, const float *in, char *out, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ff v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ff(in[12 * i + 2 * k], in[12 * i + 2 * k + 1]);
    if (!Spinor<S_INT30>::store(out, (int)n, (int)i, v)) atomicAdd(bad, 1);
}

template <int SF, typename real>
__global__ void unpack_kernel(int64_t n, const char *in, double *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    real v[6];
    Spinor<SF>::load(in, (int)n, (int)i, v);
#pragma unroll
    for (int k = 0; k < 6; k++) out[6 * i + k] = (double)v[k];
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    // non-negative doubles order like their bit patterns (NaN sorts above Inf)
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void absmax_kernel(int64_t n, const double *x, double *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(x[i]);
        m = (a > m || a != a) ? a : m;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, m, off);
        m = (o > m || o != o) ? o : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

__device__ __forceinline__ void lex_coords(const Geom &g, int lex, int c[4])
{
    c[0] = lex % g.L[0];
    int r = lex / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
}

// Largest deviation of row 2 from sign * conj(row0 x row1) over all links of
// a field (k = 1 fat, k = 3 long): zero to rounding when the field can be
// stored as 12 reals (Sec. 1, 18 -> 12 compression).
__global__ void r12_check_kernel(Geom g, const double *links, int k, double *out)
{
    const int V = 2 * g.vh;
    double m = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < 4LL * V;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)(idx / V), lex = (int)(idx % V);
        int c[4];
        lex_coords(g, lex, c);
        int ps = 0;
        for (int nu = 0; nu < mu; nu++) ps += c[nu];
        double sign = (ps & 1) ? -1.0 : 1.0;
        if (g.antiperiodic_t && mu == 3 && c[3] + k >= g.L[3]) sign = -sign;
        double U[18];
        const double *src = links + idx * 18;
        for (int j = 0; j < 18; j++) U[j] = src[j];
        double R[18];
        for (int j = 0; j < 18; j++) R[j] = U[j];
        rebuild_row2(R, sign);
        for (int j = 12; j < 18; j++) {
            const double d = fabs(R[j] - U[j]);
            m = (d > m || d != d) ? d : m;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, m, off);
        m = (o > m || o != o) ? o : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// FP64 [mu][lex][18] -> stored copy [plane][parity][mu][Vh] in format GF with
// RECON reals per link.  Fixed point: q = rint(x * inv) clamped to +-qmax,
// inv = qmax / global max (Sec. 2 footnote; Sec. 4 for 32 bits).
template <int GF, int RECON>
__global__ void quantise_kernel(Geom g, const double *links, double inv, char *out)
{
    const int vh = g.vh;
    const int64_t n = 8LL * vh;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= n) return;
    const int cb = (int)(li % vh);
    const int pm = (int)(li / vh);
    const int par = pm >> 2, mu = pm & 3;
    int r = cb / g.xh;
    const int xh = cb - r * g.xh;
    const int y = r % g.L[1];
    r /= g.L[1];
    const int z = r % g.L[2];
    const int t = r / g.L[2];
    const int x = 2 * xh + ((y + z + t + par) & 1);
    const int lex = 2 * cb + (x & 1);
    const double *src = links + ((int64_t)mu * 2 * vh + lex) * 18;
    const size_t pstride = (size_t)n * 16;
    constexpr int n16 = link_n16(GF, RECON), tail = link_tail(GF, RECON);
    if constexpr (RECON == 8) {
        // 8 reals of V = sign U (V in SU(3); sign: the long link's staggered phase and boundary
        // sign): arg V00 / pi, arg V20 / pi, V01, V02, V10.  Angles are stored as the format
        // stores a real in [-1, 1] (fixed point: rint(t qmax)), elements as every other element.
        int ps = 0;
        const int cc[4] = {x, y, z, t};
        for (int nu = 0; nu < mu; nu++) ps += cc[nu];
        double sg = (ps & 1) ? -1.0 : 1.0;
        if (g.antiperiodic_t && mu == 3 && t + 3 >= g.L[3]) sg = -sg;
        const double inv_pi = 0.31830988618379067154;
        const double pv[8] = {atan2(sg * src[1], sg * src[0]) * inv_pi, atan2(sg * src[13], sg * src[12]) * inv_pi,
                              sg * src[2], sg * src[3], sg * src[4], sg * src[5], sg * src[6], sg * src[7]};
        if constexpr (GF == G_F64) {
            for (int k = 0; k < 4; k++)
                reinterpret_cast<double2 *>(out + k * pstride)[li] = make_double2(pv[2 * k], pv[2 * k + 1]);
        } else if constexpr (GF == G_F32) {
            for (int k = 0; k < 2; k++)
                reinterpret_cast<float4 *>(out + k * pstride)[li] =
                    make_float4((float)pv[4 * k], (float)pv[4 * k + 1], (float)pv[4 * k + 2], (float)pv[4 * k + 3]);
        } else {
            constexpr double qmax = GF == G_FIX16 ? 32767.0 : 2147483647.0;
            int q[8];
            for (int k = 0; k < 8; k++) {
                double v = rint(__dmul_rn(pv[k], k < 2 ? qmax : inv));
                q[k] = (int)fmin(qmax, fmax(-qmax, v));
            }
            if constexpr (GF == G_FIX16) {
                int4 w;
                w.x = (int)((q[0] & 0xffff) | ((uint32_t)q[1] << 16));
                w.y = (int)((q[2] & 0xffff) | ((uint32_t)q[3] << 16));
                w.z = (int)((q[4] & 0xffff) | ((uint32_t)q[5] << 16));
                w.w = (int)((q[6] & 0xffff) | ((uint32_t)q[7] << 16));
                reinterpret_cast<int4 *>(out)[li] = w;
            } else {
                reinterpret_cast<int4 *>(out)[li] = make_int4(q[0], q[1], q[2], q[3]);
                reinterpret_cast<int4 *>(out + pstride)[li] = make_int4(q[4], q[5], q[6], q[7]);
            }
        }
        return;
    }
    if constexpr (GF == G_F64) {
        for (int k = 0; k < RECON / 2; k++)
            reinterpret_cast<double2 *>(out + k * pstride)[li] = make_double2(src[2 * k], src[2 * k + 1]);
    } else if constexpr (GF == G_F32) {
        for (int k = 0; k < n16; k++)
            reinterpret_cast<float4 *>(out + k * pstride)[li] =
                make_float4((float)src[4 * k], (float)src[4 * k + 1], (float)src[4 * k + 2], (float)src[4 * k + 3]);
        if constexpr (tail == 8)
            reinterpret_cast<float2 *>(out + n16 * pstride)[li] =
                make_float2((float)src[4 * n16], (float)src[4 * n16 + 1]);
    } else if constexpr (GF == G_SE15) {
        // per link: 15-bit integers with one exponent, the 30-bit rule in FP64 with scale 2^14 - 1
        // (t = max |x| / (2^14 - 1), 2^(E-127) the power of two just above t); half k = q_k << 1 | bit k
        // of E (k < 8); a link whose exponent does not fit is stored as zero with E = 1
        double mx = 0.0;
        bool ok = true;
        for (int k = 0; k < RECON; k++) {
            ok = ok && isfinite(src[k]);
            mx = fmax(mx, fabs(src[k]));
        }
        const double tq = mx / 16383.0;
        int ex = 0;
        if (tq > 0.0) frexp(tq, &ex);
        int E = tq > 0.0 ? ex + 127 : 1;
        if (E < 1) E = 1;
        if (E > 254) ok = false;
        if (!ok) E = 1;
        uint32_t h[RECON];
        for (int k = 0; k < RECON; k++) {
            const int q = ok ? (int)rint(ldexp(src[k], -(E - 127))) : 0;
            h[k] = (((uint32_t)q & 0x7fffu) << 1) | (k < 8 ? ((uint32_t)E >> k) & 1u : 0u);
        }
        for (int k = 0; k < n16; k++)
            reinterpret_cast<uint4 *>(out + k * pstride)[li] =
                make_uint4(h[8 * k] | (h[8 * k + 1] << 16), h[8 * k + 2] | (h[8 * k + 3] << 16),
                           h[8 * k + 4] | (h[8 * k + 5] << 16), h[8 * k + 6] | (h[8 * k + 7] << 16));
        if constexpr (tail == 4)
            reinterpret_cast<uint32_t *>(out + n16 * pstride)[li] = h[8 * n16] | (h[8 * n16 + 1] << 16);
        else if constexpr (tail == 8)
            reinterpret_cast<uint2 *>(out + n16 * pstride)[li] =
                make_uint2(h[8 * n16] | (h[8 * n16 + 1] << 16), h[8 * n16 + 2] | (h[8 * n16 + 3] << 16));
    } else {
        constexpr double qmax = GF == G_FIX16 ? 32767.0 : 2147483647.0;
        int q[RECON];
        for (int k = 0; k < RECON; k++) {
            double v = rint(__dmul_rn(src[k], inv));
            v = fmin(qmax, fmax(-qmax, v));
            q[k] = (int)v;
        }
        if constexpr (GF == G_FIX16) {
            for (int k = 0; k < n16; k++) {
                int4 w;
                w.x = (int)((q[8 * k] & 0xffff) | ((uint32_t)q[8 * k + 1] << 16));
                w.y = (int)((q[8 * k + 2] & 0xffff) | ((uint32_t)q[8 * k + 3] << 16));
                w.z = (int)((q[8 * k + 4] & 0xffff) | ((uint32_t)q[8 * k + 5] << 16));
                w.w = (int)((q[8 * k + 6] & 0xffff) | ((uint32_t)q[8 * k + 7] << 16));
                reinterpret_cast<int4 *>(out + k * pstride)[li] = w;
            }
            if constexpr (tail == 4) {
                reinterpret_cast<int *>(out + n16 * pstride)[li] =
                    (int)((q[8 * n16] & 0xffff) | ((uint32_t)q[8 * n16 + 1] << 16));
            } else if constexpr (tail == 8) {
                reinterpret_cast<int2 *>(out + n16 * pstride)[li] =
                    make_int2((int)((q[8 * n16] & 0xffff) | ((uint32_t)q[8 * n16 + 1] << 16)),
                              (int)((q[8 * n16 + 2] & 0xffff) | ((uint32_t)q[8 * n16 + 3] << 16)));
            }
        } else {
            for (int k = 0; k < n16; k++)
                reinterpret_cast<int4 *>(out + k * pstride)[li] =
                    make_int4(q[4 * k], q[4 * k + 1], q[4 * k + 2], q[4 * k + 3]);
            if constexpr (tail == 8)
                reinterpret_cast<int2 *>(out + n16 * pstride)[li] = make_int2(q[4 * n16], q[4 * n16 + 1]);
        }
    }
    if constexpr (RECON == 13) {
        // the 13th real: arg det U as a fraction of pi (row 2 = det(U) conj(row0 x row1) for unitary U)
        double u[18];
        for (int k = 0; k < 18; k++) u[k] = src[k];
        auto mre = [&](int i, int j) { return u[2 * (3 * i + j)]; };
        auto mim = [&](int i, int j) { return u[2 * (3 * i + j) + 1]; };
        auto cof = [&](int a, int b, int c, int d, double &r, double &im) {  // m(1,a) m(2,b) - m(1,c) m(2,d)
            r = mre(1, a) * mre(2, b) - mim(1, a) * mim(2, b) - (mre(1, c) * mre(2, d) - mim(1, c) * mim(2, d));
            im = mre(1, a) * mim(2, b) + mim(1, a) * mre(2, b) - (mre(1, c) * mim(2, d) + mim(1, c) * mre(2, d));
        };
        double c0r, c0i, c1r, c1i, c2r, c2i;
        cof(1, 2, 2, 1, c0r, c0i);
        cof(2, 0, 0, 2, c1r, c1i);
        cof(0, 1, 1, 0, c2r, c2i);
        const double dr = mre(0, 0) * c0r - mim(0, 0) * c0i + mre(0, 1) * c1r - mim(0, 1) * c1i + mre(0, 2) * c2r -
                          mim(0, 2) * c2i;
        const double di = mre(0, 0) * c0i + mim(0, 0) * c0r + mre(0, 1) * c1i + mim(0, 1) * c1r + mre(0, 2) * c2i +
                          mim(0, 2) * c2r;
        const double t = atan2(di, dr) * 0.31830988618379067154;  // 1/pi
        char *pp = out + n16 * pstride + (size_t)tail * n;
        if constexpr (GF == G_F64)
            reinterpret_cast<double *>(pp)[li] = t;
        else if constexpr (GF == G_F32)
            reinterpret_cast<float *>(pp)[li] = (float)t;
        else if constexpr (GF == G_FIX16)
            reinterpret_cast<short *>(pp)[li] = (short)rint(t * 32767.0);
        else
            reinterpret_cast<int *>(pp)[li] = (int)rint(t * 2147483647.0);
    }
}

// Error of the long links of a field stored with 8 reals, |U_stored - U| per
// real: the largest (out[0]) and the sum of squares (out[1]).  The stored
// parameters are decoded and V rebuilt in FP64 (the device rebuilds in the
// compute precision), so the result is the storage's own error, amplified
// where the rebuild is ill-conditioned (N = 1 - |V00|^2 or |V20| small).
// el: the element scale (gmax/qmax or 1), an: the angle scale (1/qmax or 1).
template <int GF>
__global__ void r8_check_kernel(Geom g, const double *links, const char *stored, double el, double an, double *out)
{
    const int vh = g.vh;
    const int64_t n = 8LL * vh;
    const size_t pstride = (size_t)n * 16;
    double m = 0.0, q = 0.0;
    for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < n; li += (int64_t)gridDim.x * blockDim.x) {
        const int cb = (int)(li % vh);
        const int pm = (int)(li / vh);
        const int par = pm >> 2, mu = pm & 3;
        int r = cb / g.xh;
        const int xh = cb - r * g.xh;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((y + z + t + par) & 1);
        const int lex = 2 * cb + (x & 1);
        const double *src = links + ((int64_t)mu * 2 * vh + lex) * 18;
        int ps = 0;
        const int cc[4] = {x, y, z, t};
        for (int nu = 0; nu < mu; nu++) ps += cc[nu];
        double sg = (ps & 1) ? -1.0 : 1.0;
        if (g.antiperiodic_t && mu == 3 && t + 3 >= g.L[3]) sg = -sg;
        double p[8];
        if constexpr (GF == G_F64) {
            for (int k = 0; k < 4; k++) {
                const double2 v = reinterpret_cast<const double2 *>(stored + k * pstride)[li];
                p[2 * k] = v.x;
                p[2 * k + 1] = v.y;
            }
        } else if constexpr (GF == G_F32) {
            for (int k = 0; k < 2; k++) {
                const float4 v = reinterpret_cast<const float4 *>(stored + k * pstride)[li];
                p[4 * k] = v.x; p[4 * k + 1] = v.y; p[4 * k + 2] = v.z; p[4 * k + 3] = v.w;
            }
        } else if constexpr (GF == G_FIX16) {
            const int4 w = reinterpret_cast<const int4 *>(stored)[li];
            const int ws[4] = {w.x, w.y, w.z, w.w};
            for (int k = 0; k < 4; k++) {
                p[2 * k] = (double)(short)(ws[k] & 0xffff);
                p[2 * k + 1] = (double)(ws[k] >> 16);
            }
        } else {
            const int4 a = reinterpret_cast<const int4 *>(stored)[li], b = reinterpret_cast<const int4 *>(stored + pstride)[li];
            p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w; p[4] = b.x; p[5] = b.y; p[6] = b.z; p[7] = b.w;
        }
        const double t1 = p[0] * an, t2 = p[1] * an;
        const double a2r = p[2] * el, a2i = p[3] * el, a3r = p[4] * el, a3i = p[5] * el, b1r = p[6] * el, b1i = p[7] * el;
        const double N = a2r * a2r + a2i * a2i + a3r * a3r + a3i * a3i;
        const double ra = sqrt(fmax(1.0 - N, 0.0)), rc = sqrt(fmax(N - b1r * b1r - b1i * b1i, 0.0));
        double s1, c1, s2, c2;
        sincospi(t1, &s1, &c1);
        sincospi(t2, &s2, &c2);
        const double a1r = ra * c1, a1i = ra * s1, cr = rc * c2, ci = rc * s2;
        // b2 = -(conj(a1) a2 b1 + conj(a3) conj(c1)) / N, b3 = (conj(a2) conj(c1) - conj(a1) a3 b1) / N
        const double a1a2r = a1r * a2r + a1i * a2i, a1a2i = a1r * a2i - a1i * a2r;    // conj(a1) a2
        const double t3r = a1a2r * b1r - a1a2i * b1i, t3i = a1a2r * b1i + a1a2i * b1r;  // * b1
        const double t4r = a3r * cr - a3i * ci, t4i = -(a3r * ci + a3i * cr);           // conj(a3) conj(c1)
        const double b2r = -(t3r + t4r) / N, b2i = -(t3i + t4i) / N;
        const double t5r = a2r * cr - a2i * ci, t5i = -(a2r * ci + a2i * cr);           // conj(a2) conj(c1)
        const double a1a3r = a1r * a3r + a1i * a3i, a1a3i = a1r * a3i - a1i * a3r;      // conj(a1) a3
        const double t6r = a1a3r * b1r - a1a3i * b1i, t6i = a1a3r * b1i + a1a3i * b1r;  // * b1
        const double b3r = (t5r - t6r) / N, b3i = (t5i - t6i) / N;
        // c2 = conj(a3 b1 - a1 b3), c3 = conj(a1 b2 - a2 b1)
        const double c2r = (a3r * b1r - a3i * b1i) - (a1r * b3r - a1i * b3i);
        const double c2i = -((a3r * b1i + a3i * b1r) - (a1r * b3i + a1i * b3r));
        const double c3r = (a1r * b2r - a1i * b2i) - (a2r * b1r - a2i * b1i);
        const double c3i = -((a1r * b2i + a1i * b2r) - (a2r * b1i + a2i * b1r));
        const double V[18] = {a1r, a1i, a2r, a2i, a3r, a3i, b1r, b1i, b2r, b2i, b3r, b3i, cr, ci, c2r, c2i, c3r, c3i};
        for (int k = 0; k < 18; k++) {
            const double d = fabs(sg * V[k] - src[k]);
            m = (d > m || d != d) ? d : m;
            q += d * d;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, m, off);
        m = (o > m || o != o) ? o : m;
        q += __shfl_down_sync(0xffffffffu, q, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out, m);
        atomicAdd(out + 1, q);
    }
}

// Largest |(U U^+)_ij - delta_ij| over all links of a field: zero to rounding
// when every link is unitary (the 13-real format applies).
__global__ void u3_check_kernel(Geom g, const double *links, double *out)
{
    const int V = 2 * g.vh;
    double m = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < 4LL * V;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const double *u = links + idx * 18;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double re = 0.0, im = 0.0;  // sum_k U_ik conj(U_jk)
                for (int k = 0; k < 3; k++) {
                    const double ar = u[2 * (3 * i + k)], ai = u[2 * (3 * i + k) + 1];
                    const double br = u[2 * (3 * j + k)], bi = u[2 * (3 * j + k) + 1];
                    re += ar * br + ai * bi;
                    im += ai * br - ar * bi;
                }
                const double d = fmax(fabs(re - (i == j ? 1.0 : 0.0)), fabs(im));
                m = (d > m || d != d) ? d : m;
            }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, m, off);
        m = (o > m || o != o) ? o : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

int nblocks(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_pack_spinor(int sf, int64_t n, const double *in, char *out, int *bad, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = nblocks(n, kBlock);
    switch (sf) {
    case S_F64: pack_kernel<S_F64><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_F32: pack_kernel<S_F32><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_HALF: pack_kernel<S_HALF><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT20: pack_kernel<S_INT20><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT14: pack_kernel<S_INT14><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT30: pack_kernel<S_INT30><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    default: break;
    }
}

void launch_pack32_spinor(int sf, int64_t n, const float *in, char *out, int *bad, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = nblocks(n, kBlock);
    switch (sf) {
    case S_F32: pack32_kernel<S_F32><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_HALF: pack32_kernel<S_HALF><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT20: pack32_kernel<S_INT20><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT14: pack32_kernel<S_INT14><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    case S_INT30: pack32_kernel<S_INT30><<<nb, kBlock, 0, s>>>(n, in, out, bad); break;
    default: break;
    }
}

void launch_pack_pair_int30(int64_t n, const float *in, char *out, int *bad, cudaStream_t s)
{
    if (n <= 0) return;
    pack_pair_kernel<<<nblocks(n, kBlock), kBlock, 0, s>>>(n, in, out, bad);
}

void launch_unpack_spinor(int sf, int cf, int64_t n, const char *in, double *out, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = nblocks(n, kBlock);
    const bool f64 = cf == HISQ_COMPUTE_F64;
    switch (sf) {
    case S_F64:
        if (f64) unpack_kernel<S_F64, double><<<nb, kBlock, 0, s>>>(n, in, out);
        else unpack_kernel<S_F64, float><<<nb, kBlock, 0, s>>>(n, in, out);
        break;
    case S_F32: unpack_kernel<S_F32, float><<<nb, kBlock, 0, s>>>(n, in, out); break;
    case S_HALF: unpack_kernel<S_HALF, float><<<nb, kBlock, 0, s>>>(n, in, out); break;
    case S_INT20: unpack_kernel<S_INT20, float><<<nb, kBlock, 0, s>>>(n, in, out); break;
    case S_INT14: unpack_kernel<S_INT14, float><<<nb, kBlock, 0, s>>>(n, in, out); break;
    case S_INT30:
        if (f64) unpack_kernel<S_INT30, double><<<nb, kBlock, 0, s>>>(n, in, out);
        else unpack_kernel<S_INT30, float><<<nb, kBlock, 0, s>>>(n, in, out);
        break;
    default: break;
    }
}

void launch_absmax(int64_t n, const double *x, double *out, cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(nblocks(n, kBlock), 4096);
    absmax_kernel<<<nb, kBlock, 0, s>>>(n, x, out);
}

void launch_r8_check(const Geom &g, int gf, const double *links, const char *stored, double el, double an,
                     double *out, cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(nblocks(8LL * g.vh, kBlock), 4096);
    switch (gf) {
    case G_F64: r8_check_kernel<G_F64><<<nb, kBlock, 0, s>>>(g, links, stored, el, an, out); break;
    case G_F32: r8_check_kernel<G_F32><<<nb, kBlock, 0, s>>>(g, links, stored, el, an, out); break;
    case G_FIX16: r8_check_kernel<G_FIX16><<<nb, kBlock, 0, s>>>(g, links, stored, el, an, out); break;
    case G_FIX32: r8_check_kernel<G_FIX32><<<nb, kBlock, 0, s>>>(g, links, stored, el, an, out); break;
    }
}

void launch_u3_check(const Geom &g, const double *links, double *out, cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(nblocks(8LL * g.vh, kBlock), 4096);
    u3_check_kernel<<<nb, kBlock, 0, s>>>(g, links, out);
}

void launch_r12_check(const Geom &g, const double *links, int k, double *out, cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(nblocks(8LL * g.vh, kBlock), 4096);
    r12_check_kernel<<<nb, kBlock, 0, s>>>(g, links, k, out);
}

void launch_quantise_links(const Geom &g, int gf, int recon, const double *links, double inv, char *out,
                           cudaStream_t s)
{
    const int nb = nblocks(8LL * g.vh, kBlock);
#define Q(GF, R) quantise_kernel<GF, R><<<nb, kBlock, 0, s>>>(g, links, inv, out)
    if (recon == 18) {
        switch (gf) {
        case G_F64: Q(G_F64, 18); break;
        case G_F32: Q(G_F32, 18); break;
        case G_FIX16: Q(G_FIX16, 18); break;
        case G_FIX32: Q(G_FIX32, 18); break;
        case G_SE15: Q(G_SE15, 18); break;
        }
    } else if (recon == 8) {
        switch (gf) {
        case G_F64: Q(G_F64, 8); break;
        case G_F32: Q(G_F32, 8); break;
        case G_FIX16: Q(G_FIX16, 8); break;
        case G_FIX32: Q(G_FIX32, 8); break;
        }
    } else if (recon == 13) {
        switch (gf) {
        case G_F64: Q(G_F64, 13); break;
        case G_F32: Q(G_F32, 13); break;
        case G_FIX16: Q(G_FIX16, 13); break;
        case G_FIX32: Q(G_FIX32, 13); break;
        }
    } else {
        switch (gf) {
        case G_F64: Q(G_F64, 12); break;
        case G_F32: Q(G_F32, 12); break;
        case G_FIX16: Q(G_FIX16, 12); break;
        case G_FIX32: Q(G_FIX32, 12); break;
        case G_SE15: Q(G_SE15, 12); break;
        }
    }
#undef Q
}

}  // namespace hisq
