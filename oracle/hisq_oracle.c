/*
 * hisq_oracle.c -- plain, slow, FP64 CPU oracle for the HISQ staggered stencil,
 * the reduced-bit storage formats and the Krylov solvers of
 * M. A. Clark, D. Howarth, J. Tu, M. Wagner, E. Weinberg,
 * "Maximizing the Bang Per Bit" (Lattice 2022).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code, header, table or
 * helper with the CUDA path; the two meet only through the seeded inputs.
 *
 * Conventions (the readings of points the paper leaves open are listed with
 * the design notes; each function below names the passage it follows):
 *   dims L = {Lx, Ly, Lz, Lt}, all even.
 *   lex = ((t*Lz + z)*Ly + y)*Lx + x,  parity = (x+y+z+t) mod 2,  cb = lex/2.
 *   gauge  : double [mu][lex][row][col][re,im]     (4*V links, 18 reals each)
 *   spinor : double [cb][color][re,im] on one parity (Vh = V/2 sites);
 *            full lattice = [parity][cb][color][re,im], even first.
 *
 * The stencil (the HISQ operator, named in Sec. 1 and Sec. 5.2 but never
 * written out) is read as
 *   (D psi)(x) = sum_mu [ F_mu(x) psi(x+mu) - F_mu(x-mu)^+ psi(x-mu)
 *                       + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^+ psi(x-3mu) ]
 * with links that already carry the staggered phases, M = 2m + D on the full
 * lattice and M_ee = 4m^2 - D_eo D_oe on the even sites.
 *
 * Every function is checked against closed forms, invariants, hand-derived
 * bit patterns or a dense direct solve by the tests; the error-estimate
 * trigger's rule (or_ru_trigger_step) against its closed form on geometric
 * residual sequences, its use inside or_mixed_cg through its limits and
 * convergence.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double kPi = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* O1 geometry                                                               */
/* ------------------------------------------------------------------------ */
static int64_t vol_of(const int *L) { return (int64_t)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int *L, int64_t lex, int c[4])
{
    for (int d = 0; d < 4; d++) {
        c[d] = (int)(lex % L[d]);
        lex /= L[d];
    }
}

static int64_t lex_of(const int *L, const int c[4])
{
    return (((int64_t)c[3] * L[2] + c[2]) * L[1] + c[1]) * L[0] + c[0];
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* Site of the given parity with checkerboard index cb: lex 2cb and 2cb+1 share
 * y, z, t and differ by one step in x, so exactly one of them has the parity. */
static int64_t lex_from_cb(const int *L, int parity, int64_t cb)
{
    int c[4];
    int64_t lex = 2 * cb;
    coords_of(L, lex, c);
    return parity_of(c) == parity ? lex : lex + 1;
}

/* lex of x + k * mu-hat with periodic wrap. */
static int64_t hop(const int *L, const int c[4], int mu, int k)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = ((d[mu] + k) % L[mu] + L[mu]) % L[mu];
    return lex_of(L, d);
}

/* Staggered phase eta_mu(x) times the antiperiodic-t sign of a fat (k=1) or
 * long (k=3) link: the sign that multiplies an SU(3) matrix in the synthetic
 * fields, used only to rebuild the third row of a compressed long link. */
static double link_sign(const int *L, const int c[4], int mu, int k, int antiperiodic_t)
{
    int s = 0;
    for (int nu = 0; nu < mu; nu++) s += c[nu];
    double eta = (s & 1) ? -1.0 : 1.0;
    if (antiperiodic_t && mu == 3 && c[3] + k >= L[3]) eta = -eta;
    return eta;
}

/* ------------------------------------------------------------------------ */
/* O3 the stencil                                                            */
/* ------------------------------------------------------------------------ */
static const cplx *link_at(const cplx *g, int64_t V, int mu, int64_t lex)
{
    return g + ((int64_t)mu * V + lex) * 9;
}

/* acc += sgn * U s */
static void mv_add(cplx acc[3], const cplx *U, const cplx *s, double sgn)
{
    for (int i = 0; i < 3; i++) {
        cplx t = 0;
        for (int j = 0; j < 3; j++) t += U[i * 3 + j] * s[j];
        acc[i] += sgn * t;
    }
}

/* acc += sgn * U^+ s */
static void mv_adj_add(cplx acc[3], const cplx *U, const cplx *s, double sgn)
{
    for (int i = 0; i < 3; i++) {
        cplx t = 0;
        for (int j = 0; j < 3; j++) t += conj(U[j * 3 + i]) * s[j];
        acc[i] += sgn * t;
    }
}

/* (D psi)(x) at one site x; psi is the half-lattice field of the other parity.
 * Terms are added per direction in the order +1, -1, +3, -3. */
static void dslash_site(const int *L, const cplx *fat, const cplx *lng, const cplx *in,
                        int64_t lex, cplx out[3])
{
    const int64_t V = vol_of(L);
    int c[4];
    coords_of(L, lex, c);
    cplx acc[3] = {0, 0, 0};
    for (int mu = 0; mu < 4; mu++) {
        int64_t p1 = hop(L, c, mu, +1), m1 = hop(L, c, mu, -1);
        int64_t p3 = hop(L, c, mu, +3), m3 = hop(L, c, mu, -3);
        mv_add(acc, link_at(fat, V, mu, lex), in + (p1 / 2) * 3, +1.0);
        mv_adj_add(acc, link_at(fat, V, mu, m1), in + (m1 / 2) * 3, -1.0);
        mv_add(acc, link_at(lng, V, mu, lex), in + (p3 / 2) * 3, +1.0);
        mv_adj_add(acc, link_at(lng, V, mu, m3), in + (m3 / 2) * 3, -1.0);
    }
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = acc[2];
}

/* out[cb] = (D in)(x) for every site x of parity out_parity; in lives on the
 * other parity.  D_eo is out_parity 0, D_oe is out_parity 1. */
void or_dslash(const int *L, const double *fat, const double *lng, int out_parity,
               const double *in, double *out)
{
    const int64_t Vh = vol_of(L) / 2;
    const cplx *F = (const cplx *)fat, *G = (const cplx *)lng, *s = (const cplx *)in;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int64_t cb = 0; cb < Vh; cb++)
        dslash_site(L, F, G, s, lex_from_cb(L, out_parity, cb), o + cb * 3);
}

/* The stencil at a list of output sites only (checkerboard indices cbs[i]). */
void or_dslash_sites(const int *L, const double *fat, const double *lng, int out_parity,
                     const double *in, int64_t n, const int64_t *cbs, double *out)
{
    const cplx *F = (const cplx *)fat, *G = (const cplx *)lng, *s = (const cplx *)in;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        dslash_site(L, F, G, s, lex_from_cb(L, out_parity, cbs[i]), o + i * 3);
}

/* y = (4 m^2 + sigma) x - D_eo D_oe x on the even sites. */
void or_mee(const int *L, const double *fat, const double *lng, double m, double sigma,
            const double *x, double *y)
{
    const int64_t n = vol_of(L) / 2 * 3;
    cplx *tmp = malloc(sizeof(cplx) * n);
    cplx *dd = malloc(sizeof(cplx) * n);
    or_dslash(L, fat, lng, 1, x, (double *)tmp);
    or_dslash(L, fat, lng, 0, (double *)tmp, (double *)dd);
    const cplx *xc = (const cplx *)x;
    cplx *yc = (cplx *)y;
    const double d = 4.0 * m * m + sigma;
    for (int64_t i = 0; i < n; i++) yc[i] = d * xc[i] - dd[i];
    free(tmp);
    free(dd);
}

/* y = 2 m x + D x on the full lattice ([parity][cb][color]). */
void or_mfull(const int *L, const double *fat, const double *lng, double m,
              const double *x, double *y)
{
    const int64_t n = vol_of(L) / 2 * 3;
    const cplx *xe = (const cplx *)x, *xo = xe + n;
    cplx *ye = (cplx *)y, *yo = ye + n;
    or_dslash(L, fat, lng, 0, (const double *)xo, (double *)ye);
    or_dslash(L, fat, lng, 1, (const double *)xe, (double *)yo);
    for (int64_t i = 0; i < n; i++) {
        ye[i] += 2.0 * m * xe[i];
        yo[i] += 2.0 * m * xo[i];
    }
}

/* ------------------------------------------------------------------------ */
/* O5 storage formats                                                        */
/* ------------------------------------------------------------------------ */
static uint32_t f2u(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

static float u2f(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* 16-bit fixed point with a site-local FP32 norm (Sec. 2, Listing 1): record
 * of 16 bytes = int16 v[6] followed by float max.  The largest |component| of
 * the site sets the scale; components are rounded to nearest-even integers in
 * [-32767, 32767].  Decoding multiplies by max * fl(1/32767).  A site whose
 * max is below 2^-110 (where 32767/max would overflow FP32) is stored as zero
 * with norm 0, like an all-zero site.
 * Returns the number of sites with a non-finite component. */
int64_t or_half_pack(int64_t n, const float *v, unsigned char *rec)
{
    int64_t bad = 0;
    for (int64_t s = 0; s < n; s++) {
        const float *x = v + 6 * s;
        float mx = 0.0f;
        int finite = 1;
        for (int i = 0; i < 6; i++) {
            if (!isfinite(x[i])) finite = 0;
            mx = fmaxf(mx, fabsf(x[i]));
        }
        int16_t q[6] = {0, 0, 0, 0, 0, 0};
        if (!finite) {
            bad++;
            mx = 0.0f;
        } else if (mx < 0x1p-110f) {
            mx = 0.0f;
        } else {
            const float inv = 32767.0f / mx;
            for (int i = 0; i < 6; i++) {
                long r = lrintf(x[i] * inv);
                if (r > 32767) r = 32767;
                if (r < -32767) r = -32767;
                q[i] = (int16_t)r;
            }
        }
        memcpy(rec + 16 * s, q, 12);
        memcpy(rec + 16 * s + 12, &mx, 4);
    }
    return bad;
}

void or_half_unpack(int64_t n, const unsigned char *rec, float *v)
{
    const float inv32767 = 1.0f / 32767.0f;
    for (int64_t s = 0; s < n; s++) {
        int16_t q[6];
        float mx;
        memcpy(q, rec + 16 * s, 12);
        memcpy(&mx, rec + 16 * s + 12, 4);
        const float scale = mx * inv32767;
        for (int i = 0; i < 6; i++) v[6 * s + i] = (float)q[i] * scale;
    }
}

/* 20-bit shared-exponent format (Sec. 4, Listing 2; the codec of Appendix A,
 * Listing 4).  Per site: six 20-bit two's-complement integers and an 8-bit
 * exponent in four 32-bit words.  Steps of the appendix:
 *   max  = largest |component| (FP32; the garbled vector initialisation of
 *          the listing is read as a scalar max over all six components);
 *   t    = max / (2^19 - 1) in FP32;
 *   E    = (biased exponent field of t) + 1, mantissa dropped, so 2^(E-127)
 *          is the power of two just above t;
 *   q_i  = round-to-nearest-even(v_i * 2^-(E-127))  (|q_i| <= 2^19 - 1);
 * and the bitfields are laid out least-significant first within each word:
 *   w0 = re0[0:20] | im0 bits 8..19 at [20:32]
 *   w1 = im0 bits 0..7 at [0:8] | re1 at [8:28] | im1 bits 16..19 at [28:32]
 *   w2 = im1 bits 0..15 at [0:16] | re2 bits 4..19 at [16:32]
 *   w3 = re2 bits 0..3 at [0:4] | im2 at [4:24] | E at [24:32]
 * Decoding sign-extends each 20-bit value and multiplies by 2^(E-127).
 * Returns the number of sites with a non-finite component (their record is
 * written as zero with E = 1). */
int64_t or_int20_pack(int64_t n, const float *v, uint32_t *w)
{
    int64_t bad = 0;
    for (int64_t s = 0; s < n; s++) {
        const float *x = v + 6 * s;
        float mx = 0.0f;
        int finite = 1;
        for (int i = 0; i < 6; i++) {
            if (!isfinite(x[i])) finite = 0;
            mx = fmaxf(mx, fabsf(x[i]));
        }
        uint32_t u[6] = {0, 0, 0, 0, 0, 0};
        uint32_t E = 1;
        if (!finite) {
            bad++;
        } else {
            const float t = mx / 524287.0f;
            E = ((f2u(t) >> 23) & 0xffu) + 1u;
            const float down = u2f((254u - E) << 23); /* 2^-(E-127) */
            for (int i = 0; i < 6; i++) {
                long q = lrintf(x[i] * down);
                u[i] = (uint32_t)(int32_t)q;
            }
        }
        uint32_t *o = w + 4 * s;
        o[0] = (u[0] & 0xfffffu) | (((u[1] >> 8) & 0xfffu) << 20);
        o[1] = (u[1] & 0xffu) | ((u[2] & 0xfffffu) << 8) | (((u[3] >> 16) & 0xfu) << 28);
        o[2] = (u[3] & 0xffffu) | (((u[4] >> 4) & 0xffffu) << 16);
        o[3] = (u[4] & 0xfu) | ((u[5] & 0xfffffu) << 4) | (E << 24);
    }
    return bad;
}

static int32_t sext(uint32_t u, int bits)
{
    const uint32_t m = 1u << (bits - 1);
    u &= (bits == 32) ? 0xffffffffu : ((1u << bits) - 1u);
    return (int32_t)((u ^ m) - m);
}

void or_int20_unpack(int64_t n, const uint32_t *w, float *v)
{
    for (int64_t s = 0; s < n; s++) {
        const uint32_t *o = w + 4 * s;
        uint32_t u[6];
        u[0] = o[0] & 0xfffffu;
        u[1] = ((o[0] >> 20) << 8) | (o[1] & 0xffu);
        u[2] = (o[1] >> 8) & 0xfffffu;
        u[3] = ((o[1] >> 28) << 16) | (o[2] & 0xffffu);
        u[4] = ((o[2] >> 16) << 4) | (o[3] & 0xfu);
        u[5] = (o[3] >> 4) & 0xfffffu;
        const uint32_t E = o[3] >> 24;
        const float up = u2f(E << 23); /* 2^(E-127) */
        for (int i = 0; i < 6; i++) v[6 * s + i] = (float)sext(u[i], 20) * up;
    }
}

/* 30-bit shared-exponent format (Sec. 4, Listing 3; no layout is given, so
 * this is our reading): six 32-bit words; bits 0..29 of word k hold the 30-bit
 * two's-complement integer q_k; bits 30..31 of words 0..3 hold bits 2k..2k+1
 * of the 8-bit exponent E; the top bits of words 4, 5 are zero.  The exponent
 * rule is the 20-bit one applied in FP64 with scale 2^29 - 1:
 * t = max / (2^29-1), 2^(E-127) the power of two just above t (E clamped to
 * [1, 254]), q_k = rint(v_k * 2^-(E-127)).  Decoding is exact in FP64.
 * Returns the number of sites that could not be encoded (non-finite, or too
 * large for the 8-bit exponent); they are written as zero with E = 1. */
int64_t or_int30_pack(int64_t n, const double *v, uint32_t *w)
{
    int64_t bad = 0;
    for (int64_t s = 0; s < n; s++) {
        const double *x = v + 6 * s;
        double mx = 0.0;
        int ok = 1;
        for (int i = 0; i < 6; i++) {
            if (!isfinite(x[i])) ok = 0;
            mx = fmax(mx, fabs(x[i]));
        }
        uint32_t E = 1;
        uint32_t u[6] = {0, 0, 0, 0, 0, 0};
        if (ok) {
            const double t = mx / 536870911.0;
            int ex = 0;
            if (t > 0.0) frexp(t, &ex); /* t = f 2^ex, f in [0.5, 1) */
            int e = (t > 0.0) ? ex + 127 : 1;
            if (e < 1) e = 1;
            if (e > 254) ok = 0;
            if (ok) {
                E = (uint32_t)e;
                for (int i = 0; i < 6; i++) {
                    long long q = llrint(ldexp(x[i], -(e - 127)));
                    u[i] = (uint32_t)(int32_t)q;
                }
            }
        }
        if (!ok) bad++;
        uint32_t *o = w + 6 * s;
        for (int k = 0; k < 6; k++) {
            o[k] = u[k] & 0x3fffffffu;
            if (k < 4) o[k] |= ((E >> (2 * k)) & 3u) << 30;
        }
    }
    return bad;
}

void or_int30_unpack(int64_t n, const uint32_t *w, double *v)
{
    for (int64_t s = 0; s < n; s++) {
        const uint32_t *o = w + 6 * s;
        uint32_t E = 0;
        for (int k = 0; k < 4; k++) E |= (o[k] >> 30) << (2 * k);
        for (int k = 0; k < 6; k++) v[6 * s + k] = ldexp((double)sext(o[k], 30), (int)E - 127);
    }
}

/* 14-bit shared-exponent format in 12 bytes: a third width of the family the
 * paper builds its two formats from (Sec. 4: the 20- and 30-bit formats are
 * two of many possible shared-exponent formats).  Per site: six 14-bit
 * two's-complement integers and an 8-bit exponent in three 32-bit words of
 * two 16-bit halves each, half k = 2j + h in word j (h = 0 low, 1 high):
 *   half k = q_k << 2 | e_k,  e_k = exponent bits 2k..2k+1 for k < 4, 0 else,
 * components in the order re0, im0, re1, im1, re2, im2.  The exponent rule is
 * Appendix A's with scale 2^13 - 1 in FP32 arithmetic:
 *   max = largest |component| (FP32);  t = max / (2^13 - 1) in FP32;
 *   E = (biased exponent field of t) + 1, so 2^(E-127) is the power of two
 *       just above t;  q_k = round-to-nearest-even(v_k 2^-(E-127));
 * decoding multiplies the sign-extended q_k by 2^(E-127).  Non-finite sites
 * are written as zero with E = 1 and counted (the return value). */
int64_t or_int14_pack(int64_t n, const float *v, uint32_t *w)
{
    int64_t bad = 0;
    for (int64_t s = 0; s < n; s++) {
        const float *x = v + 6 * s;
        float mx = 0.0f;
        int finite = 1;
        for (int i = 0; i < 6; i++) {
            if (!isfinite(x[i])) finite = 0;
            mx = fmaxf(mx, fabsf(x[i]));
        }
        uint32_t q[6] = {0, 0, 0, 0, 0, 0};
        uint32_t E = 1;
        if (!finite) {
            bad++;
        } else {
            const float t = mx / 8191.0f;
            E = ((f2u(t) >> 23) & 0xffu) + 1u;
            const float down = u2f((254u - E) << 23); /* 2^-(E-127) */
            for (int i = 0; i < 6; i++) q[i] = (uint32_t)(int32_t)lrintf(x[i] * down);
        }
        uint32_t half[6];
        for (int k = 0; k < 6; k++) {
            const uint32_t e = k < 4 ? (E >> (2 * k)) & 3u : 0u;
            half[k] = ((q[k] & 0x3fffu) << 2) | e;
        }
        for (int j = 0; j < 3; j++) w[3 * s + j] = half[2 * j] | (half[2 * j + 1] << 16);
    }
    return bad;
}

void or_int14_unpack(int64_t n, const uint32_t *w, float *v)
{
    for (int64_t s = 0; s < n; s++) {
        uint32_t half[6];
        for (int j = 0; j < 3; j++) {
            half[2 * j] = w[3 * s + j] & 0xffffu;
            half[2 * j + 1] = w[3 * s + j] >> 16;
        }
        uint32_t E = 0;
        for (int k = 0; k < 4; k++) E |= (half[k] & 3u) << (2 * k);
        const float up = u2f(E << 23); /* 2^(E-127) */
        for (int k = 0; k < 6; k++) v[6 * s + k] = (float)sext(half[k] >> 2, 14) * up;
    }
}

/* Fixed-point gauge (Sec. 2 and its footnote on smeared fields; Sec. 4 for the
 * 32-bit variant): one scale per field set by the global max |element|;
 * q = rint(x * (qmax / gmax)) in FP64, clamped to [-qmax, qmax],
 * qmax = 2^15-1 (16-bit) or 2^31-1 (32-bit). */
double or_absmax(int64_t n, const double *g)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) m = fmax(m, fabs(g[i]));
    return m;
}

static double qmax_of(int bits) { return bits == 16 ? 32767.0 : 2147483647.0; }

void or_fix_pack(int64_t n, const double *g, double gmax, int bits, int32_t *q)
{
    const double qm = qmax_of(bits);
    const double inv = gmax > 0.0 ? qm / gmax : 0.0;
    for (int64_t i = 0; i < n; i++) {
        double r = rint(g[i] * inv);
        if (r > qm) r = qm;
        if (r < -qm) r = -qm;
        q[i] = (int32_t)r;
    }
}

/* Decoded value as the computation sees it: FP64 q * (gmax/qmax), or, for FP32
 * compute, fl32(q) * fl32(gmax/qmax) rounded to FP32. */
void or_fix_unpack(int64_t n, const int32_t *q, double gmax, int bits, int compute_f32, double *out)
{
    const double s = gmax / qmax_of(bits);
    const float sf = (float)s;
    for (int64_t i = 0; i < n; i++) {
        if (compute_f32)
            out[i] = (double)((float)q[i] * sf);
        else
            out[i] = (double)q[i] * s;
    }
}

/* Shared-exponent link format (a gauge counterpart of the Sec. 4 fermion
 * formats, for smeared fat links, whose elements have no common scale across
 * the lattice): per link, its nr stored reals (18, or 12 for rows 0 and 1) as
 * 15-bit two's-complement integers sharing one 8-bit exponent.  Exponent rule
 * of the 30-bit format in FP64 with scale 2^14 - 1: mx = max |x| over the
 * link's nr reals, t = mx / (2^14 - 1), 2^(E-127) the power of two just above
 * t (E clamped to [1, 254]), q_k = rint(x_k 2^-(E-127)) (|q_k| <= 2^14 - 1).
 * Layout: one 16-bit half per real, half k = q_k << 1 | bit k of E for k < 8,
 * q_k << 1 for k >= 8 (the planar chunks of the 16-bit fixed-point format).
 * Decoding: q_k 2^(E-127), exact in FP32.  A non-finite link is stored as
 * zero with E = 1 and counted. */
int64_t or_se15_pack(int64_t nlinks, int nr, const double *g, uint16_t *h)
{
    int64_t bad = 0;
    for (int64_t l = 0; l < nlinks; l++) {
        const double *x = g + (int64_t)nr * l;
        double mx = 0.0;
        int ok = 1;
        for (int k = 0; k < nr; k++) {
            if (!isfinite(x[k])) ok = 0;
            mx = fmax(mx, fabs(x[k]));
        }
        int E = 1;
        int32_t q[18] = {0};
        if (ok) {
            const double t = mx / 16383.0;
            int ex = 0;
            if (t > 0.0) frexp(t, &ex); /* t = f 2^ex, f in [0.5, 1) */
            E = t > 0.0 ? ex + 127 : 1;
            if (E < 1) E = 1;
            if (E > 254) ok = 0;
            if (ok)
                for (int k = 0; k < nr; k++) q[k] = (int32_t)llrint(ldexp(x[k], -(E - 127)));
        }
        if (!ok) {
            bad++;
            E = 1;
            for (int k = 0; k < nr; k++) q[k] = 0;
        }
        for (int k = 0; k < nr; k++) {
            const uint32_t e = k < 8 ? ((uint32_t)E >> k) & 1u : 0u;
            h[(int64_t)nr * l + k] = (uint16_t)((((uint32_t)q[k] & 0x7fffu) << 1) | e);
        }
    }
    return bad;
}

void or_se15_unpack(int64_t nlinks, int nr, const uint16_t *h, double *g)
{
    for (int64_t l = 0; l < nlinks; l++) {
        const uint16_t *w = h + (int64_t)nr * l;
        int E = 0;
        for (int k = 0; k < 8; k++) E |= (w[k] & 1) << k;
        for (int k = 0; k < nr; k++)
            g[(int64_t)nr * l + k] = ldexp((double)sext((uint32_t)w[k] >> 1, 15), E - 127);
    }
}

/* Row 2 of a compressed link from rows 0 and 1 (Sec. 1, link compression 18 ->
 * 12): for U = sign * W with W in SU(3), row2(U) = sign * conj(row0 x row1). */
static void rebuild_row2(cplx *U, double sign)
{
    U[6] = sign * conj(U[1] * U[5] - U[2] * U[4]);
    U[7] = sign * conj(U[2] * U[3] - U[0] * U[5]);
    U[8] = sign * conj(U[0] * U[4] - U[1] * U[3]);
}

/* An angle stored as a fraction t of pi in [-1, 1] (the phases of the 13- and
 * 8-real link formats): FP64 as is, FP32 rounded, fixed point
 * q = rint(t * qmax) with qmax = 2^15-1 or 2^31-1 (no global scale: |t| <= 1). */
static double angle_round(double t, int gfmt)
{
    if (gfmt == 1) return (double)(float)t;
    if (gfmt >= 2) {
        const double qm = gfmt == 2 ? 32767.0 : 2147483647.0;
        return rint(t * qm) / qm;
    }
    return t;
}

static double round_elem(double x, int gfmt, double gmax, int compute_f32)
{
    if (gfmt == 0) return x;
    if (gfmt == 1) return (double)(float)x;
    int32_t q;
    const int bits = gfmt == 2 ? 16 : 32;
    double out;
    or_fix_pack(1, &x, gmax, bits, &q);
    or_fix_unpack(1, &q, gmax, bits, compute_f32, &out);
    return out;
}

/* 13-real link (12 + 1, for long links in U(3)): rows 0 and 1 and the phase
 * theta = arg det U, stored as t = theta/pi; for a unitary U the cofactor rule
 * gives row2 = det(U) conj(row0 x row1), i.e. row2 = e^{i pi t} conj(row0 x row1).
 * U: 9 complex elements (row-major) in and out, rows 0 and 1 already rounded. */
static void rebuild_r13(cplx *U, double t)
{
    const cplx ph = cos(kPi * t) + I * sin(kPi * t);
    U[6] = ph * conj(U[1] * U[5] - U[2] * U[4]);
    U[7] = ph * conj(U[2] * U[3] - U[0] * U[5]);
    U[8] = ph * conj(U[0] * U[4] - U[1] * U[3]);
}

/* 8-real link (Sec. 1: 18 -> 8 for SU(3) links; for U = sign * V with V in
 * SU(3)): the parameters of V are t1 = arg(V00)/pi, t2 = arg(V20)/pi and the
 * complex V01, V02, V10.  Rebuilding V from them (unitarity and det V = 1):
 *   N = |V01|^2 + |V02|^2 = 1 - |V00|^2,  V00 = sqrt(1 - N) e^{i pi t1},
 *   V20 = sqrt(N - |V10|^2) e^{i pi t2},
 *   V11 = -(conj(V00) V01 V10 + conj(V02) conj(V20)) / N,
 *   V12 = (conj(V01) conj(V20) - conj(V00) V02 V10) / N,
 *   V21 = conj(V02 V10 - V00 V12),  V22 = conj(V00 V11 - V01 V10)
 * (rows 1 and 2 orthogonal to row 0, row 2 = conj(row0 x row1)).  Needs
 * N > 0; precision falls as N or |V20| become small (links near diagonal).
 * p: the 8 reals {t1, t2, Re V01, Im V01, Re V02, Im V02, Re V10, Im V10}. */
void or_link_r8_pack(int64_t n, const double *links, const double *sign, double *p)
{
    for (int64_t i = 0; i < n; i++) {
        const cplx *U = (const cplx *)(links + 18 * i);
        cplx V[9];
        for (int e = 0; e < 9; e++) V[e] = sign[i] * U[e];
        double *q = p + 8 * i;
        q[0] = carg(V[0]) / kPi;
        q[1] = carg(V[6]) / kPi;
        q[2] = creal(V[1]); q[3] = cimag(V[1]);
        q[4] = creal(V[2]); q[5] = cimag(V[2]);
        q[6] = creal(V[3]); q[7] = cimag(V[3]);
    }
}

void or_link_r8_unpack(int64_t n, const double *p, const double *sign, double *links)
{
    for (int64_t i = 0; i < n; i++) {
        const double *q = p + 8 * i;
        const cplx a2 = q[2] + I * q[3], a3 = q[4] + I * q[5], b1 = q[6] + I * q[7];
        const double N = creal(a2 * conj(a2)) + creal(a3 * conj(a3));
        const double ra = sqrt(fmax(1.0 - N, 0.0)), rc = sqrt(fmax(N - creal(b1 * conj(b1)), 0.0));
        const cplx a1 = ra * (cos(kPi * q[0]) + I * sin(kPi * q[0]));
        const cplx c1 = rc * (cos(kPi * q[1]) + I * sin(kPi * q[1]));
        const cplx b2 = -(conj(a1) * a2 * b1 + conj(a3) * conj(c1)) / N;
        const cplx b3 = (conj(a2) * conj(c1) - conj(a1) * a3 * b1) / N;
        const cplx c2 = conj(a3 * b1 - a1 * b3);
        const cplx c3 = conj(a1 * b2 - a2 * b1);
        const cplx V[9] = {a1, a2, a3, b1, b2, b3, c1, c2, c3};
        cplx *U = (cplx *)(links + 18 * i);
        for (int e = 0; e < 9; e++) U[e] = sign[i] * V[e];
    }
}

/* Format emulation (O4): a link field as the computation sees it after storage
 * in format gfmt (0 FP64, 1 FP32, 2 fixed-16, 3 fixed-32, 4 shared-exponent
 * 15-bit, recon 18 or 12) with recon 18, 12, 13
 * or 8 (the compressions rebuild in FP64 from the rounded stored reals); r12
 * and r8 use the link's sign (long links: k = 3, fat links: k = 1).  gmax is
 * the field's scale (max |element| over all 18 reals of every link). */
void or_gauge_emulate(const int *L, const double *g, int gfmt, int recon, int k,
                      int antiperiodic_t, int compute_f32, double gmax, double *out)
{
    if (recon == 8) {
        const int64_t V = vol_of(L);
        double *sg = malloc(sizeof(double) * 4 * V);
        for (int mu = 0; mu < 4; mu++)
            for (int64_t lex = 0; lex < V; lex++) {
                int c[4];
                coords_of(L, lex, c);
                sg[(int64_t)mu * V + lex] = link_sign(L, c, mu, k, antiperiodic_t);
            }
        double *p = malloc(sizeof(double) * 8 * 4 * V);
        or_link_r8_pack(4 * V, g, sg, p);
        for (int64_t i = 0; i < 4 * V; i++) {
            p[8 * i] = angle_round(p[8 * i], gfmt);
            p[8 * i + 1] = angle_round(p[8 * i + 1], gfmt);
            for (int j = 2; j < 8; j++) p[8 * i + j] = round_elem(p[8 * i + j], gfmt, gmax, compute_f32);
        }
        or_link_r8_unpack(4 * V, p, sg, out);
        free(p);
        free(sg);
        return;
    }
    const int64_t V = vol_of(L);
    const int64_t n = 4 * V * 18;
    if (gfmt == 0) {
        memcpy(out, g, sizeof(double) * n);
    } else if (gfmt == 1) {
        for (int64_t i = 0; i < n; i++) out[i] = (double)(float)g[i];
    } else if (gfmt == 4) {
        /* the stored reals of each link (18, or 12 for rows 0 and 1) with its own exponent */
        const int nr = recon == 12 ? 12 : 18;
        double *st = malloc(sizeof(double) * 4 * V * nr);
        uint16_t *h = malloc(sizeof(uint16_t) * 4 * V * nr);
        for (int64_t i = 0; i < 4 * V; i++)
            for (int k = 0; k < nr; k++) st[i * nr + k] = g[i * 18 + k];
        or_se15_pack(4 * V, nr, st, h);
        or_se15_unpack(4 * V, nr, h, st);
        memset(out, 0, sizeof(double) * n);
        for (int64_t i = 0; i < 4 * V; i++)
            for (int k = 0; k < nr; k++) out[i * 18 + k] = st[i * nr + k];
        free(st);
        free(h);
    } else {
        const int bits = gfmt == 2 ? 16 : 32;
        int32_t *q = malloc(sizeof(int32_t) * n);
        or_fix_pack(n, g, gmax, bits, q);
        or_fix_unpack(n, q, gmax, bits, compute_f32, out);
        free(q);
    }
    if (recon == 12) {
        for (int mu = 0; mu < 4; mu++)
            for (int64_t lex = 0; lex < V; lex++) {
                int c[4];
                coords_of(L, lex, c);
                cplx *U = (cplx *)(out + ((int64_t)mu * V + lex) * 18);
                rebuild_row2(U, link_sign(L, c, mu, k, antiperiodic_t));
            }
    } else if (recon == 13) {
        for (int64_t i = 0; i < 4 * V; i++) {
            const cplx *G = (const cplx *)(g + 18 * i);
            const cplx det = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                             G[2] * (G[3] * G[7] - G[4] * G[6]);
            rebuild_r13((cplx *)(out + 18 * i), angle_round(carg(det) / kPi, gfmt));
        }
    }
}

/* Spinor format emulation: sfmt 0 FP64, 1 FP32, 2 half, 3 int20, 4 int30,
 * 5 int14. */
void or_spinor_emulate(int64_t nsites, int sfmt, const double *in, double *out)
{
    const int64_t n = nsites * 6;
    if (sfmt == 0) {
        memcpy(out, in, sizeof(double) * n);
        return;
    }
    if (sfmt == 1) {
        for (int64_t i = 0; i < n; i++) out[i] = (double)(float)in[i];
        return;
    }
    if (sfmt == 4) {
        uint32_t *w = malloc(sizeof(uint32_t) * 6 * nsites);
        or_int30_pack(nsites, in, w);
        or_int30_unpack(nsites, w, out);
        free(w);
        return;
    }
    float *f = malloc(sizeof(float) * n);
    for (int64_t i = 0; i < n; i++) f[i] = (float)in[i];
    if (sfmt == 2) {
        unsigned char *r = malloc(16 * nsites);
        or_half_pack(nsites, f, r);
        or_half_unpack(nsites, r, f);
        free(r);
    } else if (sfmt == 5) {
        uint32_t *w = malloc(sizeof(uint32_t) * 3 * nsites);
        or_int14_pack(nsites, f, w);
        or_int14_unpack(nsites, w, f);
        free(w);
    } else {
        uint32_t *w = malloc(sizeof(uint32_t) * 4 * nsites);
        or_int20_pack(nsites, f, w);
        or_int20_unpack(nsites, w, f);
        free(w);
    }
    for (int64_t i = 0; i < n; i++) out[i] = (double)f[i];
    free(f);
}

/* ------------------------------------------------------------------------ */
/* vector helpers (serial, fixed order)                                      */
/* ------------------------------------------------------------------------ */
static cplx cdot(int64_t n, const cplx *a, const cplx *b) /* a^+ b */
{
    cplx s = 0;
    for (int64_t i = 0; i < n; i++) s += conj(a[i]) * b[i];
    return s;
}

static double nrm2(int64_t n, const cplx *a)
{
    double s = 0;
    for (int64_t i = 0; i < n; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

typedef struct {
    const int *L;
    const double *fat, *lng;
    double m, sigma;
    int full; /* 0: M_ee + sigma on even sites; 1: M = 2m + D full lattice */
} op_t;

static int64_t op_len(const op_t *op) { return vol_of(op->L) / 2 * 3 * (op->full ? 2 : 1); }

static void op_apply(const op_t *op, const cplx *x, cplx *y)
{
    if (op->full)
        or_mfull(op->L, op->fat, op->lng, op->m, (const double *)x, (double *)y);
    else
        or_mee(op->L, op->fat, op->lng, op->m, op->sigma, (const double *)x, (double *)y);
}

/* ------------------------------------------------------------------------ */
/* O6 conjugate gradient (Hestenes-Stiefel), FP64                            */
/* ------------------------------------------------------------------------ */
/* Solves (M_ee + sigma) x = b.  x holds the initial guess if use_x0, else it
 * starts from zero.  Stops when the iterated residual reaches tol*|b|; then
 * *true_res = |b - (M_ee+sigma) x| / |b|.  Returns 0 on convergence, 1 when
 * maxiter was reached, 2 on breakdown. */
int or_cg(const int *L, const double *fat, const double *lng, double m, double sigma,
          const double *b_, double *x_, double tol, int maxiter, int use_x0,
          int *iters, double *true_res)
{
    op_t op = {L, fat, lng, m, sigma, 0};
    const int64_t n = op_len(&op);
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n);
    if (!use_x0) memset(x, 0, sizeof(cplx) * n);
    op_apply(&op, x, Ap);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    memcpy(p, r, sizeof(cplx) * n);
    const double bb = nrm2(n, b);
    double rr = nrm2(n, r);
    int k = 0, status = 1;
    if (sqrt(rr) <= tol * sqrt(bb)) status = 0;
    while (status == 1 && k < maxiter) {
        op_apply(&op, p, Ap);
        const double pAp = creal(cdot(n, p, Ap));
        if (!(pAp > 0.0)) {
            status = 2;
            break;
        }
        const double alpha = rr / pAp;
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        const double rr_new = nrm2(n, r);
        k++;
        if (sqrt(rr_new) <= tol * sqrt(bb)) {
            status = 0;
            break;
        }
        const double beta = rr_new / rr;
        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    op_apply(&op, x, Ap);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    *true_res = sqrt(nrm2(n, r) / bb);
    *iters = k;
    free(r);
    free(p);
    free(Ap);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O10 stabilised mixed-precision CG (Sec. 3.1), sloppy storage emulated      */
/* ------------------------------------------------------------------------ */
/* The reference for the algorithm's logic, not for the GPU's rounding: FP64
 * arithmetic throughout, with every write of a sloppy vector (r, p, A p)
 * rounded through spinor format sfmt (or_spinor_emulate), the sloppy operator
 * applied with the links (fat_s, lng_s) -- for example the format-emulated
 * copies of (fat, lng) -- and the true residuals with the exact (fat, lng).
 * Sec. 3.1 and its footnote, in the readings used throughout:
 *   reliable update when |r_k| < delta * max|r_j| over the iterations
 *     since the last one, or when |r_k| <= tol |b|: x_hi is brought up to
 *     date, the FP64 true residual r^ = b - A x_hi replaces r, and the solve
 *     ends if |r^| <= tol |b|;
 *   buffered x: the directions p_j and steps alpha_j are kept in a ring
 *     of nbuf entries and added to x_hi (FP64) when the ring is full and at
 *     each reliable update;
 *   re-projection (opts bit 1): at a reliable update
 *     p <- p - (r^+ p / r^+ r^) r^, beta = |r^|^2 / |r_old|^2 (Fletcher-Reeves),
 *     p <- r^ + beta p;
 *   Polak-Ribiere (opts bit 0): beta = (|r_new|^2 - Re r_new^+ r_old)
 *     / |r_old|^2; otherwise Fletcher-Reeves |r_new|^2 / |r_old|^2.
 *   error-estimate trigger (dyn_eps > 0, in place of delta; the "more
 *     dynamic choice based on explicit error estimation" of the Sec. 3
 *     footnote, read after the residual replacement of van der Vorst and Ye,
 *     SIAM J. Sci. Comput. 22 (2000) 835): d estimates the drift of the
 *     iterated from the true residual, growing by the rounding of each sloppy
 *     update, d_{k+1} = d_k + eps (|r_{k+1}| + |alpha_k| |A p_k|) with eps =
 *     dyn_eps, the sloppy operator's relative precision; a reliable update
 *     is made when d crosses sqrt(eps) |r| (d_k <= sqrt(eps) |r_k| and
 *     d_{k+1} > sqrt(eps) |r_{k+1}|) and d_{k+1} > 1.1 d_init, or when
 *     |r_k| <= tol |b|; after each update d = d_init = eps |r^|.
 * x_ receives x_hi (starting from zero).  hist (NULL or maxiter + 1 entries)
 * receives |r_k| / |b| for k = 0..iters: the iterated residual, replaced by
 * the recomputed true residual at the iterations that end with a reliable
 * update (the jumps of Fig. 1).  Returns 0 on convergence, 1 at maxiter, 2
 * on breakdown (p^+ A p <= 0 or non-finite). */
/* One step of the error-estimate reliable-update trigger (Sec. 3 footnote,
 * read after van der Vorst and Ye's residual replacement): the drift estimate
 * grows by the rounding of the step, d_new = d + eps (|r_{k+1}| +
 * |alpha_k| |A p_k|); an update is due when d crosses sqrt(eps) |r| in this
 * step (d <= sqrt(eps) |r_k| and d_new > sqrt(eps) |r_{k+1}|) and d_new >
 * 1.1 d_init.  Returns 1 when due, 0 otherwise; *d_out = d_new. */
int or_ru_trigger_step(double eps, double d, double d_init, double r_k, double r_k1, double alpha_ap, double *d_out)
{
    const double h = sqrt(eps);
    const double dn = d + eps * (r_k1 + alpha_ap);
    *d_out = dn;
    return d <= h * r_k && dn > h * r_k1 && dn > 1.1 * d_init;
}

/* The first step k (0-based: the step from r_k to r_{k+1}) at which the
 * trigger fires on the sequences r[0..n] and alpha_ap[0..n-1], starting from
 * d = d_init = eps r[0]; -1 if it never does. */
int or_ru_trigger_first(int n, const double *r, const double *alpha_ap, double eps)
{
    double d = eps * r[0];
    const double d_init = d;
    for (int k = 0; k < n; k++)
        if (or_ru_trigger_step(eps, d, d_init, r[k], r[k + 1], alpha_ap[k], &d)) return k;
    return -1;
}

int or_mixed_cg(const int *L, const double *fat, const double *lng, const double *fat_s,
                const double *lng_s, double m, int sfmt, const double *b_, double *x_, double tol,
                double delta, double dyn_eps, int nbuf, int opts, int maxiter, int *iters, int *reliable,
                double *true_res, double *hist)
{
    op_t op = {L, fat, lng, m, 0.0, 0}, ops = {L, fat_s, lng_s, m, 0.0, 0};
    const int64_t n = op_len(&op), ns = n / 3;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    if (nbuf < 1) nbuf = 1;
    cplx *r = malloc(sizeof(cplx) * n), *r_old = malloc(sizeof(cplx) * n), *rh = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *ring = malloc(sizeof(cplx) * n * nbuf);
    double *al = malloc(sizeof(double) * nbuf);
    int nring = 0;
#define STORE(dst, src) or_spinor_emulate(ns, sfmt, (const double *)(src), (double *)(dst))
#define FLUSH()                                                                 \
    do {                                                                        \
        for (int j_ = 0; j_ < nring; j_++)                                      \
            for (int64_t i_ = 0; i_ < n; i_++) x[i_] += al[j_] * ring[(int64_t)j_ * n + i_]; \
        nring = 0;                                                              \
    } while (0)
    memset(x, 0, sizeof(cplx) * n);
    const double bb = nrm2(n, b);
    memcpy(rh, b, sizeof(cplx) * n); /* r^ = b - A 0 */
    STORE(r, rh);
    memcpy(p, r, sizeof(cplx) * n);
    double rr = nrm2(n, r), rmax = sqrt(rr);
    double d = dyn_eps * sqrt(rr), d_init = d;
    int k = 0, ru = 0, status = 1;
    if (hist) hist[0] = sqrt(rr / bb);
    if (sqrt(nrm2(n, rh)) <= tol * sqrt(bb)) status = 0;
    while (status == 1 && k < maxiter) {
        op_apply(&ops, p, t);
        STORE(Ap, t);
        const double pAp = creal(cdot(n, p, Ap));
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            status = 2;
            break;
        }
        const double alpha = rr / pAp;
        memcpy(ring + (int64_t)nring * n, p, sizeof(cplx) * n);
        al[nring++] = alpha;
        memcpy(r_old, r, sizeof(cplx) * n);
        for (int64_t i = 0; i < n; i++) t[i] = r[i] - alpha * Ap[i];
        STORE(r, t);
        const double rr_new = nrm2(n, r);
        k++;
        if (hist) hist[k] = sqrt(rr_new / bb);
        if (nring == nbuf) FLUSH();
        int trigger = sqrt(rr_new) <= tol * sqrt(bb);
        if (dyn_eps > 0.0) {
            double d_new = d;
            trigger = or_ru_trigger_step(dyn_eps, d, d_init, sqrt(rr), sqrt(rr_new),
                                         fabs(alpha) * sqrt(nrm2(n, Ap)), &d_new) || trigger;
            d = d_new;
        } else {
            trigger = trigger || sqrt(rr_new) < delta * rmax;
        }
        if (sqrt(rr_new) > rmax) rmax = sqrt(rr_new);
        if (trigger) {
            FLUSH();
            op_apply(&op, x, t);
            for (int64_t i = 0; i < n; i++) rh[i] = b[i] - t[i];
            const double hh = nrm2(n, rh);
            ru++;
            if (hist) hist[k] = sqrt(hh / bb);
            d = d_init = dyn_eps * sqrt(hh);
            if (sqrt(hh) <= tol * sqrt(bb)) {
                status = 0;
                break;
            }
            if (opts & 2) {
                const cplx c = cdot(n, rh, p) / hh;
                for (int64_t i = 0; i < n; i++) p[i] -= c * rh[i];
            }
            const double beta = hh / rr;
            for (int64_t i = 0; i < n; i++) t[i] = rh[i] + beta * p[i];
            STORE(p, t);
            STORE(r, rh);
            rr = hh;
            rmax = sqrt(hh);
            continue;
        }
        const double beta = (opts & 1) ? (rr_new - creal(cdot(n, r, r_old))) / rr : rr_new / rr;
        if (!isfinite(beta)) {
            status = 2;
            break;
        }
        for (int64_t i = 0; i < n; i++) t[i] = r[i] + beta * p[i];
        STORE(p, t);
        rr = rr_new;
    }
    FLUSH();
#undef STORE
#undef FLUSH
    op_apply(&op, x, t);
    for (int64_t i = 0; i < n; i++) rh[i] = b[i] - t[i];
    *true_res = sqrt(nrm2(n, rh) / bb);
    *iters = k;
    *reliable = ru;
    free(r);
    free(r_old);
    free(rh);
    free(p);
    free(Ap);
    free(t);
    free(ring);
    free(al);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O7 multi-shift CG (Sec. 3.2; Jegerlehner, hep-lat/9612014), FP64          */
/* ------------------------------------------------------------------------ */
/* Solves (M_ee + sigma_i) x_i = b for i < nshift with sigma_0 the base shift.
 * With A = M_ee + sigma_0 and s_i = sigma_i - sigma_0 the shifted residuals
 * stay co-linear with the base one, r_i = zeta_i r, and
 *   zeta_i' = zeta_i zeta_i^- alpha^- /
 *             (alpha beta^- (zeta_i^- - zeta_i) + zeta_i^- alpha^- (1 + s_i alpha))
 *   alpha_i = alpha zeta_i'/zeta_i,  beta_i = beta (zeta_i'/zeta_i)^2,
 *   x_i += alpha_i p_i,  p_i = zeta_i' r + beta_i p_i,
 * starting from zeta = zeta^- = 1, alpha^- = 1, beta^- = 0.  Shift i stops
 * updating once zeta_i |r| <= tol_i |b|; the solve ends when every shift has
 * stopped.  x is [nshift][Vh][3][2]; zeta_out[i] receives the final zeta_i,
 * iters_out[i] the iteration at which shift i stopped; r_out (may be NULL)
 * the final base residual.  Returns 0 on convergence, 1 at maxiter, 2 for
 * an unsupported shift count (1..64). */
int or_multishift_cg(const int *L, const double *fat, const double *lng, double m,
                     int nshift, const double *sigma, const double *tol,
                     const double *b_, double *x_, int maxiter,
                     int *iters_out, double *zeta_out, double *r_out)
{
    if (nshift < 1 || nshift > 64) return 2;
    op_t op = {L, fat, lng, m, sigma[0], 0};
    const int64_t n = op_len(&op);
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n * nshift);
    double *z = malloc(sizeof(double) * nshift), *zm = malloc(sizeof(double) * nshift);
    int *live = malloc(sizeof(int) * nshift);
    memcpy(r, b, sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n * nshift);
    for (int i = 0; i < nshift; i++) {
        memcpy(p + i * n, b, sizeof(cplx) * n);
        z[i] = zm[i] = 1.0;
        live[i] = 1;
        iters_out[i] = 0;
    }
    const double bnorm = sqrt(nrm2(n, b));
    double rr = nrm2(n, r), alpha_m = 1.0, beta_m = 0.0;
    int k = 0, nlive = nshift;
    while (nlive > 0 && k < maxiter) {
        op_apply(&op, p, w);
        const double alpha = rr / creal(cdot(n, p, w));
        double zn[64], ai[64];
        for (int i = 0; i < nshift; i++) {
            if (!live[i]) continue;
            const double s = sigma[i] - sigma[0];
            zn[i] = z[i] * zm[i] * alpha_m /
                    (alpha * beta_m * (zm[i] - z[i]) + zm[i] * alpha_m * (1.0 + s * alpha));
            ai[i] = alpha * zn[i] / z[i];
            for (int64_t j = 0; j < n; j++) x[i * n + j] += ai[i] * p[i * n + j];
        }
        for (int64_t j = 0; j < n; j++) r[j] -= alpha * w[j];
        const double rr_new = nrm2(n, r);
        const double beta = rr_new / rr;
        k++;
        for (int i = 0; i < nshift; i++) {
            if (!live[i]) continue;
            const double bi = beta * (zn[i] / z[i]) * (zn[i] / z[i]);
            for (int64_t j = 0; j < n; j++) p[i * n + j] = zn[i] * r[j] + bi * p[i * n + j];
            zm[i] = z[i];
            z[i] = zn[i];
            if (fabs(z[i]) * sqrt(rr_new) <= tol[i] * bnorm) {
                live[i] = 0;
                iters_out[i] = k;
                nlive--;
            }
        }
        rr = rr_new;
        alpha_m = alpha;
        beta_m = beta;
    }
    for (int i = 0; i < nshift; i++) {
        zeta_out[i] = z[i];
        if (live[i]) iters_out[i] = k;
    }
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    free(r);
    free(w);
    free(p);
    free(z);
    free(zm);
    free(live);
    return nlive > 0 ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* O10 multi-shift stage with emulated sloppy storage (Sec. 3.2)              */
/* ------------------------------------------------------------------------ */
/* The multi-shift recurrences of or_multishift_cg with every write of a
 * sloppy vector (r, A p, p_i) rounded through spinor format sfmt, the sloppy
 * operator applied with (fat_s, lng_s) and, in the readings used throughout:
 * base system = sigma[0] (the smallest shift; the caller sorts); a
 * reliable update of the base system when |r| < delta * max|r| since the
 * last one (the FP64 true residual of x_0 with the exact links replaces r,
 * Fletcher-Reeves beta, the shifted p_i kept); shift i > 0 stops updating
 * once |zeta_i| |r| <= max(tol_i, 10 eps) |b| with eps the format's relative
 * precision (eps_fmt); the stage ends when every shift but the base has
 * stopped.  The x_i accumulate in FP64 here.  x is [nshift][Vh][3][2];
 * shift_iters[i] the iteration at which shift i stopped (the stage's length
 * for the base); resid[i] = |b - (M_ee + sigma_i) x_i| / |b| with the exact
 * links after the stage (before any refinement).  Returns 0 when every
 * shift but the base stopped, 1 at maxiter, 2 on breakdown or a bad shift
 * count (1..64); *iters the stage's iterations, *reliable its reliable
 * updates. */
int or_mixed_multishift(const int *L, const double *fat, const double *lng, const double *fat_s,
                        const double *lng_s, double m, int nshift, const double *sigma,
                        const double *tol, int sfmt, double eps_fmt, const double *b_, double *x_,
                        double delta, int maxiter, int *iters, int *reliable, int *shift_iters,
                        double *resid)
{
    if (nshift < 1 || nshift > 64) return 2;
    op_t op = {L, fat, lng, m, sigma[0], 0}, ops = {L, fat_s, lng_s, m, sigma[0], 0};
    const int64_t n = op_len(&op), ns = n / 3;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n * nshift);
    double z[64], zm[64], zn[64];
    int live[64];
#define STORE(dst, src) or_spinor_emulate(ns, sfmt, (const double *)(src), (double *)(dst))
    STORE(r, b);
    memset(x, 0, sizeof(cplx) * n * nshift);
    for (int i = 0; i < nshift; i++) {
        memcpy(p + i * n, r, sizeof(cplx) * n);
        z[i] = zm[i] = 1.0;
        live[i] = 1;
        shift_iters[i] = 0;
    }
    const double bnorm = sqrt(nrm2(n, b));
    double rr = nrm2(n, r), rmax = sqrt(rr), alpha_m = 1.0, beta_m = 0.0;
    int k = 0, ru = 0, nlive = nshift - 1, status = 1;
    if (nlive == 0) status = 0;
    while (status == 1 && k < maxiter) {
        op_apply(&ops, p, t);
        STORE(w, t);
        const double pAp = creal(cdot(n, p, w));
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            status = 2;
            break;
        }
        const double alpha = rr / pAp;
        for (int i = 0; i < nshift; i++) {
            if (!live[i]) continue;
            const double s = sigma[i] - sigma[0];
            zn[i] = z[i] * zm[i] * alpha_m /
                    (alpha * beta_m * (zm[i] - z[i]) + zm[i] * alpha_m * (1.0 + s * alpha));
            const double ai = alpha * zn[i] / z[i];
            for (int64_t j = 0; j < n; j++) x[i * n + j] += ai * p[i * n + j];
        }
        for (int64_t j = 0; j < n; j++) t[j] = r[j] - alpha * w[j];
        STORE(r, t);
        double rr_new = nrm2(n, r);
        k++;
        if (sqrt(rr_new) < delta * rmax) {
            /* reliable update of the base system */
            op_apply(&op, x, t);
            for (int64_t j = 0; j < n; j++) t[j] = b[j] - t[j];
            STORE(r, t);
            rr_new = nrm2(n, t);
            rmax = sqrt(rr_new);
            ru++;
        } else if (sqrt(rr_new) > rmax) {
            rmax = sqrt(rr_new);
        }
        const double beta = rr_new / rr;
        for (int i = 0; i < nshift; i++) {
            if (!live[i]) continue;
            const double bi = beta * (zn[i] / z[i]) * (zn[i] / z[i]);
            for (int64_t j = 0; j < n; j++) t[j] = zn[i] * r[j] + bi * p[i * n + j];
            STORE(p + i * n, t);
            zm[i] = z[i];
            z[i] = zn[i];
            if (i > 0 && fabs(z[i]) * sqrt(rr_new) <= fmax(tol[i], 10.0 * eps_fmt) * bnorm) {
                live[i] = 0;
                shift_iters[i] = k;
                nlive--;
            }
        }
        rr = rr_new;
        alpha_m = alpha;
        beta_m = beta;
        if (nlive == 0) status = 0;
    }
#undef STORE
    shift_iters[0] = k;
    for (int i = 1; i < nshift; i++)
        if (live[i]) shift_iters[i] = k;
    for (int i = 0; i < nshift; i++) {
        op_t oi = {L, fat, lng, m, sigma[i], 0};
        op_apply(&oi, x + i * n, t);
        for (int64_t j = 0; j < n; j++) t[j] = b[j] - t[j];
        resid[i] = sqrt(nrm2(n, t)) / bnorm;
    }
    *iters = k;
    *reliable = ru;
    free(r);
    free(w);
    free(t);
    free(p);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Full-system solve by even/odd reduction (Sec. 3; the step either side of  */
/* the even/odd solvers)                                                     */
/* ------------------------------------------------------------------------ */
/* With M = 2m + D split into parity blocks [[2m, D_eo], [D_oe, 2m]], the odd
 * unknowns are eliminated: from the odd rows x_o = (b_o - D_oe x_e) / (2m),
 * and substituting into the even rows and multiplying by 2m gives
 *   (4m^2 - D_eo D_oe) x_e = 2m b_e - D_eo b_o,
 * i.e. M_ee x_e = bt_e.  For any x_e and x_o reconstructed from it, the full
 * residual is zero on the odd sites and equals (bt_e - M_ee x_e) / (2m) on the
 * even ones.  b, x: full-lattice fields [parity][cb][color]. */
void or_schur_source(const int *L, const double *fat, const double *lng, double m, const double *b,
                     double *bt)
{
    const int64_t n = vol_of(L) / 2 * 3;
    const cplx *be = (const cplx *)b, *bo = be + n;
    cplx *t = (cplx *)bt;
    or_dslash(L, fat, lng, 0, (const double *)bo, bt); /* D_eo b_o */
    for (int64_t i = 0; i < n; i++) t[i] = 2.0 * m * be[i] - t[i];
}

/* x_o = (b_o - D_oe x_e) / (2m); b_o, x_e, x_o are half-lattice fields. */
void or_reconstruct_odd(const int *L, const double *fat, const double *lng, double m, const double *b_o,
                        const double *x_e, double *x_o)
{
    const int64_t n = vol_of(L) / 2 * 3;
    const cplx *bo = (const cplx *)b_o;
    cplx *xo = (cplx *)x_o;
    or_dslash(L, fat, lng, 1, x_e, x_o); /* D_oe x_e */
    for (int64_t i = 0; i < n; i++) xo[i] = (bo[i] - xo[i]) / (2.0 * m);
}

/* Solves (2m + D) x = b on the full lattice: textbook CG (or_cg) on
 * M_ee x_e = bt_e to the Schur tolerance tol * 2|m| |b| / |bt_e| (the even
 * residual of the full system is the Schur residual over 2m, the odd one is
 * zero), then the odd reconstruction.  *true_res = |b - M x| / |b|.  Returns
 * or_cg's status (0 converged, 1 maxiter, 2 breakdown); m must be nonzero. */
int or_solve_full(const int *L, const double *fat, const double *lng, double m, const double *b_,
                  double *x_, double tol, int maxiter, int *iters, double *true_res)
{
    const int64_t n = vol_of(L) / 2 * 3;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *bt = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * 2 * n);
    or_schur_source(L, fat, lng, m, b_, (double *)bt);
    const double bb = nrm2(2 * n, b), btn = sqrt(nrm2(n, bt));
    int status = 0;
    double tr_schur = 0.0;
    *iters = 0;
    if (btn > 0.0) {
        const double tol_s = tol * 2.0 * fabs(m) * sqrt(bb) / btn;
        status = or_cg(L, fat, lng, m, 0.0, (const double *)bt, x_, tol_s, maxiter, 0, iters, &tr_schur);
    } else {
        memset(x, 0, sizeof(cplx) * n);
    }
    or_reconstruct_odd(L, fat, lng, m, (const double *)(b + n), x_, (double *)(x + n));
    or_mfull(L, fat, lng, m, x_, (double *)r);
    for (int64_t i = 0; i < 2 * n; i++) r[i] = b[i] - r[i];
    *true_res = bb > 0.0 ? sqrt(nrm2(2 * n, r) / bb) : 0.0;
    free(bt);
    free(r);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O8 BiCGStab(l) (Sec. 6.1; Sleijpen and Fokkema 1993), FP64                */
/* ------------------------------------------------------------------------ */
/* Solves (2m + D) x = b on the full lattice from x = 0 with shadow residual
 * r~ = r_0.  Each cycle takes l BiCG steps and then minimises the residual
 * over the l new directions by modified Gram-Schmidt.  Stops when |r| <=
 * tol |b| (checked once per cycle).  *matvecs counts operator applications;
 * *true_res = |b - M x|/|b|.  Returns 0 on convergence, 1 at maxiter
 * (counted in matvecs), 2 on breakdown. */
int or_bicgstabl(const int *L, const double *fat, const double *lng, double m, int l,
                 const double *b_, double *x_, double tol, int max_matvecs,
                 int *matvecs, double *true_res)
{
    op_t op = {L, fat, lng, m, 0.0, 1};
    const int64_t n = op_len(&op);
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    if (l < 1 || l > 16) return 2;
    cplx *R = malloc(sizeof(cplx) * n * (l + 1)); /* r_0..r_l */
    cplx *U = malloc(sizeof(cplx) * n * (l + 1)); /* u_0..u_l */
    cplx *rt = malloc(sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n);
    memcpy(R, b, sizeof(cplx) * n);
    memcpy(rt, b, sizeof(cplx) * n);
    memset(U, 0, sizeof(cplx) * n);
    const double bnorm = sqrt(nrm2(n, b));
    cplx rho0 = 1, alpha = 0, omega = 1;
    cplx tau[17][17], gp[17], g[17], gpp[17];
    double sig[17];
    int mv = 0, status = 1;
    if (sqrt(nrm2(n, R)) <= tol * bnorm) status = 0;
    while (status == 1 && mv < max_matvecs) {
        rho0 = -omega * rho0;
        for (int j = 0; j < l; j++) {
            cplx rho1 = cdot(n, rt, R + j * n);
            if (cabs(rho0) == 0.0) { status = 2; break; }
            cplx beta = alpha * rho1 / rho0;
            rho0 = rho1;
            for (int i = 0; i <= j; i++)
                for (int64_t k = 0; k < n; k++) U[i * n + k] = R[i * n + k] - beta * U[i * n + k];
            op_apply(&op, U + j * n, U + (j + 1) * n);
            mv++;
            cplx gam = cdot(n, rt, U + (j + 1) * n);
            if (cabs(gam) == 0.0) { status = 2; break; }
            alpha = rho0 / gam;
            for (int i = 0; i <= j; i++)
                for (int64_t k = 0; k < n; k++) R[i * n + k] -= alpha * U[(i + 1) * n + k];
            op_apply(&op, R + j * n, R + (j + 1) * n);
            mv++;
            for (int64_t k = 0; k < n; k++) x[k] += alpha * U[k];
        }
        if (status == 2) break;
        for (int j = 1; j <= l; j++) {
            for (int i = 1; i < j; i++) {
                tau[i][j] = cdot(n, R + i * n, R + j * n) / sig[i];
                for (int64_t k = 0; k < n; k++) R[j * n + k] -= tau[i][j] * R[i * n + k];
            }
            sig[j] = nrm2(n, R + j * n);
            if (!(sig[j] > 0.0)) { status = 2; break; }
            gp[j] = cdot(n, R + j * n, R) / sig[j];
        }
        if (status == 2) break;
        g[l] = gp[l];
        omega = g[l];
        for (int j = l - 1; j >= 1; j--) {
            cplx s = 0;
            for (int i = j + 1; i <= l; i++) s += tau[j][i] * g[i];
            g[j] = gp[j] - s;
        }
        for (int j = 1; j <= l - 1; j++) {
            cplx s = 0;
            for (int i = j + 1; i <= l - 1; i++) s += tau[j][i] * g[i + 1];
            gpp[j] = g[j + 1] + s;
        }
        for (int64_t k = 0; k < n; k++) {
            x[k] += g[1] * R[k];
            R[k] -= gp[l] * R[l * n + k];
            U[k] -= g[l] * U[l * n + k];
        }
        for (int j = 1; j <= l - 1; j++)
            for (int64_t k = 0; k < n; k++) {
                U[k] -= g[j] * U[j * n + k];
                x[k] += gpp[j] * R[j * n + k];
                R[k] -= gp[j] * R[j * n + k];
            }
        if (sqrt(nrm2(n, R)) <= tol * bnorm) status = 0;
    }
    cplx *t = U; /* reuse as scratch */
    op_apply(&op, x, t);
    for (int64_t k = 0; k < n; k++) t[k] = b[k] - t[k];
    *true_res = sqrt(nrm2(n, t)) / bnorm;
    *matvecs = mv;
    free(R);
    free(U);
    free(rt);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O10 BiCGStab(l) with emulated sloppy storage (Sec. 6.1, Table 2)           */
/* ------------------------------------------------------------------------ */
/* The cycle of or_bicgstabl on M = 2m + D with every write of r_0..r_l and
 * u_0..u_l rounded through spinor format sfmt and the operator applied with
 * the sloppy links (fat_s, lng_s); x accumulates in FP64.  In the reading used
 * throughout (the CG trigger): at the end of a cycle, when |r_0| < delta *
 * max|r_0| since the last reliable update or |r_0| <= tol |b|, the FP64 true
 * residual b - M x with the exact links replaces r_0 (u_0, rho, alpha and
 * omega are kept) and the solve ends if it meets tol.  Returns 0 on
 * convergence, 1 at max_matvecs, 2 on breakdown; *matvecs counts sloppy
 * operator applications, *reliable the reliable updates. */
int or_mixed_bicgstabl(const int *L, const double *fat, const double *lng, const double *fat_s,
                       const double *lng_s, double m, int l, int sfmt, const double *b_, double *x_,
                       double tol, double delta, int max_matvecs, int *matvecs, int *reliable,
                       double *true_res)
{
    op_t op = {L, fat, lng, m, 0.0, 1}, ops = {L, fat_s, lng_s, m, 0.0, 1};
    const int64_t n = op_len(&op), ns = n / 3;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    if (l < 1 || l > 16) return 2;
    cplx *R = malloc(sizeof(cplx) * n * (l + 1)); /* r_0..r_l */
    cplx *U = malloc(sizeof(cplx) * n * (l + 1)); /* u_0..u_l */
    cplx *rt = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
#define STORE(dst) or_spinor_emulate(ns, sfmt, (const double *)(dst), (double *)(dst))
    memset(x, 0, sizeof(cplx) * n);
    memcpy(R, b, sizeof(cplx) * n);
    STORE(R);
    memcpy(rt, R, sizeof(cplx) * n);
    memset(U, 0, sizeof(cplx) * n);
    const double bnorm = sqrt(nrm2(n, b));
    cplx rho0 = 1, alpha = 0, omega = 1;
    cplx tau[17][17], gp[17], g[17], gpp[17];
    double sig[17];
    double rmax = sqrt(nrm2(n, R));
    int mv = 0, ru = 0, status = 1;
    if (rmax <= tol * bnorm) status = 0;
    while (status == 1 && mv < max_matvecs) {
        rho0 = -omega * rho0;
        for (int j = 0; j < l; j++) {
            cplx rho1 = cdot(n, rt, R + j * n);
            if (cabs(rho0) == 0.0) { status = 2; break; }
            cplx beta = alpha * rho1 / rho0;
            rho0 = rho1;
            for (int i = 0; i <= j; i++) {
                for (int64_t k = 0; k < n; k++) U[i * n + k] = R[i * n + k] - beta * U[i * n + k];
                STORE(U + i * n);
            }
            op_apply(&ops, U + j * n, U + (j + 1) * n);
            STORE(U + (j + 1) * n);
            mv++;
            cplx gam = cdot(n, rt, U + (j + 1) * n);
            if (cabs(gam) == 0.0) { status = 2; break; }
            alpha = rho0 / gam;
            for (int i = 0; i <= j; i++) {
                for (int64_t k = 0; k < n; k++) R[i * n + k] -= alpha * U[(i + 1) * n + k];
                STORE(R + i * n);
            }
            op_apply(&ops, R + j * n, R + (j + 1) * n);
            STORE(R + (j + 1) * n);
            mv++;
            for (int64_t k = 0; k < n; k++) x[k] += alpha * U[k];
        }
        if (status == 2) break;
        for (int j = 1; j <= l; j++) {
            for (int i = 1; i < j; i++) {
                tau[i][j] = cdot(n, R + i * n, R + j * n) / sig[i];
                for (int64_t k = 0; k < n; k++) R[j * n + k] -= tau[i][j] * R[i * n + k];
            }
            STORE(R + j * n);
            sig[j] = nrm2(n, R + j * n);
            if (!(sig[j] > 0.0)) { status = 2; break; }
            gp[j] = cdot(n, R + j * n, R) / sig[j];
        }
        if (status == 2) break;
        g[l] = gp[l];
        omega = g[l];
        for (int j = l - 1; j >= 1; j--) {
            cplx s = 0;
            for (int i = j + 1; i <= l; i++) s += tau[j][i] * g[i];
            g[j] = gp[j] - s;
        }
        for (int j = 1; j <= l - 1; j++) {
            cplx s = 0;
            for (int i = j + 1; i <= l - 1; i++) s += tau[j][i] * g[i + 1];
            gpp[j] = g[j + 1] + s;
        }
        for (int64_t k = 0; k < n; k++) {
            x[k] += g[1] * R[k];
            R[k] -= gp[l] * R[l * n + k];
            U[k] -= g[l] * U[l * n + k];
        }
        for (int j = 1; j <= l - 1; j++)
            for (int64_t k = 0; k < n; k++) {
                U[k] -= g[j] * U[j * n + k];
                x[k] += gpp[j] * R[j * n + k];
                R[k] -= gp[j] * R[j * n + k];
            }
        STORE(R);
        STORE(U);
        if (!isfinite(creal(omega)) || !isfinite(cimag(omega))) { status = 2; break; }
        const double rn = sqrt(nrm2(n, R));
        if (rn < delta * rmax || rn <= tol * bnorm) {
            op_apply(&op, x, t);
            for (int64_t k = 0; k < n; k++) t[k] = b[k] - t[k];
            const double hn = sqrt(nrm2(n, t));
            ru++;
            if (hn <= tol * bnorm) {
                status = 0;
                break;
            }
            memcpy(R, t, sizeof(cplx) * n);
            STORE(R);
            rmax = hn;
        } else if (rn > rmax) {
            rmax = rn;
        }
    }
#undef STORE
    op_apply(&op, x, t);
    for (int64_t k = 0; k < n; k++) t[k] = b[k] - t[k];
    *true_res = sqrt(nrm2(n, t)) / bnorm;
    *matvecs = mv;
    *reliable = ru;
    free(R);
    free(U);
    free(rt);
    free(t);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O9 dense reference                                                        */
/* ------------------------------------------------------------------------ */
/* Column k of the operator applied to unit vector e_k (complex, column-major
 * A[k*n + i] = (A e_k)_i).  which = 0: M_ee + sigma; 1: M = 2m + D full;
 * 2: the stencil D_eo (rows even, columns odd); 3: D_oe. */
void or_dense(const int *L, const double *fat, const double *lng, double m, double sigma,
              int which, double *A_)
{
    const int64_t nh = vol_of(L) / 2 * 3;
    const int64_t n = which == 1 ? 2 * nh : nh;
    cplx *A = (cplx *)A_;
    cplx *e = calloc(n, sizeof(cplx));
    op_t op = {L, fat, lng, m, sigma, which == 1};
    for (int64_t k = 0; k < n; k++) {
        e[k] = 1.0;
        if (which <= 1)
            op_apply(&op, e, A + k * n);
        else
            or_dslash(L, fat, lng, which == 2 ? 0 : 1, (const double *)e, (double *)(A + k * n));
        e[k] = 0.0;
    }
    free(e);
}

/* Solves A y = rhs in place (y overwrites rhs) by LU with partial pivoting;
 * A is complex column-major n x n and is overwritten.  Returns 0, or 1 if a
 * pivot is exactly zero. */
int or_lu_solve(int64_t n, double *A_, double *rhs_)
{
    cplx *A = (cplx *)A_, *y = (cplx *)rhs_;
#define AE(i, j) A[(j) * n + (i)]
    for (int64_t k = 0; k < n; k++) {
        int64_t piv = k;
        double best = cabs(AE(k, k));
        for (int64_t i = k + 1; i < n; i++)
            if (cabs(AE(i, k)) > best) {
                best = cabs(AE(i, k));
                piv = i;
            }
        if (best == 0.0) return 1;
        if (piv != k) {
            for (int64_t j = 0; j < n; j++) {
                cplx t = AE(k, j);
                AE(k, j) = AE(piv, j);
                AE(piv, j) = t;
            }
            cplx t = y[k];
            y[k] = y[piv];
            y[piv] = t;
        }
        for (int64_t i = k + 1; i < n; i++) {
            const cplx f = AE(i, k) / AE(k, k);
            AE(i, k) = f;
            for (int64_t j = k + 1; j < n; j++) AE(i, j) -= f * AE(k, j);
            y[i] -= f * y[k];
        }
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        cplx s = y[i];
        for (int64_t j = i + 1; j < n; j++) s -= AE(i, j) * y[j];
        y[i] = s / AE(i, i);
    }
#undef AE
    return 0;
}
