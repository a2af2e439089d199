// bicgstab.cu -- mixed-precision BiCGStab(l) (Sec. 6.1; Sleijpen and Fokkema)
// on the full-lattice operator M = 2m + D, and its C-ABI entry point.
//
// Each cycle: l BiCG steps (two matvecs each) followed by a minimal-residual
// step over the l new directions, orthogonalised by modified Gram-Schmidt.
// Vectors r_0..r_l, u_0..u_l and the shadow residual live in the sloppy
// format; x, b and true residuals in FP64; every scalar (rho, alpha, omega,
// the Gram-Schmidt coefficients tau, sigma, gamma) is computed on the device
// by the reducing kernels' finishers, so a cycle is one fixed kernel sequence
// (captured once as a CUDA graph).  A reliable update (FP64 true residual)
// ends a cycle when |r| has dropped below delta times its maximum since the
// previous one, or when the iterated residual meets the target.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <vector>

#include "blas.h"
#include "cg.h"
#include "codecs.cuh"
#include "internal.h"
#include "launch.cuh"
#include "reduce.cuh"

namespace hisq {

namespace {

constexpr int kMaxL = 8;
constexpr int kBlock = 256;
constexpr int kBSites = 2;  // sites a thread of the reductions loads before using any (in flight together)

struct BState {
    double rho_re, rho_im;         // rho_0
    double alpha_re, alpha_im;
    double omega_re, omega_im;
    double beta_re, beta_im;
    double tau_re[kMaxL + 1][kMaxL + 1], tau_im[kMaxL + 1][kMaxL + 1];
    double sigma[kMaxL + 1];
    double gp_re[kMaxL + 1], gp_im[kMaxL + 1];    // gamma'
    double g_re[kMaxL + 1], g_im[kMaxL + 1];      // gamma
    double gpp_re[kMaxL + 1], gpp_im[kMaxL + 1];  // gamma''
    double rr, rr_max, delta2, stop2, tiny2;
    double rt2;   // |rt|^2 of the shadow residual
    double brk2;  // breakdown when |<rt, v>|^2 <= brk2 |rt|^2 |v|^2
    int active, reason, cycles, l;
};

enum { OP_RHO = 1, OP_GAMMA = 2, OP_TAU = 3, OP_SIGMA = 4, OP_FINAL = 5 };

struct BArgs {
    int vh;
    size_t hb;               // bytes of one half-lattice sloppy field
    size_t fb;               // bytes of one full sloppy field (2 halves)
    char *R;                 // r_0..r_l, fb apart
    char *U;                 // u_0..u_l
    const char *rt;          // shadow residual
    double *x64;             // FP64 full field (two planar halves, 48*vh bytes each)
    int j, i;                // step indices
    int op;
    BState *b;
    const int *active;
    int *err;
    RedBuf red;
};

__device__ __forceinline__ bool skip(const int *active) { return active && *(volatile const int *)active == 0; }

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double &qr, double &qi)
{
    const double d = br * br + bi * bi;
    qr = (ar * br + ai * bi) / d;
    qi = (ai * br - ar * bi) / d;
}

__device__ void b_stop(BState *b, int reason)
{
    b->reason = reason;
    b->active = 0;
}

// finishers of the reducing kernels; sums = {Re<x,y>, Im<x,y>, extra}
__device__ void b_finish(BArgs &a, const double *s)
{
    BState *b = a.b;
    if (a.op == OP_RHO) {
        // rho1 = <rt, r_j>; beta = alpha rho1 / rho0; rho0 = rho1.  Breakdown:
        // rho1 (nearly) orthogonal relative to |rt| |r_j| (sums[2] = |r_j|^2),
        // or a rho0 too small to divide by
        const double n2 = s[0] * s[0] + s[1] * s[1];
        if (b->rho_re * b->rho_re + b->rho_im * b->rho_im <= b->tiny2 ||
            (s[2] > 0.0 && !(n2 > b->brk2 * b->rt2 * s[2])) || !isfinite(n2)) {
            b_stop(b, REASON_BREAKDOWN);
            return;
        }
        double qr, qi;
        cdiv(s[0], s[1], b->rho_re, b->rho_im, qr, qi);
        b->beta_re = b->alpha_re * qr - b->alpha_im * qi;
        b->beta_im = b->alpha_re * qi + b->alpha_im * qr;
        b->rho_re = s[0];
        b->rho_im = s[1];
    } else if (a.op == OP_GAMMA) {
        // gamma = <rt, u_{j+1}>; alpha = rho0 / gamma; breakdown relative to |rt| |u_{j+1}|
        const double n2 = s[0] * s[0] + s[1] * s[1];
        if (n2 <= b->tiny2 || !(n2 > b->brk2 * b->rt2 * s[2]) || !isfinite(s[0]) || !isfinite(s[1])) {
            b_stop(b, REASON_BREAKDOWN);
            return;
        }
        cdiv(b->rho_re, b->rho_im, s[0], s[1], b->alpha_re, b->alpha_im);
    } else if (a.op == OP_TAU) {
        // tau_ij = <r_i, r_j> / sigma_i
        b->tau_re[a.i][a.j] = s[0] / b->sigma[a.i];
        b->tau_im[a.i][a.j] = s[1] / b->sigma[a.i];
    } else if (a.op == OP_SIGMA) {
        // sums = {Re<r_j, r_0>, Im<r_j, r_0>, |r_j|^2}: sigma_j, gamma'_j
        const double sg = s[2];
        if (!(sg > 0.0) || !isfinite(sg)) {
            b_stop(b, REASON_BREAKDOWN);
            return;
        }
        b->sigma[a.j] = sg;
        b->gp_re[a.j] = s[0] / sg;
        b->gp_im[a.j] = s[1] / sg;
    } else if (a.op == OP_FINAL) {
        // sums = {|r_0|^2}
        const double rr = s[0];
        b->rr = rr;
        b->cycles += 1;
        if (!isfinite(rr)) {
            b_stop(b, REASON_BREAKDOWN);
            return;
        }
        if (rr > b->rr_max) b->rr_max = rr;
        if (rr <= b->stop2)
            b_stop(b, REASON_CONVERGED);
        else if (rr < b->delta2 * b->rr_max)
            b_stop(b, REASON_RELIABLE);
    }
}

// a field of the full lattice = two half-lattice fields; blockIdx.y = parity
__device__ __forceinline__ const char *half(const char *f, size_t hb) { return f + blockIdx.y * hb; }
__device__ __forceinline__ char *half(char *f, size_t hb) { return f + blockIdx.y * hb; }

// rho_0 <- -omega rho_0 (start of a cycle)
__global__ void cycle_start_kernel(BState *b, const int *active)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(active)) return;
    const double r = -(b->omega_re * b->rho_re - b->omega_im * b->rho_im);
    const double i = -(b->omega_re * b->rho_im + b->omega_im * b->rho_re);
    b->rho_re = r;
    b->rho_im = i;
}

// <x, y> = sum conj(x) y over the full lattice (+ |y|^2), then the finisher
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) dot_kernel(BArgs a, const char *x, const char *y)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kBSites, C = Spinor<SF>::chunks;
    const char *xf = half(x, a.hb), *yf = half(y, a.hb);
    real v[3] = {0, 0, 0};
    for (int s0 = blockIdx.x * blockDim.x * U + threadIdx.x; s0 < a.vh; s0 += gridDim.x * blockDim.x * U) {
        uint4 cx[U][C], cy[U][C];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int s = s0 + u * blockDim.x;
            if (s < a.vh) {
                Spinor<SF>::gather(xf, a.vh, s, cx[u]);
                Spinor<SF>::gather(yf, a.vh, s, cy[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (s0 + u * (int)blockDim.x >= a.vh) continue;
            real xv[6], yv[6];
            Spinor<SF>::decode(cx[u], xv);
            Spinor<SF>::decode(cy[u], yv);
            real d0 = 0, d1 = 0, d2 = 0;  // one site in the compute precision (see reduce_grid)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const real xr = xv[2 * c], xi = xv[2 * c + 1], yr = yv[2 * c], yi = yv[2 * c + 1];
                d0 += xr * yr + xi * yi;
                d1 += xr * yi - xi * yr;
                d2 += yr * yr + yi * yi;
            }
            v[0] += d0;
            v[1] += d1;
            v[2] += d2;
        }
    }
    __shared__ double tot[3];
    if (reduce_grid<3>(v, a.red, tot) && threadIdx.x == 0) b_finish(a, tot);
}

// u_i = r_i - beta u_i, i = 0..j
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) u_multi_kernel(BArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    const real br = (real)a.b->beta_re, bi = (real)a.b->beta_im;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.vh; s += gridDim.x * blockDim.x)
    for (int i = 0; i <= a.j; i++) {
        real r[6], u[6];
        Spinor<SF>::load(half(a.R + i * a.fb, a.hb), a.vh, s, r);
        char *uf = half(a.U + i * a.fb, a.hb);
        Spinor<SF>::load(uf, a.vh, s, u);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const real ur = u[2 * c], ui = u[2 * c + 1];
            u[2 * c] = r[2 * c] - (br * ur - bi * ui);
            u[2 * c + 1] = r[2 * c + 1] - (br * ui + bi * ur);
        }
        if (!Spinor<SF>::store(uf, a.vh, s, u)) atomicExch(a.err, 1);
    }
}

// r_i -= alpha u_{i+1}, i = 0..j; x += alpha u_0 (FP64)
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) r_multi_kernel(BArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    const real ar = (real)a.b->alpha_re, ai = (real)a.b->alpha_im;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.vh; s += gridDim.x * blockDim.x) {
    for (int i = 0; i <= a.j; i++) {
        real u[6], r[6];
        Spinor<SF>::load(half(a.U + (i + 1) * a.fb, a.hb), a.vh, s, u);
        char *rf = half(a.R + i * a.fb, a.hb);
        Spinor<SF>::load(rf, a.vh, s, r);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const real ur = u[2 * c], ui = u[2 * c + 1];
            r[2 * c] -= ar * ur - ai * ui;
            r[2 * c + 1] -= ar * ui + ai * ur;
        }
        if (!Spinor<SF>::store(rf, a.vh, s, r)) atomicExch(a.err, 1);
    }
    // x += alpha u_0: the increment in the compute precision, the sum in FP64
    real u0[6];
    double x[6];
    Spinor<SF>::load(half(a.U, a.hb), a.vh, s, u0);
    char *xf = reinterpret_cast<char *>(a.x64) + blockIdx.y * (size_t)48 * a.vh;
    Spinor<S_F64>::load(xf, a.vh, s, x);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        x[2 * c] += (double)(ar * u0[2 * c] - ai * u0[2 * c + 1]);
        x[2 * c + 1] += (double)(ar * u0[2 * c + 1] + ai * u0[2 * c]);
    }
    Spinor<S_F64>::store(xf, a.vh, s, x);
    }
}

// Modified Gram-Schmidt step (j, i): r_j -= tau_{i-1,j} r_{i-1} (i >= 2), then
// tau_ij = <r_i, r_j>/sigma_i (i < j) or sigma_j, gamma'_j (i == j).
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) mgs_kernel(BArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    constexpr int U = kBSites, C = Spinor<SF>::chunks;
    char *rjf = half(a.R + a.j * a.fb, a.hb);
    const char *rpf = half(a.R + (a.i >= 2 ? a.i - 1 : 0) * a.fb, a.hb);
    const int other = a.i < a.j ? a.i : 0;  // <r_i, r_j>, or <r_j, r_0> at i == j
    const char *rof = half(a.R + other * a.fb, a.hb);  // never r_j or r_{i-1}: read before r_j is stored
    const real tr = a.i >= 2 ? (real)a.b->tau_re[a.i - 1][a.j] : real(0);
    const real ti = a.i >= 2 ? (real)a.b->tau_im[a.i - 1][a.j] : real(0);
    real v[3] = {0, 0, 0};
    for (int s0 = blockIdx.x * blockDim.x * U + threadIdx.x; s0 < a.vh; s0 += gridDim.x * blockDim.x * U) {
        uint4 cj[U][C], cp[U][C], co[U][C];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int s = s0 + u * blockDim.x;
            if (s < a.vh) {
                Spinor<SF>::gather(rjf, a.vh, s, cj[u]);
                if (a.i >= 2) Spinor<SF>::gather(rpf, a.vh, s, cp[u]);
                Spinor<SF>::gather(rof, a.vh, s, co[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
        const int s = s0 + u * blockDim.x;
        if (s >= a.vh) continue;
        real rj[6], ri[6];
        Spinor<SF>::decode(cj[u], rj);
        if (a.i >= 2) {
            real rp[6];
            Spinor<SF>::decode(cp[u], rp);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const real pr = rp[2 * c], pi = rp[2 * c + 1];
                rj[2 * c] -= tr * pr - ti * pi;
                rj[2 * c + 1] -= tr * pi + ti * pr;
            }
            if (!Spinor<SF>::store(rjf, a.vh, s, rj)) atomicExch(a.err, 1);
        }
        Spinor<SF>::decode(co[u], ri);
        real d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const real jr = rj[2 * c], ji = rj[2 * c + 1], or_ = ri[2 * c], oi = ri[2 * c + 1];
            if (a.i < a.j) {  // conj(r_i) r_j
                d0 += or_ * jr + oi * ji;
                d1 += or_ * ji - oi * jr;
            } else {          // conj(r_j) r_0
                d0 += jr * or_ + ji * oi;
                d1 += jr * oi - ji * or_;
            }
            d2 += jr * jr + ji * ji;
        }
        v[0] += d0;
        v[1] += d1;
        v[2] += d2;
        }
    }
    __shared__ double tot[3];
    if (reduce_grid<3>(v, a.red, tot) && threadIdx.x == 0) b_finish(a, tot);
}

// gamma_l = gamma'_l, omega = gamma_l; gamma_j = gamma'_j - sum_{i>j} tau_ji gamma_i;
// gamma''_j = gamma_{j+1} + sum_{i=j+1}^{l-1} tau_ji gamma_{i+1}
__global__ void gamma_kernel(BState *b, const int *active)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(active)) return;
    const int l = b->l;
    b->g_re[l] = b->gp_re[l];
    b->g_im[l] = b->gp_im[l];
    b->omega_re = b->g_re[l];
    b->omega_im = b->g_im[l];
    for (int j = l - 1; j >= 1; j--) {
        double sr = 0, si = 0;
        for (int i = j + 1; i <= l; i++) {
            sr += b->tau_re[j][i] * b->g_re[i] - b->tau_im[j][i] * b->g_im[i];
            si += b->tau_re[j][i] * b->g_im[i] + b->tau_im[j][i] * b->g_re[i];
        }
        b->g_re[j] = b->gp_re[j] - sr;
        b->g_im[j] = b->gp_im[j] - si;
    }
    for (int j = 1; j <= l - 1; j++) {
        double sr = 0, si = 0;
        for (int i = j + 1; i <= l - 1; i++) {
            sr += b->tau_re[j][i] * b->g_re[i + 1] - b->tau_im[j][i] * b->g_im[i + 1];
            si += b->tau_re[j][i] * b->g_im[i + 1] + b->tau_im[j][i] * b->g_re[i + 1];
        }
        b->gpp_re[j] = b->g_re[j + 1] + sr;
        b->gpp_im[j] = b->g_im[j + 1] + si;
    }
}

// x += gamma_1 r_0 + sum gamma''_j r_j;  r_0 -= gamma'_l r_l + sum gamma'_j r_j;
// u_0 -= gamma_l u_l + sum gamma_j u_j;  |r_0|^2 -> OP_FINAL
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) final_kernel(BArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    if (skip(a.active)) return;
    const BState *b = a.b;
    const int l = b->l;
    real v[1] = {0};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.vh; s += gridDim.x * blockDim.x) {
        // updates in the compute precision; x's increment is added in FP64
        real dx[6] = {0, 0, 0, 0, 0, 0}, r0[6], u0[6], t[6];
        char *xf = reinterpret_cast<char *>(a.x64) + blockIdx.y * (size_t)48 * a.vh;
        char *r0f = half(a.R, a.hb), *u0f = half(a.U, a.hb);
        Spinor<SF>::load(r0f, a.vh, s, r0);
        Spinor<SF>::load(u0f, a.vh, s, u0);
        auto cax = [](real *y, double cr, double ci, const real *z, real sgn) {
            const real c_r = (real)cr * sgn, c_i = (real)ci * sgn;
            for (int c = 0; c < 3; c++) {
                y[2 * c] += c_r * z[2 * c] - c_i * z[2 * c + 1];
                y[2 * c + 1] += c_r * z[2 * c + 1] + c_i * z[2 * c];
            }
        };
        cax(dx, b->g_re[1], b->g_im[1], r0, real(1));
        Spinor<SF>::load(half(a.R + l * a.fb, a.hb), a.vh, s, t);
        cax(r0, b->gp_re[l], b->gp_im[l], t, real(-1));
        Spinor<SF>::load(half(a.U + l * a.fb, a.hb), a.vh, s, t);
        cax(u0, b->g_re[l], b->g_im[l], t, real(-1));
        for (int j = 1; j <= l - 1; j++) {
            Spinor<SF>::load(half(a.U + j * a.fb, a.hb), a.vh, s, t);
            cax(u0, b->g_re[j], b->g_im[j], t, real(-1));
            Spinor<SF>::load(half(a.R + j * a.fb, a.hb), a.vh, s, t);
            cax(dx, b->gpp_re[j], b->gpp_im[j], t, real(1));
            cax(r0, b->gp_re[j], b->gp_im[j], t, real(-1));
        }
        double x[6];
        Spinor<S_F64>::load(xf, a.vh, s, x);
        for (int k = 0; k < 6; k++) x[k] += (double)dx[k];
        Spinor<S_F64>::store(xf, a.vh, s, x);
        if (!Spinor<SF>::store(r0f, a.vh, s, r0)) atomicExch(a.err, 1);
        if (!Spinor<SF>::store(u0f, a.vh, s, u0)) atomicExch(a.err, 1);
        real n2 = 0;
        for (int k = 0; k < 6; k++) n2 += r0[k] * r0[k];
        v[0] += n2;
    }
    __shared__ double tot[1];
    if (reduce_grid<1>(v, a.red, tot) && threadIdx.x == 0) b_finish(a, tot);
}

// after a reliable update: rr = |r_hi|^2 (sums[0]) and iterate again
__global__ void restart_kernel(BState *b, const double *sum)
{
    pdl_wait();
    pdl_launch_dependents();
    b->rr = sum[0];
    b->rr_max = sum[0];
    b->reason = REASON_NONE;
    b->active = isfinite(sum[0]) ? 1 : 0;
    if (!b->active) b->reason = REASON_BREAKDOWN;
}

// Two rows (parities) of blocks that loop over their parity's sites: one wave
// at kernel K's occupancy (at most 4 blocks per SM per row), so that the end
// of a reducing block is paid once per resident block and no partial second
// wave trails the first (at 47 registers, five blocks fit a SM, not eight).
template <auto K>
dim3 grid2(int vh)
{
    static const int per_row = [] {
        int dev = 0, n = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, K, kBlock, 0);
        const int per_sm = occ < 1 ? 1 : occ > 8 ? 8 : occ;
        const int rows_total = (n > 0 ? n : 1) * per_sm;
        return rows_total / 2 > 0 ? rows_total / 2 : 1;
    }();
    const int need = (vh + kBlock - 1) / kBlock;
    return dim3(need < per_row ? need : per_row, 2);
}

// KERNEL<spinor format, compute type> over both parities of vh sites each.
#define B_LAUNCH(KERNEL, SF, REAL, VH, ...) \
    launch_chained(KERNEL<SF, REAL>, grid2<&KERNEL<SF, REAL>>(VH), dim3(kBlock), st, __VA_ARGS__)
#define B_DISPATCH(SF_, CF_, KERNEL, VH, ...)                                               \
    do {                                                                                    \
        const bool f64_ = (CF_) == HISQ_COMPUTE_F64;                                        \
        switch (SF_) {                                                                      \
        case S_F64: B_LAUNCH(KERNEL, S_F64, double, VH, __VA_ARGS__); break;                \
        case S_F32: B_LAUNCH(KERNEL, S_F32, float, VH, __VA_ARGS__); break;                 \
        case S_HALF: B_LAUNCH(KERNEL, S_HALF, float, VH, __VA_ARGS__); break;               \
        case S_INT20: B_LAUNCH(KERNEL, S_INT20, float, VH, __VA_ARGS__); break;             \
        case S_INT14: B_LAUNCH(KERNEL, S_INT14, float, VH, __VA_ARGS__); break;             \
        case S_INT30:                                                                       \
            if (f64_) B_LAUNCH(KERNEL, S_INT30, double, VH, __VA_ARGS__);                   \
            else B_LAUNCH(KERNEL, S_INT30, float, VH, __VA_ARGS__);                         \
            break;                                                                          \
        }                                                                                   \
    } while (0)

struct BRun {
    hisq_ctx *c;
    hisq_gauge *g;
    const hisq_solver_params &p;
    cudaStream_t st;
    Workspace ws;
    int vh, l;
    size_t hb, fb;
    char *R = nullptr, *U = nullptr, *rt = nullptr;
    double *x64 = nullptr, *r64 = nullptr, *ax64 = nullptr;
    double *park = nullptr;  // the even half's |r|^2 while the odd half is reduced
    BState *b = nullptr, *bh = nullptr;
    GaugeView gv_s{}, gv_d{};
    int mv = 0, mv_hi = 0, ru = 0;

    BRun(hisq_ctx *c_, hisq_gauge *g_, const hisq_solver_params &p_, cudaStream_t s_)
        : c(c_), g(g_), p(p_), st(s_), ws(c_, s_), vh(g_->geom.vh), l(p_.l)
    {
    }
    ~BRun()
    {
        if (bh) cudaFreeHost(bh);
    }

    BArgs args() const
    {
        BArgs a{};
        a.vh = vh;
        a.hb = hb;
        a.fb = fb;
        a.R = R;
        a.U = U;
        a.rt = rt;
        a.x64 = x64;
        a.b = b;
        a.active = &b->active;
        a.err = cur_err(c);
        a.red = cur_red(c);
        return a;
    }

    double sbytes() const { return spinor_site_bytes(p.sloppy.spinor) * 2.0 * vh; }

    // out = 2m in + D in on the full lattice (two half-lattice passes)
    void mfull(const hisq_prec &pr, const GaugeView &gv, const char *in, char *out, size_t half_bytes,
               const int *active, int kind)
    {
        for (int po = 0; po < 2; po++) {
            DslashArgs d{};
            d.g = g->geom;
            d.gv = gv;
            d.err = cur_err(c);
            d.red = cur_red(c);
            d.active = active;
            d.out_parity = po;
            d.in = in + (1 - po) * half_bytes;
            d.out = out + po * half_bytes;
            d.y = in + po * half_bytes;
            d.a = 2.0 * p.mass;
            d.sign = 1;
            d.xpay = 1;
            LaunchScope ls(c, st, kind, stencil_bytes(pr, vh, true));
            launch_dslash(pr.gauge, pr.spinor, pr.compute, pr.long_recon, false, d, st);
        }
    }

    void dot(const char *x, const char *y, int op, int j, int i)
    {
        BArgs a = args();
        a.op = op;
        a.j = j;
        a.i = i;
        LaunchScope ls(c, st, PROF_BLAS, 2.0 * sbytes());
        B_DISPATCH(p.sloppy.spinor, p.sloppy.compute, dot_kernel, vh, a, x, y);
    }

    void cycle()
    {
        const int *act = &b->active;
        {
            LaunchScope ls(c, st, PROF_BLAS, 0.0);
            launch_chained(cycle_start_kernel, dim3(1), dim3(1), st, b, act);
        }
        for (int j = 0; j < l; j++) {
            dot(rt, R + j * fb, OP_RHO, j, 0);
            BArgs a = args();
            a.j = j;
            {
                LaunchScope ls(c, st, PROF_BLAS, 3.0 * (j + 1) * sbytes());
                B_DISPATCH(p.sloppy.spinor, p.sloppy.compute, u_multi_kernel, vh, a);
            }
            mfull(p.sloppy, gv_s, U + j * fb, U + (j + 1) * fb, hb, act, PROF_STENCIL);
            dot(rt, U + (j + 1) * fb, OP_GAMMA, j, 0);
            {
                LaunchScope ls(c, st, PROF_BLAS, (3.0 * (j + 1) + 1) * sbytes() + 96.0 * 2 * vh);
                B_DISPATCH(p.sloppy.spinor, p.sloppy.compute, r_multi_kernel, vh, a);
            }
            mfull(p.sloppy, gv_s, R + j * fb, R + (j + 1) * fb, hb, act, PROF_STENCIL);
        }
        for (int j = 1; j <= l; j++)
            for (int i = 1; i <= j; i++) {
                BArgs a = args();
                a.j = j;
                a.i = i;
                a.op = i < j ? OP_TAU : OP_SIGMA;
                LaunchScope ls(c, st, PROF_BLAS, (i >= 2 ? 4.0 : 2.0) * sbytes());
                B_DISPATCH(p.sloppy.spinor, p.sloppy.compute, mgs_kernel, vh, a);
            }
        {
            LaunchScope ls(c, st, PROF_BLAS, 0.0);
            launch_chained(gamma_kernel, dim3(1), dim3(1), st, b, act);
        }
        BArgs a = args();
        a.op = OP_FINAL;
        LaunchScope ls(c, st, PROF_BLAS, (2.0 * l + 4.0) * sbytes() + 96.0 * 2 * vh);
        B_DISPATCH(p.sloppy.spinor, p.sloppy.compute, final_kernel, vh, a);
    }

    hisq_status pull()
    {
        cudaMemcpyAsync(bh, b, sizeof(BState), cudaMemcpyDeviceToHost, st);
        const cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? HISQ_OK : cuda_fail(c, e, "BiCGStab state");
    }

    // r_hi = b - M x (FP64), r_0 = r_hi (sloppy); |r_hi|^2 -> red.result[0]
    void true_residual(const double *b64, bool x_zero)
    {
        const size_t h64 = (size_t)48 * vh;
        if (!x_zero) {
            mfull(prec_f64(), gv_d, (const char *)x64, (char *)ax64, h64, nullptr, PROF_STENCIL_HI);
            mv_hi++;
        }
        for (int h = 0; h < 2; h++) {
            BlasArgs a{};
            a.n = vh;
            a.err = cur_err(c);
            a.red = cur_red(c);
            a.b64 = b64 + h * 6 * (size_t)vh;
            a.ax64 = x_zero ? nullptr : ax64 + h * 6 * (size_t)vh;
            a.r64 = r64 + h * 6 * (size_t)vh;
            a.v0 = R + h * hb;
            a.v1 = R + h * hb;
            a.fin = FIN_STORE;
            a.fst = nullptr;
            LaunchScope ls(c, st, PROF_BLAS, (48.0 * 3 + 2.0 * spinor_site_bytes(p.sloppy.spinor)) * vh);
            launch_true_residual(p.sloppy.spinor, p.sloppy.compute, a, st);
            if (h == 0) cudaMemcpyAsync(park, cur_red(c).result, sizeof(double), cudaMemcpyDeviceToDevice, st);
        }
    }

    hisq_status run(const double *b64, bool x_zero, hisq_solve_info *info)
    {
        hisq_status e = gauge_view_for(c, g, p.sloppy, &gv_s);
        if (!e) e = gauge_view_for(c, g, prec_f64(), &gv_d);
        if (e) return e;
        hb = spinor_field_bytes(p.sloppy.spinor, vh);
        fb = 2 * hb;
        const size_t f64b = (size_t)96 * vh;
        e = ws.alloc(fb * (l + 1), (void **)&R);
        if (!e) e = ws.alloc(fb * (l + 1), (void **)&U);
        if (!e) e = ws.alloc(fb, (void **)&rt);
        if (!e) e = ws.alloc(f64b, (void **)&ax64);
        if (!e) e = ws.alloc(64, (void **)&park);
        if (!e) e = ws.alloc(f64b, (void **)&r64);
        if (!e) e = ws.alloc(sizeof(BState), (void **)&b);
        if (e) return e;
        if (cudaMallocHost(&bh, sizeof(BState)) != cudaSuccess) return fail(c, HISQ_ENOMEM, "pinned host state");
        tune_stencil(c, g->geom, p.sloppy, gv_s, U, R, st);
        tune_stencil(c, g->geom, prec_f64(), gv_d, (char *)ax64, (char *)r64, st);
        cudaMemsetAsync(U, 0, fb * (l + 1), st);
        cudaMemsetAsync(R, 0, fb * (l + 1), st);
        // |b|^2 over both halves
        double bb = 0.0;
        for (int h = 0; h < 2; h++) {
            BlasArgs a{};
            a.n = vh;
            a.red = cur_red(c);
            a.x64 = const_cast<double *>(b64) + h * 6 * (size_t)vh;
            launch_norm2(a, st);
            double part = 0;
            cudaMemcpyAsync(&part, cur_red(c).result, sizeof part, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "norm");
            bb += part;
        }
        if (!std::isfinite(bb)) return fail(c, HISQ_EINVAL, "non-finite right-hand side");
        if (bb == 0.0) {
            cudaMemsetAsync(x64, 0, f64b, st);
            cudaStreamSynchronize(st);
            return HISQ_OK;
        }
        // r_0 = b - M x, shadow residual = r_0
        auto residual_norm = [&](bool xz, double &rr) -> hisq_status {
            true_residual(b64, xz);
            double parts[2] = {0, 0};
            cudaMemcpyAsync(&parts[0], park, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(&parts[1], cur_red(c).result, sizeof(double), cudaMemcpyDeviceToHost, st);
            const cudaError_t ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "true residual");
            rr = parts[0] + parts[1];
            return HISQ_OK;
        };
        double rr = 0;
        e = residual_norm(x_zero, rr);
        if (e) return e;
        cudaMemcpyAsync(rt, R, fb, cudaMemcpyDeviceToDevice, st);
        BState init{};
        init.rho_re = 1.0;
        init.omega_re = 1.0;
        init.rr = rr;
        init.rr_max = rr;
        init.delta2 = p.delta * p.delta;
        init.stop2 = p.tol * p.tol * bb;
        init.tiny2 = 1e-300;  // only guards the divisions
        init.rt2 = rr;        // rt = r_0
        init.brk2 = 1e-60;    // |<rt, v>| <= 1e-30 |rt| |v|
        init.active = 1;
        init.l = l;
        *bh = init;
        cudaMemcpyAsync(b, &init, sizeof init, cudaMemcpyHostToDevice, st);
        hisq_status status = HISQ_OK;
        bool done = rr <= init.stop2;
        const bool graph = p.use_graph && !c->prof.on;
        cudaGraphExec_t exec = nullptr;
        int64_t nodes = 0;
        while (!done) {
            if (mv >= p.maxiter) {
                status = HISQ_ENOTCONV;
                break;
            }
            if (graph) {
                if (!exec) {
                    cudaGraph_t gr = nullptr;
                    set_thread_capturing(true);
                    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                    if (ce == cudaSuccess) {
                        cycle();
                        ce = cudaStreamEndCapture(st, &gr);
                    }
                    set_thread_capturing(false);
                    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, gr, 0);
                    size_t nn = 0;
                    if (ce == cudaSuccess) ce = graph_kernel_nodes(gr, &nn);
                    if (gr) cudaGraphDestroy(gr);
                    if (ce != cudaSuccess) return cuda_fail(c, ce, "BiCGStab graph capture");
                    nodes = (int64_t)nn;
                }
                cudaGraphLaunch(exec, st);
                c->launches += nodes;
            } else {
                cycle();
            }
            mv += 2 * l;
            e = pull();
            if (e) break;
            if (bh->reason == REASON_BREAKDOWN) {
                status = fail(c, HISQ_EBREAKDOWN, "BiCGStab(%d) breakdown in cycle %d", l, bh->cycles);
                break;
            }
            if (bh->reason == REASON_RELIABLE || bh->reason == REASON_CONVERGED) {
                e = residual_norm(false, rr);
                if (e) break;
                ru++;
                {
                    LaunchScope ls(c, st, PROF_BLAS, 0.0);
                    // total of both halves was assembled on the host; hand it to the device
                    cudaMemcpyAsync(cur_red(c).result, &rr, sizeof rr, cudaMemcpyHostToDevice, st);
                    launch_chained(restart_kernel, dim3(1), dim3(1), st, b, (const double *)cur_red(c).result);
                }
                e = pull();
                if (e) break;
                done = rr <= init.stop2;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (e) return e;
        if (status != HISQ_OK) {
            e = residual_norm(false, rr);
            if (e) return e;
        }
        info->iters = bh->cycles;
        info->matvecs = mv;
        info->matvecs_hi = mv_hi;
        info->reliable_updates = ru;
        info->true_residual = std::sqrt(rr / bb);
        if (status == HISQ_ENOTCONV)
            fail(c, HISQ_ENOTCONV, "BiCGStab(%d) reached %d matvecs with true residual %.3e", l, mv,
                 info->true_residual);
        return status;
    }
};

}  // namespace

}  // namespace hisq

using namespace hisq;

extern "C" hisq_status hisq_bicgstabl(hisq_ctx *c, const hisq_gauge *gc, const hisq_solver_params *p,
                                      const double *b, double *x, hisq_solve_info *info)
{
    if (!c || !gc || !b || !x || !info) return fail(c, HISQ_EINVAL, "hisq_bicgstabl: null argument");
    *info = hisq_solve_info{};
    hisq_status e = validate_params(c, p);
    if (e) return e;
    if (p->l < 1 || p->l > 8) return fail(c, HISQ_EINVAL, "l must be in 1..8");
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    hisq_gauge *g = const_cast<hisq_gauge *>(gc);
    cudaStream_t s = pick_stream(c, p->stream);
    const int64_t vh = g->geom.vh;
    if (!solver_red_fits(vh)) return fail(c, HISQ_EINVAL, "lattice too large for the solvers' reductions");
    Workspace ws(c, s);
    double *b64 = nullptr, *x64 = nullptr;
    e = ws.alloc((size_t)96 * vh, (void **)&b64);
    if (!e) e = ws.alloc((size_t)96 * vh, (void **)&x64);
    if (e) return e;
    // the caller's full-lattice array is [even][odd]: convert per half
    for (int h = 0; h < 2 && !e; h++) e = to_planar(c, ws, b + h * 6 * vh, p->on_device, vh, b64 + h * 6 * vh, s);
    if (!e && p->use_init_guess)
        for (int h = 0; h < 2 && !e; h++) e = to_planar(c, ws, x + h * 6 * vh, p->on_device, vh, x64 + h * 6 * vh, s);
    if (!e && !p->use_init_guess) cudaMemsetAsync(x64, 0, (size_t)96 * vh, s);
    if (e) return e;
    hisq_status st;
    {
        BRun run(c, g, *p, s);
        run.x64 = x64;
        st = run.run(b64, !p->use_init_guess, info);
    }
    if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) return st;
    for (int h = 0; h < 2 && !e; h++) e = from_planar(c, ws, x64 + h * 6 * vh, vh, x + h * 6 * vh, p->on_device, s);
    if (e) return e;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}
