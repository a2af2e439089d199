// full.cu -- hisq_solve_full: the full-lattice system (2m + D) x = b solved by
// even/odd reduction around the mixed-precision CG of Sec. 3.1.
//
// With M = [[2m, D_eo], [D_oe, 2m]] in parity blocks the odd unknowns are
// eliminated: the even ones solve (4m^2 - D_eo D_oe) x_e = 2m b_e - D_eo b_o
// (the system every CG of this library works on) and the odd ones follow as
// x_o = (b_o - D_oe x_e) / (2m).  For x_o built this way the full residual is
// zero on the odd sites and (bt_e - M_ee x_e) / (2m) on the even ones, so the
// even solve is run to the tolerance tol * 2|m| |b| / |bt_e|.  The source and
// the reconstruction use the FP64 stencil, as the true residuals do.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "bcg.h"
#include "blas.h"
#include "cg.h"
#include "internal.h"

namespace hisq {

namespace {

constexpr int kBlock = 256;

// out[i] = in[i] / d over n doubles (planar FP64 fields share one layout)
__global__ void __launch_bounds__(kBlock) div_kernel(int64_t n, const double *in, double d, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] / d;
}

// out[i] = a[i] - b[i]
__global__ void __launch_bounds__(kBlock) sub_kernel(int64_t n, const double *a, const double *b, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

int grid_of(int64_t n)
{
    static const int cap = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return 8 * std::max(sms, 1);
    }();
    return (int)std::min<int64_t>((n + kBlock - 1) / kBlock, cap);
}

struct FullRun {
    hisq_ctx *c;
    hisq_gauge *g;
    cudaStream_t s;
    GaugeView gv{};
    int64_t vh;

    // out = a * y + sign * D in (FP64 stencil, output parity po)
    void stencil(int po, const double *in, const double *y, double a, int sign, double *out)
    {
        DslashArgs d{};
        d.g = g->geom;
        d.gv = gv;
        d.err = cur_err(c);
        d.red = cur_red(c);
        d.out_parity = po;
        d.in = (const char *)in;
        d.out = (char *)out;
        d.y = (const char *)y;
        d.a = a;
        d.sign = sign;
        d.xpay = 1;
        d.fin = FIN_NONE;
        LaunchScope ls(c, s, PROF_STENCIL_HI, stencil_bytes(prec_f64(), (int)vh, true));
        launch_dslash(G_F64, S_F64, HISQ_COMPUTE_F64, 18, false, d, s);
    }

    void div(const double *in, double d, double *out)
    {
        const int64_t n = 6 * vh;
        LaunchScope ls(c, s, PROF_BLAS, 16.0 * n);
        div_kernel<<<grid_of(n), kBlock, 0, s>>>(n, in, d, out);
    }

    void sub(const double *a, const double *b, double *out)
    {
        const int64_t n = 6 * vh;
        LaunchScope ls(c, s, PROF_BLAS, 24.0 * n);
        sub_kernel<<<grid_of(n), kBlock, 0, s>>>(n, a, b, out);
    }

    // |v|^2 of a planar FP64 half-lattice field (synchronises)
    hisq_status norm2(const double *v, double *out)
    {
        BlasArgs a{};
        a.n = (int)vh;
        a.err = cur_err(c);
        a.red = cur_red(c);
        a.x64 = const_cast<double *>(v);
        {
            LaunchScope ls(c, s, PROF_BLAS, 48.0 * vh);
            launch_norm2(a, s);
        }
        cudaMemcpyAsync(out, cur_red(c).result, sizeof(double), cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? HISQ_OK : cuda_fail(c, e, "norm");
    }
};

}  // namespace

}  // namespace hisq

using namespace hisq;

extern "C" hisq_status hisq_solve_full(hisq_ctx *c, const hisq_gauge *gc, const hisq_solver_params *p,
                                       const double *b, double *x, hisq_solve_info *info)
{
    if (!c || !gc || !b || !x || !info) return fail(c, HISQ_EINVAL, "hisq_solve_full: null argument");
    *info = hisq_solve_info{};
    hisq_status e = validate_params(c, p);
    if (e) return e;
    if (p->mass == 0.0) return fail(c, HISQ_EINVAL, "the full-lattice solve divides by 2m: m must be nonzero");
    const int nr = p->nrhs;
    if (nr < 1 || nr > kMaxRHS) return fail(c, HISQ_EINVAL, "nrhs must be in 1..%d", kMaxRHS);
    if (p->rhs_tile < 0 || p->rhs_tile > kMaxRHS || (p->rhs_tile > 0 && nr % p->rhs_tile))
        return fail(c, HISQ_EINVAL, "rhs_tile must divide nrhs");
    if (nr > 1 && p->history_len > 0) return fail(c, HISQ_EINVAL, "a residual history is kept for nrhs = 1 only");
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    hisq_gauge *g = const_cast<hisq_gauge *>(gc);
    cudaStream_t s = pick_stream(c, p->stream);
    const int64_t vh = g->geom.vh;
    if (!solver_red_fits(vh)) return fail(c, HISQ_EINVAL, "lattice too large for the solvers' reductions");
    FullRun fr{c, g, s, {}, vh};
    e = gauge_view_for(c, g, prec_f64(), &fr.gv);
    if (e) return e;
    const size_t h64 = (size_t)48 * vh;  // one planar FP64 half-lattice field
    const size_t hd = (size_t)6 * vh;    // its doubles
    Workspace ws(c, s);
    double *bf = nullptr, *bt = nullptr, *xe = nullptr, *xo = nullptr, *t1 = nullptr, *t2 = nullptr;
    e = ws.alloc(2 * h64 * nr, (void **)&bf);           // [rhs][parity] b
    if (!e) e = ws.alloc(h64 * nr, (void **)&bt);      // [rhs] Schur sources
    if (!e) e = ws.alloc(h64 * nr, (void **)&xe);      // [rhs] even solutions
    if (!e) e = ws.alloc(h64, (void **)&xo);
    if (!e) e = ws.alloc(h64, (void **)&t1);
    if (!e) e = ws.alloc(h64, (void **)&t2);
    if (e) return e;
    const double two_m = 2.0 * p->mass;
    std::vector<double> bb(nr), tol_s(nr);
    for (int t = 0; t < nr && !e; t++) {
        double *be = bf + 2 * hd * t, *bo = be + hd;
        e = to_planar(c, ws, b + 2 * hd * t, p->on_device, vh, be, s);
        if (!e) e = to_planar(c, ws, b + 2 * hd * t + hd, p->on_device, vh, bo, s);
        if (e) break;
        // bt_e = 2m b_e - D_eo b_o
        fr.stencil(0, bo, be, two_m, -1, bt + hd * t);
        double ne = 0, no = 0, nt = 0;
        e = fr.norm2(be, &ne);
        if (!e) e = fr.norm2(bo, &no);
        if (!e) e = fr.norm2(bt + hd * t, &nt);
        bb[t] = ne + no;
        tol_s[t] = nt > 0.0 ? p->tol * std::fabs(two_m) * std::sqrt(bb[t] / nt) : p->tol;
    }
    if (e) return e;
    // the even system, from x_e = 0
    cudaMemsetAsync(xe, 0, h64 * nr, s);
    hisq_status st;
    if (nr == 1) {
        CGConfig cfg = config_from(p, 0.0);
        cfg.tol = tol_s[0];
        cfg.hist_host = p->history;
        cfg.hist_len = p->history_len;
        st = run_cg(c, g, cfg, bt, xe, true, info, s);
    } else {
        BCGConfig bc;
        bc.nrhs = nr;
        for (int t = 0; t < nr; t++) {
            bc.diag[t] = 4.0 * p->mass * p->mass;
            bc.tol[t] = tol_s[t];
        }
        bc.sloppy = p->sloppy;
        bc.nbuf = p->nbuf;
        bc.maxiter = p->maxiter;
        bc.pr = p->pr_beta;
        bc.reproject = p->reproject;
        bc.use_graph = p->use_graph;
        bc.tile = p->rhs_tile;
        bc.kernel = p->rhs_kernel;
        bc.delta = p->delta;
        bc.dyn = p->ru_trigger;
        bc.dyn_eps = p->ru_trigger ? sloppy_eps(p->sloppy) : 0.0;
        std::vector<hisq_solve_info> infos(nr);
        st = run_bcg(c, g, bc, bt, xe, true, infos.data(), s);
        for (int t = 0; t < nr; t++) {
            info->iters = std::max(info->iters, infos[t].iters);
            info->matvecs += infos[t].matvecs;
            info->matvecs_hi += infos[t].matvecs_hi;
            info->reliable_updates += infos[t].reliable_updates;
        }
    }
    if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) return st;
    double worst = 0.0;
    for (int t = 0; t < nr && !e; t++) {
        const double *be = bf + 2 * hd * t, *bo = be + hd;
        const double *xt = xe + hd * t;
        // x_o = (b_o - D_oe x_e) / (2m)
        fr.stencil(1, xt, bo, 1.0, -1, t1);
        fr.div(t1, two_m, xo);
        // FP64 true residual of the full system: r = b - (2m x + D x), per parity
        double re = 0, ro = 0;
        fr.stencil(0, xo, xt, two_m, 1, t1);
        fr.sub(be, t1, t2);
        e = fr.norm2(t2, &re);
        if (e) break;
        fr.stencil(1, xt, xo, two_m, 1, t1);
        fr.sub(bo, t1, t2);
        e = fr.norm2(t2, &ro);
        if (e) break;
        info->matvecs_hi += 1;
        worst = std::max(worst, bb[t] > 0.0 ? std::sqrt((re + ro) / bb[t]) : 0.0);
        e = from_planar(c, ws, xt, vh, x + 2 * hd * t, p->on_device, s);
        if (!e) e = from_planar(c, ws, xo, vh, x + 2 * hd * t + hd, p->on_device, s);
    }
    if (e) return e;
    info->true_residual = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}
