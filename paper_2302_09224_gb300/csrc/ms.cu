// ms.cu -- mixed-precision multi-shift CG with refinement (Sec. 3.2) and its
// C-ABI entry point.
//
// Stage 1 (sloppy triplet): one base recurrence on A = M_ee + sigma_0 (the
// smallest shift) with reliable updates on the base system; every shift's
// solution and gradient vector are updated in one fused kernel per iteration
// that reads r once (x_i accumulators in the compute precision, flushed into
// FP64 at each reliable update).  Shift i stops updating once its iterated
// residual zeta_i |r| reaches max(tol_i, 10 eps of the sloppy format); the
// stage ends when every shift other than the base has stopped.
// Stage 2 (refinement triplet): CG on the base system continuing from its
// gradient vector (re-projected against the new residual), then CG on each
// other shift from its x_i with a clean restart, skipping shifts whose FP64
// true residual already meets their target.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "blas.h"
#include "cg.h"
#include "codecs.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "finish.cuh"

namespace hisq {

struct MSArgs {
    int n;
    int nshift;
    const char *r;        // sloppy residual
    char *p;              // nshift sloppy fields, p_bytes apart
    size_t p_bytes;
    char *acc;            // nshift accumulator fields (F32 or F64 planar), acc_bytes apart
    size_t acc_bytes;
    double *x64;          // nshift FP64 planar fields, 48*n apart
    MSState *m;
    const int *active;
    int *err;
    RedBuf red;
};

namespace {

constexpr int kBlock = 256;

// For every live shift: acc_i += alpha_i p_i, p_i = zeta_i r + beta_i p_i.
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) shift_update_kernel(MSArgs a)
{
    if (a.active && *(volatile const int *)a.active == 0) return;
    constexpr int AF = is_ff<real>::value ? S_FF : sizeof(real) == 8 ? S_F64 : S_F32;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const MSState *m = a.m;
    // the shifts' step sizes in the compute precision, converted once per block (for FP32 pairs
    // the conversion runs on the narrow FP64 pipe)
    __shared__ real cs[3][kMaxShift];
    if (threadIdx.x < a.nshift) {
        cs[0][threadIdx.x] = (real)m->alpha_i[threadIdx.x];
        cs[1][threadIdx.x] = (real)m->zeta[threadIdx.x];
        cs[2][threadIdx.x] = (real)m->beta_i[threadIdx.x];
    }
    __syncthreads();
    if (i < a.n) {
        real r[6];
        Spinor<SF>::load(a.r, a.n, i, r);
        for (int s = 0; s < a.nshift; s++) {
            if (!m->live[s]) continue;
            real p[6], x[6];
            char *ps = a.p + (size_t)s * a.p_bytes;
            char *xs = a.acc + (size_t)s * a.acc_bytes;
            Spinor<SF>::load(ps, a.n, i, p);
            Spinor<AF>::load(xs, a.n, i, x);
            const real al = cs[0][s], z = cs[1][s], be = cs[2][s];
#pragma unroll
            for (int k = 0; k < 6; k++) {
                x[k] += al * p[k];
                p[k] = z * r[k] + be * p[k];
            }
            if (!Spinor<SF>::store(ps, a.n, i, p)) atomicExch(a.err, 1);
            Spinor<AF>::store(xs, a.n, i, x);
        }
    }
    double v[1] = {0.0};
    __shared__ double tot[1];
    if (reduce_grid<1>(v, a.red, tot) && threadIdx.x == 0) run_finisher(FIN_MS_APPLY, tot, a.m, 0);
}

// x64_i += acc_i and acc_i = 0 for every shift.
template <int AF>
__global__ void __launch_bounds__(kBlock) acc_flush_kernel(MSArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    for (int s = 0; s < a.nshift; s++) {
        char *xs = a.acc + (size_t)s * a.acc_bytes;
        char *x64 = reinterpret_cast<char *>(a.x64) + (size_t)s * 48 * a.n;
        double acc[6], x[6];
        Spinor<AF>::load(xs, a.n, i, acc);
        Spinor<S_F64>::load(x64, a.n, i, x);
#pragma unroll
        for (int k = 0; k < 6; k++) {
            x[k] += acc[k];
            acc[k] = 0.0;
        }
        Spinor<S_F64>::store(x64, a.n, i, x);
        Spinor<AF>::store(xs, a.n, i, acc);
    }
}

template <int SI, int SO>
__global__ void __launch_bounds__(kBlock) convert_kernel(int n, const char *in, char *out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[6];
    Spinor<SI>::load(in, n, i, v);
    if (!Spinor<SO>::store(out, n, i, v)) atomicExch(err, 1);
}

template <int SI>
void convert_to(int so, int n, const char *in, char *out, int *err, cudaStream_t s)
{
    const int nb = (n + kBlock - 1) / kBlock;
    switch (so) {
    case S_F64: convert_kernel<SI, S_F64><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    case S_F32: convert_kernel<SI, S_F32><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    case S_HALF: convert_kernel<SI, S_HALF><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    case S_INT20: convert_kernel<SI, S_INT20><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    case S_INT14: convert_kernel<SI, S_INT14><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    case S_INT30: convert_kernel<SI, S_INT30><<<nb, kBlock, 0, s>>>(n, in, out, err); break;
    }
}

int nblk(int n) { return (n + kBlock - 1) / kBlock; }

double format_eps(int sf)
{
    switch (sf) {
    case S_F32: return std::ldexp(1.0, -24);
    case S_HALF: return std::ldexp(1.0, -15);  // Sec. 2
    case S_INT20: return std::ldexp(1.0, -19); // Sec. 4
    case S_INT30: return std::ldexp(1.0, -29); // Sec. 4
    case S_INT14: return std::ldexp(1.0, -13);
    default: return std::ldexp(1.0, -52);
    }
}

}  // namespace

// field conversion between storage formats (any pair), exposed to the drivers
void launch_convert(int si, int so, int n, const char *in, char *out, int *err, cudaStream_t s)
{
    switch (si) {
    case S_F64: convert_to<S_F64>(so, n, in, out, err, s); break;
    case S_F32: convert_to<S_F32>(so, n, in, out, err, s); break;
    case S_HALF: convert_to<S_HALF>(so, n, in, out, err, s); break;
    case S_INT20: convert_to<S_INT20>(so, n, in, out, err, s); break;
    case S_INT14: convert_to<S_INT14>(so, n, in, out, err, s); break;
    case S_INT30: convert_to<S_INT30>(so, n, in, out, err, s); break;
    }
}

namespace {

struct MSRun {
    hisq_ctx *c;
    hisq_gauge *g;
    const hisq_solver_params &p;
    cudaStream_t s;
    Workspace ws;
    int vh, ns;
    size_t sb, accb;
    int acc_fmt;
    std::vector<double> sig, tol;
    char *r_s = nullptr, *w_s = nullptr, *tmp_s = nullptr, *P = nullptr, *ACC = nullptr;
    double *X = nullptr, *r64 = nullptr, *ax64 = nullptr, *tmp64 = nullptr;
    MSState *m = nullptr, *mh = nullptr;
    GaugeView gv_s{}, gv_d{};
    int ru = 0, mv_hi = 0;

    MSRun(hisq_ctx *c_, hisq_gauge *g_, const hisq_solver_params &p_, cudaStream_t s_)
        : c(c_), g(g_), p(p_), s(s_), ws(c_, s_), vh(g_->geom.vh), ns(0)
    {
    }
    ~MSRun()
    {
        if (mh) cudaFreeHost(mh);
    }

    double *x64(int i) { return X + (size_t)i * 6 * vh; }
    char *pf(int i) { return P + (size_t)i * sb; }

    MSArgs args() const
    {
        MSArgs a{};
        a.n = vh;
        a.nshift = ns;
        a.r = r_s;
        a.p = P;
        a.p_bytes = sb;
        a.acc = ACC;
        a.acc_bytes = accb;
        a.x64 = X;
        a.m = m;
        a.err = cur_err(c);
        a.red = cur_red(c);
        return a;
    }

    hisq_status pull()
    {
        cudaMemcpyAsync(mh, m, sizeof(MSState), cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? HISQ_OK : cuda_fail(c, e, "multi-shift state");
    }

    void flush_acc()
    {
        MSArgs a = args();
        LaunchScope ls(c, s, PROF_BLAS, (double)ns * (96.0 + 2.0 * spinor_site_bytes(acc_fmt)) * vh);
        if (acc_fmt == S_F64)
            acc_flush_kernel<S_F64><<<nblk(vh), kBlock, 0, s>>>(a);
        else if (acc_fmt == S_FF)
            acc_flush_kernel<S_FF><<<nblk(vh), kBlock, 0, s>>>(a);
        else
            acc_flush_kernel<S_F32><<<nblk(vh), kBlock, 0, s>>>(a);
    }

    // FP64 |b - (M_ee + sigma) x|^2 into red.result[0]; also leaves r64/r_s.
    void residual(int shift, int fin, void *fst)
    {
        const double diag = 4.0 * p.mass * p.mass + sig[shift];
        apply_mee(c, g->geom, prec_f64(), gv_d, diag, (const char *)x64(shift), (char *)tmp64, (char *)ax64, FIN_NONE,
                  nullptr, 0, nullptr, PROF_STENCIL_HI, s);
        mv_hi++;
        BlasArgs b{};
        b.n = vh;
        b.err = cur_err(c);
        b.red = cur_red(c);
        b.b64 = b64;
        b.ax64 = ax64;
        b.r64 = r64;
        b.v0 = r_s;
        b.v1 = pf(0);
        b.fin = fin;
        b.fst = fst;
        LaunchScope ls(c, s, PROF_BLAS, (48.0 * 3 + 2.0 * spinor_site_bytes(p.sloppy.spinor)) * vh);
        launch_true_residual(p.sloppy.spinor, p.sloppy.compute, b, s);
    }

    const double *b64 = nullptr;

    void iterate_block(int nit)
    {
        const double diag0 = 4.0 * p.mass * p.mass + sig[0];
        const int *act = &m->active;
        for (int it = 0; it < nit; it++) {
            apply_mee(c, g->geom, p.sloppy, gv_s, diag0, pf(0), tmp_s, w_s, FIN_MS_ALPHA, m, 0, act, PROF_STENCIL, s);
            BlasArgs b{};
            b.n = vh;
            b.err = cur_err(c);
            b.red = cur_red(c);
            b.v0 = r_s;
            b.v1 = w_s;
            b.active = act;
            b.alpha_src = &m->alpha;
            b.fin = FIN_MS_BETA;
            b.fst = m;
            {
                LaunchScope ls(c, s, PROF_BLAS, 3.0 * spinor_site_bytes(p.sloppy.spinor) * vh);
                launch_r_update(p.sloppy.spinor, p.sloppy.compute, b, s);
            }
            MSArgs a = args();
            a.active = act;
            int live = 0;
            for (int i = 0; i < ns; i++) live += mh->live[i];
            LaunchScope ls(c, s, PROF_BLAS,
                           (spinor_site_bytes(p.sloppy.spinor) +
                            live * (2.0 * spinor_site_bytes(p.sloppy.spinor) + 2.0 * spinor_site_bytes(acc_fmt))) * vh);
            const bool f64 = p.sloppy.compute == HISQ_COMPUTE_F64;
            switch (p.sloppy.spinor) {
            case S_F64: shift_update_kernel<S_F64, double><<<nblk(vh), kBlock, 0, s>>>(a); break;
            case S_F32: shift_update_kernel<S_F32, float><<<nblk(vh), kBlock, 0, s>>>(a); break;
            case S_HALF: shift_update_kernel<S_HALF, float><<<nblk(vh), kBlock, 0, s>>>(a); break;
            case S_INT20: shift_update_kernel<S_INT20, float><<<nblk(vh), kBlock, 0, s>>>(a); break;
            case S_INT14: shift_update_kernel<S_INT14, float><<<nblk(vh), kBlock, 0, s>>>(a); break;
            case S_INT30:
                if (f64)  // FP64-class compute in FP32 pairs, pair accumulators
                    shift_update_kernel<S_INT30, ff><<<nblk(vh), kBlock, 0, s>>>(a);
                else shift_update_kernel<S_INT30, float><<<nblk(vh), kBlock, 0, s>>>(a);
                break;
            }
        }
    }

    hisq_status run(const double *b64_, int nshift, const double *sigma, const double *tolv, hisq_solve_info *info,
                    bool refine = true)
    {
        b64 = b64_;
        ns = nshift;
        sig.assign(sigma, sigma + ns);
        tol.assign(tolv, tolv + ns);
        hisq_status e = gauge_view_for(c, g, p.sloppy, &gv_s);
        if (!e) e = gauge_view_for(c, g, prec_f64(), &gv_d);
        if (e) return e;
        sb = spinor_field_bytes(p.sloppy.spinor, vh);
        acc_fmt = p.sloppy.compute != HISQ_COMPUTE_F64 ? S_F32 : p.sloppy.spinor == S_INT30 ? S_FF : S_F64;
        accb = spinor_field_bytes(acc_fmt, vh);
        const size_t b48 = (size_t)48 * vh;
        e = ws.alloc(sb, (void **)&r_s);
        if (!e) e = ws.alloc(sb, (void **)&w_s);
        if (!e) e = ws.alloc(sb, (void **)&tmp_s);
        if (!e) e = ws.alloc(sb * ns, (void **)&P);
        if (!e) e = ws.alloc(accb * ns, (void **)&ACC);
        if (!e) e = ws.alloc(b48 * ns, (void **)&X);
        if (!e) e = ws.alloc(b48, (void **)&r64);
        if (!e) e = ws.alloc(b48, (void **)&ax64);
        if (!e) e = ws.alloc(b48, (void **)&tmp64);
        if (!e) e = ws.alloc(sizeof(MSState), (void **)&m);
        if (e) return e;
        if (cudaMallocHost(&mh, sizeof(MSState)) != cudaSuccess) return fail(c, HISQ_ENOMEM, "pinned host state");
        cudaMemsetAsync(ACC, 0, accb * ns, s);
        cudaMemsetAsync(X, 0, b48 * ns, s);
        tune_stencil(c, g->geom, p.sloppy, gv_s, w_s, tmp_s, s);
        tune_stencil(c, g->geom, prec_f64(), gv_d, (char *)ax64, (char *)tmp64, s);
        // r = p_i = b
        {
            LaunchScope ls(c, s, PROF_CONVERT, (48.0 + spinor_site_bytes(p.sloppy.spinor)) * vh);
            launch_convert(S_F64, p.sloppy.spinor, vh, (const char *)b64, r_s, cur_err(c), s);
        }
        for (int i = 0; i < ns; i++) cudaMemcpyAsync(pf(i), r_s, sb, cudaMemcpyDeviceToDevice, s);
        {
            BlasArgs a{};
            a.n = vh;
            a.red = cur_red(c);
            a.x64 = const_cast<double *>(b64);
            LaunchScope ls(c, s, PROF_BLAS, 48.0 * vh);
            launch_norm2(a, s);
        }
        double bb = 0;
        cudaMemcpyAsync(&bb, cur_red(c).result, sizeof bb, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "norm");
        if (!std::isfinite(bb)) return fail(c, HISQ_EINVAL, "non-finite right-hand side");
        info->nshift = ns;
        if (bb == 0.0) return HISQ_OK;  // all x_i = 0
        MSState init{};
        init.rr = bb;
        init.rr_max = bb;
        init.bb = bb;
        init.delta2 = p.delta * p.delta;
        init.alpha_prev = 1.0;
        init.beta_prev = 0.0;
        init.nshift = ns;
        init.active = 1;
        const double floor = 10.0 * format_eps(p.sloppy.spinor);
        for (int i = 0; i < ns; i++) {
            init.shift[i] = sig[i] - sig[0];
            const double t = std::max(tol[i], floor);
            init.stop2[i] = t * t * bb;
            init.zeta[i] = init.zeta_prev[i] = 1.0;
            init.live[i] = 1;
        }
        *mh = init;
        cudaMemcpyAsync(m, &init, sizeof init, cudaMemcpyHostToDevice, s);
        const bool graph = p.use_graph && !c->prof.on;
        const int N = std::max(1, p.nbuf);
        cudaGraphExec_t exec = nullptr;
        int64_t nodes = 0;
        hisq_status status = HISQ_OK;
        while (true) {
            if (mh->k >= p.maxiter) {
                status = HISQ_ENOTCONV;
                break;
            }
            if (graph) {
                if (!exec) {
                    cudaGraph_t gr = nullptr;
                    set_thread_capturing(true);
                    cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
                    if (ce == cudaSuccess) {
                        iterate_block(N);
                        ce = cudaStreamEndCapture(s, &gr);
                    }
                    set_thread_capturing(false);
                    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, gr, 0);
                    size_t nn = 0;
                    if (ce == cudaSuccess) ce = graph_kernel_nodes(gr, &nn);
                    if (gr) cudaGraphDestroy(gr);
                    if (ce != cudaSuccess) return cuda_fail(c, ce, "multi-shift graph capture");
                    nodes = (int64_t)nn;
                }
                cudaGraphLaunch(exec, s);
                c->launches += nodes;
            } else {
                iterate_block(N);
            }
            e = pull();
            if (e) break;
            if (mh->reason == REASON_BREAKDOWN) {
                status = fail(c, HISQ_EBREAKDOWN, "multi-shift CG breakdown at iteration %d", mh->k);
                break;
            }
            if (mh->reason == REASON_CONVERGED) break;
            if (mh->reason == REASON_RELIABLE) {
                flush_acc();
                residual(0, FIN_MS_TRUE, m);
                ru++;
                e = pull();
                if (e) break;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (e) return e;
        flush_acc();
        info->iters = mh->k;
        info->matvecs += mh->k;
        info->reliable_updates += ru;
        for (int i = 0; i < ns; i++) info->shift_iters[i] = mh->live[i] ? mh->k : mh->frozen_at[i];
        // FP64 true residual of every shift after the multi-shift stage (Table 3's r_sigma)
        std::vector<double> rs(ns);
        for (int i = 0; i < ns; i++) {
            residual(i, FIN_STORE, nullptr);
            double rr = 0;
            cudaMemcpyAsync(&rr, cur_red(c).result, sizeof rr, cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "residual");
            rs[i] = std::sqrt(rr / bb);
            info->shift_resid_ms[i] = rs[i];
            info->shift_resid[i] = rs[i];
        }
        if (status == HISQ_EBREAKDOWN || !refine) {
            info->matvecs_hi += mv_hi;
            info->true_residual = info->shift_resid[0];
            return status;
        }
        const double rr_base = mh->rr;
        // refinement: the base system keeps its gradient vector, the others restart
        hisq_status worst = status;
        for (int i = 0; i < ns; i++) {
            if (rs[i] <= tol[i]) continue;
            CGConfig cfg = config_from(&p, sig[i]);
            cfg.sloppy = p.refine;
            cfg.tol = tol[i];
            if (i == 0) {
                cfg.p_init = pf(0);
                cfg.p_init_fmt = p.sloppy.spinor;
                cfg.rr_prev_init = rr_base;
            }
            hisq_solve_info ri{};
            const hisq_status st = run_cg(c, g, cfg, b64, x64(i), false, &ri, s);
            info->refine_iters[i] = ri.iters;
            info->matvecs += ri.matvecs;
            info->matvecs_hi += ri.matvecs_hi;
            info->reliable_updates += ri.reliable_updates;
            info->shift_resid[i] = ri.true_residual;
            if (st == HISQ_ENOTCONV || st == HISQ_EBREAKDOWN) {
                worst = st;
            } else if (st != HISQ_OK) {
                return st;
            }
        }
        info->matvecs_hi += mv_hi;
        info->true_residual = info->shift_resid[0];
        return worst;
    }
};

}  // namespace

hisq_status run_multishift_stage(hisq_ctx *c, hisq_gauge *g, const hisq_solver_params &p, int ns, const double *sigma,
                                 const double *tol, const double *b64, double *const *x64_out, hisq_solve_info *info,
                                 cudaStream_t s)
{
    MSRun run(c, g, p, s);
    const hisq_status st = run.run(b64, ns, sigma, tol, info, false);
    if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) return st;
    for (int i = 0; i < ns; i++)
        cudaMemcpyAsync(x64_out[i], run.x64(i), (size_t)48 * g->geom.vh, cudaMemcpyDeviceToDevice, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "multi-shift stage results");
    return st;
}

}  // namespace hisq

using namespace hisq;

extern "C" hisq_status hisq_multishift_cg(hisq_ctx *c, const hisq_gauge *gc, const hisq_solver_params *p, int nshift,
                                          const double *sigma, const double *tol, const double *b, double *const *x,
                                          hisq_solve_info *info)
{
    if (!c || !gc || !sigma || !tol || !b || !x || !info) return fail(c, HISQ_EINVAL, "hisq_multishift_cg: null argument");
    *info = hisq_solve_info{};
    hisq_status e = validate_params(c, p);
    if (e) return e;
    e = check_prec(c, p->refine);
    if (e) return e;
    if (nshift < 1 || nshift > HISQ_MAX_SHIFTS || nshift > kMaxShift)
        return fail(c, HISQ_EINVAL, "nshift must be in 1..%d", HISQ_MAX_SHIFTS);
    for (int i = 0; i < nshift; i++) {
        if (!std::isfinite(sigma[i]) || !(tol[i] > 0.0) || !x[i])
            return fail(c, HISQ_EINVAL, "shift %d: sigma must be finite, tol > 0, x non-null", i);
        if (4.0 * p->mass * p->mass + sigma[i] <= 0.0)
            return fail(c, HISQ_EINVAL, "shift %d: 4m^2 + sigma must be positive", i);
    }
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    hisq_gauge *g = const_cast<hisq_gauge *>(gc);
    cudaStream_t s = pick_stream(c, p->stream);
    const int64_t vh = g->geom.vh;
    if (!solver_red_fits(vh)) return fail(c, HISQ_EINVAL, "lattice too large for the solvers' reductions");
    // ascending shifts: the smallest is the base system
    std::vector<int> ord(nshift);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int bb) { return sigma[a] < sigma[bb]; });
    std::vector<double> ss(nshift), tt(nshift);
    for (int i = 0; i < nshift; i++) {
        ss[i] = sigma[ord[i]];
        tt[i] = tol[ord[i]];
    }
    Workspace ws(c, s);
    double *b64 = nullptr;
    e = ws.alloc((size_t)48 * vh, (void **)&b64);
    if (!e) e = to_planar(c, ws, b, p->on_device, vh, b64, s);
    if (e) return e;
    hisq_solve_info si{};
    hisq_status st;
    {
        MSRun run(c, g, *p, s);
        st = run.run(b64, nshift, ss.data(), tt.data(), &si);
        if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) return st;
        for (int i = 0; i < nshift; i++) {
            e = from_planar(c, ws, run.x64(i), vh, x[ord[i]], p->on_device, s);
            if (e) return e;
        }
    }
    // report per shift in the caller's order
    *info = si;
    for (int i = 0; i < nshift; i++) {
        info->shift_iters[ord[i]] = si.shift_iters[i];
        info->shift_resid_ms[ord[i]] = si.shift_resid_ms[i];
        info->shift_resid[ord[i]] = si.shift_resid[i];
        info->refine_iters[ord[i]] = si.refine_iters[i];
    }
    info->true_residual = si.shift_resid[0];
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}
