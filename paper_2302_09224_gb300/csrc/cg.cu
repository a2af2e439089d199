// cg.cu -- the stabilised mixed-precision even/odd CG of Sec. 3.1 and its C-ABI
// entry point.
//
// Sloppy precision (the triplet's formats): iterated residual r, gradient
// vectors p (a ring of nbuf slots) and the operator applications.  FP64: the
// solution x_hi, the right-hand side, every true residual and all reductions.
//   * reliable updates (Sec. 3, footnote): when |r| drops below delta times
//     its maximum since the last update, x_hi is brought up to date, the true
//     residual b - A x_hi is computed in FP64 and replaces r;
//   * item 1: x_hi += sum_j alpha_j p_j once per nbuf iterations (and at each
//     reliable update) from the buffered gradient vectors;
//   * item 2: at a reliable update p is re-projected against the new residual
//     and the recurrence restarts with Fletcher-Reeves beta;
//   * item 3: beta = r_new^+(r_new - r_old)/|r_old|^2 (Polak-Ribiere).
// One block of nbuf iterations is a fixed kernel sequence whose scalars live
// on the device, so it is captured once as a CUDA graph and replayed; the host
// reads the scalar state once per block.
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

Workspace::~Workspace()
{
    if (!allocs.empty()) cudaStreamSynchronize(s);
    for (auto &a : allocs) ctx_free(c, a.first, a.second);
}

hisq_status Workspace::alloc(size_t bytes, void **p)
{
    hisq_status st = ctx_alloc(c, bytes, p);
    if (!st) allocs.emplace_back(*p, bytes);
    return st;
}

double stencil_bytes(const hisq_prec &p, int vh, bool xpay)
{
    const double links = 8.0 * link_bytes(p.gauge, p.fat_recon) + 8.0 * link_bytes(p.gauge, p.long_recon);
    return (links + (xpay ? 3.0 : 2.0) * spinor_site_bytes(p.spinor)) * vh;
}

hisq_prec prec_f64()
{
    hisq_prec p;
    p.gauge = G_F64;
    p.spinor = S_F64;
    p.compute = HISQ_COMPUTE_F64;
    p.fat_recon = 18;
    p.long_recon = 18;
    return p;
}

// out_even = diag * in_even - D_eo D_oe in_even, with tmp an odd-parity field.
unsigned apply_mee(hisq_ctx *c, const Geom &geom, const hisq_prec &p, const GaugeView &gv, double diag,
                   const char *in, char *tmp, char *out, int fin, void *st, int slot, const int *active, int kind,
                   cudaStream_t s, bool leave_partials)
{
    DslashArgs d{};
    d.g = geom;
    d.gv = gv;
    d.err = cur_err(c);
    d.red = cur_red(c);
    d.active = active;
    d.st = st;
    d.slot = slot;
    d.out_parity = 1;
    d.in = in;
    d.out = tmp;
    d.sign = 1;
    DslashArgs d2 = d;
    d2.out_parity = 0;
    d2.in = tmp;
    d2.out = out;
    d2.y = in;
    d2.a = diag;
    d2.sign = -1;
    d2.xpay = 1;
    d2.fin = fin;
    if (mee_fused_available(p.gauge, p.spinor, p.compute, geom) && d2.red.sync != nullptr) {
        // one pass: links once, plus the input, tmp and output spinors
        const double links = 8.0 * link_bytes(p.gauge, 18) + 8.0 * link_bytes(p.gauge, p.long_recon);
        LaunchScope ls(c, s, kind, (links + 3.0 * spinor_site_bytes(p.spinor)) * geom.vh);
        MeeArgs m{d, d2};
        if (launch_mee_fused(p.gauge, p.spinor, p.compute, p.long_recon, m, s)) return 0;
    }
    {
        // both passes under one event pair, counted as two launches (their average duration is half
        // the span, and no event node breaks the programmatic dependent launch between them); the
        // reducing pass's summing launch is a reduction, timed with the BLAS kernels
        LaunchScope ls(c, s, kind, stencil_bytes(p, geom.vh, false) + stencil_bytes(p, geom.vh, true), 2);
        launch_dslash(p.gauge, p.spinor, p.compute, p.long_recon, false, d, s);
        d2.defer_finish = 1;
        launch_dslash(p.gauge, p.spinor, p.compute, p.long_recon, fin != FIN_NONE, d2, s);
    }
    if (fin == FIN_NONE) return 0;
    if (leave_partials) {
        // the partials of all blocks must fit the first half of the buffer
        const unsigned np = dslash_partials(p.gauge, p.spinor, p.compute, p.long_recon, geom);
        if ((size_t)np * 2 * sizeof(double) <= kSplitHalf * sizeof(double)) return np;
    }
    LaunchScope ls(c, s, PROF_BLAS, 0.0);
    launch_dslash_finish(p.gauge, p.spinor, p.compute, p.long_recon, d2, s);
    return 0;
}

void tune_stencil(hisq_ctx *c, const Geom &geom, const hisq_prec &p, const GaugeView &gv, char *zero_in, char *out,
                  cudaStream_t s)
{
    if (thread_capturing() || stream_capturing(s)) return;
    cudaMemsetAsync(zero_in, 0, spinor_field_bytes(p.spinor, geom.vh), s);
    DslashArgs d{};
    d.g = geom;
    d.gv = gv;
    d.err = cur_err(c);
    d.red = cur_red(c);
    d.out_parity = 1;
    d.in = zero_in;
    d.out = out;
    d.sign = 1;
    tune_dslash(p.gauge, p.spinor, p.compute, p.long_recon, d, s);
}

namespace {

struct CGRun {
    hisq_ctx *c;
    hisq_gauge *g;
    const CGConfig &cfg;
    cudaStream_t s;
    Workspace ws;
    int vh;
    size_t sb;
    char *r_s = nullptr, *ap_s = nullptr, *tmp_s = nullptr, *ring = nullptr;
    double *r64 = nullptr, *ax64 = nullptr, *tmp64 = nullptr;
    CGState *st = nullptr;
    CGState *st_h = nullptr;
    GaugeView gv_s{}, gv_d{};
    double diag = 0;
    int ru = 0, mv_hi = 0;
    // one mode for the whole solve (its graph is captured once); the FP64 triplet keeps the one-block
    // sums: its split r_update (82 registers, one 512-thread block a SM) measured 0.2 % slower
    const bool split = split_mode.load() != 0 && cfg.sloppy.spinor != S_F64;

    CGRun(hisq_ctx *c_, hisq_gauge *g_, const CGConfig &cfg_, cudaStream_t s_)
        : c(c_), g(g_), cfg(cfg_), s(s_), ws(c_, s_), vh(g_->geom.vh)
    {
    }
    ~CGRun()
    {
        if (st_h) cudaFreeHost(st_h);
    }

    char *slot(int j) { return ring + (size_t)j * sb; }

    BlasArgs blas() const
    {
        BlasArgs a{};
        a.n = vh;
        a.err = cur_err(c);
        a.red = cur_red(c);
        a.st = st;
        return a;
    }

    hisq_status setup()
    {
        hisq_status e = gauge_view_for(c, g, cfg.sloppy, &gv_s);
        if (!e) e = gauge_view_for(c, g, prec_f64(), &gv_d);
        if (e) return e;
        sb = spinor_field_bytes(cfg.sloppy.spinor, vh);
        const size_t b64 = (size_t)48 * vh;
        e = ws.alloc(sb, (void **)&r_s);
        if (!e) e = ws.alloc(sb, (void **)&ap_s);
        if (!e) e = ws.alloc(sb, (void **)&tmp_s);
        if (!e) e = ws.alloc(sb * cfg.nbuf, (void **)&ring);
        if (!e) e = ws.alloc(b64, (void **)&r64);
        if (!e) e = ws.alloc(b64, (void **)&ax64);
        if (!e) e = ws.alloc(b64, (void **)&tmp64);
        if (!e) e = ws.alloc(sizeof(CGState), (void **)&st);
        if (e) return e;
        if (cudaMallocHost(&st_h, sizeof(CGState)) != cudaSuccess)
            return fail(c, HISQ_ENOMEM, "pinned host state");
        cudaMemsetAsync(ring, 0, sb * cfg.nbuf, s);
        diag = 4.0 * cfg.mass * cfg.mass + cfg.sigma;
        tune_stencil(c, g->geom, cfg.sloppy, gv_s, ap_s, tmp_s, s);
        tune_stencil(c, g->geom, prec_f64(), gv_d, (char *)ax64, (char *)tmp64, s);
        return HISQ_OK;
    }

    hisq_status pull_state()
    {
        cudaMemcpyAsync(st_h, st, sizeof(CGState), cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "CG state");
        return HISQ_OK;
    }

    // x_hi += sum over the first nslots ring slots (alpha ring on the device)
    void flush(int nslots, const int *active, double *x64)
    {
        BlasArgs a = blas();
        a.v0 = ring;
        a.slot_bytes = sb;
        a.nslots = nslots;
        a.x64 = x64;
        a.active = active;
        LaunchScope ls(c, s, PROF_BLAS, (48.0 * 2 + (double)nslots * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
        launch_x_flush(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
    }

    // True residual and restart of the recurrence from p in slot j into slot 0.
    hisq_status reliable_update(const double *b64, double *x64, bool x_zero, int j)
    {
        if (!x_zero) {
            apply_mee(c, g->geom, prec_f64(), gv_d, diag, (const char *)x64, (char *)tmp64, (char *)ax64, FIN_NONE,
                      nullptr, 0, nullptr, PROF_STENCIL_HI, s);
            mv_hi++;
        }
        BlasArgs a = blas();
        a.b64 = b64;
        a.ax64 = x_zero ? nullptr : ax64;
        a.r64 = r64;
        a.v0 = r_s;
        a.v1 = slot(j);
        a.slot = j;
        {
            LaunchScope ls(c, s, PROF_BLAS, (48.0 * 3 + 2.0 * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
            launch_true_residual(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
        }
        a.v1 = slot(j);
        a.v2 = slot(0);
        {
            LaunchScope ls(c, s, PROF_BLAS, (48.0 + 2.0 * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
            launch_p_reliable(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
        }
        return pull_state();
    }

    // One block of nbuf iterations starting at ring slot 0.
    void iterate_block(double *x64)
    {
        const int N = cfg.nbuf;
        const int *act = &st->active;
        for (int i = 0; i < N; i++) {
            set_prof_tag(i);
            const unsigned np = apply_mee(c, g->geom, cfg.sloppy, gv_s, diag, slot(i), tmp_s, ap_s, FIN_CG_ALPHA, st,
                                          i, act, PROF_STENCIL, s, split);
            BlasArgs a = blas();
            a.active = act;
            a.slot = i;
            a.v0 = r_s;
            a.v1 = ap_s;
            a.split = np > 0;
            a.nparts = np;
            unsigned rp;
            {
                LaunchScope ls(c, s, PROF_BLAS, 3.0 * spinor_site_bytes(cfg.sloppy.spinor) * vh);
                rp = launch_r_update(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
            }
            a.nparts = rp;
            if (i == N - 1) flush(N, act, x64);
            a.v0 = r_s;
            a.v1 = slot(i);
            a.v2 = slot((i + 1) % N);
            a.clear_ring = i == N - 1;
            {
                LaunchScope ls(c, s, PROF_BLAS, 3.0 * spinor_site_bytes(cfg.sloppy.spinor) * vh);
                launch_p_update(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
            }
        }
        set_prof_tag(-1);
    }

    hisq_status run(const double *b64, double *x64, bool x_zero, hisq_solve_info *info)
    {
        hisq_status e = setup();
        if (e) return e;
        // |b|^2
        {
            BlasArgs a = blas();
            a.x64 = const_cast<double *>(b64);
            LaunchScope ls(c, s, PROF_BLAS, 48.0 * vh);
            launch_norm2(a, s);
        }
        double bb = 0.0;
        cudaMemcpyAsync(&bb, cur_red(c).result, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "norm");
        info->iters = 0;
        info->reliable_updates = 0;
        if (!std::isfinite(bb)) return fail(c, HISQ_EINVAL, "non-finite right-hand side");
        if (bb == 0.0) {
            cudaMemsetAsync(x64, 0, (size_t)48 * vh, s);
            info->true_residual = 0.0;
            cudaStreamSynchronize(s);
            return HISQ_OK;
        }
        CGState init{};
        init.delta2 = cfg.delta * cfg.delta;
        init.stop2 = cfg.tol * cfg.tol * bb;
        init.pr = cfg.pr;
        init.reproject = cfg.reproject;
        init.active = 1;
        init.dyn = cfg.dyn;
        init.dyn_eps = cfg.dyn_eps;
        init.dyn_hat = std::sqrt(cfg.dyn_eps);
        double *hist = nullptr;
        const int hlen = cfg.hist_host ? cfg.hist_len : 0;
        if (hlen > 0) {
            e = ws.alloc(sizeof(double) * hlen, (void **)&hist);
            if (e) return e;
            init.hist = hist;
            init.hist_len = hlen;
        }
        if (cfg.p_init) {
            // continue a previous recurrence: its gradient vector enters the
            // first restart (re-projected, with beta = |r_hi|^2 / rr_prev_init)
            LaunchScope ls(c, s, PROF_CONVERT, 2.0 * 48 * vh);
            launch_convert(cfg.p_init_fmt, cfg.sloppy.spinor, vh, cfg.p_init, slot(0), cur_err(c), s);
            init.rr_prev = cfg.rr_prev_init;
        }
        cudaMemcpyAsync(st, &init, sizeof init, cudaMemcpyHostToDevice, s);
        e = reliable_update(b64, x64, x_zero, 0);
        if (e) return e;
        hisq_status status = HISQ_OK;
        bool done = st_h->hi_rr <= init.stop2;
        // with the profiler on, the graph carries an event pair around each
        // launch; with a sample period above one, a second instance without
        // them runs the other blocks (event nodes cost device time)
        const bool graph = cfg.use_graph;
        const int every = c->prof.on ? c->prof.every : 1;
        cudaGraphExec_t exec = nullptr, exec_plain = nullptr;
        int64_t nodes = 0;
        int64_t block = 0;
        std::vector<Profiler::Rec> grecs;
        auto capture = [&](bool record, cudaGraphExec_t *out) -> cudaError_t {
            cudaGraph_t gr = nullptr;
            set_thread_capturing(true);
            if (record) set_graph_recorder(&grecs);
            cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                iterate_block(x64);
                ce = cudaStreamEndCapture(s, &gr);
            }
            set_graph_recorder(nullptr);
            set_thread_capturing(false);
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(out, gr, 0);
            size_t nn = 0;
            if (ce == cudaSuccess) ce = graph_kernel_nodes(gr, &nn);
            if (gr) cudaGraphDestroy(gr);
            nodes = (int64_t)nn;
            return ce;
        };
        while (!done) {
            if (st_h->k >= cfg.maxiter) {
                status = HISQ_ENOTCONV;
                break;
            }
            const int k0 = st_h->k;
            const bool timed = !graph || block % every == 0;
            if (graph) {
                cudaGraphExec_t *ex = (timed || !c->prof.on) ? &exec : &exec_plain;
                if (!*ex) {
                    const cudaError_t ce = capture(c->prof.on && ex == &exec, ex);
                    if (ce != cudaSuccess) {
                        if (exec) cudaGraphExecDestroy(exec);
                        if (exec_plain) cudaGraphExecDestroy(exec_plain);
                        prof_graph_release(c, grecs);
                        return cuda_fail(c, ce, "CG graph capture");
                    }
                }
                cudaGraphLaunch(*ex, s);
                c->launches += nodes;
            } else {
                iterate_block(x64);
            }
            block++;
            e = pull_state();
            if (e) break;
            if (!graph)
                prof_settle(c, st_h->k - k0);
            else if (timed)
                prof_graph_account(c, grecs, st_h->k - k0);
            const int reason = st_h->reason;
            if (reason == REASON_BREAKDOWN) {
                status = HISQ_EBREAKDOWN;
                fail(c, HISQ_EBREAKDOWN, "CG breakdown at iteration %d (non-positive p.Ap or non-finite scalar)",
                     st_h->k);
                break;
            }
            if (reason == REASON_RELIABLE || reason == REASON_CONVERGED) {
                const int j = st_h->k - k0 - 1;
                flush(j + 1, nullptr, x64);
                e = reliable_update(b64, x64, false, j);
                if (e) break;
                ru++;
                done = st_h->hi_rr <= init.stop2;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_plain) cudaGraphExecDestroy(exec_plain);
        prof_graph_release(c, grecs);
        if (e) return e;
        if (status != HISQ_OK) {
            // bring x up to date (an unfinished block's slots) and measure it
            if (status == HISQ_EBREAKDOWN) flush(cfg.nbuf, nullptr, x64);
            e = reliable_update(b64, x64, false, 0);
            if (e) return e;
        }
        int herr = 0;
        cudaMemcpyAsync(&herr, cur_err(c), sizeof herr, cudaMemcpyDeviceToHost, s);
        std::vector<double> hv;
        if (hlen > 0) {
            // entries 0..k (|r|^2 per iteration, the true residual at reliable updates)
            hv.resize(std::min(hlen, st_h->k + 1));
            cudaMemcpyAsync(hv.data(), hist, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, s);
        }
        cudaStreamSynchronize(s);
        for (size_t i = 0; i < hv.size(); i++) cfg.hist_host[i] = std::sqrt(hv[i] / bb);
        info->iters = st_h->k;
        info->matvecs += st_h->k;
        info->matvecs_hi += mv_hi;
        info->reliable_updates += ru;
        info->true_residual = std::sqrt(st_h->hi_rr / bb);
        if (herr & 2)  // a bounded wait of the fused M_ee pass gave up: its results are not trusted
            return fail(c, HISQ_ECUDA, "fused M_ee pass: a wait for earlier t-slices reached its limit");
        if (status == HISQ_ENOTCONV)
            fail(c, HISQ_ENOTCONV, "CG reached maxiter=%d with true residual %.3e", cfg.maxiter, info->true_residual);
        return status;
    }
};

}  // namespace

hisq_status run_cg(hisq_ctx *c, hisq_gauge *g, const CGConfig &cfg, const double *b64, double *x64, bool x_zero,
                   hisq_solve_info *info, cudaStream_t s)
{
    CGRun run(c, g, cfg, s);
    return run.run(b64, x64, x_zero, info);
}

hisq_status validate_params(hisq_ctx *c, const hisq_solver_params *p)
{
    if (!p) return fail(c, HISQ_EINVAL, "null parameters");
    if (!std::isfinite(p->mass) || !(p->tol > 0.0) || p->maxiter < 0 || !(p->delta >= 0.0 && p->delta < 1.0))
        return fail(c, HISQ_EINVAL, "bad solver parameters (mass, tol > 0, maxiter >= 0, 0 <= delta < 1)");
    if (p->nbuf < 1 || p->nbuf > kMaxBuf) return fail(c, HISQ_EINVAL, "nbuf must be in 1..%d", kMaxBuf);
    if (p->ru_trigger < 0 || p->ru_trigger > 1) return fail(c, HISQ_EINVAL, "ru_trigger must be 0 or 1");
    if (p->history_len < 0 || (p->history_len > 0 && !p->history))
        return fail(c, HISQ_EINVAL, "history_len must be >= 0, with a history array when > 0");
    return check_prec(c, p->sloppy);
}

double sloppy_eps(const hisq_prec &p)
{
    double es = 0x1p-29;  // 30-bit
    if (p.spinor == S_F64) es = 0x1p-53;
    if (p.spinor == S_F32) es = 0x1p-24;
    if (p.spinor == S_HALF) es = 0x1p-15;
    if (p.spinor == S_INT20) es = 0x1p-19;
    if (p.spinor == S_INT14) es = 0x1p-13;
    double eg = 0x1p-31;  // 32-bit fixed point
    if (p.gauge == G_F64) eg = 0x1p-53;
    if (p.gauge == G_F32) eg = 0x1p-24;
    if (p.gauge == G_FIX16) eg = 0x1p-15;
    const double ec = p.compute == HISQ_COMPUTE_F32 ? 0x1p-24 : 0x1p-53;
    return std::max(es, std::max(eg, ec));
}

// Caller layout [site][6] (host or device) <-> FP64 planar device field.
hisq_status to_planar(hisq_ctx *c, Workspace &ws, const double *user, int on_device, int64_t n, double *planar,
                      cudaStream_t s)
{
    const double *src = user;
    if (!on_device) {
        double *stage = nullptr;
        hisq_status e = ws.alloc((size_t)48 * n, (void **)&stage);
        if (e) return e;
        cudaMemcpyAsync(stage, user, (size_t)48 * n, cudaMemcpyHostToDevice, s);
        src = stage;
    }
    cudaMemsetAsync(cur_err(c), 0, sizeof(int), s);
    {
        LaunchScope ls(c, s, PROF_CONVERT, 96.0 * n);
        launch_pack_spinor(S_F64, n, src, (char *)planar, cur_err(c), s);
    }
    int bad = 0;
    cudaMemcpyAsync(&bad, cur_err(c), sizeof bad, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload");
    if (bad) return fail(c, HISQ_EINVAL, "non-finite input vector");
    return HISQ_OK;
}

hisq_status from_planar(hisq_ctx *c, Workspace &ws, const double *planar, int64_t n, double *user, int on_device,
                        cudaStream_t s)
{
    double *dst = user;
    if (!on_device) {
        hisq_status e = ws.alloc((size_t)48 * n, (void **)&dst);
        if (e) return e;
    }
    {
        LaunchScope ls(c, s, PROF_CONVERT, 96.0 * n);
        launch_unpack_spinor(S_F64, HISQ_COMPUTE_F64, n, (const char *)planar, dst, s);
    }
    if (!on_device) cudaMemcpyAsync(user, dst, (size_t)48 * n, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "download");
    return HISQ_OK;
}

CGConfig config_from(const hisq_solver_params *p, double sigma)
{
    CGConfig cfg;
    cfg.mass = p->mass;
    cfg.sigma = sigma;
    cfg.tol = p->tol;
    cfg.maxiter = p->maxiter;
    cfg.delta = p->delta;
    cfg.sloppy = p->sloppy;
    cfg.nbuf = p->nbuf;
    cfg.pr = p->pr_beta;
    cfg.reproject = p->reproject;
    cfg.use_graph = p->use_graph;
    cfg.dyn = p->ru_trigger;
    cfg.dyn_eps = p->ru_trigger ? sloppy_eps(p->sloppy) : 0.0;
    return cfg;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

void hisq_default_params(hisq_solver_params *p)
{
    if (!p) return;
    *p = hisq_solver_params{};
    p->mass = 0.1;
    p->tol = 1e-10;
    p->maxiter = 100000;
    p->delta = 0.1;
    hisq_prec s;
    s.gauge = HISQ_GAUGE_FIX16;
    s.spinor = HISQ_SPINOR_INT20;
    s.compute = HISQ_COMPUTE_F32;
    s.fat_recon = 18;
    s.long_recon = 12;
    p->sloppy = s;
    p->refine = s;
    p->nbuf = 8;
    p->use_init_guess = 0;
    p->on_device = 0;
    p->pr_beta = 1;
    p->reproject = 1;
    p->l = 4;
    p->use_graph = 1;
    p->nrhs = 1;
    p->rhs_tile = 0;
    p->rhs_kernel = 0;
    p->stream = nullptr;
    p->history = nullptr;
    p->history_len = 0;
    p->ru_trigger = 0;
}

hisq_status hisq_cg(hisq_ctx *c, const hisq_gauge *gc, const hisq_solver_params *p, const double *b, double *x,
                    hisq_solve_info *info)
{
    if (!c || !gc || !b || !x || !info) return fail(c, HISQ_EINVAL, "hisq_cg: null argument");
    *info = hisq_solve_info{};
    hisq_status e = validate_params(c, p);
    if (e) return e;
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    hisq_gauge *g = const_cast<hisq_gauge *>(gc);
    cudaStream_t s = pick_stream(c, p->stream);
    const int64_t vh = g->geom.vh;
    const int nr = p->nrhs;
    if (nr < 1 || nr > kMaxRHS) return fail(c, HISQ_EINVAL, "nrhs must be in 1..%d", kMaxRHS);
    if (!solver_red_fits(vh)) return fail(c, HISQ_EINVAL, "lattice too large for the solvers' reductions");
    if (p->rhs_tile < 0 || p->rhs_tile > kMaxRHS || (p->rhs_tile > 0 && nr % p->rhs_tile))
        return fail(c, HISQ_EINVAL, "rhs_tile must divide nrhs");
    if (p->rhs_kernel < 0 || p->rhs_kernel > 2 ||
        (p->rhs_kernel == 2 && p->sloppy.spinor != HISQ_SPINOR_HALF16 && p->sloppy.spinor != HISQ_SPINOR_INT20))
        return fail(c, HISQ_EINVAL, "rhs_kernel must be 0, 1, or 2 with a 16- or 20-bit sloppy fermion");
    Workspace ws(c, s);
    double *b64 = nullptr, *x64 = nullptr;
    e = ws.alloc((size_t)48 * vh * nr, (void **)&b64);
    if (!e) e = ws.alloc((size_t)48 * vh * nr, (void **)&x64);
    for (int t = 0; t < nr && !e; t++) {
        e = to_planar(c, ws, b + (size_t)t * 6 * vh, p->on_device, vh, b64 + (size_t)t * 6 * vh, s);
        if (!e && p->use_init_guess)
            e = to_planar(c, ws, x + (size_t)t * 6 * vh, p->on_device, vh, x64 + (size_t)t * 6 * vh, s);
    }
    if (!e && !p->use_init_guess) cudaMemsetAsync(x64, 0, (size_t)48 * vh * nr, s);
    if (e) return e;
    hisq_status st;
    if (nr == 1) {
        CGConfig cfg = config_from(p, 0.0);
        cfg.hist_host = p->history;
        cfg.hist_len = p->history_len;
        st = run_cg(c, g, cfg, b64, x64, !p->use_init_guess, info, s);
    } else {
        if (p->history_len > 0) return fail(c, HISQ_EINVAL, "a residual history is kept for nrhs = 1 only");
        BCGConfig bc;
        bc.nrhs = nr;
        for (int t = 0; t < nr; t++) {
            bc.diag[t] = 4.0 * p->mass * p->mass;
            bc.tol[t] = p->tol;
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
        st = run_bcg(c, g, bc, b64, x64, !p->use_init_guess, infos.data(), s);
        for (int t = 0; t < nr; t++) {
            info->iters = std::max(info->iters, infos[t].iters);
            info->matvecs += infos[t].matvecs;
            info->matvecs_hi += infos[t].matvecs_hi;
            info->reliable_updates += infos[t].reliable_updates;
            info->true_residual = std::max(info->true_residual, infos[t].true_residual);
        }
    }
    if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) return st;
    for (int t = 0; t < nr && !e; t++)
        e = from_planar(c, ws, x64 + (size_t)t * 6 * vh, vh, x + (size_t)t * 6 * vh, p->on_device, s);
    if (e) return e;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // extern "C"
