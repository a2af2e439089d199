// bcg.cu -- batched mixed-precision CG: nrhs independent even/odd systems
// (M_ee + sigma_t) x_t = b_t iterated together so that every stencil pass
// loads each link once for a tile of right-hand sides (Sec. 1, block solvers).
//
// Each right-hand side keeps the full stabilised recurrence of cg.cu (its own
// ring of buffered gradient vectors, reliable updates, re-projection,
// Polak-Ribiere beta) and its own device-side scalar state; a right-hand side
// that stops (reliable update, convergence, breakdown, maxiter) only freezes
// its own state while the others keep iterating.  Every per-RHS quantity is
// computed by the same operations whatever the batch composition, so a
// right-hand side's iterates do not depend on which others share its batch
// (only on the tile size T of the stencil).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "bcg.h"
#include "blas.h"
#include "cg.h"
#include "codecs.cuh"
#include "finish.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace hisq {

namespace {

constexpr int kBlock = 256;

struct BBArgs {
    int n, nrhs;
    size_t fb;          // bytes of one sloppy half-lattice field
    char *r, *ap;       // [nrhs] fields
    char *p_in, *p_out; // ring slots: [nrhs] fields each
    char *ring;         // [nbuf][nrhs] fields
    int nslots;
    int clear_ring;
    double *x64;        // [nrhs] FP64 planar fields (48 n bytes each)
    CGState *st;
    int *err;
    RedBuf red;
};

// r_t -= alpha_t Ap_t for active t; per-RHS |r_t|^2 and Re<r_t new, r_t old>
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) b_r_update_kernel(BBArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    real v[2 * kMaxRHS];
#pragma unroll
    for (int k = 0; k < 2 * kMaxRHS; k++) v[k] = 0;
    if (i < a.n) {
#pragma unroll
        for (int t = 0; t < kMaxRHS; t++) {
            if (t >= a.nrhs || !a.st[t].active) continue;
            real r[6], ap[6];
            char *rf = a.r + (size_t)t * a.fb;
            Spinor<SF>::load(rf, a.n, i, r);
            Spinor<SF>::load(a.ap + (size_t)t * a.fb, a.n, i, ap);
            const real alpha = (real)a.st[t].alpha;
            real n2 = 0, d = 0;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const real rn = r[k] - alpha * ap[k];
                n2 += rn * rn;
                d += rn * r[k];
                r[k] = rn;
            }
            v[2 * t] = n2;
            v[2 * t + 1] = d;
            if (!Spinor<SF>::store(rf, a.n, i, r)) atomicExch(a.err, 1);
        }
    }
    __shared__ double tot[2 * kMaxRHS];
    if (reduce_grid<2 * kMaxRHS>(v, a.red, tot) && threadIdx.x == 0)
        run_batch_finisher(FIN_CG_BETA, tot, a.st, 0, a.nrhs, 0);
}

// p_out_t = r_t + beta_t p_in_t for active t
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) b_p_update_kernel(BBArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (a.clear_ring && i == 0)
        for (int t = 0; t < a.nrhs; t++)
            if (a.st[t].active)
                for (int j = 0; j < kMaxBuf; j++) a.st[t].alpha_ring[j] = 0.0;
    if (i >= a.n) return;
    for (int t = 0; t < a.nrhs; t++) {
        if (!a.st[t].active) continue;
        real r[6], p[6];
        Spinor<SF>::load(a.r + (size_t)t * a.fb, a.n, i, r);
        Spinor<SF>::load(a.p_in + (size_t)t * a.fb, a.n, i, p);
        const real beta = (real)a.st[t].beta;
#pragma unroll
        for (int k = 0; k < 6; k++) p[k] = r[k] + beta * p[k];
        if (!Spinor<SF>::store(a.p_out + (size_t)t * a.fb, a.n, i, p)) atomicExch(a.err, 1);
    }
}

// x_t += sum_j alpha_{t,j} p_{t,j} for active t (increment in the compute precision)
template <int SF, typename real>
__global__ void __launch_bounds__(kBlock) b_flush_kernel(BBArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    for (int t = 0; t < a.nrhs; t++) {
        if (!a.st[t].active) continue;
        real dx[6] = {0, 0, 0, 0, 0, 0};
        for (int j = 0; j < a.nslots; j++) {
            const real al = (real)a.st[t].alpha_ring[j];
            if (al == real(0)) continue;
            real p[6];
            Spinor<SF>::load(a.ring + ((size_t)j * a.nrhs + t) * a.fb, a.n, i, p);
#pragma unroll
            for (int k = 0; k < 6; k++) dx[k] += al * p[k];
        }
        char *xf = reinterpret_cast<char *>(a.x64) + (size_t)t * 48 * a.n;
        double x[6];
        Spinor<S_F64>::load(xf, a.n, i, x);
#pragma unroll
        for (int k = 0; k < 6; k++) x[k] += (double)dx[k];
        Spinor<S_F64>::store(xf, a.n, i, x);
    }
}

#define BB_DISPATCH(SF_, CF_, KERNEL)                                                             \
    do {                                                                                         \
        const int nb_ = (a.n + kBlock - 1) / kBlock;                                             \
        switch (SF_) {                                                                           \
        case S_F32: KERNEL<S_F32, float><<<nb_, kBlock, 0, s>>>(a); break;                       \
        case S_HALF: KERNEL<S_HALF, float><<<nb_, kBlock, 0, s>>>(a); break;                     \
        case S_INT20: KERNEL<S_INT20, float><<<nb_, kBlock, 0, s>>>(a); break;                   \
        default: break;                                                                          \
        }                                                                                        \
    } while (0)

using TileKey = std::array<int, 10>;
// The fastest (T, variant) for a full batch, and per tile size (index log2 T)
// the time of one tile launch with its fastest variant (ms; < 0: not timed).
struct TileChoice {
    int T, variant;
    float tile_ms[5];
    int tile_var[5];
};
std::mutex tile_mu;
std::map<TileKey, TileChoice> tile_cache;

// The tile size T (dividing nrhs; only `fixed` if that is > 0) and kernel
// variant with the fastest batched pass, timed once per (triplet, nrhs,
// lattice) on zero fields.
TileChoice tune_tile(hisq_ctx *c, const Geom &geom, const hisq_prec &p, const GaugeView &gv, int nrhs, int fixed,
                     int kernel, char *in, char *out, size_t fb, cudaStream_t s)
{
    const TileKey key = {p.gauge, p.spinor, p.compute, p.long_recon, nrhs, fixed * 4 + kernel, geom.L[0], geom.L[1],
                         geom.L[2], geom.L[3]};
    {
        std::lock_guard<std::mutex> lk(tile_mu);
        auto it = tile_cache.find(key);
        if (it != tile_cache.end()) return it->second;
    }
    TileChoice best = {fixed > 0 ? fixed : 1, kernel == 2 ? 1 : 0, {-1.f, -1.f, -1.f, -1.f, -1.f}, {0, 0, 0, 0, 0}};
    if (!thread_capturing() && !stream_capturing(s)) {
        cudaMemsetAsync(in, 0, fb * nrhs, s);
        DslashMArgs d{};
        d.g = geom;
        d.gv = gv;
        d.out_parity = 1;
        d.in = in;
        d.out = out;
        d.field_bytes = fb;
        d.sign = 1;
        d.nrhs = nrhs;
        d.err = cur_err(c);
        d.red = cur_red(c);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        for (int T = 1, ti = 0; T <= 16; T *= 2, ti++) {
            if (nrhs % T || (fixed > 0 && T != fixed) || !red_fits(geom.vh, kMrhsBlock, 2 * T)) continue;
            for (int v = 0; v < 2; v++) {
                if (kernel > 0 && v != kernel - 1) continue;
                if (!launch_dslash_mrhs(p.gauge, p.spinor, p.compute, p.long_recon, false, T, v, d, s)) continue;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 2; r++) launch_dslash_mrhs(p.gauge, p.spinor, p.compute, p.long_recon, false, T, v, d, s);
                cudaEventRecord(e1, s);
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
                const float per_tile = ms / 2.0f / (float)(nrhs / T);
                if (best.tile_ms[ti] < 0.f || per_tile < best.tile_ms[ti]) {
                    best.tile_ms[ti] = per_tile;
                    best.tile_var[ti] = v;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best.T = T;
                    best.variant = v;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        (void)cudaGetLastError();
        // first result wins (a concurrent tuning of the same key keeps it)
        std::lock_guard<std::mutex> lk(tile_mu);
        return tile_cache.emplace(key, best).first->second;
    }
    return best;
}

}  // namespace

// ---------------------------------------------------------------------------
// A batch of `capacity` solver slots sharing every stencil launch.  A slot is
// loaded with a system (its right-hand side is copied in), iterated block by
// block together with the other occupied slots, and harvested when it stops;
// a freed slot can be loaded again at any block boundary (continuous
// batching).  Empty and stopped slots are inactive: the BLAS kernels skip
// them, the stencil skips tiles in which every slot is inactive (slots are
// filled lowest first).
// ---------------------------------------------------------------------------
BatchSession::BatchSession(hisq_ctx *c_, hisq_gauge *g_, const BCGConfig &cfg_, cudaStream_t s_)
    : c(c_), g(g_), cfg(cfg_), s(s_), ws(c_, s_), vh(g_->geom.vh), nr(cfg_.nrhs), N(cfg_.nbuf)
{
}

BatchSession::~BatchSession()
{
    for (auto &kv : graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (sth) cudaFreeHost(sth);
}

char *BatchSession::slot(int j, int t) { return ring + ((size_t)j * nr + t) * fb; }

double *BatchSession::x_of(int t) { return x64 + (size_t)t * 6 * vh; }

double *BatchSession::b_of(int t) { return b64 + (size_t)t * 6 * vh; }

namespace {

BBArgs bb_args(const BatchSession &b)
{
    BBArgs a{};
    a.n = b.vh;
    a.nrhs = b.nr;
    a.fb = b.fb;
    a.r = b.r_s;
    a.ap = b.ap_s;
    a.ring = b.ring;
    a.st = b.st;
    a.err = cur_err(b.c);
    a.red = cur_red(b.c);
    return a;
}

}  // namespace

void BatchSession::stencil_pass(int parity_out, const char *in, char *out, const char *y, bool red, int slot_i)
{
    DslashMArgs d{};
    d.g = g->geom;
    d.gv = gv_s;
    d.out_parity = parity_out;
    d.in = in;
    d.out = out;
    d.y = y;
    d.field_bytes = fb;
    d.nrhs = nr;
    d.err = cur_err(c);
    d.red = cur_red(c);
    d.st = st;
    d.slot = slot_i;
    d.tile_mask = tile_mask;
    if (y) {
        d.xpay = 1;
        d.sign = -1;
        d.fin = FIN_CG_ALPHA;
    } else {
        d.sign = 1;
    }
    const double links = 8.0 * link_bytes(cfg.sloppy.gauge, 18) + 8.0 * link_bytes(cfg.sloppy.gauge, cfg.sloppy.long_recon);
    const double sb = (double)spinor_site_bytes(cfg.sloppy.spinor) * vh;
    LaunchScope ls(c, s, PROF_STENCIL, links * vh * (nr / T) + (y ? 3.0 : 2.0) * sb * nr);
    launch_dslash_mrhs(cfg.sloppy.gauge, cfg.sloppy.spinor, cfg.sloppy.compute, cfg.sloppy.long_recon, red, T, variant, d,
                       s);
}

void BatchSession::iterate_block()
{
    const double sb = (double)spinor_site_bytes(cfg.sloppy.spinor) * vh;
    for (int i = 0; i < N; i++) {
        stencil_pass(1, slot(i, 0), tmp_s, nullptr, false, i);
        stencil_pass(0, tmp_s, ap_s, slot(i, 0), true, i);
        BBArgs a = bb_args(*this);
        {
            LaunchScope ls(c, s, PROF_BLAS, 3.0 * sb * nr);
            BB_DISPATCH(cfg.sloppy.spinor, cfg.sloppy.compute, b_r_update_kernel);
        }
        if (i == N - 1) {
            a.x64 = x64;
            a.nslots = N;
            LaunchScope ls(c, s, PROF_BLAS, (96.0 + N * spinor_site_bytes(cfg.sloppy.spinor)) * vh * nr);
            BB_DISPATCH(cfg.sloppy.spinor, cfg.sloppy.compute, b_flush_kernel);
        }
        a.p_in = slot(i, 0);
        a.p_out = slot((i + 1) % N, 0);
        a.clear_ring = i == N - 1;
        LaunchScope ls(c, s, PROF_BLAS, 3.0 * sb * nr);
        BB_DISPATCH(cfg.sloppy.spinor, cfg.sloppy.compute, b_p_update_kernel);
    }
}

hisq_status BatchSession::pull()
{
    cudaMemcpyAsync(sth, st, sizeof(CGState) * nr, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HISQ_OK : cuda_fail(c, e, "batched CG state");
}

void BatchSession::reliable_update(int t, int nslots, int j, bool x_zero)
{
    double *xt = x_of(t);
    const double *bt = b_of(t);
    if (nslots > 0) {
        BlasArgs f{};
        f.n = vh;
        f.err = cur_err(c);
        f.red = cur_red(c);
        f.st = st + t;
        f.v0 = slot(0, t);
        f.slot_bytes = fb * nr;
        f.nslots = nslots;
        f.x64 = xt;
        LaunchScope ls(c, s, PROF_BLAS, (96.0 + nslots * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
        launch_x_flush(cfg.sloppy.spinor, cfg.sloppy.compute, f, s);
    }
    if (!x_zero) {
        apply_mee(c, g->geom, prec_f64(), gv_d, diag[t], (const char *)xt, (char *)tmp64, (char *)ax64, FIN_NONE,
                  nullptr, 0, nullptr, PROF_STENCIL_HI, s);
        mv_hi[t]++;
    }
    BlasArgs a{};
    a.n = vh;
    a.err = cur_err(c);
    a.red = cur_red(c);
    a.st = st + t;
    a.b64 = bt;
    a.ax64 = x_zero ? nullptr : ax64;
    a.r64 = r64;
    a.v0 = r_s + (size_t)t * fb;
    a.v1 = slot(j, t);
    a.slot = j;
    {
        LaunchScope ls(c, s, PROF_BLAS, (48.0 * 3 + 2.0 * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
        launch_true_residual(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
    }
    a.v1 = slot(j, t);
    a.v2 = slot(0, t);
    LaunchScope ls(c, s, PROF_BLAS, (48.0 + 2.0 * spinor_site_bytes(cfg.sloppy.spinor)) * vh);
    launch_p_reliable(cfg.sloppy.spinor, cfg.sloppy.compute, a, s);
}

hisq_status BatchSession::setup()
{
    hisq_status e = gauge_view_for(c, g, cfg.sloppy, &gv_s);
    if (!e) e = gauge_view_for(c, g, prec_f64(), &gv_d);
    if (e) return e;
    fb = spinor_field_bytes(cfg.sloppy.spinor, vh);
    e = ws.alloc(fb * nr, (void **)&r_s);
    if (!e) e = ws.alloc(fb * nr, (void **)&ap_s);
    if (!e) e = ws.alloc(fb * nr, (void **)&tmp_s);
    if (!e) e = ws.alloc(fb * nr * N, (void **)&ring);
    if (!e) e = ws.alloc((size_t)48 * vh * nr, (void **)&b64);
    if (!e) e = ws.alloc((size_t)48 * vh * nr, (void **)&x64);
    if (!e) e = ws.alloc((size_t)48 * vh, (void **)&r64);
    if (!e) e = ws.alloc((size_t)48 * vh, (void **)&ax64);
    if (!e) e = ws.alloc((size_t)48 * vh, (void **)&tmp64);
    if (!e) e = ws.alloc(sizeof(CGState) * nr, (void **)&st);
    if (e) return e;
    if (cudaMallocHost(&sth, sizeof(CGState) * nr) != cudaSuccess) return fail(c, HISQ_ENOMEM, "pinned state");
    mv_hi.assign(nr, 0);
    ru.assign(nr, 0);
    k0.assign(nr, 0);
    occupied.assign(nr, 0);
    status.assign(nr, HISQ_OK);
    bb.assign(nr, 0.0);
    stop2.assign(nr, 0.0);
    diag.assign(nr, 0.0);
    const TileChoice tc = tune_tile(c, g->geom, cfg.sloppy, gv_s, nr, cfg.tile, cfg.kernel, ap_s, tmp_s, fb, s);
    T = tc.T;
    variant = tc.variant;
    for (int i = 0; i < 5; i++) {
        tile_ms[i] = tc.tile_ms[i];
        tile_var[i] = tc.tile_var[i];
    }
    adapt = cfg.tile == 0 && cfg.kernel == 0;
    if (nr % T) return fail(c, HISQ_EINVAL, "RHS tile %d does not divide nrhs %d", T, nr);
    if (!red_fits(vh, kMrhsBlock, 2 * T) || !red_fits(vh, kBlock, 2 * kMaxRHS))
        return fail(c, HISQ_EINVAL, "lattice too large for a batched reduction over a tile of %d", T);
    tune_stencil(c, g->geom, prec_f64(), gv_d, (char *)ax64, (char *)tmp64, s);
    cudaMemsetAsync(ring, 0, fb * nr * N, s);
    cudaMemsetAsync(r_s, 0, fb * nr, s);
    cudaMemsetAsync(b64, 0, (size_t)48 * vh * nr, s);
    cudaMemsetAsync(x64, 0, (size_t)48 * vh * nr, s);
    std::vector<CGState> zero(nr);
    for (auto &z : zero) z = CGState{};
    cudaMemcpyAsync(st, zero.data(), sizeof(CGState) * nr, cudaMemcpyHostToDevice, s);
    return pull();
}

hisq_status BatchSession::load(int t, const double *b_planar, const double *x_planar, double diag_t, double tol_t)
{
    if (t < 0 || t >= nr || occupied[t]) return fail(c, HISQ_EINVAL, "slot %d is not free", t);
    cudaMemcpyAsync(b_of(t), b_planar, (size_t)48 * vh, cudaMemcpyDeviceToDevice, s);
    if (x_planar)
        cudaMemcpyAsync(x_of(t), x_planar, (size_t)48 * vh, cudaMemcpyDeviceToDevice, s);
    else
        cudaMemsetAsync(x_of(t), 0, (size_t)48 * vh, s);
    for (int j = 0; j < N; j++) cudaMemsetAsync(slot(j, t), 0, fb, s);
    BlasArgs a{};
    a.n = vh;
    a.red = cur_red(c);
    a.x64 = b_of(t);
    launch_norm2(a, s);
    double b2 = 0.0;
    cudaMemcpyAsync(&b2, cur_red(c).result, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "norm");
    if (!std::isfinite(b2)) return fail(c, HISQ_EINVAL, "non-finite right-hand side");
    bb[t] = b2;
    diag[t] = diag_t;
    stop2[t] = tol_t * tol_t * b2;
    mv_hi[t] = 0;
    ru[t] = 0;
    status[t] = HISQ_OK;
    occupied[t] = 1;
    CGState init{};
    init.delta2 = cfg.delta * cfg.delta;
    init.dyn = cfg.dyn;
    init.dyn_eps = cfg.dyn_eps;
    init.dyn_hat = std::sqrt(cfg.dyn_eps);
    init.stop2 = stop2[t];
    init.pr = cfg.pr;
    init.reproject = cfg.reproject;
    init.diag = diag_t;
    init.active = 1;
    cudaMemcpyAsync(st + t, &init, sizeof init, cudaMemcpyHostToDevice, s);
    if (b2 == 0.0) {
        cudaMemsetAsync(x_of(t), 0, (size_t)48 * vh, s);
        cudaMemsetAsync(&st[t].active, 0, sizeof(int), s);
        finished_now.push_back(t);
        return pull();
    }
    reliable_update(t, 0, 0, x_planar == nullptr);
    hisq_status e = pull();
    if (e) return e;
    if (sth[t].hi_rr <= stop2[t]) {
        cudaMemsetAsync(&st[t].active, 0, sizeof(int), s);
        finished_now.push_back(t);
        return pull();
    }
    return HISQ_OK;
}

int BatchSession::active_slots() const
{
    int n = 0;
    for (int t = 0; t < nr; t++)
        if (occupied[t] && std::find(finished_now.begin(), finished_now.end(), t) == finished_now.end()) n++;
    return n;
}

// The tile for the next block of iterations.  Each right-hand side's
// arithmetic is the same whatever its tile and kernel (lane-wise operations,
// per-RHS partial sums over the same blocks), so the choice changes only the
// cost: with the timed cost of one tile launch per tile size, pick the size
// whose tiles holding an iterating system cost least, and launch only those
// tiles (a session whose systems are finishing one by one then pays for the
// systems left, not for the whole batch).
void BatchSession::choose_tile()
{
    unsigned live = 0;
    for (int t = 0; t < nr; t++)
        if (occupied[t] && std::find(finished_now.begin(), finished_now.end(), t) == finished_now.end())
            live |= 1u << t;
    auto tiles_of = [&](int TT) {
        unsigned m = 0;
        for (int k = 0; k * TT < nr; k++)
            if ((live >> (k * TT)) & ((1u << TT) - 1u)) m |= 1u << k;
        return m;
    };
    if (adapt) {
        float best = 1e30f;
        int bT = T, bv = variant;
        for (int TT = 1, ti = 0; TT <= kMaxRHS; TT *= 2, ti++) {
            if (nr % TT || tile_ms[ti] < 0.f) continue;
            const float cost = tile_ms[ti] * (float)__builtin_popcount(tiles_of(TT));
            if (cost < best) {
                best = cost;
                bT = TT;
                bv = tile_var[ti];
            }
        }
        T = bT;
        variant = bv;
    }
    tile_mask = tiles_of(T);
}

hisq_status BatchSession::step()
{
    for (int t = 0; t < nr; t++) k0[t] = sth[t].k;
    choose_tile();
    const bool graph = cfg.use_graph && !c->prof.on;
    if (graph) {
        const uint64_t key = (uint64_t)T | ((uint64_t)variant << 8) | ((uint64_t)tile_mask << 16);
        Graph &gg = graphs[key];
        if (!gg.exec) {
            if (graphs.size() > 64) {  // bound the cache: rebuild graphs as they are needed again
                for (auto &kv : graphs)
                    if (kv.second.exec && kv.first != key) cudaGraphExecDestroy(kv.second.exec);
                graphs.clear();
            }
            Graph &ng = graphs[key];
            cudaGraph_t gr = nullptr;
            set_thread_capturing(true);
            cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                iterate_block();
                ce = cudaStreamEndCapture(s, &gr);
            }
            set_thread_capturing(false);
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ng.exec, gr, 0);
            size_t nn = 0;
            if (ce == cudaSuccess) ce = graph_kernel_nodes(gr, &nn);
            if (gr) cudaGraphDestroy(gr);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "batched CG graph capture");
            ng.nodes = (int64_t)nn;
        }
        const Graph &run = graphs[key];
        cudaGraphLaunch(run.exec, s);
        c->launches += run.nodes;
    } else {
        iterate_block();
    }
    hisq_status e = pull();
    if (e) return e;
    bool touched = false;
    std::vector<int> stop_now;
    for (int t = 0; t < nr; t++) {
        if (!occupied[t]) continue;
        if (std::find(finished_now.begin(), finished_now.end(), t) != finished_now.end()) continue;
        const CGState &h = sth[t];
        if (h.reason == REASON_BREAKDOWN) {
            status[t] = HISQ_EBREAKDOWN;
            reliable_update(t, N, 0, false);  // bring x up to date and measure it
            stop_now.push_back(t);
            touched = true;
        } else if (h.reason == REASON_RELIABLE || h.reason == REASON_CONVERGED) {
            const int j = h.k - k0[t] - 1;
            reliable_update(t, j + 1, j, false);
            ru[t]++;
            touched = true;
        } else if (h.k >= cfg.maxiter) {
            reliable_update(t, 0, 0, false);  // a block boundary: the ring was just flushed
            status[t] = HISQ_ENOTCONV;
            stop_now.push_back(t);
            touched = true;
        }
    }
    if (touched) {
        e = pull();
        if (e) return e;
        for (int t = 0; t < nr; t++) {
            if (!occupied[t] || std::find(finished_now.begin(), finished_now.end(), t) != finished_now.end())
                continue;
            const bool stopped = std::find(stop_now.begin(), stop_now.end(), t) != stop_now.end();
            if (stopped || (sth[t].reason == REASON_NONE && sth[t].active && sth[t].hi_rr <= stop2[t])) {
                cudaMemsetAsync(&st[t].active, 0, sizeof(int), s);
                finished_now.push_back(t);
            }
        }
        e = pull();
    }
    return e;
}

std::vector<int> BatchSession::take_finished()
{
    std::vector<int> out;
    out.swap(finished_now);
    return out;
}

void BatchSession::info_of(int t, hisq_solve_info *info) const
{
    *info = hisq_solve_info{};
    info->iters = sth[t].k;
    info->matvecs = sth[t].k;
    info->matvecs_hi = mv_hi[t];
    info->reliable_updates = ru[t];
    info->true_residual = bb[t] > 0 ? std::sqrt(sth[t].hi_rr / bb[t]) : 0.0;
}

void BatchSession::release(int t)
{
    occupied[t] = 0;
    cudaMemsetAsync(&st[t].active, 0, sizeof(int), s);
}


hisq_status run_bcg(hisq_ctx *c, hisq_gauge *g, const BCGConfig &cfg, const double *b64, double *x64, bool x_zero,
                    hisq_solve_info *infos, cudaStream_t s)
{
    if (cfg.nrhs < 1 || cfg.nrhs > kMaxRHS) return fail(c, HISQ_EINVAL, "nrhs must be in 1..%d", kMaxRHS);
    if (cfg.sloppy.compute != HISQ_COMPUTE_F32 || cfg.sloppy.gauge == G_SE15 ||
        !(cfg.sloppy.spinor == S_F32 || cfg.sloppy.spinor == S_HALF || cfg.sloppy.spinor == S_INT20))
        return fail(c, HISQ_EINVAL, "batched solves support the FP32, half and 20-bit sloppy triplets");
    if (cfg.sloppy.long_recon != 12 && cfg.sloppy.long_recon != 18)
        return fail(c, HISQ_EINVAL, "batched solves support 18- and 12-real long links");
    BatchSession bs(c, g, cfg, s);
    hisq_status e = bs.setup();
    if (e) return e;
    const size_t f64 = (size_t)6 * g->geom.vh;
    for (int t = 0; t < cfg.nrhs; t++) {
        e = bs.load(t, b64 + t * f64, x_zero ? nullptr : x64 + t * f64, cfg.diag[t], cfg.tol[t]);
        if (e) return e;
    }
    int remaining = cfg.nrhs;
    hisq_status worst = HISQ_OK;
    auto harvest = [&]() {
        for (int t : bs.take_finished()) {
            cudaMemcpyAsync(x64 + t * f64, bs.x_of(t), (size_t)48 * g->geom.vh, cudaMemcpyDeviceToDevice, s);
            bs.info_of(t, &infos[t]);
            if (bs.status[t] != HISQ_OK && worst == HISQ_OK) worst = (hisq_status)bs.status[t];
            bs.release(t);
            remaining--;
        }
    };
    harvest();
    while (remaining > 0) {
        e = bs.step();
        if (e) return e;
        harvest();
    }
    cudaStreamSynchronize(s);
    return worst;
}

}  // namespace hisq
