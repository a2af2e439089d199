// context.cu -- contexts, gauge loading, the stencil and codec entry points of
// the C ABI (include/hisq.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "internal.h"

using namespace hisq;

namespace hisq {

Geom make_geom(const int dims[4], int antiperiodic_t)
{
    Geom g{};
    for (int d = 0; d < 4; d++) g.L[d] = dims[d];
    g.stride[0] = 1;
    g.stride[1] = dims[0];
    g.stride[2] = dims[0] * dims[1];
    g.stride[3] = dims[0] * dims[1] * dims[2];
    g.xh = dims[0] / 2;
    g.vh = (int)((int64_t)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    g.antiperiodic_t = antiperiodic_t;
    return g;
}

hisq_status fail(hisq_ctx *c, hisq_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lk(c->err_mu);
        c->last_error = buf;
    }
    return s;
}

hisq_status cuda_fail(hisq_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, HISQ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
thread_local const Lane *tl_lane = nullptr;
thread_local bool tl_capturing = false;
thread_local int tl_prof_tag = -1;
thread_local std::vector<Profiler::Rec> *tl_graph_rec = nullptr;
}  // namespace

void set_prof_tag(int tag) { tl_prof_tag = tag; }
void set_graph_recorder(std::vector<Profiler::Rec> *rec) { tl_graph_rec = rec; }

void set_thread_lane(const Lane *lane) { tl_lane = lane; }
const RedBuf &cur_red(hisq_ctx *c) { return tl_lane ? tl_lane->red : c->red; }
int *cur_err(hisq_ctx *c) { return tl_lane ? tl_lane->err : c->err_flag; }
void set_thread_capturing(bool on) { tl_capturing = on; }
bool thread_capturing() { return tl_capturing; }

hisq_status ctx_alloc(hisq_ctx *c, size_t bytes, void **p)
{
    *p = nullptr;
    if (bytes == 0) return HISQ_OK;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    if (c->used + bytes > c->budget)
        return fail(c, HISQ_ENOMEM, "device budget exceeded: %zu + %zu > %zu bytes", c->used, bytes, c->budget);
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return fail(c, HISQ_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    return HISQ_OK;
}

void ctx_free(hisq_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    cudaFree(p);
    c->used -= std::min(c->used, bytes);
}

cudaStream_t pick_stream(hisq_ctx *c, void *s) { return s ? (cudaStream_t)s : c->stream; }

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

LaunchScope::LaunchScope(hisq_ctx *c_, cudaStream_t s_, int kind_, double bytes_, int nl_)
    : c(c_), s(s_), kind(kind_), bytes(bytes_), tag(tl_prof_tag), nl(nl_)
{
    const bool sel = c->prof.on && ((c->prof.mask >> kind) & 1u);
    if (thread_capturing()) {  // launches are counted when the graph is replayed
        if (!sel || !tl_graph_rec) return;
        in_graph = true;
    } else {
        c->launches += nl;
        if (!sel || stream_capturing(s)) return;
    }
    std::lock_guard<std::mutex> lk(c->prof_mu);
    auto take = [&]() {
        cudaEvent_t e;
        if (!c->prof.pool.empty()) {
            e = c->prof.pool.back();
            c->prof.pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    };
    a = take();
    b = take();
    if (in_graph)
        cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    else
        cudaEventRecord(a, s);
}

LaunchScope::~LaunchScope()
{
    if (!a) return;
    if (in_graph) {
        cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
        tl_graph_rec->push_back({a, b, kind, bytes, tag, nl});
        return;
    }
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(c->prof_mu);
    c->prof.pending.push_back({a, b, kind, bytes, tag, nl});
    if (c->prof.pending.size() > 4096) prof_flush_locked(c);
}

cudaError_t graph_kernel_nodes(cudaGraph_t g, size_t *n)
{
    *n = 0;
    size_t total = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &total);
    if (e != cudaSuccess || total == 0) return e;
    std::vector<cudaGraphNode_t> nodes(total);
    e = cudaGraphGetNodes(g, nodes.data(), &total);
    if (e != cudaSuccess) return e;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) *n += 1;
    }
    return cudaSuccess;
}

void prof_settle(hisq_ctx *c, int n_exec)
{
    std::lock_guard<std::mutex> lk(c->prof_mu);
    auto &p = c->prof.pending;
    size_t w = 0;
    for (size_t i = 0; i < p.size(); i++) {
        if (p[i].tag >= n_exec) {
            c->prof.pool.push_back(p[i].a);
            c->prof.pool.push_back(p[i].b);
            continue;
        }
        p[i].tag = -1;
        p[w++] = p[i];
    }
    p.resize(w);
}

void prof_graph_account(hisq_ctx *c, const std::vector<Profiler::Rec> &recs, int n_exec)
{
    std::lock_guard<std::mutex> lk(c->prof_mu);
    for (const auto &r : recs) {
        if (r.tag >= n_exec) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof.ms[r.kind] += ms;
            c->prof.launches[r.kind] += r.nl;
            c->prof.bytes[r.kind] += r.bytes;
        }
    }
}

void prof_graph_release(hisq_ctx *c, std::vector<Profiler::Rec> &recs)
{
    std::lock_guard<std::mutex> lk(c->prof_mu);
    for (const auto &r : recs) {
        c->prof.pool.push_back(r.a);
        c->prof.pool.push_back(r.b);
    }
    recs.clear();
}

void prof_flush(hisq_ctx *c)
{
    std::lock_guard<std::mutex> lk(c->prof_mu);
    prof_flush_locked(c);
}

void prof_flush_locked(hisq_ctx *c)
{
    for (auto &r : c->prof.pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof.ms[r.kind] += ms;
            c->prof.launches[r.kind] += r.nl;
            c->prof.bytes[r.kind] += r.bytes;
        }
        c->prof.pool.push_back(r.a);
        c->prof.pool.push_back(r.b);
    }
    c->prof.pending.clear();
}

hisq_status check_prec(hisq_ctx *c, const hisq_prec &p)
{
    const bool ok = (p.gauge == G_F64 && p.spinor == S_F64 && p.compute == HISQ_COMPUTE_F64) ||
                    (p.gauge == G_F32 && p.spinor == S_F32 && p.compute == HISQ_COMPUTE_F32) ||
                    (p.gauge == G_FIX16 && p.spinor == S_HALF && p.compute == HISQ_COMPUTE_F32) ||
                    (p.gauge == G_FIX16 && p.spinor == S_INT20 && p.compute == HISQ_COMPUTE_F32) ||
                    (p.gauge == G_FIX16 && p.spinor == S_INT14 && p.compute == HISQ_COMPUTE_F32) ||
                    (p.gauge == G_SE15 && p.spinor == S_INT20 && p.compute == HISQ_COMPUTE_F32) ||
                    (p.gauge == G_FIX32 && p.spinor == S_INT30);
    if (!ok)
        return fail(c, HISQ_EINVAL, "unsupported precision triplet gauge=%d spinor=%d compute=%d", p.gauge,
                    p.spinor, p.compute);
    if (p.fat_recon != 18) return fail(c, HISQ_EINVAL, "fat links must be stored with 18 reals");
    if (p.long_recon != 18 && p.long_recon != 12 && p.long_recon != 13 && p.long_recon != 8)
        return fail(c, HISQ_EINVAL, "long_recon must be 18, 13, 12 or 8");
    if ((p.long_recon == 13 || p.long_recon == 8) &&
        !(p.compute == HISQ_COMPUTE_F32 && (p.gauge == G_FIX16 || p.gauge == G_F32)))
        return fail(c, HISQ_EINVAL, "%d-real long links need an FP32-compute triplet with 16-bit or FP32 links",
                    p.long_recon);
    return HISQ_OK;
}

static hisq_status get_copy(hisq_ctx *c, hisq_gauge *g, bool lng, int gf, int recon, const char **out)
{
    auto &copies = lng ? g->lng_copies : g->fat_copies;
    for (auto &lc : copies)
        if (lc.gf == gf && lc.recon == recon) {
            *out = lc.ptr;
            return HISQ_OK;
        }
    if (recon == 12 && !(lng ? g->lng_r12_ok : g->fat_r12_ok))
        return fail(c, HISQ_EINVAL, "%s links are not a sign times SU(3): 12-real compression refused",
                    lng ? "long" : "fat");
    if (recon == 13 && !(lng && g->lng_u3_ok))
        return fail(c, HISQ_EINVAL, "%s links are not unitary: 13-real compression refused", lng ? "long" : "fat");
    if (recon == 8 && !(lng && g->lng_r12_ok))
        return fail(c, HISQ_EINVAL, "%s links are not a sign times SU(3): 8-real compression refused",
                    lng ? "long" : "fat");
    LinkCopy lc;
    lc.gf = gf;
    lc.recon = recon;
    lc.bytes = link_field_bytes(gf, recon, g->geom.vh);
    hisq_status st = ctx_alloc(c, lc.bytes, (void **)&lc.ptr);
    if (st) return st;
    const double gmax = lng ? g->lng_max : g->fat_max;
    const double qmax = gf == G_FIX16 ? 32767.0 : 2147483647.0;
    const double inv = gmax > 0.0 ? qmax / gmax : 0.0;
    {
        LaunchScope ls(c, c->stream, PROF_CONVERT, 0.0);
        launch_quantise_links(g->geom, gf, recon, lng ? g->lng64 : g->fat64, inv, lc.ptr, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        ctx_free(c, lc.ptr, lc.bytes);
        return cuda_fail(c, e, "quantise links");
    }
    if (recon == 8) {
        // the 8-real rebuild divides by N = 1 - |V00|^2 and takes sqrt(N - |V10|^2), so single links near
        // those points come back far off; refuse a field whose rebuilt links are off by more than 4 storage
        // steps per real in the root mean square (or not finite: N = 0, e.g. a free field)
        const double step = gf == G_FIX16 ? 0x1p-15 : gf == G_FIX32 ? 0x1p-31 : gf == G_F32 ? 0x1p-24 : 0x1p-52;
        const double el = (gf == G_FIX16 || gf == G_FIX32) ? gmax / qmax : 1.0;
        const double an = (gf == G_FIX16 || gf == G_FIX32) ? 1.0 / qmax : 1.0;
        double *dev = cur_red(c).result, err[2] = {0.0, 0.0};
        e = cudaMemsetAsync(dev, 0, 2 * sizeof(double), c->stream);
        if (e == cudaSuccess) {
            launch_r8_check(g->geom, gf, g->lng64, lc.ptr, el, an, dev, c->stream);
            e = cudaMemcpyAsync(err, dev, sizeof err, cudaMemcpyDeviceToHost, c->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            ctx_free(c, lc.ptr, lc.bytes);
            return cuda_fail(c, e, "8-real link check");
        }
        const double rms = std::sqrt(err[1] / (18.0 * 8.0 * (double)g->geom.vh));
        const double bound = 4.0 * step * std::max(gmax, 1.0);
        if (!(rms <= bound)) {
            ctx_free(c, lc.ptr, lc.bytes);
            return fail(c, HISQ_EINVAL,
                        "8-real long links come back %.2e off in the root mean square (bound %.2e, largest %.2e): "
                        "too many links where the 8-real rebuild is ill-conditioned; use 12 or 13 reals",
                        rms, bound, err[0]);
        }
    }
    copies.push_back(lc);
    *out = lc.ptr;
    return HISQ_OK;
}

hisq_status gauge_view_existing(hisq_ctx *c, const hisq_gauge *g, const hisq_prec &p, GaugeView *v)
{
    hisq_status st = check_prec(c, p);
    if (st) return st;
    v->fat = v->lng = nullptr;
    // another thread may be appending a copy (gauge_view_for): look up under its lock
    std::lock_guard<std::mutex> lk(g->copy_mu);
    for (auto &lc : g->fat_copies)
        if (lc.gf == p.gauge && lc.recon == p.fat_recon) v->fat = lc.ptr;
    for (auto &lc : g->lng_copies)
        if (lc.gf == p.gauge && lc.recon == p.long_recon) v->lng = lc.ptr;
    if (!v->fat || !v->lng)
        return fail(c, HISQ_EINVAL,
                    "the gauge field has no stored copy for this precision yet (any hisq_dslash or solver call "
                    "with it builds one)");
    const double qmax = p.gauge == G_FIX16 ? 32767.0 : 2147483647.0;
    v->fat_scale_d = g->fat_max / qmax;
    v->lng_scale_d = g->lng_max / qmax;
    v->fat_scale_f = (float)v->fat_scale_d;
    v->lng_scale_f = (float)v->lng_scale_d;
    set_row2_rescale(v);
    return HISQ_OK;
}

hisq_status gauge_view_for(hisq_ctx *c, hisq_gauge *g, const hisq_prec &p, GaugeView *v)
{
    hisq_status st = check_prec(c, p);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g->copy_mu);
    st = get_copy(c, g, false, p.gauge, p.fat_recon, &v->fat);
    if (st) return st;
    st = get_copy(c, g, true, p.gauge, p.long_recon, &v->lng);
    if (st) return st;
    const double qmax = p.gauge == G_FIX16 ? 32767.0 : 2147483647.0;
    v->fat_scale_d = g->fat_max / qmax;
    v->lng_scale_d = g->lng_max / qmax;
    v->fat_scale_f = (float)v->fat_scale_d;
    v->lng_scale_f = (float)v->lng_scale_d;
    set_row2_rescale(v);
    return HISQ_OK;
}

}  // namespace hisq

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

hisq_status hisq_create(int device, size_t hbm_budget, hisq_ctx **out)
{
    if (!out) return HISQ_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        (void)cudaGetLastError();
        return HISQ_EINVAL;
    }
    hisq_ctx *c = new (std::nothrow) hisq_ctx();
    if (!c) return HISQ_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete c;
        return HISQ_ECUDA;
    }
    c->budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
    void *p = nullptr;
    const size_t red_bytes = sizeof(double) * ((size_t)kMaxRedBlocks * kMaxRed + kMaxRed) + 256 +
                             sizeof(unsigned) * kSyncWords;
    if (ctx_alloc(c, red_bytes, &p) != HISQ_OK) {
        hisq_destroy(c);
        return HISQ_ENOMEM;
    }
    c->red.partials = (double *)p;
    c->red.result = c->red.partials + (size_t)kMaxRedBlocks * kMaxRed;
    c->red.counter = (unsigned *)(c->red.result + kMaxRed);
    c->err_flag = (int *)(c->red.counter + 16);
    c->red.sync = c->red.counter + 64;  // 256 bytes past the counter
    cudaMemset(p, 0, red_bytes);
    cudaDeviceSynchronize();
    *out = c;
    return HISQ_OK;
}

void hisq_destroy(hisq_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    server_shutdown(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    prof_flush(c);
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    for (auto *g : c->gauges) {
        for (auto &lc : g->fat_copies) cudaFree(lc.ptr);
        for (auto &lc : g->lng_copies) cudaFree(lc.ptr);
        cudaFree(g->fat64);
        cudaFree(g->lng64);
        delete g;
    }
    if (c->scratch) cudaFree(c->scratch);
    if (c->red.partials) cudaFree(c->red.partials);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *hisq_last_error(hisq_ctx *c)
{
    if (!c) return "null context";
    return c->last_error.c_str();
}

size_t hisq_mem_used(hisq_ctx *c) { return c ? c->used : 0; }

hisq_status hisq_load_gauge(hisq_ctx *c, const int dims[4], const double *fat, const double *lng, unsigned flags,
                            hisq_gauge **out)
{
    if (!c || !dims || !fat || !lng || !out) return fail(c, HISQ_EINVAL, "null argument");
    *out = nullptr;
    for (int d = 0; d < 4; d++)
        if (dims[d] < 2 || dims[d] % 2)
            return fail(c, HISQ_EINVAL, "lattice extent %d of dimension %d must be even and >= 2", dims[d], d);
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    if (V / 2 > (int64_t)1 << 29) return fail(c, HISQ_EINVAL, "lattice too large");
    cudaSetDevice(c->device);
    hisq_gauge *g = new (std::nothrow) hisq_gauge();
    if (!g) return HISQ_ENOMEM;
    g->geom = make_geom(dims, (flags & HISQ_GAUGE_ANTIPERIODIC_T) ? 1 : 0);
    std::memcpy(g->dims, dims, sizeof g->dims);
    g->flags = flags;
    const size_t bytes = sizeof(double) * 18 * 4 * (size_t)V;
    hisq_status st = ctx_alloc(c, bytes, (void **)&g->fat64);
    if (!st) st = ctx_alloc(c, bytes, (void **)&g->lng64);
    if (st) {
        ctx_free(c, g->fat64, bytes);
        delete g;
        return st;
    }
    const cudaMemcpyKind kind = (flags & HISQ_GAUGE_ON_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(g->fat64, fat, bytes, kind, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->lng64, lng, bytes, kind, c->stream);
    double *scal = cur_red(c).result;  // 5 scratch doubles: fat max, long max, fat dev, long dev, long U(3) dev
    if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, 5 * sizeof(double), c->stream);
    if (e == cudaSuccess) {
        LaunchScope ls(c, c->stream, PROF_CONVERT, 0.0);
        launch_absmax(18 * 4 * V, g->fat64, scal + 0, c->stream);
        launch_absmax(18 * 4 * V, g->lng64, scal + 1, c->stream);
        launch_r12_check(g->geom, g->fat64, 1, scal + 2, c->stream);
        launch_r12_check(g->geom, g->lng64, 3, scal + 3, c->stream);
        launch_u3_check(g->geom, g->lng64, scal + 4, c->stream);
    }
    double h[5] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, scal, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        ctx_free(c, g->fat64, bytes);
        ctx_free(c, g->lng64, bytes);
        delete g;
        return cuda_fail(c, e, "gauge upload");
    }
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
        ctx_free(c, g->fat64, bytes);
        ctx_free(c, g->lng64, bytes);
        delete g;
        return fail(c, HISQ_EINVAL, "gauge field has non-finite entries");
    }
    g->fat_max = h[0];
    g->lng_max = h[1];
    g->fat_r12_ok = std::isfinite(h[2]) && h[2] <= 1e-6;
    g->lng_r12_ok = std::isfinite(h[3]) && h[3] <= 1e-6;
    g->lng_u3_ok = std::isfinite(h[4]) && h[4] <= 1e-6;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->gauges.push_back(g);
    }
    *out = g;
    return HISQ_OK;
}

void hisq_free_gauge(hisq_ctx *c, hisq_gauge *g)
{
    if (!c || !g) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->gauges.erase(std::remove(c->gauges.begin(), c->gauges.end(), g), c->gauges.end());
    }
    for (auto &lc : g->fat_copies) ctx_free(c, lc.ptr, lc.bytes);
    for (auto &lc : g->lng_copies) ctx_free(c, lc.ptr, lc.bytes);
    const size_t bytes = sizeof(double) * 18 * 4 * (size_t)g->geom.vh * 2;
    ctx_free(c, g->fat64, bytes);
    ctx_free(c, g->lng64, bytes);
    delete g;
}

double hisq_gauge_scale(const hisq_gauge *g, int which)
{
    if (!g) return 0.0;
    return which ? g->lng_max : g->fat_max;
}

size_t hisq_spinor_bytes(int sfmt, int64_t n)
{
    if (sfmt < 0 || sfmt > 5 || n < 0) return 0;
    return spinor_field_bytes(sfmt, n);
}

static hisq_status grow_scratch(hisq_ctx *c, size_t bytes)
{
    if (c->scratch_bytes >= bytes) return HISQ_OK;
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        ctx_free(c, c->scratch, c->scratch_bytes);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    hisq_status st = ctx_alloc(c, bytes, (void **)&c->scratch);
    if (!st) c->scratch_bytes = bytes;
    return st;
}

hisq_status hisq_spinor_pack(hisq_ctx *c, int sfmt, int64_t n, const double *in, void *packed, int64_t *n_bad,
                             void *stream)
{
    if (!c || !in || !packed || sfmt < 0 || sfmt > 5 || n < 0 || n > INT32_MAX)
        return fail(c, HISQ_EINVAL, "hisq_spinor_pack: bad argument");
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    int *bad = cur_err(c);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    {
        LaunchScope ls(c, s, PROF_CONVERT, (48.0 + spinor_site_bytes(sfmt)) * n);
        launch_pack_spinor(sfmt, n, in, (char *)packed, bad, s);
    }
    int h = 0;
    cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_spinor_pack");
    if (n_bad) *n_bad = h;
    return HISQ_OK;
}

hisq_status hisq_spinor_pack32(hisq_ctx *c, int sfmt, int64_t n, const float *in, void *packed, int64_t *n_bad,
                               void *stream)
{
    if (!c || !in || !packed || sfmt < 1 || sfmt > 5 || n < 0 || n > INT32_MAX)
        return fail(c, HISQ_EINVAL, "hisq_spinor_pack32: bad argument");
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    int *bad = cur_err(c);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    {
        LaunchScope ls(c, s, PROF_CONVERT, (24.0 + spinor_site_bytes(sfmt)) * n);
        launch_pack32_spinor(sfmt, n, in, (char *)packed, bad, s);
    }
    int h = 0;
    cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_spinor_pack32");
    if (n_bad) *n_bad = h;
    return HISQ_OK;
}

hisq_status hisq_spinor_pack_pair_int30(hisq_ctx *c, int64_t n, const float *in, void *packed, int64_t *n_bad,
                                        void *stream)
{
    if (!c || !in || !packed || n < 0 || n > INT32_MAX)
        return fail(c, HISQ_EINVAL, "hisq_spinor_pack_pair_int30: bad argument");
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    int *bad = cur_err(c);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    {
        LaunchScope ls(c, s, PROF_CONVERT, (48.0 + spinor_site_bytes(S_INT30)) * n);
        launch_pack_pair_int30(n, in, (char *)packed, bad, s);
    }
    int h = 0;
    cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_spinor_pack_pair_int30");
    if (n_bad) *n_bad = h;
    return HISQ_OK;
}

hisq_status hisq_spinor_unpack(hisq_ctx *c, int sfmt, int compute, int64_t n, const void *packed, double *out,
                               void *stream)
{
    if (!c || !out || !packed || sfmt < 0 || sfmt > 5 || n < 0 || n > INT32_MAX)
        return fail(c, HISQ_EINVAL, "hisq_spinor_unpack: bad argument");
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    {
        LaunchScope ls(c, s, PROF_CONVERT, (48.0 + spinor_site_bytes(sfmt)) * n);
        launch_unpack_spinor(sfmt, compute, n, (const char *)packed, out, s);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_spinor_unpack");
    return HISQ_OK;
}

hisq_status hisq_dslash(hisq_ctx *c, const hisq_gauge *gc, hisq_prec prec, int out_parity, double a,
                        const double *xpay_in, const double *in, double *out, int on_device, void *stream)
{
    if (!c || !gc || !in || !out) return fail(c, HISQ_EINVAL, "hisq_dslash: null argument");
    if (out_parity < 0 || out_parity > 2) return fail(c, HISQ_EINVAL, "out_parity must be 0, 1 or 2");
    const bool xpay = a != 0.0;
    if (xpay && !xpay_in) return fail(c, HISQ_EINVAL, "xpay_in is required when a != 0");
    cudaSetDevice(c->device);
    hisq_gauge *g = const_cast<hisq_gauge *>(gc);
    GaugeView gv{};
    hisq_status st = gauge_view_for(c, g, prec, &gv);
    if (st) return st;
    cudaStream_t s = pick_stream(c, stream);
    const int64_t vh = g->geom.vh;
    const int nhalf = out_parity == 2 ? 2 : 1;
    const int64_t n = vh * nhalf;  // sites in the caller's arrays
    const size_t b64 = (size_t)48 * n;
    const size_t bs = spinor_field_bytes(prec.spinor, vh);
    const size_t need = 3 * b64 + 3 * bs * nhalf + 256;
    st = grow_scratch(c, need);
    if (st) return st;
    char *sc = c->scratch;
    double *in64 = (double *)sc, *out64 = (double *)(sc + b64), *y64 = (double *)(sc + 2 * b64);
    char *in_s = sc + 3 * b64, *out_s = in_s + bs * nhalf, *y_s = out_s + bs * nhalf;
    const double *din = in, *dy = xpay_in;
    double *dout = on_device ? out : out64;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = cudaMemcpyAsync(in64, in, b64, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && xpay) e = cudaMemcpyAsync(y64, xpay_in, b64, cudaMemcpyHostToDevice, s);
        din = in64;
        dy = y64;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash upload");
    cudaMemsetAsync(cur_err(c), 0, sizeof(int), s);
    // the caller's full-lattice array is [even half][odd half]: pack per half
    for (int h = 0; h < nhalf; h++) {
        LaunchScope ls(c, s, PROF_CONVERT, (48.0 + spinor_site_bytes(prec.spinor)) * vh);
        launch_pack_spinor(prec.spinor, vh, din + h * vh * 6, in_s + h * bs, cur_err(c), s);
        if (xpay) launch_pack_spinor(prec.spinor, vh, dy + h * vh * 6, y_s + h * bs, cur_err(c), s);
    }
    int bad_in = 0;
    cudaMemcpyAsync(&bad_in, cur_err(c), sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash pack");
    if (bad_in) return fail(c, HISQ_EINVAL, "non-finite input spinor");
    {
        DslashArgs td{};
        td.g = g->geom;
        td.gv = gv;
        td.err = cur_err(c);
        td.red = cur_red(c);
        td.out_parity = 0;
        td.in = in_s;
        td.out = out_s;
        td.sign = 1;
        if (!stream_capturing(s)) tune_dslash(prec.gauge, prec.spinor, prec.compute, prec.long_recon, td, s);
    }
    const double link_b = 8.0 * link_bytes(prec.gauge, prec.fat_recon) + 8.0 * link_bytes(prec.gauge, prec.long_recon);
    const double site_b = spinor_site_bytes(prec.spinor);
    for (int h = 0; h < nhalf; h++) {
        const int po = out_parity == 2 ? h : out_parity;
        // half-field index of a parity inside the caller's array: full lattice
        // stores even at 0 and odd at 1; a single-parity call uses index 0
        const int oi = out_parity == 2 ? po : 0, ii = out_parity == 2 ? 1 - po : 0;
        DslashArgs da{};
        da.g = g->geom;
        da.gv = gv;
        da.out_parity = po;
        da.in = in_s + ii * bs;
        da.out = out_s + oi * bs;
        da.y = xpay ? y_s + oi * bs : nullptr;
        da.a = a;
        da.sign = xpay ? -1 : 1;
        da.xpay = xpay ? 1 : 0;
        da.active = nullptr;
        da.err = cur_err(c);
        da.red = cur_red(c);
        da.fin = FIN_NONE;
        da.st = nullptr;
        LaunchScope ls(c, s, PROF_STENCIL, (link_b + (xpay ? 3 : 2) * site_b) * vh);
        if (!launch_dslash(prec.gauge, prec.spinor, prec.compute, prec.long_recon, false, da, s))
            return fail(c, HISQ_EINVAL, "no stencil kernel for this triplet");
    }
    for (int h = 0; h < nhalf; h++) {
        LaunchScope ls(c, s, PROF_CONVERT, (48.0 + site_b) * vh);
        launch_unpack_spinor(prec.spinor, prec.compute, vh, out_s + h * bs, dout + h * vh * 6, s);
    }
    if (!on_device) e = cudaMemcpyAsync(out, out64, b64, cudaMemcpyDeviceToHost, s);
    // the stencil flags output sites it could not store
    int bad_out = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_out, cur_err(c), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "hisq_dslash");
    if (bad_out)
        return fail(c, HISQ_ERANGE,
                    "hisq_dslash: output sites not storable in the spinor format (overflow or beyond its exponent "
                    "range)");
    return HISQ_OK;
}

void hisq_profile_enable(hisq_ctx *c, int on)
{
    if (!c) return;
    if (!on) prof_flush(c);
    c->prof.on = on != 0;
}

void hisq_profile_select(hisq_ctx *c, unsigned mask)
{
    if (!c) return;
    std::lock_guard<std::mutex> lk(c->prof_mu);
    c->prof.mask = mask;
}

hisq_status hisq_profile_sample(hisq_ctx *c, int every)
{
    if (!c) return HISQ_EINVAL;
    if (every < 1) return fail(c, HISQ_EINVAL, "profile sample period must be >= 1 (got %d)", every);
    std::lock_guard<std::mutex> lk(c->prof_mu);
    c->prof.every = every;
    return HISQ_OK;
}

void hisq_profile_reset(hisq_ctx *c)
{
    if (!c) return;
    prof_flush(c);
    for (int k = 0; k < PROF_NKIND; k++) {
        c->prof.ms[k] = 0;
        c->prof.launches[k] = 0;
        c->prof.bytes[k] = 0;
    }
}

hisq_status hisq_profile_read(hisq_ctx *c, int kind, hisq_kernel_stats *out)
{
    if (!c || !out || kind < 0 || kind >= PROF_NKIND) return fail(c, HISQ_EINVAL, "hisq_profile_read: bad argument");
    prof_flush(c);
    out->ms = c->prof.ms[kind];
    out->launches = c->prof.launches[kind];
    out->bytes = c->prof.bytes[kind];
    return HISQ_OK;
}

int64_t hisq_launch_count(hisq_ctx *c) { return c ? c->launches.load() : 0; }

}  // extern "C"
