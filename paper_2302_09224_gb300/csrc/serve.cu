// serve.cu -- the request loop behind hisq_submit / hisq_poll / hisq_wait.
//
// Worker threads (each with its own CUDA stream and reduction buffers, so
// their solves overlap on the device) take requests in arrival order.  CG
// requests on the same resident gauge field with the same sloppy triplet are
// solved together in a batch session: at every block boundary the slots of
// finished systems are harvested and refilled from the queue (continuous
// batching), so a request that arrives while others iterate joins them as
// soon as a slot frees up.  Sessions are admitted only while the context's
// HBM budget allows their buffers; otherwise their requests wait.  A
// multi-shift request runs its multi-shift stage (all shifts in one fused
// update per iteration) on a worker; the refinement CG of each shift that has
// not reached its target then enters the queue as an internal CG request
// (its shifted diagonal, its target, the stage's solution as initial guess),
// so the refinements join the batch sessions of their sloppy triplet beside
// ordinary CG requests; the request is done when its last refinement is.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <numeric>
#include <memory>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "bcg.h"
#include "cg.h"
#include "internal.h"

namespace hisq {

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct MSJob;

struct Req {
    uint64_t ticket = 0;
    hisq_request r{};
    std::vector<double> sigma, tols;
    double t_submit = 0, t_done = 0;
    bool done = false;
    hisq_status status = HISQ_OK;
    hisq_solve_info info{};
    // a refinement of one shift of a multi-shift request: planar FP64 right-hand
    // side and initial guess on the device, the shifted diagonal 4m^2 + sigma
    std::shared_ptr<MSJob> job;
    int shift = -1;
    const double *b_planar = nullptr, *x0_planar = nullptr;
    double diag = 0;
};

// A multi-shift request between its stage and its last refinement: the device
// fields the refinements read (freed with the job) and the merged report.
struct MSJob {
    std::shared_ptr<Req> parent;
    std::unique_ptr<Workspace> ws;
    double *b64 = nullptr;
    std::vector<double *> x64;
    std::vector<int> ord;  // sorted shift -> the caller's index
    int remaining = 0;
    hisq_solve_info info{};  // per shift in sorted order until the end
    hisq_status worst = HISQ_OK;
};

using Key = std::tuple<const hisq_gauge *, int, int, int, int, int, int>;

Key key_of(const hisq_request &r)
{
    return Key(r.gauge, r.sloppy.gauge, r.sloppy.spinor, r.sloppy.compute, r.sloppy.long_recon, r.maxiter, 0);
}

bool batchable(const hisq_request &r)
{
    return r.kind == HISQ_REQ_CG && r.sloppy.compute == HISQ_COMPUTE_F32 && r.sloppy.gauge != G_SE15 &&
           (r.sloppy.spinor == S_F32 || r.sloppy.spinor == S_HALF || r.sloppy.spinor == S_INT20) &&
           r.sloppy.fat_recon == 18 && (r.sloppy.long_recon == 12 || r.sloppy.long_recon == 18);
}

}  // namespace

struct Server {
    hisq_ctx *c;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::map<uint64_t, std::shared_ptr<Req>> table;
    std::set<Key> busy;
    std::vector<std::thread> workers;
    bool stop = false;
    uint64_t next_ticket = 1;
    int running = 0;  // sessions or solves on the device
    std::vector<double> latencies;
    double t_first = 0, t_last = 0;
    int64_t completed = 0;

    explicit Server(hisq_ctx *c_) : c(c_) {}

    // one reduction lane (partials, result, counters, error flag) per worker,
    // allocated before the workers start: a worker never shares the
    // context's own lane with another thread
    static size_t lane_bytes()
    {
        return sizeof(double) * ((size_t)kMaxRedBlocks * kMaxRed + kMaxRed) + 256 + sizeof(unsigned) * kSyncWords;
    }

    // the merged report of a multi-shift request in the caller's shift order
    static void report_ms(MSJob &j, hisq_solve_info *out)
    {
        *out = j.info;
        const int ns = (int)j.ord.size();
        for (int i = 0; i < ns; i++) {
            out->shift_iters[j.ord[i]] = j.info.shift_iters[i];
            out->shift_resid_ms[j.ord[i]] = j.info.shift_resid_ms[i];
            out->shift_resid[j.ord[i]] = j.info.shift_resid[i];
            out->refine_iters[j.ord[i]] = j.info.refine_iters[i];
        }
        out->true_residual = j.info.shift_resid[0];
    }

    void finish(const std::shared_ptr<Req> &q, hisq_status st, const hisq_solve_info &info)
    {
        if (q->job) {  // a refinement: merge into its multi-shift request
            std::shared_ptr<Req> parent;
            hisq_solve_info rep{};
            hisq_status pst = HISQ_OK;
            {
                std::lock_guard<std::mutex> lk(mu);
                MSJob &j = *q->job;
                j.info.refine_iters[q->shift] = info.iters;
                j.info.shift_resid[q->shift] = info.true_residual;
                j.info.matvecs += info.matvecs;
                j.info.matvecs_hi += info.matvecs_hi;
                j.info.reliable_updates += info.reliable_updates;
                if (st != HISQ_OK && (j.worst == HISQ_OK || j.worst == HISQ_ENOTCONV)) j.worst = st;
                if (--j.remaining == 0) {
                    parent = j.parent;
                    report_ms(j, &rep);
                    pst = j.worst;
                }
            }
            q->job.reset();
            if (parent) finish(parent, pst, rep);
            return;
        }
        std::lock_guard<std::mutex> lk(mu);
        q->status = st;
        q->info = info;
        q->t_done = now_s();
        q->info.seconds = q->t_done - q->t_submit;
        q->done = true;
        latencies.push_back(q->info.seconds);
        t_last = q->t_done;
        completed++;
        cv_done.notify_all();
    }

    // take up to n pending batchable requests with key k (caller holds mu)
    std::vector<std::shared_ptr<Req>> take_matching(const Key &k, int n)
    {
        std::vector<std::shared_ptr<Req>> out;
        for (auto it = pending.begin(); it != pending.end() && (int)out.size() < n;) {
            if (batchable((*it)->r) && key_of((*it)->r) == k) {
                out.push_back(*it);
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
        return out;
    }

    void worker(void *lane_buf);
    void run_batch(const std::shared_ptr<Req> &first, cudaStream_t s);
    void run_single(const std::shared_ptr<Req> &q, cudaStream_t s);
};

namespace {

constexpr int kWorkers = 4;
constexpr int kBatchSlots = 8;
constexpr size_t kQueueCap = 4096;

}  // namespace

void Server::run_single(const std::shared_ptr<Req> &q, cudaStream_t s)
{
    hisq_solver_params p;
    hisq_default_params(&p);
    p.mass = q->r.mass;
    p.tol = q->r.tol;
    p.maxiter = q->r.maxiter;
    p.sloppy = q->r.sloppy;
    p.refine = q->r.refine;
    p.on_device = q->r.on_device;
    p.stream = s;
    hisq_solve_info info{};
    hisq_gauge *g = const_cast<hisq_gauge *>(q->r.gauge);
    const int64_t vh = g->geom.vh;
    if (q->job) {  // a refinement whose triplet has no batch session: the single-system CG from its guess
        CGConfig cfg = config_from(&p, q->diag - 4.0 * p.mass * p.mass);
        Workspace ws(c, s);
        double *x64 = nullptr;
        hisq_status st = ws.alloc((size_t)48 * vh, (void **)&x64);
        if (!st) {
            cudaMemcpyAsync(x64, q->x0_planar, (size_t)48 * vh, cudaMemcpyDeviceToDevice, s);
            st = run_cg(c, g, cfg, q->b_planar, x64, false, &info, s);
            if (st == HISQ_OK || st == HISQ_ENOTCONV || st == HISQ_EBREAKDOWN) {
                const hisq_status e = from_planar(c, ws, x64, vh, q->r.x, q->r.on_device, s);
                if (e) st = e;
            }
        }
        finish(q, st, info);
        return;
    }
    if (q->r.kind != HISQ_REQ_MULTISHIFT) {
        finish(q, hisq_cg(c, q->r.gauge, &p, q->r.b, q->r.x, &info), info);
        return;
    }
    // multi-shift: the stage here, then one refinement request per shift that needs one
    const int ns = q->r.nshift;
    auto job = std::make_shared<MSJob>();
    job->parent = q;
    job->ws = std::make_unique<Workspace>(c, nullptr);
    job->ord.resize(ns);
    std::iota(job->ord.begin(), job->ord.end(), 0);
    std::stable_sort(job->ord.begin(), job->ord.end(), [&](int a, int b) { return q->sigma[a] < q->sigma[b]; });
    std::vector<double> ss(ns), tt(ns);
    for (int i = 0; i < ns; i++) {
        ss[i] = q->sigma[job->ord[i]];
        tt[i] = q->tols[job->ord[i]];
    }
    hisq_status st = job->ws->alloc((size_t)48 * vh, (void **)&job->b64);
    job->x64.assign(ns, nullptr);
    for (int i = 0; i < ns && !st; i++) st = job->ws->alloc((size_t)48 * vh, (void **)&job->x64[i]);
    if (!st) st = to_planar(c, *job->ws, q->r.b, q->r.on_device, vh, job->b64, s);
    if (!st) {
        for (int i = 0; i < ns && !st; i++) {
            if (4.0 * p.mass * p.mass + ss[i] <= 0.0 || !std::isfinite(ss[i]) || !(tt[i] > 0.0))
                st = fail(c, HISQ_EINVAL, "shift %d: 4m^2 + sigma must be positive, tol > 0", i);
        }
    }
    if (!st) st = run_multishift_stage(c, g, p, ns, ss.data(), tt.data(), job->b64, job->x64.data(), &job->info, s);
    if (st != HISQ_OK && st != HISQ_ENOTCONV && st != HISQ_EBREAKDOWN) {
        hisq_solve_info none{};
        finish(q, st, none);
        return;
    }
    job->worst = st;
    const size_t f = (size_t)6 * vh;
    std::vector<std::shared_ptr<Req>> subs;
    for (int i = 0; i < ns; i++) {
        double *xi = q->r.x + job->ord[i] * f;
        if (st == HISQ_EBREAKDOWN || job->info.shift_resid[i] <= tt[i]) {  // done after the stage
            const hisq_status e = from_planar(c, *job->ws, job->x64[i], vh, xi, q->r.on_device, s);
            if (e) {
                hisq_solve_info none{};
                finish(q, e, none);
                return;
            }
            continue;
        }
        auto r = std::make_shared<Req>();
        r->r = q->r;
        r->r.kind = HISQ_REQ_CG;
        r->r.sloppy = q->r.refine;
        r->r.tol = tt[i];
        r->r.x = xi;
        r->job = job;
        r->shift = i;
        r->b_planar = job->b64;
        r->x0_planar = job->x64[i];
        r->diag = 4.0 * p.mass * p.mass + ss[i];
        r->t_submit = now_s();
        subs.push_back(r);
    }
    if (subs.empty()) {
        hisq_solve_info rep{};
        report_ms(*job, &rep);
        finish(q, st, rep);
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    job->remaining = (int)subs.size();
    for (auto it = subs.rbegin(); it != subs.rend(); ++it) pending.push_front(*it);  // ahead of new requests
    cv_work.notify_all();
}

void Server::run_batch(const std::shared_ptr<Req> &first, cudaStream_t s)
{
    hisq_gauge *g = const_cast<hisq_gauge *>(first->r.gauge);
    const int vh = g->geom.vh;
    const Key key = key_of(first->r);
    BCGConfig cfg;
    cfg.nrhs = kBatchSlots;
    cfg.sloppy = first->r.sloppy;
    cfg.maxiter = first->r.maxiter;
    std::vector<std::shared_ptr<Req>> slot(kBatchSlots);
    std::deque<std::shared_ptr<Req>> waiting{first};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &q : take_matching(key, kBatchSlots - 1)) waiting.push_back(q);
    }
    auto give_back = [&](hisq_status st) {
        hisq_solve_info none{};
        for (auto &q : waiting) finish(q, st, none);
        for (auto &q : slot)
            if (q) finish(q, st, none);
    };
    BatchSession bs(c, g, cfg, s);
    hisq_status e = bs.setup();
    // staging for one system: caller layout and the planar FP64 field
    Workspace stage(c, s);
    double *aos = nullptr, *planar = nullptr;
    if (!e) e = stage.alloc((size_t)48 * vh, (void **)&aos);
    if (!e) e = stage.alloc((size_t)48 * vh, (void **)&planar);
    if (e) {
        if (e == HISQ_ENOMEM) {
            bool alone;
            {
                std::lock_guard<std::mutex> lk(mu);
                alone = running <= 1;
                if (!alone)  // not admitted yet: requeue; running work will free memory
                    for (auto it = waiting.rbegin(); it != waiting.rend(); ++it) pending.push_front(*it);
            }
            if (!alone) {
                std::this_thread::sleep_for(std::chrono::milliseconds(5));
                return;
            }
        }
        give_back(e);  // cannot fit even with nothing else running
        return;
    }
    auto load_one = [&](int t, const std::shared_ptr<Req> &q) -> hisq_status {
        if (q->b_planar)  // a refinement: its fields are already planar on the device
            return bs.load(t, q->b_planar, q->x0_planar, q->diag, q->r.tol);
        const double *src = q->r.b;
        if (!q->r.on_device) {
            cudaMemcpyAsync(aos, q->r.b, (size_t)48 * vh, cudaMemcpyHostToDevice, s);
            src = aos;
        }
        cudaMemsetAsync(cur_err(c), 0, sizeof(int), s);
        launch_pack_spinor(S_F64, vh, src, (char *)planar, cur_err(c), s);
        c->launches += 1;
        int bad = 0;
        cudaMemcpyAsync(&bad, cur_err(c), sizeof bad, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "request upload");
        if (bad) return HISQ_EINVAL;
        return bs.load(t, planar, nullptr, 4.0 * q->r.mass * q->r.mass, q->r.tol);
    };
    auto harvest = [&]() -> hisq_status {
        for (int t : bs.take_finished()) {
            auto q = slot[t];
            if (!q) continue;
            hisq_solve_info info{};
            bs.info_of(t, &info);
            double *dst = q->r.on_device ? q->r.x : aos;
            launch_unpack_spinor(S_F64, HISQ_COMPUTE_F64, vh, (const char *)bs.x_of(t), dst, s);
            c->launches += 1;
            if (!q->r.on_device) cudaMemcpyAsync(q->r.x, aos, (size_t)48 * vh, cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "request download");
            const hisq_status st = (hisq_status)bs.status[t];
            bs.release(t);
            slot[t] = nullptr;
            finish(q, st, info);
        }
        return HISQ_OK;
    };
    while (true) {
        // refill free slots (continuous batching)
        {
            std::lock_guard<std::mutex> lk(mu);
            const int free_slots =
                (int)std::count(slot.begin(), slot.end(), nullptr) - (int)waiting.size();
            if (free_slots > 0)
                for (auto &q : take_matching(key, free_slots)) waiting.push_back(q);
        }
        for (int t = 0; t < kBatchSlots && !waiting.empty(); t++) {
            if (slot[t]) continue;
            auto q = waiting.front();
            waiting.pop_front();
            slot[t] = q;
            const hisq_status st = load_one(t, q);
            if (st != HISQ_OK) {
                slot[t] = nullptr;
                hisq_solve_info none{};
                finish(q, st, none);
            }
        }
        e = harvest();
        if (e) break;
        if (bs.active_slots() == 0 && waiting.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            bool more = false;
            for (auto &q : pending)
                if (batchable(q->r) && key_of(q->r) == key) more = true;
            if (!more) break;
            continue;
        }
        if (bs.active_slots() == 0) continue;
        e = bs.step();
        if (e) break;
        e = harvest();
        if (e) break;
    }
    if (e) give_back(e);
}

void Server::worker(void *buf)
{
    cudaSetDevice(c->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    // this thread's reduction buffer and error flag
    const size_t red_bytes = lane_bytes();
    Lane lane{};
    lane.red.partials = (double *)buf;
    lane.red.result = lane.red.partials + (size_t)kMaxRedBlocks * kMaxRed;
    lane.red.counter = (unsigned *)(lane.red.result + kMaxRed);
    lane.err = (int *)(lane.red.counter + 16);
    lane.red.sync = lane.red.counter + 64;
    set_thread_lane(&lane);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        std::shared_ptr<Req> job;
        bool batch = false;
        for (auto it = pending.begin(); it != pending.end(); ++it) {
            if (batchable((*it)->r)) {
                if (busy.count(key_of((*it)->r))) continue;  // its session will take it
                batch = true;
            }
            job = *it;
            pending.erase(it);
            break;
        }
        if (!job) {
            cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        const Key key = key_of(job->r);
        if (batch) busy.insert(key);
        running++;
        lk.unlock();
        if (batch)
            run_batch(job, s);
        else
            run_single(job, s);
        lk.lock();
        running--;
        if (batch) busy.erase(key);
        cv_work.notify_all();
    }
    lk.unlock();
    set_thread_lane(nullptr);
    cudaStreamSynchronize(s);
    ctx_free(c, buf, red_bytes);
    cudaStreamDestroy(s);
}

void server_shutdown(hisq_ctx *c)
{
    Server *sv = c->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    for (auto &t : sv->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        hisq_solve_info none{};
        for (auto &q : sv->pending) {
            q->status = HISQ_ETIMEOUT;
            q->info = none;
            q->done = true;
        }
        sv->pending.clear();
        sv->cv_done.notify_all();
    }
    delete sv;
    c->server = nullptr;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

hisq_status hisq_submit(hisq_ctx *c, const hisq_request *r, uint64_t *ticket)
{
    if (!c || !r || !ticket || !r->gauge || !r->b || !r->x) return fail(c, HISQ_EINVAL, "hisq_submit: null argument");
    if (r->kind != HISQ_REQ_CG && r->kind != HISQ_REQ_MULTISHIFT) return fail(c, HISQ_EINVAL, "unknown request kind");
    if (!std::isfinite(r->mass) || r->maxiter < 0) return fail(c, HISQ_EINVAL, "bad mass or maxiter");
    if (r->kind == HISQ_REQ_CG && !(r->tol > 0.0)) return fail(c, HISQ_EINVAL, "tol must be > 0");
    if (r->kind == HISQ_REQ_MULTISHIFT && (r->nshift < 1 || r->nshift > HISQ_MAX_SHIFTS || !r->sigma || !r->shift_tol))
        return fail(c, HISQ_EINVAL, "multi-shift requests need 1..%d shifts with targets", HISQ_MAX_SHIFTS);
    hisq_status e = check_prec(c, r->sloppy);
    if (e) return e;
    if (r->kind == HISQ_REQ_MULTISHIFT) {
        e = check_prec(c, r->refine);
        if (e) return e;
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->server) {
            // a worker per reduction lane that fits the budget (at least one)
            cudaSetDevice(c->device);
            std::vector<void *> lanes;
            for (int i = 0; i < kWorkers; i++) {
                void *buf = nullptr;
                if (ctx_alloc(c, Server::lane_bytes(), &buf) != HISQ_OK) break;
                if (cudaMemset(buf, 0, Server::lane_bytes()) != cudaSuccess) {
                    ctx_free(c, buf, Server::lane_bytes());
                    break;
                }
                lanes.push_back(buf);
            }
            if (lanes.empty()) return fail(c, HISQ_ENOMEM, "no device memory for a request worker's reduction lane");
            c->server = new Server(c);
            for (void *buf : lanes) c->server->workers.emplace_back(&Server::worker, c->server, buf);
        }
    }
    Server *sv = c->server;
    auto q = std::make_shared<Req>();
    q->r = *r;
    if (r->kind == HISQ_REQ_MULTISHIFT) {
        q->sigma.assign(r->sigma, r->sigma + r->nshift);
        q->tols.assign(r->shift_tol, r->shift_tol + r->nshift);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->pending.size() >= kQueueCap) return fail(c, HISQ_EBUSY, "request queue full");
    q->ticket = sv->next_ticket++;
    q->t_submit = now_s();
    if (sv->completed == 0 && sv->table.empty()) sv->t_first = q->t_submit;
    sv->pending.push_back(q);
    sv->table[q->ticket] = q;
    *ticket = q->ticket;
    sv->cv_work.notify_one();
    return HISQ_OK;
}

hisq_status hisq_poll(hisq_ctx *c, uint64_t ticket, int *done, hisq_solve_info *info)
{
    if (!c || !done) return fail(c, HISQ_EINVAL, "hisq_poll: null argument");
    *done = 0;
    Server *sv = c->server;
    if (!sv) return fail(c, HISQ_ENOTFOUND, "no request was submitted");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->table.find(ticket);
    if (it == sv->table.end()) return fail(c, HISQ_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done) return HISQ_OK;
    *done = 1;
    if (info) *info = it->second->info;
    const hisq_status st = it->second->status;
    sv->table.erase(it);
    return st;
}

hisq_status hisq_wait(hisq_ctx *c, uint64_t ticket, double timeout_s, hisq_solve_info *info)
{
    if (!c) return HISQ_EINVAL;
    Server *sv = c->server;
    if (!sv) return fail(c, HISQ_ENOTFOUND, "no request was submitted");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->table.find(ticket);
    if (it == sv->table.end()) return fail(c, HISQ_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto q = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (!q->done) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->done)
            return fail(c, HISQ_ETIMEOUT, "request %llu not finished within %.3f s", (unsigned long long)ticket,
                        timeout_s);
    }
    if (info) *info = q->info;
    const hisq_status st = q->status;
    sv->table.erase(ticket);
    return st;
}

hisq_status hisq_serve_stats(hisq_ctx *c, hisq_serve_stats_t *out)
{
    if (!c || !out) return fail(c, HISQ_EINVAL, "hisq_serve_stats: null argument");
    *out = hisq_serve_stats_t{};
    Server *sv = c->server;
    if (!sv) return HISQ_OK;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->completed = sv->completed;
    out->pending = (int64_t)sv->pending.size();
    if (!sv->latencies.empty()) {
        std::vector<double> l = sv->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        const double span = sv->t_last - sv->t_first;
        out->solves_per_s = span > 0 ? sv->completed / span : 0.0;
    }
    return HISQ_OK;
}

}  // extern "C"
