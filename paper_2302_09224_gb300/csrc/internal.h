// internal.h -- host/device declarations shared by the library's translation
// units (never installed; the public interface is include/hisq.h).
#pragma once

#include <cmath>

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "hisq.h"

namespace hisq {

// ---------------------------------------------------------------------------
// formats
// ---------------------------------------------------------------------------
// G_SE15: per link, 15-bit integers sharing one 8-bit exponent (2 bytes a real)
enum GaugeFmt { G_F64 = 0, G_F32 = 1, G_FIX16 = 2, G_FIX32 = 3, G_SE15 = 4 };
// S_INT14: 12 B/site, six 14-bit integers and an 8-bit exponent (a third
// shared-exponent width).  S_FF: FP32 pairs (hi, lo) per real, 48 B/site:
// internal accumulators of the FP64-class kernels only, never a storage
// format of the ABI.
enum SpinorFmt { S_F64 = 0, S_F32 = 1, S_HALF = 2, S_INT20 = 3, S_INT30 = 4, S_INT14 = 5, S_FF = 7 };

__host__ __device__ constexpr int spinor_site_bytes(int sf)
{
    return (sf == S_F64 || sf == S_FF) ? 48 : (sf == S_F32 || sf == S_INT30) ? 24 : sf == S_INT14 ? 12 : 16;
}
__host__ __device__ constexpr int spinor_n16(int sf) { return spinor_site_bytes(sf) / 16; }
__host__ __device__ constexpr int spinor_tail(int sf) { return spinor_site_bytes(sf) % 16; }

__host__ __device__ constexpr int gauge_real_bytes(int gf)
{
    return gf == G_F64 ? 8 : (gf == G_FIX16 || gf == G_SE15) ? 2 : 4;
}
// Reals of a link kept in its row planes: 18, 12, and 12 for the 13-real
// format, whose 13th real (the phase of det U) lives in a plane of its own.
__host__ __device__ constexpr int link_rows_reals(int recon) { return recon == 13 ? 12 : recon; }
__host__ __device__ constexpr int link_bytes(int gf, int recon) { return gauge_real_bytes(gf) * recon; }
__host__ __device__ constexpr int link_n16(int gf, int recon) { return gauge_real_bytes(gf) * link_rows_reals(recon) / 16; }
__host__ __device__ constexpr int link_tail(int gf, int recon) { return gauge_real_bytes(gf) * link_rows_reals(recon) % 16; }

// Bytes of a half-lattice field of n sites in the planar layout: 16-B planes
// [plane][site], then the tail plane [site] (all planes of one field are
// contiguous and start 16-B aligned).
inline size_t spinor_field_bytes(int sf, int64_t n) { return (size_t)spinor_site_bytes(sf) * (size_t)n; }

// Bytes of one stored link field: [plane][parity][mu][Vh] chunks (the
// 13-real format's phase plane follows the tail plane).
inline size_t link_field_bytes(int gf, int recon, int64_t vh)
{
    return (size_t)link_bytes(gf, recon) * 8u * (size_t)vh;
}

// ---------------------------------------------------------------------------
// lattice geometry passed to kernels
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];        // extents x, y, z, t
    int stride[4];   // lex strides 1, Lx, Lx*Ly, Lx*Ly*Lz
    int xh;          // Lx / 2
    int vh;          // sites per parity
    int antiperiodic_t;
};

Geom make_geom(const int dims[4], int antiperiodic_t);

// ---------------------------------------------------------------------------
// deterministic two-level reductions (last block finishes)
// ---------------------------------------------------------------------------
constexpr int kMaxRed = 32;         // values reduced per launch
constexpr int kMaxRedBlocks = 1 << 16;

struct RedBuf {
    double *partials;        // kMaxRedBlocks * kMaxRed values: nr per block of a launch
    unsigned int *counter;   // zero between launches
    double *result;          // [kMaxRed] written by the last block
    unsigned int *sync;      // fused M_ee pass: [0] items handed out, [32 + t] finished chunks of
                             // slice t (kMaxFusedLt slices); zero between launches
};
constexpr int kMaxFusedLt = 4096;
// Offset (in doubles) of the partials' second half: the split CG chain's
// r_update leaves its block partials there while it reads the stencil pass's
// from the first half (see blas.cu).
constexpr size_t kSplitHalf = (size_t)kMaxRedBlocks * kMaxRed / 2;
constexpr size_t kSyncWords = 32 + kMaxFusedLt;

// Whether a reducing launch over n sites (blocks of `block` threads, gy grid
// rows, nr values per block) fits the partials buffer.
inline bool red_fits(int64_t n, int block, int nr, int gy = 1)
{
    return ((n + block - 1) / block) * gy * nr <= (int64_t)kMaxRedBlocks * kMaxRed;
}

// The single-RHS solvers' reducing launches: the stencil (blocks of 128 or
// more, 2 values), the BLAS kernels (256, 3) and BiCGStab(l)'s two-parity
// grids (256, 3, 2 rows).  Holds up to Vh = 2^27 sites.
inline bool solver_red_fits(int64_t vh) { return red_fits(vh, 128, 2) && red_fits(vh, 256, 3, 2); }

// ---------------------------------------------------------------------------
// solver scalar state kept on the device (one per solve)
// ---------------------------------------------------------------------------
constexpr int kMaxBuf = 16;

struct CGState {
    double rr;          // |r_k|^2 of the iterated residual
    double rr_prev;     // |r_{k-1}|^2
    double rr_den;      // split CG chain: |r_k|^2 as r_update read it (beta's denominator, kept
                        // apart from rr, which p_update's block 0 rewrites while its other blocks run)
    double rr_max;      // max |r|^2 since the last reliable update
    double pAp;
    double alpha;
    double beta;
    double delta2;      // delta^2 (reliable-update trigger)
    double stop2;       // (tol |b|)^2: iterated residual below it asks for a check
    double alpha_ring[kMaxBuf];
    double hi_rr;       // |r_hi|^2 of the last true residual
    double proj_re, proj_im;  // projection coefficient of p onto r_hi
    double coef_re, coef_im;  // p <- coef * r_hi + beta * p at a reliable update
    double diag;        // 4 m^2 + sigma of this system (read by the batched stencil)
    double apap;        // |A p|^2 of the last operator application
    // error-estimate reliable-update trigger (dyn = 1): drift estimate d and
    // its value after the last update, the sloppy precision eps and sqrt(eps)
    double dyn_d, dyn_d_init, dyn_eps, dyn_hat;
    double *hist;       // device [hist_len]: |r_k|^2 per iteration (null: not kept)
    int hist_len;
    int active;         // kernels of an iteration run only while 1
    int reason;         // why the iteration stopped (REASON_*)
    int k;              // iterations done
    int pr;             // Polak-Ribiere beta
    int reproject;
    int dyn;            // 1: error-estimate trigger instead of delta
};

enum { REASON_NONE = 0, REASON_RELIABLE = 1, REASON_CONVERGED = 2, REASON_BREAKDOWN = 3 };

// Multi-shift CG (Sec. 3.2): the base recurrence plus, per shift, the
// co-linearity factor zeta_i (r_i = zeta_i r) and its step sizes.
constexpr int kMaxShift = 32;

struct MSState {
    double rr, rr_prev, rr_max, pAp;
    double alpha, alpha_prev, beta, beta_prev;
    double delta2;
    double bb;                         // |b|^2
    double shift[kMaxShift];           // s_i = sigma_i - sigma_0
    double stop2[kMaxShift];           // (max(tol_i, floor) |b|)^2 on zeta_i^2 |r|^2
    double zeta[kMaxShift], zeta_prev[kMaxShift], zeta_new[kMaxShift];
    double alpha_i[kMaxShift], beta_i[kMaxShift];
    int live[kMaxShift];               // shift still updated
    int freeze_next[kMaxShift];        // freeze after this iteration's update
    int frozen_at[kMaxShift];
    int nshift;
    int active, reason, pending;
    int k;
    int pad;
};

// Finisher selected by a reducing kernel: what the last block does with the
// reduced values.
enum FinOp {
    FIN_NONE = 0,
    FIN_CG_ALPHA = 1,     // values: Re<p,Ap>, |Ap|^2            -> alpha
    FIN_CG_BETA = 2,      // values: |r_new|^2, Re<r_new, r_old> -> beta, checks
    FIN_CG_TRUE = 3,      // values: |r_hi|^2, Re/Im <r_hi, p>   -> projection, coef, beta
    FIN_STORE = 4,        // copy the sums to RedBuf::result only
    FIN_MS_ALPHA = 5,     // values: Re<p0,Ap0>                  -> alpha, zeta_i', alpha_i
    FIN_MS_BETA = 6,      // values: |r_new|^2                   -> beta, beta_i, freezing, decisions
    FIN_MS_TRUE = 7,      // values: |r_hi|^2                    -> restart after a reliable update
    FIN_MS_APPLY = 8      // no values: apply pending freezes and stop decisions
};

// ---------------------------------------------------------------------------
// kernel parameter blocks
// ---------------------------------------------------------------------------
struct GaugeView {
    const char *fat;
    const char *lng;
    float fat_scale_f, lng_scale_f;    // decode scale of fixed point (FP32 compute)
    double fat_scale_d, lng_scale_d;   // decode scale (FP64 compute)
    // 2 * lng_scale_d = lng_r2_mul * 2^-(32 + lng_r2_shift), lng_r2_mul in [2^30, 2^31): the
    // integer rescale of a 12-real long link's rebuilt third row (30-bit FP64-class stencil)
    int lng_r2_mul, lng_r2_shift;
};

// lng_r2_mul and lng_r2_shift of a view whose lng_scale_d is set
inline void set_row2_rescale(GaugeView *v)
{
    int e = 0;
    const double f = std::frexp(2.0 * v->lng_scale_d, &e);  // 2s = f 2^e, f in [0.5, 1)
    long long m = std::llround(std::ldexp(f, 31));
    if (m >= (1LL << 31)) {
        m >>= 1;
        e += 1;
    }
    v->lng_r2_mul = (int)m;         // 2s = m 2^(e - 31)
    v->lng_r2_shift = -1 - e;       // 2^(e - 31) = 2^-(32 + shift)
}

struct DslashArgs {
    Geom g;
    GaugeView gv;
    int out_parity;
    const char *in;         // input parity field
    char *out;              // output parity field
    const char *y;          // xpay field (output parity), may be null
    double a;               // out = a*y + sign*D in (xpay) or sign*D in
    int sign;               // +1 or -1
    int xpay;
    const int *active;      // skip when *active == 0 (null: always run)
    int *err;               // set to 1 on a non-finite store
    RedBuf red;
    int fin;
    void *st;               // CGState or MSState, per finisher
    int slot;               // ring slot handed to the finisher
    int defer_finish;       // reducing pass: leave the summing launch to launch_dslash_finish
};

// The fused M_ee pass (d1: D_oe into tmp; d2: D_eo from tmp with xpay and the
// reduction), scheduled in t-slices through red.sync.
struct MeeArgs {
    DslashArgs d1;
    DslashArgs d2;
    int lag;            // slices between the last D_oe a D_eo slice reads and that D_eo
    int blocks_per_sm;  // resident blocks per SM asked (0: as many as fit)
    unsigned wait_polls;    // polls before a wait gives up (set by the launcher)
    unsigned wait_extra;    // added to every wait's target: nonzero only to test the bound
};

// A tile of right-hand sides for the batched stencil: right-hand side t lives
// in the fields at in/out/y + t * field_bytes.
constexpr int kMaxRHS = 16;
constexpr int kMrhsBlock = 128;  // threads per block of the batched stencil

struct DslashMArgs {
    Geom g;
    GaugeView gv;
    int out_parity;
    const char *in;
    char *out;
    const char *y;
    size_t field_bytes;
    double a[kMaxRHS];      // per right-hand side xpay coefficient
    int sign;
    int xpay;
    int nrhs;
    int t0;                 // first right-hand side of the tile (set by the launcher)
    unsigned tile_mask;     // bit k: launch tile k (0: every tile)
    const int *active_any;  // skip when *active_any == 0 (null: always run)
    int *err;
    RedBuf red;
    int fin;
    CGState *st;            // per right-hand side states (st[t])
    int slot;
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// Returns false when the (gauge, spinor, compute, long_recon) combination has
// no kernel.
bool launch_dslash(int gf, int sf, int cf, int long_recon, bool reduce, const DslashArgs &a,
                   cudaStream_t s);
// The summing launch of a reducing pass launched with a.defer_finish set.
bool launch_dslash_finish(int gf, int sf, int cf, int long_recon, const DslashArgs &a, cudaStream_t s);
// Block partials the reducing pass leaves in a.red.partials (its block count).
unsigned dslash_partials(int gf, int sf, int cf, int long_recon, const Geom &g);
// 1: the CG iteration's alpha and beta are summed by every block of the kernel
// that uses them (hisq_cg_split_scalars)
extern std::atomic<int> split_mode;
// Batched stencil over all right-hand sides in tiles of T (T in {1,2,4,8,16},
// dividing nrhs), variant 0 (register kernel) or 1 (staged neighbour loads,
// 16-byte spinor records only); false when the triplet or variant has no
// batched kernel.
bool launch_dslash_mrhs(int gf, int sf, int cf, int long_recon, bool reduce, int T, int variant, const DslashMArgs &a,
                        cudaStream_t s);
// Times each stencil launch shape on `a` (run as a plain pass: `a.out` is
// overwritten) and keeps the fastest for this triplet and lattice.  Call
// outside stream capture.
void tune_dslash(int gf, int sf, int cf, int long_recon, const DslashArgs &a, cudaStream_t s);
int stencil_config(int gf, int sf, int cf, int long_recon, bool reduce, const Geom &g);
// The fused M_ee pass (red.sync must be set); false when the triplet or the
// lattice has none, or it is switched off (hisq_mee_fused).
bool mee_fused_available(int gf, int sf, int cf, const Geom &g);
bool launch_mee_fused(int gf, int sf, int cf, int long_recon, const MeeArgs &m, cudaStream_t s);
int stencil_config_in_use(int gf, int sf, int cf, int long_recon, bool reduce, const Geom &g);

void launch_pack_spinor(int sf, int64_t n, const double *in, char *out, int *err, cudaStream_t s);
void launch_pack32_spinor(int sf, int64_t n, const float *in, char *out, int *err, cudaStream_t s);
void launch_pack_pair_int30(int64_t n, const float *in, char *out, int *err, cudaStream_t s);
void launch_unpack_spinor(int sf, int cf, int64_t n, const char *in, double *out, cudaStream_t s);

// gauge preparation
// out_max / out_maxdev must be zeroed before the launch (atomic max)
void launch_absmax(int64_t n, const double *x, double *out_max, cudaStream_t s);
void launch_r12_check(const Geom &g, const double *links, int k, double *out_maxdev, cudaStream_t s);
// FP64 rebuild error of a field stored with 8 reals: out[0] the largest
// element error, out[1] the sum of squared element errors (both zeroed before
// the launch); el / an: element and angle scales
void launch_r8_check(const Geom &g, int gf, const double *links, const char *stored, double el, double an,
                     double *out, cudaStream_t s);
// max over links of |U U^+ - 1| (out_maxdev zeroed before the launch)
void launch_u3_check(const Geom &g, const double *links, double *out_maxdev, cudaStream_t s);
void launch_quantise_links(const Geom &g, int gf, int recon, const double *links, double inv, char *out,
                           cudaStream_t s);


// ---------------------------------------------------------------------------
// host objects behind the opaque ABI handles
// ---------------------------------------------------------------------------
struct LinkCopy {
    int gf = -1, recon = 0;
    char *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace hisq

struct hisq_gauge {
    hisq::Geom geom;
    int dims[4];
    unsigned flags;
    double *fat64 = nullptr;   // device FP64 [mu][lex][18]
    double *lng64 = nullptr;
    double fat_max = 0, lng_max = 0;
    bool fat_r12_ok = false, lng_r12_ok = false;
    bool lng_u3_ok = false;    // long links unitary: the 13-real format applies
    std::vector<hisq::LinkCopy> fat_copies, lng_copies;
    mutable std::mutex copy_mu;  // guards fat_copies / lng_copies (built lazily)
};

namespace hisq {
struct Server;  // request loop (serve.cu)
void server_shutdown(hisq_ctx *c);

// Optional per-launch timing (benchmarks): launches made outside graph
// capture are bracketed by CUDA events on their own stream.
enum ProfKind { PROF_STENCIL = 0, PROF_STENCIL_HI = 1, PROF_BLAS = 2, PROF_CONVERT = 3, PROF_NKIND = 4 };
struct Profiler {
    bool on = false;
    unsigned mask = ~0u;  // classes that get event pairs
    int every = 1;        // a graph-launched solver times one block of iterations in `every`
    struct Rec {
        cudaEvent_t a, b;
        int kind;
        double bytes;
        int tag;  // iteration within a solver's block (-1: always counted), see prof_settle
        int nl;   // kernel launches between the two events
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double ms[PROF_NKIND] = {0, 0, 0, 0};
    int64_t launches[PROF_NKIND] = {0, 0, 0, 0};
    double bytes[PROF_NKIND] = {0, 0, 0, 0};
};
}  // namespace hisq

struct hisq_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    cudaStream_t stream = nullptr;
    hisq::RedBuf red{};
    int *err_flag = nullptr;         // device int
    std::string last_error;
    std::mutex mu;
    std::vector<hisq_gauge *> gauges;
    // scratch fields used by hisq_dslash (grown on demand)
    char *scratch = nullptr;
    size_t scratch_bytes = 0;
    std::atomic<int64_t> launches{0};  // kernels launched (graph replays count their nodes)
    std::mutex alloc_mu;               // device allocations and lazily built gauge copies
    std::mutex err_mu;                 // last_error
    hisq::Server *server = nullptr;    // request loop, started by the first hisq_submit
    std::mutex prof_mu;
    hisq::Profiler prof;
};

namespace hisq {

// Per-thread execution state.  A worker thread of the request loop runs its
// solves with its own reduction buffer and error flag (its "lane"); every
// other thread uses the context's.  Graph capture is per thread as well.
struct Lane {
    RedBuf red;
    int *err;
};
void set_thread_lane(const Lane *lane);
const RedBuf &cur_red(hisq_ctx *c);
int *cur_err(hisq_ctx *c);
void set_thread_capturing(bool on);
bool thread_capturing();
// Profiling tag of the launches that follow on this thread: the iteration
// within a solver's block (-1: none).  Launches of iterations that the device
// skipped (the block stopped early) are then left out of the statistics.
void set_prof_tag(int tag);

// status helpers (context.cu)
hisq_status fail(hisq_ctx *c, hisq_status s, const char *fmt, ...);
hisq_status cuda_fail(hisq_ctx *c, cudaError_t e, const char *what);
hisq_status ctx_alloc(hisq_ctx *c, size_t bytes, void **p);
void ctx_free(hisq_ctx *c, void *p, size_t bytes);
cudaStream_t pick_stream(hisq_ctx *c, void *s);

// launch bookkeeping: call before / after every kernel launch on stream s
struct LaunchScope {
    hisq_ctx *c;
    cudaStream_t s;
    int kind;
    double bytes;
    int tag = -1;
    int nl = 1;
    bool in_graph = false;
    cudaEvent_t a = nullptr, b = nullptr;
    // nl: the launches the scope encloses (counted as nl launches of kind)
    LaunchScope(hisq_ctx *c, cudaStream_t s, int kind, double bytes, int nl = 1);
    ~LaunchScope();
};
void prof_flush(hisq_ctx *c);   // resolve pending event pairs (synchronises on them)
void prof_flush_locked(hisq_ctx *c);
// After a block of iterations of which n_exec ran: drop the pending records
// tagged with a later iteration (launches that returned at once).
void prof_settle(hisq_ctx *c, int n_exec);
// Profiling inside a captured graph: while a recorder is set on the capturing
// thread, launch scopes record their event pairs as graph nodes (external
// event records) into it; after each replay of the graph and a synchronise,
// prof_graph_account adds the pairs of the first n_exec iterations to the
// statistics; prof_graph_release returns the events to the pool.
void set_graph_recorder(std::vector<Profiler::Rec> *rec);
void prof_graph_account(hisq_ctx *c, const std::vector<Profiler::Rec> &recs, int n_exec);
void prof_graph_release(hisq_ctx *c, std::vector<Profiler::Rec> &recs);
bool stream_capturing(cudaStream_t s);
// Kernel nodes of a captured graph (the launches one replay makes).
cudaError_t graph_kernel_nodes(cudaGraph_t g, size_t *n);

// A validated triplet: returns HISQ_OK and the device view of the gauge copy.
hisq_status gauge_view_for(hisq_ctx *c, hisq_gauge *g, const hisq_prec &p, GaugeView *v);
hisq_status check_prec(hisq_ctx *c, const hisq_prec &p);
// The same view without building a missing copy (never allocates).
hisq_status gauge_view_existing(hisq_ctx *c, const hisq_gauge *g, const hisq_prec &p, GaugeView *v);

}  // namespace hisq
