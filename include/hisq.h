/*
 * hisq.h -- C ABI of the GB300 (sm_103a) HISQ staggered stencil with reduced-bit
 * storage formats and the stabilised mixed-precision Krylov solvers of
 * M. A. Clark, D. Howarth, J. Tu, M. Wagner, E. Weinberg,
 * "Maximizing the Bang Per Bit" (Lattice 2022).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice extents dims = {Lx, Ly, Lz, Lt}, each even and >= 2 (the even/odd
 * decomposition needs even extents).  lex = ((t*Lz + z)*Ly + y)*Lx + x,
 * parity(x) = (x+y+z+t) mod 2, checkerboard index cb = lex/2, V = Lx*Ly*Lz*Lt,
 * Vh = V/2.
 *
 * Host gauge layout (both link fields): double [mu][t][z][y][x][3][3][re,im],
 * links already multiplied by the staggered phases eta_mu(x) (and by the
 * boundary sign if antiperiodic in t).
 *
 * Spinor layout seen by callers: double [cb][color][re,im] on one parity
 * (half lattice, Vh*6 doubles) or [parity][cb][color][re,im] on the full
 * lattice (even first, V*6 doubles).  Pointers are host pointers unless the
 * call's on_device flag is set, in which case they are device pointers of the
 * context's GPU (e.g. a torch tensor's data_ptr()).  The caller keeps
 * ownership of every pointer it passes; the library never frees them.
 *
 * The stencil (the HISQ operator of Sec. 1 and Sec. 5.2, whose form the paper
 * does not write out; see the design notes for this reading):
 *   (D psi)(x) = sum_mu [ F_mu(x) psi(x+mu) - F_mu(x-mu)^+ psi(x-mu)
 *                       + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^+ psi(x-3mu) ]
 * with fat links F and long (Naik) links L.  D is anti-Hermitian;
 * D_eo / D_oe are its parity blocks (output even / odd).  Full-lattice
 * operator M = 2m + D; even-even normal operator M_ee = 4m^2 - D_eo D_oe.
 *
 * Errors: every call returns a hisq_status; nothing aborts or exits.  After a
 * failure hisq_last_error() describes it.  A context is not safe for
 * concurrent calls from several threads except hisq_submit / hisq_poll.
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HISQ_API __attribute__((visibility("default")))
#else
#define HISQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HISQ_OK = 0,
    HISQ_EINVAL = 1,      /* bad argument, unsupported combination, non-finite input */
    HISQ_ENOMEM = 2,      /* HBM budget or device allocation exhausted */
    HISQ_ENOTCONV = 3,    /* solver hit maxiter; best x returned, info filled */
    HISQ_EBREAKDOWN = 4,  /* solver recurrence broke down (zero or non-finite scalar) */
    HISQ_ECUDA = 5,       /* a CUDA runtime call failed */
    HISQ_EBUSY = 6,       /* request queue full */
    HISQ_ETIMEOUT = 7,    /* bounded wait expired */
    HISQ_ENOTFOUND = 8,   /* unknown ticket or gauge */
    HISQ_ERANGE = 9       /* a result could not be stored in its storage format (non-finite, or beyond
                             the format's exponent range): the packed formats write such a site as
                             zero, FP64 and FP32 keep the non-finite value */
} hisq_status;

/* Storage format of the gauge field (Sec. 4, the three-precision triplet). */
typedef enum {
    HISQ_GAUGE_F64 = 0,
    HISQ_GAUGE_F32 = 1,
    HISQ_GAUGE_FIX16 = 2, /* 16-bit fixed point, scale = global max (Sec. 2 footnote) */
    HISQ_GAUGE_FIX32 = 3, /* 32-bit fixed point, scale = global max (Sec. 4) */
    HISQ_GAUGE_SE15 = 4   /* per link: 15-bit integers sharing one 8-bit exponent (a shared-exponent
                             gauge format for smeared fat links; 2 bytes a real) */
} hisq_gauge_fmt;

/* Storage format of the fermion (spinor) field. */
typedef enum {
    HISQ_SPINOR_F64 = 0,    /* 48 B/site */
    HISQ_SPINOR_F32 = 1,    /* 24 B/site */
    HISQ_SPINOR_HALF16 = 2, /* 16 B/site: int16 v[6] + FP32 site max (Sec. 2, Listing 1) */
    HISQ_SPINOR_INT20 = 3,  /* 16 B/site: 6 x int20 + 8-bit exponent (Sec. 4 Listing 2; Appendix A) */
    HISQ_SPINOR_INT30 = 4,  /* 24 B/site: 6 x int30 + 8-bit exponent (Sec. 4, Listing 3) */
    HISQ_SPINOR_INT14 = 5   /* 12 B/site: 6 x int14 + 8-bit exponent (a third width of the Sec. 4
                               shared-exponent family; the Appendix A rule with scale 2^13 - 1) */
} hisq_spinor_fmt;

/* Arithmetic precision (the third member of the triplet, Sec. 4). */
typedef enum { HISQ_COMPUTE_F32 = 0, HISQ_COMPUTE_F64 = 1 } hisq_compute_fmt;

/* Precision triplet gauge / fermion / compute plus link compression (Sec. 1:
 * 18 -> 12 reals by SU(3) unitarity).  Supported combinations:
 *   F64/F64/F64, F32/F32/F32, FIX16/HALF16/F32, FIX16/INT20/F32,
 *   FIX32/INT30/F64, FIX32/INT30/F32, and, in the single-right-hand-side
 *   solvers only, FIX16/INT14/F32 and SE15/INT20/F32;
 * fat_recon must be 18 (smeared fat links are not unitary); long_recon 18,
 * 12, 13 or 8:
 *   12: rows 0 and 1; needs long links that are a sign times SU(3) (checked
 *       at load, EINVAL otherwise);
 *   13: rows 0, 1 and arg(det U)/pi; needs unitary long links (U(3));
 *   8:  arg V00, arg V20, V01, V02, V10 of V = sign * U in SU(3), rebuilt
 *       from unitarity and det V = 1; needs a sign times SU(3), and the first
 *       use of a format builds the copy, rebuilds it in FP64 and returns
 *       EINVAL when its root-mean-square error per real exceeds 4 storage
 *       steps or is not finite (links with V00 = 1, e.g. a free field);
 *   13 and 8 are supported on FP32-compute triplets with FIX16 or F32 links
 *   and in the single-right-hand-side solvers (EINVAL elsewhere). */
typedef struct {
    int32_t gauge;      /* hisq_gauge_fmt */
    int32_t spinor;     /* hisq_spinor_fmt */
    int32_t compute;    /* hisq_compute_fmt */
    int32_t fat_recon;  /* 18 */
    int32_t long_recon; /* 18, 12, 13 or 8 */
} hisq_prec;

typedef struct hisq_ctx hisq_ctx;
typedef struct hisq_gauge hisq_gauge;

/* hisq_load_gauge flags */
#define HISQ_GAUGE_ANTIPERIODIC_T 0x1u /* links crossing the t boundary carry -1 */
#define HISQ_GAUGE_ON_DEVICE 0x2u      /* fat/lng are device pointers */

/* Create a context on CUDA device `device`.  hbm_budget bounds the device
 * memory the context may hold (0: 90% of the free memory at creation).  The
 * context owns every device buffer, stream and scratch area it makes.
 * Errors: EINVAL (bad device, out == NULL), ECUDA. */
HISQ_API hisq_status hisq_create(int device, size_t hbm_budget, hisq_ctx **out);

/* Release a context and everything it owns (gauge fields included). */
HISQ_API void hisq_destroy(hisq_ctx *ctx);

/* Message of the last failed call on this context (never NULL). */
HISQ_API const char *hisq_last_error(hisq_ctx *ctx);

/* Device bytes the context currently holds. */
HISQ_API size_t hisq_mem_used(hisq_ctx *ctx);

/* Load a gauge configuration (Sec. 2 footnote, Sec. 4: one global scale per
 * fixed-point field).  fat and lng are FP64 in the host gauge layout
 * (4*V*18 doubles each).  The data are copied: an FP64 copy of each field
 * stays resident for true residuals; reduced formats are built from it on
 * first use.  Checks: extents even and >= 2 (EINVAL), every entry finite
 * (EINVAL), budget (ENOMEM).  Whether each field can be compressed to 12 reals
 * (a sign times SU(3), to 1e-6) is recorded; asking for r12 on a field that
 * cannot be returns EINVAL at use.  Free with hisq_free_gauge. */
HISQ_API hisq_status hisq_load_gauge(hisq_ctx *ctx, const int dims[4], const double *fat, const double *lng,
                            unsigned flags, hisq_gauge **out);

HISQ_API void hisq_free_gauge(hisq_ctx *ctx, hisq_gauge *g);

/* Global max |element| of the fat (which = 0) or long (which = 1) field: the
 * fixed-point scale of Sec. 2 footnote. */
HISQ_API double hisq_gauge_scale(const hisq_gauge *g, int which);

/* One application of the stencil in precision `prec` (Sec. 5.2-5.3: the
 * fields are stored in the reduced formats, unpacked to the compute precision
 * in registers and repacked on store):
 *   out = a * xpay_in - D in      (a != 0)
 *   out = D in                    (a == 0; xpay_in may be NULL)
 * out_parity 0: out on even sites, in on odd sites (D_eo); 1: the reverse
 * (D_oe); 2: full lattice (in, out, xpay_in full-lattice arrays).
 * in / out / xpay_in are FP64 arrays in the caller's spinor layout; the input
 * (and xpay_in) is rounded into the spinor storage format first, and the
 * output is the decoded storage-format result.  on_device selects device or
 * host pointers; stream is a cudaStream_t (NULL: the context's stream).
 * Errors: EINVAL (unsupported prec, r12 not possible, non-finite input),
 * ERANGE (some output sites could not be stored in the spinor format: the
 * result overflowed the compute precision or the format's exponent range;
 * out holds zero there for the packed formats, the non-finite value for FP64
 * and FP32), ENOMEM, ECUDA. */
HISQ_API hisq_status hisq_dslash(hisq_ctx *ctx, const hisq_gauge *g, hisq_prec prec, int out_parity, double a,
                        const double *xpay_in, const double *in, double *out, int on_device,
                        void *stream);

/* Sites per parity accepted by hisq_dslash_noalloc: 2^15, e.g. a 16^4 lattice
 * (its fixed scratch is 3 x 48 B x 2 x 2^15 = 9 MiB plus 256 B). */
#define HISQ_NOALLOC_MAX_SITES 32768

/* hisq_dslash for callers that cannot allocate device memory.  The paper has
 * no counterpart; it exists because some callers may not call cudaMalloc: an
 * application whose own pool allocator has already reserved the GPU's memory
 * (an allocation would fail or fragment that pool), or a long-running loop
 * that must not allocate, since cudaMalloc and cudaFree synchronise the device
 * and can fail partway through a run.  Same arguments and result as
 * hisq_dslash with on_device = 1 (in, out, xpay_in are device pointers) but
 * it allocates nothing: its scratch (the fields in the storage format and a
 * non-finite counter) is one fixed device array of this library, which every
 * GPU that loads the library holds until the process exits.
 * Limits and rules:
 *  - at most HISQ_NOALLOC_MAX_SITES sites per parity, else EINVAL;
 *  - the gauge field must already hold its stored copy for `prec` (any earlier
 *    hisq_dslash or solver call with that precision builds it), else EINVAL;
 *  - the call copies a counter back to the host and synchronises `stream`,
 *    so it must not be made while `stream` is being captured (EINVAL);
 *  - the first call on a device looks up the scratch array's device address
 *    once (cudaGetSymbolAddress);
 *  - output sites that cannot be stored in the spinor format return ERANGE,
 *    as in hisq_dslash;
 *  - every call uses the same scratch array, which keeps the previous call's
 *    contents (the counter is cleared at each call): calls whose work overlaps
 *    on the GPU (several streams or host threads) race, so serialise them. */
HISQ_API hisq_status hisq_dslash_noalloc(hisq_ctx *ctx, const hisq_gauge *g, hisq_prec prec, int out_parity,
                                         double a, const double *xpay_in, const double *in, double *out,
                                         void *stream);

/* Device bytes of one half-lattice (n sites) spinor field in format sfmt, in
 * this library's planar layout: the site record is split into 16-byte planes
 * [plane][site] followed by one narrower tail plane (F32 and INT30: 16 + 8 B;
 * F64: 3 x 16 B; HALF16 and INT20: one 16-B record = the paper's struct;
 * INT14: an 8-B plane (words 0, 1) and a 4-B plane (word 2)). */
HISQ_API size_t hisq_spinor_bytes(int sfmt, int64_t n);

/* Encode n sites (FP64 [n][6] on the device) into format sfmt (planar layout
 * above) on the device, exactly as every kernel of the library stores a
 * field: HALF16, INT20 and INT14 round the input to FP32 first and encode in
 * FP32 (Appendix A arithmetic for INT20 and INT14); INT30 encodes in FP64.  *n_bad receives
 * the number of sites with a non-finite (or, for INT30, unencodable)
 * component; such sites are stored as zero.  Device pointers only. */
HISQ_API hisq_status hisq_spinor_pack(hisq_ctx *ctx, int sfmt, int64_t n, const double *in, void *packed,
                             int64_t *n_bad, void *stream);

/* Encode n sites of FP32 [n][6] input (device) into format sfmt (F32, HALF16,
 * INT20, INT30 or INT14) exactly as the FP32-compute kernels store a field; for
 * INT30 the bits equal those of hisq_spinor_pack on the same (FP32-exact)
 * values.  *n_bad counts non-finite sites (stored as zero). */
HISQ_API hisq_status hisq_spinor_pack32(hisq_ctx *ctx, int sfmt, int64_t n, const float *in, void *packed,
                               int64_t *n_bad, void *stream);

/* Encode n sites given as FP32 pairs [n][6][hi, lo] (value hi + lo, |lo| at
 * most half an ulp of hi; device) into INT30 exactly as the FP64-class
 * kernels store a field: the 30-bit rule applied to the exact value hi + lo,
 * so the bits equal those of hisq_spinor_pack wherever hi + lo is exact in
 * FP64. */
HISQ_API hisq_status hisq_spinor_pack_pair_int30(hisq_ctx *ctx, int64_t n, const float *in, void *packed,
                                        int64_t *n_bad, void *stream);

/* Decode n sites of format sfmt into FP64 [n][6] (device pointers).  compute
 * selects the precision of the decode (F32 decodes as the F32 kernels do). */
HISQ_API hisq_status hisq_spinor_unpack(hisq_ctx *ctx, int sfmt, int compute, int64_t n, const void *packed,
                               double *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* Kernel classes timed by the profiler. */
#define HISQ_PROF_STENCIL 0     /* stencil passes in the call's (sloppy) precision */
#define HISQ_PROF_STENCIL_HI 1  /* FP64 stencil passes of true residuals */
#define HISQ_PROF_BLAS 2        /* fused BLAS-1 / reduction kernels */
#define HISQ_PROF_CONVERT 3     /* format conversions */

typedef struct {
    double ms;          /* summed device time of the timed launches */
    int64_t launches;   /* launches timed */
    double bytes;       /* summed algorithmic bytes of those launches: each
                           array touched once per launch (links, input and
                           output spinors, xpay input) */
} hisq_kernel_stats;

/* While enabled, every launch of a selected class is bracketed by CUDA events
 * on its own stream and accumulated per class.  The CG solver keeps its
 * graphs: the event pairs are then recorded as graph nodes and read after
 * each block of iterations, and launches of iterations the device skipped
 * (the block stopped early) are not counted; the other solvers run without
 * graphs while profiling.  Reading synchronises on the events. */
HISQ_API void hisq_profile_enable(hisq_ctx *ctx, int on);
HISQ_API void hisq_profile_reset(hisq_ctx *ctx);
HISQ_API hisq_status hisq_profile_read(hisq_ctx *ctx, int kind, hisq_kernel_stats *out);
/* Classes that get event pairs: bit k selects class k (default all).  Each
 * event pair costs some device time, so a caller timing a solve may select
 * only the class it needs.  Unselected classes are not counted. */
HISQ_API void hisq_profile_select(hisq_ctx *ctx, unsigned mask);
/* Sample period of the CG solver's graphs: with every > 1 the solver keeps a
 * second graph without event pairs and times only one block of iterations in
 * `every` (the first of each solve included), so that the event nodes (each
 * costs device time) perturb a timed solve less; the per-class averages then
 * come from the sampled blocks.  Other solvers time every launch.  every = 1
 * (default) times every block.  EINVAL when every < 1. */
HISQ_API hisq_status hisq_profile_sample(hisq_ctx *ctx, int every);

/* Launch shape of the stencil kernels: -1 (default) lets the library time the
 * shapes the first time a (precision, lattice) pair is used and keep the
 * fastest (separately for the plain pass and for the pass with the fused
 * reduction); 0..4 forces one shape for every later launch in the process.
 * hisq_stencil_config sets the plain pass and, unless
 * hisq_stencil_config_reduce has set its own, the reducing pass too.
 * Returns the previous setting, or -2 for an invalid value.  For benchmarking
 * and testing the shapes. */
HISQ_API int hisq_stencil_config(int cfg);
/* The normal operator M_ee as one fused pass (D_oe and D_eo swept over
 * t-slices in one persistent kernel so that each link is read from HBM about
 * once) instead of two stencil passes: 1 on, 0 off (default).  FP32-compute
 * triplets, Lt <= 4096.  Returns the previous setting, or -2 for an invalid
 * value.  Has no counterpart in the paper (a cache-blocking of its operator). */
HISQ_API int hisq_mee_fused(int mode);
/* Schedule of the fused pass: lag = t-slices between the last D_oe slice a
 * D_eo slice reads and that D_eo slice in the work order (default 4; larger
 * waits less, keeps more of the lattice in L2), blocks_per_sm = resident
 * blocks asked per SM (0, the default: as many as fit).  Negative values leave
 * a setting unchanged.  For benchmarking. */
HISQ_API void hisq_mee_fused_shape(int lag, int blocks_per_sm);
/* Test control of the fused pass's bounded waits (a block waits for earlier
 * t-slices of the same launch): polls = polls before a wait gives up (0: the
 * default, 2^22 polls of at least 64 ns each); unreachable = 1 raises every
 * wait's target past what the launch can reach, so each wait runs to its
 * limit, the kernel flags the error and goes on, and the solver returns
 * ECUDA.  Only for testing that a wait ends; 0 restores normal waits. */
HISQ_API void hisq_mee_fused_wait_test(unsigned polls, int unreachable);
HISQ_API int hisq_stencil_config_reduce(int cfg);
/* Programmatic dependent launch of the solvers' kernel chains (stencil
 * passes, their finish kernel and the fused BLAS kernels): 1 (default) lets
 * each kernel's blocks be scheduled while its predecessor's last wave runs
 * (every kernel waits for its predecessor's results before touching them, so
 * results are identical either way); 0 launches them one after another.
 * Returns the previous setting, or -2 for an invalid value.  For benchmarking;
 * no counterpart in the paper. */
HISQ_API int hisq_programmatic_launch(int mode);
/* The scalar steps of the CG iteration (Sec. 3.1: alpha = |r|^2 / p.Ap and
 * beta): 1 (default) every block of the residual update sums the reducing
 * stencil pass's per-block partials itself, in one fixed order, and takes
 * alpha from them, and every block of the gradient update does the same for
 * beta, so no one-block launch or last-block tail sits between the kernels;
 * 0 sums them once, in a one-block launch after the stencil pass and in the
 * last block of the residual update.  The sums are deterministic in both
 * modes; their rounding differs between the two (other block shapes).  The
 * FP64 triplet (FP64 sloppy storage) always takes the second form (faster
 * there).  Returns the previous setting, or -2 for an invalid value.  Read
 * when a solve starts.  For benchmarking; no counterpart in the paper. */
HISQ_API int hisq_cg_split_scalars(int mode);
/* The shape in use for triplet p on gauge g's lattice (plain pass, or the
 * reducing pass if reduce != 0): the forced one, else the tuned one, else -1
 * when that pair has not been tuned yet. */
HISQ_API int hisq_stencil_config_in_use(const hisq_gauge *g, hisq_prec p, int reduce);

/* Kernels this context has launched so far (graph replays add their nodes). */
HISQ_API int64_t hisq_launch_count(hisq_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Solvers                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double mass;          /* m */
    double tol;           /* target |b - A x| / |b| on the FP64 true residual */
    int32_t maxiter;      /* iteration cap (CG iterations; BiCGStab(l): matvecs) */
    double delta;         /* reliable-update trigger (Sec. 3 footnote: 0.1) */
    hisq_prec sloppy;     /* precision of the iterated vectors and matvecs */
    hisq_prec refine;     /* multi-shift: precision of the refinement CG (Sec. 3.2) */
    int32_t nbuf;         /* gradient vectors buffered before x is updated (Sec. 3.1 item 1); 1..16 */
    int32_t use_init_guess; /* x holds the initial guess */
    int32_t on_device;    /* b and x are device pointers */
    int32_t pr_beta;      /* 1: Polak-Ribiere beta (Sec. 3.1 item 3), 0: Fletcher-Reeves */
    int32_t reproject;    /* 1: re-project p at each reliable update (Sec. 3.1 item 2) */
    int32_t l;            /* BiCGStab(l): l (Sec. 6.1 uses 4), 1..8 */
    int32_t use_graph;    /* 1: replay each block of iterations as a CUDA graph */
    int32_t nrhs;         /* hisq_cg: right-hand sides solved together (1..16, Sec. 1 block solvers) */
    int32_t rhs_tile;     /* right-hand sides per stencil launch (1,2,4,8,16 dividing nrhs; 0: tuned) */
    int32_t rhs_kernel;   /* batched stencil kernel: 0 tuned, 1 registers, 2 staged neighbour loads
                             (16-bit and 20-bit fermions only; EINVAL otherwise) */
    void *stream;         /* cudaStream_t; NULL: the context's stream */
    double *history;      /* host array or NULL: with nrhs = 1, hisq_cg and hisq_solve_full write
                             |r_k| / |b| of the CG's iterated residual for k = 0, 1, ... (at most
                             history_len entries, up to the last iteration); at an iteration that
                             ends with a reliable update the entry is the recomputed FP64 true
                             residual instead (the jumps of Fig. 1) */
    int32_t history_len;  /* entries of history (0: none kept) */
    int32_t ru_trigger;   /* CG reliable-update trigger: 0 when |r| drops below delta times its
                             maximum since the last update (Sec. 3 footnote); 1 an error estimate
                             (the footnote's dynamic choice, after van der Vorst and Ye's residual
                             replacement): the drift d of the iterated from the true residual grows
                             by eps (|r_k+1| + |alpha_k| |A p_k|) per iteration, eps the sloppy
                             triplet's coarsest unit roundoff, and an update is made when d
                             crosses sqrt(eps) |r| (and exceeds 1.1 times its value after the last
                             update) */
} hisq_solver_params;

/* Fills params with the defaults: delta 0.1, nbuf 8, pr_beta 1, reproject 1,
 * l 4, use_graph 1, nrhs 1, rhs_tile 0, rhs_kernel 0, maxiter 100000, tol 1e-10, sloppy
 * and refine FIX16/INT20/F32 with r12 long links, no history, ru_trigger 0. */
HISQ_API void hisq_default_params(hisq_solver_params *p);

#define HISQ_MAX_SHIFTS 32

typedef struct {
    int32_t iters;              /* iterations (CG) or BiCGStab(l) cycles */
    int32_t matvecs;            /* operator applications in the sloppy precision */
    int32_t matvecs_hi;         /* operator applications in FP64 (true residuals) */
    int32_t reliable_updates;
    double true_residual;       /* |b - A x| / |b| in FP64 at exit */
    double seconds;             /* wall time of the solve */
    int32_t nshift;
    int32_t shift_iters[HISQ_MAX_SHIFTS];    /* multi-shift: iteration at which shift i froze */
    double shift_resid_ms[HISQ_MAX_SHIFTS];  /* true residual of shift i after the multi-shift stage */
    double shift_resid[HISQ_MAX_SHIFTS];     /* final true residual of shift i */
    int32_t refine_iters[HISQ_MAX_SHIFTS];   /* refinement CG iterations of shift i */
} hisq_solve_info;

/* Even/odd CG (Sec. 3.1): solves (4m^2 - D_eo D_oe) x = b on the even sites
 * with the sloppy triplet for the iterated residual and gradient vectors,
 * FP64 for x (accumulated from nbuf buffered gradient vectors), reliable
 * updates with an FP64 true residual whenever |r| drops below delta times its
 * maximum since the last update, re-projection of p and Polak-Ribiere beta.
 * With sloppy = F64/F64/F64 this is plain FP64 CG.  b, x: half-lattice FP64.
 * With nrhs > 1, b and x hold nrhs half-lattice fields back to back and the
 * systems are iterated together: every stencil launch applies each link it
 * loads to a tile of rhs_tile right-hand sides (sloppy triplets F32, half and
 * 20-bit); each right-hand side keeps its own recurrence and stops on its own;
 * info then reports the largest iteration count and true residual and the
 * summed operator applications.
 * Returns OK, ENOTCONV (x is the best iterate, info filled), EBREAKDOWN,
 * EINVAL, ENOMEM, ECUDA. */
HISQ_API hisq_status hisq_cg(hisq_ctx *ctx, const hisq_gauge *g, const hisq_solver_params *p, const double *b,
                    double *x, hisq_solve_info *info);

/* Full-lattice solve of (2m + D) x = b (m != 0) by even/odd reduction
 * around the CG of hisq_cg (Sec. 3: the solvers work on the even-site
 * system; this is the step either side of them).  With M = [[2m, D_eo],
 * [D_oe, 2m]] in parity blocks:
 *   bt_e = 2m b_e - D_eo b_o                     (FP64 stencil),
 *   (4m^2 - D_eo D_oe) x_e = bt_e                (hisq_cg with p),
 *   x_o  = (b_o - D_oe x_e) / (2m)               (FP64 stencil).
 * The even residual of the full system is the CG's residual over 2m and the
 * odd one vanishes, so the CG runs to the tolerance tol * 2|m| |b| / |bt_e|,
 * which makes |b - M x| / |b| <= tol.  b, x: full-lattice FP64 arrays
 * ([parity][cb][color][re,im], even first), nrhs of them back to back;
 * p->use_init_guess is ignored (the even CG starts from zero).
 * info->true_residual is the FP64 |b - M x| / |b| (the largest over the
 * right-hand sides); iters, matvecs and reliable updates are the CG's.
 * Returns OK, ENOTCONV, EBREAKDOWN, EINVAL (m == 0 or as hisq_cg), ENOMEM,
 * ECUDA. */
HISQ_API hisq_status hisq_solve_full(hisq_ctx *ctx, const hisq_gauge *g, const hisq_solver_params *p,
                                     const double *b, double *x, hisq_solve_info *info);

/* Multi-shift CG (Sec. 3.2): solves (M_ee + sigma_i) x_i = b for nshift
 * shifts (<= HISQ_MAX_SHIFTS) in the sloppy precision with reliable updates on
 * the base (smallest) shift; shift i freezes when its iterated residual
 * reaches tol[i] or the sloppy format's precision floor; then refinement CG in
 * p->refine: the base system continuing with its gradient vector, the other
 * shifts restarted from their x_i.  x[i]: half-lattice FP64 arrays. */
HISQ_API hisq_status hisq_multishift_cg(hisq_ctx *ctx, const hisq_gauge *g, const hisq_solver_params *p, int nshift,
                               const double *sigma, const double *tol, const double *b, double *const *x,
                               hisq_solve_info *info);

/* BiCGStab(l) (Sec. 6.1) on the full-lattice M = 2m + D with sloppy vectors,
 * FP64 x and a reliable update at the end of a cycle when triggered. */
HISQ_API hisq_status hisq_bicgstabl(hisq_ctx *ctx, const hisq_gauge *g, const hisq_solver_params *p, const double *b,
                           double *x, hisq_solve_info *info);

/* ------------------------------------------------------------------------ */
/* Request loop (continuous batching)                                        */
/* ------------------------------------------------------------------------ */

#define HISQ_REQ_CG 0          /* (4m^2 - D_eo D_oe) x = b */
#define HISQ_REQ_MULTISHIFT 1  /* (M_ee + sigma_i) x_i = b, i < nshift */

typedef struct {
    const hisq_gauge *gauge; /* resident gauge field: its lattice is the request's volume */
    int32_t kind;            /* HISQ_REQ_CG or HISQ_REQ_MULTISHIFT */
    double mass;
    double tol;              /* CG: target true residual */
    int32_t nshift;          /* multi-shift: number of shifts (<= HISQ_MAX_SHIFTS) */
    const double *sigma;     /* multi-shift: shifts (copied at submit) */
    const double *shift_tol; /* multi-shift: per-shift targets (copied at submit) */
    const double *b;         /* half-lattice FP64 source */
    double *x;               /* CG: one half-lattice field; multi-shift: nshift fields back to back */
    int32_t on_device;       /* b and x are device pointers */
    hisq_prec sloppy;        /* CG sloppy / multi-shift stage triplet */
    hisq_prec refine;        /* multi-shift refinement triplet */
    int32_t maxiter;
} hisq_request;

typedef struct {
    int64_t completed;
    int64_t pending;
    double latency_p50_s;  /* submit -> done */
    double latency_p99_s;
    double solves_per_s;   /* completed / (last completion - first submission) */
} hisq_serve_stats_t;

/* Queue a solve and return at once with a ticket.  Worker threads of the
 * context (each with its own stream, so their work overlaps on the device)
 * take requests in arrival order.  CG requests on the same gauge field with
 * the same sloppy triplet (FP32, half or 20-bit) share batch sessions: at
 * every block of iterations finished systems leave and queued ones join
 * (continuous batching).  A multi-shift request runs its multi-shift stage
 * on a worker; the refinement CG of each shift that has not reached its
 * target (the shifted system from the stage's solution, in the request's
 * refine triplet; unlike hisq_multishift_cg, the base system restarts too)
 * then joins the batch sessions like a CG request.  A session
 * starts only when the context's HBM budget has room for it; otherwise its
 * requests wait.  b and x stay owned by the caller and must stay valid until
 * the request is done; the gauge must not be freed while requests use it.
 * The first call starts the workers, one per reduction lane (partial sums,
 * counters, error flag; about 17 MB each) that fits the budget, up to four.
 * Errors: EINVAL (bad request), EBUSY (queue full), ENOMEM (first call: not
 * even one worker's lane fits the budget). */
HISQ_API hisq_status hisq_submit(hisq_ctx *ctx, const hisq_request *req, uint64_t *ticket);

/* Non-blocking: *done = 1 and info filled once the request finished (the
 * return value is then the solve's status and the ticket is released);
 * *done = 0 while it is queued or running.  ENOTFOUND for unknown tickets. */
HISQ_API hisq_status hisq_poll(hisq_ctx *ctx, uint64_t ticket, int *done, hisq_solve_info *info);

/* Bounded wait for a request: its status once done, ETIMEOUT after timeout_s. */
HISQ_API hisq_status hisq_wait(hisq_ctx *ctx, uint64_t ticket, double timeout_s, hisq_solve_info *info);

/* Completed requests, queue length, latency percentiles and throughput. */
HISQ_API hisq_status hisq_serve_stats(hisq_ctx *ctx, hisq_serve_stats_t *out);

#ifdef __cplusplus
}
#endif

#endif /* HISQ_H */
