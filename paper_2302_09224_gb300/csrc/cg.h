// cg.h -- shared pieces of the solver drivers (CG core, operator, buffers).
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "internal.h"

namespace hisq {

// Device allocations owned by one solve; freed (after the stream drains) on
// destruction.
struct Workspace {
    hisq_ctx *c;
    cudaStream_t s;
    std::vector<std::pair<void *, size_t>> allocs;
    Workspace(hisq_ctx *c_, cudaStream_t s_) : c(c_), s(s_) {}
    ~Workspace();
    hisq_status alloc(size_t bytes, void **p);
};

struct CGConfig {
    double mass = 0, sigma = 0, tol = 1e-10;
    int maxiter = 100000;
    double delta = 0.1;
    hisq_prec sloppy{};
    int nbuf = 8;
    int pr = 1, reproject = 1, use_graph = 1;
    // continuation (multi-shift refinement of the base system): a gradient
    // vector in format p_init_fmt and the |r|^2 it was built against
    const char *p_init = nullptr;
    int p_init_fmt = 0;
    double rr_prev_init = 0.0;
    // error-estimate reliable-update trigger (dyn = 1) with the sloppy precision dyn_eps
    int dyn = 0;
    double dyn_eps = 0.0;
    // residual history: host array of hist_len entries, |r_k|/|b| per iteration
    double *hist_host = nullptr;
    int hist_len = 0;
};

// Relative precision of the sloppy operator: the largest unit roundoff of the
// triplet's gauge format, spinor format and compute precision (the precision
// the error-estimate trigger accumulates).
double sloppy_eps(const hisq_prec &p);

// field conversion between any two storage formats (ms.cu)
void launch_convert(int si, int so, int n, const char *in, char *out, int *err, cudaStream_t s);

hisq_prec prec_f64();
// Tune the stencil's launch shape for this triplet and lattice (zeroes zero_in,
// overwrites out); a no-op during stream capture or once tuned.
void tune_stencil(hisq_ctx *c, const Geom &geom, const hisq_prec &p, const GaugeView &gv, char *zero_in, char *out,
                  cudaStream_t s);
double stencil_bytes(const hisq_prec &p, int vh, bool xpay);

// Returns the number of block partials left for the next kernel when
// leave_partials is set and the reducing pass's finisher was not run (the
// caller's next kernel sums them: the split CG chain), else 0.
unsigned apply_mee(hisq_ctx *c, const Geom &geom, const hisq_prec &p, const GaugeView &gv, double diag,
                   const char *in, char *tmp, char *out, int fin, void *st, int slot, const int *active, int kind,
                   cudaStream_t s, bool leave_partials = false);

// Mixed-precision CG on (M_ee + sigma) x = b; b64 / x64 are FP64 planar device
// fields (x64 holds the initial guess unless x_zero).
hisq_status run_cg(hisq_ctx *c, hisq_gauge *g, const CGConfig &cfg, const double *b64, double *x64, bool x_zero,
                   hisq_solve_info *info, cudaStream_t s);

// The multi-shift stage alone (Sec. 3.2, without the refinement CG): shifts in
// ascending order, b64 and x64_out[i] device FP64 planar fields (x64_out
// owned by the caller, 48 Vh bytes each); info->shift_resid[i] is each
// shift's FP64 true residual over |b| after the stage.
hisq_status run_multishift_stage(hisq_ctx *c, hisq_gauge *g, const hisq_solver_params &p, int ns, const double *sigma,
                                 const double *tol, const double *b64, double *const *x64_out, hisq_solve_info *info,
                                 cudaStream_t s);

hisq_status validate_params(hisq_ctx *c, const hisq_solver_params *p);
CGConfig config_from(const hisq_solver_params *p, double sigma);
hisq_status to_planar(hisq_ctx *c, Workspace &ws, const double *user, int on_device, int64_t n, double *planar,
                      cudaStream_t s);
hisq_status from_planar(hisq_ctx *c, Workspace &ws, const double *planar, int64_t n, double *user, int on_device,
                        cudaStream_t s);

}  // namespace hisq
