// bcg.h -- batched (multi right-hand side) CG driver.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "cg.h"
#include "internal.h"

namespace hisq {

struct BCGConfig {
    int nrhs = 1;
    double diag[kMaxRHS] = {};  // 4 m_t^2 + sigma_t per right-hand side
    double tol[kMaxRHS] = {};
    hisq_prec sloppy{};
    int nbuf = 8, maxiter = 100000, pr = 1, reproject = 1, use_graph = 1;
    int tile = 0;               // RHS per stencil launch (0: tuned)
    int kernel = 0;             // batched stencil: 0 tuned, 1 registers, 2 staged
    double delta = 0.1;
    int dyn = 0;                // error-estimate trigger (every right-hand side)
    double dyn_eps = 0.0;
};

// b64 / x64: nrhs FP64 planar half-lattice fields, 48*Vh bytes apart; infos:
// nrhs entries.
hisq_status run_bcg(hisq_ctx *c, hisq_gauge *g, const BCGConfig &cfg, const double *b64, double *x64, bool x_zero,
                    hisq_solve_info *infos, cudaStream_t s);

// A batch of cfg.nrhs solver slots sharing each stencil launch (bcg.cu).
struct BatchSession {
    hisq_ctx *c;
    hisq_gauge *g;
    BCGConfig cfg;
    cudaStream_t s;
    Workspace ws;
    int vh, nr, N, T = 1, variant = 0;
    size_t fb = 0;
    char *r_s = nullptr, *ap_s = nullptr, *tmp_s = nullptr, *ring = nullptr;
    double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *ax64 = nullptr, *tmp64 = nullptr;
    CGState *st = nullptr, *sth = nullptr;
    GaugeView gv_s{}, gv_d{};
    std::vector<int> mv_hi, ru, k0, occupied, status;
    std::vector<double> bb, stop2, diag;
    std::vector<int> finished_now;
    // graphs of one block of iterations, per (tile, variant, launched tiles)
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int64_t nodes = 0;
    };
    std::map<uint64_t, Graph> graphs;
    float tile_ms[5] = {-1.f, -1.f, -1.f, -1.f, -1.f};  // one tile launch per tile size (log2 T)
    int tile_var[5] = {0, 0, 0, 0, 0};
    bool adapt = false;      // the tile may change between blocks (not fixed by the caller)
    unsigned tile_mask = 0;  // tiles launched in the current block

    BatchSession(hisq_ctx *c, hisq_gauge *g, const BCGConfig &cfg, cudaStream_t s);
    ~BatchSession();
    hisq_status setup();
    // Load a system into free slot t: b_planar (device FP64 planar, copied),
    // x_planar initial guess or null for zero.  A system that is already
    // solved goes straight to the finished list.
    hisq_status load(int t, const double *b_planar, const double *x_planar, double diag, double tol);
    hisq_status step();                // one block of iterations plus the stopped slots' updates
    std::vector<int> take_finished();  // slots that stopped since the last call
    void info_of(int t, hisq_solve_info *info) const;
    void release(int t);               // free slot t (after its x has been read)
    int active_slots() const;
    double *x_of(int t);
    double *b_of(int t);

  private:
    char *slot(int j, int t);
    void stencil_pass(int parity_out, const char *in, char *out, const char *y, bool red, int slot_i);
    void iterate_block();
    void choose_tile();
    hisq_status pull();
    void reliable_update(int t, int nslots, int j, bool x_zero);
};

}  // namespace hisq
