// finish.cuh -- scalar recurrences of the CG iteration, run by thread 0 of the
// last block of a reducing kernel (so alpha, beta and the reliable-update and
// convergence decisions never leave the device).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hisq {

__device__ __forceinline__ void stop_iterating(CGState *st, int reason)
{
    st->reason = reason;
    st->active = 0;
}

// sums: the grid totals of the reducing kernel; slot: ring slot of p.
__device__ __forceinline__ void run_finisher(int fin, const double *sums, CGState *st, int slot)
{
    if (fin == FIN_CG_ALPHA) {
        // sums = {Re<p, A p>, |A p|^2}
        const double pAp = sums[0];
        const double alpha = st->rr / pAp;
        if (!(pAp > 0.0) || !isfinite(alpha)) {
            st->alpha = 0.0;
            stop_iterating(st, REASON_BREAKDOWN);
            return;
        }
        st->pAp = pAp;
        st->alpha = alpha;
        st->alpha_ring[slot] = alpha;
    } else if (fin == FIN_CG_BETA) {
        // sums = {|r_new|^2, Re<r_new, r_old>}; Polak-Ribiere beta (Sec. 2.1
        // item 3) = r_new^+(r_new - r_old) / |r_old|^2, else Fletcher-Reeves
        const double rr_new = sums[0];
        const double num = st->pr ? rr_new - sums[1] : rr_new;
        const double beta = num / st->rr;
        st->rr_prev = st->rr;
        st->rr = rr_new;
        st->beta = beta;
        st->k += 1;
        if (!isfinite(rr_new) || !isfinite(beta)) {
            stop_iterating(st, REASON_BREAKDOWN);
            return;
        }
        if (rr_new > st->rr_max) st->rr_max = rr_new;
        if (rr_new <= st->stop2)
            stop_iterating(st, REASON_CONVERGED);
        else if (rr_new < st->delta2 * st->rr_max)  // |r| < delta max|r| (Sec. 2 footnote)
            stop_iterating(st, REASON_RELIABLE);
    } else if (fin == FIN_CG_TRUE) {
        // sums = {|r_hi|^2, Re<r_hi, p>, Im<r_hi, p>}.  Re-projection (Sec. 2.1
        // item 2): p <- p - (<r_hi,p>/|r_hi|^2) r_hi, then Fletcher-Reeves
        // beta = |r_hi|^2/|r_old|^2 and p_new = r_hi + beta p, i.e.
        // p_new = (1 - beta c) r_hi + beta p with c = <r_hi,p>/|r_hi|^2.
        const double rr = sums[0];
        st->hi_rr = rr;
        const double beta = st->rr_prev > 0.0 ? rr / st->rr_prev : 0.0;
        double cr = 0.0, ci = 0.0;
        if (st->reproject && rr > 0.0) {
            cr = sums[1] / rr;
            ci = sums[2] / rr;
        }
        st->proj_re = cr;
        st->proj_im = ci;
        st->beta = beta;
        st->coef_re = 1.0 - beta * cr;
        st->coef_im = -beta * ci;
        st->rr = rr;
        st->rr_max = rr;
        st->reason = REASON_NONE;
        st->active = 1;
        if (!isfinite(rr)) stop_iterating(st, REASON_BREAKDOWN);
    }
}

}  // namespace hisq
