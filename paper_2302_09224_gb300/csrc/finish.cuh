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

__device__ __forceinline__ void ms_stop(MSState *m, int reason)
{
    m->reason = reason;
    m->active = 0;
}

// Multi-shift finishers (Sec. 3.2; the shifted recurrences of Jegerlehner,
// hep-lat/9612014): r_i = zeta_i r with
//   zeta_i' = zeta_i zeta_i^- a^- / (a b^- (zeta_i^- - zeta_i) + zeta_i^- a^- (1 + s_i a))
//   alpha_i = a zeta_i'/zeta_i,  beta_i = b (zeta_i'/zeta_i)^2.
__device__ __forceinline__ void run_ms_finisher(int fin, const double *sums, MSState *m)
{
    if (fin == FIN_MS_ALPHA) {
        const double pAp = sums[0];
        const double a = m->rr / pAp;
        if (!(pAp > 0.0) || !isfinite(a)) {
            m->alpha = 0.0;
            ms_stop(m, REASON_BREAKDOWN);
            return;
        }
        m->pAp = pAp;
        m->alpha = a;
        for (int i = 0; i < m->nshift; i++) {
            if (!m->live[i]) {
                m->alpha_i[i] = 0.0;
                continue;
            }
            const double z = m->zeta[i], zm = m->zeta_prev[i];
            const double den = a * m->beta_prev * (zm - z) + zm * m->alpha_prev * (1.0 + m->shift[i] * a);
            const double zn = z * zm * m->alpha_prev / den;
            if (!isfinite(zn) || zn == 0.0) {  // the shift has converged beyond representability
                m->live[i] = 0;
                m->frozen_at[i] = m->k;
                m->alpha_i[i] = 0.0;
                continue;
            }
            m->zeta_new[i] = zn;
            m->alpha_i[i] = a * zn / z;
        }
    } else if (fin == FIN_MS_BETA) {
        const double rr_new = sums[0];
        const double b = rr_new / m->rr;
        m->k += 1;
        if (!isfinite(rr_new) || !isfinite(b)) {
            ms_stop(m, REASON_BREAKDOWN);
            return;
        }
        m->beta = b;
        bool all_frozen = true;
        for (int i = 0; i < m->nshift; i++) {
            if (!m->live[i]) continue;
            const double q = m->zeta_new[i] / m->zeta[i];
            m->beta_i[i] = b * q * q;
            m->zeta_prev[i] = m->zeta[i];
            m->zeta[i] = m->zeta_new[i];
            const double zr2 = m->zeta[i] * m->zeta[i] * rr_new;
            m->freeze_next[i] = zr2 <= m->stop2[i];
            if (i > 0 && !m->freeze_next[i]) all_frozen = false;
        }
        if (m->nshift == 1) all_frozen = m->freeze_next[0] != 0;
        m->alpha_prev = m->alpha;
        m->beta_prev = b;
        m->rr_prev = m->rr;
        m->rr = rr_new;
        if (rr_new > m->rr_max) m->rr_max = rr_new;
        if (all_frozen)
            m->pending = REASON_CONVERGED;
        else if (rr_new < m->delta2 * m->rr_max)
            m->pending = REASON_RELIABLE;
    } else if (fin == FIN_MS_APPLY) {
        for (int i = 0; i < m->nshift; i++)
            if (m->live[i] && m->freeze_next[i] && (i > 0 || m->nshift == 1)) {
                m->live[i] = 0;
                m->frozen_at[i] = m->k;
            }
        if (m->pending != REASON_NONE) {
            ms_stop(m, m->pending);
            m->pending = REASON_NONE;
        }
    } else if (fin == FIN_MS_TRUE) {
        m->rr = sums[0];
        m->rr_max = sums[0];
        m->reason = REASON_NONE;
        m->active = isfinite(sums[0]) ? 1 : 0;
        if (!m->active) m->reason = REASON_BREAKDOWN;
    }
}

// sums: the grid totals of the reducing kernel; slot: ring slot of p.
__device__ __forceinline__ void run_finisher(int fin, const double *sums, void *state, int slot)
{
    if (state == nullptr || fin == FIN_NONE || fin == FIN_STORE) return;  // sums stay in RedBuf::result
    if (fin >= FIN_MS_ALPHA) {
        run_ms_finisher(fin, sums, static_cast<MSState *>(state));
        return;
    }
    CGState *st = static_cast<CGState *>(state);
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
        st->apap = sums[1];
        st->alpha = alpha;
        st->alpha_ring[slot] = alpha;
    } else if (fin == FIN_CG_BETA) {
        // sums = {|r_new|^2, Re<r_new, r_old>}; Polak-Ribiere beta (Sec. 3.1
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
        if (st->hist != nullptr && st->k < st->hist_len) st->hist[st->k] = rr_new;
        if (rr_new > st->rr_max) st->rr_max = rr_new;
        bool update;
        if (st->dyn) {
            // error estimate (the Sec. 3 footnote's dynamic choice, after van der
            // Vorst and Ye's residual replacement): the drift of the iterated
            // from the true residual grows by the rounding of this update; act
            // when it crosses sqrt(eps) |r|
            const double rn = sqrt(rr_new), ro = sqrt(st->rr_prev);
            const double dn = st->dyn_d + st->dyn_eps * (rn + fabs(st->alpha) * sqrt(st->apap));
            update = st->dyn_d <= st->dyn_hat * ro && dn > st->dyn_hat * rn && dn > 1.1 * st->dyn_d_init;
            st->dyn_d = dn;
        } else {
            update = rr_new < st->delta2 * st->rr_max;  // |r| < delta max|r| (Sec. 3 footnote)
        }
        if (rr_new <= st->stop2)
            stop_iterating(st, REASON_CONVERGED);
        else if (update)
            stop_iterating(st, REASON_RELIABLE);
    } else if (fin == FIN_CG_TRUE) {
        // sums = {|r_hi|^2, Re<r_hi, p>, Im<r_hi, p>}.  Re-projection (Sec. 3.1
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
        st->dyn_d = st->dyn_d_init = st->dyn_eps * sqrt(rr);
        if (st->hist != nullptr && st->k < st->hist_len) st->hist[st->k] = rr;  // the recomputed residual
        st->reason = REASON_NONE;
        st->active = 1;
        if (!isfinite(rr)) stop_iterating(st, REASON_BREAKDOWN);
    }
}

// Batched solver: the CG finisher for each active right-hand side of a tile
// (stopped right-hand sides keep their state untouched).
__device__ __forceinline__ void run_batch_finisher(int fin, const double *sums, CGState *st, int t0, int T, int slot)
{
    if (st == nullptr) return;
    for (int j = 0; j < T; j++)
        if (st[t0 + j].active) run_finisher(fin, sums + 2 * j, &st[t0 + j], slot);
}

}  // namespace hisq
