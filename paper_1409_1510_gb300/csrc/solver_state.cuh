// Device-resident per-bundle solver state and the scalar steps ("hooks") that the last block of
// a reducing kernel runs once the bundle-wide dot products are complete.
#pragma once
#include "hisq_internal.cuh"

namespace hisq {

enum RhsStatus { RHS_RUNNING = 0, RHS_CONVERGED = 1, RHS_NOT_CONVERGED = 2, RHS_BREAKDOWN = 3 };

enum Hook {
    HOOK_NONE = 0,
    HOOK_INIT = 1,      // dots = |b|^2: set up norms and masks
    HOOK_ALPHA = 2,     // dots = <p, A p>: alpha = rr / pAp          (plain CG)
    HOOK_DECIDE = 3,    // dots = |r|^2 after the update: beta or reliable update
    HOOK_RELIABLE = 4,  // dots = |b - A x_hi|^2 (FP64): convergence, restart of r
    HOOK_LOOP = 5,      // (unused: HOOK_DECIDE and HOOK_RELIABLE set the loop condition)
    HOOK_FCG_ALPHA = 6, // dots = <p, A p>; with <p, r> from HOOK_FCG_PR: alpha for flexible CG
    HOOK_FCG_BETA = 7,  // dots = <r - r_old, z> (complex): beta for flexible CG
    HOOK_FCG_PR = 8,    // dots = <p, r> (complex) of the new direction
    HOOK_CG1 = 9,       // dots = |r|^2 (n), then Re<r, A r> (n): one-reduction CG step
};

struct SolverState {
    double rr[HISQ_MAX_BUNDLE];       // |r|^2 of the iterated residual
    double rr_prev[HISQ_MAX_BUNDLE];  // |r|^2 one iteration earlier
    double alpha[HISQ_MAX_BUNDLE][2]; // complex (imaginary part 0 for plain CG)
    double beta[HISQ_MAX_BUNDLE][2];
    double rp_old[HISQ_MAX_BUNDLE][2];// flexible CG: <r_{k-1}, p_{k-1}>
    double pr[HISQ_MAX_BUNDLE][2];    // flexible CG: <p_k, r_k>
    double r_upd[HISQ_MAX_BUNDLE];    // |r| at the last FP64 residual recomputation
    double r_win[HISQ_MAX_BUNDLE];    // flexible CG: |r| at the start of the stall window
    double bnorm[HISQ_MAX_BUNDLE];
    double true_res[HISQ_MAX_BUNDLE]; // last FP64 relative true residual
    int active[HISQ_MAX_BUNDLE];      // 1 while iterating
    int update[HISQ_MAX_BUNDLE];      // 1 when an FP64 residual recomputation is due
    int iters[HISQ_MAX_BUNDLE];
    int updates[HISQ_MAX_BUNDLE];
    int status[HISQ_MAX_BUNDLE];
    int win_start[HISQ_MAX_BUNDLE];   // flexible CG: iteration where the stall window began
    int fallback[HISQ_MAX_BUNDLE];    // flexible CG: 1 once switched to plain CG
    int restart[HISQ_MAX_BUNDLE];     // flexible CG: next direction starts afresh (beta = 0)
    int fallbacks;
    int any_update;
    int update_rounds;                // iterations that ran the FP64 residual recomputation
    int any_active;
    int bundle_iters;
    int n;
    int max_iter;
    int inner_fp64;                   // 1: iterated residual is FP64 (update only at tol)
    int use_pc;
    int stall_window;
    double stall_factor;
    double tol;
    double delta;
    unsigned long long h_loop;        // conditional handles (0 when not in a graph)
    unsigned long long h_upd;
    int cond_loop;                    // last value given to each handle (the graph assigns the
    int cond_upd;                     // defaults 1 and 0 at every launch)
    int cg1;                          // 1: single-reduction CG (HOOK_CG1 drives the iteration)
};
static_assert(sizeof(SolverState) % sizeof(uint32_t) == 0, "the state is copied as 32-bit words");

// Sets a graph condition only when its value changes (the call is not free and most iterations
// leave both conditions as they are).
__device__ __forceinline__ void set_condition(unsigned long long handle, int *last, unsigned int value) {
    if (handle && (unsigned int)*last != value) {
        cudaGraphSetConditional((cudaGraphConditionalHandle)handle, value);
        *last = (int)value;
    }
}

// Scalar step of the solver for one bundle.  Called by thread 0 of the last block of a reducing
// kernel after the bundle-wide dots are final (dots[k] for right-hand side k; complex dots use
// dots[2k], dots[2k+1]; HOOK_FCG_BETA has a second array of n complex dots after the first).
__device__ __forceinline__ void run_hook(int hook, SolverState *st, const double *dots, int n) {
    switch (hook) {
    case HOOK_INIT: {
        int any = 0;
        for (int k = 0; k < n; k++) {
            double b2 = dots[k];
            st->bnorm[k] = sqrt(b2);
            st->rr[k] = b2;
            st->rr_prev[k] = b2;
            st->r_upd[k] = sqrt(b2);
            st->r_win[k] = sqrt(b2);
            st->win_start[k] = 0;
            st->fallback[k] = 0;
            st->restart[k] = 1;
            st->iters[k] = 0;
            st->updates[k] = 0;
            st->update[k] = 0;
            st->alpha[k][0] = st->alpha[k][1] = 0.0;
            st->beta[k][0] = st->beta[k][1] = 0.0;
            st->rp_old[k][0] = 1.0; st->rp_old[k][1] = 0.0;
            bool ok = isfinite(b2);
            st->active[k] = (ok && b2 > 0.0) ? 1 : 0;
            st->status[k] = !ok ? RHS_BREAKDOWN : (b2 > 0.0 ? RHS_RUNNING : RHS_CONVERGED);
            st->true_res[k] = (b2 > 0.0 || !ok) ? 1.0 : 0.0;
            any |= st->active[k];
        }
        for (int k = n; k < HISQ_MAX_BUNDLE; k++) { st->active[k] = 0; st->update[k] = 0; }
        st->fallbacks = 0;
        st->update_rounds = 0;
        st->any_active = any;
        st->any_update = 0;
        st->bundle_iters = 0;
        break;
    }
    case HOOK_ALPHA: {
        for (int k = 0; k < n; k++) {
            if (!st->active[k]) continue;
            double pap = dots[k];
            if (!(pap > 0.0) || !isfinite(pap)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                st->alpha[k][0] = 0.0;
                continue;
            }
            st->alpha[k][0] = st->rr[k] / pap;
            st->alpha[k][1] = 0.0;
        }
        break;
    }
    case HOOK_FCG_ALPHA: {
        // dots[k] = <p, A p>; alpha = <p, r> / <p, A p> (complex); <r, p> kept for the next beta
        for (int k = 0; k < n; k++) {
            if (!st->active[k]) continue;
            double pap = dots[k];
            double pr_re = st->pr[k][0], pr_im = st->pr[k][1];
            if (!(pap > 0.0) || !isfinite(pap) || !isfinite(pr_re) || !isfinite(pr_im)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                st->alpha[k][0] = st->alpha[k][1] = 0.0;
                continue;
            }
            st->alpha[k][0] = pr_re / pap;
            st->alpha[k][1] = pr_im / pap;
            st->rp_old[k][0] = pr_re;   // <r, p> = conj(<p, r>)
            st->rp_old[k][1] = -pr_im;
        }
        break;
    }
    case HOOK_FCG_PR: {
        for (int k = 0; k < n; k++) {
            st->pr[k][0] = dots[2 * k];
            st->pr[k][1] = dots[2 * k + 1];
        }
        break;
    }
    case HOOK_FCG_BETA: {
        // beta = <r_k - r_{k-1}, z_k> / <r_{k-1}, p_{k-1}> (Polak-Ribiere form of flexible CG);
        // zero on the first iteration and when the direction restarts (stall fallback)
        for (int k = 0; k < n; k++) {
            if (!st->active[k]) continue;
            if (st->restart[k]) {
                st->beta[k][0] = st->beta[k][1] = 0.0;
                st->restart[k] = 0;
                continue;
            }
            double nr = dots[2 * k], ni = dots[2 * k + 1];
            double dr = st->rp_old[k][0], di = st->rp_old[k][1];
            double den = dr * dr + di * di;
            if (!(den > 0.0) || !isfinite(nr) || !isfinite(ni)) {
                st->beta[k][0] = st->beta[k][1] = 0.0;
                continue;
            }
            st->beta[k][0] = (nr * dr + ni * di) / den;
            st->beta[k][1] = (ni * dr - nr * di) / den;
        }
        break;
    }
    case HOOK_CG1: {
        // Chronopoulos & Gear (1989): with gamma = |r_k|^2 and delta = <r_k, A r_k> from one
        // reduction, beta = gamma / gamma_prev and alpha = gamma / (delta - beta gamma / alpha_prev)
        // (= gamma / <p_k, A p_k>); the update phase then forms p = r + beta p, q = A r + beta q
        // (= A p), x += alpha p, r -= alpha q.  The FP64 recomputation decision is taken on
        // gamma (the residual of the current iterate) and runs after that update.
        int any = 0;
        for (int k = 0; k < n; k++) {
            st->update[k] = 0;
            if (!st->active[k]) continue;
            const double g = dots[k], d = dots[n + k];
            if (!isfinite(g) || !isfinite(d)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                continue;
            }
            double beta = 0.0;
            if (st->restart[k]) st->restart[k] = 0;
            else beta = g / st->rr[k];
            double den = beta == 0.0 ? d : d - beta * g / st->alpha[k][0];
            if (!(den > 0.0) || !isfinite(den)) {
                // <p, A p> from the recurrence lost to rounding (it is a difference): restart the
                // direction, p = r and q = A r, for which it is <r, A r> itself
                beta = 0.0;
                den = d;
            }
            if (!(den > 0.0)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                continue;
            }
            st->beta[k][0] = beta;
            st->beta[k][1] = 0.0;
            st->alpha[k][0] = g / den;
            st->alpha[k][1] = 0.0;
            st->rr_prev[k] = st->rr[k];
            st->rr[k] = g;
            st->iters[k] += 1;
            const double rn = sqrt(g);
            const bool at_tol = rn <= st->tol * st->bnorm[k];
            const bool drop = (!st->inner_fp64) && rn < st->delta * st->r_upd[k];
            const bool last = st->iters[k] >= st->max_iter;
            if (at_tol || drop || last) any = 1;
        }
        if (any) {  // bundle-wide, as in HOOK_DECIDE
            for (int k = 0; k < n; k++)
                if (st->active[k]) st->update[k] = 1;
        }
        st->any_update = any;
        st->update_rounds += any;
        int act = 0;
        for (int k = 0; k < n; k++) act |= st->active[k];
        st->any_active = act;
        st->bundle_iters += 1;
        break;
    }
    case HOOK_DECIDE: {
        int any = 0;
        for (int k = 0; k < n; k++) {
            st->update[k] = 0;
            if (!st->active[k]) continue;
            st->iters[k] += 1;
            double rr = dots[k];
            if (!isfinite(rr)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                continue;
            }
            double rn = sqrt(rr);
            bool at_tol = rn <= st->tol * st->bnorm[k];
            bool drop = (!st->inner_fp64) && rn < st->delta * st->r_upd[k];
            bool last = st->iters[k] >= st->max_iter;
            if (at_tol || drop || last) {
                st->update[k] = 1;
                any = 1;
            }
            st->rr_prev[k] = st->rr[k];
            st->beta[k][0] = rr / st->rr[k];
            st->beta[k][1] = 0.0;
            st->rr[k] = rr;
            if (st->use_pc && !st->fallback[k]) {
                // stall detection for flexible CG: the residual must drop by stall_factor
                // within stall_window iterations, else continue as plain CG
                if (rn * st->stall_factor <= st->r_win[k]) {
                    st->r_win[k] = rn;
                    st->win_start[k] = st->iters[k];
                } else if (st->iters[k] - st->win_start[k] >= st->stall_window) {
                    st->fallback[k] = 1;
                    st->restart[k] = 1;
                    st->fallbacks += 1;
                }
            }
        }
        if (any) {
            // bundle-wide recomputation: once one right-hand side needs its FP64 residual, all
            // active ones get it in the same pass.  The FP64 residual Dslash is FP64-arithmetic
            // bound, so a pass for one of n right-hand sides would cost nearly what a pass for
            // all n does; updating together also aligns their later triggers (each restarts its
            // 10x-drop reference here), so a bundle needs about as many passes as one RHS.
            for (int k = 0; k < n; k++)
                if (st->active[k]) st->update[k] = 1;
        }
        st->any_update = any;
        st->update_rounds += any;
        set_condition(st->h_upd, &st->cond_upd, any);
        // end of the iteration's scalar work: count it and decide whether the loop continues
        // (right-hand sides flagged for an update stay active until HOOK_RELIABLE decides)
        int act = 0;
        for (int k = 0; k < n; k++) act |= st->active[k];
        st->any_active = act;
        st->bundle_iters += 1;
        set_condition(st->h_loop, &st->cond_loop, (act && st->bundle_iters < st->max_iter) ? 1u : 0u);
        break;
    }
    case HOOK_RELIABLE: {
        for (int k = 0; k < n; k++) {
            if (!st->update[k]) continue;
            double r2 = dots[k];
            st->updates[k] += 1;
            if (!isfinite(r2)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                continue;
            }
            double rn = sqrt(r2);
            st->true_res[k] = rn / st->bnorm[k];
            if (st->true_res[k] <= st->tol) {
                st->active[k] = 0;
                st->status[k] = RHS_CONVERGED;
            } else if (st->iters[k] >= st->max_iter) {
                st->active[k] = 0;
                st->status[k] = RHS_NOT_CONVERGED;
            } else if (st->cg1) {
                // single-reduction CG: the next step measures |r_true|^2 itself and takes
                // beta = |r_true|^2 / |r_previous|^2 against the gamma kept in rr
                st->r_upd[k] = rn;
            } else {
                // restart the iterated residual from the true one; keep the search direction
                // with beta = |r_true|^2 / |r_previous|^2 (Sleijpen & van der Vorst reliable update)
                st->beta[k][0] = r2 / st->rr_prev[k];
                st->beta[k][1] = 0.0;
                st->rr[k] = r2;
                st->r_upd[k] = rn;
            }
        }
        int act = 0;
        for (int k = 0; k < n; k++) act |= st->active[k];
        st->any_active = act;
        set_condition(st->h_loop, &st->cond_loop, (act && st->bundle_iters < st->max_iter) ? 1u : 0u);
        break;
    }
    default:
        break;
    }
}

}  // namespace hisq
