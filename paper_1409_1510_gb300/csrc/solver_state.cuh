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
    HOOK_CG1 = 9,       // dots = <p, A p>, |r|^2, |A p|^2 (n each): one-reduction CG step
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
    double tolk[HISQ_MAX_BUNDLE];     // relative tolerance of each right-hand side
    double mass2[HISQ_MAX_BUNDLE];    // m^2 of each right-hand side's operator m^2 - D_eo D_oe
                                      // (one value for a plain solve; the persistent driver also
                                      // solves bundles of shifted systems)
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
    double delta;
    unsigned long long h_loop;        // conditional handles (0 when not in a graph)
    unsigned long long h_upd;
    int cond_loop;                    // last value given to each handle (the graph assigns the
    int cond_upd;                     // defaults 1 and 0 at every launch)
    int pad_;
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
        // Hestenes-Stiefel CG with one reduction per iteration.  The reduction after A p brings
        // <p, A p> and |A p|^2 together with |r|^2, which the previous update phase published
        // (or, right after setup or an FP64 recomputation, the exact value kept in rr): then
        // alpha = |r|^2 / <p, A p> and, since <r, A p> = <p, A p> (A-conjugacy), the next
        // residual norm |r - alpha A p|^2 = alpha^2 |A p|^2 - |r|^2 gives beta and the
        // reliable-update decision before the update phase, which then also forms p = r + beta p.
        // |r|^2 is measured every iteration and A p recomputed, so no rounding accumulates.
        int any = 0;
        for (int k = 0; k < n; k++) {
            const bool exact = st->restart[k] || st->update[k];  // rr holds the measured |r|^2
            st->restart[k] = 0;
            st->update[k] = 0;
            if (!st->active[k]) continue;
            const double pap = dots[k], apap = dots[2 * n + k];
            const double g = exact ? st->rr[k] : dots[n + k];
            if (!(pap > 0.0) || !isfinite(pap) || !isfinite(g) || !isfinite(apap)) {
                st->active[k] = 0;
                st->status[k] = RHS_BREAKDOWN;
                st->alpha[k][0] = 0.0;
                continue;
            }
            // one division and no square root on the critical path (an FP64 division or square
            // root is a long dependent sequence on this part): with q = |A p|^2 / <p, A p>,
            // beta = |r_new|^2 / |r|^2 = alpha^2 |A p|^2 / |r|^2 - 1 = alpha q - 1, and the
            // stopping tests compare squares
            const double inv = 1.0 / pap;
            const double al = g * inv;
            double be = al * (apap * inv) - 1.0;
            if (!(be > 0.0)) be = 0.0;  // cancellation at convergence: the FP64 check decides
            const double gn = be * g;
            st->alpha[k][0] = al;
            st->alpha[k][1] = 0.0;
            st->iters[k] += 1;
            st->rr_prev[k] = g;
            st->beta[k][0] = be;
            st->beta[k][1] = 0.0;
            st->rr[k] = gn;
            const double tb = st->tolk[k] * st->bnorm[k], du = st->delta * st->r_upd[k];
            const bool at_tol = gn <= tb * tb;
            const bool drop = (!st->inner_fp64) && gn < du * du;
            const bool last = st->iters[k] >= st->max_iter;
            if (at_tol || drop || last) {
                st->update[k] = 1;
                any = 1;
            }
        }
        // per right-hand side: the persistent kernel's FP64 passes run over only the right-hand
        // sides that recompute, so a pass costs in proportion to them
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
            bool at_tol = rn <= st->tolk[k] * st->bnorm[k];
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
            if (st->true_res[k] <= st->tolk[k]) {
                st->active[k] = 0;
                st->status[k] = RHS_CONVERGED;
            } else if (st->iters[k] >= st->max_iter) {
                st->active[k] = 0;
                st->status[k] = RHS_NOT_CONVERGED;
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
