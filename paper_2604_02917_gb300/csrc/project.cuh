// Block-cooperative exact projection onto F = {mu^T x >= R, 1^T x = 1, x >= 0}
// (Sec. 3.1, Eqs. simplex-tau, simplex-proj, projF-dualpath), FP64.
//
// One thread block owns one problem.  Every step is one block-wide reduction
// of five FP64 sums over a candidate support S = {i : v_i + nu mu_i > tau}:
//     |S|, sum_S v, sum_S mu, sum_S mu v, sum_S mu^2.
// From these the two scalar searches of the paper are driven:
//
//  * inner (simplex threshold, Eq. simplex-tau): h(tau) = sum max(w - tau, 0) - 1
//    is convex, decreasing and piecewise linear in tau.  A Newton step from
//    any tau lands at or left of the root, and from the left the iterates
//    rise monotonically with nested supports, so the iteration ends exactly
//    when |S| stops changing:  tau = (sum_S w - 1) / |S|.  This replaces the
//    sort of the paper by a few reductions and yields the same threshold.
//
//  * outer (return multiplier, Eq. projF-dualpath): phi(nu) = mu^T x(nu) is
//    continuous, nondecreasing and piecewise linear.  On the support S found
//    at the current nu, the budget and return rows
//        |S| tau - nu sum_S mu = sum_S v - 1
//        sum_S mu tau - nu sum_S mu^2 = sum_S mu v - R
//    give the exact (tau, nu) of that linear piece (a Newton step on phi).
//    The iteration keeps a bracket psi(lo) < 0 <= psi(hi) with psi = phi - R,
//    falls back to the paper's geometric expansion nu = 1, 2, 4, ... and to
//    bisection when the Newton point leaves the bracket, and stops when the
//    support at nu reproduces nu (the exact finish).  When psi(0) >= 0 the
//    return row is inactive and the simplex projection is the answer.
//
// The warm start (nu, tau of the previous call) only changes where the
// search begins, never the point it returns: the projection is unique.
#pragma once

#include "mv_internal.cuh"

namespace mv {

struct ProjSums {
    double cnt, sv, sm, smv, smm;
};

struct ProjOut {
    double nu, tau;
    ProjSums s;
    int status;
    int steps;
};

template <int NT>
struct Projector {
    const double *V;    // n points (shared or global memory)
    const double *MU;   // n expected returns
    int n;
    double *red;        // (NT/32 + 1) * 5 doubles of shared memory
    int steps;

    __device__ __forceinline__ ProjSums support_sums(double nu, double tau) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = threadIdx.x; i < n; i += NT) {
            const double v = V[i], m = MU[i];
            const double w = fma(nu, m, v);
            if (w > tau) {
                acc[0] += 1.0;
                acc[1] += v;
                acc[2] += m;
                acc[3] = fma(m, v, acc[3]);
                acc[4] = fma(m, m, acc[4]);
            } else if (!(w == w)) {
                acc[1] = NAN;                 // poison the sums: reported as MV_ERR_NUMERIC
            }
        }
        block_sum<5, NT>(acc, red);
        ++steps;
        return ProjSums{acc[0], acc[1], acc[2], acc[3], acc[4]};
    }

    // Newton on the simplex threshold at fixed nu.  tau may start anywhere
    // (-inf gives the all-assets start).  Returns false if the budget ran out.
    __device__ bool simplex_tau(double nu, double &tau, ProjSums &s, int budget) {
        if (!(tau == tau)) tau = -INFINITY;
        s = support_sums(nu, tau);
        for (int it = 0; it < budget; ++it) {
            if (s.cnt == 0.0) {          // tau >= max w: restart from the left
                tau = -INFINITY;
                s = support_sums(nu, tau);
                continue;
            }
            const double tn = (fma(nu, s.sm, s.sv) - 1.0) / s.cnt;
            const ProjSums s2 = support_sums(nu, tn);
            const bool same = (s2.cnt == s.cnt);
            tau = tn;
            s = s2;
            if (same) return true;
        }
        return false;
    }

    // Full search.  mode: MV_RETURN_GE or MV_RETURN_EQ.
    __device__ ProjOut solve(double R, int mode, double mu_min, double mu_max,
                             double nu_hint, double tau_hint, int budget) {
        ProjOut o;
        o.steps = 0;
        steps = 0;
        o.status = MV_OK;
        if (!(R <= mu_max) || (mode == MV_RETURN_EQ && !(R >= mu_min))) {
            o.status = MV_ERR_INFEASIBLE;
            o.nu = o.tau = NAN;
            o.s = ProjSums{0, 0, 0, 0, 0};
            return o;
        }
        const double scaleR = fmax(fabs(R), fmax(fabs(mu_max), fabs(mu_min)));
        const bool ge = (mode == MV_RETURN_GE);
        double lo = -INFINITY, hi = INFINITY;   // psi(lo) < 0 <= psi(hi)
        bool have_lo = false, have_hi = false, zero_done = false;
        double nu = (nu_hint == nu_hint) ? nu_hint : 0.0;
        if (ge && !(nu > 0.0)) nu = 0.0;
        double tau = tau_hint;
        ProjSums s;
        for (int it = 0; it < budget; ++it) {
            if (!simplex_tau(nu, tau, s, 96)) {
                o.status = MV_ERR_NOT_CONVERGED;
                break;
            }
            if (!(tau == tau) || !isfinite(s.sv) || !isfinite(s.smv)) {
                o.status = MV_ERR_NUMERIC;
                break;
            }
            if (nu == 0.0) zero_done = true;
            const double a = s.cnt, b = s.sm, c = s.smm;
            const double det = a * c - b * b;            // |S| sum_S (mu - mean)^2
            const bool flat = !(det > 1e-13 * a * c);    // mu constant on S
            double psi;
            if (flat) {
                psi = b / a - R;                         // phi = mean of mu on S
            } else {
                psi = (fma(nu, c, s.smv) - tau * b) - R;
            }
            if (ge && nu == 0.0 && psi >= 0.0) break;    // return row inactive
            if (psi == 0.0) break;
            double nu_c = NAN;
            if (flat) {
                if (fabs(psi) <= 1e-12 * scaleR) break;  // target met on a flat piece
            } else {
                const double d1 = s.sv - 1.0, d2 = s.smv - R;
                nu_c = (b * d1 - a * d2) / det;
                if (fabs(nu_c - nu) <= 1e-13 * fmax(1.0, fabs(nu))) break;   // exact finish
            }
            if (psi < 0.0) {
                lo = nu;
                have_lo = true;
            } else {
                hi = nu;
                have_hi = true;
            }
            double nxt = nu_c;
            if (ge && nxt == nxt && nxt <= 0.0 && !zero_done) nxt = 0.0;
            const bool inside = (nxt == nxt) && (!have_lo || nxt > lo) && (!have_hi || nxt < hi) &&
                                (!ge || nxt >= 0.0);
            if (!inside) {
                if (have_lo && have_hi) {
                    nxt = 0.5 * (lo + hi);
                } else if (have_lo) {                    // expand right: 1, 2, 4, ...
                    nxt = (lo < 0.0) ? 0.0 : (lo == 0.0 ? 1.0 : 2.0 * lo);
                    if (nxt == 0.0 && zero_done) nxt = 1.0;
                } else {                                 // expand left (EQ) or test nu = 0 (GE)
                    if (ge) {
                        nxt = 0.0;
                    } else {
                        nxt = (hi > 0.0) ? 0.0 : (hi == 0.0 ? -1.0 : 2.0 * hi);
                        if (nxt == 0.0 && zero_done) nxt = -1.0;
                    }
                }
            }
            if (nxt == nu) {                             // bracket exhausted in FP64
                o.status = MV_ERR_NOT_CONVERGED;
                break;
            }
            // Start the inner search from the threshold this support predicts.
            tau = (fma(nxt, b, s.sv) - 1.0) / a;
            nu = nxt;
            if (it == budget - 1) o.status = MV_ERR_NOT_CONVERGED;
        }
        o.nu = nu;
        o.tau = tau;
        o.s = s;
        o.steps = steps;
        return o;
    }
};

}  // namespace mv
