// finish.cuh -- the scalar updates that end each phase of a level solve (run
// on one thread once the phase's inner products are reduced).  Shared by the
// per-phase kernels and the persistent level kernels.
//
// The inner products arrive as double-float totals and the recurrence scalars
// are kept and updated as double-float pairs (44-48 significant bits, see
// common.cuh): these updates sit on the critical path of every iteration, and
// on GB300 the FP64 form of the MR-II rotation update took about 3000 cycles
// (1.45 us) per iteration against a few hundred in pairs.  The stopping limit
// is formed once per solve in FP64; totals the host reads (||r||^2, ||g||^2)
// are also kept in FP64.
//
// stopped: 0 running; 1 a stopping rule fired; 2 breakdown, no further step;
//          3 non-finite value; 4 breakdown after deciding a last step
//          (applied by the final phase).
#pragma once

#include <math.h>

#include "common.cuh"

namespace eecmg {

__device__ __forceinline__ DF df_one() { return DF{1.f, 0.f}; }
__device__ __forceinline__ DF df_zero() { return DF{0.f, 0.f}; }

// r = g - H u: ||r||^2, ||g||^2; the stopping limit and the test before
// iteration 1 (Section 2 discrepancy rule and the convergence stop).
__device__ __forceinline__ void fin_resid(Scalars* sc, DF rr2, DF gg2, double conv_tol2,
                                          double disc2, int early = 1) {
    const double rr = df_to_double(rr2), gg = df_to_double(gg2);
    sc->rr = rr;
    sc->gg = gg;
    const double l1 = conv_tol2 * gg;
    const double lim2 = l1 > disc2 ? l1 : disc2;
    sc->lim2 = lim2;
    sc->lim2d = df_from_double(lim2);
    sc->iters = 0;
    sc->loops = 0;
    sc->spec = 0;
    sc->applied = 0;
    // MR-II predicts ||r_k|| (fin_mr_b) only where the discrepancy limit is the one that binds:
    // there the residual stays within a small factor of ||r_0|| and the prediction is accurate
    // to rounding; at a convergence limit far below ||r_0|| it would be all cancellation.
    // early = 0 never checks early, 2 checks before every step (the same result).
    sc->lim2spec = early == 2 ? DF{3.0e38f, 0.f}
                   : (early == 1 && disc2 > 0.0 && disc2 >= l1) ? df_from_double(lim2 * (1.0 + 1.0 / 64.0))
                                                                 : DF{-1.f, 0.f};
    if (!(rr < 1.0e300)) sc->stopped = 3;
    else sc->stopped = (rr <= lim2) ? 1 : 0;
}

// MR-II start: v_1 = H r_0, ||v_1||, phi_1 = <w_1, r_0>, identity rotations.
__device__ __forceinline__ void fin_mr_v1(Scalars* sc, DF vv, DF vr) {
    if (!df_finite(vv)) {
        sc->stopped = 3;
    } else if (!(vv.hi > 0.f)) {
        sc->stopped = 2;  // H r_0 = 0: no step
    } else {
        const DF inv = df_rsqrt(vv);
        sc->nrm = df_mul(vv, inv);
        sc->inv_nrm = inv;
        sc->nrm_prev = df_zero();
        sc->inv_nrm_prev = df_zero();
        sc->phi = df_mul(vr, inv);
        sc->f_scale = inv.hi;
        sc->cs1 = df_one();
        sc->sn1 = df_zero();
        sc->cs2 = df_one();
        sc->sn2 = df_zero();
    }
}

// alpha_k = <H w_k, w_k> from <H w_k, v_k>.
__device__ __forceinline__ void fin_mr_a(Scalars* sc, DF hv) {
    const DF inv = sc->inv_nrm;
    const DF alpha = df_mul(hv, inv);
    sc->alpha = alpha;
    sc->loops += 1;
    // phase B of this iteration: v_{k+1} = H w_k - (alpha/||v_k||) v_k - (||v_k||/||v_{k-1}||) v_{k-1},
    // with both coefficients applied as (hi, lo) pairs
    const DF ca = df_mul(alpha, inv), cb = df_mul(sc->nrm, sc->inv_nrm_prev);
    sc->f_ca = ca.hi;
    sc->f_ca_lo = ca.lo;
    sc->f_cb = cb.hi;
    sc->f_cb_lo = cb.lo;
}

// MR-II phase B of iteration k: rr = ||r_{k-1}||^2 (k >= 2), vv = ||v_{k+1}||^2,
// vr = <v_{k+1}, r_{k-1}>.  Stopping rules, then the Givens rotation of
// column k of the tridiagonal T (||v_k|| above the diagonal, 0 for k = 1;
// alpha_k on it; ||v_{k+1}|| below): apply G_{k-2}, G_{k-1}, form G_k, and
// record the coefficients of step k.
__device__ __forceinline__ void fin_mr_b(Scalars* sc, int k, DF rr, DF vv, DF vr) {
    const bool step = k >= 2;
    sc->spec = 0;
    if (step) {
        if (!df_finite(rr)) {
            sc->stopped = 3;
            sc->rr = df_to_double(rr);
            return;
        }
        if (df_le(rr, sc->lim2d)) {  // stopping rule on ||r_{k-1}||, before iteration k
            sc->stopped = 1;
            sc->rr = df_to_double(rr);
            return;
        }
    }
    if (!df_finite(vv)) {
        sc->stopped = 3;
        if (step) sc->rr = df_to_double(rr);
        return;
    }
    const DF inv_new = vv.hi > 0.f ? df_rsqrt(vv) : df_zero();
    const DF nrm_new = df_mul(vv, inv_new);
    const DF c_new = df_mul(vr, inv_new);
    const DF alpha = sc->alpha;
    const DF cpl = step ? sc->nrm : df_zero();
    const DF e = df_mul(sc->sn2, cpl);
    const DF t = df_mul(sc->cs2, cpl);
    const DF r1 = df_add2(df_mul(sc->cs1, t), df_mul(sc->sn1, alpha));
    const DF a2 = df_sub2(df_mul(sc->cs1, alpha), df_mul(sc->sn1, t));
    const DF rho2 = df_add2(df_mul(a2, a2), vv);  // rho = hypot(a2, ||v_{k+1}||)
    if (!(rho2.hi > 0.f) || !df_finite(rho2)) {
        sc->stopped = rho2.hi > 0.f ? 3 : 2;
        if (step) sc->rr = df_to_double(rr);
        return;
    }
    const DF inv_rho = df_rsqrt(rho2);
    const DF cs = df_mul(a2, inv_rho), sn = df_mul(nrm_new, inv_rho);
    const DF phi = sc->phi;
    const DF tau = df_add2(df_mul(cs, phi), df_mul(sn, c_new));
    sc->phi = df_sub2(df_mul(cs, c_new), df_mul(sn, phi));
    sc->tau = tau;
    sc->dinv = inv_rho;
    const DF dw = df_mul(inv_rho, sc->inv_nrm);
    const DF d1 = df_mul(r1, inv_rho);
    const DF d2 = df_mul(e, inv_rho);
    sc->dw = dw;
    sc->d1 = d1;
    sc->d2 = d2;
    sc->cs2 = sc->cs1;
    sc->sn2 = sc->sn1;
    sc->cs1 = cs;
    sc->sn1 = sn;
    sc->nrm_prev = sc->nrm;
    sc->inv_nrm_prev = sc->inv_nrm;
    sc->nrm = nrm_new;
    sc->inv_nrm = inv_new;
    sc->iters = k;
    sc->f_dw = dw.hi;
    sc->f_d1 = d1.hi;
    sc->f_d2 = d2.hi;
    sc->f_dinv = inv_rho.hi;
    sc->f_tau = tau.hi;
    sc->f_scale = inv_new.hi;
    if (!(nrm_new.hi > 0.f)) sc->stopped = 4;  // Krylov space exhausted: step k is the last
    // Step k moves tau_k out of the residual: ||r_k||^2 = ||r_{k-1}||^2 - tau_k^2 (the Givens
    // rotation is orthogonal).  When this prediction is at or below the limit (with a margin),
    // the kernel applies step k at once and checks ||r_k|| explicitly (fin_mr_check) instead of
    // first spending the convolution of iteration k + 1, whose phase B would find the stop.
    // The step and its check are the same arithmetic either way, so the prediction changes the
    // work done, never the result.
    const DF rprev = step ? rr : df_from_double(sc->rr);  // k = 1: ||r_0||^2
    sc->spec = (sc->stopped == 0 && df_le(df_sub2(rprev, df_mul(tau, tau)), sc->lim2spec)) ? 1 : 0;
    // the FP64 copy for the host last: its conversion is off the coefficients' path
    if (step) sc->rr = df_to_double(rr);
}

// The early check of step k, applied by the phase just ended: ||r_k||^2 against the limit.
// If it does not stop, phase B of iteration k + 1 skips the step it would otherwise apply.
__device__ __forceinline__ void fin_mr_check(Scalars* sc, int k, DF rr) {
    sc->applied = k;
    sc->spec = 0;
    sc->rr = df_to_double(rr);
    if (!df_finite(rr)) sc->stopped = 3;
    else if (df_le(rr, sc->lim2d)) sc->stopped = 1;
}

__device__ __forceinline__ void fin_mr_final(Scalars* sc, DF rr) {
    sc->rr = df_to_double(rr);
    if (!df_finite(rr)) sc->stopped = 3;
}

// CGLS start: s = H^T r, gamma = <s, s>.
__device__ __forceinline__ void fin_cg_s0(Scalars* sc, DF gm) {
    if (!df_finite(gm)) sc->stopped = 3;
    else if (!(gm.hi > 0.f)) sc->stopped = 2;
    else sc->gamma = gm;
}

// CGLS: q = H p, alpha = gamma / <q, q>.
__device__ __forceinline__ void fin_cg_q(Scalars* sc, DF qq) {
    sc->loops += 1;
    if (!df_finite(qq)) {
        sc->stopped = 3;
    } else if (!(qq.hi > 0.f)) {
        sc->stopped = 2;
    } else {
        sc->qq = qq;
        const DF a = df_div(sc->gamma, qq);
        sc->cg_alpha = a;
        sc->f_cg_alpha = a.hi;
        sc->iters += 1;
    }
}

// CGLS: after u += alpha p, r -= alpha q: the stopping rule on the new residual.
__device__ __forceinline__ void fin_cg_step(Scalars* sc, DF rr) {
    if (!df_finite(rr)) sc->stopped = 3;
    else if (df_le(rr, sc->lim2d)) sc->stopped = 1;
    sc->rr = df_to_double(rr);
}

// CGLS: s = H^T r, beta = <s, s> / gamma.
__device__ __forceinline__ void fin_cg_s(Scalars* sc, DF gn) {
    if (!df_finite(gn)) {
        sc->stopped = 3;
        return;
    }
    const DF b = df_div(gn, sc->gamma);
    sc->beta = b;
    sc->f_beta = b.hi;
    sc->gamma = gn;
    if (!(gn.hi > 0.f)) sc->stopped = 2;
}

}  // namespace eecmg
