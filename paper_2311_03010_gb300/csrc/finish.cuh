// finish.cuh -- the FP64 scalar updates that end each phase of a level solve
// (run on one thread once the phase's inner products are reduced).  Shared
// by the per-phase kernels and the persistent level kernels.
//
// stopped: 0 running; 1 a stopping rule fired; 2 breakdown, no further step;
//          3 non-finite value; 4 breakdown after deciding a last step
//          (applied by the final phase).
#pragma once

#include <math.h>

#include "common.cuh"

namespace eecmg {

// r = g - H u: ||r||^2, ||g||^2; the stopping limit and the test before
// iteration 1 (Section 2 discrepancy rule and the convergence stop).
__device__ __forceinline__ void fin_resid(Scalars* sc, double rr, double gg, double conv_tol2,
                                          double disc2) {
    sc->rr = rr;
    sc->gg = gg;
    const double l1 = conv_tol2 * gg;
    sc->lim2 = l1 > disc2 ? l1 : disc2;
    sc->iters = 0;
    sc->loops = 0;
    if (!(rr < 1.0e300)) sc->stopped = 3;
    else sc->stopped = (rr <= sc->lim2) ? 1 : 0;
}

// MR-II start: v_1 = H r_0, ||v_1||, phi_1 = <w_1, r_0>, identity rotations.
__device__ __forceinline__ void fin_mr_v1(Scalars* sc, double vv, double vr) {
    if (!(vv < 1.0e300)) {
        sc->stopped = 3;
    } else if (!(vv > 0.0)) {
        sc->stopped = 2;  // H r_0 = 0: no step
    } else {
        const double inv = rsqrt(vv);
        sc->nrm = vv * inv;
        sc->inv_nrm = inv;
        sc->nrm_prev = 0.0;
        sc->inv_nrm_prev = 0.0;
        sc->phi = vr * inv;
        sc->f_scale = (float)inv;
        sc->cs1 = 1.0;
        sc->sn1 = 0.0;
        sc->cs2 = 1.0;
        sc->sn2 = 0.0;
    }
}

// alpha_k = <H w_k, w_k> from <H w_k, v_k>.
__device__ __forceinline__ void fin_mr_a(Scalars* sc, double hv) {
    const double inv = sc->inv_nrm;
    const double alpha = hv * inv;
    sc->alpha = alpha;
    sc->loops += 1;
    // phase B of this iteration: v_{k+1} = H w_k - (alpha/||v_k||) v_k - (||v_k||/||v_{k-1}||) v_{k-1}
    // double-float (hi + lo) coefficients for the Lanczos update of phase B
    const double ca = alpha * inv, cb = sc->nrm * sc->inv_nrm_prev;
    sc->f_ca = (float)ca;
    sc->f_ca_lo = (float)(ca - (double)sc->f_ca);
    sc->f_cb = (float)cb;
    sc->f_cb_lo = (float)(cb - (double)sc->f_cb);
}

// MR-II phase B of iteration k: rr = ||r_{k-1}||^2 (k >= 2), vv = ||v_{k+1}||^2,
// vr = <v_{k+1}, r_{k-1}>.  Stopping rules, then the Givens rotation of
// column k of the tridiagonal T (||v_k|| above the diagonal, 0 for k = 1;
// alpha_k on it; ||v_{k+1}|| below): apply G_{k-2}, G_{k-1}, form G_k, and
// record the coefficients of step k.
__device__ __forceinline__ void fin_mr_b(Scalars* sc, int k, double rr, double vv, double vr) {
    const bool step = k >= 2;
    if (step) {
        sc->rr = rr;
        if (!(rr < 1.0e300)) {
            sc->stopped = 3;
            return;
        }
        if (rr <= sc->lim2) {  // stopping rule on ||r_{k-1}||, before iteration k
            sc->stopped = 1;
            return;
        }
    }
    if (!(vv < 1.0e300)) {
        sc->stopped = 3;
        return;
    }
    const double inv_new = vv > 0.0 ? rsqrt(vv) : 0.0;
    const double nrm_new = vv * inv_new;
    const double c_new = vr * inv_new;
    const double alpha = sc->alpha;
    const double cpl = step ? sc->nrm : 0.0;
    const double e = sc->sn2 * cpl;
    const double t = sc->cs2 * cpl;
    const double r1 = sc->cs1 * t + sc->sn1 * alpha;
    const double a2 = -sc->sn1 * t + sc->cs1 * alpha;
    const double rho2 = a2 * a2 + vv;  // rho = hypot(a2, ||v_{k+1}||)
    if (!(rho2 > 0.0) || !(rho2 < 1.0e300)) {
        sc->stopped = rho2 > 0.0 ? 3 : 2;
        return;
    }
    const double inv_rho = rsqrt(rho2);
    const double cs = a2 * inv_rho, sn = nrm_new * inv_rho;
    const double phi = sc->phi;
    sc->tau = cs * phi + sn * c_new;
    sc->phi = -sn * phi + cs * c_new;
    sc->dinv = inv_rho;
    sc->dw = inv_rho * sc->inv_nrm;
    sc->d1 = r1 * inv_rho;
    sc->d2 = e * inv_rho;
    sc->cs2 = sc->cs1;
    sc->sn2 = sc->sn1;
    sc->cs1 = cs;
    sc->sn1 = sn;
    sc->nrm_prev = sc->nrm;
    sc->inv_nrm_prev = sc->inv_nrm;
    sc->nrm = nrm_new;
    sc->inv_nrm = inv_new;
    sc->iters = k;
    sc->f_dw = (float)sc->dw;
    sc->f_d1 = (float)sc->d1;
    sc->f_d2 = (float)sc->d2;
    sc->f_dinv = (float)inv_rho;
    sc->f_tau = (float)sc->tau;
    sc->f_scale = (float)inv_new;
    if (!(nrm_new > 0.0)) sc->stopped = 4;  // Krylov space exhausted: step k is the last
}

__device__ __forceinline__ void fin_mr_final(Scalars* sc, double rr) {
    sc->rr = rr;
    if (!(rr < 1.0e300)) sc->stopped = 3;
}

// CGLS start: s = H^T r, gamma = <s, s>.
__device__ __forceinline__ void fin_cg_s0(Scalars* sc, double gm) {
    if (!(gm < 1.0e300)) sc->stopped = 3;
    else if (!(gm > 0.0)) sc->stopped = 2;
    else sc->gamma = gm;
}

// CGLS: q = H p, alpha = gamma / <q, q>.
__device__ __forceinline__ void fin_cg_q(Scalars* sc, double qq) {
    sc->loops += 1;
    if (!(qq < 1.0e300)) {
        sc->stopped = 3;
    } else if (!(qq > 0.0)) {
        sc->stopped = 2;
    } else {
        sc->qq = qq;
        sc->cg_alpha = sc->gamma / qq;
        sc->f_cg_alpha = (float)sc->cg_alpha;
        sc->iters += 1;
    }
}

// CGLS: after u += alpha p, r -= alpha q: the stopping rule on the new residual.
__device__ __forceinline__ void fin_cg_step(Scalars* sc, double rr) {
    sc->rr = rr;
    if (!(rr < 1.0e300)) sc->stopped = 3;
    else if (rr <= sc->lim2) sc->stopped = 1;
}

// CGLS: s = H^T r, beta = <s, s> / gamma.
__device__ __forceinline__ void fin_cg_s(Scalars* sc, double gn) {
    sc->beta = gn / sc->gamma;
    sc->f_beta = (float)sc->beta;
    sc->gamma = gn;
    if (!(gn < 1.0e300)) sc->stopped = 3;
    else if (!(gn > 0.0)) sc->stopped = 2;
}

}  // namespace eecmg
