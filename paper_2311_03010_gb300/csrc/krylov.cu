// krylov.cu -- elementwise phases of the level smoothers C_l^m (Section 2):
// MR-II (reading of "MR") and CGLS (reading of "CG").
//
// MR-II is run in its Lanczos / Givens form: the Lanczos process on the
// symmetric H_l started from H r_0 builds an orthonormal basis w_1..w_k of
// K_k(H, H r_0) with H W_k = W_{k+1} T_k (T_k tridiagonal), and the iterate
// u_k = u_0 + W_k y_k minimises ||r_0 - W_{k+1} T_k y|| + const, a small
// least-squares problem with right-hand side c_j = <w_j, r_0> solved by
// progressive Givens rotations (as in MINRES).  In exact arithmetic these are
// the iterates of the three-term MR-II recurrence; in FP32 this form keeps
// the iterates far closer to the FP64 ones.  The residual r_k = r_0 - H(u_k -
// u_0) is carried through H d_j (from the stored H w_j) for the stopping
// rules, exactly as the recurrence residual.
//
// The projection c_{k+1} = <w_{k+1}, r_0> is taken as <w_{k+1}, r_{k-1}>:
// r_0 - r_{k-1} = H (u_{k-1} - u_0) lies in H span(W_{k-1}) = span(W_k),
// which is orthogonal to w_{k+1}, so the two are equal in exact arithmetic.
// In FP32 the Lanczos vectors lose orthogonality to w_1, which carries the
// large first coefficient; against the small current residual that loss no
// longer sets a residual floor above the convergence threshold.
//
// Vectors are FP32; every inner product goes through the deterministic FP64
// grid reduction, and all scalars (Lanczos coefficients, rotations, stop
// flags) are decided on the device by the last block.  Each thread handles
// 8 elements strided by the block size, so loads and stores are coalesced.
#include <math.h>

#include "finish.cuh"
#include "launch.hpp"

namespace eecmg {

// Applies step j: d_j, H d_j, u += tau d_j, r -= tau H d_j; returns r_i.
__device__ __forceinline__ float mr_apply_step(const MrVecs& V, int j, size_t i, float dw,
                                               float d1, float d2, float dinv, float tau) {
    const int sj = j & 1, sj1 = sj ^ 1;  // d_{j-1} lives in slot (j-1)&1, d_{j-2} in slot j&1
    float dj = dw * V.v[sj][i];
    float hj = dinv * V.aw[sj][i];
    if (j >= 2) {
        dj = fmaf(-d1, V.d[sj1][i], dj);
        hj = fmaf(-d1, V.hd[sj1][i], hj);
    }
    if (j >= 3) {
        dj = fmaf(-d2, V.d[sj][i], dj);
        hj = fmaf(-d2, V.hd[sj][i], hj);
    }
    V.d[sj][i] = dj;
    V.hd[sj][i] = hj;
    V.u[i] = fmaf(tau, dj, V.u[i]);
    const float rv = fmaf(-tau, hj, V.r[i]);
    V.r[i] = rv;
    return rv;
}

// Phase B of iteration k (see launch.hpp).  The dot for c_{k+1} uses the
// residual after the pending step k-1 (r_{k-1}; r_0 when k = 1).
__global__ void __launch_bounds__(NTHREADS)
    k_mr_b(MrVecs V, int k, size_t n, Scalars* sc, double* partials) {
    if (*(volatile int*)&sc->stopped) return;
    const bool step = k >= 2;  // step k-1 is pending
    const float dw = sc->f_dw, d1 = sc->f_d1, d2 = sc->f_d2, dinv = sc->f_dinv, tau = sc->f_tau;
    const float ca = sc->f_ca, ca_lo = sc->f_ca_lo;  // alpha_k / ||v_k||, double-float
    const float cb = step ? sc->f_cb : 0.f;          // ||v_k|| / ||v_{k-1}||
    const float cb_lo = step ? sc->f_cb_lo : 0.f;
    const int sk = k & 1, sk1 = sk ^ 1;
    float arr = 0.f, avv = 0.f, avr = 0.f;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const size_t i = base + (size_t)jj * NTHREADS;
        if (i < n) {
            if (step) {
                const float rv = mr_apply_step(V, k - 1, i, dw, d1, d2, dinv, tau);
                arr = fmaf(rv, rv, arr);
            }
            // v_{k+1} = H w_k - alpha_k w_k - ||v_k|| w_{k-1}
            const float vk = V.v[sk][i];
            float vn = fmaf(-ca_lo, vk, fmaf(-ca, vk, V.aw[sk][i]));
            if (step) {
                const float vk1 = V.v[sk1][i];
                vn = fmaf(-cb_lo, vk1, fmaf(-cb, vk1, vn));
            }
            V.v[sk1][i] = vn;
            avv = fmaf(vn, vn, avv);
            avr = fmaf(vn, V.r[i], avr);
        }
    }
    double vals[3] = {(double)arr, (double)avv, (double)avr};
    if (!block_partials_arrive<3>(vals, partials, &sc->counter, gridDim.x, blockIdx.x)) return;
    double tot[3];
    grid_total<3>(partials, gridDim.x, &sc->counter, tot);
    if (threadIdx.x != 0) return;
    fin_mr_b(sc, k, df_from_double(tot[0]), df_from_double(tot[1]), df_from_double(tot[2]));
}

// Applies the step decided last (its index is sc->iters) and reduces ||r||^2.
__global__ void __launch_bounds__(NTHREADS)
    k_mr_final(MrVecs V, size_t n, Scalars* sc, double* partials) {
    const int st = *(volatile int*)&sc->stopped;
    if (st != 0 && st != 4) return;
    const int j = sc->iters;
    if (j < 1) return;
    const float dw = sc->f_dw, d1 = sc->f_d1, d2 = sc->f_d2, dinv = sc->f_dinv, tau = sc->f_tau;
    float arr = 0.f;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const size_t i = base + (size_t)jj * NTHREADS;
        if (i < n) {
            const float rv = mr_apply_step(V, j, i, dw, d1, d2, dinv, tau);
            arr = fmaf(rv, rv, arr);
        }
    }
    double vals[1] = {(double)arr};
    if (!block_partials_arrive<1>(vals, partials, &sc->counter, gridDim.x, blockIdx.x)) return;
    double tot[1];
    grid_total<1>(partials, gridDim.x, &sc->counter, tot);
    if (threadIdx.x != 0) return;
    fin_mr_final(sc, df_from_double(tot[0]));
}

// CGLS: u += alpha p, r -= alpha q, ||r||^2, then the stopping rule on the
// new residual (checked before the next iteration, as in the oracle).
__global__ void __launch_bounds__(NTHREADS)
    k_cg_step(float* __restrict__ u, const float* __restrict__ p, float* __restrict__ r,
              const float* __restrict__ q, size_t n, Scalars* sc, double* partials) {
    if (*(volatile int*)&sc->stopped) return;
    const float a = sc->f_cg_alpha;
    float arr = 0.f;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * NTHREADS;
        if (i < n) {
            u[i] = fmaf(a, p[i], u[i]);
            const float rv = fmaf(-a, q[i], r[i]);
            r[i] = rv;
            arr = fmaf(rv, rv, arr);
        }
    }
    double v[1] = {(double)arr};
    if (!block_partials_arrive<1>(v, partials, &sc->counter, gridDim.x, blockIdx.x)) return;
    double tot[1];
    grid_total<1>(partials, gridDim.x, &sc->counter, tot);
    if (threadIdx.x != 0) return;
    fin_cg_step(sc, df_from_double(tot[0]));
}

// CGLS direction update p = s + beta p (beta decided by the H^T launch).
__global__ void __launch_bounds__(NTHREADS)
    k_cg_p(float* __restrict__ p, const float* __restrict__ s, size_t n, Scalars* sc) {
    if (*(volatile int*)&sc->stopped) return;
    const float b = sc->f_beta;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * NTHREADS;
        if (i < n) p[i] = fmaf(b, p[i], s[i]);
    }
}

cudaError_t launch_mr_b(const MrVecs& V, int k, size_t n, Scalars* sc, double* partials,
                        cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_mr_b<<<ew_blocks(n), NTHREADS, 0, s>>>(V, k, n, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_mr_final(const MrVecs& V, size_t n, Scalars* sc, double* partials,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_mr_final<<<ew_blocks(n), NTHREADS, 0, s>>>(V, n, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_step(float* u, const float* p, float* r, const float* q, size_t n,
                           Scalars* sc, double* partials, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_cg_step<<<ew_blocks(n), NTHREADS, 0, s>>>(u, p, r, q, n, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_p(float* p, const float* sv, size_t n, Scalars* sc, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_cg_p<<<ew_blocks(n), NTHREADS, 0, s>>>(p, sv, n, sc);
    return cudaGetLastError();
}

}  // namespace eecmg
