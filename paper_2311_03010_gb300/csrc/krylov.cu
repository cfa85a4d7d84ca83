// krylov.cu -- elementwise phases of the level smoothers C_l^m (Section 2):
// MR-II (reading of "MR") and CGLS (reading of "CG").
//
// Vectors are FP32; every inner product goes through the deterministic FP64
// grid reduction, and the scalars (alpha, beta, norms, stop flags) are
// decided on the device by the last block, so a whole level runs without a
// host round trip.  Each thread handles 8 elements, strided by the block
// size so that every load and store is coalesced.
#include "launch.hpp"

namespace eecmg {

// MR-II, phase B of iteration k >= 2 (the convolution z = H q_{k-1} and the
// betas came from the previous launch):
//   u += alpha_{k-1} p_{k-1},  r -= alpha_{k-1} q_{k-1}          (step k-1)
//   q_k = z - b1 q_{k-1} - b2 q_{k-2},  p_k = q_{k-1} - b1 p_{k-1} - b2 p_{k-2}
// q_k overwrites q_{k-2} (q2) and p_k overwrites p_{k-2} (p2) in place.
// The last block applies the stopping rules to ||r_{k-1}|| (checked before
// iteration k, as in the oracle), then the breakdown test on <q_k, q_k>,
// and decides alpha_k = <r_{k-1}, q_k> / <q_k, q_k>.
__global__ void __launch_bounds__(NTHREADS)
    k_mr_b(const float* __restrict__ z, const float* __restrict__ q1, float* q2,
           const float* __restrict__ p1, float* p2, float* __restrict__ u, float* __restrict__ r,
           size_t n, int has2, Scalars* sc, double* partials) {
    if (*(volatile int*)&sc->stopped) return;
    const float a = (float)sc->alpha;
    const float b1 = (float)sc->b1;
    const float b2 = has2 ? (float)sc->b2 : 0.f;
    float arq = 0.f, aqq = 0.f, arr = 0.f;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * NTHREADS;
        if (i < n) {
            const float q1v = q1[i], p1v = p1[i];
            const float rv = fmaf(-a, q1v, r[i]);
            u[i] = fmaf(a, p1v, u[i]);
            r[i] = rv;
            float qk = fmaf(-b1, q1v, z[i]);
            float pk = fmaf(-b1, p1v, q1v);
            if (has2) {
                qk = fmaf(-b2, q2[i], qk);
                pk = fmaf(-b2, p2[i], pk);
            }
            q2[i] = qk;
            p2[i] = pk;
            arq = fmaf(rv, qk, arq);
            aqq = fmaf(qk, qk, aqq);
            arr = fmaf(rv, rv, arr);
        }
    }
    double v[3] = {(double)arq, (double)aqq, (double)arr};
    if (!block_partials_arrive<3>(v, partials, &sc->counter, gridDim.x, blockIdx.x)) return;
    double tot[3];
    grid_total<3>(partials, gridDim.x, &sc->counter, tot);
    if (threadIdx.x != 0) return;
    const double rr = tot[2], qq = tot[1];
    sc->rr = rr;
    if (!(rr < 1.0e300)) {
        sc->stopped = 3;
    } else if (rr <= sc->lim2) {
        sc->stopped = 1;
    } else if (!(qq < 1.0e300)) {
        sc->stopped = 3;
    } else if (!(qq > 0.0)) {
        sc->stopped = 2;
    } else {
        sc->rq = tot[0];
        sc->alpha = tot[0] / qq;
        sc->qq_prev = sc->qq;
        sc->qq = qq;
        sc->iters += 1;
    }
}

// u += alpha p, r -= alpha q, and ||r||^2.  check = 1: apply the stopping
// rule to the new residual (CGLS, before its next iteration).
__global__ void __launch_bounds__(NTHREADS)
    k_step(float* __restrict__ u, const float* __restrict__ p, float* __restrict__ r,
           const float* __restrict__ q, size_t n, int check, Scalars* sc, double* partials) {
    if (*(volatile int*)&sc->stopped) return;
    const float a = (float)sc->alpha;
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
    sc->rr = tot[0];
    if (!(tot[0] < 1.0e300)) sc->stopped = 3;
    else if (check && tot[0] <= sc->lim2) sc->stopped = 1;
}

// CGLS direction update p = s + beta p (beta decided by the H^T launch).
__global__ void __launch_bounds__(NTHREADS)
    k_cg_p(float* __restrict__ p, const float* __restrict__ s, size_t n, Scalars* sc) {
    if (*(volatile int*)&sc->stopped) return;
    const float b = (float)sc->b1;
    const size_t base = (size_t)blockIdx.x * EW_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * NTHREADS;
        if (i < n) p[i] = fmaf(b, p[i], s[i]);
    }
}

cudaError_t launch_mr_b(const float* z, const float* q1, float* q2, const float* p1, float* p2,
                        float* u, float* r, size_t n, int has2, Scalars* sc, double* partials,
                        cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_mr_b<<<ew_blocks(n), NTHREADS, 0, s>>>(z, q1, q2, p1, p2, u, r, n, has2, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_step(float* u, const float* p, float* r, const float* q, size_t n, int check,
                        Scalars* sc, double* partials, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_step<<<ew_blocks(n), NTHREADS, 0, s>>>(u, p, r, q, n, check, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_p(float* p, const float* sv, size_t n, Scalars* sc, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_cg_p<<<ew_blocks(n), NTHREADS, 0, s>>>(p, sv, n, sc);
    return cudaGetLastError();
}

}  // namespace eecmg
