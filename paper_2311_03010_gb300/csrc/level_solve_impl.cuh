// level_solve_impl.cuh -- persistent level smoothers C_l^m (Section 2): one
// cooperative launch runs a whole level solve, MR-II (Lanczos / Givens form,
// see krylov.cu) or CGLS.
//
// Every phase of an iteration is a grid-stride pass over the level's tiles
// (convolution phases, 32 x 64 tiles with halo in shared memory) or pixels
// (elementwise phases), ended by a reduction barrier (persistent.cuh): the
// deterministic double-float sums of the phase's inner products and its scalar
// update (finish.cuh), run by every block on its own replica of the scalars.  Compared with one launch per phase this removes the
// launch latency of every phase and, because the loop tests the stop flag,
// the iterations that a stopping rule makes unnecessary are never launched.
// Vectors written inside the launch are read back through L2 (ld.global.cg).
#pragma once

#include <type_traits>

#include "conv_tile.cuh"
#include "finish.cuh"
#include "level_ops.cuh"
#include "level_solve.hpp"
#include "persistent.cuh"

namespace eecmg {


namespace ls_detail {

__device__ __forceinline__ int volatile_stopped(const Scalars* sc) {
    return *(volatile const int*)&sc->stopped;
}

__device__ __forceinline__ float vldf(const float* p) { return *(volatile const float*)p; }

struct StepCoef {
    float dw, d1, d2, dinv, tau;
};

__device__ __forceinline__ StepCoef step_coef(const Scalars* sc) {
    return StepCoef{vldf(&sc->f_dw), vldf(&sc->f_d1), vldf(&sc->f_d2), vldf(&sc->f_dinv),
                    vldf(&sc->f_tau)};
}

// The MR-II vectors of a solve: the directions d as HT (FP32, or BF16 in the
// BF16-storage variant); the Lanczos vectors v, their images H w, the images
// H d, u, r and g stay FP32.  Neither v nor the images can be rounded: the
// Lanczos update v_{k+1} = H w_k - alpha v_k - beta v_{k-1} cancels to a small
// fraction of H w on smooth operators, so a rounding of v_k or H w_k there is
// amplified in v_{k+1}, and H d carries the residual recurrence.
template <typename HT>
struct MrVec {
    float* v[2];
    float* aw[2];
    HT* d[2];
    float* hd[2];
    __device__ __forceinline__ explicit MrVec(const LevelJob& J) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            v[i] = J.v[i];
            aw[i] = J.aw[i];
            d[i] = reinterpret_cast<HT*>(J.d[i]);
            hd[i] = J.hd[i];
        }
    }
};

// MR-II step j on pixels 4q..4q+3 (coherent loads), u alone: u += tau d_j;
// returns the new r without storing it, nor d_j and H d_j.  This is the step
// of an early check or of the solve's end, whose r, d_j and H d_j are dead
// unless the solve goes on (phase B of the next iteration then stores them).
// Every operand is loaded before the store (the stores may alias nothing the
// compiler can see, so a load after a store would wait for it).
template <typename HT>
__device__ __forceinline__ float4 mr_step4_u(const LevelJob& J, const MrVec<HT>& M, int j, size_t q,
                                             const StepCoef& c) {
    using IO = VecIO<HT>;
    const int sj = j & 1, sj1 = sj ^ 1;
    const float4 vj = ld4cg(M.v[sj], q), awj = ld4cg(M.aw[sj], q);
    const float4 uu = ld4cg(J.u, q), rr = ld4cg(J.r, q);
    float4 dA = vj, hA = vj, dB = vj, hB = vj;
    if (j >= 2) {
        dA = IO::ld4(M.d[sj1], q);
        hA = ld4cg(M.hd[sj1], q);
    }
    if (j >= 3) {
        dB = IO::ld4(M.d[sj], q);
        hB = ld4cg(M.hd[sj], q);
    }
    float4 dj = mul4(c.dw, vj);
    float4 hj = mul4(c.dinv, awj);
    if (j >= 2) {
        dj = fma4(-c.d1, dA, dj);
        hj = fma4(-c.d1, hA, hj);
    }
    if (j >= 3) {
        dj = fma4(-c.d2, dB, dj);
        hj = fma4(-c.d2, hB, hj);
    }
    st4(J.u, q, fma4(c.tau, dj, uu));
    return fma4(-c.tau, hj, rr);
}

// Applies MR-II step j at pixel i (coherent loads, all before the stores);
// returns the new r_i.  MODE 0: the whole step; 1: u alone (as mr_step4_u);
// 2: the rest of a step whose u is updated (d_j, H d_j, r).
template <typename HT, int MODE = 0>
__device__ __forceinline__ float mr_step_px(const LevelJob& J, const MrVec<HT>& M, int j, size_t i,
                                            float dw, float d1, float d2, float dinv, float tau) {
    using IO = VecIO<HT>;
    const int sj = j & 1, sj1 = sj ^ 1;
    const float vj = ldcg(M.v[sj] + i), awj = ldcg(M.aw[sj] + i);
    const float uu = MODE == 2 ? 0.f : ldcg(J.u + i), rr = ldcg(J.r + i);
    float dA = 0.f, hA = 0.f, dB = 0.f, hB = 0.f;
    if (j >= 2) {
        dA = IO::ld(M.d[sj1], i);
        hA = ldcg(M.hd[sj1] + i);
    }
    if (j >= 3) {
        dB = IO::ld(M.d[sj], i);
        hB = ldcg(M.hd[sj] + i);
    }
    float dj = dw * vj;
    float hj = dinv * awj;
    if (j >= 2) {
        dj = fmaf(-d1, dA, dj);
        hj = fmaf(-d1, hA, hj);
    }
    if (j >= 3) {
        dj = fmaf(-d2, dB, dj);
        hj = fmaf(-d2, hB, hj);
    }
    const float rv = fmaf(-tau, hj, rr);
    if (MODE != 1) {
        IO::st(M.d[sj], i, dj);
        M.hd[sj][i] = hj;
        J.r[i] = rv;
    }
    if (MODE != 2) J.u[i] = fmaf(tau, dj, uu);
    return rv;
}

// One convolution phase over the level: y = scale * (C (*) x) for every tile,
// with epilogue E(idx, z, center, pre) accumulating into acc0/acc1.  pre is
// the value of the read-only vector `pre` at the pixel (0 if pre is null): its
// loads are issued before the tile is convolved, so their latency overlaps
// the compute (loaded inside the epilogue, each would wait behind the
// epilogue's stores, which the compiler cannot tell apart from it).
template <int R, bool SEP, bool PREC, bool ZERO, typename TIN = float, class Epi>
__device__ __forceinline__ void conv_phase(ConvSmem<R, SEP>& S, const TIN* x, int h, int w,
                                           unsigned int nb, unsigned int bid, const float* pre, Epi&& epi) {
    using SM = ConvSmem<R, SEP>;
    const int tiles_x = (w + CONV_TW - 1) / CONV_TW, tiles_y = (h + CONV_TH - 1) / CONV_TH;
    const int ntiles = tiles_x * tiles_y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // software pipeline: the loads of the block's next tile are issued before the
    // current tile is convolved, so their latency overlaps the compute and the epilogue
    ConvRegs<R, SEP, TIN> V;
    if (!ZERO && (int)bid < ntiles)
        conv_fetch<R, SEP, true, TIN>(V, x, h, w, ((int)bid / tiles_x) * CONV_TH,
                                      ((int)bid % tiles_x) * CONV_TW);
    for (int t = (int)bid; t < ntiles; t += (int)nb) {
        const int y0 = (t / tiles_x) * CONV_TH, x0 = (t % tiles_x) * CONV_TW;
        if (!ZERO) {
            conv_put<R, SEP, TIN>(S, V);
            __syncthreads();
            const int tn = t + (int)nb;
            if (tn < ntiles)
                conv_fetch<R, SEP, true, TIN>(V, x, h, w, (tn / tiles_x) * CONV_TH, (tn % tiles_x) * CONV_TW);
        }
        float pv[CONV_TH / 8][2];
#pragma unroll
        for (int it = 0; it < CONV_TH / 8; ++it)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int gy = y0 + warp + 8 * it, gx = x0 + lane + 32 * hf;
                pv[it][hf] = (pre && gy < h && gx < w) ? __ldg(pre + (size_t)gy * w + gx) : 0.f;
            }
        if (!ZERO) {
            conv_compute<R, SEP, PREC>(S);
            __syncthreads();
        }
#pragma unroll
        for (int it = 0; it < CONV_TH / 8; ++it) {
            const int r = warp + 8 * it, gy = y0 + r;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int c = lane + 32 * hf, gx = x0 + c;
                if (gy < h && gx < w) {
                    const size_t idx = (size_t)gy * w + gx;
                    const float z = ZERO ? 0.f : S.out[r * SM::PO + c];
                    const float ctr = ZERO ? 0.f : S.in[SM::at(r + R, c + R)];
                    epi(idx, z, ctr, pv[it][hf]);
                }
            }
        }
        __syncthreads();  // S is reused by the next tile
    }
}

// Phase 0 of a solve that starts its own level (J.start): u = D(S(P(Pi(u1, u2)))) over the
// level's 32 x 64 tiles, then a barrier (the r_0 phase reads u with its halo).  Returns false
// if the job is in error.
__device__ __forceinline__ bool start_phase(PsdSmem& M, const LevelJob& J, unsigned int nb,
                                            unsigned int bid, LevelSync& sy) {
    const int h = J.h, w = J.w;
    const int tiles_x = (w + PSD_TW - 1) / PSD_TW, ntiles = tiles_x * ((h + PSD_TH - 1) / PSD_TH);
    float* u = J.u;
    for (int t = (int)bid; t < ntiles; t += (int)nb) {
        const int y0 = (t / tiles_x) * PSD_TH, x0 = (t % tiles_x) * PSD_TW;
        tile_psd(M, J.s_u1, J.s_h1, J.s_w1, J.s_u2, J.s_h2, J.s_w2, h, w, J.s_scale, J.s_tau, J.s_ik2,
                 y0, x0, [&](int rr, int cc, float v) { u[(size_t)(y0 + rr) * w + x0 + cc] = v; });
        __syncthreads();
    }
    float v[1] = {0.f};
    return sy.reduce<1>(v, [&](DF*) {});
}

// Algorithmic bytes per pixel of the level's start: the zero start written into u, or the
// fused start reading both coarser solutions and writing u.
__device__ __forceinline__ double start_bytes(const LevelJob& J) {
    if (J.start)
        return 4.0 + 4.0 * ((double)J.s_h1 * J.s_w1 + (double)J.s_h2 * J.s_w2) / ((double)J.h * J.w);
    return J.zero_start ? 4.0 : 0.0;
}

}  // namespace ls_detail

using namespace ls_detail;

template <int R, bool SEP, bool PREC, typename HT>
__device__ __forceinline__ void mr2_body(ConvSmem<R, SEP>& S, PsdSmem& M, const LevelJob& J, Scalars* sc,
                                         unsigned int nb, unsigned int bid, LevelSync& sy) {
    const int h = J.h, w = J.w;
    const size_t n = (size_t)h * w;
    const size_t stride = (size_t)nb * NTHREADS;
    using IO = VecIO<HT>;
    const MrVec<HT> K(J);
    if (J.start && !start_phase(M, J, nb, bid, sy)) return;
    conv_stage_taps<R, SEP>(S, J.taps);
    __syncthreads();

    // r_0 = g - H u_0, ||r_0||^2, ||g||^2, stopping limit (a zero start is written into u here)
    {
        float a0 = 0.f, a1 = 0.f;
        const bool zs = J.zero_start != 0;
        auto epi = [&](size_t idx, float z, float, float gv) {
            const float rv = gv - z;
            J.r[idx] = rv;
            if (zs) J.u[idx] = 0.f;
            a0 = fmaf(rv, rv, a0);
            a1 = fmaf(gv, gv, a1);
        };
        if (zs)
            conv_phase<R, SEP, PREC, true>(S, J.u, h, w, nb, bid, J.g, epi);
        else
            conv_phase<R, SEP, PREC, false>(S, J.u, h, w, nb, bid, J.g, epi);
        float v[2] = {a0, a1};
        const double ct2 = J.conv_tol2, d2 = J.disc2;
        const int ear = J.early;
        const double b0 = (J.zero_start ? 8.0 : 12.0) + start_bytes(J);
        if (!sy.reduce<2>(v, [&](DF* t) {
                fin_resid(sc, t[0], t[1], ct2, d2, ear);
                sc->bpp = b0;
            }))
            return;
    }
    if (J.m <= 0 || volatile_stopped(sc)) return;

    // bytes per pixel of the vector phases (each operand read or written once;
    // d stored as HT, everything else FP32)
    constexpr double E = (double)sizeof(HT);
    auto hist = [](int j) { return (4.0 + E) * ((j >= 2 ? 1 : 0) + (j >= 3 ? 1 : 0)); };

    // v_1 = H r_0, ||v_1||, <v_1, r_0>
    {
        float a0 = 0.f, a1 = 0.f;
        float* v1 = K.v[1];
        conv_phase<R, SEP, PREC, false>(S, J.r, h, w, nb, bid, nullptr, [&](size_t idx, float z, float ctr, float) {
            v1[idx] = z;
            a0 = fmaf(z, z, a0);
            a1 = fmaf(z, ctr, a1);
        });
        float v[2] = {a0, a1};
        if (!sy.reduce<2>(v, [&](DF* t) {
                fin_mr_v1(sc, t[0], t[1]);
                sc->bpp += 8.0;
            }))
            return;
    }

    for (int k = 1; k <= J.m; ++k) {
        if (volatile_stopped(sc)) break;
        const int sk = k & 1, sk1 = sk ^ 1;
        // phase A: H w_k = H v_k / ||v_k||, alpha_k = <H w_k, w_k>
        {
            const float scale = vldf(&sc->f_scale);
            float a0 = 0.f;
            float* aw = K.aw[sk];
            conv_phase<R, SEP, PREC, false>(S, K.v[sk], h, w, nb, bid, nullptr,
                                            [&](size_t idx, float z, float ctr, float) {
                                                const float hz = z * scale;
                                                aw[idx] = hz;
                                                a0 = fmaf(hz, ctr, a0);
                                            });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) {
                    fin_mr_a(sc, t[0]);
                    sc->bpp += 8.0;
                }))
                return;
        }
        // phase B: pending step k-1 (its d, H d and r only, if an early check updated u
        // already), v_{k+1}, stopping rules, rotation of column k
        {
            const bool step = k >= 2;
            const bool apply = step && *(volatile const int*)&sc->applied != k - 1;
            const bool rest = step && !apply;  // the early check of step k-1 did not hold
            const StepCoef c = step_coef(sc);
            // Lanczos coefficients in double-float: the update below cancels
            const float ca = vldf(&sc->f_ca), ca_lo = vldf(&sc->f_ca_lo);
            const float cb = step ? vldf(&sc->f_cb) : 0.f, cb_lo = step ? vldf(&sc->f_cb_lo) : 0.f;
            float arr = 0.f, avv = 0.f, avr = 0.f;
            const size_t n4 = n >> 2;
            const int j = k - 1, sj = j & 1, sj1 = sj ^ 1;  // sj == sk1
            for (size_t q = (size_t)bid * NTHREADS + threadIdx.x; q < n4; q += stride) {
                // every operand is loaded before the first store, so the pass
                // costs one round trip to L2 (the stores alias none of the
                // loads except the same elements, already read)
                const float4 vk = ld4cg(K.v[sk], q), awk = ld4cg(K.aw[sk], q);
                const float4 rr = ld4cg(J.r, q);
                float4 vj = make_float4(0.f, 0.f, 0.f, 0.f), awj = vj, uu = vj;
                float4 dA = vj, hA = vj, dB = vj, hB = vj;
                if (step) vj = ld4cg(K.v[sj], q);
                if (step) {
                    awj = ld4cg(K.aw[sj], q);
                    if (apply) uu = ld4cg(J.u, q);
                    if (j >= 2) {
                        dA = IO::ld4(K.d[sj1], q);
                        hA = ld4cg(K.hd[sj1], q);
                    }
                    if (j >= 3) {
                        dB = IO::ld4(K.d[sj], q);
                        hB = ld4cg(K.hd[sj], q);
                    }
                }
                float4 rv = rr;
                if (step) {  // step j = k - 1 (same operation order as mr_step4)
                    float4 dj = mul4(c.dw, vj);
                    float4 hj = mul4(c.dinv, awj);
                    if (j >= 2) {
                        dj = fma4(-c.d1, dA, dj);
                        hj = fma4(-c.d1, hA, hj);
                    }
                    if (j >= 3) {
                        dj = fma4(-c.d2, dB, dj);
                        hj = fma4(-c.d2, hB, hj);
                    }
                    IO::st4(K.d[sj], q, dj);
                    st4(K.hd[sj], q, hj);
                    if (apply) st4(J.u, q, fma4(c.tau, dj, uu));
                    rv = fma4(-c.tau, hj, rr);
                    st4(J.r, q, rv);
                }
                if (step) arr = dot4(rv, rv, arr);
                float4 vn = fma4(-ca_lo, vk, fma4(-ca, vk, awk));
                if (step) vn = fma4(-cb_lo, vj, fma4(-cb, vj, vn));
                st4(K.v[sk1], q, vn);
                avv = dot4(vn, vn, avv);
                avr = dot4(vn, rv, avr);
            }
            if (bid == 0) {  // the n mod 4 tail
                for (size_t i = 4 * n4 + threadIdx.x; i < n; i += NTHREADS) {
                    const float rv = apply  ? mr_step_px<HT>(J, K, k - 1, i, c.dw, c.d1, c.d2, c.dinv, c.tau)
                                     : rest ? mr_step_px<HT, 2>(J, K, k - 1, i, c.dw, c.d1, c.d2, c.dinv, c.tau)
                                            : ldcg(J.r + i);
                    if (step) arr = fmaf(rv, rv, arr);
                    const float vki = ldcg(K.v[sk] + i);
                    float vn = fmaf(-ca_lo, vki, fmaf(-ca, vki, ldcg(K.aw[sk] + i)));
                    if (step) {
                        const float vk1 = ldcg(K.v[sk1] + i);
                        vn = fmaf(-cb_lo, vk1, fmaf(-cb, vk1, vn));
                    }
                    K.v[sk1][i] = vn;
                    avv = fmaf(vn, vn, avv);
                    avr = fmaf(vn, rv, avr);
                }
            }
            float v[3] = {arr, avv, avr};
            const double bb = k == 1 ? 16.0 : (apply ? 40.0 + E + hist(k - 1) : 32.0 + E + hist(k - 1));
            if (!sy.reduce<3>(v, [&](DF* t) {
                    fin_mr_b(sc, k, t[0], t[1], t[2]);
                    sc->bpp += bb;
                }))
                return;
        }
        // early check of step k (fin_mr_b predicted ||r_k|| at the limit): apply it now and
        // test ||r_k||, so that a solve that stops here skips iteration k + 1's convolution
        if (k < J.m && *(volatile const int*)&sc->spec && !volatile_stopped(sc)) {
            const StepCoef c = step_coef(sc);
            float arr = 0.f;
            const size_t n4 = n >> 2;
            for (size_t q = (size_t)bid * NTHREADS + threadIdx.x; q < n4; q += stride) {
                const float4 rv = mr_step4_u<HT>(J, K, k, q, c);
                arr = dot4(rv, rv, arr);
            }
            if (bid == 0)
                for (size_t i = 4 * n4 + threadIdx.x; i < n; i += NTHREADS) {
                    const float rv = mr_step_px<HT, 1>(J, K, k, i, c.dw, c.d1, c.d2, c.dinv, c.tau);
                    arr = fmaf(rv, rv, arr);
                }
            float v[1] = {arr};
            const double bc = 20.0 + hist(k);
            if (!sy.reduce<1>(v, [&](DF* t) {
                    fin_mr_check(sc, k, t[0]);
                    sc->bpp += bc;
                }))
                return;
        }
    }

    // the step decided last (breakdown-with-step or the schedule's end), unless an early
    // check applied it already
    const int st = volatile_stopped(sc);
    const int j = *(volatile const int*)&sc->iters;
    if ((st == 0 || st == 4) && j >= 1 && *(volatile const int*)&sc->applied != j) {
        const StepCoef c = step_coef(sc);
        float arr = 0.f;
        const size_t n4 = n >> 2;
        for (size_t q = (size_t)bid * NTHREADS + threadIdx.x; q < n4; q += stride) {
            const float4 rv = mr_step4_u<HT>(J, K, j, q, c);
            arr = dot4(rv, rv, arr);
        }
        if (bid == 0)
            for (size_t i = 4 * n4 + threadIdx.x; i < n; i += NTHREADS) {
                const float rv = mr_step_px<HT, 1>(J, K, j, i, c.dw, c.d1, c.d2, c.dinv, c.tau);
                arr = fmaf(rv, rv, arr);
            }
        float v[1] = {arr};
        const double bf = 20.0 + hist(j);
        sy.reduce<1>(v, [&](DF* t) {
            fin_mr_final(sc, t[0]);
            sc->bpp += bf;
        });
    }
}

template <int R, bool SEP, bool PREC, typename HT>
__device__ __forceinline__ void cgls_body(ConvSmem<R, SEP>& S, PsdSmem& M, const LevelJob& J, Scalars* sc,
                                          unsigned int nb, unsigned int bid, LevelSync& sy) {
    // s and p are stored as HT; q = H p stays FP32 (computed from the stored
    // p), so u and the residual recurrence see the same direction
    using IO = VecIO<HT>;
    const int h = J.h, w = J.w;
    const size_t n = (size_t)h * w;
    const size_t stride = (size_t)nb * NTHREADS;
    float* rv_ = J.r;
    HT* sv = reinterpret_cast<HT*>(J.v[0]);   // s
    HT* pv = reinterpret_cast<HT*>(J.v[1]);   // p
    float* qv = J.aw[0];                      // q
    if (J.start && !start_phase(M, J, nb, bid, sy)) return;
    conv_stage_taps<R, SEP>(S, J.taps);
    __syncthreads();
    {
        float a0 = 0.f, a1 = 0.f;
        const bool zs = J.zero_start != 0;
        auto epi = [&](size_t idx, float z, float, float gv) {
            const float rv = gv - z;
            rv_[idx] = rv;
            if (zs) J.u[idx] = 0.f;
            a0 = fmaf(rv, rv, a0);
            a1 = fmaf(gv, gv, a1);
        };
        if (zs)
            conv_phase<R, SEP, PREC, true>(S, J.u, h, w, nb, bid, J.g, epi);
        else
            conv_phase<R, SEP, PREC, false>(S, J.u, h, w, nb, bid, J.g, epi);
        float v[2] = {a0, a1};
        const double ct2 = J.conv_tol2, d2 = J.disc2;
        const int ear = J.early;
        const double sb = start_bytes(J);  // the host counts the CGLS phases themselves
        if (!sy.reduce<2>(v, [&](DF* t) {
                fin_resid(sc, t[0], t[1], ct2, d2, ear);
                sc->bpp = sb;
            }))
            return;
    }
    if (J.m <= 0 || volatile_stopped(sc)) return;
    __syncthreads();
    conv_stage_taps<R, SEP>(S, J.tapsT);  // s = H^T r, p = s
    __syncthreads();
    {
        float a0 = 0.f;
        conv_phase<R, SEP, PREC, false>(S, rv_, h, w, nb, bid, nullptr, [&](size_t idx, float z, float, float) {
            IO::st(sv, idx, z);
            IO::st(pv, idx, z);
            a0 = fmaf(z, z, a0);
        });
        float v[1] = {a0};
        if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_s0(sc, t[0]); }))
            return;
    }
    for (int k = 1; k <= J.m; ++k) {
        if (volatile_stopped(sc)) break;
        __syncthreads();
        conv_stage_taps<R, SEP>(S, J.taps);  // q = H p, alpha
        __syncthreads();
        {
            float a0 = 0.f;
            conv_phase<R, SEP, PREC, false, HT>(S, pv, h, w, nb, bid, nullptr, [&](size_t idx, float z, float, float) {
                qv[idx] = z;
                a0 = fmaf(z, z, a0);
            });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_q(sc, t[0]); }))
                return;
        }
        if (volatile_stopped(sc)) break;
        {  // u += alpha p, r -= alpha q, stopping rule
            const float a = vldf(&sc->f_cg_alpha);
            float arr = 0.f;
            const size_t n4 = n >> 2;
            for (size_t q = (size_t)bid * NTHREADS + threadIdx.x; q < n4; q += stride) {
                const float4 pq = IO::ld4(pv, q), uq = ld4cg(J.u, q);  // all loads first
                const float4 qq = ld4cg(qv, q), rq = ld4cg(rv_, q);
                st4(J.u, q, fma4(a, pq, uq));
                const float4 r = fma4(-a, qq, rq);
                st4(rv_, q, r);
                arr = dot4(r, r, arr);
            }
            if (bid == 0)
                for (size_t i = 4 * n4 + threadIdx.x; i < n; i += NTHREADS) {
                    J.u[i] = fmaf(a, IO::ld(pv, i), ldcg(J.u + i));
                    const float r = fmaf(-a, ldcg(qv + i), ldcg(rv_ + i));
                    rv_[i] = r;
                    arr = fmaf(r, r, arr);
                }
            float v[1] = {arr};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_step(sc, t[0]); }))
                return;
        }
        if (k == J.m || volatile_stopped(sc)) break;
        __syncthreads();
        conv_stage_taps<R, SEP>(S, J.tapsT);  // s = H^T r, beta
        __syncthreads();
        {
            float a0 = 0.f;
            conv_phase<R, SEP, PREC, false>(S, rv_, h, w, nb, bid, nullptr, [&](size_t idx, float z, float, float) {
                IO::st(sv, idx, z);
                a0 = fmaf(z, z, a0);
            });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_s(sc, t[0]); }))
                return;
        }
        if (volatile_stopped(sc)) break;
        {  // p = s + beta p
            const float b = vldf(&sc->f_beta);
            const size_t n4 = n >> 2;
            for (size_t q = (size_t)bid * NTHREADS + threadIdx.x; q < n4; q += stride)
                IO::st4(pv, q, fma4(b, IO::ld4(pv, q), IO::ld4(sv, q)));
            if (bid == 0)
                for (size_t i = 4 * n4 + threadIdx.x; i < n; i += NTHREADS)
                    IO::st(pv, i, fmaf(b, IO::ld(pv, i), IO::ld(sv, i)));
            float v[1] = {0.f};
            if (!sy.reduce<1>(v, [&](DF*) {})) return;
        }
    }
}

// One level solve per job: a cooperative grid (LL.cluster == 0; the job's
// blocks meet at bounded grid barriers) or one thread-block cluster of
// LL.cluster blocks per job (reductions through distributed shared memory).
// Shared memory of a streaming solve: the convolution tile of every phase, or
// the level-start tile of phase 0.
template <int R, bool SEP>
union LevelSmem {
    ConvSmem<R, SEP> conv;
    PsdSmem psd;
};

template <int R, bool SEP, bool PREC, typename HT, bool CGLS>
__device__ __forceinline__ void level_kernel(const LevelLaunch& LL) {
    __shared__ LevelSmem<R, SEP> U;
    ConvSmem<R, SEP>& S = U.conv;
    __shared__ LevelJob sJ;
    __shared__ ClusterState CS;
    if (threadIdx.x == 0) sJ = LL.jobs ? LL.jobs[LL.block_job[blockIdx.x]] : LL.job;
    __syncthreads();
    const LevelJob& J = sJ;
    const unsigned int nb = LL.jobs ? (unsigned int)J.nblocks : gridDim.x;
    const unsigned int bid = LL.jobs ? blockIdx.x - (unsigned int)J.block0 : blockIdx.x;
    const bool cl = LL.cluster > 0;
    if (cl) {
        cluster_begin(CS, J.sc, nb);
    } else {
        if (threadIdx.x == 0) CS.sc = *J.sc;
        __syncthreads();
    }
    LevelSync sy{J.partials, J.gs, nb, bid, &CS, cl, 0u};
    Scalars* sc = &CS.sc;  // this block's replica (identical in every block)
    if constexpr (CGLS)
        cgls_body<R, SEP, PREC, HT>(S, U.psd, J, sc, nb, bid, sy);
    else
        mr2_body<R, SEP, PREC, HT>(S, U.psd, J, sc, nb, bid, sy);
    if (cl) {
        cluster_end(CS, J.sc, bid);
    } else {
        __syncthreads();
        if (bid == 0 && threadIdx.x == 0) *J.sc = CS.sc;
        grid_exit(J.gs, nb);
    }
}

template <int R, bool SEP, bool PREC, typename HT>
__global__ void __launch_bounds__(NTHREADS, 2) k_level_mr2(LevelLaunch LL) {
    level_kernel<R, SEP, PREC, HT, false>(LL);
}

template <int R, bool SEP, bool PREC, typename HT>
__global__ void __launch_bounds__(NTHREADS, 3) k_level_cgls(LevelLaunch LL) {
    level_kernel<R, SEP, PREC, HT, true>(LL);
}

}  // namespace eecmg

#include "level_resident.cuh"

namespace eecmg {

template <class K>
inline cudaError_t coop_launch(K kernel, const LevelLaunch& L, int blocks, cudaStream_t s) {
    LevelLaunch arg = L;
    void* params[] = {&arg};
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(blocks), dim3(NTHREADS), params, 0, s);
}

template <class K>
inline cudaError_t cluster_launch(K kernel, const LevelLaunch& L, int blocks, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned int)L.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, L);
}

template <class K>
inline int coresident_blocks(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NTHREADS, 0);
    return per_sm * sms;
}

// Largest cluster (<= CLUSTER_MAX) the kernel can run as; 0 if none.
template <class K>
inline int max_cluster(K kernel) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLUSTER_MAX);
    cfg.blockDim = dim3(NTHREADS);
    int c = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&c, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return c < CLUSTER_MAX ? c : CLUSTER_MAX;
}

// One instantiation: op selects a cooperative launch of `blocks` blocks, a
// cluster launch of `blocks` blocks in clusters of L.cluster, or a query
// (*out = co-resident capacity, or the largest usable cluster).
template <class K>
inline cudaError_t level_op(K kern, int& cap, int& cmax, const LevelLaunch& L, int op, int blocks,
                            cudaStream_t s, int* out) {
    switch (op) {
        case LS_CAPACITY:
            if (cap < 0) cap = coresident_blocks(kern);
            if (out) *out = cap;
            return cudaSuccess;
        case LS_CLUSTER_MAX:
            if (cmax < 0) cmax = max_cluster(kern);
            if (out) *out = cmax;
            return cudaSuccess;
        case LS_COOP:
            return coop_launch(kern, L, blocks, s);
        case LS_CLUSTER:
            if (cmax < 0) cmax = max_cluster(kern);
            if (L.cluster < 1 || L.cluster > cmax || blocks % L.cluster) return cudaErrorInvalidValue;
            return cluster_launch(kern, L, blocks, s);
        default:
            return cudaErrorInvalidValue;
    }
}

// The resident solver of one instantiation: a cluster launch with
// res_smem_bytes(L.resident) of dynamic shared memory, or the largest cluster
// it can run as with that much (cached per tile count).
template <class K>
inline bool res_attrs(K kern) {
    const bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)res_smem_bytes(RES_TMAX)) == cudaSuccess &&
                    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                        cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
}

// attrs: res_attrs() of this kernel (set once per instantiation by the caller)
template <class K>
inline cudaError_t res_op(K kern, bool attrs, int (&cmax)[RES_TMAX + 1], const LevelLaunch& L, int op,
                          int blocks, cudaStream_t s, int* out) {
    const int T = L.resident;
    if (T < 1 || T > RES_TMAX) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = res_smem_bytes(T);
    cfg.stream = s;
    if (op == LS_RESIDENT_MAX) {
        if (cmax[T] < 0) {
            int c = 0;
            cfg.gridDim = dim3(CLUSTER_MAX);
            if (!attrs || cudaOccupancyMaxPotentialClusterSize(&c, kern, &cfg) != cudaSuccess) {
                cudaGetLastError();
                c = 0;
            }
            cmax[T] = c < CLUSTER_MAX ? c : CLUSTER_MAX;
        }
        if (out) *out = cmax[T];
        return cudaSuccess;
    }
    if (!attrs || L.cluster < 1 || L.cluster > CLUSTER_MAX || blocks % L.cluster) return cudaErrorInvalidValue;
    cfg.gridDim = dim3(blocks);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned int)L.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, L);
}

template <int R, bool SEP, bool PREC, bool CGLS, typename HT>
cudaError_t launch_level_t(const LevelLaunch& L, int op, int blocks, cudaStream_t s, int* out) {
    static int cap = -1, cmax = -1;  // per instantiation; the library runs on one GPU model
    if (op == LS_RESIDENT || op == LS_RESIDENT_MAX) {
        if constexpr (std::is_same<HT, float>::value && R <= RES_RMAX) {
            static int rmax[RES_TMAX + 1] = {-1, -1, -1};
            if constexpr (CGLS) {
                static const bool attrs = res_attrs(k_level_cgls_res<R, SEP, PREC>);  // per instantiation
                return res_op(k_level_cgls_res<R, SEP, PREC>, attrs, rmax, L, op, blocks, s, out);
            } else {
                static const bool attrs = res_attrs(k_level_mr2_res<R, SEP, PREC>);
                return res_op(k_level_mr2_res<R, SEP, PREC>, attrs, rmax, L, op, blocks, s, out);
            }
        } else {
            if (out) *out = 0;
            return op == LS_RESIDENT_MAX ? cudaSuccess : cudaErrorInvalidValue;
        }
    }
    if constexpr (CGLS)
        return level_op(k_level_cgls<R, SEP, PREC, HT>, cap, cmax, L, op, blocks, s, out);
    else
        return level_op(k_level_mr2<R, SEP, PREC, HT>, cap, cmax, L, op, blocks, s, out);
}

template <int R, bool CGLS, typename HT>
cudaError_t launch_level_r(const LevelLaunch& L, int sep, int prec, int op, int blocks,
                           cudaStream_t s, int* out) {
    if (sep && prec) return launch_level_t<R, true, true, CGLS, HT>(L, op, blocks, s, out);
    if (sep) return launch_level_t<R, true, false, CGLS, HT>(L, op, blocks, s, out);
    return launch_level_t<R, false, false, CGLS, HT>(L, op, blocks, s, out);
}

// Per translation unit: one solver, one storage type, a range of radii
// (names: launch_level_<solver>_<storage>_<lo|hi>).
#define EECMG_LS_DECL(name)                                                                \
    cudaError_t name(const LevelLaunch& L, int rt, int sep, int prec, int op, int blocks,      \
                     cudaStream_t s, int* out);
EECMG_LS_DECL(launch_level_mr2_f32_lo)
EECMG_LS_DECL(launch_level_mr2_f32_hi)
EECMG_LS_DECL(launch_level_mr2_bf16_lo)
EECMG_LS_DECL(launch_level_mr2_bf16_hi)
EECMG_LS_DECL(launch_level_cgls_f32_lo)
EECMG_LS_DECL(launch_level_cgls_f32_hi)
EECMG_LS_DECL(launch_level_cgls_bf16_lo)
EECMG_LS_DECL(launch_level_cgls_bf16_hi)
#undef EECMG_LS_DECL

}  // namespace eecmg
