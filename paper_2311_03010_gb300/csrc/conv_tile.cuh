// conv_tile.cuh -- one 32 x 64 output tile of the zero-boundary convolution
// y = C (*) x (Eqs. 1, 7), shared by the single-launch convolution kernel and
// the persistent level solvers.
//
// The input tile plus a halo of R pixels is staged in shared memory (zero
// outside the image: the block-Toeplitz boundary of Eq. 7).  Separable PSFs
// run a vertical then a horizontal pass, each thread sliding a register
// window over 8 outputs; other PSFs run over their non-zero taps.  PREC
// selects a compensated horizontal pass: each product is split exactly into
// p + pe with an FMA, the p are summed with Kahan compensation and the pe in
// a separate accumulator (7 FP32 operations per tap instead of 1).  The result lands in S.out (row r, column c at r * PO + c) and the
// staged input stays in S.in (pixel (r, c) of the tile at (r + R) * IW + c + R).
#pragma once

#include "launch.hpp"

namespace eecmg {

template <int R, bool SEP>
struct ConvSmem {
    static constexpr int TH = CONV_TH, TW = CONV_TW;
    static constexpr int IH = TH + 2 * R, IW = TW + 2 * R;
    static constexpr int PT = TW + 2 * R + 1;  // odd pitch: conflict-free column walks
    static constexpr int PO = TW + 1;
    static constexpr int NT = SEP ? 1 : (2 * R + 1) * (2 * R + 1);
    float in[IH * IW];
    float tmp[SEP ? TH * PT : 1];
    float out[TH * PO];
    float cy[2 * R + 1], cx[2 * R + 1];
    int off[NT];
    float wt[NT];
    int ntap;
};

// Stages the level's taps (then __syncthreads()).  The kernel radius R may
// exceed the taps' own radius (a batched launch uses the largest radius of
// its jobs): separable factors are placed centred and padded with zeros.
template <int R, bool SEP>
__device__ __forceinline__ void conv_stage_taps(ConvSmem<R, SEP>& S, const Taps* taps) {
    const int tid = threadIdx.x;
    if (SEP) {
        const int rt = taps->rt;
        for (int d = tid; d < 2 * R + 1; d += NTHREADS) {
            const int e = d - R + rt;
            const bool in = e >= 0 && e <= 2 * rt;
            S.cy[d] = in ? taps->cy[e] : 0.f;
            S.cx[d] = in ? taps->cx[e] : 0.f;
        }
    } else {
        const int nt = taps->ntap;
        if (tid == 0) S.ntap = nt;
        for (int t = tid; t < nt; t += NTHREADS) {
            S.off[t] = (taps->dy[t] + R) * ConvSmem<R, SEP>::IW + (taps->dx[t] + R);
            S.wt[t] = taps->wt[t];
        }
    }
}

// Loads the tile at (y0, x0) with halo.  COHERENT loads go through L2 only
// (ld.global.cg): required when x was written earlier in the same launch by
// other blocks.
template <int R, bool SEP, bool COHERENT, typename TIN = float>
__device__ __forceinline__ void conv_load(ConvSmem<R, SEP>& S, const TIN* __restrict__ x, int h,
                                          int w, int y0, int x0) {
    constexpr int IH = ConvSmem<R, SEP>::IH, IW = ConvSmem<R, SEP>::IW;
    constexpr int NTOT = IH * IW;
    constexpr int ITERS = (NTOT + NTHREADS - 1) / NTHREADS;
    const int tid = threadIdx.x;
    float vals[ITERS];
#pragma unroll
    for (int k = 0; k < ITERS; ++k) {
        const int i = tid + k * NTHREADS;
        const int r = i / IW, c = i - r * IW;
        const int gy = y0 - R + r, gx = x0 - R + c;
        float v = 0.f;
        if (i < NTOT && gy >= 0 && gy < h && gx >= 0 && gx < w) {
            const size_t idx = (size_t)gy * w + gx;
            if constexpr (sizeof(TIN) == 4)
                v = COHERENT ? __ldcg((const float*)x + idx) : __ldg((const float*)x + idx);
            else
                v = VecIO<TIN>::ld(x, idx);
        }
        vals[k] = v;
    }
#pragma unroll
    for (int k = 0; k < ITERS; ++k) {
        const int i = tid + k * NTHREADS;
        if (i < NTOT) S.in[i] = vals[k];
    }
}

// Computes S.out from S.in (the caller synchronises before and after).
template <int R, bool SEP, bool PREC>
__device__ __forceinline__ void conv_compute(ConvSmem<R, SEP>& S) {
    constexpr int IW = ConvSmem<R, SEP>::IW, PT = ConvSmem<R, SEP>::PT, PO = ConvSmem<R, SEP>::PO;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (SEP) {
        // Each thread slides a register window over 8 outputs; the taps are
        // read from shared memory (a broadcast) once per tap, tap-outer, so the
        // window and the 8 accumulators are all that live in registers.  Every
        // output still sums its taps in increasing order.
        // vertical pass: tmp(r, c) = sum_d cy[d] in(r + d, c), r < TH, all IW columns
        for (int item = tid; item < 4 * IW; item += NTHREADS) {
            const int rg = item / IW, c = item - rg * IW;
            float v[8 + 2 * R];
#pragma unroll
            for (int j = 0; j < 8 + 2 * R; ++j) v[j] = S.in[(rg * 8 + j) * IW + c];
            float acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
            for (int d = 0; d < 2 * R + 1; ++d) {
                const float cd = S.cy[d];
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fmaf(cd, v[i + d], acc[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) S.tmp[(rg * 8 + i) * PT + c] = acc[i];
        }
        __syncthreads();
        // horizontal pass: one row per lane, 8 consecutive columns per warp
        const int r = lane, cg = warp;
        float v[8 + 2 * R];
#pragma unroll
        for (int j = 0; j < 8 + 2 * R; ++j) v[j] = S.tmp[r * PT + cg * 8 + j];
        float acc[8], lo[8], comp[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i] = 0.f;
            lo[i] = 0.f;
            comp[i] = 0.f;
        }
#pragma unroll
        for (int d = 0; d < 2 * R + 1; ++d) {
            const float cd = S.cx[d];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (PREC) {
                    // exact product p + pe (FMA), Kahan-compensated sum of the p,
                    // product errors summed apart: 7 operations per tap
                    const float p = __fmul_rn(cd, v[i + d]);
                    const float pe = fmaf(cd, v[i + d], -p);
                    const float y = __fsub_rn(p, comp[i]);
                    const float t = __fadd_rn(acc[i], y);
                    comp[i] = __fsub_rn(__fsub_rn(t, acc[i]), y);
                    acc[i] = t;
                    lo[i] = __fadd_rn(lo[i], pe);
                } else {
                    acc[i] = fmaf(cd, v[i + d], acc[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            S.out[r * PO + cg * 8 + i] = PREC ? __fadd_rn(acc[i], __fsub_rn(lo[i], comp[i])) : acc[i];
    } else {
        const int c = tid & 63, rg = tid >> 6;
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        const int nt = S.ntap;
        const float* base = S.in + (rg * 8) * IW + c;
        for (int t = 0; t < nt; ++t) {
            const float wt = S.wt[t];
            const float* p = base + S.off[t];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt, p[i * IW], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) S.out[(rg * 8 + i) * PO + c] = acc[i];
    }
}

}  // namespace eecmg
