// conv_tile.cuh -- one 32 x 64 output tile of the zero-boundary convolution
// y = C (*) x (Eqs. 1, 7), shared by the single-launch convolution kernel and
// the persistent level solvers.
//
// The input tile plus a halo of R pixels is staged in shared memory (zero
// outside the image: the block-Toeplitz boundary of Eq. 7).  Separable PSFs
// run a vertical then a horizontal pass, each thread sliding a register
// window over its outputs; other PSFs run over their non-zero taps.  PREC
// selects a compensated horizontal pass: each product is split exactly into
// p + pe with an FMA, the p are summed with Kahan compensation and the pe in
// a separate accumulator (7 FP32 operations per tap instead of 1).  The result
// lands in S.out (row r, column c at r * PO + c) and the staged input stays in
// S.in (pixel (r, c) of the tile at S.at(r + R, c + R)).
#pragma once

#include "launch.hpp"

namespace eecmg {

template <int R, bool SEP>
struct ConvSmem {
    static constexpr int TH = CONV_TH, TW = CONV_TW;
    static constexpr int IH = TH + 2 * R, IW = TW + 2 * R;
    // Input rows start 16-byte aligned and hold the window from column -X0:
    // the halo rounded up to whole 4-float chunks, so that a row of the
    // window arrives as aligned 16-byte chunks (one shared store each).
    static constexpr int PADX = (R + 3) / 4 * 4;
    static constexpr int X0 = PADX - R;
    static constexpr int IP = TW + 2 * PADX;
    // tmp pitch: the window rounded up to whole 16-byte vectors (rows are read as
    // 16-byte vectors), an odd number of them, so the 8 rows of a quarter warp's
    // 16-byte loads fall on distinct banks
    static constexpr int PT0 = (IW + 3) / 4 * 4;
    static constexpr int PT = (PT0 / 4) % 2 == 1 ? PT0 : PT0 + 4;
    static constexpr int PO = TW + 1;
    static constexpr int NTAP4 = (2 * R + 1 + 3) / 4 * 4;  // taps padded to whole float4
    static constexpr int NT = SEP ? 1 : (2 * R + 1) * (2 * R + 1);
    // Vertical pass of the separable form: VG groups of VR consecutive rows
    // per window column, one group per thread, every thread busy in one
    // round (the last group starts at TH - VR and overlaps the one before).
    static constexpr int VG = 3 * IW <= NTHREADS ? 3 : 2;
    static constexpr int VR = (TH + VG - 1) / VG;
    alignas(16) float in[IH * IP];
    alignas(16) float tmp[SEP ? TH * PT : 4];
    float out[TH * PO];
    // separable factors, zero-padded to whole float4: each 16-byte load is one
    // broadcast carrying four taps
    alignas(16) float cy[NTAP4];
    alignas(16) float cx[NTAP4];
    int off[NT];
    float wt[NT];
    int ntap;
    // index in `in` of window pixel (r, c), r in [0, IH), c in [0, IW)
    static __device__ __forceinline__ int at(int r, int c) { return r * IP + X0 + c; }
};

// Stages the level's taps (then __syncthreads()).  The kernel radius R may
// exceed the taps' own radius (a batched launch uses the largest radius of
// its jobs): separable factors are placed centred and padded with zeros.
template <int R, bool SEP>
__device__ __forceinline__ void conv_stage_taps(ConvSmem<R, SEP>& S, const Taps* taps) {
    const int tid = threadIdx.x;
    if (SEP) {
        const int rt = taps->rt;
        for (int d = tid; d < ConvSmem<R, SEP>::NTAP4; d += NTHREADS) {
            const int e = d - R + rt;
            const bool in = d <= 2 * R && e >= 0 && e <= 2 * rt;
            S.cy[d] = in ? taps->cy[e] : 0.f;
            S.cx[d] = in ? taps->cx[e] : 0.f;
        }
    } else {
        const int nt = taps->ntap;
        if (tid == 0) S.ntap = nt;
        for (int t = tid; t < nt; t += NTHREADS) {
            // offset of tap (dy, dx) from window pixel (r, c) to (r + dy + R, c + dx + R)
            S.off[t] = (taps->dy[t] + R) * ConvSmem<R, SEP>::IP + (taps->dx[t] + R);
            S.wt[t] = taps->wt[t];
        }
    }
}

// Per-thread share of a tile with halo, held in registers between its global
// loads and its shared-memory stores.  Rows are fetched as 16-byte chunks (4
// FP32 or 8 BF16 values) starting PADX (the halo rounded up to a chunk) left
// of the tile, so that every chunk is aligned whenever the row pitch is: an
// element costs a fraction of an address computation and bounds test.
template <int R, bool SEP, typename TIN = float>
struct ConvRegs {
    static constexpr int EPC = 16 / (int)sizeof(TIN);       // elements per chunk
    static constexpr int PADX = (R + EPC - 1) / EPC * EPC;
    static constexpr int XOFF = PADX - R;                   // loaded columns left of the halo
    static constexpr int CPR = (CONV_TW + 2 * PADX) / EPC;  // chunks per row
    static constexpr int IH = ConvSmem<R, SEP>::IH;
    static constexpr int NC = IH * CPR;
    static constexpr int ITERS = (NC + NTHREADS - 1) / NTHREADS;
    uint4 q[ITERS];
};

__device__ __forceinline__ float chunk_elem(const uint4& c, int e, float) {
    const unsigned int b = e == 0 ? c.x : (e == 1 ? c.y : (e == 2 ? c.z : c.w));
    return __uint_as_float(b);
}
__device__ __forceinline__ float chunk_elem(const uint4& c, int e, __nv_bfloat16) {
    const unsigned int b = (e >> 1) == 0 ? c.x : ((e >> 1) == 1 ? c.y : ((e >> 1) == 2 ? c.z : c.w));
    return __uint_as_float((e & 1) ? (b & 0xffff0000u) : (b << 16));
}
// The raw bits of element i of x (an FP32 or BF16 vector), through L2 or the read-only path.
template <bool COHERENT>
__device__ __forceinline__ unsigned int elem_bits(const float* x, size_t i) {
    const unsigned int* p = reinterpret_cast<const unsigned int*>(x) + i;
    return COHERENT ? __ldcg(p) : __ldg(p);
}
template <bool COHERENT>
__device__ __forceinline__ unsigned int elem_bits(const __nv_bfloat16* x, size_t i) {
    const unsigned short* p = reinterpret_cast<const unsigned short*>(x) + i;
    return (unsigned int)(COHERENT ? __ldcg(p) : __ldg(p));
}

// Issues the global loads of the tile at (y0, x0) with halo into registers
// (zero outside the image).  COHERENT loads go through L2 only
// (ld.global.cg): required when x was written earlier in the same launch by
// other blocks.  Aligned 16-byte loads when x is 16-byte aligned and w a
// multiple of the chunk; element loads otherwise (same values).
template <int R, bool SEP, bool COHERENT, typename TIN = float>
__device__ __forceinline__ void conv_fetch(ConvRegs<R, SEP, TIN>& V, const TIN* __restrict__ x, int h,
                                           int w, int y0, int x0) {
    using CR = ConvRegs<R, SEP, TIN>;
    constexpr int EPC = CR::EPC;
    const int tid = threadIdx.x;
    const bool vec = (w % EPC) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
#pragma unroll
    for (int k = 0; k < CR::ITERS; ++k) {
        const int i = tid + k * NTHREADS;
        const int r = i / CR::CPR, c = i - r * CR::CPR;
        const int gy = y0 - R + r, gx = x0 - CR::PADX + EPC * c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i < CR::NC && gy >= 0 && gy < h) {
            const size_t row = (size_t)gy * w;
            if (vec) {
                if (gx >= 0 && gx < w) {
                    const uint4* p = reinterpret_cast<const uint4*>(x + row + gx);
                    v = COHERENT ? __ldcg(p) : __ldg(p);
                }
            } else {
                unsigned int b[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int gxe = gx + e;
                    if (gxe >= 0 && gxe < w)
                        b[e * (int)sizeof(TIN) / 4] |= elem_bits<COHERENT>(x, row + gxe)
                                                       << (8 * ((e * (int)sizeof(TIN)) & 3));
                }
                v = make_uint4(b[0], b[1], b[2], b[3]);
            }
        }
        V.q[k] = v;
    }
}

// Stores a fetched tile into S.in as FP32 (the caller synchronises before reading it).
// FP32 chunks land whole (their columns line up with the rows of S.in); BF16
// chunks are widened element by element, the parts outside the window dropped.
template <int R, bool SEP, typename TIN = float>
__device__ __forceinline__ void conv_put(ConvSmem<R, SEP>& S, const ConvRegs<R, SEP, TIN>& V) {
    using CR = ConvRegs<R, SEP, TIN>;
    using SM = ConvSmem<R, SEP>;
    constexpr int IW = SM::IW, EPC = CR::EPC;
    const int tid = threadIdx.x;
    if constexpr (EPC == 4) {
        static_assert(CR::PADX == SM::PADX && CR::CPR * 4 == SM::IP, "FP32 chunks must tile the rows of S.in");
#pragma unroll
        for (int k = 0; k < CR::ITERS; ++k) {
            const int i = tid + k * NTHREADS;
            if (i < CR::NC) reinterpret_cast<uint4*>(S.in)[i] = V.q[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < CR::ITERS; ++k) {
            const int i = tid + k * NTHREADS;
            if (i < CR::NC) {
                const int r = i / CR::CPR, c = i - r * CR::CPR;
                const int lc = EPC * c - CR::XOFF;  // window column of the chunk's first element
                float* dst = S.in + SM::at(r, lc);
                if (lc >= 0 && lc + EPC - 1 < IW) {
#pragma unroll
                    for (int e = 0; e < EPC; ++e) dst[e] = chunk_elem(V.q[k], e, TIN());
                } else {
#pragma unroll
                    for (int e = 0; e < EPC; ++e)
                        if (lc + e >= 0 && lc + e < IW) dst[e] = chunk_elem(V.q[k], e, TIN());
                }
            }
        }
    }
}

// Loads the tile at (y0, x0) with halo into S.in.
template <int R, bool SEP, bool COHERENT, typename TIN = float>
__device__ __forceinline__ void conv_load(ConvSmem<R, SEP>& S, const TIN* __restrict__ x, int h,
                                          int w, int y0, int x0) {
    ConvRegs<R, SEP, TIN> V;
    conv_fetch<R, SEP, COHERENT, TIN>(V, x, h, w, y0, x0);
    conv_put<R, SEP, TIN>(S, V);
}

// Computes S.out from S.in (the caller synchronises before and after).
template <int R, bool SEP, bool PREC>
__device__ __forceinline__ void conv_compute(ConvSmem<R, SEP>& S) {
    using SM = ConvSmem<R, SEP>;
    constexpr int IW = SM::IW, PT = SM::PT, PO = SM::PO, VR = SM::VR, VG = SM::VG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (SEP) {
        // Each thread slides a register window over its outputs; the taps are
        // read from shared memory (a broadcast) once per tap, tap-outer, so the
        // window and the accumulators are all that live in registers.  Every
        // output still sums its taps in increasing order.
        // vertical pass: tmp(r, c) = sum_d cy[d] in(r + d, c), r < TH, all IW columns;
        // thread (g, c) takes rows r0 .. r0 + VR - 1 of column c
        const int g = tid / IW, c = tid - g * IW;
        if (g < VG) {
            const int r0 = g == VG - 1 ? CONV_TH - VR : g * VR;
            float v[VR + 2 * R];
#pragma unroll
            for (int j = 0; j < VR + 2 * R; ++j) v[j] = S.in[SM::at(r0 + j, c)];
            float acc[VR];
#pragma unroll
            for (int i = 0; i < VR; ++i) acc[i] = 0.f;
#pragma unroll
            for (int d4 = 0; d4 < 2 * R + 1; d4 += 4) {
                const float4 c4 = *reinterpret_cast<const float4*>(S.cy + d4);
                const float cq[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (d4 + e <= 2 * R) {
#pragma unroll
                        for (int i = 0; i < VR; ++i) acc[i] = fmaf(cq[e], v[i + d4 + e], acc[i]);
                    }
            }
            // rows the group before already wrote are skipped
#pragma unroll
            for (int i = 0; i < VR; ++i)
                if (g < VG - 1 || i >= VG * VR - CONV_TH) S.tmp[(r0 + i) * PT + c] = acc[i];
        }
        __syncthreads();
        // horizontal pass: one row per lane, 8 consecutive columns per warp; the
        // window (8 + 2R values from column 8 cg, a multiple of 4) as 16-byte loads
        const int r = lane, cg = warp;
        constexpr int NW = 8 + 2 * R, NW4 = (NW + 3) / 4;
        float v[4 * NW4];
#pragma unroll
        for (int j4 = 0; j4 < NW4; ++j4) {
            const float4 q = *reinterpret_cast<const float4*>(S.tmp + r * PT + cg * 8 + 4 * j4);
            v[4 * j4] = q.x;
            v[4 * j4 + 1] = q.y;
            v[4 * j4 + 2] = q.z;
            v[4 * j4 + 3] = q.w;
        }
        float acc[8], lo[8], comp[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i] = 0.f;
            lo[i] = 0.f;
            comp[i] = 0.f;
        }
#pragma unroll
        for (int d = 0; d < 2 * R + 1; ++d) {
            const float4 c4 = *reinterpret_cast<const float4*>(S.cx + (d & ~3));
            const float cd = (d & 3) == 0 ? c4.x : ((d & 3) == 1 ? c4.y : ((d & 3) == 2 ? c4.z : c4.w));
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
        const float* base = S.in + SM::at(rg * 8, c);
        for (int t = 0; t < nt; ++t) {
            const float wt = S.wt[t];
            const float* p = base + S.off[t];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt, p[i * SM::IP], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) S.out[(rg * 8 + i) * PO + c] = acc[i];
    }
}

}  // namespace eecmg
