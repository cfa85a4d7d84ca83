// common.cuh -- shared device definitions of the EECMG CUDA library.
//
// Layout conventions: images are FP32, row-major, pitch = width.  A level's
// PSF is held in *correlation* form C(dy, dx) so that every kernel computes
//     y(i, j) = sum_{dy, dx} C(dy, dx) * x(i + dy, j + dx),   x = 0 outside,
// which is H (Eq. 7, zero boundary) with C(dy, dx) = K(-dy, -dx) and H^T
// with C = K.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eecmg.h"

namespace eecmg {

constexpr int RMAX = EECMG_MAX_RADIUS;
constexpr int KMAX = 2 * RMAX + 1;
constexpr int TAPS_MAX = KMAX * KMAX;

// One level's PSF in correlation form.  Device resident (plan-owned).
struct Taps {
    int ry, rx;           // radii: dy in [-ry, ry], dx in [-rx, rx]
    int rt;               // template radius used by the kernels (max(ry, rx))
    int sep;              // 1: C(dy, dx) = cy[dy + rt] * cx[dx + rt]
    int ntap;             // non-separable path: number of non-zero taps
    int pad[3];
    float cy[KMAX];       // separable factors, indexed by d + rt
    float cx[KMAX];
    int dy[TAPS_MAX];     // non-zero taps (dy, dx, weight)
    int dx[TAPS_MAX];
    float wt[TAPS_MAX];
};

// A double-float value hi + lo (two floats, |lo| <= ulp(hi) / 2).
struct DF {
    float hi, lo;
};

// Per-solve device scalars: totals and stopping limits in FP64 for the host,
// the Krylov recurrence scalars as double-float pairs.  One per level of a plan.
struct alignas(64) Scalars {
    double rr;            // last ||r||^2
    double gg;            // ||g||^2
    double lim2;          // stop when ||r||^2 <= lim2
    int stopped;          // 0 running; 1 stopping rule; 2 breakdown (no further step);
                          // 3 non-finite; 4 breakdown after deciding a last step
    int iters;            // iterations whose step has been decided
    unsigned int counter; // last-block arrival counter (reset by the last block)
    int loops;            // iterations whose first phase ran (for byte accounting)
    DF lim2d;             // lim2 as a double-float pair (the per-iteration tests)
    // MR-II early check (see fin_mr_b): a step applied ahead of its iteration's phase B
    DF lim2spec;          // threshold on the predicted ||r_k||^2 (-1: never predict)
    int spec;             // 1: the next phase applies step `iters` and checks ||r||
    int applied;          // the last step applied by such a check (0: none)
    double bpp;           // algorithmic bytes per pixel of the phases run so far
    // MR-II, Lanczos / Givens form (double-float scalars: see finish.cuh)
    DF nrm, nrm_prev;     // ||v_k||, ||v_{k-1}|| (w_k = v_k / ||v_k||)
    DF inv_nrm, inv_nrm_prev;  // their reciprocals
    DF alpha;             // alpha_k = <H w_k, w_k>
    DF cs1, sn1;          // rotation G_{k-1}
    DF cs2, sn2;          // rotation G_{k-2}
    DF phi;               // pending entry of the rotated right-hand side
    // pending step j: d_j = dw v_j - d1 d_{j-1} - d2 d_{j-2}  (= (w_j - r1 d_{j-1} -
    // e d_{j-2}) / rho), H d_j = dinv H w_j - d1 H d_{j-1} - d2 H d_{j-2},
    // u += tau d_j, r -= tau H d_j
    DF dw, d1, d2, dinv, tau;
    // CGLS
    DF gamma;             // <s, s>
    DF qq;                // <q, q>
    DF cg_alpha, beta;
    // FP32 coefficients for the vector phases, rounded once from the
    // scalars by the thread that updates them (no FP64 work per element)
    float f_scale;        // 1 / ||v_k||            (H w_k = f_scale * H v_k)
    float f_ca, f_cb;     // alpha_k / ||v_k||, ||v_k|| / ||v_{k-1}||
    float f_ca_lo, f_cb_lo;  // their FP32 rounding errors: v_{k+1} = H w - (ca + ca_lo) v - ...
                             // cancels to ~1e-4 of H w on near-scalar levels, where a
                             // single-float ca would stall the Lanczos recurrence
    float f_dw, f_d1, f_d2, f_dinv, f_tau;  // pending step
    float f_cg_alpha, f_beta;
};

constexpr int NTHREADS = 256;
constexpr int NPART = 4;  // partial sums per block

// ---------------------------------------------------------------------------
// Deterministic reductions.  Each thread sums a few products in FP32 (a
// handful of terms).  The warp and block trees add those partials in
// double-float (an FP32 pair kept exact by TwoSum, ~48-bit significand), so
// the tree runs on the FP32 pipes instead of the narrow FP64 pipe; each
// block's total is then one FP64 value, block b writing partials[b*NPART+j].
// The grid total is summed in a fixed order, so the result does not depend
// on block scheduling.
// ---------------------------------------------------------------------------

// Error-free sum of two floats (Knuth's TwoSum).
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return DF{s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return two_sum(s.hi, lo);
}

// ---------------------------------------------------------------------------
// Double-float scalar arithmetic for the solvers' scalar updates (Dekker's
// pair arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2, sums by
// Knuth's TwoSum, products made exact by one FMA).  On GB300 a dependent FP64
// FMA takes about 66 cycles and an FP64 reciprocal square root about 400;
// these run on the FP32 pipes in 4-cycle steps and keep 44-48 significant
// bits.  Every operation ends normalised, so hi is the value rounded to
// float.
// ---------------------------------------------------------------------------

// a + b when |a| >= |b| (or a == 0).
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// Sum keeping the rounding errors of both parts (accurate under cancellation).
__device__ __forceinline__ DF df_add2(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ DF df_sub2(DF a, DF b) { return df_add2(a, df_neg(b)); }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const DF p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ DF df_mulf(DF a, float b) {
    const DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// a / b: the float quotient corrected once by the remainder a - b q.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r = df_sub2(a, df_mulf(b, q1));
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// 1 / sqrt(x), x > 0: the FP32 estimate y refined by one Newton step
// y (1 + e / 2), e = 1 - x y^2 formed in double-float (relative error about
// 3 e^2 / 8, below 2^-44).  x is first scaled by 2^-80 or 2^80 when far from
// 1 so that y^2 stays in range.
__device__ __forceinline__ DF df_rsqrt(DF x) {
    float sc = 1.f;
    if (x.hi < 0x1p-60f) {
        x = DF{x.hi * 0x1p80f, x.lo * 0x1p80f};
        sc = 0x1p40f;
    } else if (x.hi > 0x1p60f) {
        x = DF{x.hi * 0x1p-80f, x.lo * 0x1p-80f};
        sc = 0x1p-40f;
    }
    const float y = rsqrtf(x.hi);
    const DF e = df_sub2(DF{1.f, 0.f}, df_mul(x, two_prod(y, y)));
    const DF c = two_prod(y, 0.5f * e.hi);
    const DF r = two_sum(y, c.hi);
    const DF n = fast_two_sum(r.hi, __fadd_rn(r.lo, c.lo));
    return DF{n.hi * sc, n.lo * sc};
}

// a <= b, a < b (normalised pairs compare by hi, then lo)
__device__ __forceinline__ bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool df_finite(DF a) { return isfinite(a.hi) && isfinite(a.lo); }

__device__ __forceinline__ DF df_from_double(double x) {
    const float hi = (float)x;
    return DF{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// Butterfly sums over groups of W lanes (W a power of two <= 32) of NV values
// at once: each level issues the shuffles of all values, then their adds, so
// the NV dependency chains overlap.  Same additions, in the same order, as
// NV separate warp_sum_df calls (zero lanes beyond W would add exact zeros).
template <int NV, int W = 32>
__device__ __forceinline__ void warp_sum_df_n(DF (&v)[NV]) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        DF w[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            w[j].hi = __shfl_xor_sync(0xffffffffu, v[j].hi, o);
            w[j].lo = __shfl_xor_sync(0xffffffffu, v[j].lo, o);
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = df_add(v[j], w[j]);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Block-wide double-float sum of NV values per thread, entirely on the FP32
// pipes (GB300's FP64 pipe is narrow).  Every lane of warp 0 returns lane
// 0's totals (the butterfly's lanes may differ in the last bit otherwise).
// Ends with __syncthreads().
template <int NV>
__device__ __forceinline__ void block_sum_df(const DF (&v)[NV], DF (&out)[NV]) {
    __shared__ DF red_df[NV][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    DF s[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = v[j];
    warp_sum_df_n<NV>(s);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) red_df[j][warp] = s[j];
    }
    __syncthreads();
    if (warp == 0) {
        DF t[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) t[j] = lane < NTHREADS / 32 ? red_df[j][lane] : DF{0.f, 0.f};
        warp_sum_df_n<NV, NTHREADS / 32>(t);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            out[j].hi = __shfl_sync(0xffffffffu, t[j].hi, 0);
            out[j].lo = __shfl_sync(0xffffffffu, t[j].lo, 0);
        }
    }
    __syncthreads();
}

// Block-wide sum of NV values per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(const double (&v)[NV], double (&out)[NV]) {
    __shared__ DF red[NV][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const DF s = warp_sum_df(df_from_double(v[j]));
        if (lane == 0) red[j][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            DF s = lane < NTHREADS / 32 ? red[j][lane] : DF{0.f, 0.f};
            s = warp_sum_df(s);
            out[j] = (double)s.hi + (double)s.lo;
        }
    }
    __syncthreads();
}

// Writes this block's partials and returns true in every thread of the last
// block to arrive.  Must be called by all threads of the block.
template <int NV>
__device__ __forceinline__ bool block_partials_arrive(const double (&v)[NV], double* partials,
                                                      unsigned int* counter, unsigned int nblocks,
                                                      unsigned int bid) {
    double out[NV];
    block_sum<NV>(v, out);
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)bid * NPART + j] = out[j];
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == nblocks - 1);
    }
    __syncthreads();
    return is_last;
}

// In the last block: fixed-order sum of all blocks' partials.  Result in
// thread 0 (out), and the counter is reset for the next launch.
template <int NV>
__device__ __forceinline__ void grid_total(const double* partials, unsigned int nblocks,
                                           unsigned int* counter, double (&out)[NV]) {
    __threadfence();
    double v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = 0.0;
    for (unsigned int b = threadIdx.x; b < nblocks; b += NTHREADS) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] += __ldcg(partials + (size_t)b * NPART + j);
    }
    block_sum<NV>(v, out);
    if (threadIdx.x == 0) *counter = 0u;
}

__device__ __forceinline__ bool finite_pos(double x) { return x > 0.0 && x < 1.0e300; }

// float4 helpers (vectors are 256-byte aligned; index q addresses pixels 4q..4q+3)
__device__ __forceinline__ float4 ld4cg(const float* p, size_t q) {
    return __ldcg(reinterpret_cast<const float4*>(p) + q);
}
__device__ __forceinline__ void st4(float* p, size_t q, float4 v) {
    reinterpret_cast<float4*>(p)[q] = v;
}
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 mul4(float a, float4 x) {
    return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}
// Coherent (L2) element and float4 access to a vector stored as T (FP32, or
// BF16 for the streamed vectors of the BF16-storage variant).  BF16 values
// are rounded to nearest even on store and widened exactly on load.
template <typename T>
struct VecIO;
template <>
struct VecIO<float> {
    static __device__ __forceinline__ float ld(const float* p, size_t i) { return __ldcg(p + i); }
    static __device__ __forceinline__ void st(float* p, size_t i, float v) { p[i] = v; }
    static __device__ __forceinline__ float4 ld4(const float* p, size_t q) {
        return __ldcg(reinterpret_cast<const float4*>(p) + q);
    }
    static __device__ __forceinline__ void st4(float* p, size_t q, float4 v) {
        reinterpret_cast<float4*>(p)[q] = v;
    }
};
template <>
struct VecIO<__nv_bfloat16> {
    static __device__ __forceinline__ float widen(unsigned int bits16) {
        return __uint_as_float(bits16 << 16);
    }
    static __device__ __forceinline__ unsigned int narrow(float v) {
        return (unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) {
        return widen(__ldcg(reinterpret_cast<const unsigned short*>(p) + i));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, size_t i, float v) {
        p[i] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float4 ld4(const __nv_bfloat16* p, size_t q) {
        const uint2 w = __ldcg(reinterpret_cast<const uint2*>(p) + q);
        return make_float4(widen(w.x & 0xffffu), widen(w.x >> 16), widen(w.y & 0xffffu),
                           widen(w.y >> 16));
    }
    static __device__ __forceinline__ void st4(__nv_bfloat16* p, size_t q, float4 v) {
        uint2 w;
        w.x = narrow(v.x) | (narrow(v.y) << 16);
        w.y = narrow(v.z) | (narrow(v.w) << 16);
        reinterpret_cast<uint2*>(p)[q] = w;
    }
};

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

}  // namespace eecmg
