// launch.hpp -- host-side launchers of the EECMG kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace eecmg {

// Epilogues fused into the convolution y = C (*) x.
enum ConvMode : int {
    CM_STORE = 0,   // y = C (*) x
    CM_RESID = 1,   // r = g - H u (e0 = g; y2 = optional copy): ||r||^2, ||g||^2 -> limit, stop test
    CM_MR_V1 = 2,   // v_1 = H r_0 (x = r_0): <v_1, v_1>, <v_1, r_0> -> ||v_1||, phi_1
    CM_MR_A = 3,    // H w_k = H v_k / ||v_k|| (x = v_k): <H w_k, w_k> -> alpha_k
    CM_CG_S0 = 4,   // s = H^T r, p = s (y2): <s, s> -> gamma
    CM_CG_Q = 5,    // q = H p: <q, q> -> alpha = gamma / <q, q>
    CM_CG_S = 6,    // s = H^T r: <s, s> -> beta, gamma
};

struct ConvArgs {
    const float* x = nullptr;
    float* y = nullptr;
    float* y2 = nullptr;
    const float* e0 = nullptr;
    const float* e1 = nullptr;
    const Taps* taps = nullptr;
    Scalars* sc = nullptr;
    double* partials = nullptr;
    double conv_tol2 = 0.0;
    double disc2 = 0.0;
    int h = 0, w = 0;
    int mode = CM_STORE;
    int has_e1 = 0;
    int zero_input = 0;
};

// Tile of the convolution kernels.
constexpr int CONV_TH = 32;
constexpr int CONV_TW = 64;

inline unsigned int conv_blocks(int h, int w) {
    return (unsigned int)(((w + CONV_TW - 1) / CONV_TW) * ((h + CONV_TH - 1) / CONV_TH));
}

// Elementwise kernels: 8 elements per thread.
constexpr int EW_PER_BLOCK = NTHREADS * 8;
inline unsigned int ew_blocks(size_t n) {
    return (unsigned int)((n + EW_PER_BLOCK - 1) / EW_PER_BLOCK);
}

cudaError_t launch_conv(const ConvArgs& a, int rt, int sep, int prec, cudaStream_t s);

// MR-II (Lanczos / Givens form), phase B of iteration k: applies the
// pending step k-1 (d, Hd, u, r), forms v_{k+1} and reduces ||r||^2,
// <v_{k+1}, v_{k+1}>, <v_{k+1}, r_{k-1}>; the last block applies the stopping
// rules and the Givens rotation of column k.  Buffers are indexed by step
// parity: v[k & 1] = v_k, aw[k & 1] = H w_k, d/hd[j & 1] = d_j / H d_j.
struct MrVecs {
    float* v[2];
    float* aw[2];
    float* d[2];
    float* hd[2];
    float* u;
    float* r;
};
cudaError_t launch_mr_b(const MrVecs& V, int k, size_t n, Scalars* sc, double* partials,
                        cudaStream_t s);
// Applies the pending step (index read on the device) and reduces ||r||^2.
cudaError_t launch_mr_final(const MrVecs& V, size_t n, Scalars* sc, double* partials,
                            cudaStream_t s);
// CGLS: u += alpha p, r -= alpha q, ||r||^2 and the stopping rule.
cudaError_t launch_cg_step(float* u, const float* p, float* r, const float* q, size_t n,
                           Scalars* sc, double* partials, cudaStream_t s);
// CGLS: p = s + beta p.
cudaError_t launch_cg_p(float* p, const float* sv, size_t n, Scalars* sc, cudaStream_t s);

// Level operators.
// Batched per-level operations (one launch per kind for many images).
enum OpKind : int {
    OP_RESTRICT = 0, OP_EXTRAPOLATE, OP_QUADRATIC, OP_LINEAR, OP_SMOOTH, OP_DENOISE, OP_ZERO, OP_COPY,
    OP_PROLONG, OP_PSD, OP_KINDS
};
// One image's operation: output grid h x w (restriction: the coarse grid,
// w1 = fine width; Pi: the level-(l-1) grid, inputs h1 x w1 and h2 x w2;
// fused P(Pi): output h x w, inputs a = u_{l-1} (h1 x w1), b = u_{l-2} (h2 x w2);
// P / L: input h1 x w1; S: p0 = scale; D: p0 = tau, p1 = 1 / k^2; fused D(S(P(Pi))):
// the inputs of P(Pi), s0 = scale, p0 = tau, p1 = 1 / k^2).  bx and
// block0 place its blocks within the launch (filled by the host).
struct OpItem {
    const float* a = nullptr;
    const float* b = nullptr;
    float* out = nullptr;
    int h = 0, w = 0, h1 = 0, w1 = 0, h2 = 0, w2 = 0;
    float p0 = 0.f, p1 = 0.f, s0 = 0.f;
    int bx = 0, block0 = 0;
    int th = 0;  // OP_PSD: rows of the item's tiles
};
int op_blocks(int op, int h, int w);  // blocks of operation kind op covering an h x w output
int psd_tile_rows();                  // rows of the fused level start's tiles (process-wide tuning)
int op_blocks_x(int op, int w);       // of which along x
cudaError_t launch_ops_batch(int op, const OpItem* d_items, int n, int total_blocks, cudaStream_t s);

cudaError_t launch_restrict(const float* fine, int hf, int wf, float* coarse, int hc, int wc,
                            cudaStream_t s);
cudaError_t launch_extrapolate(const float* u1, int h1, int w1, const float* u2, int h2, int w2,
                               float* out, cudaStream_t s);
// The nonlinear prolongation P(Pi(u1, u2)) of Section 3.2 in one pass (out h x w).
cudaError_t launch_prolong(const float* u1, int h1, int w1, const float* u2, int h2, int w2,
                           float* out, int h, int w, cudaStream_t s);
// D(S(P(Pi(u1, u2)))) in one pass (out h x w): the start of a prolonged level of Algorithm 2
// with one Perona-Malik step.
cudaError_t launch_psd(const float* u1, int h1, int w1, const float* u2, int h2, int w2, float* out,
                       int h, int w, float scale, float tau, float kpm, cudaStream_t s);
cudaError_t launch_quadratic(const float* ut, int h1, int w1, float* out, int h, int w,
                             cudaStream_t s);
cudaError_t launch_linear(const float* uc, int hc, int wc, float* out, int h, int w,
                          cudaStream_t s);
cudaError_t launch_smooth(const float* in, float* out, int h, int w, float scale, cudaStream_t s);
cudaError_t launch_denoise(const float* in, float* out, int h, int w, float tau, float kpm,
                           cudaStream_t s);

}  // namespace eecmg
