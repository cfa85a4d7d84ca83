// level_ops.cu -- per-level operators of the cascade: restriction (Eqs.
// 12-13), the new extrapolation Pi and quadratic interpolation P (Section
// 3.2), linear prolongation L (Eq. 15), local smoothing S (Section 3.3,
// Eqs. 18-19) and one explicit Perona-Malik step D (Section 4, Eqs. 21-24).
// Each runs once per level per restoration; they are simple stencils with
// 32 x 8 thread blocks over the output image.
#include "launch.hpp"
#include "level_ops.cuh"

namespace eecmg {

namespace {
constexpr int BX = 32, BY = 8;
inline dim3 grid2(int h, int w) { return dim3((w + BX - 1) / BX, (h + BY - 1) / BY); }
}  // namespace

// g_l(a, b) = g_{l+1}(2a, 2b): the paper's 1-based 2k - 1, per dimension.
// step = 2^j restricts j levels at once: g_{l}(a, b) = g_{l+j}(2^j a, 2^j b).
__device__ __forceinline__ void px_restrict(const float* __restrict__ fine, int wf,
                                            float* __restrict__ coarse, int hc, int wc, int a, int b,
                                            int step = 2) {
    if (a < hc && b < wc) coarse[(size_t)a * wc + b] = fine[(size_t)(step * a) * wf + step * b];
}
__global__ void k_restrict(const float* __restrict__ fine, int wf, float* __restrict__ coarse,
                           int hc, int wc) {
    px_restrict(fine, wf, coarse, hc, wc, blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x);
}

__device__ __forceinline__ void px_extrapolate(const float* __restrict__ u1, int h1, int w1,
                                               const float* __restrict__ u2, int h2, int w2,
                                               float* __restrict__ out, int a, int b) {
    if (a >= h1 || b >= w1) return;
    out[(size_t)a * w1 + b] = pi_at(u1, w1, u2, h2, w2, a, b);
}
__global__ void k_extrapolate(const float* __restrict__ u1, int h1, int w1,
                              const float* __restrict__ u2, int h2, int w2,
                              float* __restrict__ out) {
    px_extrapolate(u1, h1, w1, u2, h2, w2, out, blockIdx.y * BY + threadIdx.y,
                   blockIdx.x * BX + threadIdx.x);
}

// P: tensor-product quadratic interpolation of ut (h1 x w1) onto h x w.
__device__ __forceinline__ void px_quadratic(const float* __restrict__ ut, int h1, int w1,
                                             float* __restrict__ out, int h, int w, int y, int x) {
    if (y >= h || x >= w) return;
    const int A = y >> 2, ty = y & 3, B = x >> 2, tx = x & 3;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int ar = min(2 * A + i, h1 - 1);
        float row = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int bc = min(2 * B + j, w1 - 1);
            row = fmaf(c_qw[tx][j], ut[(size_t)ar * w1 + bc], row);
        }
        s = fmaf(c_qw[ty][i], row, s);
    }
    out[(size_t)y * w + x] = s;
}
__global__ void k_quadratic(const float* __restrict__ ut, int h1, int w1, float* __restrict__ out,
                            int h, int w) {
    px_quadratic(ut, h1, w1, out, h, w, blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x);
}

// The nonlinear prolongation P(Pi(u1, u2)) of Section 3.2 fused for one
// BY x BX block of fine pixels at (y0, x0): the level-(l-1) values of Pi that
// the block's quadratic interpolation reads (a window of at most 7 x 19,
// indices clamped as in P) are computed into shared memory first, with the
// same arithmetic as k_extrapolate, then P reads them as k_quadratic reads
// its input.  The result equals k_extrapolate followed by k_quadratic, without
// the round trip of Pi's output through memory.  Called by every thread of
// the block.
constexpr int PI_ROWS = 2 * ((BY + 3) / 4) + 3, PI_COLS = 2 * ((BX + 3) / 4) + 3;
__device__ __forceinline__ void tile_prolong(const float* __restrict__ u1, int h1, int w1,
                                             const float* __restrict__ u2, int h2, int w2,
                                             float* __restrict__ out, int h, int w, int y0, int x0) {
    __shared__ float ext[PI_ROWS][PI_COLS];
    const int r0 = 2 * (y0 >> 2), c0 = 2 * (x0 >> 2);
    const int nr = 2 * (((y0 + BY - 1) >> 2) - (y0 >> 2)) + 3;
    const int nc = 2 * (((x0 + BX - 1) >> 2) - (x0 >> 2)) + 3;
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int k = tid; k < nr * nc; k += BX * BY) {
        const int rr = k / nc, cc = k - rr * nc;
        ext[rr][cc] = pi_at(u1, w1, u2, h2, w2, min(r0 + rr, h1 - 1), min(c0 + cc, w1 - 1));
    }
    __syncthreads();
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    if (y >= h || x >= w) return;
    const int A = y >> 2, ty = y & 3, B = x >> 2, tx = x & 3;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // staged row 2A + i - r0 holds level-(l-1) row min(2A + i, h1 - 1), as P reads
        const float* er = ext[2 * A + i - r0];
        float row = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) row = fmaf(c_qw[tx][j], er[2 * B + j - c0], row);
        acc = fmaf(c_qw[ty][i], row, acc);
    }
    out[(size_t)y * w + x] = acc;
}
__global__ void __launch_bounds__(BX* BY) k_prolong(const float* __restrict__ u1, int h1, int w1,
                                                   const float* __restrict__ u2, int h2, int w2,
                                                   float* __restrict__ out, int h, int w) {
    tile_prolong(u1, h1, w1, u2, h2, w2, out, h, w, blockIdx.y * BY, blockIdx.x * BX);
}

// L of Eq. 15 in 0-based indices: copy at (2a, 2b); horizontal / vertical
// averages at (2a, 2b+1) / (2a+1, 2b); the diagonal pair (a, b), (a+1, b+1)
// at (2a+1, 2b+1).  Indices past the last coarse node are clamped.
__device__ __forceinline__ void px_linear(const float* __restrict__ uc, int hc, int wc,
                                          float* __restrict__ out, int h, int w, int y, int x) {
    if (y >= h || x >= w) return;
    const int a = y >> 1, b = x >> 1;
    const int a1 = min(a + 1, hc - 1), b1 = min(b + 1, wc - 1);
    const float u00 = uc[(size_t)a * wc + b];
    float v;
    if (!(y & 1) && !(x & 1)) v = u00;
    else if (!(y & 1)) v = 0.5f * (u00 + uc[(size_t)a * wc + b1]);
    else if (!(x & 1)) v = 0.5f * (u00 + uc[(size_t)a1 * wc + b]);
    else v = 0.5f * (u00 + uc[(size_t)a1 * wc + b1]);
    out[(size_t)y * w + x] = v;
}
__global__ void k_linear(const float* __restrict__ uc, int hc, int wc, float* __restrict__ out,
                         int h, int w) {
    px_linear(uc, hc, wc, out, h, w, blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x);
}

template <class Rd>
__device__ __forceinline__ void px_smooth_rd(Rd rd, float* __restrict__ out, int h, int w, float scale,
                                             int i, int j) {
    if (i >= h || j >= w) return;
    out[(size_t)i * w + j] = smooth_value_rd(rd, h, w, scale, i, j);
}
// S for one BY x BX block at (y0, x0): the input with a 1-pixel halo is staged
// in shared memory once (the 3 x 3 fits read it nine times); same arithmetic
// as the per-pixel form px_smooth_rd.  Called by every thread of the block.
__device__ __forceinline__ void tile_smooth(const float* __restrict__ in, float* __restrict__ out,
                                            int h, int w, float scale, int y0, int x0) {
    __shared__ float U[BY + 2][BX + 2];
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int k = tid; k < (BY + 2) * (BX + 2); k += BX * BY) {
        const int r = k / (BX + 2), c = k - r * (BX + 2);
        const int gy = y0 - 1 + r, gx = x0 - 1 + c;
        U[r][c] = (gy >= 0 && gy < h && gx >= 0 && gx < w) ? in[(size_t)gy * w + gx] : 0.f;
    }
    __syncthreads();
    px_smooth_rd([&](int a, int b) { return U[a - y0 + 1][b - x0 + 1]; }, out, h, w, scale,
                 y0 + threadIdx.y, x0 + threadIdx.x);
}

__global__ void __launch_bounds__(BX* BY) k_smooth(const float* __restrict__ in, float* __restrict__ out,
                                                  int h, int w, float scale) {
    tile_smooth(in, out, h, w, scale, blockIdx.y * BY, blockIdx.x * BX);
}

template <class Ud, class Cd>
__device__ __forceinline__ void px_denoise_rd(Ud in, Cd c, float* __restrict__ out, int h, int w,
                                              float tau, int i, int j) {
    if (i >= h || j >= w) return;
    out[(size_t)i * w + j] = denoise_value_rd(in, c, h, w, tau, i, j);
}
// D for one BY x BX block at (y0, x0): the input with a 2-pixel halo and the
// diffusivities c with a 1-pixel halo are staged in shared memory (c computed
// once per pixel instead of five times); same arithmetic as the per-pixel form.
// Called by every thread of the block.
__device__ __forceinline__ void tile_denoise(const float* __restrict__ in, float* __restrict__ out,
                                             int h, int w, float tau, float inv_k2, int y0, int x0) {
    __shared__ float U[BY + 4][BX + 4];
    __shared__ float C[BY + 2][BX + 2];
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int k = tid; k < (BY + 4) * (BX + 4); k += BX * BY) {
        const int r = k / (BX + 4), cc = k - r * (BX + 4);
        const int gy = y0 - 2 + r, gx = x0 - 2 + cc;
        U[r][cc] = (gy >= 0 && gy < h && gx >= 0 && gx < w) ? in[(size_t)gy * w + gx] : 0.f;
    }
    __syncthreads();
    auto u = [&](int a, int b) { return U[a - y0 + 2][b - x0 + 2]; };
    for (int k = tid; k < (BY + 2) * (BX + 2); k += BX * BY) {
        const int r = k / (BX + 2), cc = k - r * (BX + 2);
        const int gy = y0 - 1 + r, gx = x0 - 1 + cc;
        // only in-image pixels are ever read back
        C[r][cc] = (gy >= 0 && gy < h && gx >= 0 && gx < w) ? pm_c_rd(u, h, w, gy, gx, inv_k2) : 0.f;
    }
    __syncthreads();
    px_denoise_rd(u, [&](int a, int b) { return C[a - y0 + 1][b - x0 + 1]; }, out, h, w, tau,
                  y0 + threadIdx.y, x0 + threadIdx.x);
}

__global__ void __launch_bounds__(BX* BY) k_denoise(const float* __restrict__ in, float* __restrict__ out,
                                                   int h, int w, float tau, float inv_k2) {
    tile_denoise(in, out, h, w, tau, inv_k2, blockIdx.y * BY, blockIdx.x * BX);
}

__global__ void __launch_bounds__(BX* BY) k_psd(const float* __restrict__ u1, int h1, int w1,
                                               const float* __restrict__ u2, int h2, int w2,
                                               float* __restrict__ out, int h, int w, float scale,
                                               float tau, float inv_k2, int th) {
    __shared__ PsdSmem M;
    const int y0 = blockIdx.y * th, x0 = blockIdx.x * PSD_TW;
    auto store = [&](int rr, int cc, float v) { out[(size_t)(y0 + rr) * w + x0 + cc] = v; };
    if (th == 16)
        tile_psd<16>(M, u1, h1, w1, u2, h2, w2, h, w, scale, tau, inv_k2, y0, x0, store);
    else
        tile_psd<PSD_TH>(M, u1, h1, w1, u2, h2, w2, h, w, scale, tau, inv_k2, y0, x0, store);
}

// Many operations of one kind in one launch (the server's ticks): block b
// serves the item whose block range holds b (binary search over block0),
// with the same per-pixel code as the single launches above.
template <int OP>
__global__ void __launch_bounds__(BX* BY) k_ops_batch(const OpItem* __restrict__ items, int n) {
    const int blk = (int)blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].block0 <= blk) lo = mid;
        else hi = mid - 1;
    }
    const OpItem& it = items[lo];
    const int local = blk - it.block0;
    const int by = local / it.bx, bx = local - by * it.bx;
    const int x = bx * BX + threadIdx.x, y = by * BY + threadIdx.y;
    if constexpr (OP == OP_RESTRICT) px_restrict(it.a, it.w1, it.out, it.h, it.w, y, x, it.h2);
    if constexpr (OP == OP_EXTRAPOLATE) px_extrapolate(it.a, it.h1, it.w1, it.b, it.h2, it.w2, it.out, y, x);
    if constexpr (OP == OP_QUADRATIC) px_quadratic(it.a, it.h1, it.w1, it.out, it.h, it.w, y, x);
    if constexpr (OP == OP_LINEAR) px_linear(it.a, it.h1, it.w1, it.out, it.h, it.w, y, x);
    if constexpr (OP == OP_SMOOTH) tile_smooth(it.a, it.out, it.h, it.w, it.p0, by * BY, bx * BX);
    if constexpr (OP == OP_DENOISE) tile_denoise(it.a, it.out, it.h, it.w, it.p0, it.p1, by * BY, bx * BX);
    if constexpr (OP == OP_PROLONG)
        tile_prolong(it.a, it.h1, it.w1, it.b, it.h2, it.w2, it.out, it.h, it.w, by * BY, bx * BX);
    if constexpr (OP == OP_PSD) {
        __shared__ PsdSmem M;
        // this block's tile of the th x 64 grid (bx counts PSD_TW-wide tiles)
        const int y0 = by * it.th, x0 = bx * PSD_TW;
        float* out = it.out;
        const int w = it.w;
        auto store = [&](int rr, int cc, float v) { out[(size_t)(y0 + rr) * w + x0 + cc] = v; };
        if (it.th == 16)
            tile_psd<16>(M, it.a, it.h1, it.w1, it.b, it.h2, it.w2, it.h, it.w, it.s0, it.p0, it.p1, y0, x0, store);
        else
            tile_psd<PSD_TH>(M, it.a, it.h1, it.w1, it.b, it.h2, it.w2, it.h, it.w, it.s0, it.p0, it.p1, y0, x0,
                             store);
    }
    if constexpr (OP == OP_ZERO || OP == OP_COPY) {
        if (y < it.h && x < it.w) it.out[(size_t)y * it.w + x] = OP == OP_ZERO ? 0.f : it.a[(size_t)y * it.w + x];
    }
}

namespace {
template <int OP>
cudaError_t launch_op(const OpItem* d_items, int n, int total_blocks, cudaStream_t s) {
    k_ops_batch<OP><<<dim3((unsigned int)total_blocks), dim3(BX, BY), 0, s>>>(d_items, n);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_restrict(const float* fine, int hf, int wf, float* coarse, int hc, int wc,
                            cudaStream_t s) {
    (void)hf;
    if (hc <= 0 || wc <= 0) return cudaSuccess;
    k_restrict<<<grid2(hc, wc), dim3(BX, BY), 0, s>>>(fine, wf, coarse, hc, wc);
    return cudaGetLastError();
}

cudaError_t launch_extrapolate(const float* u1, int h1, int w1, const float* u2, int h2, int w2,
                               float* out, cudaStream_t s) {
    if (h1 <= 0 || w1 <= 0) return cudaSuccess;
    k_extrapolate<<<grid2(h1, w1), dim3(BX, BY), 0, s>>>(u1, h1, w1, u2, h2, w2, out);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const float* u1, int h1, int w1, const float* u2, int h2, int w2,
                           float* out, int h, int w, cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    k_prolong<<<grid2(h, w), dim3(BX, BY), 0, s>>>(u1, h1, w1, u2, h2, w2, out, h, w);
    return cudaGetLastError();
}

cudaError_t launch_psd(const float* u1, int h1, int w1, const float* u2, int h2, int w2, float* out,
                       int h, int w, float scale, float tau, float kpm, cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    const int th = psd_tile_rows();
    const dim3 grid((w + PSD_TW - 1) / PSD_TW, (h + th - 1) / th);
    k_psd<<<grid, dim3(BX, BY), 0, s>>>(u1, h1, w1, u2, h2, w2, out, h, w, scale, tau, 1.f / (kpm * kpm), th);
    return cudaGetLastError();
}

cudaError_t launch_quadratic(const float* ut, int h1, int w1, float* out, int h, int w,
                             cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    k_quadratic<<<grid2(h, w), dim3(BX, BY), 0, s>>>(ut, h1, w1, out, h, w);
    return cudaGetLastError();
}

cudaError_t launch_linear(const float* uc, int hc, int wc, float* out, int h, int w,
                          cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    k_linear<<<grid2(h, w), dim3(BX, BY), 0, s>>>(uc, hc, wc, out, h, w);
    return cudaGetLastError();
}

cudaError_t launch_smooth(const float* in, float* out, int h, int w, float scale, cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    k_smooth<<<grid2(h, w), dim3(BX, BY), 0, s>>>(in, out, h, w, scale);
    return cudaGetLastError();
}

cudaError_t launch_denoise(const float* in, float* out, int h, int w, float tau, float kpm,
                           cudaStream_t s) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    k_denoise<<<grid2(h, w), dim3(BX, BY), 0, s>>>(in, out, h, w, tau, 1.f / (kpm * kpm));
    return cudaGetLastError();
}

int op_blocks(int op, int h, int w) {
    if (h <= 0 || w <= 0) return 0;
    if (op == OP_PSD) return ((w + PSD_TW - 1) / PSD_TW) * ((h + psd_tile_rows() - 1) / psd_tile_rows());
    const dim3 g = grid2(h, w);
    return (int)(g.x * g.y);
}

int op_blocks_x(int op, int w) { return op == OP_PSD ? (w + PSD_TW - 1) / PSD_TW : (w + BX - 1) / BX; }

cudaError_t launch_ops_batch(int op, const OpItem* d_items, int n, int total_blocks, cudaStream_t s) {
    if (n <= 0 || total_blocks <= 0) return cudaSuccess;
    switch (op) {
        case OP_RESTRICT: return launch_op<OP_RESTRICT>(d_items, n, total_blocks, s);
        case OP_EXTRAPOLATE: return launch_op<OP_EXTRAPOLATE>(d_items, n, total_blocks, s);
        case OP_QUADRATIC: return launch_op<OP_QUADRATIC>(d_items, n, total_blocks, s);
        case OP_LINEAR: return launch_op<OP_LINEAR>(d_items, n, total_blocks, s);
        case OP_SMOOTH: return launch_op<OP_SMOOTH>(d_items, n, total_blocks, s);
        case OP_DENOISE: return launch_op<OP_DENOISE>(d_items, n, total_blocks, s);
        case OP_ZERO: return launch_op<OP_ZERO>(d_items, n, total_blocks, s);
        case OP_COPY: return launch_op<OP_COPY>(d_items, n, total_blocks, s);
        case OP_PROLONG: return launch_op<OP_PROLONG>(d_items, n, total_blocks, s);
        case OP_PSD: return launch_op<OP_PSD>(d_items, n, total_blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
