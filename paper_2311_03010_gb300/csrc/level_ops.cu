// level_ops.cu -- per-level operators of the cascade: restriction (Eqs.
// 12-13), the new extrapolation Pi and quadratic interpolation P (Section
// 3.2), linear prolongation L (Eq. 15), local smoothing S (Section 3.3,
// Eqs. 18-19) and one explicit Perona-Malik step D (Section 4, Eqs. 21-24).
// Each runs once per level per restoration; they are simple stencils with
// 32 x 8 thread blocks over the output image.
#include "launch.hpp"

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

// Pi on the level-(l-1) grid: u1 + (1/4) * (bilinear interpolant of
// d = u1|coarse - u2), i.e. (5 u1 - u2)/4 at coarse nodes, u1 + (d_a + d_b)/8
// at edge midpoints and u1 + (sum of four d)/16 at cell centres; indices
// past the last level-(l-2) node are clamped to it.  The differences of the
// two near-equal iterates are taken exactly (TwoSum: each is a double-float
// pair, as exact as an FP64 difference of two FP32 values) and summed in
// double-float, all on the FP32 pipes: GB300's FP64 pipe is narrow, and an
// FP64 form of this made the prolongation 20x slower than its memory traffic.
// The result is the double-float value rounded once to FP32.
__device__ __forceinline__ float pi_at(const float* __restrict__ u1, int w1,
                                      const float* __restrict__ u2, int h2, int w2, int a, int b) {
    const int A0 = a >> 1, B0 = b >> 1;
    const int A1 = (a & 1) ? min(A0 + 1, h2 - 1) : A0;
    const int B1 = (b & 1) ? min(B0 + 1, w2 - 1) : B0;
    auto d = [&](int A, int B) -> DF {
        return two_sum(u1[(size_t)(2 * A) * w1 + 2 * B], -u2[(size_t)A * w2 + B]);
    };
    const DF dsum = df_add2(df_add2(d(A0, B0), d(A0, B1)), df_add2(d(A1, B0), d(A1, B1)));
    const DF e = df_add2(DF{u1[(size_t)a * w1 + b], 0.f}, DF{0.0625f * dsum.hi, 0.0625f * dsum.lo});
    return __fadd_rn(e.hi, e.lo);
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

// Three-point Lagrange weights at offsets 0, 1/4, 1/2, 3/4 of a level-(l-2)
// cell spanned by the level-(l-1) triplet (2A, 2A+1, 2A+2).
__constant__ float c_qw[4][3] = {
    {1.f, 0.f, 0.f}, {0.375f, 0.75f, -0.125f}, {0.f, 1.f, 0.f}, {-0.125f, 0.75f, 0.375f}};

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

// S: weighted least-squares plane fit over the in-image 3 x 3 neighbourhood
// with weights exp(-(scale * (u_c - u_nb))^2) (Eqs. 18-19), output the fitted
// constant.  Solved in centred form: with W, the weighted means (sb, tb, vb)
// of the offsets and of v = u_nb - u_c, the 2 x 2 moment matrix C and the
// cross vector c, slope = C^+ c (eigenvalues below 1e-6 W dropped) and
// a0 = u_c + vb - slope . (sb, tb).
template <class Rd>
__device__ __forceinline__ float smooth_value_rd(Rd rd, int h, int w, float scale, int i, int j) {
    const float uc = rd(i, j);
    float ws[9], ss[9], ts[9], vs[9];
    float W = 0.f, sb = 0.f, tb = 0.f, vb = 0.f;
#pragma unroll
    for (int s = -1; s <= 1; ++s) {
#pragma unroll
        for (int t = -1; t <= 1; ++t) {
            const int k = (s + 1) * 3 + (t + 1);
            const int ii = i + s, jj = j + t;
            const bool inside = ii >= 0 && ii < h && jj >= 0 && jj < w;
            const float v = inside ? rd(ii, jj) - uc : 0.f;
            const float e = scale * v;
            const float wt = inside ? __expf(-e * e) : 0.f;  // MUFU exp: ~2 ulp, ample for a weight
            ws[k] = wt;
            ss[k] = (float)s;
            ts[k] = (float)t;
            vs[k] = v;
            W += wt;
            sb = fmaf(wt, (float)s, sb);
            tb = fmaf(wt, (float)t, tb);
            vb = fmaf(wt, v, vb);
        }
    }
    const float inv_w = 1.f / W;  // W >= 1: the centre always has weight 1
    sb *= inv_w;
    tb *= inv_w;
    vb *= inv_w;
    float css = 0.f, cst = 0.f, ctt = 0.f, csv = 0.f, ctv = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float ds = ss[k] - sb, dt = ts[k] - tb, dv = vs[k] - vb;
        const float wd = ws[k];
        css = fmaf(wd * ds, ds, css);
        cst = fmaf(wd * ds, dt, cst);
        ctt = fmaf(wd * dt, dt, ctt);
        csv = fmaf(wd * ds, dv, csv);
        ctv = fmaf(wd * dt, dv, ctv);
    }
    const float tr = 0.5f * (css + ctt), df = 0.5f * (css - ctt);
    const float rad = sqrtf(df * df + cst * cst);
    const float l1 = tr + rad;
    // small eigenvalue from the determinant: no cancellation
    const float l2 = l1 > 0.f ? (css * ctt - cst * cst) / l1 : 0.f;
    const float thr = 1e-6f * W;
    float e1s = 1.f, e1t = 0.f;
    if (rad > 0.f) {
        const float a0 = css - l2, c0 = ctt - l2;
        if (fabsf(a0) >= fabsf(c0)) {
            const float nn = rsqrtf(a0 * a0 + cst * cst);
            e1s = a0 * nn;
            e1t = cst * nn;
        } else {
            const float nn = rsqrtf(cst * cst + c0 * c0);
            e1s = cst * nn;
            e1t = c0 * nn;
        }
    }
    const float e2s = -e1t, e2t = e1s;
    float gs = 0.f, gt = 0.f;
    if (l1 > thr) {
        const float c1 = (e1s * csv + e1t * ctv) / l1;
        gs = fmaf(c1, e1s, gs);
        gt = fmaf(c1, e1t, gt);
    }
    if (l2 > thr) {
        const float c2 = (e2s * csv + e2t * ctv) / l2;
        gs = fmaf(c2, e2s, gs);
        gt = fmaf(c2, e2t, gt);
    }
    return uc + vb - (gs * sb + gt * tb);
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

// D: u + tau * sum over in-image 4-neighbours of (c_nb + c_c)/2 (u_nb - u_c),
// c = 1 / (1 + |grad u|^2 / k^2) with central differences (an out-of-image
// neighbour replaced by the centre value).
template <class Rd>
__device__ __forceinline__ float pm_c_rd(Rd u, int h, int w, int i, int j, float inv_k2) {
    const float uc = u(i, j);
    const float ue = (j + 1 < w) ? u(i, j + 1) : uc;
    const float uw = (j > 0) ? u(i, j - 1) : uc;
    const float us = (i + 1 < h) ? u(i + 1, j) : uc;
    const float un = (i > 0) ? u(i - 1, j) : uc;
    const float gx = 0.5f * (ue - uw), gy = 0.5f * (us - un);
    return 1.f / (1.f + (gx * gx + gy * gy) * inv_k2);
}
// c at (i, j) from a reader Cd of precomputed c, u from Ud.
template <class Ud, class Cd>
__device__ __forceinline__ float denoise_value_rd(Ud in, Cd c, int h, int w, float tau, int i, int j) {
    const float uc = in(i, j);
    const float cc = c(i, j);
    float f = 0.f;
    if (i + 1 < h) f += 0.5f * (c(i + 1, j) + cc) * (in(i + 1, j) - uc);
    if (i > 0) f += 0.5f * (c(i - 1, j) + cc) * (in(i - 1, j) - uc);
    if (j + 1 < w) f += 0.5f * (c(i, j + 1) + cc) * (in(i, j + 1) - uc);
    if (j > 0) f += 0.5f * (c(i, j - 1) + cc) * (in(i, j - 1) - uc);
    return fmaf(tau, f, uc);
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

// The start of a prolonged level (Algorithm 2, Step 2) in one pass: D(S(P(Pi(u1, u2)))) for
// one PSD_TH x PSD_TW block of fine pixels at (y0, x0).  D needs S's output with a 2-pixel halo
// (its own 4 neighbours and their diffusivities), S needs P's with a 1-pixel halo beyond that,
// and P the level-(l-1) window of Pi values its triplets read; each stage is computed for its
// whole region into shared memory (pixels outside the image are never read), with the
// per-pixel arithmetic of k_prolong, k_smooth and k_denoise, so the result equals those three
// kernels in sequence bitwise, while the two intermediate images never leave the SM.  Halo
// work: P on 1.30x, S on 1.20x, c on 1.10x the block's pixels.  Called by every thread of a
// 256-thread block.
constexpr int PSD_TH = 32, PSD_TW = 64;
constexpr int PSD_PH = PSD_TH + 6, PSD_PW = PSD_TW + 6;  // P: 3-pixel halo
constexpr int PSD_SH = PSD_TH + 4, PSD_SW = PSD_TW + 4;  // S: 2
constexpr int PSD_CH = PSD_TH + 2, PSD_CW = PSD_TW + 2;  // c: 1
// Pi window: n consecutive fine indices read level-(l-1) indices 2A .. 2A' + 2 with
// A' - A <= (n + 2) / 4
constexpr int PSD_XR = 2 * ((PSD_PH + 2) / 4) + 3, PSD_XC = 2 * ((PSD_PW + 2) / 4) + 3;
struct PsdSmem {
    float X[PSD_XR][PSD_XC];
    float P[PSD_PH][PSD_PW];
    float S[PSD_SH][PSD_SW];
    float C[PSD_CH][PSD_CW];
};
__device__ __forceinline__ void tile_psd(PsdSmem& M, const float* __restrict__ u1, int h1, int w1,
                                         const float* __restrict__ u2, int h2, int w2,
                                         float* __restrict__ out, int h, int w, float scale, float tau,
                                         float inv_k2, int y0, int x0) {
    const int tid = threadIdx.y * BX + threadIdx.x;
    constexpr int NT = BX * BY;
    // fine region of P (clipped to the image) and its Pi window
    const int py0 = max(y0 - 3, 0), px0 = max(x0 - 3, 0);
    const int py1 = min(y0 + PSD_TH + 3, h), px1 = min(x0 + PSD_TW + 3, w);  // exclusive
    const int r0 = 2 * (py0 >> 2), c0 = 2 * (px0 >> 2);
    const int nr = 2 * (((py1 - 1) >> 2) - (py0 >> 2)) + 3;
    const int nc = 2 * (((px1 - 1) >> 2) - (px0 >> 2)) + 3;
    for (int k = tid; k < nr * nc; k += NT) {
        const int rr = k / nc, cc = k - rr * nc;
        M.X[rr][cc] = pi_at(u1, w1, u2, h2, w2, min(r0 + rr, h1 - 1), min(c0 + cc, w1 - 1));
    }
    __syncthreads();
    // P on rows y0-3 .. y0+TH+2 and columns x0-3 .. x0+TW+2 (in-image part)
    for (int k = tid; k < PSD_PH * PSD_PW; k += NT) {
        const int rr = k / PSD_PW, cc = k - rr * PSD_PW;
        const int y = y0 - 3 + rr, x = x0 - 3 + cc;
        float acc = 0.f;
        if (y >= 0 && y < h && x >= 0 && x < w) {
            const int A = y >> 2, ty = y & 3, B = x >> 2, tx = x & 3;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                // staged row 2A + i - r0 holds level-(l-1) row min(2A + i, h1 - 1), as P reads
                const float* er = M.X[2 * A + i - r0];
                float row = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) row = fmaf(c_qw[tx][j], er[2 * B + j - c0], row);
                acc = fmaf(c_qw[ty][i], row, acc);
            }
        }
        M.P[rr][cc] = acc;
    }
    __syncthreads();
    auto pr = [&](int a, int b) { return M.P[a - y0 + 3][b - x0 + 3]; };
    for (int k = tid; k < PSD_SH * PSD_SW; k += NT) {
        const int rr = k / PSD_SW, cc = k - rr * PSD_SW;
        const int y = y0 - 2 + rr, x = x0 - 2 + cc;
        M.S[rr][cc] = (y >= 0 && y < h && x >= 0 && x < w) ? smooth_value_rd(pr, h, w, scale, y, x) : 0.f;
    }
    __syncthreads();
    auto sr = [&](int a, int b) { return M.S[a - y0 + 2][b - x0 + 2]; };
    for (int k = tid; k < PSD_CH * PSD_CW; k += NT) {
        const int rr = k / PSD_CW, cc = k - rr * PSD_CW;
        const int y = y0 - 1 + rr, x = x0 - 1 + cc;
        M.C[rr][cc] = (y >= 0 && y < h && x >= 0 && x < w) ? pm_c_rd(sr, h, w, y, x, inv_k2) : 0.f;
    }
    __syncthreads();
    auto cr = [&](int a, int b) { return M.C[a - y0 + 1][b - x0 + 1]; };
    for (int k = tid; k < PSD_TH * PSD_TW; k += NT) {
        const int rr = k / PSD_TW, cc = k - rr * PSD_TW;
        px_denoise_rd(sr, cr, out, h, w, tau, y0 + rr, x0 + cc);
    }
}

__global__ void __launch_bounds__(BX* BY) k_psd(const float* __restrict__ u1, int h1, int w1,
                                               const float* __restrict__ u2, int h2, int w2,
                                               float* __restrict__ out, int h, int w, float scale,
                                               float tau, float inv_k2) {
    __shared__ PsdSmem M;
    tile_psd(M, u1, h1, w1, u2, h2, w2, out, h, w, scale, tau, inv_k2, blockIdx.y * PSD_TH,
             blockIdx.x * PSD_TW);
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
        // this block's tile of the 32 x 64 grid (bx counts PSD_TW-wide tiles)
        tile_psd(M, it.a, it.h1, it.w1, it.b, it.h2, it.w2, it.out, it.h, it.w, it.s0, it.p0, it.p1,
                 by * PSD_TH, bx * PSD_TW);
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
    const dim3 grid((w + PSD_TW - 1) / PSD_TW, (h + PSD_TH - 1) / PSD_TH);
    k_psd<<<grid, dim3(BX, BY), 0, s>>>(u1, h1, w1, u2, h2, w2, out, h, w, scale, tau, 1.f / (kpm * kpm));
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
    if (op == OP_PSD) return ((w + PSD_TW - 1) / PSD_TW) * ((h + PSD_TH - 1) / PSD_TH);
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
