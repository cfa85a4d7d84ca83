// level_ops.cuh -- per-pixel arithmetic of the per-level operators of the
// cascade (Section 3.2: the new extrapolation Pi and quadratic interpolation P;
// Section 3.3: local smoothing S; Section 4: the Perona-Malik step D) and the
// fused start of a prolonged level, D(S(P(Pi))), over one 32 x 64 tile.
// Shared by the standalone operator kernels (level_ops.cu) and the level
// solvers, whose first phase can start a level itself, so that every path
// runs the same arithmetic.
#pragma once

#include "common.cuh"

namespace eecmg {

// Pi on the level-(l-1) grid: u1 + (1/4) * (bilinear interpolant of
// d = u1|coarse - u2), i.e. (5 u1 - u2)/4 at coarse nodes, u1 + (d_a + d_b)/8
// at edge midpoints and u1 + (sum of four d)/16 at cell centres; indices
// past the last level-(l-2) node are clamped to it.  The differences of the
// two near-equal iterates are taken exactly (TwoSum: each is a double-float
// pair, as exact as an FP64 difference of two FP32 values) and summed in
// double-float, all on the FP32 pipes: GB300's FP64 pipe is narrow, and an
// FP64 form of this made the prolongation 20x slower than its memory traffic.
// The result is the double-float value rounded once to FP32.
// Pi from the centre value u1(a, b) and the four exact differences d of the
// level-(l-2) nodes around it (d00 = d(A0, B0), d01 = d(A0, B1), ...).
__device__ __forceinline__ float pi_from(float u1c, DF d00, DF d01, DF d10, DF d11) {
    const DF dsum = df_add2(df_add2(d00, d01), df_add2(d10, d11));
    const DF e = df_add2(DF{u1c, 0.f}, DF{0.0625f * dsum.hi, 0.0625f * dsum.lo});
    return __fadd_rn(e.hi, e.lo);
}
// The exact difference d(A, B) = u1(2A, 2B) - u2(A, B) as a double-float pair.
__device__ __forceinline__ DF pi_diff(const float* __restrict__ u1, int w1, const float* __restrict__ u2,
                                      int w2, int A, int B) {
    return two_sum(u1[(size_t)(2 * A) * w1 + 2 * B], -u2[(size_t)A * w2 + B]);
}
// The level-(l-2) nodes (A0, A1) x (B0, B1) that Pi at (a, b) reads.
__device__ __forceinline__ void pi_nodes(int a, int b, int h2, int w2, int& A0, int& A1, int& B0, int& B1) {
    A0 = a >> 1;
    B0 = b >> 1;
    A1 = (a & 1) ? min(A0 + 1, h2 - 1) : A0;
    B1 = (b & 1) ? min(B0 + 1, w2 - 1) : B0;
}
__device__ __forceinline__ float pi_at(const float* __restrict__ u1, int w1,
                                      const float* __restrict__ u2, int h2, int w2, int a, int b) {
    int A0, A1, B0, B1;
    pi_nodes(a, b, h2, w2, A0, A1, B0, B1);
    return pi_from(u1[(size_t)a * w1 + b], pi_diff(u1, w1, u2, w2, A0, B0), pi_diff(u1, w1, u2, w2, A0, B1),
                   pi_diff(u1, w1, u2, w2, A1, B0), pi_diff(u1, w1, u2, w2, A1, B1));
}
// Three-point Lagrange weights at offsets 0, 1/4, 1/2, 3/4 of a level-(l-2)
// cell spanned by the level-(l-1) triplet (2A, 2A+1, 2A+2).
static __constant__ float c_qw[4][3] = {
    {1.f, 0.f, 0.f}, {0.375f, 0.75f, -0.125f}, {0.f, 1.f, 0.f}, {-0.125f, 0.75f, 0.375f}};

// S: weighted least-squares plane fit over the in-image 3 x 3 neighbourhood
// with weights exp(-(scale * (u_c - u_nb))^2) (Eqs. 18-19), output the fitted
// constant.  Solved in centred form: with W, the weighted means (sb, tb, vb)
// of the offsets and of v = u_nb - u_c, the 2 x 2 moment matrix C and the
// cross vector c, slope = C^+ c (eigenvalues below 1e-6 W dropped) and
// a0 = u_c + vb - slope . (sb, tb).
// EDGE = false: the caller guarantees that the whole 3 x 3 neighbourhood lies in
// the image (the same arithmetic without the bounds tests).
template <bool EDGE = true, class Rd>
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
            const bool inside = !EDGE || (ii >= 0 && ii < h && jj >= 0 && jj < w);
            // the centre term is v = 0, weight exp(0) = 1 exactly (as the exponential gives it)
            const bool ctr = s == 0 && t == 0;
            const float v = ctr ? 0.f : (inside ? rd(ii, jj) - uc : 0.f);
            const float e = scale * v;
            const float wt = ctr ? 1.f : (inside ? __expf(-e * e) : 0.f);  // MUFU exp: ~2 ulp, ample for a weight
            ws[k] = wt;
            ss[k] = (float)s;
            ts[k] = (float)t;
            vs[k] = v;
            W += wt;
            // a zero offset (or the centre's v = 0) adds exactly nothing: no FMA for it
            if (s != 0) sb = fmaf(wt, (float)s, sb);
            if (t != 0) tb = fmaf(wt, (float)t, tb);
            if (!ctr) vb = fmaf(wt, v, vb);
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
    // the slope's components along the eigenvectors: no decision depends on them, so the
    // fast division (2 ulp) serves; the eigenvalues, which the cut tests, stay IEEE-rounded
    float gs = 0.f, gt = 0.f;
    if (l1 > thr) {
        const float c1 = __fdividef(e1s * csv + e1t * ctv, l1);
        gs = fmaf(c1, e1s, gs);
        gt = fmaf(c1, e1t, gt);
    }
    if (l2 > thr) {
        const float c2 = __fdividef(e2s * csv + e2t * ctv, l2);
        gs = fmaf(c2, e2s, gs);
        gt = fmaf(c2, e2t, gt);
    }
    return uc + vb - (gs * sb + gt * tb);
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
// The start of a prolonged level (Algorithm 2, Step 2) in one pass: D(S(P(Pi(u1, u2)))) for
// one TH x PSD_TW block of fine pixels at (y0, x0), TH <= PSD_TH (the shared-memory stages are
// sized for PSD_TH rows; a block's result does not depend on TH).  D needs S's output with a 2-pixel halo
// (its own 4 neighbours and their diffusivities), S needs P's with a 1-pixel halo beyond that,
// and P the level-(l-1) window of Pi values its triplets read; each stage is computed for its
// whole region into shared memory (pixels outside the image are never read), with the
// per-pixel arithmetic of k_prolong, k_smooth and k_denoise, so the result equals those three
// kernels in sequence bitwise, while the two intermediate images never leave the SM.  Halo
// work at TH = 32: P on 1.30x, S on 1.20x, c on 1.10x the block's pixels.  Called by every thread of a
// 256-thread block; store(rr, cc, v) receives the block's in-image outputs (row rr, column cc of
// the tile).
constexpr int PSD_TH = 32, PSD_TW = 64, PSD_THREADS = 256;
constexpr int PSD_PH = PSD_TH + 6, PSD_PW = PSD_TW + 6;  // P: 3-pixel halo
constexpr int PSD_SH = PSD_TH + 4, PSD_SW = PSD_TW + 4;  // S: 2
constexpr int PSD_CH = PSD_TH + 2, PSD_CW = PSD_TW + 2;  // c: 1
// Pi window: n consecutive fine indices read level-(l-1) indices 2A .. 2A' + 2 with
// A' - A <= (n + 2) / 4
constexpr int PSD_XR = 2 * ((PSD_PH + 2) / 4) + 3, PSD_XC = 2 * ((PSD_PW + 2) / 4) + 3;
// level-(l-2) nodes under the Pi window: rows 2A of the window and one more
constexpr int PSD_DR = (PSD_XR - 1) / 2 + 2, PSD_DC = (PSD_XC - 1) / 2 + 2;
struct PsdSmem {
    float2 D[PSD_DR][PSD_DC];  // exact differences d(A, B) as (hi, lo)
    float X[PSD_XR][PSD_XC];
    float P[PSD_PH][PSD_PW];
    float S[PSD_SH][PSD_SW];
    float C[PSD_CH][PSD_CW];
};
template <int TH = PSD_TH, class Store>
__device__ __forceinline__ void tile_psd(PsdSmem& M, const float* __restrict__ u1, int h1, int w1,
                                         const float* __restrict__ u2, int h2, int w2, int h, int w,
                                         float scale, float tau, float inv_k2, int y0, int x0,
                                         Store&& store) {
    static_assert(TH >= 1 && TH <= PSD_TH, "the stages are sized for PSD_TH rows");
    constexpr int th = TH;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    constexpr int NT = PSD_THREADS;
    // fine region of P (clipped to the image) and its Pi window
    const int py0 = max(y0 - 3, 0), px0 = max(x0 - 3, 0);
    const int py1 = min(y0 + th + 3, h), px1 = min(x0 + PSD_TW + 3, w);  // exclusive
    const int r0 = 2 * (py0 >> 2), c0 = 2 * (px0 >> 2);
    const int nr = 2 * (((py1 - 1) >> 2) - (py0 >> 2)) + 3;
    const int nc = 2 * (((px1 - 1) >> 2) - (px0 >> 2)) + 3;
    // the differences d(A, B) of the nodes under the window, each taken once (a node
    // serves up to nine Pi values), then Pi from them: the same operations as pi_at
    const int A0w = r0 >> 1, B0w = c0 >> 1;
    const int nA = min(((min(r0 + nr - 1, h1 - 1)) >> 1) + 1, h2 - 1) - A0w + 1;
    const int nB = min(((min(c0 + nc - 1, w1 - 1)) >> 1) + 1, w2 - 1) - B0w + 1;
    for (int k = tid; k < nA * nB; k += NT) {
        const int ra = k / nB, cb = k - ra * nB;
        const DF d = pi_diff(u1, w1, u2, w2, A0w + ra, B0w + cb);
        M.D[ra][cb] = make_float2(d.hi, d.lo);
    }
    __syncthreads();
    for (int k = tid; k < nr * nc; k += NT) {
        const int rr = k / nc, cc = k - rr * nc;
        const int a = min(r0 + rr, h1 - 1), b = min(c0 + cc, w1 - 1);
        int A0, A1, B0, B1;
        pi_nodes(a, b, h2, w2, A0, A1, B0, B1);
        auto dd = [&](int A, int B) {
            const float2 q = M.D[A - A0w][B - B0w];
            return DF{q.x, q.y};
        };
        M.X[rr][cc] = pi_from(u1[(size_t)a * w1 + b], dd(A0, B0), dd(A0, B1), dd(A1, B0), dd(A1, B1));
    }
    __syncthreads();
    // P on rows y0-3 .. y0+TH+2 and columns x0-3 .. x0+TW+2 (in-image part)
    for (int k = tid; k < (th + 6) * PSD_PW; k += NT) {
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
    // a block whose P region lies inside the image needs no bounds tests in S (most blocks)
    const bool interior = y0 >= 3 && x0 >= 3 && y0 + th + 3 <= h && x0 + PSD_TW + 3 <= w;
    if (interior) {
        for (int k = tid; k < (th + 4) * PSD_SW; k += NT) {
            const int rr = k / PSD_SW, cc = k - rr * PSD_SW;
            M.S[rr][cc] = smooth_value_rd<false>(pr, h, w, scale, y0 - 2 + rr, x0 - 2 + cc);
        }
    } else {
        for (int k = tid; k < (th + 4) * PSD_SW; k += NT) {
            const int rr = k / PSD_SW, cc = k - rr * PSD_SW;
            const int y = y0 - 2 + rr, x = x0 - 2 + cc;
            M.S[rr][cc] = (y >= 0 && y < h && x >= 0 && x < w) ? smooth_value_rd(pr, h, w, scale, y, x) : 0.f;
        }
    }
    __syncthreads();
    auto sr = [&](int a, int b) { return M.S[a - y0 + 2][b - x0 + 2]; };
    for (int k = tid; k < (th + 2) * PSD_CW; k += NT) {
        const int rr = k / PSD_CW, cc = k - rr * PSD_CW;
        const int y = y0 - 1 + rr, x = x0 - 1 + cc;
        M.C[rr][cc] = (y >= 0 && y < h && x >= 0 && x < w) ? pm_c_rd(sr, h, w, y, x, inv_k2) : 0.f;
    }
    __syncthreads();
    auto cr = [&](int a, int b) { return M.C[a - y0 + 1][b - x0 + 1]; };
    for (int k = tid; k < th * PSD_TW; k += NT) {
        const int rr = k / PSD_TW, cc = k - rr * PSD_TW;
        const int y = y0 + rr, x = x0 + cc;
        if (y < h && x < w) store(rr, cc, denoise_value_rd(sr, cr, h, w, tau, y, x));
    }
}

}  // namespace eecmg
