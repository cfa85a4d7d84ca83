// conv.cu -- the blur operator H_l and H_l^T (Eqs. 1, 7, 14: zero-boundary
// 2-D convolution with the level's PSF) with the Krylov epilogues fused.
//
// One CTA computes a 32 x 64 output tile.  The input tile plus a halo of R
// pixels is staged in shared memory (zero outside the image, which is the
// block-Toeplitz boundary of Eq. 7).  Separable PSFs (the Gaussian of
// Section 5, H = h (x) h, and its Galerkin coarsenings) run a vertical then
// a horizontal pass, each thread sliding a register window over 8 outputs;
// other PSFs (motion blur) run over their non-zero taps.  The finished tile
// is then streamed out row-major (coalesced) through the fused epilogue,
// whose inner products enter the deterministic grid reduction.
//
// PREC selects a compensated horizontal pass: each product's rounding error
// (from an FMA) and each addition's rounding error (TwoSum) are carried in a
// second FP32 accumulator, so the output is nearly correctly rounded.  The
// semi-convergent Krylov levels amplify the rounding of H, and this halves
// the FP32-vs-FP64 gap of the whole cascade at some ALU cost.
#include "launch.hpp"

namespace eecmg {

template <int R, bool SEP, bool PREC>
__global__ void __launch_bounds__(NTHREADS) k_conv(ConvArgs a) {
    constexpr int TH = CONV_TH, TW = CONV_TW;
    constexpr int IH = TH + 2 * R, IW = TW + 2 * R;
    constexpr int PT = TW + 2 * R + 1;  // odd pitch: conflict-free column walks
    constexpr int PO = TW + 1;
    constexpr int NT = SEP ? 1 : (2 * R + 1) * (2 * R + 1);

    __shared__ float s_in[IH * IW];
    __shared__ float s_tmp[SEP ? TH * PT : 1];
    __shared__ float s_out[TH * PO];
    __shared__ float s_cy[2 * R + 1], s_cx[2 * R + 1];
    __shared__ int s_off[NT];
    __shared__ float s_wt[NT];
    __shared__ int s_ntap;

    const int mode = a.mode;
    if (a.sc != nullptr && mode != CM_RESID) {
        if (*(volatile int*)&a.sc->stopped) return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
    const int h = a.h, w = a.w;

    if (!a.zero_input) {
        if (SEP) {
            for (int d = tid; d < 2 * R + 1; d += NTHREADS) {
                s_cy[d] = a.taps->cy[d];
                s_cx[d] = a.taps->cx[d];
            }
        } else {
            const int nt = a.taps->ntap;
            if (tid == 0) s_ntap = nt;
            for (int t = tid; t < nt; t += NTHREADS) {
                s_off[t] = (a.taps->dy[t] + R) * IW + (a.taps->dx[t] + R);
                s_wt[t] = a.taps->wt[t];
            }
        }
        // input tile with halo, zero outside the image
        const float* __restrict__ x = a.x;
        for (int i = tid; i < IH * IW; i += NTHREADS) {
            const int r = i / IW, c = i - r * IW;
            const int gy = y0 - R + r, gx = x0 - R + c;
            float v = 0.f;
            if (gy >= 0 && gy < h && gx >= 0 && gx < w) v = __ldg(x + (size_t)gy * w + gx);
            s_in[i] = v;
        }
        __syncthreads();

        if (SEP) {
            float cyr[2 * R + 1], cxr[2 * R + 1];
#pragma unroll
            for (int d = 0; d < 2 * R + 1; ++d) {
                cyr[d] = s_cy[d];
                cxr[d] = s_cx[d];
            }
            // vertical pass: tmp(r, c) = sum_d cy[d] in(r + d, c), r < TH, all IW columns
            for (int item = tid; item < 4 * IW; item += NTHREADS) {
                const int rg = item / IW, c = item - rg * IW;
                float v[8 + 2 * R];
#pragma unroll
                for (int j = 0; j < 8 + 2 * R; ++j) v[j] = s_in[(rg * 8 + j) * IW + c];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float acc = 0.f;
#pragma unroll
                    for (int d = 0; d < 2 * R + 1; ++d) acc = fmaf(cyr[d], v[i + d], acc);
                    s_tmp[(rg * 8 + i) * PT + c] = acc;
                }
            }
            __syncthreads();
            // horizontal pass: one row per lane, 8 consecutive columns per warp
            {
                const int r = lane, cg = warp;
                float v[8 + 2 * R];
#pragma unroll
                for (int j = 0; j < 8 + 2 * R; ++j) v[j] = s_tmp[r * PT + cg * 8 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float acc = 0.f;
                    if (PREC) {
                        float lo = 0.f;
#pragma unroll
                        for (int d = 0; d < 2 * R + 1; ++d) {
                            const float p = __fmul_rn(cxr[d], v[i + d]);
                            const float pe = fmaf(cxr[d], v[i + d], -p);  // exact product error
                            const float s = __fadd_rn(acc, p);
                            const float bp = __fsub_rn(s, acc);
                            const float se = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, bp)), __fsub_rn(p, bp));
                            acc = s;
                            lo = __fadd_rn(lo, __fadd_rn(pe, se));
                        }
                        acc = __fadd_rn(acc, lo);
                    } else {
#pragma unroll
                        for (int d = 0; d < 2 * R + 1; ++d) acc = fmaf(cxr[d], v[i + d], acc);
                    }
                    s_out[r * PO + cg * 8 + i] = acc;
                }
            }
        } else {
            const int c = tid & 63, rg = tid >> 6;
            float acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = 0.f;
            const int nt = s_ntap;
            const float* base = s_in + (rg * 8) * IW + c;
            for (int t = 0; t < nt; ++t) {
                const float wt = s_wt[t];
                const float* p = base + s_off[t];
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt, p[i * IW], acc[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) s_out[(rg * 8 + i) * PO + c] = acc[i];
        }
        __syncthreads();
    }

    // epilogue: row-major, coalesced
    float scale = 1.f;
    if (mode == CM_MR_A) scale = (float)(1.0 / a.sc->nrm);
    float acc0 = 0.f, acc1 = 0.f;
    float* __restrict__ y = a.y;
#pragma unroll
    for (int it = 0; it < TH / 8; ++it) {
        const int r = warp + 8 * it;
        const int gy = y0 + r;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int c = lane + 32 * hf;
            const int gx = x0 + c;
            if (gy < h && gx < w) {
                const size_t idx = (size_t)gy * w + gx;
                const float z = a.zero_input ? 0.f : s_out[r * PO + c];
                switch (mode) {
                    case CM_RESID: {
                        const float gv = __ldg(a.e0 + idx);
                        const float rv = gv - z;
                        y[idx] = rv;
                        if (a.y2) a.y2[idx] = rv;
                        acc0 = fmaf(rv, rv, acc0);
                        acc1 = fmaf(gv, gv, acc1);
                    } break;
                    case CM_MR_V1: {  // v_1 = H r_0, with <v, v>, <v, r_0>
                        y[idx] = z;
                        acc0 = fmaf(z, z, acc0);
                        acc1 = fmaf(z, s_in[(r + R) * IW + c + R], acc1);
                    } break;
                    case CM_MR_A: {   // H w_k = H v_k / ||v_k||, with <H w_k, v_k>
                        const float hz = z * scale;
                        y[idx] = hz;
                        acc0 = fmaf(hz, s_in[(r + R) * IW + c + R], acc0);
                    } break;
                    case CM_CG_S0: {
                        y[idx] = z;
                        a.y2[idx] = z;
                        acc0 = fmaf(z, z, acc0);
                    } break;
                    case CM_CG_Q:
                    case CM_CG_S: {
                        y[idx] = z;
                        acc0 = fmaf(z, z, acc0);
                    } break;
                    default:
                        y[idx] = z;
                }
            }
        }
    }
    if (mode == CM_STORE) return;

    const unsigned int nblocks = gridDim.x * gridDim.y;
    const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x;
    Scalars* sc = a.sc;
    double v[2] = {(double)acc0, (double)acc1};
    if (!block_partials_arrive<2>(v, a.partials, &sc->counter, nblocks, bid)) return;
    double tot[2];
    grid_total<2>(a.partials, nblocks, &sc->counter, tot);
    if (tid != 0) return;
    switch (mode) {
        case CM_RESID: {
            const double rr = tot[0], gg = tot[1];
            sc->rr = rr;
            sc->gg = gg;
            const double l1 = a.conv_tol2 * gg;
            sc->lim2 = l1 > a.disc2 ? l1 : a.disc2;
            sc->iters = 0;
            if (!(rr < 1.0e300)) sc->stopped = 3;
            else sc->stopped = (rr <= sc->lim2) ? 1 : 0;
        } break;
        case CM_MR_V1: {
            const double vv = tot[0];
            if (!(vv < 1.0e300)) {
                sc->stopped = 3;
            } else if (!(vv > 0.0)) {
                sc->stopped = 2;  // H r_0 = 0: no step
            } else {
                const double nrm = sqrt(vv);
                sc->nrm = nrm;
                sc->nrm_prev = 0.0;
                sc->phi = tot[1] / nrm;  // <w_1, r_0>
                sc->cs1 = 1.0;
                sc->sn1 = 0.0;
                sc->cs2 = 1.0;
                sc->sn2 = 0.0;
            }
        } break;
        case CM_MR_A: {
            sc->alpha = tot[0] / sc->nrm;
        } break;
        case CM_CG_S0: {
            const double gm = tot[0];
            if (!(gm < 1.0e300)) sc->stopped = 3;
            else if (!(gm > 0.0)) sc->stopped = 2;
            else sc->gamma = gm;
        } break;
        case CM_CG_Q: {
            const double qq = tot[0];
            if (!(qq < 1.0e300)) {
                sc->stopped = 3;
            } else if (!(qq > 0.0)) {
                sc->stopped = 2;
            } else {
                sc->qq = qq;
                sc->cg_alpha = sc->gamma / qq;
                sc->iters += 1;
            }
        } break;
        case CM_CG_S: {
            const double gn = tot[0];
            sc->beta = gn / sc->gamma;
            sc->gamma = gn;
            if (!(gn < 1.0e300)) sc->stopped = 3;
            else if (!(gn > 0.0)) sc->stopped = 2;
        } break;
        default:
            break;
    }
}

template <int R>
static cudaError_t launch_conv_r(const ConvArgs& a, int sep, int prec, cudaStream_t s) {
    dim3 grid((a.w + CONV_TW - 1) / CONV_TW, (a.h + CONV_TH - 1) / CONV_TH);
    if (sep && prec)
        k_conv<R, true, true><<<grid, NTHREADS, 0, s>>>(a);
    else if (sep)
        k_conv<R, true, false><<<grid, NTHREADS, 0, s>>>(a);
    else
        k_conv<R, false, false><<<grid, NTHREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv(const ConvArgs& a, int rt, int sep, int prec, cudaStream_t s) {
    if (a.h <= 0 || a.w <= 0) return cudaSuccess;
    switch (rt) {
        case 0: return launch_conv_r<0>(a, sep, prec, s);
        case 1: return launch_conv_r<1>(a, sep, prec, s);
        case 2: return launch_conv_r<2>(a, sep, prec, s);
        case 3: return launch_conv_r<3>(a, sep, prec, s);
        case 4: return launch_conv_r<4>(a, sep, prec, s);
        case 5: return launch_conv_r<5>(a, sep, prec, s);
        case 6: return launch_conv_r<6>(a, sep, prec, s);
        case 7: return launch_conv_r<7>(a, sep, prec, s);
        case 8: return launch_conv_r<8>(a, sep, prec, s);
        case 9: return launch_conv_r<9>(a, sep, prec, s);
        case 10: return launch_conv_r<10>(a, sep, prec, s);
        case 11: return launch_conv_r<11>(a, sep, prec, s);
        case 12: return launch_conv_r<12>(a, sep, prec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
