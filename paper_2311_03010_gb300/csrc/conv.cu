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
#include "conv_tile.cuh"
#include "finish.cuh"

namespace eecmg {

template <int R, bool SEP, bool PREC>
__global__ void __launch_bounds__(NTHREADS) k_conv(ConvArgs a) {
    using SM = ConvSmem<R, SEP>;
    __shared__ SM S;
    constexpr int PO = SM::PO, TH = SM::TH;

    const int mode = a.mode;
    if (a.sc != nullptr && mode != CM_RESID) {
        if (*(volatile int*)&a.sc->stopped) return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y0 = blockIdx.y * CONV_TH, x0 = blockIdx.x * CONV_TW;
    const int h = a.h, w = a.w;

    if (!a.zero_input) {
        conv_stage_taps<R, SEP>(S, a.taps);
        conv_load<R, SEP, false>(S, a.x, h, w, y0, x0);
        __syncthreads();
        conv_compute<R, SEP, PREC>(S);
        __syncthreads();
    }

    // epilogue: row-major, coalesced
    float scale = 1.f;
    if (mode == CM_MR_A) scale = *(volatile const float*)&a.sc->f_scale;
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
                const float z = a.zero_input ? 0.f : S.out[r * PO + c];
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
                        acc1 = fmaf(z, S.in[SM::at(r + R, c + R)], acc1);
                    } break;
                    case CM_MR_A: {   // H w_k = H v_k / ||v_k||, with <H w_k, v_k>
                        const float hz = z * scale;
                        y[idx] = hz;
                        acc0 = fmaf(hz, S.in[SM::at(r + R, c + R)], acc0);
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
        case CM_RESID: fin_resid(sc, df_from_double(tot[0]), df_from_double(tot[1]), a.conv_tol2, a.disc2); break;
        case CM_MR_V1: fin_mr_v1(sc, df_from_double(tot[0]), df_from_double(tot[1])); break;
        case CM_MR_A: fin_mr_a(sc, df_from_double(tot[0])); break;
        case CM_CG_S0: fin_cg_s0(sc, df_from_double(tot[0])); break;
        case CM_CG_Q: fin_cg_q(sc, df_from_double(tot[0])); break;
        case CM_CG_S: fin_cg_s(sc, df_from_double(tot[0])); break;
        default: break;
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
