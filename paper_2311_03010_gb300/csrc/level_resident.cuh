// level_resident.cuh -- the level solves (Section 2: MR-II in Lanczos / Givens
// form, and CGLS) with the whole level held in shared memory: FP32 storage, one
// thread-block cluster of C <= 16 blocks per solve.  Block b owns T (1 or 2)
// consecutive 32 x 64 tiles of the level in row-major tile order and keeps
// the solver vectors of its tiles (MR-II: u, r, v_k, v_{k+1}, H w_k, H w_{k+1},
// two directions d, two H d; CGLS: u, r, s, p, q) in its shared memory, tile-major, for the whole
// solve: T x 2048 x 10 floats.  A convolution phase stages each tile with its
// halo from the blocks that own the halo pixels (distributed shared memory
// loads after the phase barrier); elementwise phases read and write shared
// memory only; the reductions are the in-cluster exchange of persistent.cuh.
// Only u0 and g are read from global memory (start phase) and only u is
// written back (end).  Entries of partial tiles outside the level are zero
// at the start and stay zero (every update is a linear combination of zero
// entries), so the elementwise phases run over whole tiles.
//
// Per pixel and per scalar this is the arithmetic of mr2_body / cgls_body;
// only the partition of the inner products into block sums differs.
#pragma once

namespace eecmg {

constexpr int RES_TMAX = 2;                 // tiles per block
constexpr int RES_NVEC = 10;
constexpr int RES_RMAX = 5;                 // instantiated radii 0..RES_RMAX
constexpr int TILE_PX = CONV_TH * CONV_TW;  // 2048

__host__ __device__ constexpr size_t res_smem_bytes(int T) {
    return (size_t)T * TILE_PX * RES_NVEC * sizeof(float);
}

namespace res_detail {

enum { VU = 0, VR = 1, VV = 2, VAW = 4, VD = 6, VHD = 8 };  // vector slots (VV + 0/1 etc.)

struct ResCtx {
    float* base;                        // this block's vectors: RES_NVEC x NL floats
    int T, NL, bid, tiles_x, ntiles, h, w;
    __device__ __forceinline__ float* vec(int k) const { return base + (size_t)k * NL; }
};

__device__ __forceinline__ unsigned int cluster_addr(unsigned int shared_addr, unsigned int rank) {
    unsigned int r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(shared_addr), "r"(rank));
    return r;
}

__device__ __forceinline__ float ld_cluster(unsigned int addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ float ld_local(unsigned int addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

constexpr unsigned int RES_NONE = 0xffffffffu;

// Stages vector k's window of tile t (halo R, zero outside the level) into
// S.in.  nbr[3 (dy + 1) + dx + 1] receives the distributed-shared-memory
// address of vector k of the tile (dy, dx) away from t in the block that owns
// it (RES_NONE outside the tile grid); each window pixel then reads its own
// tile's copy.  Padding entries of partial tiles are zero, so pixels beyond
// the level inside existing tiles need no test.
template <int R, bool SEP>
__device__ __forceinline__ void conv_load_res(ConvSmem<R, SEP>& S, unsigned int (&nbr)[9], const ResCtx& X,
                                              int k, int t) {
    constexpr int IW = ConvSmem<R, SEP>::IW;
    constexpr int NTOT = ConvSmem<R, SEP>::IH * IW;
    constexpr int ITERS = (NTOT + NTHREADS - 1) / NTHREADS;
    if (threadIdx.x < 9) {
        const int dy = (int)threadIdx.x / 3 - 1, dx = (int)threadIdx.x % 3 - 1;
        const int ty = t / X.tiles_x + dy, tx = t % X.tiles_x + dx;
        const int tiles_y = X.ntiles / X.tiles_x;
        unsigned int a = RES_NONE;
        if (ty >= 0 && ty < tiles_y && tx >= 0 && tx < X.tiles_x) {
            const int tn = ty * X.tiles_x + tx;
            const int owner = tn / X.T;
            const unsigned int local =
                (unsigned int)__cvta_generic_to_shared(X.base + (size_t)k * X.NL + (size_t)(tn - owner * X.T) * TILE_PX);
            a = cluster_addr(local, (unsigned int)owner);
        }
        nbr[threadIdx.x] = a;
    }
    __syncthreads();
    // the tile itself is this block's (plain shared-memory loads when R = 0)
    const unsigned int own = (unsigned int)__cvta_generic_to_shared(
        X.base + (size_t)k * X.NL + (size_t)(t - X.bid * X.T) * TILE_PX);
    float vals[ITERS];
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int i = threadIdx.x + it * NTHREADS;
        float v = 0.f;
        if (i < NTOT) {
            const int ry = i / IW - R, rx = i % IW - R;
            const int sy = ry < 0 ? 0 : (ry >= CONV_TH ? 2 : 1), sx = rx < 0 ? 0 : (rx >= CONV_TW ? 2 : 1);
            const unsigned int off = 4u * (unsigned int)((ry - (sy - 1) * CONV_TH) * CONV_TW + rx - (sx - 1) * CONV_TW);
            if constexpr (R == 0) {
                v = ld_local(own + off);  // the window is the tile
            } else {  // one load form for every pixel: no divergence at the window's edges
                const unsigned int a = nbr[3 * sy + sx];
                if (a != RES_NONE) v = ld_cluster(a + off);
            }
        }
        vals[it] = v;
    }
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int i = threadIdx.x + it * NTHREADS;
        if (i < NTOT) S.in[ConvSmem<R, SEP>::at(i / IW, i % IW)] = vals[it];
    }
}

// One convolution phase over this block's tiles: the input is u0 in global
// memory (GLOBAL) or vector k of the cluster (ZERO: an all-zero input, no
// loads); the epilogue gets (local index, level index, (C (*) x)(p), x(p)).
// conv_compute on two staged tiles at once: every thread carries the outputs
// of both tiles through the same loops (twice the independent chains while a
// block holds one SM), with the operations of conv_compute per output.
template <int R, bool SEP, bool PREC>
__device__ __forceinline__ void conv_compute2(ConvSmem<R, SEP>& A, ConvSmem<R, SEP>& B) {
    using SM = ConvSmem<R, SEP>;
    constexpr int IW = SM::IW, PT = SM::PT, PO = SM::PO, VR = SM::VR, VG = SM::VG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ConvSmem<R, SEP>* S[2] = {&A, &B};
    if (SEP) {
        // vertical pass: thread (g, c) takes rows r0 .. r0 + VR - 1 of column c of both tiles
        const int g = tid / IW, c = tid - g * IW;
        if (g < VG) {
            const int r0 = g == VG - 1 ? CONV_TH - VR : g * VR;
            float v[2][VR + 2 * R];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int j = 0; j < VR + 2 * R; ++j) v[s][j] = S[s]->in[SM::at(r0 + j, c)];
            float acc[2][VR];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < VR; ++i) acc[s][i] = 0.f;
#pragma unroll
            for (int d = 0; d < 2 * R + 1; ++d) {
                const float cd = A.cy[d];
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int i = 0; i < VR; ++i) acc[s][i] = fmaf(cd, v[s][i + d], acc[s][i]);
            }
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < VR; ++i)
                    if (g < VG - 1 || i >= VG * VR - CONV_TH) S[s]->tmp[(r0 + i) * PT + c] = acc[s][i];
        }
        __syncthreads();
        const int r = lane, cg = warp;
        constexpr int NW4 = (8 + 2 * R + 3) / 4;
        float v[2][4 * NW4];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int j4 = 0; j4 < NW4; ++j4) {
                const float4 q = *reinterpret_cast<const float4*>(S[s]->tmp + r * PT + cg * 8 + 4 * j4);
                v[s][4 * j4] = q.x;
                v[s][4 * j4 + 1] = q.y;
                v[s][4 * j4 + 2] = q.z;
                v[s][4 * j4 + 3] = q.w;
            }
        float acc[2][8], lo[2][8], comp[2][8];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[s][i] = 0.f;
                lo[s][i] = 0.f;
                comp[s][i] = 0.f;
            }
#pragma unroll
        for (int d = 0; d < 2 * R + 1; ++d) {
            const float cd = A.cx[d];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (PREC) {
                        const float p = __fmul_rn(cd, v[s][i + d]);
                        const float pe = fmaf(cd, v[s][i + d], -p);
                        const float y = __fsub_rn(p, comp[s][i]);
                        const float t = __fadd_rn(acc[s][i], y);
                        comp[s][i] = __fsub_rn(__fsub_rn(t, acc[s][i]), y);
                        acc[s][i] = t;
                        lo[s][i] = __fadd_rn(lo[s][i], pe);
                    } else {
                        acc[s][i] = fmaf(cd, v[s][i + d], acc[s][i]);
                    }
                }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                S[s]->out[r * PO + cg * 8 + i] =
                    PREC ? __fadd_rn(acc[s][i], __fsub_rn(lo[s][i], comp[s][i])) : acc[s][i];
    } else {
        const int c = tid & 63, rg = tid >> 6;
        float acc[2][8];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[s][i] = 0.f;
        const int nt = A.ntap;
        for (int t = 0; t < nt; ++t) {
            const float wt = A.wt[t];
            const int off = A.off[t] + ConvSmem<R, SEP>::at(rg * 8, c);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[s][i] = fmaf(wt, S[s]->in[off + i * ConvSmem<R, SEP>::IP], acc[s][i]);
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 8; ++i) S[s]->out[(rg * 8 + i) * PO + c] = acc[s][i];
    }
}

// One convolution phase over this block's tiles: the input is u0 in global
// memory (GLOBAL) or vector k of the cluster (ZERO: an all-zero input, no
// loads); the epilogue gets (local index, level index, (C (*) x)(p), x(p)).
// S[0] stages one tile at a time; with two tiles of the cluster's vector
// both are staged (S[0], S[1]) and computed together.  Only S[0] holds taps.
template <int R, bool SEP, bool PREC, bool ZERO, bool GLOBAL, class Epi>
__device__ __forceinline__ void conv_phase_res(ConvSmem<R, SEP> (&S)[2], const ResCtx& X, int k,
                                               const float* xg, Epi&& epi) {
    using SM = ConvSmem<R, SEP>;
    __shared__ unsigned int nbr[2][9];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto epilogue = [&](const SM& T, int lt, int y0, int x0) {
#pragma unroll
        for (int it = 0; it < CONV_TH / 8; ++it) {
            const int r = warp + 8 * it, gy = y0 + r;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int c = lane + 32 * hf, gx = x0 + c;
                if (gy < X.h && gx < X.w) {
                    const float z = ZERO ? 0.f : T.out[r * SM::PO + c];
                    const float ctr = ZERO ? 0.f : T.in[SM::at(r + R, c + R)];
                    epi(lt * TILE_PX + r * CONV_TW + c, (size_t)gy * X.w + gx, z, ctr);
                }
            }
        }
    };
    const int t0 = X.bid * X.T;
    if (!ZERO && !GLOBAL && X.T == 2 && t0 + 1 < X.ntiles) {
        conv_load_res<R, SEP>(S[0], nbr[0], X, k, t0);
        conv_load_res<R, SEP>(S[1], nbr[1], X, k, t0 + 1);
        __syncthreads();
        conv_compute2<R, SEP, PREC>(S[0], S[1]);
        __syncthreads();
        for (int lt = 0; lt < 2; ++lt)
            epilogue(S[lt], lt, ((t0 + lt) / X.tiles_x) * CONV_TH, ((t0 + lt) % X.tiles_x) * CONV_TW);
        __syncthreads();
        return;
    }
    for (int lt = 0; lt < X.T; ++lt) {
        const int t = t0 + lt;
        if (t >= X.ntiles) break;
        const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
        if (!ZERO) {
            if (GLOBAL)
                conv_load<R, SEP, true, float>(S[0], xg, X.h, X.w, y0, x0);
            else
                conv_load_res<R, SEP>(S[0], nbr[0], X, k, t);
            __syncthreads();
            conv_compute<R, SEP, PREC>(S[0]);
            __syncthreads();
        }
        epilogue(S[0], lt, y0, x0);
        __syncthreads();  // S[0] is reused by the next tile
    }
}

__device__ __forceinline__ float4 lds4(const float* p, int q) {
    return reinterpret_cast<const float4*>(p)[q];
}
__device__ __forceinline__ void sts4(float* p, int q, float4 v) { reinterpret_cast<float4*>(p)[q] = v; }

// MR-II step j on local float4 q; returns the new r.
__device__ __forceinline__ float4 res_step4(const ResCtx& X, int j, int q, const StepCoef& c) {
    const int sj = j & 1, sj1 = sj ^ 1;
    float4 dj = mul4(c.dw, lds4(X.vec(VV + sj), q));
    float4 hj = mul4(c.dinv, lds4(X.vec(VAW + sj), q));
    if (j >= 2) {
        dj = fma4(-c.d1, lds4(X.vec(VD + sj1), q), dj);
        hj = fma4(-c.d1, lds4(X.vec(VHD + sj1), q), hj);
    }
    if (j >= 3) {
        dj = fma4(-c.d2, lds4(X.vec(VD + sj), q), dj);
        hj = fma4(-c.d2, lds4(X.vec(VHD + sj), q), hj);
    }
    sts4(X.vec(VD + sj), q, dj);
    sts4(X.vec(VHD + sj), q, hj);
    sts4(X.vec(VU), q, fma4(c.tau, dj, lds4(X.vec(VU), q)));
    const float4 rv = fma4(-c.tau, hj, lds4(X.vec(VR), q));
    sts4(X.vec(VR), q, rv);
    return rv;
}

// Phase 0 of a resident solve that starts its own level (J.start): D(S(P(Pi))) of each of the
// block's tiles into its resident u and into u in global memory (the r_0 phase stages its
// halo windows from there), then a cluster barrier.  Returns false if the job is in error.
__device__ __forceinline__ bool res_start_phase(PsdSmem& M, const LevelJob& J, const ResCtx& X,
                                                float* ures, LevelSync& sy) {
    for (int lt = 0; lt < X.T; ++lt) {
        const int t = X.bid * X.T + lt;
        if (t >= X.ntiles) break;
        const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
        float* ul = ures + lt * TILE_PX;
        tile_psd(M, J.s_u1, J.s_h1, J.s_w1, J.s_u2, J.s_h2, J.s_w2, X.h, X.w, J.s_scale, J.s_tau,
                 J.s_ik2, y0, x0, [&](int rr, int cc, float v) {
                     ul[rr * CONV_TW + cc] = v;
                     J.u[(size_t)(y0 + rr) * X.w + x0 + cc] = v;
                 });
        __syncthreads();
    }
    float v[1] = {0.f};
    return sy.reduce<1>(v, [&](DF*) {});
}

template <int R, bool SEP, bool PREC>
__device__ __forceinline__ void mr2_res_body(ConvSmem<R, SEP> (&S)[2], PsdSmem& M, const LevelJob& J, Scalars* sc,
                                             const ResCtx& X, LevelSync& sy) {
    const int n4 = X.NL >> 2;
    {  // every vector zero, then u0 (or the level's start, phase 0)
        float4* b4 = reinterpret_cast<float4*>(X.base);
        for (int q = threadIdx.x; q < RES_NVEC * n4; q += NTHREADS) b4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        if (J.start) {
            if (!res_start_phase(M, J, X, X.vec(VU), sy)) return;
        } else if (!J.zero_start) {
            float* u = X.vec(VU);
            for (int lt = 0; lt < X.T; ++lt) {
                const int t = X.bid * X.T + lt;
                if (t >= X.ntiles) break;
                const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
                for (int p = threadIdx.x; p < TILE_PX; p += NTHREADS) {
                    const int gy = y0 + p / CONV_TW, gx = x0 + p % CONV_TW;
                    if (gy < X.h && gx < X.w) u[lt * TILE_PX + p] = __ldcg(J.u + (size_t)gy * X.w + gx);
                }
            }
        }
        __syncthreads();
    }
    conv_stage_taps<R, SEP>(S[0], J.taps);  // after phase 0, whose tile shares this memory
    __syncthreads();

    // r_0 = g - H u_0, ||r_0||^2, ||g||^2, stopping limit
    {
        float a0 = 0.f, a1 = 0.f;
        float* rv_ = X.vec(VR);
        const bool zs = J.zero_start != 0;
        auto epi = [&](int li, size_t gi, float z, float) {
            const float gv = __ldg(J.g + gi);
            const float rv = gv - z;
            rv_[li] = rv;
            if (zs) J.u[gi] = 0.f;  // the zero start, in global memory for an early return
            a0 = fmaf(rv, rv, a0);
            a1 = fmaf(gv, gv, a1);
        };
        if (J.zero_start)
            conv_phase_res<R, SEP, PREC, true, true>(S, X, 0, J.u, epi);
        else
            conv_phase_res<R, SEP, PREC, false, true>(S, X, 0, J.u, epi);
        float v[2] = {a0, a1};
        const double ct2 = J.conv_tol2, d2 = J.disc2;
        const int ear = J.early;
        const double b0 = (J.zero_start ? 8.0 : 12.0) + ls_detail::start_bytes(J);
        if (!sy.reduce<2>(v, [&](DF* t) {
                fin_resid(sc, t[0], t[1], ct2, d2, ear);
                sc->bpp = b0;
            }))
            return;
    }
    if (J.m <= 0 || volatile_stopped(sc)) return;  // u in global memory holds the start
    // algorithmic bytes per pixel of the vector phases (as the streaming solver counts them)
    auto hist = [](int j) { return 8.0 * ((j >= 2 ? 1 : 0) + (j >= 3 ? 1 : 0)); };

    // v_1 = H r_0, ||v_1||, <v_1, r_0>
    {
        float a0 = 0.f, a1 = 0.f;
        float* v1 = X.vec(VV + 1);
        conv_phase_res<R, SEP, PREC, false, false>(S, X, VR, nullptr,
                                                   [&](int li, size_t, float z, float ctr) {
                                                       v1[li] = z;
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
            float* aw = X.vec(VAW + sk);
            conv_phase_res<R, SEP, PREC, false, false>(S, X, VV + sk, nullptr,
                                                       [&](int li, size_t, float z, float ctr) {
                                                           const float hz = z * scale;
                                                           aw[li] = hz;
                                                           a0 = fmaf(hz, ctr, a0);
                                                       });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) {
                    fin_mr_a(sc, t[0]);
                    sc->bpp += 8.0;
                }))
                return;
        }
        // phase B: pending step k-1 (unless an early check applied it), v_{k+1}, stopping
        // rules, rotation of column k
        {
            const bool step = k >= 2;
            const bool apply = step && *(volatile const int*)&sc->applied != k - 1;
            const StepCoef c = step_coef(sc);
            const float ca = vldf(&sc->f_ca), ca_lo = vldf(&sc->f_ca_lo);
            const float cb = step ? vldf(&sc->f_cb) : 0.f, cb_lo = step ? vldf(&sc->f_cb_lo) : 0.f;
            float arr = 0.f, avv = 0.f, avr = 0.f;
            const int j = k - 1, sj = j & 1, sj1 = sj ^ 1;  // sj == sk1
            for (int q = threadIdx.x; q < n4; q += NTHREADS) {
                const float4 vk = lds4(X.vec(VV + sk), q), awk = lds4(X.vec(VAW + sk), q);
                const float4 rr = lds4(X.vec(VR), q);
                float4 vj = make_float4(0.f, 0.f, 0.f, 0.f), awj = vj, uu = vj;
                float4 dA = vj, hA = vj, dB = vj, hB = vj;
                if (step) vj = lds4(X.vec(VV + sj), q);
                if (apply) {
                    awj = lds4(X.vec(VAW + sj), q);
                    uu = lds4(X.vec(VU), q);
                    if (j >= 2) {
                        dA = lds4(X.vec(VD + sj1), q);
                        hA = lds4(X.vec(VHD + sj1), q);
                    }
                    if (j >= 3) {
                        dB = lds4(X.vec(VD + sj), q);
                        hB = lds4(X.vec(VHD + sj), q);
                    }
                }
                float4 rv = rr;
                if (apply) {  // step j = k - 1 (the operation order of mr_step4)
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
                    sts4(X.vec(VD + sj), q, dj);
                    sts4(X.vec(VHD + sj), q, hj);
                    sts4(X.vec(VU), q, fma4(c.tau, dj, uu));
                    rv = fma4(-c.tau, hj, rr);
                    sts4(X.vec(VR), q, rv);
                }
                if (step) arr = dot4(rv, rv, arr);
                float4 vn = fma4(-ca_lo, vk, fma4(-ca, vk, awk));
                if (step) vn = fma4(-cb_lo, vj, fma4(-cb, vj, vn));
                sts4(X.vec(VV + sk1), q, vn);
                avv = dot4(vn, vn, avv);
                avr = dot4(vn, rv, avr);
            }
            float v[3] = {arr, avv, avr};
            const double bb = k == 1 ? 16.0 : (apply ? 44.0 + hist(k - 1) : 20.0);
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
            for (int q = threadIdx.x; q < n4; q += NTHREADS) {
                const float4 rv = res_step4(X, k, q, c);
                arr = dot4(rv, rv, arr);
            }
            float v[1] = {arr};
            const double bc = 32.0 + hist(k);
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
        for (int q = threadIdx.x; q < n4; q += NTHREADS) {
            const float4 rv = res_step4(X, j, q, c);
            arr = dot4(rv, rv, arr);
        }
        float v[1] = {arr};
        const double bf = 32.0 + hist(j);
        if (!sy.reduce<1>(v, [&](DF* t) {
                fin_mr_final(sc, t[0]);
                sc->bpp += bf;
            }))
            return;
    }
    // u back to global memory
    const float* u = X.vec(VU);
    for (int lt = 0; lt < X.T; ++lt) {
        const int t = X.bid * X.T + lt;
        if (t >= X.ntiles) break;
        const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
        for (int p = threadIdx.x; p < TILE_PX; p += NTHREADS) {
            const int gy = y0 + p / CONV_TW, gx = x0 + p % CONV_TW;
            if (gy < X.h && gx < X.w) J.u[(size_t)gy * X.w + gx] = u[lt * TILE_PX + p];
        }
    }
}

// CGLS (Section 2) on the resident vectors: the phases and per-pixel
// arithmetic of cgls_body (u, r, s = H^T r, p, q = H p; s and p FP32).
enum { CU = 0, CR = 1, CS_ = 2, CP = 3, CQ = 4 };

template <int R, bool SEP, bool PREC>
__device__ __forceinline__ void cgls_res_body(ConvSmem<R, SEP> (&S)[2], PsdSmem& M, const LevelJob& J, Scalars* sc,
                                              const ResCtx& X, LevelSync& sy) {
    const int n4 = X.NL >> 2;
    {  // every vector zero, then u0 (or the level's start, phase 0)
        float4* b4 = reinterpret_cast<float4*>(X.base);
        for (int q = threadIdx.x; q < RES_NVEC * n4; q += NTHREADS) b4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        if (J.start) {
            if (!res_start_phase(M, J, X, X.vec(CU), sy)) return;
        } else if (!J.zero_start) {
            float* u = X.vec(CU);
            for (int lt = 0; lt < X.T; ++lt) {
                const int t = X.bid * X.T + lt;
                if (t >= X.ntiles) break;
                const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
                for (int p = threadIdx.x; p < TILE_PX; p += NTHREADS) {
                    const int gy = y0 + p / CONV_TW, gx = x0 + p % CONV_TW;
                    if (gy < X.h && gx < X.w) u[lt * TILE_PX + p] = __ldcg(J.u + (size_t)gy * X.w + gx);
                }
            }
        }
        __syncthreads();
    }
    conv_stage_taps<R, SEP>(S[0], J.taps);  // after phase 0, whose tile shares this memory
    __syncthreads();
    float* rv_ = X.vec(CR);
    float* sv = X.vec(CS_);
    float* pv = X.vec(CP);
    float* qv = X.vec(CQ);
    {  // r_0 = g - H u_0
        float a0 = 0.f, a1 = 0.f;
        const bool zs = J.zero_start != 0;
        auto epi = [&](int li, size_t gi, float z, float) {
            const float gv = __ldg(J.g + gi);
            const float rv = gv - z;
            rv_[li] = rv;
            if (zs) J.u[gi] = 0.f;  // the zero start, in global memory for an early return
            a0 = fmaf(rv, rv, a0);
            a1 = fmaf(gv, gv, a1);
        };
        if (J.zero_start)
            conv_phase_res<R, SEP, PREC, true, true>(S, X, 0, J.u, epi);
        else
            conv_phase_res<R, SEP, PREC, false, true>(S, X, 0, J.u, epi);
        float v[2] = {a0, a1};
        const double ct2 = J.conv_tol2, d2 = J.disc2;
        const int ear = J.early;
        const double sb = ls_detail::start_bytes(J);  // the host counts the CGLS phases themselves
        if (!sy.reduce<2>(v, [&](DF* t) {
                fin_resid(sc, t[0], t[1], ct2, d2, ear);
                sc->bpp = sb;
            }))
            return;
    }
    if (J.m <= 0 || volatile_stopped(sc)) return;  // u in global memory holds the start
    conv_stage_taps<R, SEP>(S[0], J.tapsT);  // s = H^T r, p = s
    __syncthreads();
    {
        float a0 = 0.f;
        conv_phase_res<R, SEP, PREC, false, false>(S, X, CR, nullptr, [&](int li, size_t, float z, float) {
            sv[li] = z;
            pv[li] = z;
            a0 = fmaf(z, z, a0);
        });
        float v[1] = {a0};
        if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_s0(sc, t[0]); })) return;
    }
    bool ok = true;
    for (int k = 1; k <= J.m && ok; ++k) {
        if (volatile_stopped(sc)) break;
        __syncthreads();
        conv_stage_taps<R, SEP>(S[0], J.taps);  // q = H p, alpha
        __syncthreads();
        {
            float a0 = 0.f;
            conv_phase_res<R, SEP, PREC, false, false>(S, X, CP, nullptr, [&](int li, size_t, float z, float) {
                qv[li] = z;
                a0 = fmaf(z, z, a0);
            });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_q(sc, t[0]); })) return;
        }
        if (volatile_stopped(sc)) break;
        {  // u += alpha p, r -= alpha q, stopping rule
            const float a = vldf(&sc->f_cg_alpha);
            float arr = 0.f;
            for (int q = threadIdx.x; q < n4; q += NTHREADS) {
                const float4 pq = lds4(pv, q), uq = lds4(X.vec(CU), q);
                const float4 qq = lds4(qv, q), rq = lds4(rv_, q);
                sts4(X.vec(CU), q, fma4(a, pq, uq));
                const float4 r = fma4(-a, qq, rq);
                sts4(rv_, q, r);
                arr = dot4(r, r, arr);
            }
            float v[1] = {arr};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_step(sc, t[0]); })) return;
        }
        if (k == J.m || volatile_stopped(sc)) break;
        __syncthreads();
        conv_stage_taps<R, SEP>(S[0], J.tapsT);  // s = H^T r, beta
        __syncthreads();
        {
            float a0 = 0.f;
            conv_phase_res<R, SEP, PREC, false, false>(S, X, CR, nullptr, [&](int li, size_t, float z, float) {
                sv[li] = z;
                a0 = fmaf(z, z, a0);
            });
            float v[1] = {a0};
            if (!sy.reduce<1>(v, [&](DF* t) { fin_cg_s(sc, t[0]); })) return;
        }
        if (volatile_stopped(sc)) break;
        {  // p = s + beta p; the reduction is the barrier before other blocks read p's halo
            const float b = vldf(&sc->f_beta);
            for (int q = threadIdx.x; q < n4; q += NTHREADS) sts4(pv, q, fma4(b, lds4(pv, q), lds4(sv, q)));
            float v[1] = {0.f};
            ok = sy.reduce<1>(v, [&](DF*) {});
        }
    }
    if (!ok) return;
    const float* u = X.vec(CU);  // u back to global memory
    for (int lt = 0; lt < X.T; ++lt) {
        const int t = X.bid * X.T + lt;
        if (t >= X.ntiles) break;
        const int y0 = (t / X.tiles_x) * CONV_TH, x0 = (t % X.tiles_x) * CONV_TW;
        for (int p = threadIdx.x; p < TILE_PX; p += NTHREADS) {
            const int gy = y0 + p / CONV_TW, gx = x0 + p % CONV_TW;
            if (gy < X.h && gx < X.w) J.u[(size_t)gy * X.w + gx] = u[lt * TILE_PX + p];
        }
    }
}

}  // namespace res_detail

// One resident solve (MR-II, or CGLS) per cluster of LL.cluster blocks,
// LL.resident tiles per block; dynamic shared memory res_smem_bytes(LL.resident).
template <int R, bool SEP, bool PREC, bool CGLS>
__device__ __forceinline__ void level_res_kernel(const LevelLaunch& LL) {
    using namespace res_detail;
    __shared__ union {
        ConvSmem<R, SEP> conv[2];
        PsdSmem psd;  // phase 0: the level's start
    } U;
    ConvSmem<R, SEP>(&S)[2] = U.conv;
    __shared__ LevelJob sJ;
    __shared__ ClusterState CS;
    extern __shared__ float4 res_smem[];
    if (threadIdx.x == 0) sJ = LL.jobs ? LL.jobs[LL.block_job[blockIdx.x]] : LL.job;
    __syncthreads();
    const LevelJob& J = sJ;
    const unsigned int nb = LL.jobs ? (unsigned int)J.nblocks : gridDim.x;
    const unsigned int bid = LL.jobs ? blockIdx.x - (unsigned int)J.block0 : blockIdx.x;
    float* base = reinterpret_cast<float*>(res_smem);
    cluster_begin(CS, J.sc, nb);  // ends with a cluster barrier (every block's mbarrier ready)
    const int tiles_x = (J.w + CONV_TW - 1) / CONV_TW, tiles_y = (J.h + CONV_TH - 1) / CONV_TH;
    const ResCtx X{base, LL.resident, LL.resident * TILE_PX, (int)bid, tiles_x,
                   tiles_x * tiles_y, J.h, J.w};
    LevelSync sy{nullptr, J.gs, nb, bid, &CS, true, 0u};
    if constexpr (CGLS)
        cgls_res_body<R, SEP, PREC>(S, U.psd, J, &CS.sc, X, sy);
    else
        mr2_res_body<R, SEP, PREC>(S, U.psd, J, &CS.sc, X, sy);
    cluster_end(CS, J.sc, bid);
}

template <int R, bool SEP, bool PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_level_mr2_res(LevelLaunch LL) {
    level_res_kernel<R, SEP, PREC, false>(LL);
}

template <int R, bool SEP, bool PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_level_cgls_res(LevelLaunch LL) {
    level_res_kernel<R, SEP, PREC, true>(LL);
}

}  // namespace eecmg
