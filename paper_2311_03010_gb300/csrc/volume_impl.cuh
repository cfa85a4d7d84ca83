// volume_impl.cuh -- the level solve of the volume path (internal): the
// convolution tile and the persistent MR-II kernel, templated on the level
// PSF's radius R.  The instantiations R = 0 .. EECMG_VOL_MAX_RADIUS are split
// over the volume_r*.cu translation units (compile time); volume.cu holds the
// voxel kernels of the level start, the planner and the C ABI.
#pragma once

#include <cstdint>

#include "../../include/eecmg.h"
#include "common.cuh"
#include "persistent.cuh"

namespace eecmg {
namespace vol {

constexpr int VR = EECMG_VOL_MAX_RADIUS;
constexpr int VK = 2 * VR + 1;
constexpr int TX = 32, TY = 8, TZ = 8;  // output tile (columns, rows, slices)

// Taps of one level in correlation form, y(v) = sum_d C(d) x(v + d), C(d) = K(-d),
// centred at r = the level PSF's largest radius (shorter axes padded with zeros).
struct VolTaps {
    int r;
    int sep;                       // 1: C = cz (x) cy (x) cx
    float cz[VK], cy[VK], cx[VK];  // factors, index d + r
    int ntap;                      // general form: taps in the job's tap list
};

struct VolJob {
    int d, h, w;
    long long n;    // voxels
    long long n4;   // padded voxels / 4
    const float* g;
    float* u;
    float* R;
    float* P[3];
    float* Q[3];
    float* Z;
    VolTaps taps;
    const int4* gtaps;  // general form: (dz, dy, dx, weight bits)
    int m;
    int zero_start;
    double stop_tol;    // discrepancy: stop once ||r||_RMS <= stop_tol (0: off)
    double conv_tol;    // stop once ||r|| <= conv_tol ||g|| (0: off)
    double* partials;
    GroupSync* gs;
    double* out;        // [0] iterations, [1] ||r||^2, [2] stop reason
};

// Per-block replica of the solve's scalars (identical in every block).
struct VolScal {
    double rr, gg, qq, qqp, qqn, a, b1, b2;
    int k, done;
};

// -------------------------------------------------------------------- tile
//
// A block loops over its output tiles t = blockIdx.x, + gridDim.x, ...  The
// input window of a tile (the tile plus an r-voxel halo, zero outside the
// volume) is fetched with cp.async (16-byte chunks where rows are 16-byte
// aligned, else 4-byte copies; zero fill past the volume) into one of two
// shared-memory buffers while the previous tile is convolved from the other.
// The separable form runs three passes in shared memory: slices over every
// staged (row, column) into B, rows over B into C (C reuses the tile's own
// input buffer), columns over C; the first two slide a register window along
// their axis, so each staged value is read once.  The general form sums its
// tap list over the window.

template <int R>
struct VolTile {
    // a staged row starts PADX = R rounded up to 4 voxels left of the tile, so
    // rows are whole 16-byte chunks; voxel x of the window sits at X0 + x
    static constexpr int PADX = (R + 3) / 4 * 4, X0 = PADX - R;
    static constexpr int NZ = TZ + 2 * R, NY = TY + 2 * R, AX = TX + 2 * PADX;
    static constexpr int IN = NZ * NY * AX;  // one input buffer
    static constexpr int MID = TZ * NY * AX; // B: the slice pass's output
    static constexpr size_t bytes(bool sep) { return sizeof(float) * (2 * (size_t)IN + (sep ? MID : 0)); }
};

__device__ __forceinline__ int num_tiles(const VolJob& J) {
    return ((J.w + TX - 1) / TX) * ((J.h + TY - 1) / TY) * ((J.d + TZ - 1) / TZ);
}

__device__ __forceinline__ void tile_origin(const VolJob& J, int t, int& x0, int& y0, int& z0) {
    const int ntx = (J.w + TX - 1) / TX, nty = (J.h + TY - 1) / TY;
    x0 = (t % ntx) * TX;
    y0 = ((t / ntx) % nty) * TY;
    z0 = (t / ntx / nty) * TZ;
}

template <int R>
__device__ __forceinline__ void stage_tile(const VolJob& J, const float* __restrict__ x, int t, float* A) {
    using T = VolTile<R>;
    int x0, y0, z0;
    tile_origin(J, t, x0, y0, z0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int base = (unsigned int)__cvta_generic_to_shared(A);
    if ((J.w & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        // 16-byte chunks: rows are 16-byte aligned in memory (w a multiple of 4,
        // x 16-byte aligned) and a chunk is
        // either inside the row or wholly past one of its ends (zero fill)
        constexpr int CH = T::AX / 4;           // chunks per row
        constexpr int RPW = 32 / CH;            // rows per warp instruction
        constexpr int ROWS = T::NZ * T::NY;
        const int sub = lane / CH, c = lane - sub * CH;
        for (int r0 = warp * RPW; r0 < ROWS; r0 += (NTHREADS / 32) * RPW) {
            const int row = r0 + sub;
            if (sub >= RPW || row >= ROWS) continue;
            const int za = row / T::NY, ya = row - za * T::NY;
            const int gz = z0 - R + za, gy = y0 - R + ya, gx = x0 - T::PADX + 4 * c;
            const bool in = gz >= 0 && gz < J.d && gy >= 0 && gy < J.h && gx >= 0 && gx < J.w;
            const float* g = in ? x + ((long long)gz * J.h + gy) * J.w + gx : x;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             base + 4u * (unsigned int)(row * T::AX + 4 * c)),
                         "l"(g), "r"(in ? 16 : 0)
                         : "memory");
        }
    } else {
        for (int row = warp; row < T::NZ * T::NY; row += NTHREADS / 32) {
            const int za = row / T::NY, ya = row - za * T::NY;
            const int gz = z0 - R + za, gy = y0 - R + ya;
            const bool rin = gz >= 0 && gz < J.d && gy >= 0 && gy < J.h;
            const float* src = x + ((long long)(rin ? gz : 0) * J.h + (rin ? gy : 0)) * J.w;
#pragma unroll
            for (int xa = lane; xa < T::AX; xa += 32) {
                const int gx = x0 - T::PADX + xa;
                const bool in = rin && gx >= 0 && gx < J.w;
                const float* g = in ? src + gx : x;  // a valid address either way
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                 base + 4u * (unsigned int)(row * T::AX + xa)),
                             "l"(g), "r"(in ? 4 : 0)
                             : "memory");
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Convolves the staged tile t (buffer A) and calls epi(voxel index, (H x)(v))
// for every in-volume output.  Ends with __syncthreads().
template <int R, class Epi>
__device__ __forceinline__ void compute_tile(const VolJob& J, int t, float* A, float* B, Epi&& epi) {
    using T = VolTile<R>;
    const VolTaps& K = J.taps;
    int x0, y0, z0;
    tile_origin(J, t, x0, y0, z0);
    const int xo = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp = output row within a slice
    const int gx = x0 + xo, gy = y0 + warp;
    // the epilogue's read-only operands of this thread's outputs, fetched
    // before the passes so that their latency hides behind the convolution
    const bool col_in = gy < J.h && gx < J.w;
    float2 pre[TZ];
#pragma unroll
    for (int zo = 0; zo < TZ; ++zo)
        pre[zo] = (col_in && z0 + zo < J.d) ? epi.pre(((long long)(z0 + zo) * J.h + gy) * J.w + gx)
                                            : make_float2(0.f, 0.f);
    if (K.sep) {
        // slices first: B[z][y][x] = sum_dz cz A[z + dz][y][x] for the TZ output
        // slices, every staged (y, x) column; each thread slides a register
        // window down its column, so a staged value is read once
        constexpr int COLS = T::NY * T::AX;
        for (int c = threadIdx.x; c < COLS; c += NTHREADS) {
            float win[T::NZ];
#pragma unroll
            for (int z = 0; z < T::NZ; ++z) win[z] = A[z * COLS + c];
#pragma unroll
            for (int zo = 0; zo < TZ; ++zo) {
                float s = 0.f;
#pragma unroll
                for (int o = 0; o <= 2 * R; ++o) s = fmaf(K.cz[o], win[zo + o], s);
                B[zo * COLS + c] = s;
            }
        }
        __syncthreads();
        // rows: C[z][y][x] = sum_dy cy B[z][y + dy][x] for the TY output rows,
        // every (z, x) column (C over the window's own buffer)
        float* C = A;
        constexpr int COLS2 = TZ * T::AX;
        for (int c = threadIdx.x; c < COLS2; c += NTHREADS) {
            const int z = c / T::AX, x = c - z * T::AX;
            const float* b = B + z * COLS + x;
            float win[T::NY];
#pragma unroll
            for (int y = 0; y < T::NY; ++y) win[y] = b[y * T::AX];
#pragma unroll
            for (int yo = 0; yo < TY; ++yo) {
                float s = 0.f;
#pragma unroll
                for (int p = 0; p <= 2 * R; ++p) s = fmaf(K.cy[p], win[yo + p], s);
                C[(z * TY + yo) * T::AX + x] = s;
            }
        }
        __syncthreads();
        // columns: out[z][y][x] = sum_dx cx C[z][y][X0 + x + dx]
        float s[TZ];
#pragma unroll
        for (int zo = 0; zo < TZ; ++zo) {
            s[zo] = 0.f;
            const float* c = C + (zo * TY + warp) * T::AX + T::X0 + xo;
#pragma unroll
            for (int q = 0; q <= 2 * R; ++q) s[zo] = fmaf(K.cx[q], c[q], s[zo]);
        }
        if (col_in) {
#pragma unroll
            for (int zo = 0; zo < TZ; ++zo)
                if (z0 + zo < J.d) epi(((long long)(z0 + zo) * J.h + gy) * J.w + gx, s[zo], pre[zo]);
        }
    } else {
#pragma unroll
        for (int zo = 0; zo < TZ; ++zo) {
            const float* a = A + ((zo + R) * T::NY + warp + R) * T::AX + T::X0 + xo + R;
            float s = 0.f;
            for (int k = 0; k < K.ntap; ++k) {
                const int4 tp = __ldg(J.gtaps + k);
                s = fmaf(__int_as_float(tp.w), a[(tp.x * T::NY + tp.y) * T::AX + tp.z], s);
            }
            if (z0 + zo < J.d && col_in) epi(((long long)(z0 + zo) * J.h + gy) * J.w + gx, s, pre[zo]);
        }
    }
    __syncthreads();  // the buffers are restaged after this
}

// An epilogue: pre(v) loads the operands output v needs (at most two floats,
// issued before the convolution), op(v, (H x)(v), operands) consumes them.
template <class Pre, class Op>
struct Epilogue {
    Pre pre;
    Op op;
    __device__ __forceinline__ void operator()(long long v, float hx, float2 p) { op(v, hx, p); }
};
template <class Pre, class Op>
__device__ __forceinline__ Epilogue<Pre, Op> epilogue(Pre pre, Op op) {
    return Epilogue<Pre, Op>{pre, op};
}
__device__ __forceinline__ float2 no_pre(long long) { return make_float2(0.f, 0.f); }

// One convolution phase: H x over all the block's tiles, the next tile's
// window in flight while the current one is convolved.
template <int R, class Epi>
__device__ __forceinline__ void conv_phase(const VolJob& J, const float* __restrict__ x, float* sm,
                                           Epi&& epi) {
    using T = VolTile<R>;
    const int ntiles = num_tiles(J), nb = gridDim.x;
    int t = blockIdx.x;
    if (t >= ntiles) return;  // the whole block
    float* B = sm + 2 * T::IN;
    int buf = 0;
    stage_tile<R>(J, x, t, sm);
    for (; t < ntiles; t += nb) {
        if (t + nb < ntiles) {
            stage_tile<R>(J, x, t + nb, sm + (buf ^ 1) * T::IN);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        compute_tile<R>(J, t, sm + buf * T::IN, B, epi);
        buf ^= 1;
    }
}



// per-thread compensated sum (cascaded: the rounding errors are kept in lo)
__device__ __forceinline__ void acc_add(DF& a, float v) {
    const DF s = two_sum(a.hi, v);
    a.hi = s.hi;
    a.lo += s.lo;
}

__device__ __forceinline__ double tot2(const DF (&t)[4], int j) {
    return df_to_double(t[2 * j]) + df_to_double(t[2 * j + 1]);
}

// A vector phase over float4 elements i = gtid, gtid + gstr, ...: two elements
// per step, every load of both issued before the first store (the stores may
// alias nothing the loads need, but the compiler cannot prove it).
// f(x, y) maps the NL loaded values to the NS stored ones.
template <int NL, int NS, class F>
__device__ __forceinline__ void vec_phase(long long n4, long long gtid, long long gstr,
                                          const float4* const (&in)[NL], float4* const (&out)[NS],
                                          F&& f) {
    for (long long i = gtid; i < n4; i += 2 * gstr) {
        const long long j = i + gstr;
        const bool second = j < n4;
        float4 x0[NL], x1[NL], y[NS];
#pragma unroll
        for (int k = 0; k < NL; ++k) x0[k] = __ldcg(in[k] + i);
        if (second) {
#pragma unroll
            for (int k = 0; k < NL; ++k) x1[k] = __ldcg(in[k] + j);
        }
        f(x0, y);
#pragma unroll
        for (int k = 0; k < NS; ++k) out[k][i] = y[k];
        if (second) {
            f(x1, y);
#pragma unroll
            for (int k = 0; k < NS; ++k) out[k][j] = y[k];
        }
    }
}

// ------------------------------------------------------------- level solve

// Stop test of the oracle's level smoother, checked before every iteration.
__device__ __forceinline__ bool level_done(const VolJob& J, double rr, double gg) {
    if (J.stop_tol > 0.0 && sqrt(rr / (double)J.n) <= J.stop_tol) return true;
    if (J.conv_tol > 0.0 && sqrt(rr) <= J.conv_tol * sqrt(gg)) return true;
    return false;
}

__device__ __forceinline__ bool pos_finite(double x) { return x > 0.0 && isfinite(x); }

// MR-II (the three-term recurrence of the oracle's level smoother):
//   r0 = g - H u0;  p1 = H r0, q1 = H p1, a = <r,q>/<q,q>, u += a p, r -= a q;
//   then while k < m and the stop test fails:
//   z = H q_k, b1 = <z,q_k>/<q_k,q_k>, b2 = <z,q_{k-1}>/<q_{k-1},q_{k-1}> (k >= 2),
//   q_{k+1} = z - b1 q_k - b2 q_{k-1}, p_{k+1} = q_k - b1 p_k - b2 p_{k-1},
//   a = <r,q_{k+1}>/<q_{k+1},q_{k+1}>, u += a p_{k+1}, r -= a q_{k+1}.
// p and q live in rings of three buffers: p_k = P[(k - 1) % 3].
template <int R>
__global__ void __launch_bounds__(NTHREADS, 2) k_vol_mr2(VolJob J) {
    extern __shared__ __align__(16) float sm[];
    __shared__ VolScal S;
    const unsigned int nb = gridDim.x, bid = blockIdx.x;
    const long long gtid = (long long)bid * NTHREADS + threadIdx.x, gstr = (long long)nb * NTHREADS;
    unsigned int phase = 0;
    bool ok = true;
    auto reduce = [&](const DF (&acc)[2], auto&& fin) {
        float v[4] = {acc[0].hi, acc[0].lo, acc[1].hi, acc[1].lo};
        return grid_reduce<4>(v, J.partials, J.gs, nb, bid, phase++, fin);
    };
    float4* u4 = reinterpret_cast<float4*>(J.u);
    float4* r4 = reinterpret_cast<float4*>(J.R);
    const float4* g4 = reinterpret_cast<const float4*>(J.g);

    // r0 = g - H u0 (a zero start writes u = 0, r = g); ||r||^2, ||g||^2
    {
        // the vector phases run on whole float4s: zero the (at most 3) padding
        // voxels past n of every vector this solve reads, whatever an earlier
        // use of the shared buffers left there
        const long long pad = 4 * J.n4 - J.n;
        if (gtid < pad) {
            const long long i = J.n + gtid;
            J.u[i] = 0.f;
            J.R[i] = 0.f;
            J.Z[i] = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                J.P[b][i] = 0.f;
                J.Q[b][i] = 0.f;
            }
        }
        DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
        if (J.zero_start) {
            for (long long i = gtid; i < J.n4; i += gstr) {
                const float4 g = __ldcg(g4 + i);
                u4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                r4[i] = g;
                acc_add(acc[0], dot4(g, g, 0.f));
                acc_add(acc[1], dot4(g, g, 0.f));
            }
        } else {
            conv_phase<R>(J, J.u, sm, epilogue(
                [&](long long i) { return make_float2(__ldcg(J.g + i), 0.f); },
                [&](long long i, float hx, float2 p) {
                    const float g = p.x;
                    const float r = g - hx;
                    J.R[i] = r;
                    acc_add(acc[0], r * r);
                    acc_add(acc[1], g * g);
                }));
        }
        ok = reduce(acc, [&](const DF (&t)[4]) {
            S.rr = tot2(t, 0);
            S.gg = tot2(t, 1);
            S.k = 0;
            S.done = (J.m <= 0 || level_done(J, S.rr, S.gg)) ? 1 : 0;
        });
    }
    if (ok && !S.done) {
        // p1 = H r0
        conv_phase<R>(J, J.R, sm, epilogue(no_pre, [&](long long i, float hx, float2) { J.P[0][i] = hx; }));
        DF none[2] = {{0.f, 0.f}, {0.f, 0.f}};
        ok = reduce(none, [&](const DF (&)[4]) {});
    }
    if (ok && !S.done) {
        // q1 = H p1; <q,q>, <r,q>
        DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
        conv_phase<R>(J, J.P[0], sm, epilogue(
            [&](long long i) { return make_float2(__ldcg(J.R + i), 0.f); },
            [&](long long i, float hx, float2 p) {
                J.Q[0][i] = hx;
                acc_add(acc[0], hx * hx);
                acc_add(acc[1], p.x * hx);
            }));
        ok = reduce(acc, [&](const DF (&t)[4]) {
            const double qq = tot2(t, 0), rq = tot2(t, 1);
            if (!pos_finite(qq)) {
                S.done = 2;
            } else {
                S.qq = qq;
                S.a = rq / qq;
            }
        });
    }
    if (ok && !S.done) {
        // u += a p1, r -= a q1; ||r||^2
        DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
        const float a = (float)S.a;
        const float4* const in[4] = {reinterpret_cast<const float4*>(J.P[0]),
                                     reinterpret_cast<const float4*>(J.Q[0]), u4, r4};
        float4* const out[2] = {u4, r4};
        vec_phase<4, 2>(J.n4, gtid, gstr, in, out, [&](const float4 (&x)[4], float4 (&y)[2]) {
            y[0] = fma4(a, x[0], x[2]);
            y[1] = fma4(-a, x[1], x[3]);
            acc_add(acc[0], dot4(y[1], y[1], 0.f));
        });
        ok = reduce(acc, [&](const DF (&t)[4]) {
            S.rr = tot2(t, 0);
            S.k = 1;
            S.qqp = 0.0;
            S.done = (S.k >= J.m || level_done(J, S.rr, S.gg)) ? 1 : 0;
        });
    }
    while (ok && !S.done) {
        const int k = S.k;
        const int cur = (k - 1) % 3, prv = (k + 1) % 3, nxt = k % 3;
        const float* q = J.Q[cur];
        const float* qp = J.Q[prv];
        const bool two = k >= 2;
        // z = H q_k; <z, q_k>, <z, q_{k-1}>
        {
            DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
            conv_phase<R>(J, q, sm, epilogue(
                [&](long long i) { return make_float2(__ldcg(q + i), two ? __ldcg(qp + i) : 0.f); },
                [&](long long i, float hx, float2 p) {
                    J.Z[i] = hx;
                    acc_add(acc[0], hx * p.x);
                    if (two) acc_add(acc[1], hx * p.y);
                }));
            ok = reduce(acc, [&](const DF (&t)[4]) {
                S.b1 = tot2(t, 0) / S.qq;
                S.b2 = two ? tot2(t, 1) / S.qqp : 0.0;
            });
            if (!ok) break;
        }
        // q_{k+1}, p_{k+1}; <q_{k+1}, q_{k+1}>, <r, q_{k+1}>
        {
            DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
            const float b1 = (float)S.b1, b2 = (float)S.b2;
            float4* const out[2] = {reinterpret_cast<float4*>(J.Q[nxt]), reinterpret_cast<float4*>(J.P[nxt])};
            if (two) {
                const float4* const in[6] = {reinterpret_cast<const float4*>(J.Z),
                                             reinterpret_cast<const float4*>(J.Q[cur]),
                                             reinterpret_cast<const float4*>(J.P[cur]), r4,
                                             reinterpret_cast<const float4*>(J.Q[prv]),
                                             reinterpret_cast<const float4*>(J.P[prv])};
                vec_phase<6, 2>(J.n4, gtid, gstr, in, out, [&](const float4 (&x)[6], float4 (&y)[2]) {
                    y[0] = fma4(-b2, x[4], fma4(-b1, x[1], x[0]));
                    y[1] = fma4(-b2, x[5], fma4(-b1, x[2], x[1]));
                    acc_add(acc[0], dot4(y[0], y[0], 0.f));
                    acc_add(acc[1], dot4(x[3], y[0], 0.f));
                });
            } else {
                const float4* const in[4] = {reinterpret_cast<const float4*>(J.Z),
                                             reinterpret_cast<const float4*>(J.Q[cur]),
                                             reinterpret_cast<const float4*>(J.P[cur]), r4};
                vec_phase<4, 2>(J.n4, gtid, gstr, in, out, [&](const float4 (&x)[4], float4 (&y)[2]) {
                    y[0] = fma4(-b1, x[1], x[0]);
                    y[1] = fma4(-b1, x[2], x[1]);
                    acc_add(acc[0], dot4(y[0], y[0], 0.f));
                    acc_add(acc[1], dot4(x[3], y[0], 0.f));
                });
            }
            ok = reduce(acc, [&](const DF (&t)[4]) {
                const double qqn = tot2(t, 0), rqn = tot2(t, 1);
                if (!pos_finite(qqn)) {
                    S.done = 2;
                } else {
                    S.qqn = qqn;
                    S.a = rqn / qqn;
                }
            });
            if (!ok || S.done) break;
        }
        // u += a p_{k+1}, r -= a q_{k+1}; ||r||^2
        {
            DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
            const float a = (float)S.a;
            const float4* const in[4] = {reinterpret_cast<const float4*>(J.P[nxt]),
                                         reinterpret_cast<const float4*>(J.Q[nxt]), u4, r4};
            float4* const out[2] = {u4, r4};
            vec_phase<4, 2>(J.n4, gtid, gstr, in, out, [&](const float4 (&x)[4], float4 (&y)[2]) {
                y[0] = fma4(a, x[0], x[2]);
                y[1] = fma4(-a, x[1], x[3]);
                acc_add(acc[0], dot4(y[1], y[1], 0.f));
            });
            ok = reduce(acc, [&](const DF (&t)[4]) {
                S.rr = tot2(t, 0);
                S.qqp = S.qq;
                S.qq = S.qqn;
                S.k = S.k + 1;
                S.done = (S.k >= J.m || level_done(J, S.rr, S.gg)) ? 1 : 0;
            });
        }
    }
    if (bid == 0 && threadIdx.x == 0) {
        J.out[0] = S.k;
        J.out[1] = S.rr;
        J.out[2] = ok ? S.done : -1;
    }
    grid_exit(J.gs, nb);
}

// H x (or H^T x with the transposed taps) of a whole level, one tile per block.
template <int R>
__global__ void __launch_bounds__(NTHREADS) k_vol_apply(VolJob J, const float* __restrict__ x,
                                                        float* __restrict__ y) {
    extern __shared__ __align__(16) float sm[];
    stage_tile<R>(J, x, blockIdx.x, sm);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    compute_tile<R>(J, blockIdx.x, sm, sm + 2 * VolTile<R>::IN,
                    epilogue(no_pre, [&](long long i, float hx, float2) { y[i] = hx; }));
}

// ------------------------------------------------------------ level start

// The solve and apply kernels of radius r (0 .. EECMG_VOL_MAX_RADIUS), from the
// translation unit that instantiates them; false if r is outside its range.
bool vol_kernels_r012(int r, const void** solve, const void** apply);
bool vol_kernels_r34(int r, const void** solve, const void** apply);
bool vol_kernels_r56(int r, const void** solve, const void** apply);

}  // namespace vol
}  // namespace eecmg
