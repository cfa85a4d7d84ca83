// volume.cu -- EECMG on volumes (Algorithm 2 with every operator carried over
// to three dimensions; the paper names volumes as the method's next
// application without writing the 3-D operators out).
//
// The slice axis is treated exactly like the row and column axes:
//   restriction  coarse (a, b, c) = fine (2a, 2b, 2c)                (Eqs. 12-13)
//   H_l          zero-boundary 3-D convolution, K_l(o,p,q) = rho K(2o,2p,2q),
//                rho = N_{l+1} / N_l                                  (Eq. 14)
//   Pi           u^{l-1} + 1/4 of the trilinear interpolant of the level-(l-2)
//                differences                                         (Section 3.2)
//   P            the three-point quadratic rule along all three axes (Section 3.2)
//   S            weighted hyperplane fit over the 3x3x3 neighbourhood with the
//                Eq. 18 weights, pseudo-inverse of the 3x3 moment matrix
//                (eigenvalues under 1e-6 W dropped)                  (Section 3.3)
//   D            one explicit Perona-Malik step with six face neighbours
//                                                                    (Section 4)
//   C_l^m        MR-II with the discrepancy stop of Section 2 and m_l as its cap.
//
// GPU design.  A volume of d x h x w voxels is stored slice-major, x[(k h + i)
// w + j]; every level vector of the workspace is padded with zeros to a
// multiple of 4 voxels so the vector phases run on float4.  Each level solve is
// ONE cooperative launch (all blocks co-resident): its phases are separated by
// the grid barrier with the fused deterministic reduction of persistent.cuh
// (every block sums all blocks' partials in a fixed order and keeps its own
// replica of the scalars), so the m_l iterations never return to the host and
// the stop decision is taken on the device.  The convolution phases loop over
// 8 x 8 x 32 output tiles: a tile and its halo are staged in shared memory and
// a separable PSF runs as three passes (slices, rows, columns) inside the tile;
// a general PSF runs its non-zero taps from the staged tile (the level solve is
// in volume_impl.cuh).  The level start (Pi, P, S, D) is a chain of
// voxel-parallel kernels in this file.  The cascade is captured once as a CUDA
// graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.hpp"
#include "volume_impl.cuh"

namespace eecmg {
namespace vol {

// Voxel kernels run on a 3-D grid of 32 x 8 blocks: x = column, y = row,
// z = slice (no index division).
constexpr int VBX = 32, VBY = 8;

#define VOXEL_INDEX(d, h, w)                                          \
    const int j = blockIdx.x * VBX + (threadIdx.x & (VBX - 1));       \
    const int i = blockIdx.y * VBY + (threadIdx.x / VBX);             \
    const int k = blockIdx.z;                                         \
    if (j >= (w) || i >= (h)) return;                                 \
    const long long v = ((long long)k * (h) + i) * (w) + j;

__global__ void __launch_bounds__(VBX * VBY) k_vol_restrict(const float* __restrict__ f, int hf, int wf,
                                                            float* __restrict__ c, int dc, int hc, int wc) {
    VOXEL_INDEX(dc, hc, wc)
    c[v] = f[((long long)(2 * k) * hf + 2 * i) * wf + 2 * j];
}

// Pi: out = u1 + (1/4) * mean of the level-(l-2) differences d over the cell's
// eight corners (indices past the last level-(l-2) node clamp to it).
__global__ void __launch_bounds__(VBX * VBY) k_vol_pi(const float* __restrict__ u1, int d1, int h1, int w1,
                                                      const float* __restrict__ u2, int d2, int h2, int w2,
                                                      float* __restrict__ out) {
    VOXEL_INDEX(d1, h1, w1)
    const int c = k, a = i, b = j;
    const int C0 = c >> 1, C1 = (c & 1) ? min(C0 + 1, d2 - 1) : C0;
    const int A0 = a >> 1, A1 = (a & 1) ? min(A0 + 1, h2 - 1) : A0;
    const int B0 = b >> 1, B1 = (b & 1) ? min(B0 + 1, w2 - 1) : B0;
    const int Cs[2] = {C0, C1}, As[2] = {A0, A1}, Bs[2] = {B0, B1};
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int z = 0; z < 2; ++z)
                s += __ldg(u1 + ((long long)(2 * Cs[x]) * h1 + 2 * As[y]) * w1 + 2 * Bs[z]) -
                     __ldg(u2 + ((long long)Cs[x] * h2 + As[y]) * w2 + Bs[z]);
    out[v] = u1[v] + 0.03125f * s;
}

__constant__ float c_vqw[4][3] = {
    {1.f, 0.f, 0.f}, {0.375f, 0.75f, -0.125f}, {0.f, 1.f, 0.f}, {-0.125f, 0.75f, 0.375f}};

// P: the three-point quadratic rule along all three axes (clamped indices).
__global__ void __launch_bounds__(VBX * VBY) k_vol_quad(const float* __restrict__ ut, int d1, int h1, int w1,
                                                        float* __restrict__ out, int d, int h, int w) {
    VOXEL_INDEX(d, h, w)
    const int tz = k & 3, ty = i & 3, tx = j & 3;
    const int Z = (k >> 2) * 2, Y = (i >> 2) * 2, X = (j >> 2) * 2;
    int xs[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) xs[q] = min(X + q, w1 - 1);
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const float wz = c_vqw[tz][o];
        if (wz == 0.f) continue;
        const int c = min(Z + o, d1 - 1);
        float sy = 0.f;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float wy = c_vqw[ty][p];
            if (wy == 0.f) continue;
            const float* row = ut + ((long long)c * h1 + min(Y + p, h1 - 1)) * w1;
            float sx = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) sx = fmaf(c_vqw[tx][q], __ldg(row + xs[q]), sx);
            sy = fmaf(wy, sx, sy);
        }
        s = fmaf(wz, sy, s);
    }
    out[v] = s;
}

// slope . ob for slope = C^+ c (eigenvalues of C at most thr dropped), by the
// cyclic Jacobi method (Golub & Van Loan, Sec. 8.5): rotations in the (0,1),
// (0,2), (1,2) planes diagonalise the symmetric C; instead of accumulating
// the eigenvector matrix V, each rotation is applied to c and ob directly, so
// y = V^T c and z = V^T ob and the result is sum_k [lambda_k > thr] y_k z_k /
// lambda_k.  A rotation's angle needs no correct rounding (the rotation stays
// orthogonal to rounding whatever its angle, and the next sweep removes what
// it left), so t uses the fast division (its denominator is at least 1).
// Four sweeps.
__device__ __forceinline__ float jacobi_pinv_dot(float (&A)[3][3], float (&y)[3], float (&z)[3],
                                                 float thr) {
#pragma unroll
    for (int sweep = 0; sweep < 4; ++sweep) {
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2, r = 3 - p - q;
            const float apq = A[p][q];
            if (apq == 0.f) continue;
            const float th = (A[q][q] - A[p][p]) / (2.f * apq);  // IEEE: apq may be subnormal
            const float t = __fdividef(copysignf(1.f, th), fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
            const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
            A[p][p] = fmaf(-t, apq, A[p][p]);
            A[q][q] = fmaf(t, apq, A[q][q]);
            A[p][q] = A[q][p] = 0.f;
            const float arp = A[r][p], arq = A[r][q];
            A[r][p] = A[p][r] = c * arp - s * arq;
            A[r][q] = A[q][r] = s * arp + c * arq;
            const float yp = y[p], yq = y[q], zp = z[p], zq = z[q];
            y[p] = c * yp - s * yq;
            y[q] = s * yp + c * yq;
            z[p] = c * zp - s * zq;
            z[q] = s * zp + c * zq;
        }
    }
    float g = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (A[k][k] > thr) g = fmaf(__fdividef(y[k], A[k][k]), z[k], g);
    return g;
}

// S: per voxel, the weighted hyperplane fit over the in-volume 3x3x3
// neighbourhood (weights exp(-(scale v)^2), v = neighbour - centre) in centred
// form; the output is u + vb - slope . ob with slope = C^+ c.  When
// Gershgorin's bound puts every eigenvalue of C above 1e-2 W (far above the
// 1e-6 W cut), C^+ = C^-1 and the slope comes from the adjugate; otherwise from
// the Jacobi eigen-decomposition with the cut.
__global__ void __launch_bounds__(VBX * VBY) k_vol_smooth(const float* __restrict__ u, int d, int h, int w,
                                                          float scale, float* __restrict__ out) {
    VOXEL_INDEX(d, h, w)
    const float uc = u[v];
    float W = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f, vb = 0.f;
    float m00 = 0.f, m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    // raw weighted moments; centred afterwards (offsets are small integers)
#pragma unroll
    for (int r = -1; r <= 1; ++r) {
        if (k + r < 0 || k + r >= d) continue;
#pragma unroll
        for (int s = -1; s <= 1; ++s) {
            if (i + s < 0 || i + s >= h) continue;
            const float* row = u + ((long long)(k + r) * h + i + s) * w + j;
#pragma unroll
            for (int t = -1; t <= 1; ++t) {
                if (j + t < 0 || j + t >= w) continue;
                const float val = __ldg(row + t) - uc;
                const float e = scale * val;
                const float wt = (r == 0 && s == 0 && t == 0) ? 1.f : __expf(-e * e);
                W += wt;
                const float wv = wt * val;
                vb += wv;
                if (r) { o0 = fmaf(wt, (float)r, o0); m00 += wt; c0 = fmaf(wv, (float)r, c0); }
                if (s) { o1 = fmaf(wt, (float)s, o1); m11 += wt; c1 = fmaf(wv, (float)s, c1); }
                if (t) { o2 = fmaf(wt, (float)t, o2); m22 += wt; c2 = fmaf(wv, (float)t, c2); }
                if (r && s) m01 = fmaf(wt, (float)(r * s), m01);
                if (r && t) m02 = fmaf(wt, (float)(r * t), m02);
                if (s && t) m12 = fmaf(wt, (float)(s * t), m12);
            }
        }
    }
    const float iW = 1.f / W;
    o0 *= iW; o1 *= iW; o2 *= iW; vb *= iW;
    // centred moments: sum w (o - ob)(o' - ob') = sum w o o' - W ob ob'
    float A[3][3];
    A[0][0] = fmaf(-W * o0, o0, m00);
    A[1][1] = fmaf(-W * o1, o1, m11);
    A[2][2] = fmaf(-W * o2, o2, m22);
    A[0][1] = A[1][0] = fmaf(-W * o0, o1, m01);
    A[0][2] = A[2][0] = fmaf(-W * o0, o2, m02);
    A[1][2] = A[2][1] = fmaf(-W * o1, o2, m12);
    // sum w (o - ob)(v - vb) = sum w o v - W ob vb
    const float cv0 = fmaf(-W * o0, vb, c0), cv1 = fmaf(-W * o1, vb, c1), cv2 = fmaf(-W * o2, vb, c2);
    const float gersh = fminf(A[0][0] - fabsf(A[0][1]) - fabsf(A[0][2]),
                              fminf(A[1][1] - fabsf(A[0][1]) - fabsf(A[1][2]),
                                    A[2][2] - fabsf(A[0][2]) - fabsf(A[1][2])));
    float gob;
    if (gersh > 1e-2f * W) {
        const float k00 = A[1][1] * A[2][2] - A[1][2] * A[1][2];
        const float k01 = A[0][2] * A[1][2] - A[0][1] * A[2][2];
        const float k02 = A[0][1] * A[1][2] - A[0][2] * A[1][1];
        const float k11 = A[0][0] * A[2][2] - A[0][2] * A[0][2];
        const float k12 = A[0][1] * A[0][2] - A[0][0] * A[1][2];
        const float k22 = A[0][0] * A[1][1] - A[0][1] * A[0][1];
        const float idet = 1.f / (A[0][0] * k00 + A[0][1] * k01 + A[0][2] * k02);
        const float g0 = (k00 * cv0 + k01 * cv1 + k02 * cv2) * idet;
        const float g1 = (k01 * cv0 + k11 * cv1 + k12 * cv2) * idet;
        const float g2 = (k02 * cv0 + k12 * cv1 + k22 * cv2) * idet;
        gob = g0 * o0 + g1 * o1 + g2 * o2;
    } else {
        float y[3] = {cv0, cv1, cv2}, z[3] = {o0, o1, o2};
        gob = jacobi_pinv_dot(A, y, z, 1e-6f * W);
    }
    out[v] = uc + vb - gob;
}

// D, first half: the diffusivity c = 1 / (1 + |grad u|^2 / k^2), central
// differences, an out-of-volume neighbour replaced by the centre.
__global__ void __launch_bounds__(VBX * VBY) k_vol_pm_c(const float* __restrict__ u, int d, int h, int w,
                                                        float ik2, float* __restrict__ c) {
    VOXEL_INDEX(d, h, w)
    const long long sl = (long long)h * w;
    const float uc = u[v];
    const float ub = k + 1 < d ? u[v + sl] : uc, ua = k > 0 ? u[v - sl] : uc;
    const float us = i + 1 < h ? u[v + w] : uc, un = i > 0 ? u[v - w] : uc;
    const float ue = j + 1 < w ? u[v + 1] : uc, uw = j > 0 ? u[v - 1] : uc;
    const float gx = 0.5f * (ue - uw), gy = 0.5f * (us - un), gz = 0.5f * (ub - ua);
    c[v] = 1.f / (1.f + (gx * gx + gy * gy + gz * gz) * ik2);
}

// D, second half: u' = u + tau sum over in-volume face neighbours of
// (c_nb + c) / 2 (u_nb - u) (no flux through the volume's faces).
__global__ void __launch_bounds__(VBX * VBY) k_vol_pm_step(const float* __restrict__ u, const float* __restrict__ c,
                                                           int d, int h, int w, float tau,
                                                           float* __restrict__ out) {
    VOXEL_INDEX(d, h, w)
    const long long sl = (long long)h * w;
    const float uc = u[v], cc = c[v];
    float f = 0.f;
    if (k + 1 < d) f = fmaf(0.5f * (c[v + sl] + cc), u[v + sl] - uc, f);
    if (k > 0) f = fmaf(0.5f * (c[v - sl] + cc), u[v - sl] - uc, f);
    if (i + 1 < h) f = fmaf(0.5f * (c[v + w] + cc), u[v + w] - uc, f);
    if (i > 0) f = fmaf(0.5f * (c[v - w] + cc), u[v - w] - uc, f);
    if (j + 1 < w) f = fmaf(0.5f * (c[v + 1] + cc), u[v + 1] - uc, f);
    if (j > 0) f = fmaf(0.5f * (c[v - 1] + cc), u[v - 1] - uc, f);
    out[v] = fmaf(tau, f, uc);
}

}  // namespace vol
}  // namespace eecmg

// ====================================================================== host

using namespace eecmg;
using namespace eecmg::vol;

struct eecmg_vol_s {
    int W = 0, H = 0, D = 0, L = 0;
    double tau = 0.2, kpm = 10.0;
    eecmg_options opt{};
    int device = 0, sms = 0;
    std::vector<int> ds, hs, ws, m;
    std::vector<long long> n, n4;
    std::vector<VolTaps> taps, tapsT;                  // H_l and H_l^T
    std::vector<std::vector<int4>> gt, gtT;            // general-form tap lists (host)
    char* wsp = nullptr;
    size_t ws_bytes = 0;
    std::vector<float*> g, u;                          // per level (padded)
    float* vec[8] = {};                                // R, P0..2, Q0..2, Z (finest size)
    int4* dtaps = nullptr;                             // all tap lists, [2l] H, [2l+1] H^T
    std::vector<size_t> dtap_off;
    GroupSync* gs = nullptr;                           // one per level
    double* partials = nullptr;
    double* out = nullptr;                             // 4 doubles per level
    std::vector<int> grid;                             // level solve blocks
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // optional per-launch timing (eager launches with an event pair around
    // each level start and each level solve)
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // [4l .. 4l+3]: start begin/end, solve begin/end
    std::vector<int> ev_used;
};

namespace {

#define VCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_error(EECMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Correlation-form taps of the PSF K (kd x kh x kw): C(d) = K(-d) for H,
// C(d) = K(d) for H^T.  A PSF that is an outer product of three vectors (to
// FP64 rounding) is stored as its three factors.
void make_vol_taps(const std::vector<double>& K, int kd, int kh, int kw, bool transpose,
                   VolTaps* t, std::vector<int4>* list) {
    std::memset(t, 0, sizeof(VolTaps));
    const int rz = kd / 2, ry = kh / 2, rx = kw / 2;
    const int r = std::max(rz, std::max(ry, rx));
    t->r = r;
    auto C = [&](int o, int p, int q) {
        if (!transpose) { o = -o; p = -p; q = -q; }
        return K[((size_t)(o + rz) * kh + (p + ry)) * kw + (q + rx)];
    };
    int o0 = 0, p0 = 0, q0 = 0;
    double mx = -1.0;
    for (int o = -rz; o <= rz; ++o)
        for (int p = -ry; p <= ry; ++p)
            for (int q = -rx; q <= rx; ++q)
                if (std::fabs(C(o, p, q)) > mx) {
                    mx = std::fabs(C(o, p, q));
                    o0 = o;
                    p0 = p;
                    q0 = q;
                }
    bool sep = mx > 0.0;
    if (sep) {
        // C(o,p,q) = a(o) b(p) c(q) through the largest entry k0:
        // a(o) = C(o,p0,q0), b(p) = C(o0,p,q0) / k0, c(q) = C(o0,p0,q) / k0
        const double k0 = C(o0, p0, q0);
        std::vector<double> a(kd), b(kh), c(kw);
        for (int o = -rz; o <= rz; ++o) a[o + rz] = C(o, p0, q0);
        for (int p = -ry; p <= ry; ++p) b[p + ry] = C(o0, p, q0) / k0;
        for (int q = -rx; q <= rx; ++q) c[q + rx] = C(o0, p0, q) / k0;
        for (int o = -rz; o <= rz && sep; ++o)
            for (int p = -ry; p <= ry && sep; ++p)
                for (int q = -rx; q <= rx; ++q)
                    if (std::fabs(C(o, p, q) - a[o + rz] * b[p + ry] * c[q + rx]) > 1e-12 * mx) {
                        sep = false;
                        break;
                    }
        if (sep) {
            for (int o = 0; o < kd; ++o) t->cz[o - rz + r] = (float)a[o];
            for (int p = 0; p < kh; ++p) t->cy[p - ry + r] = (float)b[p];
            for (int q = 0; q < kw; ++q) t->cx[q - rx + r] = (float)c[q];
        }
    }
    t->sep = sep ? 1 : 0;
    list->clear();
    if (!sep) {
        for (int o = -rz; o <= rz; ++o)
            for (int p = -ry; p <= ry; ++p)
                for (int q = -rx; q <= rx; ++q) {
                    const double v = C(o, p, q);
                    if (v == 0.0) continue;
                    float f = (float)v;
                    int bits;
                    std::memcpy(&bits, &f, 4);
                    // offsets into the staged tile relative to the output voxel
                    list->push_back(make_int4(o, p, q, bits));
                }
    }
    t->ntap = (int)list->size();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t tile_bytes(const VolTaps& t) {
    const int NZ = TZ + 2 * t.r, NY = TY + 2 * t.r, AX = TX + 2 * ((t.r + 3) / 4 * 4);
    return sizeof(float) * (2 * (size_t)NZ * NY * AX + (t.sep ? (size_t)TZ * NY * AX : 0));
}

// The kernels of every radius 0 .. EECMG_VOL_MAX_RADIUS (instantiated in the
// volume_r*.cu translation units).
struct VolKernels {
    const void* solve[VR + 1];
    const void* apply[VR + 1];
};
const VolKernels& vol_kernels() {
    static_assert(VR == 6, "instantiate every radius");
    static const VolKernels k = [] {
        VolKernels t{};
        for (int r = 0; r <= VR; ++r)
            if (!vol_kernels_r012(r, &t.solve[r], &t.apply[r]) &&
                !vol_kernels_r34(r, &t.solve[r], &t.apply[r]))
                vol_kernels_r56(r, &t.solve[r], &t.apply[r]);
        return t;
    }();
    return k;
}

// The 3-D grid of the voxel kernels for a d x h x w volume.
dim3 vgrid(int d, int h, int w) { return dim3((w + VBX - 1) / VBX, (h + VBY - 1) / VBY, d); }
constexpr int VTHREADS = VBX * VBY;

VolJob make_job(eecmg_vol_s* P, int l, bool transpose) {
    VolJob J{};
    J.d = P->ds[l];
    J.h = P->hs[l];
    J.w = P->ws[l];
    J.n = P->n[l];
    J.n4 = P->n4[l];
    J.g = P->g[l];
    J.u = P->u[l];
    J.R = P->vec[0];
    for (int i = 0; i < 3; ++i) {
        J.P[i] = P->vec[1 + i];
        J.Q[i] = P->vec[4 + i];
    }
    J.Z = P->vec[7];
    J.taps = transpose ? P->tapsT[l] : P->taps[l];
    J.gtaps = P->dtaps + P->dtap_off[2 * l + (transpose ? 1 : 0)];
    // general-form offsets index the staged tile: (dz + rz) NY AX + ...; the
    // kernel adds the output's own position, so store dz, dy, dx as they are
    J.m = P->m[l];
    J.stop_tol = P->opt.stop == EECMG_STOP_DISCREPANCY ? P->opt.c * P->opt.delta : 0.0;
    J.conv_tol = P->opt.conv_tol;
    J.partials = P->partials;
    J.gs = P->gs + l;
    J.out = P->out + 4 * l;
    return J;
}

int level_tiles(const VolJob& J) {
    return ((J.w + TX - 1) / TX) * ((J.h + TY - 1) / TY) * ((J.d + TZ - 1) / TZ);
}

eecmg_status launch_solve(eecmg_vol_s* P, int l, bool zero_start, cudaStream_t s) {
    VolJob J = make_job(P, l, false);
    J.zero_start = zero_start ? 1 : 0;
    void* args[] = {&J};
    const size_t smem = tile_bytes(J.taps);
    VCK(cudaLaunchCooperativeKernel(vol_kernels().solve[J.taps.r], dim3(P->grid[l]), dim3(NTHREADS),
                                    args, smem, s));
    return EECMG_OK;
}

eecmg_status launch_apply(eecmg_vol_s* P, int l, bool transpose, const float* x, float* y,
                          cudaStream_t s) {
    VolJob J = make_job(P, l, transpose);
    const size_t smem = tile_bytes(J.taps);
    const float* xx = x;
    void* args[] = {&J, (void*)&xx, (void*)&y};
    VCK(cudaLaunchKernel(vol_kernels().apply[J.taps.r], dim3(level_tiles(J)), dim3(NTHREADS), args,
                         smem, s));
    return EECMG_OK;
}

// D(S(P(Pi(u1, u2)))) of level l (l >= 2) into out; uses R, Z, P0, Q0 as
// temporaries (none of them is live between level solves).
eecmg_status launch_start(eecmg_vol_s* P, int l, const float* u1, const float* u2, float* out,
                          cudaStream_t s) {
    const int d1 = P->ds[l - 1], h1 = P->hs[l - 1], w1 = P->ws[l - 1];
    const int d = P->ds[l], h = P->hs[l], w = P->ws[l];
    float* ue = P->vec[4];   // Q0: Pi on level l-1
    float* ut = P->vec[0];   // R: P(Pi)
    float* sa = P->vec[1];   // P0
    float* cc = P->vec[7];   // Z: diffusivity
    k_vol_pi<<<vgrid(d1, h1, w1), VTHREADS, 0, s>>>(u1, d1, h1, w1, u2, P->ds[l - 2], P->hs[l - 2],
                                                    P->ws[l - 2], ue);
    k_vol_quad<<<vgrid(d, h, w), VTHREADS, 0, s>>>(ue, d1, h1, w1, ut, d, h, w);
    const int steps = P->opt.diffusion_steps;
    float* cur = steps == 0 ? out : sa;
    k_vol_smooth<<<vgrid(d, h, w), VTHREADS, 0, s>>>(ut, d, h, w, (float)P->opt.s_scale, cur);
    const float ik2 = (float)(1.0 / (P->kpm * P->kpm));
    for (int st = 0; st < steps; ++st) {
        float* nxt = st == steps - 1 ? out : (cur == sa ? ut : sa);
        k_vol_pm_c<<<vgrid(d, h, w), VTHREADS, 0, s>>>(cur, d, h, w, ik2, cc);
        k_vol_pm_step<<<vgrid(d, h, w), VTHREADS, 0, s>>>(cur, cc, d, h, w, (float)P->tau, nxt);
        cur = nxt;
    }
    VCK(cudaGetLastError());
    return EECMG_OK;
}

eecmg_status cascade(eecmg_vol_s* P, cudaStream_t s) {
    const int L = P->L;
    auto mark = [&](int l, int which) -> eecmg_status {
        if (!P->prof) return EECMG_OK;
        VCK(cudaEventRecord(P->ev[4 * l + which], s));
        P->ev_used[4 * l + which] = 1;
        return EECMG_OK;
    };
    for (int l = L - 1; l > 0; --l) {
        k_vol_restrict<<<vgrid(P->ds[l - 1], P->hs[l - 1], P->ws[l - 1]), VTHREADS, 0, s>>>(P->g[l], P->hs[l], P->ws[l],
                                                             P->g[l - 1], P->ds[l - 1],
                                                             P->hs[l - 1], P->ws[l - 1]);
        VCK(cudaGetLastError());
    }
    for (int l = 0; l < L; ++l) {
        eecmg_status st;
        if (l >= 2) {
            if ((st = mark(l, 0)) != EECMG_OK) return st;
            st = launch_start(P, l, P->u[l - 1], P->u[l - 2], P->u[l], s);
            if (st != EECMG_OK) return st;
            if ((st = mark(l, 1)) != EECMG_OK) return st;
        }
        if ((st = mark(l, 2)) != EECMG_OK) return st;
        st = launch_solve(P, l, l < 2, s);
        if (st != EECMG_OK) return st;
        if ((st = mark(l, 3)) != EECMG_OK) return st;
    }
    return EECMG_OK;
}

// Algorithmic bytes of level l's solve from the iterations it ran (each
// operand read or written once per phase, FP32): r0 12 per voxel; p1 = H r 8;
// q1 = H p with <r, q> 12; the first update 24; then per iteration k >= 1:
// z = H q_k with <z, q_k> (and <z, q_{k-1}> for k >= 2) 8 (12), the new
// directions 24 (32), the update 24.  A breakdown ends a level after the
// phase that found it.
double solve_bytes(const eecmg_vol_s* P, int l, int k, int reason) {
    double b = 12.0;
    const bool ran_first = k >= 1 || reason == 2;
    if (ran_first) b += 8.0 + 12.0;
    if (k >= 1) b += 24.0;
    for (int j = 1; j < k; ++j) b += (j >= 2 ? 12.0 : 8.0) + (j >= 2 ? 32.0 : 24.0) + 24.0;
    if (k >= 1 && reason == 2) b += (k >= 2 ? 12.0 : 8.0) + (k >= 2 ? 32.0 : 24.0);
    return b * (double)P->n[l];
}

// The cascade on the workspace's g_L (filled by the caller), as one CUDA graph
// captured at the first call (use_graph) or as plain launches.
eecmg_status run_cascade(eecmg_vol_s* P, cudaStream_t s) {
    if (!P->opt.use_graph || P->prof) return cascade(P, s);
    if (!P->gexec) {
        VCK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
        eecmg_status st = cascade(P, P->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(P->cap, &graph);
        if (st != EECMG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess)
            return set_error(EECMG_ERR_CUDA, std::string("volume graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->gexec = nullptr;
            return set_error(EECMG_ERR_CUDA, std::string("volume graph instantiate: ") + cudaGetErrorString(e));
        }
    }
    VCK(cudaGraphLaunch(P->gexec, s));
    return EECMG_OK;
}

eecmg_status check_level(eecmg_vol_s* P, int level, const char* who) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, std::string(who) + ": NULL plan");
    if (level < 0 || level >= P->L)
        return set_error(EECMG_ERR_INVALID_ARG, std::string(who) + ": level out of range");
    return EECMG_OK;
}

}  // namespace

extern "C" {

eecmg_status eecmg_vol_plan(int width, int height, int depth, int levels, const double* psf,
                            int psf_w, int psf_h, int psf_d, double alpha, double k,
                            const int* iters, const eecmg_options* opt, eecmg_vol_t* out) {
    if (!out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: out is NULL");
    *out = nullptr;
    if (width < 1 || height < 1 || depth < 1 || levels < 1 || levels > 16)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: bad volume size or levels");
    if ((long long)width * height * depth > (1LL << 31) || depth > 65535)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_vol_plan: volume above 2^31 voxels or 65535 slices");
    if (!psf || psf_w < 1 || psf_h < 1 || psf_d < 1 || !(psf_w & 1) || !(psf_h & 1) || !(psf_d & 1) ||
        psf_w / 2 > VR || psf_h / 2 > VR || psf_d / 2 > VR)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_vol_plan: PSF sides must be odd with radius <= EECMG_VOL_MAX_RADIUS");
    if (!(alpha >= 0.0 && alpha <= 0.25) || !(k > 0.0))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: need 0 <= alpha <= 0.25 and k > 0");
    eecmg_options o;
    eecmg_default_options(&o);
    if (opt) o = *opt;
    if (o.smoother != EECMG_SMOOTHER_MR2 || o.prolong != EECMG_PROLONG_EECMG ||
        o.storage != EECMG_STORAGE_FP32 || !o.workspace)
        return set_error(EECMG_ERR_UNSUPPORTED,
                         "eecmg_vol_plan: volumes run MR-II, Algorithm 2, FP32, with a workspace");
    if ((o.coarse_op != EECMG_COARSE_GALERKIN_RMS && o.coarse_op != EECMG_COARSE_GALERKIN_RENORM) ||
        (o.stop != EECMG_STOP_FIXED && o.stop != EECMG_STOP_DISCREPANCY) || !(o.c > 1.0) ||
        !(o.delta >= 0.0) || o.diffusion_steps < 0 || o.diffusion_steps > 64 || !(o.conv_tol >= 0.0) ||
        !std::isfinite(o.s_scale))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: invalid option");
    const int nk = psf_w * psf_h * psf_d;
    std::vector<double> K(psf, psf + nk);
    double ksum = 0.0;
    for (double v : K) {
        if (!std::isfinite(v)) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: PSF not finite");
        ksum += v;
    }
    if (!(ksum > 0.0)) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: PSF sum must be positive");
    for (int i = 0; i < nk; ++i)  // MR-II needs H symmetric: K(d) = K(-d)
        if (std::fabs(K[i] - K[nk - 1 - i]) > 1e-12 * std::fabs(ksum))
            return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_vol_plan: MR-II needs a centrosymmetric PSF");
    if (iters)
        for (int l = 0; l < levels; ++l)
            if (iters[l] < 0) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan: iters < 0");

    auto* P = new eecmg_vol_s();
    P->W = width;
    P->H = height;
    P->D = depth;
    P->L = levels;
    P->tau = alpha;
    P->kpm = k;
    P->opt = o;
    const int L = levels;
    P->ds.resize(L);
    P->hs.resize(L);
    P->ws.resize(L);
    P->m.resize(L);
    P->ds[L - 1] = depth;
    P->hs[L - 1] = height;
    P->ws[L - 1] = width;
    for (int l = L - 1; l > 0; --l) {
        P->ds[l - 1] = (P->ds[l] + 1) / 2;
        P->hs[l - 1] = (P->hs[l] + 1) / 2;
        P->ws[l - 1] = (P->ws[l] + 1) / 2;
    }
    for (int l = 0; l < L; ++l) P->m[l] = iters ? iters[l] : schedule_m(L, l + 1);
    P->n.resize(L);
    P->n4.resize(L);
    for (int l = 0; l < L; ++l) {
        P->n[l] = (long long)P->ds[l] * P->hs[l] * P->ws[l];
        P->n4[l] = (P->n[l] + 3) / 4;
    }
    // level PSFs (Eq. 14 in 3-D; RENORM rescales to the fine PSF's sum)
    std::vector<std::vector<double>> Kl(L);
    std::vector<int> kdl(L), khl(L), kwl(L);
    Kl[L - 1] = K;
    kdl[L - 1] = psf_d;
    khl[L - 1] = psf_h;
    kwl[L - 1] = psf_w;
    for (int l = L - 1; l > 0; --l) {
        const double rho = (double)P->n[l] / (double)P->n[l - 1];
        const int rz = kdl[l] / 2, ry = khl[l] / 2, rx = kwl[l] / 2;
        const int cz = rz / 2, cy = ry / 2, cx = rx / 2;
        kdl[l - 1] = 2 * cz + 1;
        khl[l - 1] = 2 * cy + 1;
        kwl[l - 1] = 2 * cx + 1;
        Kl[l - 1].assign((size_t)kdl[l - 1] * khl[l - 1] * kwl[l - 1], 0.0);
        for (int a = -cz; a <= cz; ++a)
            for (int b = -cy; b <= cy; ++b)
                for (int c = -cx; c <= cx; ++c)
                    Kl[l - 1][((size_t)(a + cz) * khl[l - 1] + (b + cy)) * kwl[l - 1] + (c + cx)] =
                        rho * Kl[l][((size_t)(2 * a + rz) * khl[l] + (2 * b + ry)) * kwl[l] + (2 * c + rx)];
        if (o.coarse_op == EECMG_COARSE_GALERKIN_RENORM) {
            double s = 0.0;
            bool nz = false;
            for (double v : Kl[l - 1]) {
                s += v;
                nz = nz || v != 0.0;
            }
            if (s != 0.0 && nz)
                for (double& v : Kl[l - 1]) v *= ksum / s;
        }
    }
    P->taps.resize(L);
    P->tapsT.resize(L);
    P->gt.resize(L);
    P->gtT.resize(L);
    size_t ntaps = 0;
    for (int l = 0; l < L; ++l) {
        make_vol_taps(Kl[l], kdl[l], khl[l], kwl[l], false, &P->taps[l], &P->gt[l]);
        make_vol_taps(Kl[l], kdl[l], khl[l], kwl[l], true, &P->tapsT[l], &P->gtT[l]);
        ntaps += P->gt[l].size() + P->gtT[l].size() + 2;
    }
    // workspace: g and u per level, 8 solver vectors, taps, barriers, partials
    eecmg_status st = EECMG_OK;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_vol_plan: ") + cudaGetErrorString(e));
    }
    P->grid.resize(L);
    int maxgrid = 1;
    for (int l = 0; l < L; ++l) {
        const int r = std::max(P->taps[l].r, P->tapsT[l].r);
        const size_t smem = std::max(tile_bytes(P->taps[l]), tile_bytes(P->tapsT[l]));
        e = cudaFuncSetAttribute(vol_kernels().solve[r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(vol_kernels().apply[r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        int per = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vol_kernels().solve[r], NTHREADS, smem);
        if (e != cudaSuccess || per < 1) {
            delete P;
            return set_error(EECMG_ERR_CUDA, "eecmg_vol_plan: level solve does not fit an SM");
        }
        VolJob J{};
        J.d = P->ds[l];
        J.h = P->hs[l];
        J.w = P->ws[l];
        const long long want = std::max<long long>(level_tiles(J), (P->n4[l] + NTHREADS - 1) / NTHREADS);
        const long long cap = (long long)per * P->sms;
        P->grid[l] = (int)std::max<long long>(1, std::min(want, cap));
        maxgrid = std::max(maxgrid, P->grid[l]);
    }
    size_t off = 0;
    std::vector<size_t> goff(L), uoff(L), voff(8);
    for (int l = 0; l < L; ++l) {
        goff[l] = off;
        off = align256(off + (size_t)P->n4[l] * 16);
        uoff[l] = off;
        off = align256(off + (size_t)P->n4[l] * 16);
    }
    for (int i = 0; i < 8; ++i) {
        voff[i] = off;
        off = align256(off + (size_t)P->n4[L - 1] * 16);
    }
    const size_t taps_off = off;
    off = align256(off + ntaps * sizeof(int4));
    const size_t gs_off = off;
    off = align256(off + (size_t)L * sizeof(GroupSync));
    const size_t out_off = off;
    off = align256(off + (size_t)L * 4 * sizeof(double));
    const size_t part_off = off;
    off = align256(off + (size_t)2 * maxgrid * NPART * sizeof(double));
    e = cudaMalloc((void**)&P->wsp, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return set_error(EECMG_ERR_OOM, "eecmg_vol_plan: workspace allocation failed");
    }
    P->ws_bytes = off;
    e = cudaMemset(P->wsp, 0, off);
    P->g.resize(L);
    P->u.resize(L);
    for (int l = 0; l < L; ++l) {
        P->g[l] = (float*)(P->wsp + goff[l]);
        P->u[l] = (float*)(P->wsp + uoff[l]);
    }
    for (int i = 0; i < 8; ++i) P->vec[i] = (float*)(P->wsp + voff[i]);
    P->dtaps = (int4*)(P->wsp + taps_off);
    P->gs = (GroupSync*)(P->wsp + gs_off);
    P->out = (double*)(P->wsp + out_off);
    P->partials = (double*)(P->wsp + part_off);
    std::vector<int4> all;
    P->dtap_off.resize(2 * L);
    for (int l = 0; l < L; ++l) {
        P->dtap_off[2 * l] = all.size();
        all.insert(all.end(), P->gt[l].begin(), P->gt[l].end());
        all.push_back(make_int4(0, 0, 0, 0));
        P->dtap_off[2 * l + 1] = all.size();
        all.insert(all.end(), P->gtT[l].begin(), P->gtT[l].end());
        all.push_back(make_int4(0, 0, 0, 0));
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(P->dtaps, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        st = set_error(EECMG_ERR_CUDA, std::string("eecmg_vol_plan: ") + cudaGetErrorString(e));
        cudaFree(P->wsp);
        delete P;
        return st;
    }
    *out = P;
    return EECMG_OK;
}

eecmg_status eecmg_vol_plan_destroy(eecmg_vol_t P) {
    if (!P) return EECMG_OK;
    cudaDeviceSynchronize();
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->cap) cudaStreamDestroy(P->cap);
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    if (P->wsp) cudaFree(P->wsp);
    delete P;
    return EECMG_OK;
}

eecmg_status eecmg_vol_plan_info(eecmg_vol_t P, int* levels, int* level_w, int* level_h,
                                 int* level_d, int* iters, size_t* workspace_bytes) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan_info: NULL plan");
    if (levels) *levels = P->L;
    for (int l = 0; l < P->L; ++l) {
        if (level_w) level_w[l] = P->ws[l];
        if (level_h) level_h[l] = P->hs[l];
        if (level_d) level_d[l] = P->ds[l];
        if (iters) iters[l] = P->m[l];
    }
    if (workspace_bytes) *workspace_bytes = P->ws_bytes;
    return EECMG_OK;
}

eecmg_status eecmg_vol_restore(eecmg_vol_t P, const float* g, float* u, cudaStream_t s) {
    if (!P || !g || !u) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_restore: NULL argument");
    const size_t bytes = (size_t)P->n[P->L - 1] * sizeof(float);
    VCK(cudaMemcpyAsync(P->g[P->L - 1], g, bytes, cudaMemcpyDeviceToDevice, s));
    eecmg_status st = run_cascade(P, s);
    if (st != EECMG_OK) return st;
    VCK(cudaMemcpyAsync(u, P->u[P->L - 1], bytes, cudaMemcpyDeviceToDevice, s));
    return EECMG_OK;
}

eecmg_status eecmg_vol_restore_host(eecmg_vol_t P, const float* g_host, float* u_host,
                                    cudaStream_t s) {
    if (!P || !g_host || !u_host)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_restore_host: NULL argument");
    const size_t bytes = (size_t)P->n[P->L - 1] * sizeof(float);
    VCK(cudaMemcpyAsync(P->g[P->L - 1], g_host, bytes, cudaMemcpyHostToDevice, s));
    eecmg_status st = run_cascade(P, s);
    if (st != EECMG_OK) return st;
    VCK(cudaMemcpyAsync(u_host, P->u[P->L - 1], bytes, cudaMemcpyDeviceToHost, s));
    VCK(cudaStreamSynchronize(s));
    return EECMG_OK;
}

eecmg_status eecmg_vol_plan_stats(eecmg_vol_t P, int* iters_done, double* res_rms) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan_stats: NULL plan");
    VCK(cudaDeviceSynchronize());
    std::vector<double> h(4 * (size_t)P->L);
    VCK(cudaMemcpy(h.data(), P->out, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<GroupSync> gs(P->L);
    VCK(cudaMemcpy(gs.data(), P->gs, gs.size() * sizeof(GroupSync), cudaMemcpyDeviceToHost));
    for (int l = 0; l < P->L; ++l) {
        if (iters_done) iters_done[l] = (int)h[4 * l];
        if (res_rms) res_rms[l] = std::sqrt(h[4 * l + 1] / (double)P->n[l]);
        if (gs[l].err) return set_error(EECMG_ERR_TIMEOUT, "eecmg_vol_plan_stats: a grid barrier timed out");
    }
    return EECMG_OK;
}

eecmg_status eecmg_vol_apply_H(eecmg_vol_t P, int level, const float* x, float* y, int transpose,
                               cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_apply_H");
    if (st != EECMG_OK) return st;
    if (!x || !y || x == y) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_apply_H: bad buffers");
    return launch_apply(P, level, transpose != 0, x, y, s);
}

eecmg_status eecmg_vol_start_level(eecmg_vol_t P, int level, const float* u1, const float* u2,
                                   float* out, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_start_level");
    if (st != EECMG_OK) return st;
    if (level < 2 || !u1 || !u2 || !out)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_start_level: needs level >= 2 and buffers");
    return launch_start(P, level, u1, u2, out, s);
}

eecmg_status eecmg_vol_smooth(eecmg_vol_t P, int level, const float* x, float* y, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_smooth");
    if (st != EECMG_OK) return st;
    if (!x || !y || x == y) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_smooth: bad buffers");
    k_vol_smooth<<<vgrid(P->ds[level], P->hs[level], P->ws[level]), VTHREADS, 0, s>>>(x, P->ds[level], P->hs[level], P->ws[level],
                                                        (float)P->opt.s_scale, y);
    VCK(cudaGetLastError());
    return EECMG_OK;
}

eecmg_status eecmg_vol_denoise(eecmg_vol_t P, int level, const float* x, float* y, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_denoise");
    if (st != EECMG_OK) return st;
    if (!x || !y || x == y) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_denoise: bad buffers");
    const int d = P->ds[level], h = P->hs[level], w = P->ws[level];
    k_vol_pm_c<<<vgrid(d, h, w), VTHREADS, 0, s>>>(x, d, h, w, (float)(1.0 / (P->kpm * P->kpm)),
                                                      P->vec[7]);
    k_vol_pm_step<<<vgrid(d, h, w), VTHREADS, 0, s>>>(x, P->vec[7], d, h, w, (float)P->tau, y);
    VCK(cudaGetLastError());
    return EECMG_OK;
}

eecmg_status eecmg_vol_restrict(eecmg_vol_t P, int level, const float* fine, float* coarse,
                                cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_restrict");
    if (st != EECMG_OK) return st;
    if (level >= P->L - 1 || !fine || !coarse)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_restrict: level must be below the finest");
    k_vol_restrict<<<vgrid(P->ds[level], P->hs[level], P->ws[level]), VTHREADS, 0, s>>>(fine, P->hs[level + 1], P->ws[level + 1],
                                                          coarse, P->ds[level], P->hs[level],
                                                          P->ws[level]);
    VCK(cudaGetLastError());
    return EECMG_OK;
}

eecmg_status eecmg_vol_level_solve(eecmg_vol_t P, int level, const float* g, float* u, int m,
                                   cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_vol_level_solve");
    if (st != EECMG_OK) return st;
    if (!g || !u || m < 0) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_level_solve: bad arguments");
    const size_t bytes = (size_t)P->n[level] * sizeof(float);
    VCK(cudaMemcpyAsync(P->g[level], g, bytes, cudaMemcpyDeviceToDevice, s));
    VCK(cudaMemcpyAsync(P->u[level], u, bytes, cudaMemcpyDeviceToDevice, s));
    const int keep = P->m[level];
    P->m[level] = m;
    st = launch_solve(P, level, false, s);
    P->m[level] = keep;
    if (st != EECMG_OK) return st;
    VCK(cudaMemcpyAsync(u, P->u[level], bytes, cudaMemcpyDeviceToDevice, s));
    return EECMG_OK;
}

eecmg_status eecmg_vol_plan_profile(eecmg_vol_t P, int enable) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan_profile: NULL plan");
    if (enable && P->ev.empty()) {
        P->ev.resize(4 * (size_t)P->L);
        for (auto& e : P->ev) VCK(cudaEventCreate(&e));
    }
    P->ev_used.assign(4 * (size_t)P->L, 0);
    P->prof = enable != 0;
    return EECMG_OK;
}

eecmg_status eecmg_vol_plan_profile_read(eecmg_vol_t P, double* start_ms, double* solve_ms,
                                         double* solve_bytes_out) {
    if (!P || !P->prof) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_vol_plan_profile_read: profiling is off");
    VCK(cudaDeviceSynchronize());
    std::vector<double> h(4 * (size_t)P->L);
    VCK(cudaMemcpy(h.data(), P->out, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int l = 0; l < P->L; ++l) {
        float a = 0.f, b = 0.f;
        if (P->ev_used[4 * l] && P->ev_used[4 * l + 1])
            VCK(cudaEventElapsedTime(&a, P->ev[4 * l], P->ev[4 * l + 1]));
        if (P->ev_used[4 * l + 2] && P->ev_used[4 * l + 3])
            VCK(cudaEventElapsedTime(&b, P->ev[4 * l + 2], P->ev[4 * l + 3]));
        if (start_ms) start_ms[l] = a;
        if (solve_ms) solve_ms[l] = b;
        if (solve_bytes_out) solve_bytes_out[l] = solve_bytes(P, l, (int)h[4 * l], (int)h[4 * l + 2]);
    }
    return EECMG_OK;
}

}  // extern "C"
