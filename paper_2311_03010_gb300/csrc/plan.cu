// plan.cu -- planner, cascade driver and C ABI of the EECMG library.
//
// A plan fixes the level sizes (Section 2: each coarser side is ceil(n/2)),
// the per-level PSFs of the Galerkin coarse operators (Eq. 14), the
// economy iteration schedule (Section 2) and a device workspace.  A
// restoration enqueues Algorithm 2 on a stream without any host round trip
// (all Krylov scalars are decided on the device) and is captured once as a
// CUDA graph, then replayed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "launch.hpp"
#include "level_solve.hpp"
#include "plan.hpp"

using namespace eecmg;

namespace eecmg {

thread_local std::string g_last_error = "no error";

eecmg_status set_error(eecmg_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

static eecmg_status no_ws(const char* who) {
    return set_error(EECMG_ERR_INVALID_ARG,
                     std::string(who) + ": the plan is a description only (workspace = 0)");
}

// Economy schedule m_l (Section 2) in exact integer arithmetic, l = 1..L:
//   l > L/2:  m_l = ceil((L - L/2)^2 4^(L-l)) = ceil(L^2 4^(L-l) / 4)
//   l <= L/2: m_l = ceil((L - 1.5 l) 4^(l-1)) = ceil((2L - 3l) 4^(l-1) / 2)
// and at least 1 ("the smallest positive integer not less than t").
int schedule_m(int L, int l) {
    long long v;
    if (2 * l > L) {
        long long num = (long long)L * L;
        for (int i = 0; i < L - l; ++i) num *= 4;
        v = (num + 3) / 4;
    } else {
        long long num = 2LL * L - 3LL * l;
        for (int i = 0; i < l - 1; ++i) num *= 4;
        v = num > 0 ? (num + 1) / 2 : 1;
    }
    return v < 1 ? 1 : (int)v;
}

}  // namespace eecmg

namespace {

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_error(EECMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Host PSF in convolution form, kh x kw, centred.
struct Psf {
    int kh = 1, kw = 1;
    std::vector<double> k{1.0};
    double at(int p, int q) const { return k[(size_t)(p + kh / 2) * kw + (q + kw / 2)]; }
};

// Eq. 14 with the RMS adjoint: K_c(p, q) = rho * K(2p, 2q).
Psf coarsen(const Psf& f, double rho) {
    Psf c;
    const int ry = f.kh / 2 / 2, rx = f.kw / 2 / 2;
    c.kh = 2 * ry + 1;
    c.kw = 2 * rx + 1;
    c.k.assign((size_t)c.kh * c.kw, 0.0);
    for (int p = -ry; p <= ry; ++p)
        for (int q = -rx; q <= rx; ++q) c.k[(size_t)(p + ry) * c.kw + (q + rx)] = rho * f.at(2 * p, 2 * q);
    return c;
}

bool centrosymmetric(const Psf& f) {
    double mx = 0.0;
    for (double v : f.k) mx = std::fmax(mx, std::fabs(v));
    for (int p = -f.kh / 2; p <= f.kh / 2; ++p)
        for (int q = -f.kw / 2; q <= f.kw / 2; ++q)
            if (std::fabs(f.at(p, q) - f.at(-p, -q)) > 1e-12 * mx) return false;
    return true;
}

// Fills the device descriptor (correlation form) for H (transpose = 0:
// C(dy, dx) = K(-dy, -dx)) or H^T (C = K).  Separable PSFs K = a b^T are
// detected to FP64 rounding and stored as two factors.
void make_taps(const Psf& f, bool transpose, Taps* t) {
    std::memset(t, 0, sizeof(Taps));
    const int ry = f.kh / 2, rx = f.kw / 2;
    const int rt = ry > rx ? ry : rx;
    t->ry = ry;
    t->rx = rx;
    t->rt = rt;
    auto C = [&](int dy, int dx) { return transpose ? f.at(dy, dx) : f.at(-dy, -dx); };
    // separability: K = a b^T through the largest entry
    int p0 = 0, q0 = 0;
    double mx = -1.0;
    for (int p = -ry; p <= ry; ++p)
        for (int q = -rx; q <= rx; ++q)
            if (std::fabs(C(p, q)) > mx) {
                mx = std::fabs(C(p, q));
                p0 = p;
                q0 = q;
            }
    bool sep = mx > 0.0;
    if (sep) {
        const double k00 = C(p0, q0);
        const double sc = 1.0 / std::sqrt(std::fabs(k00));
        const double sg = k00 < 0 ? -1.0 : 1.0;
        std::vector<double> a(2 * ry + 1), b(2 * rx + 1);
        for (int p = -ry; p <= ry; ++p) a[p + ry] = C(p, q0) * sc;
        for (int q = -rx; q <= rx; ++q) b[q + rx] = C(p0, q) * sc * sg;
        for (int p = -ry; p <= ry && sep; ++p)
            for (int q = -rx; q <= rx; ++q)
                if (std::fabs(C(p, q) - a[p + ry] * b[q + rx]) > 1e-12 * mx) {
                    sep = false;
                    break;
                }
        if (sep) {
            for (int p = -ry; p <= ry; ++p) t->cy[p + rt] = (float)a[p + ry];
            for (int q = -rx; q <= rx; ++q) t->cx[q + rt] = (float)b[q + rx];
        }
    }
    t->sep = sep ? 1 : 0;
    int n = 0;
    for (int dy = -ry; dy <= ry; ++dy)
        for (int dx = -rx; dx <= rx; ++dx) {
            const double v = C(dy, dx);
            if (v != 0.0) {
                t->dy[n] = dy;
                t->dx[n] = dx;
                t->wt[n] = (float)v;
                ++n;
            }
        }
    t->ntap = n;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace eecmg {

cudaEvent_t prof_event(Profiler& pr) {
    if (!pr.free_events.empty()) {
        cudaEvent_t e = pr.free_events.back();
        pr.free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Algorithmic bytes of a persistent level solve, from the iterations it ran
// (each operand read or written once per phase, FP32).
double level_solve_bytes(const eecmg_plan_s* P, int l, const Scalars& sc, bool zero_start) {
    const double n = (double)P->lv[l].h * P->lv[l].w;
    // bytes per element of the BF16-able direction vectors (MR-II d; CGLS s,
    // p): 2 in the BF16-storage variant
    const double e = P->opt.storage == EECMG_STORAGE_BF16 ? 2.0 : 4.0;
    // MR-II: the solver adds each phase's bytes per pixel as it runs (the early
    // checks of the discrepancy rule change which phases run)
    if (P->opt.smoother == EECMG_SMOOTHER_MR2) return sc.bpp * n;
    // CGLS: the solver records the bytes of the level's start (if it ran one) in bpp
    double b = (zero_start ? 8.0 : 12.0) * n + sc.bpp * n;  // start; r = g - H u
    const int K = sc.loops;
    {
        if (K > 0 || sc.iters > 0) b += (4.0 + 2 * e) * n;  // s = H^T r, p = s
        b += (e + 4.0 + e + 4.0 + 16.0) * n * K;          // q = H p; u, r update
        if (K > 1) b += (4.0 + e + 3 * e) * n * (K - 1);  // s = H^T r; p = s + beta p
    }
    return b;
}

// Folds the recorded launches into the per-class totals (synchronises).
cudaError_t prof_flush(eecmg_plan_s* P) {
    Profiler& pr = P->prof;
    for (auto& r : pr.recs) {
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        double bytes = r.bytes;
        if (r.level >= 0) {
            Scalars sc;
            e = cudaMemcpy(&sc, P->sc + r.level, sizeof(Scalars), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return e;
            bytes = level_solve_bytes(P, r.level, sc, r.bytes != 0.0);
        }
        pr.ms[r.cls] += ms;
        pr.bytes[r.cls] += bytes;
        pr.launches[r.cls] += 1;
        pr.free_events.push_back(r.e0);
        pr.free_events.push_back(r.e1);
    }
    pr.recs.clear();
    return cudaSuccess;
}

}  // namespace eecmg

// Launch with optional profiling: an event pair around the launch and its
// algorithmic byte count.
#define LK(P, s, cls, nbytes, call)                                              \
    do {                                                                         \
        if ((P)->prof.on) {                                                      \
            eecmg::Profiler::Rec rec_{(cls), (double)(nbytes), prof_event((P)->prof), \
                                      prof_event((P)->prof)};                    \
            cudaEventRecord(rec_.e0, (s));                                       \
            CK(call);                                                            \
            cudaEventRecord(rec_.e1, (s));                                       \
            (P)->prof.recs.push_back(rec_);                                      \
            if ((P)->prof.recs.size() > 8192) CK(prof_flush(P));         \
        } else {                                                                 \
            CK(call);                                                            \
        }                                                                        \
    } while (0)

// ---------------------------------------------------------------------------
// cascade enqueue
// ---------------------------------------------------------------------------

namespace eecmg {

void bind_workspace(eecmg_plan_s* P, char* ws) {
    const PlanLayout& Y = P->layout;
    P->ws = ws;
    for (int l = 0; l < P->L; ++l) {
        P->lv[l].g = (float*)(ws + Y.g_off[l]);
        P->lv[l].u = (float*)(ws + Y.u_off[l]);
    }
    for (int i = 0; i < eecmg_plan_s::NVEC; ++i) P->vec[i] = (float*)(ws + Y.vec_off[i]);
    P->dtaps = (Taps*)(ws + Y.taps_off);
    P->sc = (Scalars*)(ws + Y.sc_off);
    P->gsync = (GroupSync*)(ws + Y.gs_off);
    P->partials = (double*)(ws + Y.part_off);
}

bool level_fused_start(const eecmg_plan_s* P, int l) {
    return P->opt.fuse_start && P->opt.persistent && P->opt.prolong == EECMG_PROLONG_EECMG &&
           P->opt.diffusion_steps == 1 && l >= 2;
}

void set_level_start(const eecmg_plan_s* P, int l, LevelJob& J) {
    if (!level_fused_start(P, l)) return;
    const LevelPlan& L1 = P->lv[l - 1];
    const LevelPlan& L2 = P->lv[l - 2];
    J.start = 1;
    J.s_u1 = L1.u;
    J.s_u2 = L2.u;
    J.s_h1 = L1.h;
    J.s_w1 = L1.w;
    J.s_h2 = L2.h;
    J.s_w2 = L2.w;
    J.s_scale = (float)P->opt.s_scale;
    J.s_tau = (float)P->tau;
    const float kpm = (float)P->kpm;
    J.s_ik2 = 1.f / (kpm * kpm);
}

eecmg_status solve_level_enqueue(eecmg_plan_s* P, int l, const float* g, float* u, int m,
                                 bool zero_start, cudaStream_t s, bool own_start) {
    LevelPlan& L = P->lv[l];
    const size_t n = (size_t)L.h * L.w;
    Scalars* sc = P->sc + l;
    const Taps* tH = P->dtaps + 2 * l;
    const Taps* tHT = P->dtaps + 2 * l + 1;
    const int rt = L.rt, sepH = L.sepH, sepHT = L.sepHT, prec = P->opt.precise_conv;
    const bool mr2 = P->opt.smoother == EECMG_SMOOTHER_MR2;
    const int bf16 = P->opt.storage == EECMG_STORAGE_BF16 ? 1 : 0;
    float** V = P->vec;

    if (P->opt.persistent) {
        LevelJob J;
        J.g = g;
        J.u = u;
        for (int i = 0; i < 2; ++i) {
            J.v[i] = V[0 + i];
            J.aw[i] = V[2 + i];
            J.d[i] = V[4 + i];
            J.hd[i] = V[6 + i];
        }
        J.r = V[8];
        J.taps = tH;
        J.tapsT = tHT;
        J.sc = sc;
        J.partials = P->partials;
        J.gs = P->gsync + l;
        J.conv_tol2 = P->conv_tol2;
        J.disc2 = L.disc2;
        J.early = P->opt.early_check;
        J.h = L.h;
        J.w = L.w;
        J.m = m;
        J.zero_start = zero_start ? 1 : 0;
        if (own_start) set_level_start(P, l, J);
        int used = 0;
        if (P->prof.on) {
            // bytes field flags a zero start; the count itself is taken after the run
            Profiler::Rec rec{KC_LEVEL, zero_start ? 1.0 : 0.0, prof_event(P->prof),
                              prof_event(P->prof), l};
            cudaEventRecord(rec.e0, s);
            CK(launch_level_solve(J, rt, sepH, prec, mr2 ? 0 : 1, bf16, s, &used));
            cudaEventRecord(rec.e1, s);
            P->prof.recs.push_back(rec);
        } else {
            CK(launch_level_solve(J, rt, sepH, prec, mr2 ? 0 : 1, bf16, s, &used));
        }
        return EECMG_OK;
    }

    ConvArgs ra;
    ra.x = u;
    ra.y = V[8];                      // r
    ra.e0 = g;
    ra.taps = tH;
    ra.sc = sc;
    ra.partials = P->partials;
    ra.conv_tol2 = P->conv_tol2;
    ra.disc2 = L.disc2;
    ra.h = L.h;
    ra.w = L.w;
    ra.mode = CM_RESID;
    ra.zero_input = zero_start ? 1 : 0;
    LK(P, s, KC_CONV, 4.0 * n * 3 - (zero_start ? 4.0 * n : 0.0), launch_conv(ra, rt, sepH, prec, s));
    if (m <= 0) return EECMG_OK;

    if (mr2) {
        MrVecs mv;
        mv.v[0] = V[0];
        mv.v[1] = V[1];
        mv.aw[0] = V[2];
        mv.aw[1] = V[3];
        mv.d[0] = V[4];
        mv.d[1] = V[5];
        mv.hd[0] = V[6];
        mv.hd[1] = V[7];
        mv.u = u;
        mv.r = V[8];
        ConvArgs c;
        c.taps = tH;
        c.sc = sc;
        c.partials = P->partials;
        c.h = L.h;
        c.w = L.w;
        c.x = V[8];  // v_1 = H r_0
        c.y = mv.v[1];
        c.mode = CM_MR_V1;
        LK(P, s, KC_CONV, 8.0 * n, launch_conv(c, rt, sepH, prec, s));
        for (int k = 1; k <= m; ++k) {
            c.x = mv.v[k & 1];  // H w_k
            c.y = mv.aw[k & 1];
            c.mode = CM_MR_A;
            LK(P, s, KC_CONV, 8.0 * n, launch_conv(c, rt, sepH, prec, s));
            // step k-1 (k >= 2): reads v, Hw, u, r and 2/4 of the d/Hd history, writes d, Hd, u, r;
            // Lanczos: reads Hw_k, v_k (and r, v_{k-1} when k = 1), writes v_{k+1}
            const int j = k - 1;
            const double step_vec = j >= 1 ? 4 + (j >= 2 ? 2 : 0) + (j >= 3 ? 2 : 0) + 4 : 0;
            LK(P, s, KC_MR_B, 4.0 * n * (step_vec + (j >= 1 ? 3 : 4)),
               launch_mr_b(mv, k, n, sc, P->partials, s));
        }
        LK(P, s, KC_MR_FINAL, 4.0 * n * (4 + (m >= 2 ? 2 : 0) + (m >= 3 ? 2 : 0) + 4),
           launch_mr_final(mv, n, sc, P->partials, s));
    } else {
        float* rv = V[8];
        float* sv = V[0];
        float* pv = V[1];
        float* qv = V[2];
        ConvArgs c;
        c.sc = sc;
        c.partials = P->partials;
        c.h = L.h;
        c.w = L.w;
        c.x = rv;
        c.y = sv;
        c.y2 = pv;
        c.taps = tHT;
        c.mode = CM_CG_S0;
        LK(P, s, KC_CONV, 12.0 * n, launch_conv(c, rt, sepHT, prec, s));
        for (int k = 1; k <= m; ++k) {
            ConvArgs q = c;
            q.x = pv;
            q.y = qv;
            q.y2 = nullptr;
            q.taps = tH;
            q.mode = CM_CG_Q;
            LK(P, s, KC_CONV, 8.0 * n, launch_conv(q, rt, sepH, prec, s));
            LK(P, s, KC_CG_STEP, 24.0 * n, launch_cg_step(u, pv, rv, qv, n, sc, P->partials, s));
            if (k < m) {
                ConvArgs t = c;
                t.y2 = nullptr;
                t.mode = CM_CG_S;
                LK(P, s, KC_CONV, 8.0 * n, launch_conv(t, rt, sepHT, prec, s));
                LK(P, s, KC_CG_P, 12.0 * n, launch_cg_p(pv, sv, n, sc, s));
            }
        }
    }
    return EECMG_OK;
}

// Starting guess of level l >= the number of zero-started levels, written
// into u_l (Algorithm 2 Step 2 items 1-4, or Algorithm 1 Step 2 items 1-3).
eecmg_status prolong_enqueue(eecmg_plan_s* P, int l, cudaStream_t s) {
    LevelPlan& L = P->lv[l];
    LevelPlan& L1 = P->lv[l - 1];
    float* up = P->vec[0];  // prolonged, level l
    const int steps = P->opt.diffusion_steps;
    if (P->opt.prolong == EECMG_PROLONG_EECMG && steps >= 1) {
        // D(S(P(Pi(u_{l-1}, u_{l-2})))) in one pass, then the further D steps
        LevelPlan& L2 = P->lv[l - 2];
        float* sm = P->vec[1];
        float* first = steps == 1 ? L.u : sm;
        LK(P, s, KC_PROLONG, 4.0 * ((double)L1.h * L1.w + (double)L2.h * L2.w + (double)L.h * L.w),
           launch_psd(L1.u, L1.h, L1.w, L2.u, L2.h, L2.w, first, L.h, L.w, (float)P->opt.s_scale,
                      (float)P->tau, (float)P->kpm, s));
        float* cur = first;
        for (int d = 1; d < steps; ++d) {
            float* nxt = (d == steps - 1) ? L.u : (cur == sm ? up : sm);
            LK(P, s, KC_DENOISE, 8.0 * L.h * L.w,
               launch_denoise(cur, nxt, L.h, L.w, (float)P->tau, (float)P->kpm, s));
            cur = nxt;
        }
        return EECMG_OK;
    }
    if (P->opt.prolong == EECMG_PROLONG_EECMG) {  // P(Pi(u_{l-1}, u_{l-2})), one fused pass
        LevelPlan& L2 = P->lv[l - 2];
        LK(P, s, KC_PROLONG, 4.0 * ((double)L1.h * L1.w + (double)L2.h * L2.w + (double)L.h * L.w),
           launch_prolong(L1.u, L1.h, L1.w, L2.u, L2.h, L2.w, up, L.h, L.w, s));
    } else if (P->opt.prolong == EECMG_PROLONG_IECMG_P) {
        LK(P, s, KC_PROLONG, 4.0 * ((double)L1.h * L1.w + (double)L.h * L.w),
           launch_quadratic(L1.u, L1.h, L1.w, up, L.h, L.w, s));
    } else {
        LK(P, s, KC_PROLONG, 4.0 * ((double)L1.h * L1.w + (double)L.h * L.w),
           launch_linear(L1.u, L1.h, L1.w, up, L.h, L.w, s));
    }
    float* sm = P->vec[1];
    LK(P, s, KC_SMOOTH, 8.0 * L.h * L.w, launch_smooth(up, sm, L.h, L.w, (float)P->opt.s_scale, s));
    if (steps <= 0) {
        LK(P, s, KC_COPY, 8.0 * L.h * L.w,
           cudaMemcpyAsync(L.u, sm, sizeof(float) * L.h * L.w, cudaMemcpyDeviceToDevice, s));
        return EECMG_OK;
    }
    float* cur = sm;
    for (int d = 0; d < steps; ++d) {
        float* nxt = (d == steps - 1) ? L.u : (cur == sm ? up : sm);
        LK(P, s, KC_DENOISE, 8.0 * L.h * L.w,
           launch_denoise(cur, nxt, L.h, L.w, (float)P->tau, (float)P->kpm, s));
        cur = nxt;
    }
    return EECMG_OK;
}

eecmg_status cascade_enqueue(eecmg_plan_s* P, cudaStream_t s) {
    const int L = P->L;
    for (int l = L - 1; l > 0; --l)
        LK(P, s, KC_RESTRICT, 8.0 * P->lv[l - 1].h * P->lv[l - 1].w,
           launch_restrict(P->lv[l].g, P->lv[l].h, P->lv[l].w, P->lv[l - 1].g, P->lv[l - 1].h,
                           P->lv[l - 1].w, s));
    const int nzero = P->opt.prolong == EECMG_PROLONG_EECMG ? 2 : 1;
    for (int l = 0; l < L; ++l) {
        const bool zero = l < nzero;
        // a persistent solve writes its zero start, or runs the fused start of its level,
        // itself (one launch per cascade step)
        if (zero) {
            if (!P->opt.persistent)
                LK(P, s, KC_COPY, 4.0 * P->lv[l].h * P->lv[l].w,
                   cudaMemsetAsync(P->lv[l].u, 0, sizeof(float) * P->lv[l].h * P->lv[l].w, s));
        } else if (!level_fused_start(P, l)) {
            eecmg_status st = prolong_enqueue(P, l, s);
            if (st != EECMG_OK) return st;
        }
        eecmg_status st = solve_level_enqueue(P, l, P->lv[l].g, P->lv[l].u, P->lv[l].m, zero, s, true);
        if (st != EECMG_OK) return st;
    }
    return EECMG_OK;
}

eecmg_status run_cascade(eecmg_plan_s* P, cudaStream_t s) {
    if (!P->opt.use_graph || P->prof.on) return cascade_enqueue(P, s);
    if (!P->gexec) {
        CK(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
        eecmg_status st = cascade_enqueue(P, P->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(P->cap_stream, &graph);
        if (st != EECMG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return set_error(EECMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->gexec = nullptr;
            return set_error(EECMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
    }
    CK(cudaGraphLaunch(P->gexec, s));
    return EECMG_OK;
}

}  // namespace eecmg

namespace eecmg {

std::atomic<int> g_live_owners{0};

// Allocates, zeroes and fills the plan's device workspace (layout already
// computed) and its capture stream.  On failure nothing is left allocated.
eecmg_status plan_allocate(eecmg_plan_s* P, const char* who) {
    const size_t off = P->layout.bytes;
    cudaError_t e = cudaMalloc((void**)&P->ws, off);
    if (e != cudaSuccess) {
        P->ws = nullptr;
        cudaGetLastError();
        return set_error(EECMG_ERR_OOM, std::string(who) + ": workspace allocation failed: " +
                                            cudaGetErrorString(e));
    }
    bind_workspace(P, P->ws);
    e = cudaMemset(P->ws, 0, off);
    if (e == cudaSuccess)
        e = cudaMemcpy(P->dtaps, P->htaps.data(), sizeof(Taps) * 2 * P->L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(P->ws);
        P->ws = nullptr;
        if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
        P->cap_stream = nullptr;
        return set_error(EECMG_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
    }
    P->owns_ws = true;
    g_live_owners.fetch_add(1);
    return EECMG_OK;
}

// A new plan with D's description and its own workspace.
eecmg_status plan_materialize(const eecmg_plan_s* D, eecmg_plan_s** out) {
    *out = nullptr;
    auto* P = new (std::nothrow) eecmg_plan_s();
    if (!P) return set_error(EECMG_ERR_OOM, "host allocation failed");
    P->W = D->W;
    P->H = D->H;
    P->L = D->L;
    P->tau = D->tau;
    P->kpm = D->kpm;
    P->conv_tol2 = D->conv_tol2;
    P->opt = D->opt;
    P->opt.workspace = 1;
    P->device = D->device;
    P->lv = D->lv;
    P->htaps = D->htaps;
    P->layout = D->layout;
    P->ws_bytes = D->ws_bytes;
    P->max_blocks = D->max_blocks;
    eecmg_status st = plan_allocate(P, "plan_materialize");
    if (st != EECMG_OK) {
        delete P;
        return st;
    }
    *out = P;
    return EECMG_OK;
}

}  // namespace eecmg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* eecmg_last_error(void) { return g_last_error.c_str(); }

const char* eecmg_version(void) { return "eecmg-gb300 0.1 (sm_103a)"; }

eecmg_status eecmg_default_options(eecmg_options* o) {
    if (!o) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_default_options: NULL");
    o->smoother = EECMG_SMOOTHER_MR2;
    o->coarse_op = EECMG_COARSE_GALERKIN_RMS;
    o->storage = EECMG_STORAGE_FP32;
    o->stop = EECMG_STOP_DISCREPANCY;
    o->c = 1.1;
    o->delta = 0.0;
    o->diffusion_steps = 1;
    o->s_scale = 1.0;
    o->conv_tol = 1e-5;
    o->prolong = EECMG_PROLONG_EECMG;
    o->use_graph = 1;
    o->precise_conv = -1;
    o->persistent = 1;
    o->workspace = 1;
    o->fuse_start = 0;
    o->early_check = 1;
    return EECMG_OK;
}

eecmg_status eecmg_plan(int width, int height, int levels, const double* psf, int psf_w, int psf_h,
                        double alpha, double k, const int* iters, const eecmg_options* opt,
                        eecmg_plan_t* out) {
    if (!out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: out is NULL");
    *out = nullptr;
    if (width < 1 || height < 1 || levels < 1 || levels > 30)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: need width, height >= 1 and 1 <= levels <= 30");
    if (!psf || psf_w < 1 || psf_h < 1 || !(psf_w & 1) || !(psf_h & 1))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: PSF must be non-NULL with odd sizes");
    if (psf_w / 2 > EECMG_MAX_RADIUS || psf_h / 2 > EECMG_MAX_RADIUS)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: PSF radius exceeds EECMG_MAX_RADIUS");
    if (!(alpha >= 0.0 && alpha <= 0.25))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: alpha (tau) must be in [0, 0.25]");
    if (!(k > 0.0) || !std::isfinite(k)) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: k must be > 0");
    eecmg_options o;
    eecmg_default_options(&o);
    if (opt) o = *opt;
    if (o.smoother < 0 || o.smoother > 1 || o.coarse_op < 0 || o.coarse_op > 1 || o.storage < 0 ||
        o.storage > 1 || o.stop < 0 || o.stop > 1 || o.prolong < 0 || o.prolong > 2 ||
        o.diffusion_steps < 0 || !(o.conv_tol >= 0.0) || !(o.s_scale >= 0.0) ||
        o.precise_conv < -1 || o.precise_conv > 1 || o.fuse_start < 0 || o.fuse_start > 1 ||
        o.early_check < 0 || o.early_check > 2)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: invalid option value");
    if (o.stop == EECMG_STOP_DISCREPANCY && (!(o.c > 0.0) || !(o.delta >= 0.0)))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: discrepancy rule needs c > 0, delta >= 0");
    // compensated convolution where a level can run many iterations (the fixed schedule, or
    // no noise level): there FP32 rounding of the second pass grows with the count
    if (o.precise_conv < 0)
        o.precise_conv = (o.stop == EECMG_STOP_FIXED || !(o.delta > 0.0)) ? 1 : 0;
    if (o.storage == EECMG_STORAGE_BF16 && !o.persistent)
        return set_error(EECMG_ERR_UNSUPPORTED,
                         "eecmg_plan: BF16 storage needs the persistent level solve (persistent = 1)");
    double sum = 0.0;
    for (int i = 0; i < psf_w * psf_h; ++i) {
        if (!std::isfinite(psf[i])) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: PSF has non-finite entries");
        sum += psf[i];
    }
    if (!(sum > 0.0)) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: PSF sum must be positive");
    if (iters)
        for (int l = 0; l < levels; ++l)
            if (iters[l] < 0) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan: negative iteration count");

    Psf fine;
    fine.kh = psf_h;
    fine.kw = psf_w;
    fine.k.assign(psf, psf + (size_t)psf_w * psf_h);
    if (o.smoother == EECMG_SMOOTHER_MR2 && !centrosymmetric(fine))
        return set_error(EECMG_ERR_UNSUPPORTED,
                         "eecmg_plan: MR-II needs a symmetric H (centrosymmetric PSF); use CGLS");

    auto* P = new (std::nothrow) eecmg_plan_s();
    if (!P) return set_error(EECMG_ERR_OOM, "eecmg_plan: host allocation failed");
    P->W = width;
    P->H = height;
    P->L = levels;
    P->tau = alpha;
    P->kpm = k;
    P->opt = o;
    P->conv_tol2 = o.conv_tol * o.conv_tol;
    CK(cudaGetDevice(&P->device));
    P->lv.resize(levels);
    P->lv[levels - 1].h = height;
    P->lv[levels - 1].w = width;
    for (int l = levels - 1; l > 0; --l) {
        P->lv[l - 1].h = (P->lv[l].h + 1) / 2;
        P->lv[l - 1].w = (P->lv[l].w + 1) / 2;
    }
    std::vector<Psf> psfs(levels);
    psfs[levels - 1] = fine;
    for (int l = levels - 1; l > 0; --l) {
        const double rho = ((double)P->lv[l].h * P->lv[l].w) / ((double)P->lv[l - 1].h * P->lv[l - 1].w);
        psfs[l - 1] = coarsen(psfs[l], rho);
        if (o.coarse_op == EECMG_COARSE_GALERKIN_RENORM) {
            double s = 0.0;
            for (double v : psfs[l - 1].k) s += v;
            if (s != 0.0)
                for (double& v : psfs[l - 1].k) v *= sum / s;
        }
    }
    std::vector<Taps> htaps(2 * levels);
    size_t max_n = 0, sum_n = 0;
    for (int l = 0; l < levels; ++l) {
        LevelPlan& L = P->lv[l];
        L.m = iters ? iters[l] : schedule_m(levels, l + 1);
        make_taps(psfs[l], false, &htaps[2 * l]);
        make_taps(psfs[l], true, &htaps[2 * l + 1]);
        L.rt = htaps[2 * l].rt;
        L.sepH = htaps[2 * l].sep;
        L.sepHT = htaps[2 * l + 1].sep;
        const size_t n = (size_t)L.h * L.w;
        L.disc2 = o.stop == EECMG_STOP_DISCREPANCY ? (o.c * o.delta) * (o.c * o.delta) * (double)n : 0.0;
        max_n = n > max_n ? n : max_n;
        sum_n += n;
    }
    const size_t fine_n = (size_t)width * height;
    size_t max_blocks = 1;
    for (int l = 0; l < levels; ++l) {
        const size_t n = (size_t)P->lv[l].h * P->lv[l].w;
        size_t b = conv_blocks(P->lv[l].h, P->lv[l].w);
        if (ew_blocks(n) > b) b = ew_blocks(n);
        const size_t pb = (n + 4 * NTHREADS - 1) / (4 * NTHREADS);  // persistent grid bound
        if (pb > b) b = pb;
        if (b > max_blocks) max_blocks = b;
    }
    (void)fine_n;
    // workspace: g and u pyramids, solver vectors, taps, scalars, partials
    PlanLayout& Y = P->layout;
    size_t off = 0;
    Y.g_off.resize(levels);
    Y.u_off.resize(levels);
    for (int l = 0; l < levels; ++l) {
        Y.g_off[l] = off;
        off = align_up(off + sizeof(float) * P->lv[l].h * P->lv[l].w, 256);
    }
    for (int l = 0; l < levels; ++l) {
        Y.u_off[l] = off;
        off = align_up(off + sizeof(float) * P->lv[l].h * P->lv[l].w, 256);
    }
    for (int i = 0; i < eecmg_plan_s::NVEC; ++i) {
        Y.vec_off[i] = off;
        off = align_up(off + sizeof(float) * max_n, 256);
    }
    Y.taps_off = off;
    off = align_up(off + sizeof(Taps) * 2 * levels, 256);
    Y.sc_off = off;
    off = align_up(off + sizeof(Scalars) * levels, 256);
    Y.gs_off = off;
    off = align_up(off + sizeof(GroupSync) * levels, 256);
    Y.part_off = off;
    off = align_up(off + sizeof(double) * 2 * NPART * max_blocks, 256);  // double-buffered
    Y.bytes = off;
    P->ws_bytes = off;
    P->max_blocks = max_blocks;
    P->htaps = htaps;
    if (o.workspace) {
        eecmg_status st = plan_allocate(P, "eecmg_plan");
        if (st != EECMG_OK) {
            delete P;
            return st;
        }
    }
    *out = P;
    return EECMG_OK;
}

eecmg_status eecmg_plan_destroy(eecmg_plan_t P) {
    if (!P) return EECMG_OK;
    cudaDeviceSynchronize();
    forget_plan_batches(P);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    prof_flush(P);
    for (cudaEvent_t e : P->prof.free_events) cudaEventDestroy(e);
    if (P->owns_ws) {
        cudaFree(P->ws);
        g_live_owners.fetch_sub(1);
    }
    delete P;
    return EECMG_OK;
}

eecmg_status eecmg_plan_info(eecmg_plan_t P, int* levels, int* level_w, int* level_h, int* iters,
                             size_t* workspace_bytes) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan_info: NULL plan");
    if (levels) *levels = P->L;
    for (int l = 0; l < P->L; ++l) {
        if (level_w) level_w[l] = P->lv[l].w;
        if (level_h) level_h[l] = P->lv[l].h;
        if (iters) iters[l] = P->lv[l].m;
    }
    if (workspace_bytes) *workspace_bytes = P->ws_bytes;
    return EECMG_OK;
}

eecmg_status eecmg_level_partition(eecmg_plan_t P, int level, int* cluster, int* blocks, int* resident) {
    if (!P || level < 0 || level >= P->L)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_level_partition: NULL plan or level out of range");
    const LevelPlan& L = P->lv[level];
    const int cg = P->opt.smoother == EECMG_SMOOTHER_CGLS ? 1 : 0;
    const int bf = P->opt.storage == EECMG_STORAGE_BF16 ? 1 : 0;
    const LevelShape sh = level_shape(L.h, L.w, L.rt, cg, bf);
    int nb = sh.blocks;
    if (sh.cluster == 0) {
        const int cap = level_capacity(L.rt, L.sepH, P->opt.precise_conv, cg, bf);
        if (cap <= 0) return set_error(EECMG_ERR_CUDA, "eecmg_level_partition: occupancy query failed");
        nb = std::max(1, std::min(nb, cap));
    }
    if (cluster) *cluster = sh.cluster;
    if (blocks) *blocks = nb;
    if (resident) *resident = sh.resident;
    return EECMG_OK;
}

eecmg_status eecmg_restore(eecmg_plan_t P, const float* g, float* u, cudaStream_t s) {
    if (!P || !g || !u) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore: NULL argument");
    if (!P->ws) return no_ws("eecmg_restore");
    const size_t bytes = sizeof(float) * P->W * P->H;
    LevelPlan& F = P->lv[P->L - 1];
    if (g != F.g) CK(cudaMemcpyAsync(F.g, g, bytes, cudaMemcpyDeviceToDevice, s));
    eecmg_status st = run_cascade(P, s);
    if (st != EECMG_OK) return st;
    if (u != F.u) CK(cudaMemcpyAsync(u, F.u, bytes, cudaMemcpyDeviceToDevice, s));
    P->last_stream = s;
    return EECMG_OK;
}

eecmg_status eecmg_restore_host(eecmg_plan_t P, const float* g, float* u, cudaStream_t s) {
    if (!P || !g || !u) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_host: NULL argument");
    if (!P->ws) return no_ws("eecmg_restore_host");
    const size_t bytes = sizeof(float) * P->W * P->H;
    LevelPlan& F = P->lv[P->L - 1];
    CK(cudaMemcpyAsync(F.g, g, bytes, cudaMemcpyHostToDevice, s));
    eecmg_status st = run_cascade(P, s);
    if (st != EECMG_OK) return st;
    CK(cudaMemcpyAsync(u, F.u, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    P->last_stream = s;
    return EECMG_OK;
}

eecmg_status eecmg_plan_stats(eecmg_plan_t P, int* iters_done, double* res_rms) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan_stats: NULL plan");
    if (!P->ws) return no_ws("eecmg_plan_stats");
    CK(cudaStreamSynchronize(P->last_stream));
    CK(cudaStreamSynchronize(P->cap_stream));
    std::vector<Scalars> h(P->L);
    CK(cudaMemcpy(h.data(), P->sc, sizeof(Scalars) * P->L, cudaMemcpyDeviceToHost));
    bool numeric = false;
    for (int l = 0; l < P->L; ++l) {
        if (iters_done) iters_done[l] = h[l].iters;
        if (res_rms) res_rms[l] = std::sqrt(h[l].rr / ((double)P->lv[l].h * P->lv[l].w));
        if (h[l].stopped == 3) numeric = true;
    }
    if (numeric) return set_error(EECMG_ERR_NUMERIC, "eecmg_plan_stats: a level produced a non-finite scalar");
    return EECMG_OK;
}

static eecmg_status check_level(eecmg_plan_t P, int level, const char* who) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, std::string(who) + ": NULL plan");
    if (!P->ws) return no_ws(who);
    if (level < 0 || level >= P->L) return set_error(EECMG_ERR_INVALID_ARG, std::string(who) + ": level out of range");
    return EECMG_OK;
}

eecmg_status eecmg_apply_H(eecmg_plan_t P, int level, const float* x, float* y, int transpose,
                           cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_apply_H");
    if (st != EECMG_OK) return st;
    if (!x || !y || x == y) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_apply_H: NULL or aliased buffers");
    LevelPlan& L = P->lv[level];
    ConvArgs a;
    a.x = x;
    a.y = y;
    a.h = L.h;
    a.w = L.w;
    a.taps = P->dtaps + 2 * level + (transpose ? 1 : 0);
    a.mode = CM_STORE;
    CK(launch_conv(a, L.rt, transpose ? L.sepHT : L.sepH, P->opt.precise_conv, s));
    return EECMG_OK;
}

eecmg_status eecmg_restrict(eecmg_plan_t P, int level, const float* fine, float* coarse,
                            cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_restrict");
    if (st != EECMG_OK) return st;
    if (level + 1 >= P->L) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restrict: level must be < levels - 1");
    if (!fine || !coarse) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restrict: NULL buffer");
    LevelPlan& F = P->lv[level + 1];
    LevelPlan& C = P->lv[level];
    CK(launch_restrict(fine, F.h, F.w, coarse, C.h, C.w, s));
    return EECMG_OK;
}

eecmg_status eecmg_prolong(eecmg_plan_t P, int level, const float* u1, const float* u2, float* out,
                           cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_prolong");
    if (st != EECMG_OK) return st;
    if (level < 2) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_prolong: level must be >= 2");
    if (!u1 || !u2 || !out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_prolong: NULL buffer");
    LevelPlan& L = P->lv[level];
    LevelPlan& L1 = P->lv[level - 1];
    LevelPlan& L2 = P->lv[level - 2];
    CK(launch_prolong(u1, L1.h, L1.w, u2, L2.h, L2.w, out, L.h, L.w, s));
    return EECMG_OK;
}

eecmg_status eecmg_prolong_single(eecmg_plan_t P, int level, const float* u1, float* out,
                                  int quadratic, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_prolong_single");
    if (st != EECMG_OK) return st;
    if (level < 1) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_prolong_single: level must be >= 1");
    if (!u1 || !out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_prolong_single: NULL buffer");
    LevelPlan& L = P->lv[level];
    LevelPlan& L1 = P->lv[level - 1];
    if (quadratic)
        CK(launch_quadratic(u1, L1.h, L1.w, out, L.h, L.w, s));
    else
        CK(launch_linear(u1, L1.h, L1.w, out, L.h, L.w, s));
    return EECMG_OK;
}

eecmg_status eecmg_start_level(eecmg_plan_t P, int level, const float* u1, const float* u2, float* out,
                               cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_start_level");
    if (st != EECMG_OK) return st;
    if (level < 2) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_start_level: level must be >= 2");
    if (!u1 || !u2 || !out || out == u1 || out == u2)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_start_level: NULL or aliased buffers");
    if (P->opt.diffusion_steps != 1)
        return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_start_level: needs diffusion_steps = 1");
    LevelPlan& L = P->lv[level];
    LevelPlan& L1 = P->lv[level - 1];
    LevelPlan& L2 = P->lv[level - 2];
    CK(launch_psd(u1, L1.h, L1.w, u2, L2.h, L2.w, out, L.h, L.w, (float)P->opt.s_scale, (float)P->tau,
                  (float)P->kpm, s));
    return EECMG_OK;
}

eecmg_status eecmg_smooth(eecmg_plan_t P, int level, const float* in, float* out, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_smooth");
    if (st != EECMG_OK) return st;
    if (!in || !out || in == out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_smooth: NULL or aliased buffers");
    CK(launch_smooth(in, out, P->lv[level].h, P->lv[level].w, (float)P->opt.s_scale, s));
    return EECMG_OK;
}

eecmg_status eecmg_denoise(eecmg_plan_t P, int level, const float* in, float* out, cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_denoise");
    if (st != EECMG_OK) return st;
    if (!in || !out || in == out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_denoise: NULL or aliased buffers");
    CK(launch_denoise(in, out, P->lv[level].h, P->lv[level].w, (float)P->tau, (float)P->kpm, s));
    return EECMG_OK;
}

eecmg_status eecmg_level_solve(eecmg_plan_t P, int level, const float* g, float* u, int m,
                               cudaStream_t s) {
    eecmg_status st = check_level(P, level, "eecmg_level_solve");
    if (st != EECMG_OK) return st;
    if (!g || !u || m < 0) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_level_solve: bad arguments");
    st = solve_level_enqueue(P, level, g, u, m, false, s);
    P->last_stream = s;
    return st;
}

eecmg_status eecmg_plan_profile(eecmg_plan_t P, int enable) {
    if (!P) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan_profile: NULL plan");
    if (!P->ws) return no_ws("eecmg_plan_profile");
    CK(prof_flush(P));
    P->prof.on = enable != 0;
    for (int c = 0; c < KC_COUNT; ++c) {
        P->prof.ms[c] = 0.0;
        P->prof.bytes[c] = 0.0;
        P->prof.launches[c] = 0;
    }
    return EECMG_OK;
}

eecmg_status eecmg_plan_profile_read(eecmg_plan_t P, eecmg_kernel_stat* out, int max, int* n) {
    static const char* names[KC_COUNT] = {"conv", "mr_b", "mr_final", "cg_step", "cg_p",
                                          "restrict", "prolong", "smooth", "denoise", "copy",
                                          "level_solve"};
    if (!P || !n) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_plan_profile_read: NULL argument");
    CK(prof_flush(P));
    int k = 0;
    for (int c = 0; c < KC_COUNT; ++c) {
        if (out && k < max) {
            std::snprintf(out[k].name, sizeof(out[k].name), "%s", names[c]);
            out[k].launches = P->prof.launches[c];
            out[k].ms = P->prof.ms[c];
            out[k].bytes = P->prof.bytes[c];
        }
        ++k;
    }
    *n = k;
    return EECMG_OK;
}

static eecmg_status restore_batched_host_impl(const eecmg_plan_t* plans, const float* const* g,
                                              float* const* u, int n, cudaStream_t s, bool sync) {
    if (n < 0 || (n > 0 && (!plans || !g || !u)))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched_host: bad arguments");
    if (n == 0) return EECMG_OK;
    std::vector<const float*> gd(n);
    std::vector<float*> ud(n);
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !g[i] || !u[i])
            return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched_host: NULL plan or buffer");
        if (!plans[i]->ws) return no_ws("eecmg_restore_batched_host");
        if (plans[i]->prof.on)
            return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched_host: disable profiling first");
        LevelPlan& F = plans[i]->lv[plans[i]->L - 1];
        CK(cudaMemcpyAsync(F.g, g[i], sizeof(float) * plans[i]->W * plans[i]->H, cudaMemcpyHostToDevice, s));
        gd[i] = F.g;  // already in place: the batched call copies nothing more
        ud[i] = F.u;
    }
    eecmg_status st = restore_batched_impl(plans, gd.data(), ud.data(), n, s);
    if (st != EECMG_OK) return st;
    for (int i = 0; i < n; ++i) {
        LevelPlan& F = plans[i]->lv[plans[i]->L - 1];
        CK(cudaMemcpyAsync(u[i], F.u, sizeof(float) * plans[i]->W * plans[i]->H, cudaMemcpyDeviceToHost, s));
    }
    if (sync) CK(cudaStreamSynchronize(s));
    return EECMG_OK;
}

eecmg_status eecmg_restore_batched_host(const eecmg_plan_t* plans, const float* const* g,
                                        float* const* u, int n, cudaStream_t s) {
    return restore_batched_host_impl(plans, g, u, n, s, true);
}

eecmg_status eecmg_restore_batched_host_async(const eecmg_plan_t* plans, const float* const* g,
                                              float* const* u, int n, cudaStream_t s) {
    return restore_batched_host_impl(plans, g, u, n, s, false);
}

eecmg_status eecmg_batch_info(const eecmg_plan_t* plans, int n, int* graph_nodes) {
    if (!plans || n < 1 || !graph_nodes) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_batch_info: bad arguments");
    return batch_graph_nodes(plans, n, graph_nodes);
}

eecmg_status eecmg_batch_time_step(const eecmg_plan_t* plans, int n, int step, int enable) {
    if (!plans || n < 1) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_batch_time_step: bad arguments");
    return batch_time_step(plans, n, step, enable);
}

eecmg_status eecmg_batch_step_time(const eecmg_plan_t* plans, int n, float* ms, int* launches,
                                   double* bytes) {
    if (!plans || n < 1) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_batch_step_time: bad arguments");
    return batch_step_time(plans, n, ms, launches, bytes);
}

eecmg_status eecmg_restore_batched(const eecmg_plan_t* plans, const float* const* g, float* const* u,
                                   int n, cudaStream_t s) {
    if (n < 0 || (n > 0 && (!plans || !g || !u)))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched: bad arguments");
    if (n == 0) return EECMG_OK;
    for (int i = 0; i < n; ++i)
        if (plans[i] && !plans[i]->ws) return no_ws("eecmg_restore_batched");
    for (int i = 0; i < n; ++i)
        if (plans[i] && plans[i]->prof.on)
            return set_error(EECMG_ERR_INVALID_ARG,
                             "eecmg_restore_batched: disable profiling on the plans first");
    return restore_batched_impl(plans, g, u, n, s);
}

}  // extern "C"
