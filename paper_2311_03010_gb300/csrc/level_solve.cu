// level_solve.cu -- dispatch of the persistent level solve (kernels in
// level_solve_impl.cuh, instantiated in the ls_*.cu translation units).
#include <atomic>
#include <cstdlib>

#include "level_solve_impl.cuh"

namespace eecmg {

namespace {

cudaError_t dispatch(const LevelLaunch& L, int rt, int sep, int prec, int cgls, int bf16, int op,
                     int blocks, cudaStream_t s, int* out) {
    if (rt < 0 || rt > RMAX) return cudaErrorInvalidValue;
    const bool lo = rt < 6;
    if (cgls) {
        if (bf16)
            return lo ? launch_level_cgls_bf16_lo(L, rt, sep, prec, op, blocks, s, out)
                      : launch_level_cgls_bf16_hi(L, rt, sep, prec, op, blocks, s, out);
        return lo ? launch_level_cgls_f32_lo(L, rt, sep, prec, op, blocks, s, out)
                  : launch_level_cgls_f32_hi(L, rt, sep, prec, op, blocks, s, out);
    }
    if (bf16)
        return lo ? launch_level_mr2_bf16_lo(L, rt, sep, prec, op, blocks, s, out)
                  : launch_level_mr2_bf16_hi(L, rt, sep, prec, op, blocks, s, out);
    return lo ? launch_level_mr2_f32_lo(L, rt, sep, prec, op, blocks, s, out)
              : launch_level_mr2_f32_hi(L, rt, sep, prec, op, blocks, s, out);
}

// Largest cluster every instantiation can run as (queried on the kernels
// with the most shared memory: the largest radius, non-separable).
int cluster_limit() {
    static int lim = -1;
    if (lim < 0) {
        LevelLaunch L;
        int m = CLUSTER_MAX;
        for (int cgls = 0; cgls < 2; ++cgls)
            for (int bf16 = 0; bf16 < 2; ++bf16) {
                int c = 0;
                if (dispatch(L, RMAX, 0, 0, cgls, bf16, LS_CLUSTER_MAX, 0, nullptr, &c) != cudaSuccess) c = 0;
                m = c < m ? c : m;
            }
        lim = m;
    }
    return lim;
}

// Largest cluster of the resident solver with T tiles per block on every
// instantiation (queried on the ones with the most static shared memory).
int resident_cluster_limit(int T) {
    static int lim[RES_TMAX + 1] = {-1, -1, -1};
    if (T < 1 || T > RES_TMAX) return 0;
    if (lim[T] < 0) {
        LevelLaunch L;
        L.resident = T;
        int m = CLUSTER_MAX;
        for (int cgls = 0; cgls < 2; ++cgls)
            for (int sep = 0; sep < 2; ++sep) {
                int c = 0;
                if (dispatch(L, RES_RMAX, sep, 1, cgls, 0, LS_RESIDENT_MAX, 0, nullptr, &c) != cudaSuccess)
                    c = 0;
                m = c < m ? c : m;
            }
        lim[T] = m;
    }
    return lim[T];
}

}  // namespace

// ---------------------------------------------------------------------------
// Partition parameters (eecmg_tuning).  Process-wide; the C ABI changes them
// only while no plan with a workspace and no server exists, so every solve
// of a process is partitioned the same way alone, batched or served.
// Initial values: the GB300 optimum measured by sweeps, overridable through
// EECMG_PX_PER_BLOCK, EECMG_CLUSTER_MAX_PX and EECMG_BLOCKS_PER_SM.
// ---------------------------------------------------------------------------

namespace {

std::atomic<int> g_px_per_block{0}, g_blocks_per_sm{0}, g_resident_max_tiles{0}, g_psd_tile_h{32};
std::atomic<long long> g_cluster_max_px{-1};

void tuning_init() {
    if (g_px_per_block.load() > 0) return;
    const char* a = std::getenv("EECMG_PX_PER_BLOCK");
    const char* b = std::getenv("EECMG_CLUSTER_MAX_PX");
    const char* c = std::getenv("EECMG_BLOCKS_PER_SM");
    const char* d = std::getenv("EECMG_RESIDENT_MAX_TILES");
    const char* e = std::getenv("EECMG_PSD_TILE_H");
    Tuning t;
    if (a) t.px_per_block = std::atoi(a);
    if (b) t.cluster_max_px = std::atoll(b);
    if (c) t.blocks_per_sm = std::atoi(c);
    if (d) t.resident_max_tiles = std::atoi(d);
    if (e) t.psd_tile_h = std::atoi(e);
    set_tuning_raw(t);
}

}  // namespace

bool tuning_valid(const Tuning& t) {
    return t.px_per_block >= 1024 && t.px_per_block <= (1 << 22) && t.cluster_max_px >= 0 &&
           t.blocks_per_sm >= 1 && t.blocks_per_sm <= 3 && t.resident_max_tiles >= 0 &&
           t.resident_max_tiles <= CLUSTER_MAX * RES_TMAX && (t.psd_tile_h == 16 || t.psd_tile_h == 32);
}

void set_tuning_raw(const Tuning& t0) {
    Tuning t = t0;
    // the plan sizes its reduction partials for at least 1024 pixels per block
    if (t.px_per_block < 1024) t.px_per_block = 1024;
    if (t.cluster_max_px < 0) t.cluster_max_px = 0;
    t.blocks_per_sm = t.blocks_per_sm < 1 ? 1 : (t.blocks_per_sm > 3 ? 3 : t.blocks_per_sm);
    const int rmt = CLUSTER_MAX * RES_TMAX;
    t.resident_max_tiles = t.resident_max_tiles < 0 ? 0 : (t.resident_max_tiles > rmt ? rmt : t.resident_max_tiles);
    g_resident_max_tiles.store(t.resident_max_tiles);
    g_psd_tile_h.store(t.psd_tile_h == 16 ? 16 : 32);
    g_cluster_max_px.store(t.cluster_max_px);
    g_blocks_per_sm.store(t.blocks_per_sm);
    g_px_per_block.store(t.px_per_block);
}

Tuning get_tuning() {
    tuning_init();
    Tuning t;
    t.px_per_block = g_px_per_block.load();
    t.cluster_max_px = g_cluster_max_px.load();
    t.blocks_per_sm = g_blocks_per_sm.load();
    t.resident_max_tiles = g_resident_max_tiles.load();
    t.psd_tile_h = g_psd_tile_h.load();
    return t;
}

int psd_tile_rows() { return get_tuning().psd_tile_h; }

// Blocks of a grid-mode level solve: the larger of the 32 x 64 tile count and
// pixels / px_per_block, at most blocks_per_sm per SM (the MR-II solvers fit
// two per SM, CGLS three; a solve never exceeds its instantiation's
// capacity).  Measured on GB300: one block per tile (px_per_block 2048) beats
// one per 1024 pixels by 10-25 % on the 512^2 and batched cascades (cheaper
// barriers, no idle blocks in the convolution phases).
int level_want_blocks(int h, int w) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const Tuning t = get_tuning();
    const int cap = t.blocks_per_sm * sms;
    const size_t n = (size_t)h * w;
    const int tiles = (int)conv_blocks(h, w);
    const int elem = (int)((n + (size_t)t.px_per_block - 1) / (size_t)t.px_per_block);
    const int want = tiles > elem ? tiles : elem;
    return want < cap ? want : cap;
}

// Levels of at most cluster_max_px pixels run in cluster mode (0: never).
// Measured on GB300: 128^2 and below gain from the in-GPC exchange; from
// 256^2 up a 16-SM cluster is throughput-bound and the grid form is faster.
LevelShape level_shape(int h, int w, int rt, int cgls, int bf16) {
    LevelShape sh;
    // FP32 storage: levels of at most resident_max_tiles tiles (<= 32) keep their
    // vectors in the shared memory of one cluster, T = 1 or 2 tiles per block
    (void)cgls;
    const int tiles = (int)conv_blocks(h, w);
    if (!bf16 && rt >= 0 && rt <= RES_RMAX && tiles <= get_tuning().resident_max_tiles) {
        const int T = (tiles + CLUSTER_MAX - 1) / CLUSTER_MAX;
        const int C = (tiles + T - 1) / T;
        if (T <= RES_TMAX && C <= resident_cluster_limit(T)) {
            sh.cluster = C;
            sh.blocks = C;
            sh.resident = T;
            return sh;
        }
    }
    const int want = level_want_blocks(h, w);
    const size_t n = (size_t)h * w;
    const int lim = n <= (size_t)get_tuning().cluster_max_px ? cluster_limit() : 0;
    if (lim >= 1) {
        sh.cluster = want < lim ? want : lim;
        sh.blocks = sh.cluster;
    } else {
        sh.blocks = want;
    }
    return sh;
}

cudaError_t launch_level_solve(const LevelJob& J, int rt, int sep, int prec, int cgls, int bf16,
                               cudaStream_t s, int* blocks_used) {
    if (J.h <= 0 || J.w <= 0) return cudaSuccess;
    LevelLaunch L;
    L.job = J;
    const LevelShape sh = level_shape(J.h, J.w, rt, cgls, bf16);
    if (sh.cluster > 0) {
        L.cluster = sh.cluster;
        L.resident = sh.resident;
        if (blocks_used) *blocks_used = sh.blocks;
        return dispatch(L, rt, sep, prec, cgls, bf16, sh.resident > 0 ? LS_RESIDENT : LS_CLUSTER,
                        sh.blocks, s, nullptr);
    }
    int cap = 0;
    cudaError_t e = dispatch(L, rt, sep, prec, cgls, bf16, LS_CAPACITY, 0, nullptr, &cap);
    if (e != cudaSuccess) return e;
    int blocks = sh.blocks < cap ? sh.blocks : cap;
    if (blocks < 1) blocks = 1;
    if (blocks_used) *blocks_used = blocks;
    return dispatch(L, rt, sep, prec, cgls, bf16, LS_COOP, blocks, s, nullptr);
}

cudaError_t launch_level_batch(const LevelJob* d_jobs, const unsigned short* d_block_job, int njobs,
                               int total_blocks, int rt, int sep, int prec, int cgls, int bf16,
                               int cluster, int resident, cudaStream_t s) {
    if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
    LevelLaunch L;
    L.jobs = d_jobs;
    L.block_job = d_block_job;
    L.njobs = njobs;
    L.cluster = cluster;
    L.resident = resident;
    const int op = resident > 0 ? LS_RESIDENT : (cluster > 0 ? LS_CLUSTER : LS_COOP);
    return dispatch(L, rt, sep, prec, cgls, bf16, op, total_blocks, s, nullptr);
}

int level_capacity(int rt, int sep, int prec, int cgls, int bf16) {
    LevelLaunch L;
    int cap = 0;
    if (dispatch(L, rt, sep, prec, cgls, bf16, LS_CAPACITY, 0, nullptr, &cap) != cudaSuccess) return 0;
    return cap;
}

}  // namespace eecmg

