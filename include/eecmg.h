/*
 * eecmg.h -- C ABI of the GB300 (sm_103a) implementation of the
 * Extrapolation Economy Cascadic Multigrid method (EECMG) for image
 * restoration (Chu, Yan & Li, "A New Extrapolation Economy Cascadic
 * Multigrid Method for Image Restoration Problems").
 *
 * The method restores u from H u = g_delta (Eqs. 3 and 9), H the
 * zero-boundary (block-Toeplitz) convolution with a point-spread function
 * (PSF).  It runs a coarse-to-fine cascade (Algorithm 2): the two coarsest
 * levels are solved from zero with a few Krylov iterations; every finer
 * level starts from the new extrapolation of the two previous solutions
 * (Section 3.2), quadratic interpolation, local smoothing (Section 3.3) and
 * one Perona-Malik denoising step (Section 4), then runs its economy number
 * of Krylov iterations (Section 2).
 *
 * Conventions for every entry point:
 *   - Images are single-channel FP32, row-major, pitch = width, values on
 *     the [0, 255] grey scale.  "device" pointers are CUDA global memory of
 *     the current device; "host" pointers are CPU memory.  The library never
 *     takes ownership of caller buffers; asynchronous calls require the
 *     caller to keep them alive until the stream reaches the call.
 *   - PSFs are host FP64, row-major, odd sizes, centred; they are copied.
 *   - Levels are numbered 0 (coarsest) .. levels-1 (finest, the input size).
 *   - Every function returns an eecmg_status; on failure a description is
 *     available from eecmg_last_error() (thread-local).  No function throws
 *     or aborts.  Invalid arguments are detected on the host before any work
 *     is enqueued.
 *   - A plan owns device memory (its workspace) and is not safe to use from
 *     two streams at once; use one plan per concurrent restoration.
 */
#ifndef EECMG_H
#define EECMG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EECMG_OK = 0,
    EECMG_ERR_INVALID_ARG = 1,  /* bad size, pointer, option or PSF            */
    EECMG_ERR_UNSUPPORTED = 2,  /* e.g. MR-II with a non-centrosymmetric PSF   */
    EECMG_ERR_OOM = 3,          /* device allocation or memory budget failed   */
    EECMG_ERR_CUDA = 4,         /* a CUDA runtime call failed                  */
    EECMG_ERR_NUMERIC = 5,      /* non-finite scalar in a level solve          */
    EECMG_ERR_TIMEOUT = 6,      /* a bounded device wait gave up               */
    EECMG_ERR_BUSY = 7          /* server queue full / resource in use         */
} eecmg_status;

enum { EECMG_SMOOTHER_MR2 = 0, EECMG_SMOOTHER_CGLS = 1 };
enum { EECMG_COARSE_GALERKIN_RMS = 0, EECMG_COARSE_GALERKIN_RENORM = 1 };
enum { EECMG_STORAGE_FP32 = 0, EECMG_STORAGE_BF16 = 1 };
enum { EECMG_STOP_FIXED = 0, EECMG_STOP_DISCREPANCY = 1 };
enum { EECMG_PROLONG_EECMG = 0, EECMG_PROLONG_IECMG_P = 1, EECMG_PROLONG_IECMG_L = 2 };

/* Largest PSF radius supported (PSF up to 25 x 25). */
#define EECMG_MAX_RADIUS 12

/*
 * Options.  eecmg_default_options() fills:
 *   smoother = MR2        "MR" of Section 2 read as MR-II (needs a
 *                         centrosymmetric PSF); CGLS is the reading of "CG".
 *   coarse_op = GALERKIN_RMS  H_l = R_l H_{l+1} R_l^* (Eq. 14) with R_l^* the
 *                         adjoint under the RMS inner product of Eq. 10;
 *                         GALERKIN_RENORM rescales each coarse PSF to the
 *                         fine PSF's sum.
 *   storage = FP32        BF16 stores the Krylov search directions (MR-II: the
 *                         d history; CGLS: s and p) as bf16, rounded to
 *                         nearest even.  Lanczos vectors, H d, q = H p, u and
 *                         r stay FP32, arithmetic is FP32 and scalars FP64,
 *                         so residuals and stopping decisions follow the
 *                         stored directions exactly.  Needs persistent = 1
 *                         (else EECMG_ERR_UNSUPPORTED).
 *   stop = DISCREPANCY    the stopping rule of Section 2 (after Eq. 10): a
 *                         level stops before an iteration once
 *                         ||g_l - H_l u||_RMS <= c * delta, and after at
 *                         most m_l iterations (the economy schedule is the
 *                         cap).  FIXED runs exactly m_l iterations (the note
 *                         of Algorithm 2), which on noisy data iterates far
 *                         past the noise level and amplifies it.
 *   c = 1.1, delta = 0    discrepancy constant c > 1 and the noise level
 *                         delta = ||e||_RMS of the data (the same on every
 *                         level: the RMS norm does not depend on the grid
 *                         size).  delta = 0 (noise-free data) leaves only
 *                         the cap, i.e. the FIXED schedule: pass the data's
 *                         noise level to get the rule.
 *   diffusion_steps = 1   explicit Perona-Malik steps per prolonged level.
 *   s_scale = 1           scale of the weight argument of Eq. 18.
 *   conv_tol = 1e-5       a level also stops once ||r|| <= conv_tol ||g_l||
 *                         (the exact method takes no step after a zero
 *                         residual; see the design notes); 0 disables.
 *   prolong = EECMG       Algorithm 2; IECMG_P / IECMG_L run Algorithm 1
 *                         with quadratic / linear (Eq. 15) prolongation.
 *   use_graph = 1         capture the cascade as a CUDA graph per plan.
 *   precise_conv = -1     1: compensated (error-free product + Kahan) FP32
 *                         accumulation in the second pass of separable
 *                         convolutions; 0: plain FMA accumulation; -1
 *                         (auto): 1 where a level can run many iterations
 *                         (stop = FIXED, or delta = 0), else 0.  Under the
 *                         discrepancy rule a level stops within a few
 *                         iterations and the plain pass stays within the
 *                         FP32 bar of the FP64 result; over a long fixed
 *                         schedule its rounding grows with the count.
 *   persistent = 1        one cooperative launch per level solve (grid
 *                         barriers inside); 0 = one launch per phase.
 *   workspace = 1         allocate the plan's device workspace; 0 = the plan
 *                         is a description only (no device memory), usable
 *                         with eecmg_server_submit and eecmg_plan_info; every
 *                         entry point that runs kernels on it returns
 *                         EECMG_ERR_INVALID_ARG.
 *   fuse_start = 0        1: every prolonged level's persistent solve runs
 *                         the level's start D(S(P(Pi))) itself as its first
 *                         phase, so a restoration is one launch per cascade
 *                         step (Algorithm 2 with diffusion_steps = 1; the
 *                         same arithmetic, bitwise the same result).  0: the
 *                         start is its own launch at full occupancy, which
 *                         is faster on GB300 (the start is compute-bound and
 *                         a solve runs two blocks per SM).  The two coarsest
 *                         levels write their zero start inside their solve
 *                         either way.
 *   early_check = 1       MR-II's early stop check under the discrepancy
 *                         rule (Section 2): when the rotation predicts
 *                         ||r_k|| within 1/64 of the limit, the solve updates
 *                         u with step k and tests the explicit ||r_k|| before
 *                         spending iteration k + 1's convolution; if the test
 *                         fails, the next iteration completes the step.  The
 *                         iterate and every decision are the same as without
 *                         the check.  0: no early check; 2: a check before
 *                         every step (the same result; for tests).
 */
typedef struct {
    int smoother;
    int coarse_op;
    int storage;
    int stop;
    double c;
    double delta;
    int diffusion_steps;
    double s_scale;
    double conv_tol;
    int prolong;
    int use_graph;
    int precise_conv;
    int persistent;
    int workspace;
    int fuse_start;
    int early_check;
} eecmg_options;

typedef struct eecmg_plan_s *eecmg_plan_t;

/* Fills *opt with the defaults listed above.  Errors: INVALID_ARG if NULL. */
eecmg_status eecmg_default_options(eecmg_options *opt);

/*
 * Creates a restoration plan for width x height images (Section 2, Eqs.
 * 11-14; Section 5 for the PSF and the paper's parameters).
 *   levels   number of grid levels L >= 1 (the two coarsest are solved from
 *            zero; L = 1 is the standalone smoother); each coarser side is
 *            ceil(side / 2) (Section 2).
 *   psf      host FP64 PSF, psf_h rows x psf_w cols, odd sizes, radius
 *            <= EECMG_MAX_RADIUS, positive sum; copied.
 *   alpha    step tau of the explicit Perona-Malik step (Eq. 24),
 *            0 <= alpha <= 0.25 (the API's alpha is read as tau).
 *   k        Perona-Malik threshold of Eq. 21, k > 0.
 *   iters    host array of `levels` iteration counts m_l (coarsest first),
 *            or NULL for the economy schedule of Section 2.
 *   opt      options, or NULL for the defaults.
 *   out      receives the plan.  The plan allocates its device workspace
 *            (see eecmg_plan_info) on the current device.
 * Errors: INVALID_ARG (sizes, PSF, alpha, k, iters < 0), UNSUPPORTED (MR-II
 * with a PSF that is not centrosymmetric), OOM, CUDA.
 */
eecmg_status eecmg_plan(int width, int height, int levels, const double *psf, int psf_w,
                        int psf_h, double alpha, double k, const int *iters,
                        const eecmg_options *opt, eecmg_plan_t *out);

/* Releases the plan and its device memory (synchronises the device first). */
eecmg_status eecmg_plan_destroy(eecmg_plan_t plan);

/*
 * Plan geometry: level_w/level_h/iters (each `levels` entries, may be NULL)
 * receive the level sizes and scheduled m_l, coarsest first;
 * workspace_bytes (may be NULL) the device memory the plan holds.
 */
eecmg_status eecmg_plan_info(eecmg_plan_t plan, int *levels, int *level_w, int *level_h,
                             int *iters, size_t *workspace_bytes);

/*
 * How the persistent solve of level `level` (0 = coarsest) is partitioned
 * (system design, no counterpart in the paper; see eecmg_tuning): *cluster
 * receives the blocks per thread-block cluster (0: one cooperative grid),
 * *blocks the blocks of the solve, *resident the 32x64 tiles each block
 * keeps in shared memory (0: the vectors stream through L2).  Follows the
 * current eecmg_tuning; NULL outputs are skipped.  INVALID_ARG for a NULL
 * plan or a level outside 0 .. levels-1; CUDA if the device query fails.
 */
eecmg_status eecmg_level_partition(eecmg_plan_t plan, int level, int *cluster, int *blocks,
                                   int *resident);

/*
 * Restores one image (Algorithm 2, Step 1 - Step 3).  g_delta and u_out are
 * device buffers of height x width floats; they may alias.  Asynchronous on
 * `stream` (0 = legacy default stream).  Errors: INVALID_ARG (NULL
 * pointers), CUDA.  Numeric breakdowns are not errors: a level whose Krylov
 * denominator vanishes ends early (see eecmg_plan_stats).
 */
eecmg_status eecmg_restore(eecmg_plan_t plan, const float *g_delta, float *u_out,
                           cudaStream_t stream);

/*
 * As eecmg_restore, with HOST buffers: copies g_host to the device, restores
 * and copies the result to u_host, then synchronises `stream`.  For callers
 * that keep their images in CPU memory.
 */
eecmg_status eecmg_restore_host(eecmg_plan_t plan, const float *g_host, float *u_host,
                                cudaStream_t stream);

/*
 * eecmg_restore_batched with HOST buffers: copies every g_host[i] into its
 * plan's workspace, runs the batched restoration, copies every result to
 * u_host[i] and synchronises `stream` once.  Pinned host memory makes the
 * copies asynchronous.  Errors as eecmg_restore_batched.
 */
eecmg_status eecmg_restore_batched_host(const eecmg_plan_t *plans, const float *const *g_host,
                                        float *const *u_host, int n, cudaStream_t stream);

/*
 * eecmg_restore_batched_host without the final synchronisation: the copies
 * in, the batched restoration and the copies out are queued on `stream` and
 * the call returns.  The host buffers must stay valid (and the plans unused
 * elsewhere) until the stream has passed this point; with pinned host memory
 * the copies run asynchronously, so a caller that alternates two sets of
 * plans on two streams overlaps one batch's copies with the other's
 * restoration.  Errors as eecmg_restore_batched.
 */
eecmg_status eecmg_restore_batched_host_async(const eecmg_plan_t *plans, const float *const *g_host,
                                              float *const *u_host, int n, cudaStream_t stream);

/*
 * Restores n images with their own plans (sizes, PSFs, levels and options
 * may differ) as one batch: per cascade step (levels counted from the
 * coarsest), one persistent cooperative launch per kind of level solver
 * covers every image, each image's solve owning its own block range.
 * plans[i], g[i] (device), u[i] (device); the plans must be distinct, use
 * the persistent level solve and not be profiling.  The first call with a
 * given set of plans builds device job tables and a CUDA graph for it (an
 * allocation; make it before any stream capture); later calls replay it.
 * Destroying any of the plans drops the cached batch.  Image i's finest
 * level is solved in g[i] and u[i] themselves (g is only read) when u[i]
 * overlaps no g[j] and no other u[j]; otherwise g[i] is copied into the
 * plan's workspace first and the result copied out after the batch, so
 * u[i] may alias g[i] or another image's input.  When the buffers differ
 * from the previous call's, the job tables are rebound (a small upload on
 * `stream` ahead of the batch).  Asynchronous on `stream`.  Errors:
 * INVALID_ARG, OOM, CUDA.
 */
eecmg_status eecmg_restore_batched(const eecmg_plan_t *plans, const float *const *g,
                                   float *const *u, int n, cudaStream_t stream);

/*
 * Kernel nodes of the CUDA graph that eecmg_restore_batched replays for
 * exactly these plans in this order (after its first call; INVALID_ARG
 * before): the library's kernel launches per batched restoration.
 */
eecmg_status eecmg_batch_info(const eecmg_plan_t *plans, int n, int *graph_nodes);

/*
 * Measurement hook (system design, no counterpart in the paper).  With
 * enable = 1, the CUDA graph that eecmg_restore_batched replays for exactly
 * these plans in this order also records a pair of CUDA events, as
 * event-record nodes on the launch stream, immediately before the first and
 * after the last level-solve launch of cascade step `step` (0 = every
 * image's coarsest level).  enable = 0 removes them.  A change synchronises
 * the device and drops the cached graph, which is captured again at the next
 * eecmg_restore_batched (do not call it during a stream capture).  Errors:
 * INVALID_ARG if these plans were never restored as a batch or step is out
 * of range; CUDA.
 */
eecmg_status eecmg_batch_time_step(const eecmg_plan_t *plans, int n, int step, int enable);

/*
 * Reads the hook of the most recent replay: waits for its second event, then
 * *ms receives the elapsed time between the two events, *launches the
 * level-solve launches between them and *bytes their algorithmic bytes (each
 * solver vector read or written once per phase, FP32 or BF16 as stored,
 * counted from the iterations each solve actually ran).  NULL outputs are
 * skipped.  INVALID_ARG without an enabled hook and a replay.
 */
eecmg_status eecmg_batch_step_time(const eecmg_plan_t *plans, int n, float *ms, int *launches,
                                   double *bytes);

/*
 * Per-level outcome of the most recent restoration with this plan:
 * iters_done[l] (iterations actually taken) and res_rms[l] (||g_l - H_l
 * u_l||_RMS as carried by the recurrence, Eq. 10).  Synchronises the plan's
 * last stream.  Either pointer may be NULL.
 */
eecmg_status eecmg_plan_stats(eecmg_plan_t plan, int *iters_done, double *res_rms);

/*
 * Per-launch profiling (for measurement, not the paper): with enable = 1 the
 * plan's restorations run eagerly (no graph) with a CUDA event pair around
 * every kernel launch on the caller's stream; eecmg_plan_profile_read
 * synchronises and returns, per kernel class, the launches, the summed
 * event time (ms) and the summed algorithmic bytes (the reads and writes
 * each operator needs, counted once).  Enabling or disabling resets the
 * totals.  *n receives the number of classes; at most max are written.
 */
typedef struct {
    char name[24];
    long long launches;
    double ms;
    double bytes;
} eecmg_kernel_stat;
eecmg_status eecmg_plan_profile(eecmg_plan_t plan, int enable);
eecmg_status eecmg_plan_profile_read(eecmg_plan_t plan, eecmg_kernel_stat *out, int max, int *n);

/* ---- operator-level entry points (one level of a plan) ----------------- */

/*
 * y = H_l x (transpose = 0) or y = H_l^T x (transpose = 1): zero-boundary
 * convolution with the level's PSF (Eqs. 1, 7; Eq. 14 for l < L-1).  x, y
 * device, level_h x level_w floats, must not alias.  Asynchronous.
 */
eecmg_status eecmg_apply_H(eecmg_plan_t plan, int level, const float *x, float *y, int transpose,
                           cudaStream_t stream);

/*
 * Restriction of Eqs. 12-13: coarse(a, b) = fine(2a, 2b) from level+1 to
 * level.  fine: level+1 sizes, coarse: level sizes, device.  Asynchronous.
 */
eecmg_status eecmg_restrict(eecmg_plan_t plan, int level, const float *fine, float *coarse,
                            cudaStream_t stream);

/*
 * Nonlinear prolongation of Section 3.2 to `level` (>= 2): the new
 * extrapolation Pi from u1 (level-1 solution) and u2 (level-2 solution),
 * then quadratic interpolation P onto `level`.  out: level sizes.  Device,
 * asynchronous.
 */
eecmg_status eecmg_prolong(eecmg_plan_t plan, int level, const float *u1, const float *u2,
                           float *out, cudaStream_t stream);

/*
 * Prolongation of Algorithm 1 to `level` (>= 1) from the level-1 solution
 * u1 only: quadratic = 1 for P (IECMG-P), 0 for the linear L of Eq. 15
 * (IECMG-L).  Device, asynchronous.
 */
eecmg_status eecmg_prolong_single(eecmg_plan_t plan, int level, const float *u1, float *out,
                                  int quadratic, cudaStream_t stream);

/*
 * The start of a prolonged level in Algorithm 2 (Step 2): out = D_l(S_l(P_l(
 * Pi_l(u1, u2)))), the new extrapolation and quadratic interpolation of
 * Section 3.2, the local smoothing of Section 3.3 and one Perona-Malik step of
 * Section 4, as one pass (bitwise equal to eecmg_prolong, eecmg_smooth and
 * eecmg_denoise in sequence).  level >= 2; u1, u2: device solutions of
 * levels level-1 and level-2; out: device, level sizes, aliasing neither.
 * UNSUPPORTED unless the plan has diffusion_steps = 1.  Asynchronous.
 */
eecmg_status eecmg_start_level(eecmg_plan_t plan, int level, const float *u1, const float *u2,
                               float *out, cudaStream_t stream);

/* Local smoothing S_l of Section 3.3 (Eqs. 18-19).  in != out.  Device. */
eecmg_status eecmg_smooth(eecmg_plan_t plan, int level, const float *in, float *out,
                          cudaStream_t stream);

/* One explicit Perona-Malik step D_l, Section 4 (Eqs. 21, 23-24).  in != out. */
eecmg_status eecmg_denoise(eecmg_plan_t plan, int level, const float *in, float *out,
                           cudaStream_t stream);

/*
 * The level smoother C_l^m of Section 2 (MR-II or CGLS per the plan's
 * options) on level `level`: g device data, u device start vector on entry
 * and result on exit, at most m iterations (with the plan's stopping
 * rules).  Uses the plan's workspace.  Asynchronous; the outcome is read
 * with eecmg_plan_stats (entry `level`).
 */
eecmg_status eecmg_level_solve(eecmg_plan_t plan, int level, const float *g, float *u, int m,
                               cudaStream_t stream);

/*
 * r = g - H u and its norms, for callers that cannot allocate device memory
 * (a process that forbids cudaMalloc after start-up because it can stall
 * the device mid-request, or code under a framework allocator that already
 * holds all of the GPU's memory).  The paper has no counterpart: this is the
 * first step of a level solve (the residual of Section 2's stopping rule)
 * without a plan.  H is the zero-boundary convolution with psf (host FP64,
 * psf_h x psf_w, odd, radius <= EECMG_MAX_RADIUS).  g, u, r: device,
 * height x width floats (r must not alias g or u); norms: device, 2
 * doubles receiving ||r||^2 and ||g||^2 (Euclidean).  width and height must
 * be in [1, 4096].  Asynchronous on `stream`.
 * Scratch: the PSF taps, the reduction's per-block partial sums and its
 * scalars live in one fixed __device__ array (about 264 KB) that every GPU
 * which loads the library holds until the process exits; no call allocates
 * or frees memory.  The first call on a device looks up that array's device
 * address (once per device); under lazy module loading (CUDA's default) that
 * lookup is also what loads the library's device code and reserves the
 * array, so the first call is a warm-up: make it at start-up, before any
 * stream capture and before a framework allocator reserves the GPU's memory.
 * Later calls allocate nothing.
 * Every call shares the array and reinitialises it, so calls whose work
 * overlaps on the GPU (other streams, other threads) race: serialise them.
 * Errors: INVALID_ARG (sizes, PSF, NULL or aliased buffers), CUDA.
 */
eecmg_status eecmg_residual_noalloc(int width, int height, const double *psf, int psf_w,
                                    int psf_h, const float *g, const float *u, float *r,
                                    double *norms, cudaStream_t stream);

/* ---- partition of the level solves and its autotuner ------------------ */

/*
 * How the persistent level solves are split over the GPU (system design, no
 * counterpart in the paper).  A level with FP32 storage (MR-II or CGLS), a
 * kernel radius of at most 5 and at most resident_max_tiles 32x64 tiles runs on one
 * thread-block cluster whose blocks keep all the solve's vectors in shared
 * memory for the whole solve (one or two tiles per block, at most 16 blocks).
 * Otherwise a level of at most cluster_max_px pixels runs on one cluster of
 * up to 16 blocks that exchange their sums through distributed shared memory
 * and stream the vectors through L2; larger levels run as a cooperative grid
 * of max(32x64 tiles, pixels / px_per_block) blocks, at most blocks_per_sm
 * per SM.  The fused start of a prolonged level runs on tiles of psd_tile_h
 * x 64 pixels (16 rows give small levels more blocks; its result does not
 * depend on the tile).  Process-wide.  Initial values: the GB300 optimum of
 * measured sweeps (resident_max_tiles 32, cluster_max_px 16384, px_per_block
 * 2048, blocks_per_sm 2, psd_tile_h 32), overridable by the environment
 * variables EECMG_RESIDENT_MAX_TILES, EECMG_CLUSTER_MAX_PX,
 * EECMG_PX_PER_BLOCK, EECMG_BLOCKS_PER_SM, EECMG_PSD_TILE_H read at first
 * use.
 */
typedef struct {
    long long cluster_max_px; /* >= 0; 0 = never cluster mode                 */
    int px_per_block;         /* 1024 .. 4194304                              */
    int blocks_per_sm;        /* 1 .. 3                                       */
    int resident_max_tiles;   /* 0 .. 32; 0 = never shared-memory resident     */
    int psd_tile_h;           /* 16 or 32: rows of the fused level start's
                                 64-column tiles (Algorithm 2, Step 2)        */
} eecmg_tuning;

eecmg_status eecmg_get_tuning(eecmg_tuning *out);

/*
 * Sets the partition.  Every solve of a process must be partitioned the same
 * way (that is what keeps batched and served results bitwise equal to a
 * plan's own restoration), so this returns EECMG_ERR_BUSY while any plan
 * owning a workspace or any server exists.  INVALID_ARG outside the ranges.
 */
eecmg_status eecmg_set_tuning(const eecmg_tuning *t);

/*
 * Autotuner: times one batched restoration (eecmg_restore_batched) of the n
 * plans on the inputs g[i] (device, plan i's size) under candidate
 * partitions -- a coordinate search over resident_max_tiles in {0, 16, 32},
 * then cluster_max_px in {0, 4096, 16384, 65536, 262144}, then px_per_block
 * in {1024, 2048, 4096}, then blocks_per_sm in {1, 2, 3}, from the current
 * setting -- with `reps` timed
 * runs each (CUDA events on `stream`, after two warm-up runs), and keeps the
 * fastest (a candidate must beat the incumbent by 3 %; also written to *best
 * if non-NULL).  The plans are descriptions:
 * the tuner restores private copies with their own workspaces and frees
 * them.  Needs the same conditions as eecmg_set_tuning (BUSY otherwise: pass
 * plans created with workspace = 0).  Synchronises the stream.
 */
eecmg_status eecmg_autotune(const eecmg_plan_t *plans, const float *const *g, int n, int reps,
                            cudaStream_t stream, eecmg_tuning *best);

/*
 * Diagnostic of the failure path (no counterpart in the paper).  Every wait
 * inside a level solve (grid barrier poll, cluster mbarrier wait) gives up
 * after a clock limit, sets the job's error flag and returns, so a stuck
 * solve surfaces as EECMG_ERR_TIMEOUT instead of a hung GPU.  This call runs
 * one such barrier whose arrival count can never be reached (cluster = 0:
 * the grid barrier; 1: the cluster mbarrier) with a limit of about 10 us on
 * one block, then reads the flag.  Returns EECMG_ERR_TIMEOUT when the wait
 * gave up as designed, EECMG_OK if it did not (a defect), CUDA/OOM on
 * failures.  Synchronises the stream; allocates and frees a small scratch.
 */
eecmg_status eecmg_selftest_bounded_wait(int cluster, cudaStream_t stream);

/*
 * Diagnostic (no counterpart in the paper): the FP32 FMA rate of the current
 * GPU, the compute half of the roofline of the convolution and stencil
 * kernels.  One warm-up and `reps` timed launches (CUDA events on `stream`)
 * of a kernel running independent fmaf chains on every SM at full
 * occupancy; *tflops receives the best rate as 2 x FMAs per second / 1e12.
 * Synchronises the stream; allocates and frees a 1 KB buffer.  Errors:
 * INVALID_ARG (reps < 1, NULL output), OOM, CUDA.
 */
eecmg_status eecmg_probe_fp32_fma(int reps, cudaStream_t stream, double *tflops);

/* ---- serving: continuous batching of restoration requests -------------- */

typedef struct eecmg_server_s *eecmg_server_t;

/*
 * Creates a server that admits restoration requests while their workspace
 * fits in mem_budget_bytes of device memory and at most max_slots are
 * active, keeps each request's level pyramid and solver state resident,
 * and advances all active requests together, one cascade step per
 * scheduler tick, on its own stream and host thread.
 */
eecmg_status eecmg_server_create(size_t mem_budget_bytes, int max_slots, eecmg_server_t *out);

/*
 * Queues one request.  plan: a plan describing the request (size, PSF,
 * options; shared and read-only, only its description is used; it may be a
 * workspace = 0 plan and must stay alive until the request completes);
 * g_delta, u_out: device buffers that stay valid until the request completes.
 * *ticket receives an id.  Errors: INVALID_ARG (also a plan with more than 30
 * levels or more than 16 diffusion steps: the server's per-tick tables are
 * sized for these at creation and nothing is allocated while serving), BUSY
 * (queue full), OOM (the request alone exceeds the budget).
 */
eecmg_status eecmg_server_submit(eecmg_server_t srv, eecmg_plan_t plan, const float *g_delta,
                                 float *u_out, uint64_t *ticket);

/* *done = 1 once the result is in u_out; *latency_ms = submit -> done. */
eecmg_status eecmg_server_poll(eecmg_server_t srv, uint64_t ticket, int *done,
                               double *latency_ms);

/* Blocks until every queued request has completed. */
eecmg_status eecmg_server_drain(eecmg_server_t srv);

/* Drains, stops the scheduler thread and frees all device memory. */
eecmg_status eecmg_server_destroy(eecmg_server_t srv);

/* ------------------------------------------------------------------ */
/* Volumes: the method on 3-D data (the paper's Section 6 names volumes  */
/* as the next application; every operator carries over with the slice  */
/* axis treated exactly like the row and column axes).                  */
/* ------------------------------------------------------------------ */

/* Largest PSF radius per axis for volumes (PSF up to 13 x 13 x 13). */
#define EECMG_VOL_MAX_RADIUS 6

typedef struct eecmg_vol_s *eecmg_vol_t;

/*
 * Creates a restoration plan for width x height x depth volumes, stored
 * slice-major: x[(k * height + i) * width + j] (FP32, [0, 255] grey scale),
 * at most 2^31 voxels and 65535 slices.
 * The cascade is Algorithm 2 with, per level:
 *   restriction  coarse (a, b, c) = fine (2a, 2b, 2c) (Eqs. 12-13 per axis);
 *   H_l          zero-boundary 3-D convolution with
 *                K_l(o, p, q) = rho K_{l+1}(2o, 2p, 2q), rho = N_{l+1} / N_l
 *                (Eq. 14 with the RMS adjoint; GALERKIN_RENORM rescales to the
 *                fine PSF's sum);
 *   Pi           u^{l-1} + 1/4 of the trilinear interpolant of the level-(l-2)
 *                differences (Section 3.2 per axis);
 *   P            the three-point quadratic rule along all three axes;
 *   S            weighted least-squares hyperplane fit over the 3 x 3 x 3
 *                neighbourhood with the weights of Eq. 18 (Section 3.3);
 *   D            explicit Perona-Malik steps (Eqs. 20-24) with the six face
 *                neighbours;
 *   C_l^m        MR-II with the stopping rules of eecmg_options.
 * Each side of a coarser level is ceil(side / 2).  psf: host FP64, psf_d x
 * psf_h x psf_w (slice-major), odd sides, radius <= EECMG_VOL_MAX_RADIUS per
 * axis, positive sum, centrosymmetric (MR-II needs H symmetric); copied.  A
 * PSF that is an outer product of three vectors runs as three 1-D passes.
 * alpha is the Perona-Malik step tau, 0 <= alpha <= 0.25 as for images (the
 * step keeps the discrete maximum principle for alpha <= 1/6); k > 0.  iters: `levels` caps m_l (coarsest first) or
 * NULL for the economy schedule of Section 2.  opt: NULL for the defaults;
 * smoother must be MR2, prolong EECMG, storage FP32, workspace 1 (else
 * UNSUPPORTED); use_graph selects one CUDA graph per plan; the other fields
 * mean what they mean for images (precise_conv, persistent, fuse_start and
 * early_check are ignored: every level solve is one cooperative launch).
 * The plan allocates its workspace on the current device: the data and
 * solution pyramids plus eight solver vectors of the finest size.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
eecmg_status eecmg_vol_plan(int width, int height, int depth, int levels, const double *psf,
                            int psf_w, int psf_h, int psf_d, double alpha, double k,
                            const int *iters, const eecmg_options *opt, eecmg_vol_t *out);

/* Releases the plan and its device memory (synchronises the device first). */
eecmg_status eecmg_vol_plan_destroy(eecmg_vol_t plan);

/*
 * Plan geometry: per level (coarsest first; NULL outputs skipped) the sides
 * and the scheduled cap m_l, plus the workspace bytes.  INVALID_ARG for NULL.
 */
eecmg_status eecmg_vol_plan_info(eecmg_vol_t plan, int *levels, int *level_w, int *level_h,
                                 int *level_d, int *iters, size_t *workspace_bytes);

/*
 * Restores one volume (Algorithm 2).  g_delta and u_out: device buffers of
 * depth x height x width floats; they may alias (g is copied into the
 * workspace first).  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA.
 */
eecmg_status eecmg_vol_restore(eecmg_vol_t plan, const float *g_delta, float *u_out,
                               cudaStream_t stream);

/* As eecmg_vol_restore with HOST buffers; synchronises `stream`. */
eecmg_status eecmg_vol_restore_host(eecmg_vol_t plan, const float *g_host, float *u_host,
                                    cudaStream_t stream);

/*
 * Per level (coarsest first) of the last restoration or level solve: the
 * iterations run and ||g_l - H_l u_l||_RMS.  Synchronises the device.
 * TIMEOUT if a level solve's bounded grid barrier gave up.
 */
eecmg_status eecmg_vol_plan_stats(eecmg_vol_t plan, int *iters_done, double *res_rms);

/*
 * Per-launch timing of a volume plan.  enable = 1: later restorations launch
 * eagerly (no graph) with an event pair around each level start and each
 * level solve; profile_read (synchronises the device) returns per level,
 * coarsest first, the start's and the solve's milliseconds of the last
 * restoration and the solve's algorithmic bytes (each operand read or
 * written once per phase, counted from the iterations it ran); NULL outputs
 * are skipped.  INVALID_ARG if profiling is off; CUDA.
 */
eecmg_status eecmg_vol_plan_profile(eecmg_vol_t plan, int enable);
eecmg_status eecmg_vol_plan_profile_read(eecmg_vol_t plan, double *start_ms, double *solve_ms,
                                         double *solve_bytes);

/* Operators of one level, for tests and composition (device buffers of the
 * level's size, not aliased; asynchronous on `stream`):
 *   apply_H      y = H_l x (transpose = 0) or H_l^T x;
 *   restrict     coarse = level `level`'s injection of level level+1's fine;
 *   start_level  out = D(S(P(Pi(u1, u2)))), u1 on level-1, u2 on level-2
 *                (level >= 2), with the plan's diffusion_steps;
 *   smooth       y = S(x);  denoise  y = one Perona-Malik step of x;
 *   level_solve  u <- C_l^m u (MR-II from the start in u, at most m
 *                iterations, the plan's stopping rules); see plan_stats.
 * Errors: INVALID_ARG (level, buffers), CUDA. */
eecmg_status eecmg_vol_apply_H(eecmg_vol_t plan, int level, const float *x, float *y,
                               int transpose, cudaStream_t stream);
eecmg_status eecmg_vol_restrict(eecmg_vol_t plan, int level, const float *fine, float *coarse,
                                cudaStream_t stream);
eecmg_status eecmg_vol_start_level(eecmg_vol_t plan, int level, const float *u1,
                                   const float *u2, float *out, cudaStream_t stream);
eecmg_status eecmg_vol_smooth(eecmg_vol_t plan, int level, const float *x, float *y,
                              cudaStream_t stream);
eecmg_status eecmg_vol_denoise(eecmg_vol_t plan, int level, const float *x, float *y,
                               cudaStream_t stream);
eecmg_status eecmg_vol_level_solve(eecmg_vol_t plan, int level, const float *g, float *u, int m,
                                   cudaStream_t stream);

/* Thread-local description of the last error (never NULL). */
const char *eecmg_last_error(void);

/* Library version string. */
const char *eecmg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EECMG_H */
