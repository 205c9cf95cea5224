/*
 * libms -- cosine mean-shift with the online seed optimisation policy (OSOP)
 * on one GPU (sm_103a). C ABI: plain pointers and sizes, no C++ types.
 *
 * Method: "Faster Mean-shift: GPU-accelerated clustering for cosine
 * embedding-based cell segmentation and tracking" (Zhao et al.).
 *   Problem statement: given a vector set S and a bandwidth h, return the
 *   modes and a vector-to-mode assignment (Algorithm 1 and 2, Require/Ensure).
 *   Cosine distance d = 1 - cos (Eq. 9); the flat kernel k_h = [d <= h]
 *   (Eq. 11), so a window is {i : cos(x, p_i) >= c} with c = 1 - h.
 *   Update x <- normalise(mean of the window) (Eq. 6-8, Sec. 3.2.1).
 *   Seeds in rounds sized by OSOP (Eq. 19-21, Sec. 3.2.2-3.2.4), early
 *   stopping at gamma (Sec. 3.2.3), prune/merge and labelling (the last
 *   steps of Algorithm 2).
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers, h_* are HOST pointers; other
 *    pointers to scalars (e.g. n_seeded_out) are host pointers.
 *  - Device inputs passed to ms_create are BORROWED: the caller keeps them
 *    alive and unchanged until ms_destroy. Every ms_ctx OWNS its workspace,
 *    allocated in ms_create and freed by ms_destroy.
 *  - Work is enqueued on the stream given to ms_create (NULL = legacy default
 *    stream). Calls that return counts synchronise that stream.
 *  - Errors: every call returns an ms_status; the library never aborts,
 *    exits or prints. ms_last_error() gives a thread-local message for the
 *    last failing call on the calling thread. After MS_ERR_CUDA the context
 *    should be destroyed.
 *  - A context is not thread safe; distinct contexts may be used from
 *    distinct threads.
 */
#ifndef MS_H
#define MS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MS_API __attribute__((visibility("default")))
#else
#define MS_API
#endif

typedef struct ms_ctx ms_ctx;
typedef int32_t ms_status;

#define MS_OK 0
#define MS_ERR_INVALID_ARG 1   /* bad argument or input values (rejected before any work) */
#define MS_ERR_CUDA 2          /* a CUDA call failed; see ms_last_error() */
#define MS_ERR_OOM 3           /* device or pinned-host allocation failed */
#define MS_ERR_NOT_CONVERGED 4 /* a round ended with no converged seed */
#define MS_ERR_STATE 5         /* call out of order (e.g. ms_iterate before ms_seed_batch) */
#define MS_ERR_TIMEOUT 6       /* a bounded device-side wait gave up */

#define MS_FLAT 0 /* flat kernel, Eq. 11 */
#define MS_VMF 1  /* smooth kernel exp(kappa * cos): only the ms_vmf_* calls */

#define MS_FP32 0 /* plain FP32 SIMT similarity and sums */
#define MS_BF16 1 /* BF16 tensor-core GEMMs with FP32 accumulation and an FP32 recheck band (the
                     shift, coverage, labelling and, in batches and single frames, the merge's
                     two contractions; every decision equal to the FP32 form's) */

#define MS_MAX_DIM 32

/* Hyper-parameters; ms_config_default() fills the paper's values. */
typedef struct ms_config {
    int32_t dim;          /* embedding dimension d, 1..MS_MAX_DIM */
    int32_t kernel;       /* MS_FLAT (MS_VMF is only for ms_vmf_*) */
    double bandwidth_cos; /* c = 1 - h; default 0.9 (h = 0.1, Sec. 4.2/4.3) */
    double kappa;         /* vMF concentration for MS_VMF */
    double tol;           /* convergence ||x' - x||_2 < tol, evaluated in FP64; default 1e-6 */
    int32_t max_iter;     /* iterations per round before the round is cut; default 300 */
    int32_t n_initial;    /* N_initial = 128 (Sec. 3.2.4) */
    double gamma;         /* early stop when #converged > gamma * N; 0.9 (Sec. 3.2.3) */
    double L;             /* lower schedule bound (Eq. 21); 2 */
    double H;             /* upper schedule bound; 8 (Sec. 3.2.4) */
    double P_target;      /* P in Eq. 19; 0.99 */
    double alpha;         /* Eq. 20; only used when L <= 0, then L = alpha / gamma */
    double merge_cos;     /* modes closer than this cosine are merged; default = bandwidth_cos */
    uint64_t seed;        /* seed-order permutation offset: SplitMix64(seed ^ frame_id) */
    uint64_t frame_id;
    int32_t precision;    /* MS_FP32 or MS_BF16 */
    int32_t max_rounds;   /* guard on OSOP rounds; default 1000000 */
    double eps_band;      /* reserved, 0: the BF16 recheck band is the library's derived bound
                             (2^-14 around c; other values are ignored) */
    int32_t all_seeds;    /* 1 = Algorithm 1: every pixel seeds a single round, gamma = 1 */
    int32_t batch_split;  /* ms_batch_* only: 0 = each frame split into work items as on its own
                             (results bit-identical to ms_run on that frame); 1 = the batch's
                             work items shared out by each frame's seed x pixel work */
    int32_t batch_max_passes; /* ms_batch_* only: guard on passes of the graph's loop body (every
                                 iterating frame advances one iteration per pass); a batch still
                                 unfinished after it stops with MS_ERR_TIMEOUT. 0 = 200000 */
    int32_t video_restart; /* ms_video_* only: 1 = every frame starts from n_initial instead of the
                              seed count carried from the previous frame */
    int32_t tc_shape;     /* BF16 form: warp arrangement of the shift kernel, the same arithmetic in
                             each (results bit-identical). Mask warps x pixels each per tile, GEMM2
                             issuers: 0 = 16 x 32, two (default); 1 = 16 x 32, one; 2 = 8 x 64,
                             two; 3 = 8 x 64, one; 4 = two groups of 8 x 64 taking alternate
                             tiles, two; 5 = the same groups, one; 6 = GEMM1 on 64-pixel units
                             (four S buffers, six mask buffers), two groups of 8 x 32 taking
                             alternate units, two issuers; 7 = as 6, one issuer */
    int32_t reserved[3];  /* zero */
} ms_config;

/* Per-context counters, filled by ms_stats_get. */
typedef struct ms_stats {
    int32_t rounds;        /* OSOP rounds run */
    int32_t n_modes;       /* modes kept */
    int32_t iters_total;   /* iterations summed over rounds */
    int32_t reserved0;
    int64_t n_fg;          /* foreground pixels */
    int64_t seeds;         /* seeds drawn */
    int64_t seed_iters;    /* seed-iterations: one seed shifted once against all pixels */
    int64_t candidates;    /* converged seeds offered to the merge */
    int64_t dropped;       /* seeds not converged when their round ended (Sec. 3.2.3) */
    int64_t band_pairs;    /* BF16 form: seed-pixel pairs rechecked in FP32 */
    int64_t uncovered;     /* foreground pixels not yet covered */
    int64_t workspace_bytes;
    int64_t launches;      /* kernels launched by this context */
    int64_t shift_launches;   /* shift-kernel launches that did work (profiling on) */
    double shift_ms;       /* their summed CUDA-event time (profiling on) */
} ms_stats;

/* Fill *cfg with the paper's defaults for dimension 16 and MS_FP32: h = 0.1
 * (Sec. 4.2 and 4.3), gamma = 0.9 (Sec. 3.2.3), N_initial = 128, L = 2 and
 * H = 8 (Sec. 3.2.4), P = 0.99 (Eq. 19). Cannot fail. */
MS_API void ms_config_default(ms_config* cfg);

/* Message describing the last failure on the calling thread ("" if none).
 * No counterpart in the paper. Cannot fail; the string is thread-local and is
 * overwritten by the thread's next failing call. */
MS_API const char* ms_last_error(void);

/* Testing hook for the allocation-failure path (no counterpart in the paper):
 * the next `count` workspace allocations of this process (ms_create,
 * ms_batch_create) fail with MS_ERR_OOM as if cudaMalloc had failed, without
 * calling it; nothing is left allocated. count <= 0 clears it. */
MS_API void ms_inject_alloc_failure(int32_t count);

/* Device bytes ms_create would allocate for n_pixels pixels with cfg (no
 * counterpart in the paper; the layout is the one in ms_create). Allocates
 * nothing. MS_ERR_INVALID_ARG for a bad cfg, a NULL bytes_out or n_pixels
 * outside [0, 2^24). */
MS_API ms_status ms_workspace_bytes(const ms_config* cfg, int64_t n_pixels, int64_t* bytes_out);

/* Bind a frame (the vector set S of Algorithm 2) and allocate the workspace.
 * d_emb: device float32 [n_pixels, cfg->dim] row-major embeddings (any norm;
 *        each foreground vector is normalised, Eq. 9). Borrowed.
 * d_mask: device uint8 [n_pixels], nonzero = foreground; NULL = all
 *        foreground. Borrowed.
 * stream: a cudaStream_t (NULL for the legacy default stream).
 * Enqueues normalisation and foreground compaction and synchronises.
 * MS_ERR_INVALID_ARG for a bad cfg, n_pixels < 0 or >= 2^24, or a foreground
 * vector with zero or non-finite norm (nothing is allocated then). */
MS_API ms_status ms_create(const ms_config* cfg, const float* d_emb, const uint8_t* d_mask,
                    int64_t n_pixels, void* stream, ms_ctx** out);

/* Draw the next seed batch (the seed-selection step of Algorithm 2): the next n uncovered
 * positions of the frame's fixed seed order pi(j) = (b + a j) mod n_fg.
 * n_requested <= 0 uses the OSOP schedule's current N (Sec. 3.2.4).
 * Drawn pixels count as covered. *n_seeded_out = 0 means every foreground
 * pixel is covered. MS_ERR_STATE if a previous batch was not merged. */
MS_API ms_status ms_seed_batch(ms_ctx* ctx, int32_t n_requested, int32_t* n_seeded_out);

/* Shift the current batch in lockstep (the shift loop of Algorithm 2) until more
 * than gamma of it has converged, none is still moving, or max_iter
 * (<= 0: cfg->max_iter) iterations; unconverged seeds are dropped
 * (Sec. 3.2.3). MS_ERR_NOT_CONVERGED if no seed converged (the batch is still
 * consumed). MS_ERR_STATE without a pending batch. */
MS_API ms_status ms_iterate(ms_ctx* ctx, int32_t max_iter, int32_t* n_converged_out,
                     int32_t* n_iters_out);

/* Prune and merge the batch's converged modes into the kept set (the
 * prune/merge step of Algorithm 2): in order of support (descending) then seed order, a mode is kept
 * when its FP64 cosine to every kept mode is < merge_cos. Then marks pixels
 * within c of a new mode as covered and updates N by Eq. 19-21.
 * MS_ERR_STATE unless ms_iterate ran on the current batch. */
MS_API ms_status ms_merge_modes(ms_ctx* ctx, int32_t* n_modes_out, int64_t* n_uncovered_out);

/* Cluster every vector by its distance to the modes (the
 * labelling step of Algorithm 2): label = argmax_k cos(p_i, m_k), lowest k on ties, -1 for
 * background. d_labels_out: device int32 [n_pixels], caller-owned.
 * d_modes_out: device float32 [cap, dim] or NULL. MS_ERR_INVALID_ARG if
 * d_modes_out is given and cap < the mode count (nothing written). */
MS_API ms_status ms_label(ms_ctx* ctx, int32_t* d_labels_out, float* d_modes_out, int32_t cap,
                   int32_t* n_modes_out);

/* Free the workspace (no counterpart in the paper). Synchronises the
 * context's stream first. Accepts NULL; cannot fail. */
MS_API void ms_destroy(ms_ctx* ctx);

/* The whole method for the bound frame (Algorithm 2): OSOP rounds (seed,
 * iterate, merge) until every foreground pixel is covered or max_rounds, then
 * ms_label. A round in which no seed converged is not an error here (its
 * batch is consumed and the next round starts), nor is stopping at
 * max_rounds (ms_stats.uncovered > 0 then). Errors: MS_ERR_INVALID_ARG for a
 * NULL ctx, MS_ERR_STATE while a seed batch is pending, otherwise those of
 * ms_seed_batch, ms_iterate, ms_merge_modes and ms_label. */
MS_API ms_status ms_run(ms_ctx* ctx, int32_t* d_labels_out, float* d_modes_out, int32_t cap,
                 int32_t* n_modes_out);

/* Measurement only (no counterpart in the paper): record CUDA events around
 * every shift-kernel launch on the context's stream (enable = 1) so ms_stats
 * reports its device time; off by default. MS_ERR_INVALID_ARG for a NULL ctx,
 * MS_ERR_CUDA if the events cannot be created. */
MS_API ms_status ms_profile(ms_ctx* ctx, int32_t enable);

/* Counters of the context so far (no counterpart in the paper). Does not
 * synchronise. MS_ERR_INVALID_ARG for a NULL argument. */
MS_API ms_status ms_stats_get(const ms_ctx* ctx, ms_stats* out);

/* OSOP state carried across frames of a video (Sec. 3.2.4; Sec. 4.3, Table 3):
 * the seed count N that a next frame starts from. It follows the same Eq. 19-21
 * updates as the frame's own schedule, from the frame's starting N, without
 * the clamp to the frame's uncovered pixel count (that clamp bounds the draws
 * at the frame's end), and is bounded by the largest seed batch the frame drew
 * (no frame can use more seeds than it has uncovered pixels). ms_set_state
 * sets the frame's starting N; it returns MS_ERR_STATE once the frame's first
 * round has run. MS_ERR_INVALID_ARG for a NULL argument or (ms_set_state)
 * n_next < 1. */
MS_API ms_status ms_get_state(const ms_ctx* ctx, int64_t* n_next_out);
MS_API ms_status ms_set_state(ms_ctx* ctx, int64_t n_next);

/* Copy an internal array to host memory for inspection (tests, debugging;
 * no counterpart in the paper). what: MS_INSPECT_* below. Writes min(cap,
 * available) elements to h_out and the available count to *count_out.
 * Synchronises the stream. MS_ERR_INVALID_ARG for a NULL ctx, a NULL h_out
 * with cap > 0 or an unknown code; MS_ERR_CUDA if a copy fails. */
#define MS_INSPECT_SEED_LOG 1  /* int32: foreground index of every seed in draw order */
#define MS_INSPECT_MODES 2     /* float32 [K, dim]: kept modes in keep order */
#define MS_INSPECT_SUPPORT 3   /* int32 [K]: window size of each kept mode */
#define MS_INSPECT_COVERED 4   /* uint8 [n_fg]: coverage flags */
#define MS_INSPECT_ROUND_LOG 5 /* int64 [rounds, 4]: N requested, seeds, modes kept, uncovered */
#define MS_INSPECT_PIXELS 6    /* float32 [n_fg, dim]: normalised foreground */
MS_API ms_status ms_inspect(const ms_ctx* ctx, int32_t what, void* h_out, int64_t cap,
                     int64_t* count_out);

/* The whole method (Algorithm 2) on one frame held in HOST memory: copies h_emb and h_mask
 * to the device, runs ms_create + ms_run, and copies labels (and modes, when
 * h_modes is not NULL) back, all on `stream`; returns after the copies end.
 * h_emb: float32 [n_pixels, cfg->dim]; h_mask: uint8 [n_pixels] or NULL;
 * h_labels: int32 [n_pixels]; h_modes: float32 [cap, dim] or NULL. Pinned
 * host buffers make the copies asynchronous. Allocates and frees its own
 * device memory. stats_out (nullable) receives the run's counters. Errors:
 * MS_ERR_INVALID_ARG for a bad cfg, n_pixels outside [0, 2^24) or a NULL
 * h_emb or h_labels with n_pixels > 0; MS_ERR_OOM if the device buffer cannot
 * be allocated; otherwise those of ms_create and ms_run (nothing is copied
 * back after a failure). */
MS_API ms_status ms_run_host(const ms_config* cfg, const float* h_emb, const uint8_t* h_mask,
                             int64_t n_pixels, void* stream, int32_t* h_labels, float* h_modes,
                             int32_t cap, int32_t* n_modes_out, ms_stats* stats_out);

/* Smooth-kernel form: T unrolled mean-shift steps with the exponential
 * (von Mises-Fisher) profile of the Eq. 2 kernel family instead of the flat
 * kernel, every seed moved to the weighted mean of all pixels (the dense
 * update of Sec. 3.2.1) and renormalised:
 *   x_{t+1} = normalise( sum_i exp(kappa (x_t . p_i - 1)) p_i ).
 * d_P: device float32 [N, dim] pixels (used as given, not normalised);
 * d_X0: device float32 [M, dim] starting seeds; dim must be 16; 0 <= kappa < 80.
 * ms_vmf_forward writes x_T to d_XT [M, dim].
 * ms_vmf_backward takes d_GT = dL/dx_T [M, dim] and writes dL/dP to d_dP
 * [N, dim] and dL/dx_0 to d_dX0 [M, dim]. It recomputes the iterates by
 * re-running the forward and recomputes every kernel weight on the fly; no
 * M x N matrix is stored. Both allocate their workspace stream-ordered on
 * `stream` from the library's own memory pool (which keeps freed memory mapped
 * for the next call) and return without synchronising. Results are
 * deterministic. MS_ERR_INVALID_ARG on NULL pointers or bad sizes. */
MS_API ms_status ms_vmf_forward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                double kappa, int32_t T, float* d_XT, void* stream);
MS_API ms_status ms_vmf_backward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                 double kappa, int32_t T, const float* d_GT, float* d_dP, float* d_dX0,
                                 void* stream);
/* The same with a precision: MS_FP32 is the calls above; MS_BF16 runs every
 * forward step on the tensor cores. There, GEMM1 scores kappa log2(e) (s - 1)
 * from three-term BF16 splits of kappa log2(e) x and of p (six products, FP32
 * accumulation), the weight w = exp(kappa (s - 1)) is formed in FP32 and split
 * as w = wh + wl (BF16), and GEMM2 accumulates wh.[ph | pm | pl] + wl.[ph | pm]
 * in FP32; per-chunk sums are
 * added in a fixed order, so results are deterministic. ms_vmf_backward_ex
 * with MS_BF16 also runs both reverse passes of every step on the tensor
 * cores (the derivative of the step above): with gy = (g - x'(x'.g))/|y|,
 * the scores kappa log2(e) x.p and gy.p come from six products of three-term
 * splits each, w and ds = kappa w (gy.p) are split into two BF16 terms, and
 * dL/dx = sum_i ds p_i (seeds as rows) and dL/dp_i += sum_m w gy_m + ds x_m
 * (pixels as rows) accumulate in FP32, per-chunk sums again added in a fixed
 * order. With MS_BF16 the forward synchronises `stream` once at the end, the
 * backward twice (after the re-run forward and at the end), to read the
 * device status: MS_ERR_TIMEOUT if a bounded wait inside a kernel gave up
 * (the outputs are then NaN). */
MS_API ms_status ms_vmf_forward_ex(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                   double kappa, int32_t T, int32_t precision, float* d_XT, void* stream);
MS_API ms_status ms_vmf_backward_ex(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                    double kappa, int32_t T, int32_t precision, const float* d_GT, float* d_dP,
                                    float* d_dX0, void* stream);

/* Other distances and kernel profiles (Eq. 2-6 with Eq. 3, 4 and 9): T steps
 * of the dense mean-shift update, every seed against every vector,
 *     t = (d(x, p) / h)^2,   w = k(t),   x' = sum w p / sum w   (Eq. 6),
 * with d the Euclidean distance ||x - p|| (Eq. 4, vectors as given) or the
 * cosine distance 1 - cos (Eq. 9: vectors and seeds are normalised, x' is
 * renormalised), and k flat [t <= 1] (Eq. 3), Epanechnikov max(0, 1 - t) or
 * Gaussian exp(-t / 2). A seed whose weights are all zero stays put.
 * d_P: device float32 [N, dim]; d_X0: device float32 [M, dim] starting seeds;
 * d_XT: device float32 [M, dim] receives x_T; d_counts (nullable): device int32
 * [M] receives each seed's count of vectors with nonzero weight in the last
 * step. 1 <= dim <= 32, h > 0, T >= 0. FP32 arithmetic; results are
 * deterministic. Allocates its workspace stream-ordered on `stream` from the
 * library's own memory pool and synchronises it once, after validating the inputs on the
 * device: MS_ERR_INVALID_ARG for a non-finite component or (cosine) a zero
 * norm. */
#define MS_DIST_COSINE 0
#define MS_DIST_EUCLID 1
#define MS_PROFILE_FLAT 0
#define MS_PROFILE_EPANECHNIKOV 1
#define MS_PROFILE_GAUSSIAN 2
MS_API ms_status ms_kernel_shift(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                 int32_t distance, int32_t profile, double h, int32_t T, float* d_XT,
                                 int32_t* d_counts, void* stream);

/* Check of the BF16 tensor-core shift tile (Eq. 11 window, Eq. 8 sums) on
 * one work item: 128 seeds d_X [128, 16] (device, unit FP32) against n_pix
 * pixels d_P [n_pix, 16] (device FP32, normalised inside) with bandwidth c.
 * It runs the production kernel once and returns, in HOST buffers,
 * h_S [128, n_pad] the raw accumulator Xh.Ph + Xh.Pm + Xl.Ph - c (c rounded
 * up to FP32; n_pad = n_pix rounded up to 128) and h_acc [128, 17] each seed's window
 * sums (units of 2^-36) and window size. 1 <= n_pix <= 4096. Allocates and
 * frees its own device memory; synchronises the device. MS_ERR_INVALID_ARG
 * for NULL pointers or n_pix out of range, MS_ERR_TIMEOUT if a bounded wait
 * inside the kernel gave up. */
MS_API ms_status ms_tc_selftest(const float* d_X, const float* d_P, int32_t n_pix, double c, float* h_S,
                                int64_t* h_acc);

/* Window sums with no device allocation. The paper has no counterpart: this
 * is for callers that cannot allocate device memory (an arena or pool that
 * owns the device, allocation forbidden while a stream is captured, a host
 * application that hands a plugin only its buffers). It computes, for m
 * seeds d_X [m, 16] (device FP32) against n pixels d_P [n, 16] (device FP32,
 * each of nonzero finite norm; normalised inside in FP32), every seed's
 * flat-kernel window sum and window size at bandwidth c, into the caller's
 * d_acc_out [m, 17] (device int64: 16 sums in units of 2^-36, then the count)
 * -- the same quantities ms_tc_selftest returns.
 * Scratch lives in one fixed file-scope device array of about 1.2 MB that
 * every GPU loading the library holds until the process exits; it limits
 * m <= 1024 and n <= 16384 (larger sizes return MS_ERR_INVALID_ARG). No
 * cudaMalloc, cudaFree or other allocating call is made. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before capturing a stream. All calls on a device share the
 * array, which keeps the last call's contents (each call clears what must
 * start at zero): calls whose work overlaps on the GPU, e.g. on two streams,
 * race. Work is enqueued on `stream`; the call does not synchronise, so a
 * pixel of zero or non-finite norm cannot be rejected up front: the call then
 * returns MS_OK and every row of d_acc_out reads sums 0 and count -1 (check
 * the counts after synchronising). Each call clears that error state. */
MS_API ms_status ms_window_sums_static(const float* d_X, int32_t m, const float* d_P, int32_t n, double c,
                                       int64_t* d_acc_out, void* stream);

/* Video form (Sec. 3.2.4; Sec. 4.3 and Table 3): the frames of one sequence
 * clustered in order, each as its own vector set (Algorithm 2), with the seed
 * count N carried from each frame into the next (the ms_get_state value; the
 * first frame of the video starts at cfg->n_initial). Frame t of the video
 * (counting over every ms_video_run call) uses the seed order of frame_id =
 * cfg->frame_id + t, so its results equal ms_create + ms_set_state(carried N)
 * + ms_run on that frame with that frame_id.
 *
 * With cfg->video_restart = 1 every frame starts from cfg->n_initial instead
 * (frames then equal ms_create + ms_run on their own; the second stream and the
 * reused workspaces remain).
 *
 * ms_video_create allocates two workspaces for frames of up to max_pixels
 * pixels (0 <= max_pixels < 2^24) and a second, internal stream; cfg as for
 * ms_create (MS_FLAT, all_seeds = 0). Work runs on `stream` (NULL = legacy
 * default stream).
 * ms_video_run clusters T more frames: d_embs[t] device float32
 * [n_pixels[t], dim], d_masks (NULL, or entries NULL = all foreground) device
 * uint8 [n_pixels[t]], d_labels[t] device int32 [n_pixels[t]] receives the
 * labels (-1 background). All borrowed for the duration of the call; the host
 * arrays are read during the call only. While frame t runs its rounds on
 * `stream`, frame t+1 is compacted, normalised and (MS_BF16) split on the
 * internal stream into the other workspace. h_n_start (nullable, host int64
 * [T]) receives the N each frame started from, h_n_modes (nullable, host int32
 * [T]) its mode count. Returns after the last frame's rounds; its labels are
 * written when `stream` reaches them. Errors as ms_create/ms_run for the
 * failing frame; frames before it are complete.
 * ms_video_state gives the N the next frame will start from and the frames
 * clustered so far; ms_video_stats the counters of the last (which = 0) or the
 * previous (which = 1) frame. ms_video_destroy synchronises and frees. */
typedef struct ms_video ms_video;
MS_API ms_status ms_video_create(const ms_config* cfg, int64_t max_pixels, void* stream, ms_video** out);
MS_API ms_status ms_video_run(ms_video* v, int32_t T, const float* const* d_embs, const uint8_t* const* d_masks,
                              const int64_t* n_pixels, int32_t* const* d_labels, int64_t* h_n_start,
                              int32_t* h_n_modes);
MS_API ms_status ms_video_state(const ms_video* v, int64_t* n_carry_out, int64_t* frames_out);
MS_API ms_status ms_video_stats(const ms_video* v, int32_t which, ms_stats* out);
MS_API void ms_video_destroy(ms_video* v);

/* Batched form: B frames (e.g. the frames of a time-lapse sequence, each its
 * own vector set S of Algorithm 2) clustered by one CUDA graph. Every frame
 * runs exactly the single-frame method (same seeds, rounds, modes and labels
 * as ms_create + ms_run on that frame with cfg->frame_id = cfg->frame_id + f)
 * but the OSOP control (Sec. 3.2.2-3.2.4: seed batches, early stop at gamma,
 * merge, coverage, the Eq. 19 schedule) runs on the device, one state
 * machine per frame, and the shift kernel of each iteration is one launch
 * over the work of all frames still iterating. Frames of different sizes are
 * in different rounds at the same time.
 *
 * ms_batch_create binds the frames and builds the graph (a set-up stage, a
 * conditional WHILE node whose body advances every frame by one iteration,
 * then labelling); it allocates the workspace (one cudaMalloc) and
 * synchronises `stream`. Arguments:
 *  cfg       as for ms_create (MS_FLAT).
 *  B         1..4096 frames.
 *  d_embs    host array of B device pointers, frame f float32 [n_pixels[f], dim]. Borrowed.
 *  d_masks   host array of B device pointers (uint8 [n_pixels[f]], NULL entry = all
 *            foreground), or NULL for no masks. Borrowed.
 *  n_pixels  host array of B sizes, each 0 <= n < 2^24, sum < 2^31.
 *  d_labels  host array of B device pointers, int32 [n_pixels[f]]: written by every
 *            ms_batch_run (background -1). Borrowed.
 *  stream    the cudaStream_t the graph is launched on (NULL = legacy default).
 * The pointer arrays are copied; the buffers they point to must stay alive
 * and must not move until ms_batch_destroy. MS_ERR_INVALID_ARG for a bad
 * cfg or frame.
 *
 * ms_batch_run launches the graph once on `stream` (the whole method on all
 * frames, from the embeddings as they are now). With sync = 0 it returns at
 * once; with sync != 0 it waits, reads the per-frame counters back, and
 * returns MS_ERR_INVALID_ARG if a foreground vector had zero or non-finite
 * norm, MS_ERR_TIMEOUT if a bounded device wait gave up.
 * ms_batch_stats fills *out for frame f (or summed over all frames for
 * f = -1) from the last synchronised run; for f = -1 it also gives launches
 * (kernels the graph ran), reserved0 (passes of the loop body), band_pairs
 * and, with profiling on, shift_ms / shift_launches (time of the shift
 * kernels that had work, from the GPU global timer read by one-thread
 * kernels placed before and after each shift launch; includes one launch gap
 * each). ms_batch_profile(b, 1) rebuilds the graph with those timer kernels
 * (0 removes them); ms_batch_profile(b, 2) adds one-thread timer kernels
 * between the phases of the graph as well (see ms_batch_phase_ms); it
 * synchronises the stream. ms_batch_modes copies frame f's K kept modes, float32
 * [K, dim], to h_out (cap >= K; h_out NULL only reports K). ms_batch_destroy
 * synchronises the stream and frees everything. */
typedef struct ms_batch ms_batch;
MS_API ms_status ms_batch_create(const ms_config* cfg, int32_t B, const float* const* d_embs,
                                 const uint8_t* const* d_masks, const int64_t* n_pixels,
                                 int32_t* const* d_labels, void* stream, ms_batch** out);
MS_API ms_status ms_batch_run(ms_batch* b, int32_t sync);
/* ms_batch_run from HOST memory: copies every frame's embeddings (and mask,
 * for frames bound with one) from h_embs[f] / h_masks[f] into the device
 * buffers bound at ms_batch_create, runs the graph, copies each frame's
 * labels into h_labels[f] (int32 [n_pixels[f]]), and synchronises. One
 * cudaMemcpyAsync per buffer on the batch's stream; pinned host buffers make
 * them asynchronous. Host arrays as for ms_batch_create (entries of empty
 * frames are ignored). Errors as ms_batch_run with sync. */
MS_API ms_status ms_batch_run_host(ms_batch* b, const float* const* h_embs, const uint8_t* const* h_masks,
                                   int32_t* const* h_labels);
MS_API ms_status ms_batch_stats(const ms_batch* b, int32_t frame, ms_stats* out);
/* The same work as one ms_batch_run, issued as ordinary kernel launches on
 * the batch's stream instead of the graph: set-up, `passes` passes of the
 * loop body and labelling (for profilers that do not look inside conditional
 * graph nodes). Passes after every frame has finished change nothing, so
 * results equal ms_batch_run's when passes >= the loop's pass count
 * (ms_batch_stats(-1).reserved0 after a graph run). Synchronises;
 * MS_ERR_STATE if a frame is still unfinished after `passes`. */
MS_API ms_status ms_batch_run_eager(ms_batch* b, int32_t passes);
MS_API ms_status ms_batch_profile(ms_batch* b, int32_t enable);
/* Measurement only (no counterpart in the paper): with profiling level 2, the
 * time of the last synchronised run split by phase, in ms, from the GPU
 * global timer: out[0] set-up (compaction, normalisation, packing); summed
 * over the loop's passes out[1] relaunch of the loop body, seed selection and
 * work plan, out[2] the shift, out[3] its finalisation and early-stop check,
 * out[4] the merge chain, out[5] coverage, out[6] the schedule and loop
 * condition; out[7] labelling. Each phase includes the launch gaps inside
 * it. Writes min(cap, 8) values (zeros below level 2) and *n_out = 8.
 * MS_ERR_INVALID_ARG on NULL b or out with cap > 0. */
MS_API ms_status ms_batch_phase_ms(const ms_batch* b, double* out, int32_t cap, int32_t* n_out);
MS_API ms_status ms_batch_modes(const ms_batch* b, int32_t frame, float* h_out, int32_t cap,
                                int32_t* n_modes_out);
MS_API void ms_batch_destroy(ms_batch* b);

/* Work split and tile shape of a batch's shift launches (the autotuned
 * parameters; no counterpart in the paper): batch_split 0 gives every frame the single-frame split
 * (results equal ms_run's frame by frame; target_mult is then unused);
 * batch_split 1 shares target_mult x (shift grid) work items across the
 * iterating frames in proportion to their seed x pixel work (target_mult
 * 1..64). tc_shape is ms_config.tc_shape (0..7; the BF16 form's warp
 * arrangement; the FP32 form ignores it). ms_batch_configure rebuilds the
 * graph (synchronises the stream).
 * ms_batch_autotune times ms_batch_run on the batch's own frames as the
 * median of `reps` graph launches (CUDA events on the batch's stream, after
 * one warm-up launch). Phase 1 times the splits (0, 2), (1, 1), (1, 2),
 * (1, 4), (1, 8) on tc_shape 0; for a BF16 batch, phase 2 times tc_shapes
 * 1..7 on phase 1's fastest split. It keeps the fastest of all, runs it once
 * more so the batch's outputs come from it, and writes min(cap, 5 or 12)
 * results to `results` (host), in the order timed. Both are for speed only
 * (the paper fixes no work split): every tile shape gives the same results,
 * and batch_split 0 equals ms_run frame by frame; batch_split 1 cuts each
 * seed's window sums into other chunks, so its rounding may differ while it
 * meets the same bar against the FP64 method. MS_ERR_INVALID_ARG for a NULL batch, batch_split not 0 or 1,
 * target_mult outside 1..64, tc_shape outside 0..7, reps outside 1..100 or
 * cap < 0; otherwise the errors of ms_batch_run with sync. */
typedef struct ms_tune_result {
    int32_t batch_split;
    int32_t target_mult;
    int32_t tc_shape;
    int32_t reserved;
    double ms;
} ms_tune_result;
MS_API ms_status ms_batch_configure(ms_batch* b, int32_t batch_split, int32_t target_mult, int32_t tc_shape);
MS_API ms_status ms_batch_autotune(ms_batch* b, int32_t reps, ms_tune_result* results, int32_t cap,
                                   int32_t* n_results);

#ifdef __cplusplus
}
#endif
#endif /* MS_H */
