/*
 * FP64 CPU oracle for cosine mean-shift driven by the online seed
 * optimisation policy (OSOP) of "Faster Mean-shift" (Zhao et al.).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path
 * (libms) never calls it and shares no code, header or table with it.
 *
 * Conventions: row-major arrays, caller-owned buffers, FP64 arithmetic,
 * dimensions 1..OR_MAX_DIM. Return codes: 0 ok, OR_EINVAL bad argument,
 * OR_ENOMEM allocation failure, OR_ECAP an output capacity is too small.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_DIM 256
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ECAP (-3)

typedef struct or_config {
    int32_t dim;          /* embedding dimension d */
    double bandwidth_cos; /* c = 1 - h; window is cos >= c (Eq. 9, Eq. 11) */
    double tol;           /* convergence: ||x' - x||_2 < tol (Sec. 3.2.1) */
    int32_t max_iter;     /* guard on iterations per round */
    double gamma;         /* early stop: round ends when #conv > gamma * N (Sec. 3.2.3) */
    int32_t n_initial;    /* N_initial (Sec. 3.2.4) */
    double L, H;          /* N schedule bounds (Eq. 21, Sec. 3.2.4) */
    double P_target;      /* P in Eq. 19 */
    double alpha;         /* Eq. 20; used only when L <= 0 (then L = alpha / gamma) */
    double merge_cos;     /* modes with cos >= merge_cos are merged */
    uint64_t seed;        /* seed-order permutation: b = SplitMix64(seed ^ frame_id) mod n */
    uint64_t frame_id;
    int32_t max_rounds;   /* guard on OSOP rounds */
    int32_t all_seeds;    /* 1: Algorithm 1, every pixel seeds one round, gamma forced to 1 */
} or_config;

typedef struct or_stats {
    int32_t rounds;
    int32_t n_modes;
    int32_t iters_total;      /* sum over rounds of iterations run */
    int32_t pad_;
    int64_t seeds;            /* seeds drawn */
    int64_t seed_iters;       /* seed-iterations (one seed shifted once) */
    int64_t candidates;       /* converged seeds offered to the merge */
    int64_t dropped;          /* seeds that did not converge before the round ended */
    double min_window_margin; /* min |cos - c| over every window decision */
    double min_cover_margin;  /* min |max_k cos - c| over every coverage decision */
    double min_merge_margin;  /* min |max_kept cos - merge_cos| over every merge decision */
    int64_t n_carry;          /* seed count carried to the next frame of a video (Sec. 3.2.4,
                                 Sec. 4.3 / Table 3): the Eq. 19-21 updates from n_initial over
                                 the frame's rounds without the clamp to the frame's uncovered
                                 count, bounded by the largest batch the frame drew */
} or_stats;

/* SplitMix64 (Steele, Lea, Flood 2014): advance *state and return the output. */
uint64_t or_splitmix64_next(uint64_t* state);

/* Seed order: pi(j) = (b + a*j) mod n, a the integer in [1, n-1] coprime to n
 * nearest round(0.6180339887 n) (lower candidate first on a tie), and
 * b = SplitMix64(seed ^ frame_id) mod n. n = 1 gives a = 1, b = 0. */
void or_perm_params(int64_t n, uint64_t seed, uint64_t frame_id, int64_t* a, int64_t* b);
int64_t or_perm_at(int64_t j, int64_t n, int64_t a, int64_t b);

/* Compact the foreground (mask != 0, or every pixel when mask is NULL) in
 * row-major order and normalise each vector to unit length in FP64.
 * p_out [n_pixels*dim], pnorm_out [n_pixels] (norm of the normalised vector),
 * idx_out [n_pixels]. Returns the foreground count, or OR_EINVAL when a
 * foreground vector has zero or non-finite norm. */
int64_t or_normalize(const float* emb, const uint8_t* mask, int64_t n_pixels, int32_t dim,
                     double* p_out, double* pnorm_out, int64_t* idx_out);

/* Cosine similarity, Eq. 1. */
double or_cos(const double* a, double an, const double* b, double bn, int32_t dim);

/* One mean-shift update with the flat kernel (Eq. 6-8, Eq. 11):
 * x_new = normalise(sum of p_i with cos(x, p_i) >= c). Returns |W(x)|; on an
 * empty window x_new is left untouched. min_margin (nullable) is lowered to
 * the smallest |cos - c| seen. */
int64_t or_shift_step(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                      const double* x, double* x_new, double* min_margin);

/* Iterate one seed until ||x' - x|| < tol or max_iter steps. traj gets
 * x_0..x_T ((max_iter+1)*dim), counts gets |W(x_t)| for t < T. Returns T,
 * or -T when the window emptied at step T. */
int32_t or_trajectory(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                      double tol, int32_t max_iter, const double* x0, double* traj,
                      int64_t* counts);

/* Shift a batch of m seeds in lockstep (the shift loop of Algorithm 2) with early
 * stopping: after each sweep, stop when #converged > gamma*m or no seed is
 * still moving. X [m*dim] in/out; state[s] = 1 converged, 2 empty window,
 * 0 still moving (dropped); support[s] = window size of the last update;
 * conv_iter[s] = sweep of convergence. Returns the sweeps run. */
int32_t or_shift_round(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                       double tol, int32_t max_iter, double gamma, double* X, int32_t m,
                       uint8_t* state, int64_t* support, int32_t* conv_iter,
                       int64_t* seed_iters, double* min_margin);

/* Prune and merge (the prune/merge step of Algorithm 2): candidates taken in order of
 * support (descending) then seed order (ascending); each is kept when its
 * cosine to every mode kept so far (kept[0..n_kept) and those kept in this
 * call) is < merge_cos. Kept modes are appended to kept (capacity cap) and
 * kept_src gets the candidate index of each new mode. Returns the new count,
 * or OR_ECAP. */
int32_t or_merge(const double* cand, const int64_t* support, const int64_t* order, int32_t k,
                 int32_t dim, double merge_cos, double* kept, int32_t n_kept, int32_t cap,
                 int32_t* kept_src, double* min_margin);

/* Coverage: an uncovered pixel becomes covered when max over modes
 * [k0, k1) of cos(p_i, m) >= c. Returns the number still uncovered. */
int64_t or_cover(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                 const double* modes, int32_t k0, int32_t k1, uint8_t* covered,
                 double* min_margin);

/* Eq. 19: N_min = ln(1 - e^(ln P / I)) / ln(1 - r/I). */
double or_nmin(double I, double r, double P);
/* Eq. 14: probability that each of I equal clusters receives a seed. */
double or_p_all_seeded(double N, double I, double r);
/* N schedule (Sec. 3.2.4): with N_min from Eq. 19, double N when
 * N < L*N_min, else N <- N - ceil(N_min) when N > H*N_min; I <= 0 keeps N.
 * The result is clamped to [1, max(1, uncovered)]. */
int64_t or_next_n(int64_t N, int64_t I, double r, double P, double L, double H,
                  int64_t uncovered);

/* Cluster every vector by its distance to the modes (the
 * labelling step of Algorithm 2): label = argmax_k cos(p_i, m_k), lowest k on ties; background -1.
 * labels [n_pixels]; margin (nullable) [n] = top1 - top2 (+inf for K = 1). */
void or_label(const double* P, const double* pn, const int64_t* idx, int64_t n, int32_t dim,
              const double* modes, int32_t K, int64_t n_pixels, int32_t* labels,
              double* margin);

/* Whole method on one frame: normalise, OSOP rounds (seed, shift, merge,
 * cover, schedule) until every foreground pixel is covered, then label.
 * modes_out [mode_cap*dim]; mode_support (nullable) [mode_cap];
 * label_margin (nullable) [n_pixels] indexed like labels (NaN on
 * background); round_log (nullable) [4*max_rounds]: per round the N
 * requested, seeds drawn, modes kept after it and pixels left uncovered.
 * seed_log (nullable) [n_pixels]: foreground index of every seed in draw
 * order. */
int32_t or_run(const or_config* cfg, const float* emb, const uint8_t* mask, int64_t n_pixels,
               int32_t* labels, double* modes_out, int32_t mode_cap, int32_t* n_modes_out,
               int64_t* mode_support, double* label_margin, int64_t* round_log,
               int64_t* seed_log, or_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
