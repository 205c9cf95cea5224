/*
 * FP64 CPU oracle for cosine mean-shift with the online seed optimisation
 * policy (OSOP), "Faster Mean-shift" (Zhao et al., arXiv 2007.14283).
 *
 * TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library against the
 * paper. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does.
 *
 * It is deliberately plain: every dot product runs k = 0..d-1 in order, every
 * window is a scan over all pixels in index order, and nothing is blocked,
 * fused or reordered. OpenMP (when available) only spreads independent seeds
 * or pixels over cores; each one's arithmetic is the same sequence. The build
 * uses -ffp-contract=off so results do not depend on FMA contraction.
 *
 * Readings of the paper taken here (the paper leaves them open):
 *  - Pixels are normalised once in FP64; the window compares cos >= c with
 *    c = 1 - h, the inclusive boundary of Eq. 11.
 *  - The update is the sample mean of Eq. 8 over the window, renormalised to
 *    the unit sphere (Eq. 10 as printed sums distances, which cannot give a
 *    vector; the renormalisation does not change any cosine).
 *  - Seeds are taken in a fixed affine permutation of the foreground, the
 *    next N uncovered positions per round; merge keeps modes in order of
 *    support then seed order with threshold merge_cos; a pixel is covered
 *    once seeded or once within c of a kept mode.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

uint64_t or_splitmix64_next(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b != 0) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

void or_perm_params(int64_t n, uint64_t seed, uint64_t frame_id, int64_t* a, int64_t* b) {
    if (n <= 1) {
        *a = 1;
        *b = 0;
        return;
    }
    int64_t a0 = (int64_t)floor(0.6180339887 * (double)n + 0.5);
    int64_t pick = 1;
    for (int64_t k = 0; k <= n; ++k) {
        int64_t lo = a0 - k, hi = a0 + k;
        if (lo >= 1 && lo <= n - 1 && gcd64(lo, n) == 1) { pick = lo; break; }
        if (hi >= 1 && hi <= n - 1 && gcd64(hi, n) == 1) { pick = hi; break; }
    }
    uint64_t st = seed ^ frame_id;
    *a = pick;
    *b = (int64_t)(or_splitmix64_next(&st) % (uint64_t)n);
}

int64_t or_perm_at(int64_t j, int64_t n, int64_t a, int64_t b) {
    uint64_t aj = ((uint64_t)a * (uint64_t)j) % (uint64_t)n;
    return (int64_t)((aj + (uint64_t)b) % (uint64_t)n);
}

static double dot(const double* a, const double* b, int32_t d) {
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) s += a[k] * b[k];
    return s;
}

static double norm2(const double* a, int32_t d) { return sqrt(dot(a, a, d)); }

double or_cos(const double* a, double an, const double* b, double bn, int32_t dim) {
    return dot(a, b, dim) / (an * bn);
}

int64_t or_normalize(const float* emb, const uint8_t* mask, int64_t n_pixels, int32_t dim,
                     double* p_out, double* pnorm_out, int64_t* idx_out) {
    if (dim < 1 || dim > OR_MAX_DIM || n_pixels < 0) return OR_EINVAL;
    int64_t n = 0;
    for (int64_t i = 0; i < n_pixels; ++i) {
        if (mask != NULL && mask[i] == 0) continue;
        const float* e = emb + i * dim;
        double s = 0.0;
        for (int32_t k = 0; k < dim; ++k) s += (double)e[k] * (double)e[k];
        double nrm = sqrt(s);
        if (!(nrm > 0.0) || !isfinite(nrm)) return OR_EINVAL;
        double* p = p_out + n * dim;
        for (int32_t k = 0; k < dim; ++k) p[k] = (double)e[k] / nrm;
        pnorm_out[n] = norm2(p, dim);
        idx_out[n] = i;
        ++n;
    }
    return n;
}

int64_t or_shift_step(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                      const double* x, double* x_new, double* min_margin) {
    double y[OR_MAX_DIM];
    for (int32_t k = 0; k < dim; ++k) y[k] = 0.0;
    double xn = norm2(x, dim);
    int64_t cnt = 0;
    double mm = min_margin ? *min_margin : 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double* p = P + i * dim;
        double cs = or_cos(x, xn, p, pn[i], dim);
        if (min_margin) {
            double m = fabs(cs - c);
            if (m < mm) mm = m;
        }
        if (cs >= c) {
            for (int32_t k = 0; k < dim; ++k) y[k] += p[k];
            ++cnt;
        }
    }
    if (min_margin) *min_margin = mm;
    if (cnt == 0) return 0;
    double yn = norm2(y, dim);
    for (int32_t k = 0; k < dim; ++k) x_new[k] = y[k] / yn;
    return cnt;
}

static double dist2(const double* a, const double* b, int32_t d) {
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        s += t * t;
    }
    return sqrt(s);
}

int32_t or_trajectory(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                      double tol, int32_t max_iter, const double* x0, double* traj,
                      int64_t* counts) {
    memcpy(traj, x0, sizeof(double) * (size_t)dim);
    for (int32_t t = 0; t < max_iter; ++t) {
        const double* x = traj + (int64_t)t * dim;
        double* xn = traj + (int64_t)(t + 1) * dim;
        int64_t cnt = or_shift_step(P, pn, n, dim, c, x, xn, NULL);
        counts[t] = cnt;
        if (cnt == 0) return -(t + 1);
        if (dist2(xn, x, dim) < tol) return t + 1;
    }
    return max_iter;
}

int32_t or_shift_round(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                       double tol, int32_t max_iter, double gamma, double* X, int32_t m,
                       uint8_t* state, int64_t* support, int32_t* conv_iter,
                       int64_t* seed_iters, double* min_margin) {
    for (int32_t s = 0; s < m; ++s) {
        state[s] = 0;
        support[s] = 0;
        conv_iter[s] = 0;
    }
    double mm = min_margin ? *min_margin : INFINITY;
    int64_t si = 0;
    int32_t sweeps = 0;
    for (int32_t t = 1; t <= max_iter; ++t) {
        sweeps = t;
        int64_t active = 0;
        for (int32_t s = 0; s < m; ++s) active += (state[s] == 0);
        si += active;
#pragma omp parallel for schedule(dynamic, 4) reduction(min : mm)
        for (int32_t s = 0; s < m; ++s) {
            if (state[s] != 0) continue;
            double* x = X + (int64_t)s * dim;
            double xn[OR_MAX_DIM];
            double local = INFINITY;
            int64_t cnt = or_shift_step(P, pn, n, dim, c, x, xn, &local);
            if (local < mm) mm = local;
            if (cnt == 0) {
                state[s] = 2;
                continue;
            }
            double delta = dist2(xn, x, dim);
            memcpy(x, xn, sizeof(double) * (size_t)dim);
            support[s] = cnt;
            if (delta < tol) {
                state[s] = 1;
                conv_iter[s] = t;
            }
        }
        int64_t nconv = 0, nmove = 0;
        for (int32_t s = 0; s < m; ++s) {
            nconv += (state[s] == 1);
            nmove += (state[s] == 0);
        }
        if ((double)nconv > gamma * (double)m || nmove == 0) break;
    }
    if (seed_iters) *seed_iters += si;
    if (min_margin) *min_margin = mm;
    return sweeps;
}

typedef struct {
    int64_t support;
    int64_t order;
    int32_t idx;
} cand_key;

static int cand_cmp(const void* pa, const void* pb) {
    const cand_key* a = (const cand_key*)pa;
    const cand_key* b = (const cand_key*)pb;
    if (a->support != b->support) return a->support > b->support ? -1 : 1;
    if (a->order != b->order) return a->order < b->order ? -1 : 1;
    return 0;
}

int32_t or_merge(const double* cand, const int64_t* support, const int64_t* order, int32_t k,
                 int32_t dim, double merge_cos, double* kept, int32_t n_kept, int32_t cap,
                 int32_t* kept_src, double* min_margin) {
    if (k <= 0) return n_kept;
    cand_key* keys = (cand_key*)malloc(sizeof(cand_key) * (size_t)k);
    if (!keys) return OR_ENOMEM;
    for (int32_t a = 0; a < k; ++a) {
        keys[a].support = support[a];
        keys[a].order = order[a];
        keys[a].idx = a;
    }
    qsort(keys, (size_t)k, sizeof(cand_key), cand_cmp);
    int32_t n0 = n_kept;
    double mm = min_margin ? *min_margin : INFINITY;
    for (int32_t r = 0; r < k; ++r) {
        const double* m = cand + (int64_t)keys[r].idx * dim;
        double mn = norm2(m, dim);
        double best = -INFINITY;
        for (int32_t j = 0; j < n_kept; ++j) {
            const double* q = kept + (int64_t)j * dim;
            double cs = or_cos(m, mn, q, norm2(q, dim), dim);
            if (cs > best) best = cs;
        }
        if (n_kept > 0) {
            double marg = fabs(best - merge_cos);
            if (marg < mm) mm = marg;
        }
        if (n_kept == 0 || best < merge_cos) {
            if (n_kept >= cap) {
                free(keys);
                return OR_ECAP;
            }
            memcpy(kept + (int64_t)n_kept * dim, m, sizeof(double) * (size_t)dim);
            if (kept_src) kept_src[n_kept - n0] = keys[r].idx;
            ++n_kept;
        }
    }
    if (min_margin) *min_margin = mm;
    free(keys);
    return n_kept;
}

int64_t or_cover(const double* P, const double* pn, int64_t n, int32_t dim, double c,
                 const double* modes, int32_t k0, int32_t k1, uint8_t* covered,
                 double* min_margin) {
    double mm = min_margin ? *min_margin : INFINITY;
    int64_t left = 0;
#pragma omp parallel for schedule(static) reduction(min : mm) reduction(+ : left)
    for (int64_t i = 0; i < n; ++i) {
        if (covered[i]) continue;
        if (k1 > k0) {
            const double* p = P + i * dim;
            double best = -INFINITY;
            for (int32_t k = k0; k < k1; ++k) {
                const double* q = modes + (int64_t)k * dim;
                double cs = or_cos(p, pn[i], q, norm2(q, dim), dim);
                if (cs > best) best = cs;
            }
            double marg = fabs(best - c);
            if (marg < mm) mm = marg;
            if (best >= c) {
                covered[i] = 1;
                continue;
            }
        }
        ++left;
    }
    if (min_margin) *min_margin = mm;
    return left;
}

double or_nmin(double I, double r, double P) { return log(1.0 - exp(log(P) / I)) / log(1.0 - r / I); }

double or_p_all_seeded(double N, double I, double r) { return pow(1.0 - pow(1.0 - r / I, N), I); }

int64_t or_next_n(int64_t N, int64_t I, double r, double P, double L, double H,
                  int64_t uncovered) {
    int64_t nn = N;
    if (I > 0) {
        double nmin = or_nmin((double)I, r, P);
        if ((double)N < L * nmin)
            nn = 2 * N;
        else if ((double)N > H * nmin)
            nn = N - (int64_t)ceil(nmin);
    }
    int64_t hi = uncovered > 1 ? uncovered : 1;
    if (nn > hi) nn = hi;
    if (nn < 1) nn = 1;
    return nn;
}

void or_label(const double* P, const double* pn, const int64_t* idx, int64_t n, int32_t dim,
              const double* modes, int32_t K, int64_t n_pixels, int32_t* labels,
              double* margin) {
    for (int64_t i = 0; i < n_pixels; ++i) labels[i] = -1;
    double* mnorm = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    for (int32_t k = 0; k < K; ++k) mnorm[k] = norm2(modes + (int64_t)k * dim, dim);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double* p = P + i * dim;
        int32_t best = -1;
        double b1 = -INFINITY, b2 = -INFINITY;
        for (int32_t k = 0; k < K; ++k) {
            double cs = or_cos(p, pn[i], modes + (int64_t)k * dim, mnorm[k], dim);
            if (cs > b1) {
                b2 = b1;
                b1 = cs;
                best = k;
            } else if (cs > b2) {
                b2 = cs;
            }
        }
        labels[idx[i]] = best;
        if (margin) margin[i] = b1 - b2;
    }
    free(mnorm);
}

int32_t or_run(const or_config* cfg, const float* emb, const uint8_t* mask, int64_t n_pixels,
               int32_t* labels, double* modes_out, int32_t mode_cap, int32_t* n_modes_out,
               int64_t* mode_support, double* label_margin, int64_t* round_log,
               int64_t* seed_log, or_stats* stats) {
    const int32_t d = cfg->dim;
    if (d < 1 || d > OR_MAX_DIM || n_pixels < 0 || n_pixels > INT32_MAX || cfg->max_iter < 1 ||
        cfg->n_initial < 1 || cfg->max_rounds < 1 || !(cfg->tol > 0.0) || mode_cap < 0)
        return OR_EINVAL;
    or_stats st;
    memset(&st, 0, sizeof(st));
    st.min_window_margin = INFINITY;
    st.min_cover_margin = INFINITY;
    st.min_merge_margin = INFINITY;
    const double c = cfg->bandwidth_cos;
    const double gamma = cfg->all_seeds ? 1.0 : cfg->gamma;
    const double L = cfg->L > 0.0 ? cfg->L : cfg->alpha / gamma;

    double* P = (double*)malloc(sizeof(double) * (size_t)(n_pixels * d + 1));
    double* pn = (double*)malloc(sizeof(double) * (size_t)(n_pixels + 1));
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    uint8_t* covered = (uint8_t*)calloc((size_t)(n_pixels + 1), 1);
    double* X = (double*)malloc(sizeof(double) * (size_t)(n_pixels * d + 1));
    int64_t* seed_pix = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    int64_t* seed_order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    uint8_t* sstate = (uint8_t*)malloc((size_t)(n_pixels + 1));
    int64_t* support = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    int32_t* conv_iter = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_pixels + 1));
    double* cand = (double*)malloc(sizeof(double) * (size_t)(n_pixels * d + 1));
    int64_t* csup = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    int64_t* cord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    int32_t* ksrc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_pixels + 1));
    double* kept = (double*)malloc(sizeof(double) * (size_t)(n_pixels * d + 1));
    int64_t* ksup = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_pixels + 1));
    double* lmargin = (double*)malloc(sizeof(double) * (size_t)(n_pixels + 1));
    int32_t rc = 0;
    if (!P || !pn || !idx || !covered || !X || !seed_pix || !seed_order || !sstate || !support ||
        !conv_iter || !cand || !csup || !cord || !ksrc || !kept || !ksup || !lmargin) {
        rc = OR_ENOMEM;
        goto done;
    }
    int64_t n = or_normalize(emb, mask, n_pixels, d, P, pn, idx);
    if (n < 0) {
        rc = (int32_t)n;
        goto done;
    }
    int64_t a = 1, b = 0;
    or_perm_params(n, cfg->seed, cfg->frame_id, &a, &b);
    int64_t cursor = 0, uncovered = n, N = cfg->n_initial, drawn = 0;
    int32_t n_kept = 0;
    int64_t n_free = N, max_draw = 0;
    st.n_carry = N;
    while (uncovered > 0 && st.rounds < cfg->max_rounds) {
        int64_t want = cfg->all_seeds ? n : N;
        if (want > uncovered) want = uncovered;
        /* Seed selection (the seed-selection step of Algorithm 2): next uncovered positions. */
        int32_t m = 0;
        while (m < want && cursor < n) {
            int64_t i = or_perm_at(cursor, n, a, b);
            ++cursor;
            if (covered[i]) continue;
            covered[i] = 1;
            seed_pix[m] = i;
            if (seed_log) seed_log[drawn] = i;
            seed_order[m] = drawn++;
            memcpy(X + (int64_t)m * d, P + i * d, sizeof(double) * (size_t)d);
            ++m;
        }
        if (m == 0) break;
        st.seeds += m;
        int32_t sweeps = or_shift_round(P, pn, n, d, c, cfg->tol, cfg->max_iter, gamma, X, m,
                                        sstate, support, conv_iter, &st.seed_iters,
                                        &st.min_window_margin);
        st.iters_total += sweeps;
        int32_t k = 0;
        for (int32_t s = 0; s < m; ++s) {
            if (sstate[s] != 1) {
                st.dropped += 1;
                continue;
            }
            memcpy(cand + (int64_t)k * d, X + (int64_t)s * d, sizeof(double) * (size_t)d);
            csup[k] = support[s];
            cord[k] = seed_order[s];
            ++k;
        }
        st.candidates += k;
        int32_t k0 = n_kept;
        int32_t nk = or_merge(cand, csup, cord, k, d, cfg->merge_cos, kept, n_kept, (int32_t)n,
                              ksrc, &st.min_merge_margin);
        if (nk < 0) {
            rc = nk;
            goto done;
        }
        for (int32_t j = k0; j < nk; ++j) ksup[j] = csup[ksrc[j - k0]];
        n_kept = nk;
        uncovered = or_cover(P, pn, n, d, c, kept, k0, n_kept, covered, &st.min_cover_margin);
        if (round_log) {
            round_log[4 * st.rounds + 0] = want;
            round_log[4 * st.rounds + 1] = m;
            round_log[4 * st.rounds + 2] = n_kept;
            round_log[4 * st.rounds + 3] = uncovered;
        }
        st.rounds += 1;
        /* A video carries N into its next frame (Sec. 3.2.4; Sec. 4.3, Table 3).
           The carried value follows the same Eq. 19-21 updates from n_initial
           without the clamp to this frame's uncovered pixels (which only
           bounds the draws at the frame's end), and is bounded by the largest
           batch the frame actually drew: no frame can use more seeds than it
           has uncovered pixels. */
        if (m > max_draw) max_draw = m;
        n_free = or_next_n(n_free, n_kept, 1.0, cfg->P_target, L, cfg->H, INT64_MAX);
        st.n_carry = n_free < max_draw ? n_free : max_draw;
        N = or_next_n(N, n_kept, 1.0, cfg->P_target, L, cfg->H, uncovered);
    }
    if (n_kept > mode_cap) {
        rc = OR_ECAP;
        goto done;
    }
    or_label(P, pn, idx, n, d, kept, n_kept, n_pixels, labels, lmargin);
    if (label_margin) {
        for (int64_t i = 0; i < n_pixels; ++i) label_margin[i] = NAN;
        for (int64_t i = 0; i < n; ++i) label_margin[idx[i]] = lmargin[i];
    }
    memcpy(modes_out, kept, sizeof(double) * (size_t)n_kept * (size_t)d);
    if (mode_support) memcpy(mode_support, ksup, sizeof(int64_t) * (size_t)n_kept);
    *n_modes_out = n_kept;
    st.n_modes = n_kept;
done:
    if (stats) *stats = st;
    free(P); free(pn); free(idx); free(covered); free(X); free(seed_pix); free(seed_order);
    free(sstate); free(support); free(conv_iter); free(cand); free(csup); free(cord);
    free(ksrc); free(kept); free(ksup); free(lmargin);
    return rc;
}
