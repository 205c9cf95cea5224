// C ABI of libms: context lifetime, workspace, OSOP round control.
//
// Host control follows Sec. 3.2.4: N starts at N_initial; after every round
// N_min is recomputed from the kept-mode count I by Eq. 19 (r = 1: seeds are
// drawn from the foreground only); N doubles while N < L*N_min and shrinks by
// N_min when N > H*N_min. The GPU does all per-pixel and per-seed work; the
// host reads back a few counters per call.
#include <atomic>
#include <stdint.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "ms_internal.cuh"

#include <mutex>

namespace ms {

static thread_local char g_err[512] = "";

ms_status set_error(ms_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

static std::atomic<int32_t> g_fail_allocs{0};

cudaError_t workspace_malloc(void** p, size_t bytes) {
    int32_t left = g_fail_allocs.load();
    while (left > 0 && !g_fail_allocs.compare_exchange_weak(left, left - 1)) {
    }
    if (left > 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// The library's own stream-ordered pool on each device. It keeps freed memory
// mapped (release threshold: never), so calls that allocate a workspace per
// call and synchronise do not re-map it each time; the process's default
// pool is left as the caller configured it.
cudaError_t scratch_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&pools[dev], &props)) != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

ms_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MS_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(MS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(MS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).
uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

int64_t gcd(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Seed order pi(j) = (b + a j) mod n with a coprime to n, closest to
// round(0.6180339887 n) (the smaller of two equally close), b from SplitMix64.
void seed_order_params(int64_t n, uint64_t seed, uint64_t frame_id, int64_t* a, int64_t* b) {
    if (n <= 1) {
        *a = 1;
        *b = 0;
        return;
    }
    const int64_t centre = (int64_t)floor(0.6180339887 * (double)n + 0.5);
    int64_t pick = 1;
    for (int64_t off = 0; off <= n; ++off) {
        const int64_t lo = centre - off;
        if (lo >= 1 && lo < n && gcd(lo, n) == 1) {
            pick = lo;
            break;
        }
        const int64_t hi = centre + off;
        if (hi >= 1 && hi < n && gcd(hi, n) == 1) {
            pick = hi;
            break;
        }
    }
    *a = pick;
    *b = (int64_t)(splitmix64(seed ^ frame_id) % (uint64_t)n);
}

// Eq. 19: smallest N for which every one of I clusters holds a seed with
// probability P, for a cluster share r/I.
double eq19_nmin(double I, double r, double P) {
    return log(1.0 - exp(log(P) / I)) / log(1.0 - r / I);
}

int64_t schedule_next(int64_t N, int64_t I, double P, double L, double H, int64_t uncovered) {
    int64_t next = N;
    if (I > 0) {
        const double nmin = eq19_nmin((double)I, 1.0, P);
        if ((double)N < L * nmin)
            next = 2 * N;
        else if ((double)N > H * nmin)
            next = N - (int64_t)ceil(nmin);
    }
    const int64_t cap = uncovered > 1 ? uncovered : 1;
    if (next > cap) next = cap;
    if (next < 1) next = 1;
    return next;
}

ms_status validate(const ms_config* c) {
    if (!c) return set_error(MS_ERR_INVALID_ARG, "config is NULL");
    if (c->dim < 1 || c->dim > MS_MAX_DIM) return set_error(MS_ERR_INVALID_ARG, "dim %d not in 1..%d", c->dim, MS_MAX_DIM);
    if (c->kernel != MS_FLAT) return set_error(MS_ERR_INVALID_ARG, "ms_create supports the flat kernel only");
    if (!(c->bandwidth_cos > -1.0 && c->bandwidth_cos <= 1.0)) return set_error(MS_ERR_INVALID_ARG, "bandwidth_cos must be in (-1, 1]");
    if (!(c->merge_cos > -1.0 && c->merge_cos <= 1.0)) return set_error(MS_ERR_INVALID_ARG, "merge_cos must be in (-1, 1]");
    if (!(c->tol > 0.0)) return set_error(MS_ERR_INVALID_ARG, "tol must be > 0");
    if (c->max_iter < 1) return set_error(MS_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (c->n_initial < 1) return set_error(MS_ERR_INVALID_ARG, "n_initial must be >= 1");
    if (!(c->gamma >= 0.0 && c->gamma <= 1.0)) return set_error(MS_ERR_INVALID_ARG, "gamma must be in [0, 1]");
    if (!(c->P_target > 0.0 && c->P_target < 1.0)) return set_error(MS_ERR_INVALID_ARG, "P_target must be in (0, 1)");
    if (!(c->H >= 0.0)) return set_error(MS_ERR_INVALID_ARG, "H must be >= 0");
    if (c->L <= 0.0 && !(c->alpha > 0.0)) return set_error(MS_ERR_INVALID_ARG, "L <= 0 needs alpha > 0");
    if (c->precision != MS_FP32 && c->precision != MS_BF16) return set_error(MS_ERR_INVALID_ARG, "unknown precision");
    if (c->max_rounds < 1) return set_error(MS_ERR_INVALID_ARG, "max_rounds must be >= 1");
    if (c->batch_max_passes < 0) return set_error(MS_ERR_INVALID_ARG, "batch_max_passes must be >= 0");
    if (c->tc_shape < 0 || c->tc_shape >= kTcShapes) return set_error(MS_ERR_INVALID_ARG, "unknown tc_shape");
    return MS_OK;
}

constexpr size_t kAlign = 256;

struct Layout {
    size_t off[29];
    size_t total;

};

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

Layout plan(int64_t np, int Dp, bool bf16) {
    Layout L;
    const size_t n = (size_t)(np > 0 ? np : 1);
    const size_t sizes[] = {
        n * Dp * sizeof(float),           // 0 P32
        n * sizeof(int32_t),              // 1 pix
        n,                                // 2 covered
        n * Dp * sizeof(float),           // 3 X
        n * sizeof(int32_t),              // 4 seed_pix
        n * sizeof(int32_t),              // 5 seed_order
        n,                                // 6 sstate
        n * sizeof(int32_t),              // 7 support
        n * sizeof(int32_t),              // 8 active0
        n * sizeof(int32_t),              // 9 active1
        n * sizeof(int32_t),              // 10 seed_log
        n * (Dp + 1) * sizeof(unsigned long long),  // 11 acc
        n * Dp * sizeof(float),           // 12 modes
        n * sizeof(int32_t),              // 13 mode_support
        n * sizeof(int32_t),              // 14 cand
        n * sizeof(int32_t),              // 15 cand_rank
        n * sizeof(int32_t),              // 16 rank_cand
        n,                                // 17 cand_state
        n * sizeof(int32_t),              // 18 conf_deg
        n * kMergeCap * sizeof(int32_t),  // 19 conf
        ((n + 1023) / 1024 + 1) * sizeof(int32_t),  // 20 block_tmp
        sizeof(DevCounters),              // 21 dc
        bf16 ? (n + 127) / 128 * 128 * 128 * (Dp / 16) : 0,  // 22 Pk (one array per 16 dimensions)
        bf16 ? (n + 127) / 128 * 128 * 128 * (Dp / 16) : 0,  // 23 Mk (labelling on the tensor cores)
        bf16 ? n * sizeof(int2) + 16 : 0,                     // 24 label_fix + count
        bf16 ? n * Dp * sizeof(float) : 0,                    // 25 Xr (merge candidates in rank order)
        bf16 ? n : 0,                                         // 26 removed_r
        bf16 ? (n + 127) / 128 * 128 * 128 * (Dp / 16) : 0,  // 27 Ck (their BF16 split rows)
    };
    size_t t = 0;
    for (int i = 0; i < 28; ++i) {
        L.off[i] = t;
        t += align_up(sizes[i]);
    }
    L.total = t;
    return L;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

ms_status readback(ms_ctx* ctx) {
    MS_CUDA(cudaMemcpyAsync(ctx->hc, ctx->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, ctx->stream));
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    return MS_OK;
}

void free_ctx(ms_ctx* ctx) {
    if (!ctx) return;
    for (int i = 0; i < 64; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->hc) cudaFreeHost(ctx->hc);
    delete[] ctx->round_log;
    delete ctx;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" void ms_inject_alloc_failure(int32_t count) { g_fail_allocs.store(count > 0 ? count : 0); }

extern "C" {

void ms_config_default(ms_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->dim = 16;
    c->kernel = MS_FLAT;
    c->bandwidth_cos = 0.9;
    c->kappa = 20.0;
    c->tol = 1e-6;
    c->max_iter = 300;
    c->n_initial = 128;
    c->gamma = 0.9;
    c->L = 2.0;
    c->H = 8.0;
    c->P_target = 0.99;
    c->alpha = 1.0;
    c->merge_cos = 0.9;
    c->seed = 0;
    c->frame_id = 0;
    c->precision = MS_FP32;
    c->max_rounds = 1000000;
    c->eps_band = 0.0;
    c->all_seeds = 0;
}

const char* ms_last_error(void) { return g_err; }

ms_status ms_workspace_bytes(const ms_config* cfg, int64_t n_pixels, int64_t* bytes_out) {
    ms_status s = validate(cfg);
    if (s != MS_OK) return s;
    if (!bytes_out || n_pixels < 0 || n_pixels >= (1LL << 24))
        return set_error(MS_ERR_INVALID_ARG, "n_pixels must be in [0, 2^24)");
    *bytes_out = (int64_t)plan(n_pixels, padded_dim(cfg->dim), cfg->precision == MS_BF16).total;
    return MS_OK;
}

}  // extern "C"

namespace ms {

// Workspace for frames of up to max_pixels pixels; no frame bound yet.
ms_status ctx_alloc(const ms_config* cfg, int64_t max_pixels, cudaStream_t stream, ms_ctx** out) {
    *out = nullptr;
    ms_ctx* ctx = new (std::nothrow) ms_ctx();
    if (!ctx) return set_error(MS_ERR_OOM, "host allocation failed");
    ctx->cfg = *cfg;
    ctx->d = cfg->dim;
    ctx->Dp = padded_dim(cfg->dim);
    ctx->stream = stream;
    ctx->max_pixels = max_pixels;
    ctx->num_sms = device_sms();
    ctx->shift_grid = ctx->num_sms * shift_blocks_per_sm();
    ctx->target_items = 2 * ctx->shift_grid;
    const Layout L = plan(max_pixels, ctx->Dp, cfg->precision == MS_BF16);
    ctx->ws_bytes = L.total;
    cudaError_t e = workspace_malloc(&ctx->ws, L.total);
    if (e != cudaSuccess) {
        free_ctx(ctx);
        return cuda_check(e, "cudaMalloc(workspace)");
    }
    e = cudaMallocHost((void**)&ctx->hc, sizeof(DevCounters));
    if (e != cudaSuccess) {
        free_ctx(ctx);
        return cuda_check(e, "cudaMallocHost(counters)");
    }
    char* b = (char*)ctx->ws;
    ctx->P32 = (float*)(b + L.off[0]);
    ctx->pix = (int32_t*)(b + L.off[1]);
    ctx->covered = (uint8_t*)(b + L.off[2]);
    ctx->X = (float*)(b + L.off[3]);
    ctx->seed_pix = (int32_t*)(b + L.off[4]);
    ctx->seed_order = (int32_t*)(b + L.off[5]);
    ctx->sstate = (uint8_t*)(b + L.off[6]);
    ctx->support = (int32_t*)(b + L.off[7]);
    ctx->active[0] = (int32_t*)(b + L.off[8]);
    ctx->active[1] = (int32_t*)(b + L.off[9]);
    ctx->seed_log = (int32_t*)(b + L.off[10]);
    ctx->acc = (unsigned long long*)(b + L.off[11]);
    ctx->modes = (float*)(b + L.off[12]);
    ctx->mode_support = (int32_t*)(b + L.off[13]);
    ctx->cand = (int32_t*)(b + L.off[14]);
    ctx->cand_rank = (int32_t*)(b + L.off[15]);
    ctx->rank_cand = (int32_t*)(b + L.off[16]);
    ctx->cand_state = (uint8_t*)(b + L.off[17]);
    ctx->conf_deg = (int32_t*)(b + L.off[18]);
    ctx->conf = (int32_t*)(b + L.off[19]);
    ctx->block_tmp = (int32_t*)(b + L.off[20]);
    ctx->dc = (DevCounters*)(b + L.off[21]);
    ctx->Pk = cfg->precision == MS_BF16 ? (void*)(b + L.off[22]) : nullptr;
    ctx->Mk = cfg->precision == MS_BF16 ? (void*)(b + L.off[23]) : nullptr;
    ctx->label_fix = cfg->precision == MS_BF16 ? (int2*)(b + L.off[24]) : nullptr;
    ctx->Xr = cfg->precision == MS_BF16 ? (float*)(b + L.off[25]) : nullptr;
    ctx->removed_r = cfg->precision == MS_BF16 ? (uint8_t*)(b + L.off[26]) : nullptr;
    ctx->Ck = cfg->precision == MS_BF16 ? (void*)(b + L.off[27]) : nullptr;
    ctx->round_log_cap = 64;
    ctx->round_log = new (std::nothrow) int64_t[ctx->round_log_cap * 4];
    if (!ctx->round_log) {
        free_ctx(ctx);
        return set_error(MS_ERR_OOM, "host allocation failed");
    }
    *out = ctx;
    return MS_OK;
}

// Enqueue on `st` everything that binds a frame to the workspace and needs no
// host decision: clearing, foreground compaction and normalisation, and the
// BF16 split rows (sized on the device from the foreground count).
ms_status ctx_bind_async(ms_ctx* ctx, const float* d_emb, const uint8_t* d_mask, int64_t n_pixels,
                         cudaStream_t st) {
    ctx->emb = d_emb;
    ctx->mask = d_mask;
    ctx->n_pixels = n_pixels;
    const size_t nn = (size_t)(n_pixels > 0 ? n_pixels : 1);
    MS_CUDA(cudaMemsetAsync(ctx->covered, 0, nn, st));
    MS_CUDA(cudaMemsetAsync(ctx->dc, 0, sizeof(DevCounters), st));
    MS_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(unsigned long long) * (size_t)(ctx->Dp + 1) * nn, st));
    const cudaStream_t keep = ctx->stream;
    ctx->stream = st;
    ms_status s = launch_ingest(ctx);
    if (s == MS_OK && ctx->cfg.precision == MS_BF16) s = tc_pack_async(ctx);
    ctx->stream = keep;
    return s;
}

// Wait for the bind on `st`, check its inputs, and set the frame's host state:
// foreground count, seed order of frame_id, N starting at n_start.
ms_status ctx_bind_finish(ms_ctx* ctx, cudaStream_t st, uint64_t frame_id, int64_t n_start) {
    MS_CUDA(cudaMemcpyAsync(ctx->hc, ctx->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    if (ctx->hc->status != 0) return set_error(MS_ERR_INVALID_ARG, "a foreground embedding has zero or non-finite norm");
    ctx->cfg.frame_id = frame_id;
    ctx->n = ctx->hc->n_fg;
    ctx->uncovered = ctx->n;
    seed_order_params(ctx->n, ctx->cfg.seed, frame_id, &ctx->perm_a, &ctx->perm_b);
    ctx->n_pad = ctx->n > 0 ? (ctx->n + 127) / 128 * 128 : 0;
    if (ctx->cfg.precision == MS_BF16 && ctx->n > 0) {
        ms_status s = tc_finish(ctx);
        if (s != MS_OK) return s;
    }
    ctx->N = n_start;
    ctx->N_carry = n_start;
    ctx->max_draw = 0;
    ctx->phase = 0;
    ctx->n_kept = 0;
    ctx->m_round = 0;
    const int64_t launches = ctx->stats.launches;
    ctx->stats = ms_stats{};
    ctx->stats.launches = launches;
    ctx->stats.n_fg = ctx->n;
    ctx->stats.uncovered = ctx->n;
    ctx->stats.workspace_bytes = (int64_t)ctx->ws_bytes;
    return MS_OK;
}

void ctx_free(ms_ctx* ctx) { free_ctx(ctx); }

int64_t carried_n(const ms_ctx* ctx) {
    if (ctx->max_draw <= 0) return ctx->N_carry;
    return ctx->N_carry < ctx->max_draw ? ctx->N_carry : ctx->max_draw;
}

}  // namespace ms

extern "C" {

ms_status ms_create(const ms_config* cfg, const float* d_emb, const uint8_t* d_mask, int64_t n_pixels,
                    void* stream, ms_ctx** out) {
    g_err[0] = 0;
    if (!out) return set_error(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ms_status s = validate(cfg);
    if (s != MS_OK) return s;
    if (n_pixels < 0 || n_pixels >= (1LL << 24)) return set_error(MS_ERR_INVALID_ARG, "n_pixels must be in [0, 2^24)");
    if (n_pixels > 0 && !d_emb) return set_error(MS_ERR_INVALID_ARG, "d_emb is NULL");
    ms_ctx* ctx = nullptr;
    s = ctx_alloc(cfg, n_pixels, (cudaStream_t)stream, &ctx);
    if (s != MS_OK) return s;
    s = ctx_bind_async(ctx, d_emb, d_mask, n_pixels, ctx->stream);
    if (s == MS_OK) s = ctx_bind_finish(ctx, ctx->stream, cfg->frame_id, cfg->n_initial);
    if (s != MS_OK) {
        free_ctx(ctx);
        return s;
    }
    *out = ctx;
    return MS_OK;
}

ms_status ms_seed_batch(ms_ctx* ctx, int32_t n_requested, int32_t* n_seeded_out) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->phase != 0) return set_error(MS_ERR_STATE, "the previous seed batch was not merged");
    int64_t want = ctx->cfg.all_seeds ? ctx->n : (n_requested > 0 ? n_requested : ctx->N);
    if (want > ctx->uncovered) want = ctx->uncovered;
    if (want <= 0 || ctx->uncovered == 0) {
        if (n_seeded_out) *n_seeded_out = 0;
        return MS_OK;
    }
    ms_status s = launch_seed_select(ctx, (int32_t)want);
    if (s != MS_OK) return s;
    s = readback(ctx);
    if (s != MS_OK) return s;
    const int32_t m = ctx->hc->n_seeded;
    ctx->m_round = m;
    if (m > ctx->max_draw) ctx->max_draw = m;
    ctx->uncovered = ctx->hc->n_uncovered;
    ctx->stats.seeds += m;
    if ((int64_t)ctx->stats.rounds >= ctx->round_log_cap) {
        int64_t* nl = new (std::nothrow) int64_t[ctx->round_log_cap * 8];
        if (!nl) return set_error(MS_ERR_OOM, "host allocation failed");
        memcpy(nl, ctx->round_log, sizeof(int64_t) * 4 * ctx->round_log_cap);
        delete[] ctx->round_log;
        ctx->round_log = nl;
        ctx->round_log_cap *= 2;
    }
    int64_t* row = ctx->round_log + 4 * ctx->stats.rounds;
    row[0] = want;
    row[1] = m;
    row[2] = ctx->n_kept;
    row[3] = ctx->uncovered;
    if (m > 0) ctx->phase = 1;
    if (n_seeded_out) *n_seeded_out = m;
    return MS_OK;
}

ms_status ms_iterate(ms_ctx* ctx, int32_t max_iter, int32_t* n_converged_out, int32_t* n_iters_out) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->phase != 1) return set_error(MS_ERR_STATE, "no seed batch is pending");
    const int mi = max_iter > 0 ? max_iter : ctx->cfg.max_iter;
    const int64_t seed_iters0 = ctx->hc->seed_iters;
    int t = 0, batch = 4;
    for (;;) {
        const int iters_before = ctx->hc->iters;
        int launched = 0;
        for (int j = 0; j < batch && t < mi; ++j, ++t, ++launched) {
            cudaEvent_t e0 = ctx->prof ? ctx->ev[2 * j] : nullptr;
            cudaEvent_t e1 = ctx->prof ? ctx->ev[2 * j + 1] : nullptr;
            ms_status s = launch_shift_iteration(ctx, t, mi, e0, e1);
            if (s != MS_OK) return s;
        }
        ms_status s = readback(ctx);
        if (s != MS_OK) return s;
        if (ctx->prof) {
            // only launches that ran an iteration (the rest returned at once)
            const int real = ctx->hc->iters - iters_before;
            for (int j = 0; j < real && j < launched; ++j) {
                float ms_ = 0.f;
                MS_CUDA(cudaEventElapsedTime(&ms_, ctx->ev[2 * j], ctx->ev[2 * j + 1]));
                ctx->stats.shift_ms += ms_;
                ctx->stats.shift_launches += 1;
            }
        }
        if (ctx->hc->done || t >= mi) break;
        batch = batch < 32 ? batch * 2 : 32;
    }
    const DevCounters& h = *ctx->hc;
    ctx->phase = 2;
    ctx->stats.iters_total += h.iters;
    ctx->stats.seed_iters += h.seed_iters - seed_iters0;
    ctx->stats.dropped += (int64_t)h.m_round - h.conv_total;
    ctx->stats.candidates += h.conv_total;
    if (n_converged_out) *n_converged_out = h.conv_total;
    if (n_iters_out) *n_iters_out = h.iters;
    if (h.conv_total == 0) return set_error(MS_ERR_NOT_CONVERGED, "no seed of the batch converged");
    return MS_OK;
}

ms_status ms_merge_modes(ms_ctx* ctx, int32_t* n_modes_out, int64_t* n_uncovered_out) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->phase != 2) return set_error(MS_ERR_STATE, "ms_iterate has not run on the current batch");
    const int32_t k = ctx->hc->conv_total;
    const int32_t k0 = ctx->n_kept;
    ms_status s = launch_collect(ctx);
    if (s == MS_OK) s = launch_merge_prepare(ctx, k);
    if (s == MS_OK) s = launch_merge_resolve(ctx, k, 8);
    if (s == MS_OK) s = readback(ctx);
    for (int extra = 0; s == MS_OK && k > 0 && ctx->hc->undecided > 0 && extra < 7; ++extra) {
        s = launch_merge_resolve(ctx, k, 8);
        if (s == MS_OK) s = readback(ctx);
    }
    if (s == MS_OK && k > 0 && ctx->hc->undecided > 0) s = launch_merge_sequential(ctx, k);
    if (s == MS_OK) s = launch_merge_append(ctx, k);
    if (s == MS_OK) s = readback(ctx);
    if (s != MS_OK) return s;
    const int32_t k1 = ctx->hc->n_kept;
    s = launch_cover(ctx, k0, k1);
    if (s == MS_OK) s = readback(ctx);
    if (s != MS_OK) return s;
    ctx->n_kept = k1;
    ctx->uncovered = ctx->hc->n_uncovered;
    int64_t* row = ctx->round_log + 4 * ctx->stats.rounds;
    row[2] = ctx->n_kept;
    row[3] = ctx->uncovered;
    ctx->stats.rounds += 1;
    ctx->stats.n_modes = ctx->n_kept;
    ctx->stats.uncovered = ctx->uncovered;
    const double gamma = ctx->cfg.all_seeds ? 1.0 : ctx->cfg.gamma;
    const double L = ctx->cfg.L > 0.0 ? ctx->cfg.L : ctx->cfg.alpha / gamma;
    ctx->N = schedule_next(ctx->N, ctx->n_kept, ctx->cfg.P_target, L, ctx->cfg.H, ctx->uncovered);
    // the value a video carries into its next frame: the same updates without
    // the clamp to this frame's uncovered pixels, bounded (in ms_get_state) by
    // the largest batch the frame drew
    ctx->N_carry = schedule_next(ctx->N_carry, ctx->n_kept, ctx->cfg.P_target, L, ctx->cfg.H, INT64_MAX);
    ctx->phase = 0;
    if (n_modes_out) *n_modes_out = ctx->n_kept;
    if (n_uncovered_out) *n_uncovered_out = ctx->uncovered;
    return MS_OK;
}

ms_status ms_label(ms_ctx* ctx, int32_t* d_labels_out, float* d_modes_out, int32_t cap, int32_t* n_modes_out) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->phase != 0) return set_error(MS_ERR_STATE, "a seed batch is still pending");
    if (!d_labels_out && ctx->n_pixels > 0) return set_error(MS_ERR_INVALID_ARG, "d_labels_out is NULL");
    if (d_modes_out && cap < ctx->n_kept)
        return set_error(MS_ERR_INVALID_ARG, "cap %d < %d modes", cap, ctx->n_kept);
    if (ctx->n_pixels > 0) {
        ms_status s = launch_label(ctx, d_labels_out);
        if (s != MS_OK) return s;
    }
    if (d_modes_out && ctx->n_kept > 0)
        MS_CUDA(cudaMemcpy2DAsync(d_modes_out, sizeof(float) * ctx->d, ctx->modes, sizeof(float) * ctx->Dp,
                                  sizeof(float) * ctx->d, (size_t)ctx->n_kept, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    if (n_modes_out) *n_modes_out = ctx->n_kept;
    return MS_OK;
}

void ms_destroy(ms_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

ms_status ms_run(ms_ctx* ctx, int32_t* d_labels_out, float* d_modes_out, int32_t cap, int32_t* n_modes_out) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->phase != 0) return set_error(MS_ERR_STATE, "a seed batch is still pending");
    int rounds = 0;
    while (ctx->uncovered > 0 && rounds < ctx->cfg.max_rounds) {
        int32_t m = 0;
        ms_status s = ms_seed_batch(ctx, 0, &m);
        if (s != MS_OK) return s;
        if (m == 0) break;
        s = ms_iterate(ctx, 0, nullptr, nullptr);
        if (s != MS_OK && s != MS_ERR_NOT_CONVERGED) return s;
        s = ms_merge_modes(ctx, nullptr, nullptr);
        if (s != MS_OK) return s;
        ++rounds;
        if (ctx->cfg.all_seeds) break;
    }
    return ms_label(ctx, d_labels_out, d_modes_out, cap, n_modes_out);
}

ms_status ms_stats_get(const ms_ctx* ctx, ms_stats* out) {
    if (!ctx || !out) return set_error(MS_ERR_INVALID_ARG, "NULL argument");
    *out = ctx->stats;
    out->band_pairs = ctx->hc->band_pairs;
    out->launches = ctx->launches;
    return MS_OK;
}

ms_status ms_profile(ms_ctx* ctx, int32_t enable) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (enable && !ctx->ev[0])
        for (int i = 0; i < 64; ++i) MS_CUDA(cudaEventCreate(&ctx->ev[i]));
    ctx->prof = enable != 0;
    return MS_OK;
}

ms_status ms_run_host(const ms_config* cfg, const float* h_emb, const uint8_t* h_mask, int64_t n_pixels,
                      void* stream, int32_t* h_labels, float* h_modes, int32_t cap, int32_t* n_modes_out,
                      ms_stats* stats_out) {
    g_err[0] = 0;
    ms_status s = validate(cfg);
    if (s != MS_OK) return s;
    if (n_pixels < 0 || n_pixels >= (1LL << 24)) return set_error(MS_ERR_INVALID_ARG, "n_pixels must be in [0, 2^24)");
    if (n_pixels > 0 && (!h_emb || !h_labels)) return set_error(MS_ERR_INVALID_ARG, "NULL host buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t eb = sizeof(float) * (size_t)n_pixels * (size_t)cfg->dim;
    const size_t mb = h_mask ? (size_t)n_pixels : 0;
    const size_t lb = sizeof(int32_t) * (size_t)n_pixels;
    const size_t modes_b = h_modes ? sizeof(float) * (size_t)(cap > 0 ? cap : 0) * (size_t)cfg->dim : 0;
    char* buf = nullptr;
    const size_t o_mask = align_up(eb), o_lab = o_mask + align_up(mb), o_modes = o_lab + align_up(lb);
    MS_CUDA(cudaMalloc(&buf, o_modes + align_up(modes_b) + kAlign));
    ms_ctx* ctx = nullptr;
    int32_t k = 0;
    s = cuda_check(cudaMemcpyAsync(buf, h_emb, eb, cudaMemcpyHostToDevice, st), "copy h_emb");
    if (s == MS_OK && mb) s = cuda_check(cudaMemcpyAsync(buf + o_mask, h_mask, mb, cudaMemcpyHostToDevice, st), "copy h_mask");
    if (s == MS_OK) s = ms_create(cfg, (const float*)buf, mb ? (const uint8_t*)(buf + o_mask) : nullptr, n_pixels, stream, &ctx);
    if (s == MS_OK) s = ms_run(ctx, (int32_t*)(buf + o_lab), h_modes ? (float*)(buf + o_modes) : nullptr, cap, &k);
    if (s == MS_OK && lb) s = cuda_check(cudaMemcpyAsync(h_labels, buf + o_lab, lb, cudaMemcpyDeviceToHost, st), "copy labels");
    if (s == MS_OK && h_modes && k > 0)
        s = cuda_check(cudaMemcpyAsync(h_modes, buf + o_modes, sizeof(float) * (size_t)k * cfg->dim,
                                       cudaMemcpyDeviceToHost, st), "copy modes");
    if (s == MS_OK) s = cuda_check(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (s == MS_OK && stats_out) ms_stats_get(ctx, stats_out);
    if (n_modes_out) *n_modes_out = k;
    ms_destroy(ctx);
    cudaFree(buf);
    return s;
}

ms_status ms_get_state(const ms_ctx* ctx, int64_t* n_next_out) {
    if (!ctx || !n_next_out) return set_error(MS_ERR_INVALID_ARG, "NULL argument");
    *n_next_out = carried_n(ctx);
    return MS_OK;
}

ms_status ms_set_state(ms_ctx* ctx, int64_t n_next) {
    if (!ctx) return set_error(MS_ERR_INVALID_ARG, "ctx is NULL");
    if (n_next < 1) return set_error(MS_ERR_INVALID_ARG, "n_next must be >= 1");
    if (ctx->phase != 0 || ctx->stats.rounds != 0)
        return set_error(MS_ERR_STATE, "the seed count can be set only before the frame's first round");
    ctx->N = n_next;
    ctx->N_carry = n_next;
    ctx->max_draw = 0;
    return MS_OK;
}

ms_status ms_inspect(const ms_ctx* cctx, int32_t what, void* h_out, int64_t cap, int64_t* count_out) {
    ms_ctx* ctx = const_cast<ms_ctx*>(cctx);
    if (!ctx || (cap > 0 && !h_out)) return set_error(MS_ERR_INVALID_ARG, "NULL argument");
    int64_t avail = 0;
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    switch (what) {
        case MS_INSPECT_SEED_LOG: {
            avail = ctx->stats.seeds;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0) MS_CUDA(cudaMemcpy(h_out, ctx->seed_log, sizeof(int32_t) * c, cudaMemcpyDeviceToHost));
            break;
        }
        case MS_INSPECT_MODES: {
            avail = ctx->n_kept;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0)
                MS_CUDA(cudaMemcpy2D(h_out, sizeof(float) * ctx->d, ctx->modes, sizeof(float) * ctx->Dp,
                                     sizeof(float) * ctx->d, (size_t)c, cudaMemcpyDeviceToHost));
            break;
        }
        case MS_INSPECT_SUPPORT: {
            avail = ctx->n_kept;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0) MS_CUDA(cudaMemcpy(h_out, ctx->mode_support, sizeof(int32_t) * c, cudaMemcpyDeviceToHost));
            break;
        }
        case MS_INSPECT_COVERED: {
            avail = ctx->n;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0) MS_CUDA(cudaMemcpy(h_out, ctx->covered, (size_t)c, cudaMemcpyDeviceToHost));
            break;
        }
        case MS_INSPECT_ROUND_LOG: {
            avail = ctx->stats.rounds;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0) memcpy(h_out, ctx->round_log, sizeof(int64_t) * 4 * (size_t)c);
            break;
        }
        case MS_INSPECT_PIXELS: {
            avail = ctx->n;
            const int64_t c = avail < cap ? avail : cap;
            if (c > 0)
                MS_CUDA(cudaMemcpy2D(h_out, sizeof(float) * ctx->d, ctx->P32, sizeof(float) * ctx->Dp,
                                     sizeof(float) * ctx->d, (size_t)c, cudaMemcpyDeviceToHost));
            break;
        }
        default:
            return set_error(MS_ERR_INVALID_ARG, "unknown inspect code %d", what);
    }
    if (count_out) *count_out = avail;
    return MS_OK;
}

}  // extern "C"

extern "C" ms_status ms_tc_selftest(const float* d_X, const float* d_P, int32_t n_pix, double c, float* h_S,
                                    int64_t* h_acc) {
    g_err[0] = 0;
    if (!d_X || !d_P || !h_S || !h_acc || n_pix < 1 || n_pix > 4096)
        return set_error(MS_ERR_INVALID_ARG, "bad self-test arguments");
    ms_config cfg;
    ms_config_default(&cfg);
    cfg.precision = MS_BF16;
    cfg.bandwidth_cos = c;
    ms_ctx* ctx = nullptr;
    ms_status s = ms_create(&cfg, d_P, nullptr, n_pix, nullptr, &ctx);
    if (s != MS_OK) return s;
    float* dbg = nullptr;
    const size_t n_pad = (size_t)ctx->n_pad;
    int32_t iota[128];
    for (int i = 0; i < 128; ++i) iota[i] = i;
    DevCounters dc0;
    memset(&dc0, 0, sizeof(dc0));
    dc0.n_active = 128;
    dc0.m_round = 128;
    s = cuda_check(cudaMalloc(&dbg, sizeof(float) * 128 * n_pad), "cudaMalloc");
    if (s == MS_OK) s = cuda_check(cudaMemset(dbg, 0, sizeof(float) * 128 * n_pad), "cudaMemset");
    if (s == MS_OK) s = cuda_check(cudaMemcpy(ctx->X, d_X, sizeof(float) * 128 * 16, cudaMemcpyDeviceToDevice), "copy X");
    if (s == MS_OK) s = cuda_check(cudaMemcpy(ctx->active[0], iota, sizeof(iota), cudaMemcpyHostToDevice), "copy active");
    if (s == MS_OK) s = cuda_check(cudaMemcpy(ctx->dc, &dc0, sizeof(dc0), cudaMemcpyHostToDevice), "copy counters");
    if (s == MS_OK) s = launch_shift_tc(ctx, ctx->active[0], 1, 1, dbg);
    if (s == MS_OK) s = cuda_check(cudaDeviceSynchronize(), "self-test kernel");
    if (s == MS_OK) s = readback(ctx);
    if (s == MS_OK && ctx->hc->status != 0) s = set_error(MS_ERR_TIMEOUT, "tensor-core tile timed out");
    if (s == MS_OK) s = cuda_check(cudaMemcpy(h_S, dbg, sizeof(float) * 128 * n_pad, cudaMemcpyDeviceToHost), "copy S");
    if (s == MS_OK)
        s = cuda_check(cudaMemcpy(h_acc, ctx->acc, sizeof(int64_t) * 128 * 17, cudaMemcpyDeviceToHost), "copy acc");
    if (dbg) cudaFree(dbg);
    ms_destroy(ctx);
    return s;
}
