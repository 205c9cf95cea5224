// Internal declarations shared by the libms translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ms.h"

namespace ms {

// Pixels and seeds are stored with their dimension padded by zeros to Dp = 16
// or 32: padding changes no dot product or norm, and keeps rows 64/128-byte
// aligned for vector loads.
inline int padded_dim(int d) { return d <= 16 ? 16 : 32; }

// FP32 similarity is decided directly when it clears the threshold by more
// than kEpsF32; inside that band the decision is recomputed in FP64. For unit
// vectors with d <= 32 the FP32 dot product, including the normalisation
// error of both operands, is within 2.3e-6 of the exact value.
constexpr float kEpsF32 = 1e-5f;

// Normalised pixel components below 2^-100 in magnitude are stored as 0. This
// changes no dot product by more than 2^-95 and keeps every stored component
// in the range where its three-term BF16 split (tensor-core form) rebuilds
// the FP32 value exactly.
constexpr float kTinyComponent = 7.8886090522101181e-31f;  // 2^-100
__host__ __device__ inline float flush_tiny(float v) { return fabsf(v) < kTinyComponent ? 0.f : v; }

constexpr int kShiftThreads = 128;
constexpr int kSeedsPerThread = 2;
constexpr int kSeedsPerTile = kShiftThreads * kSeedsPerThread;  // 256
constexpr int kPixTile = 128;                                    // pixels per smem stage
constexpr int kMergeCap = 32;  // stored higher-ranked conflicts per merge candidate

enum SeedState : uint8_t { kMoving = 0, kConverged = 1, kFailed = 2 };
enum CandState : uint8_t { kUndecided = 0, kKept = 1, kRemoved = 2 };

// Device-resident control block of one frame.
struct DevCounters {
    int32_t n_active;    // seeds in the current iteration's active list
    int32_t n_next;      // seeds still moving after this iteration
    int32_t conv_new;    // converged during this iteration
    int32_t conv_total;  // converged in this round
    int32_t fail_total;  // empty windows in this round
    int32_t done;        // round finished
    int32_t iters;       // iterations run in this round
    int32_t m_round;     // seeds in this round
    int32_t status;      // nonzero: device-side input error
    int32_t n_seeded;    // seeds drawn by the last selection
    int32_t cursor;      // next seed-order position
    int32_t drawn;       // seeds drawn over all rounds
    int32_t n_kept;      // kept modes
    int32_t n_cand;      // merge candidates
    int32_t undecided;   // merge candidates still undecided
    int32_t n_uncovered; // foreground pixels not covered
    int32_t n_fg;        // foreground pixels
    int32_t pad;
    int64_t seed_iters;  // seed-iterations summed
    int64_t band_pairs;  // BF16 form: pairs rechecked in FP32
};

// Work split of one shift iteration: seed tiles x pixel chunks.
struct ShiftSplit {
    int tiles, chunks, chunk_len;
};

__host__ __device__ inline ShiftSplit shift_split(int n_active, int n, int target_items) {
    ShiftSplit s;
    s.tiles = (n_active + kSeedsPerTile - 1) / kSeedsPerTile;
    if (s.tiles == 0 || n == 0) {
        s.chunks = 0;
        s.chunk_len = kPixTile;
        return s;
    }
    int max_chunks = (n + kPixTile - 1) / kPixTile;
    int ch = (target_items + s.tiles - 1) / s.tiles;
    ch = ch < 1 ? 1 : (ch > max_chunks ? max_chunks : ch);
    int per = (n + ch - 1) / ch;
    per = (per + kPixTile - 1) / kPixTile * kPixTile;
    s.chunk_len = per;
    s.chunks = (n + per - 1) / per;
    return s;
}

}  // namespace ms

struct ms_ctx {
    ms_config cfg;
    int d, Dp;
    cudaStream_t stream;
    const float* emb;
    const uint8_t* mask;
    int64_t n_pixels;
    int64_t n;          // foreground count
    int64_t perm_a, perm_b;
    int num_sms;
    int shift_grid;     // persistent grid of the shift kernel
    int target_items;   // work items per shift iteration
    // workspace (one allocation)
    void* ws;
    size_t ws_bytes;
    float* P32;          // [n_pixels, Dp] normalised foreground
    int32_t* pix;        // [n_pixels] foreground index -> pixel index
    uint8_t* covered;    // [n_pixels]
    float* X;            // [n_pixels, Dp] seed positions by slot
    int32_t* seed_pix;   // [n_pixels]
    int32_t* seed_order; // [n_pixels]
    uint8_t* sstate;     // [n_pixels]
    int32_t* support;    // [n_pixels]
    int32_t* active[2];  // [n_pixels] each
    int32_t* seed_log;   // [n_pixels]
    unsigned long long* acc;  // [n_pixels, Dp + 1] fixed-point window sums and counts (2^-36 units)
    float* modes;        // [n_pixels, Dp] kept modes
    int32_t* mode_support;
    int32_t* cand;       // [n_pixels] candidate slots
    int32_t* cand_rank;  // [n_pixels]
    int32_t* rank_cand;  // [n_pixels] inverse of cand_rank
    uint8_t* cand_state; // [n_pixels]
    int32_t* conf_deg;   // [n_pixels]
    int32_t* conf;       // [n_pixels * kMergeCap]
    int32_t* block_tmp;  // ingest scan scratch
    ms::DevCounters* dc;
    ms::DevCounters* hc; // pinned host mirror
    int64_t* round_log;  // host [cap * 4]
    int64_t round_log_cap;
    // host-side OSOP state
    int phase;           // 0 idle, 1 seeded, 2 iterated
    int64_t N;           // seed count for the next batch
    int64_t N_carry;     // the schedule's N without the clamp to uncovered pixels (carried across video frames)
    int64_t max_draw;    // the largest seed batch of the frame so far (bounds the carried N)
    int64_t max_pixels;  // the workspace holds frames of up to this many pixels
    int64_t uncovered;
    int32_t n_kept;
    int32_t m_round;
    ms_stats stats;
    // BF16 tensor-core form
    void* Pk;            // [n_pad, 64] bf16: [Ph | Pm | Pl | 0] per pixel
    int64_t n_pad;       // n rounded up to 128 (0 when n = 0)
    CUtensorMap pmap;    // TMA map of Pk: boxes of 128 rows x 128 bytes, 128-byte swizzle
    CUtensorMap pmap1;   // d = 32: the same for dimensions 16..31 (the second Pk array)
    int tc_grid;         // persistent grid of the tensor-core shift kernel
    void* Mk;            // [n_pad, 64] bf16 split rows of the kept modes (labelling)
    int2* label_fix;     // [n] near-tie queue of the tensor-core labelling, then its count
    float* Xr;           // BF16 form: [n, Dp] merge candidates' positions in rank order
    uint8_t* removed_r;  // BF16 form: [n] candidates removed by an earlier mode, by rank
    void* Ck;            // BF16 form: [n_pad, 64] bf16 split rows of Xr (a second array for Dp = 32)
    // measurement
    bool prof;
    cudaEvent_t ev[64];  // start/end pairs around shift launches of one batch
    int64_t launches;
};

namespace ms {

// Error plumbing (ms_api.cu).
ms_status set_error(ms_status code, const char* fmt, ...);
ms_status cuda_check(cudaError_t e, const char* what);
// cudaMalloc of a context's or batch's workspace, failing first when a test
// asked for it through ms_inject_alloc_failure (ms_api.cu).
cudaError_t workspace_malloc(void** p, size_t bytes);
// Stream-ordered scratch from the library's own pool (kept mapped between calls); free with cudaFreeAsync.
cudaError_t scratch_malloc_async(void** p, size_t bytes, cudaStream_t st);
#define MS_CUDA(call)                                                 \
    do {                                                              \
        ms_status _s = ::ms::cuda_check((call), #call);               \
        if (_s != MS_OK) return _s;                                   \
    } while (0)
#define MS_LAUNCH(what)                                               \
    do {                                                              \
        ms_status _s = ::ms::cuda_check(cudaGetLastError(), what);    \
        if (_s != MS_OK) return _s;                                   \
    } while (0)

// Kernel launchers. Each enqueues on ctx->stream and returns MS_OK or MS_ERR_CUDA.
ms_status launch_ingest(ms_ctx* ctx);                       // ms_ingest.cu
ms_status launch_seed_select(ms_ctx* ctx, int32_t want);    // ms_seed.cu
ms_status launch_shift_iteration(ms_ctx* ctx, int t, int max_iter, cudaEvent_t e0, cudaEvent_t e1);  // ms_shift_fp32.cu
float ceil_to_float(double c);  // smallest float >= c
ms_status launch_merge_prepare(ms_ctx* ctx, int32_t k);     // ms_merge.cu
ms_status launch_merge_resolve(ms_ctx* ctx, int32_t k, int sweeps);
ms_status launch_merge_sequential(ms_ctx* ctx, int32_t k);
ms_status launch_merge_append(ms_ctx* ctx, int32_t k);
ms_status launch_cover(ms_ctx* ctx, int32_t k0, int32_t k1);
ms_status launch_label(ms_ctx* ctx, int32_t* d_labels);     // ms_label.cu
ms_status launch_collect(ms_ctx* ctx);                      // ms_merge.cu
int shift_blocks_per_sm();                                  // ms_shift_fp32.cu
// Window sums of the seeds active[0..dc->n_active) into acc (fixed point), d = 16.
ms_status launch_window_sums_fp32(const float* P32, int32_t n, const int32_t* active, const float* X,
                                  unsigned long long* acc, float c, const DevCounters* dc,
                                  cudaStream_t stream);
ms_status tc_pack_async(ms_ctx* ctx);                       // ms_shift_tc.cu: split rows on ctx->stream
ms_status tc_finish(ms_ctx* ctx);                           // kernel attributes, TMA map of the n_pad rows
// ms_api.cu: a context's workspace, and binding frames to it (ms_create and the video form)
ms_status ctx_alloc(const ms_config* cfg, int64_t max_pixels, cudaStream_t stream, ms_ctx** out);
ms_status ctx_bind_async(ms_ctx* ctx, const float* d_emb, const uint8_t* d_mask, int64_t n_pixels, cudaStream_t st);
ms_status ctx_bind_finish(ms_ctx* ctx, cudaStream_t st, uint64_t frame_id, int64_t n_start);
void ctx_free(ms_ctx* ctx);
int64_t carried_n(const ms_ctx* ctx);   // the N a video carries into its next frame
ms_status launch_shift_tc(ms_ctx* ctx, const int32_t* active, int grid, int target_items, float* dbg_S);
int tc_smem_bytes(int D);
constexpr int kTcShapes = 8;  // values of ms_config.tc_shape (warp arrangements of k_shift_tc)
ms_status encode_pk_map(void* Pk, int rows, CUtensorMap* map);  // ms_shift_tc.cu: TMA map of split rows

// ms_vmf_tc.cu: the smooth-kernel step on the tensor cores.
struct VmfTcPlan {
    int n_ptiles, chunks, tpc, items, grid;  // 128-pixel tiles, chunks of tpc tiles, work items, CTAs
};
VmfTcPlan vmf_tc_plan(int32_t M, int64_t N, int grid);
size_t vmf_tc_pk_bytes(int64_t N);
// Packs P [N, 16] into BF16 split rows and encodes their TMA map (on st).
ms_status vmf_tc_prepare(const float* P, int64_t N, void* Pk, CUtensorMap* map, cudaStream_t st);
// One step x_t -> x_{t+1}; partial holds plan.items x 128 x 16 floats.
ms_status vmf_tc_step(const CUtensorMap& map, const float* Xt, int32_t M, float kappa, const VmfTcPlan& plan,
                      float* partial, int* status, float* Xn, float* ynorm, cudaStream_t st);

// ms_vmf_tc_adj.cu: the smooth-kernel adjoint step on the tensor cores.
struct VmfAdjPlan {
    int row_tiles, n_sub, chunks, spc, items, grid;  // 128-row tiles x chunks of spc 64-column sub-tiles
};
struct VmfAdjWork {
    CUtensorMap pk_rows, pk_cols;  // Pk (BF16 split pixel rows) in 128-row and 64-row boxes
    CUtensorMap v_rows, v_cols;    // Vk: split rows of kappa log2(e) x_t (and the -kappa log2(e) column)
    CUtensorMap g_cols;            // Gk: split rows of gy (pass B's seed columns)
    CUtensorMap ga_rows;           // Gak: split rows of kappa gy (pass A's seed rows)
    void* Vk;
    void* Gk;
    void* Gak;
    float* partial_a;              // pass A: per item 128 seed rows x 16 sums
    float* partial_b;              // pass B: per item 128 pixel rows x 16 sums, over every step
    VmfAdjPlan pa, pb;             // pass A (rows: seeds), pass B (rows: pixels)
    int32_t M, Mp;
    int64_t N;
};
// Workspace bytes of vmf_adj_prepare for M seeds, N pixels and `grid` CTAs.
size_t vmf_adj_bytes(int32_t M, int64_t N, int grid);
// Lays out the workspace ws and encodes the TMA maps; Pk as vmf_tc_prepare wrote it.
ms_status vmf_adj_prepare(void* Pk, int64_t N, int32_t M, int grid, void* ws, VmfAdjWork* w);
// The whole reverse sweep over T steps on the tensor cores, from the
// forward's iterates (iters: x_0..x_T, [T+1, M, 16]) and |y_t| ([T, M]):
// dX0 = dL/dx_0, dP = dL/dP (overwritten). A raised *status poisons both (NaN).
ms_status vmf_adj_backward(VmfAdjWork* w, const float* iters, const float* ynorm, int32_t T, float kappa,
                           const float* GT, int* status, float* dP, float* dX0, cudaStream_t st);

}  // namespace ms
