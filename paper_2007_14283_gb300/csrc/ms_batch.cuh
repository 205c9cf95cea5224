// Batched form: B frames of uneven size clustered together, every frame's
// OSOP control on the device (a per-frame state machine advanced by one CUDA
// graph whose body runs until all frames finish).
#pragma once

#include "ms_internal.cuh"

namespace ms {

// Per-frame phase of the OSOP loop.
enum BPhase : int32_t { kNeedSeed = 0, kIterating = 1, kRoundDone = 2, kFinished = 3 };

// Per-frame constants, fixed after set-up. Frame f owns the rows
// [pix0, pix0 + n) of every per-pixel, per-seed, per-candidate and per-mode
// array, and the Pk rows [pk_row0, pk_row0 + n_ptiles * 128).
struct BFrame {
    int64_t pix0;
    int64_t in0;        // offset of the frame's input pixels (labels, masks)
    int64_t n_pixels;   // input pixels
    int32_t n;          // foreground pixels
    int32_t n_ptiles;   // ceil(n / 128)
    int32_t pk_row0;
    int32_t pad;
    uint64_t perm_a, perm_b;
    const float* emb;   // borrowed input [n_pixels, d]
    const uint8_t* mask;
};

// Per-frame state, advanced only by device code.
struct BState {
    DevCounters dc;
    int64_t N;          // seeds requested next round (Sec. 3.2.4)
    int32_t phase;
    int32_t rounds;
    int32_t k0;         // kept modes before the current merge
    int32_t iters_total;
    int64_t seeds_total;
    int64_t cands_total;
    int64_t dropped_total;
};

// Work split of the current iteration, computed on the device.
// item_off / seed_off: exclusive prefix sums over frames (B + 1 entries).
struct BPlan {
    int32_t* item_off;
    int32_t* seed_off;
    int32_t* chunks;    // per frame
    int32_t* tpc;       // per frame: pixel tiles (TC) or pixels (FP32) per chunk
};

// Tensor-core shift over all iterating frames (ms_shift_tc.cu).
ms_status tc_batch_setup(int D);
ms_status launch_shift_tc_batch(const CUtensorMap& pmap, const CUtensorMap& pmap1, int D, const float* P32,
                                const float* X, unsigned long long* acc, float c_f, const BFrame* frames,
                                const BState* states, BPlan plan, const int32_t* act0, const int32_t* act1, int nf,
                                int* status, unsigned long long* band, int grid, int shape, cudaStream_t st);
// FP32 shift over all iterating frames (ms_shift_fp32.cu).
ms_status launch_shift_fp32_batch(const float* P32, const float* X, unsigned long long* acc, float c_f, int Dp,
                                  const BFrame* frames, const BState* states, BPlan plan, const int32_t* act0,
                                  const int32_t* act1, int nf, int grid, cudaStream_t st);

// Index of the frame whose [off[f], off[f+1]) holds i (off has nf + 1 entries).
__device__ __forceinline__ int locate(const int32_t* off, int nf, int i) {
    int lo = 0, hi = nf;  // invariant: off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Scratch of the tensor-core labelling: the near-tie queue (capacity: the
// foreground pixels) and, in batch form, the per-frame item offsets (B + 1).
struct LabelTcScratch {
    int2* fix;
    int* fix_count;
    int32_t* off;
};

ms_status label_tc_setup();
// Labelling on the tensor cores (BF16 form, Dp = 16 or 32): exact FP64-argmax
// labels, near-ties re-decided as the FP32 form decides them. pmap1: the
// pixels' dimensions 16-31 (Dp = 32); Mk holds the modes' split rows, for
// Dp = 32 followed by a second array of n_pad (mk_rows) rows.
ms_status launch_label_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad, int Dp,
                                 const float* modes, int K, int n, const float* P32, const int32_t* pix,
                                 const float* emb, int d, int32_t* labels, LabelTcScratch sc, int grid, int* status,
                                 cudaStream_t st);
// Coverage against one frame's new modes [k0, k1) on the tensor cores (BF16
// form): exact decisions, the near-threshold pixels re-decided as the FP32
// form decides them.
ms_status launch_cover_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad, int Dp,
                                 const float* modes, int k0, int k1, int n, const float* P32, const int32_t* pix,
                                 const float* emb, int d, double c, uint8_t* covered, int* n_uncovered,
                                 LabelTcScratch sc, int grid, int* status, cudaStream_t st);
// The same for the frames of a batch whose round ended (tile_off: their pixel
// tiles, from k_b_blocks with 128 pixels per block).
ms_status launch_cover_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                                const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, int Dp, const BFrame* frames,
                                BState* states, int B, int max_pk_rows, const float* modes, const float* P32,
                                const int32_t* pix, int d, double c, uint8_t* covered, const int32_t* tile_off,
                                LabelTcScratch sc, int grid, int* status, cudaStream_t st);
// The merge's two contractions on the tensor cores for the frames whose round
// ended (tile_off: their candidates in blocks of 128): the candidates in rank
// order (Xr, packed into Ck) against their earlier modes (Mk), then against
// one another; exact decisions (merge_cos), the near-threshold pairs decided
// by the FP32-then-FP64 test. Sets removed_r / cand_state and fills the
// conflict lists as k_b_merge_old and k_b_merge_pairs do.
ms_status launch_merge_tc_batch(const CUtensorMap& cmap, const CUtensorMap& cmap1, const CUtensorMap& mmap,
                                const CUtensorMap& mmap1, void* Ck, int64_t rows, int Dp, const BFrame* frames,
                                BState* states, int B, int max_pk_rows, const float* Xr, const float* modes,
                                const int32_t* rank_cand, uint8_t* cand_state, uint8_t* removed_r, int32_t* conf_deg,
                                int32_t* conf, float thr_f, double thr, const int32_t* tile_off, LabelTcScratch sc,
                                int grid, int* status, cudaStream_t st);
// The same for one frame: k candidates (Xr, packed into Ck) against its K_old
// earlier modes (Mk), then against one another.
ms_status launch_merge_tc_single(void* Ck, void* Mk, int64_t n_pad, int Dp, int k, int K_old, const float* Xr,
                                 const float* modes, const int32_t* rank_cand, uint8_t* cand_state, uint8_t* removed_r,
                                 int32_t* conf_deg, int32_t* conf, float thr_f, double thr, LabelTcScratch sc,
                                 int grid, int* status, cudaStream_t st);
ms_status launch_label_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                                const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, int Dp, const BFrame* frames,
                                const BState* states, int B, int max_pk_rows, const float* modes, const float* P32,
                                const int32_t* pix, int d, int32_t* const* labels, LabelTcScratch sc, int grid,
                                int* status, cudaStream_t st);

// Pixel tiles per chunk when a frame's seed tiles (128 seeds each) are cut
// into tiles x chunks work items for the tensor-core shift. The plain rule
// spreads `target` items over the seed tiles. With grid > 0 the items are
// also fitted to the launch's CTAs, which each take items in turn: among the
// chunk counts that fill 2..8 whole waves of the grid (at least two items per
// CTA, so one item's pipeline fill overlaps the previous item's drain) and the
// plain rule's,
// the one with the smallest makespan waves x (tiles per item + 2 tiles of
// per-item overhead) wins (ties: the earlier candidate). Integer arithmetic
// only, so every caller with the same arguments cuts a frame the same way.
__host__ __device__ inline int tc_tiles_per_chunk(int tiles, int n_ptiles, int target, int grid) {
    if (tiles <= 0 || n_ptiles <= 0) return 1;
    int ch = (target + tiles - 1) / tiles;
    ch = ch < 1 ? 1 : (ch > n_ptiles ? n_ptiles : ch);
    int best = (n_ptiles + ch - 1) / ch;
    if (grid <= 0) return best;
    auto cost = [&](int tpc) {
        const long long items = (long long)tiles * ((n_ptiles + tpc - 1) / tpc);
        return ((items + grid - 1) / grid) * (long long)(tpc + 2);
    };
    long long best_cost = cost(best);
    for (int w = 2; w <= 8; ++w) {
        int c = (int)((long long)w * grid / tiles);
        if (c < 1) continue;
        c = c > n_ptiles ? n_ptiles : c;
        const int tpc = (n_ptiles + c - 1) / c;
        const long long k = cost(tpc);
        if (k < best_cost) {
            best_cost = k;
            best = tpc;
        }
    }
    return best;
}

}  // namespace ms
