// Labelling, BF16 tensor-core form (the labelling step of Algorithm 2): every
// foreground vector takes the mode of highest cosine, lowest index on ties.
//
// The pixel-by-mode score matrix is a GEMM with K = d = 16 (or 32, as two
// 16-dimensional halves with their own pixel and mode tiles). A work item is
// one tile of 128 pixels (the GEMM's M rows) against every 128-mode tile of
// its frame (N columns); the scores live only in TMEM:
//     S = Ph.Mh + Ph.Mm + Pm.Mh          (3 tcgen05 MMAs per half, FP32 accumulate)
// with p = Ph + Pm + Pl and m = Mh + Mm + Ml the exact BF16 splits of the FP32
// vectors, so |S - p.m| <= LbDim<D>::kEps (the bound is derived there).
// Sixteen warps read S from TMEM, one pixel per lane and 32 mode columns per
// warp, and keep the best and second-best score of each pixel. A pixel whose
// best leads its second by more than 2 * kEps has the exact FP64 argmax as its
// winner; the others (near-ties) are queued and re-decided by k_label_fix
// exactly as the FP32 form decides them: FP32 scores over all modes, then
// FP64 among those within 2 * kEpsF32 of the best.
//
// Warp roles (576 threads, one CTA per SM): warps 0-15 read S (warp w reaches
// TMEM lanes 32 * (w % 4) + 0..31); warp 16 issues TMA loads (the item's pixel
// tile, double-buffered, and mode tiles into a 4- or 8-stage ring); warp 17 owns the
// 512 TMEM columns (four S buffers of 128) and issues the MMAs from a converged
// warp, one elected lane issuing. Waits are bounded as in the shift kernel.
#include <cudaTypedefs.h>

#include "ms_batch.cuh"
#include "ms_device.cuh"
#include "ms_tc.cuh"

namespace ms {
namespace {

using namespace tc;

constexpr int kLEpi = 16;                   // score-reading warps
constexpr int kLWarpTma = kLEpi;
constexpr int kLWarpMma = kLEpi + 1;
constexpr int kLThreads = (kLEpi + 2) * 32;  // 576
constexpr int kLSBufs = 4;                  // S buffers, 128 TMEM columns each
constexpr int kLTile = 128 * 128;           // bytes of a 128-row operand tile
constexpr uint32_t kLTmemCols = 512;

// Layout and score bound for embedding dimension D (16, or 32 as two halves).
// Bound of |S - p.m| for unit vectors: per component the three products leave
// out ph.ml + pm.(mm + ml) + pl.m. Each round-to-nearest BF16 residual is at
// most 2^-8 of the value it splits (8 significant bits), so the three terms
// are at most 2^-16 (1 + 2^-8) |p_k||m_k| each: at most 4.64e-5 over a unit
// pair (a search over the split's rounding cases reaches about 2 * 2^-16 =
// 3.0e-5). The tensor cores add the 3 * D exact products in FP32 in an
// unspecified order; with partial sums below 1.01 an addition loses at most
// 2^-22 even if it truncates both addends and the result: 48 * 2^-22 =
// 1.14e-5 (D = 16) or 96 * 2^-22 = 2.29e-5 (D = 32). Hence kEps.
template <int D>
struct LbDim {
    static constexpr int kHalves = D / 16;
    static constexpr int kStages = D == 16 ? 8 : 4;                        // mode-tile ring
    static constexpr int kOffA = 0;                                        // 2 pixel tiles per half
    static constexpr int kOffB = 2 * kHalves * kLTile;                     // kStages mode tiles per half
    static constexpr int kOffX = kOffB + kStages * kHalves * kLTile;       // exchange: [4][128] x (b1, i1, b2)
    static constexpr int kOffBar = kOffX + 4 * 128 * 12;
    static constexpr int kNumBars = 2 * 2 + 2 * kStages + 2 * kLSBufs + 2;
    static constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16 + 1024;
    static constexpr float kEps = D == 16 ? 6e-5f : 7e-5f;
    static_assert(D == 16 || D == 32, "embedding dimension 16 or 32");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

// What an item covers.
struct LbItem {
    int frame;
    int pk_row0;   // Pk / Mk row of the frame's pixel 0 and mode 0 (multiple of 128)
    int pt;        // pixel tile
    int n;         // the frame's foreground count
    int K;         // the frame's kept modes (the end of the scored mode range)
    int k0;        // the first scored mode (0 for labelling; coverage scores a round's new modes)
};

struct LbSingle {
    int n, K;
    __device__ __forceinline__ bool init() { return n > 0; }
    __device__ __forceinline__ int total() const { return (n + 127) / 128; }
    int k0 = 0;
    __device__ __forceinline__ LbItem item(int i) const { return LbItem{0, 0, i, n, K, k0}; }
};

struct LbBatch {
    const BFrame* frames;
    const BState* states;
    const int32_t* off;   // pixel-tile offsets over frames (B + 1)
    int B;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = off[B];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ LbItem item(int i) const {
        const int f = locate(off, B, i);
        const BFrame& fr = frames[f];
        return LbItem{f, fr.pk_row0, i - off[f], fr.n, states[f].dc.n_kept, 0};
    }
};

// Coverage in the batch: the pixel tiles of the frames whose round ended
// (off from k_b_blocks with 128 pixels per block), each against its frame's
// new modes [k0, n_kept).
struct LbBatchCover {
    const BFrame* frames;
    const BState* states;
    const int32_t* off;
    int B;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = off[B];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ LbItem item(int i) const {
        const int f = locate(off, B, i);
        const BFrame& fr = frames[f];
        return LbItem{f, fr.pk_row0, i - off[f], fr.n, states[f].dc.n_kept, states[f].k0};
    }
};

// The merge of the frames whose round ended (off from k_b_blocks with 128
// candidates per block): row tile t of a frame's k candidates, in rank order
// (Ck rows), against its modes kept in earlier rounds (Mk, LbBatchOld) or
// against the candidates ranked up to the tile's end (Ck, LbBatchPairs).
struct LbBatchOld {
    const BFrame* frames;
    const BState* states;
    const int32_t* off;
    int B;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = off[B];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ LbItem item(int i) const {
        const int f = locate(off, B, i);
        return LbItem{f, frames[f].pk_row0, i - off[f], states[f].dc.n_cand, states[f].dc.n_kept, 0};
    }
};
struct LbBatchPairs {
    const BFrame* frames;
    const BState* states;
    const int32_t* off;
    int B;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = off[B];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ LbItem item(int i) const {
        const int f = locate(off, B, i);
        const int t = i - off[f], k = states[f].dc.n_cand;
        return LbItem{f, frames[f].pk_row0, t, k, min(k, (t + 1) * 128), 0};
    }
};

// The same for one frame (row base 0): k candidates against K earlier modes,
// or against one another (pairs).
struct LbSingleMerge {
    int k, K, pairs;
    __device__ __forceinline__ bool init() { return k > 0; }
    __device__ __forceinline__ int total() const { return (k + 127) / 128; }
    __device__ __forceinline__ LbItem item(int i) const {
        return LbItem{0, 0, i, k, pairs ? min(k, (i + 1) * 128) : K, 0};
    }
};

__device__ __forceinline__ bool lwarp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

__device__ __forceinline__ void ldrain(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

// Output of one pixel: where its label goes and, for a near-tie, the queue.
// Batch form: per-frame label pointers and pixel offsets from the frames;
// single form: labels1 and offset 0.
struct LbOut {
    int32_t* const* labels;    // per frame, or nullptr
    int32_t* labels1;
    const BFrame* frames;      // pixel offsets (pix0), or nullptr
    const int32_t* pix;        // foreground index -> pixel index, all frames
    int2* fix;                 // near-ties (frame, foreground index)
    int* fix_count;
    // coverage: the covered flags (all frames), the uncovered count (single
    // form) or the frames' states (batch form), and c
    uint8_t* covered;
    int* n_uncovered;
    float c_f;             // coverage: c; merge: merge_cos rounded to FP32
    BState* states;
    // merge (rows are candidates in rank order): their FP32 positions, the
    // removed-by-an-earlier-mode flags by rank, rank -> candidate, the
    // candidates' states and conflict lists, and merge_cos
    const float* Xr;
    uint8_t* removed_r;
    const int32_t* rank_cand;
    uint8_t* cand_state;
    int32_t* conf_deg;
    int32_t* conf;
    double thr;
};

// What k_label_tc's score readers do with a row's scores.
enum LbMode {
    kLbLabel = 0,   // best and second-best column (labelling)
    kLbCover = 1,   // best column against c (OSOP coverage)
    kLbOld = 2,     // best column against merge_cos (candidates against earlier modes)
    kLbPairs = 3,   // every column ranked above the row at or above merge_cos (conflict lists)
};

// kMode = kLbLabel: labelling (best and second-best mode of every pixel).
// kMode = kLbCover: coverage of the OSOP stop rule against the modes [k0, K):
// an uncovered pixel whose best score clears c by kEpsTc is covered; one
// within kEpsTc of c is queued for the FP32 form's exact test.
// kMode = kLbOld, kLbPairs: the merge's two contractions, rows being the
// candidates in rank order. A score farther than kDelta = kEpsTc + 2e-6 from
// merge_cos decides the pair as the exact test does (kEpsTc bounds the split
// score, 2e-6 the gap between x.m and the FP64 cosine of near-unit FP32
// vectors); nearer ones take the exact test itself (cos_at_least). kLbOld:
// a candidate within merge_cos of an earlier mode is removed; near ones are
// queued for k_merge_old_fix. kLbPairs: every candidate ranked above the row
// that is not removed and within merge_cos joins the row's conflict list.
// pmap / mmap: the pixel and mode split rows (dimensions 0-15); pmap1 /
// mmap1: dimensions 16-31 (D = 32 only).
template <class Map, int kMode, int kD>
__global__ void __launch_bounds__(kLThreads, 1)
k_label_tc(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap mmap,
           const __grid_constant__ CUtensorMap pmap1, const __grid_constant__ CUtensorMap mmap1, Map map, LbOut out,
           int* status) {
    using L = LbDim<kD>;
    constexpr int kHalves = L::kHalves, kLStages = L::kStages;
    constexpr float kEpsTc = L::kEps;
    constexpr float kDelta = L::kEps + 2e-6f;
    constexpr bool kCover = kMode == kLbCover || kMode == kLbOld;  // best column against a threshold
    if (!map.init()) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* Ab = smem + L::kOffA;
    uint8_t* Bst = smem + L::kOffB;
    float* xb1 = (float*)(smem + L::kOffX);        // [4][128]
    int* xi1 = (int*)(xb1 + 4 * 128);              // [4][128]
    float* xb2 = (float*)(xi1 + 4 * 128);          // [4][128]
    uint64_t* bars = (uint64_t*)(smem + L::kOffBar);
    uint64_t* a_full = bars;                       // [2]
    uint64_t* a_empty = a_full + 2;                // [2]
    uint64_t* b_full = a_empty + 2;                // [kLStages]
    uint64_t* b_empty = b_full + kLStages;         // [kLStages]
    uint64_t* s_full = b_empty + kLStages;         // [kLSBufs]
    uint64_t* s_empty = s_full + kLSBufs;          // [kLSBufs]
    uint64_t* aux = s_empty + kLSBufs;             // [2] drain
    uint32_t* tmem_slot = (uint32_t*)(bars + L::kNumBars);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
        }
        for (int s = 0; s < kLStages; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int b = 0; b < kLSBufs; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_empty[b], kLEpi);
        }
        mbar_init(&aux[0], 1);
        mbar_init(&aux[1], 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == kLWarpTma && lane == 0) {
        tma_prefetch_desc(&pmap);
        tma_prefetch_desc(&mmap);
        if (kHalves > 1) {
            tma_prefetch_desc(&pmap1);
            tma_prefetch_desc(&mmap1);
        }
    }
    if (warp == kLWarpMma) {
        tmem_alloc(tmem_slot, kLTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int items = map.total();

    if (warp == kLWarpTma) {
        // ------------------------------------------------ TMA producer
        int g = 0, ia = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const LbItem ii = map.item(item);
            const int nmt = (ii.K - ii.k0 + 127) / 128;
            if (nmt <= 0) continue;
            const int ab = ia & 1;
            if (ia >= 2 && !(ok = lwarp_wait(&a_empty[ab], ((ia >> 1) - 1) & 1, abort))) break;
            if (lane == 0) {
                mbar_arrive_expect_tx(&a_full[ab], kHalves * kLTile);
                tma_load_2d(Ab + ab * kHalves * kLTile, &pmap, 0, ii.pk_row0 + ii.pt * 128, &a_full[ab]);
                if (kHalves > 1)
                    tma_load_2d(Ab + (ab * kHalves + 1) * kLTile, &pmap1, 0, ii.pk_row0 + ii.pt * 128, &a_full[ab]);
            }
            __syncwarp();
            ++ia;
            for (int mt = 0; mt < nmt; ++mt, ++g) {
                const int s = g % kLStages;
                if (g >= kLStages && !(ok = lwarp_wait(&b_empty[s], ((g / kLStages) - 1) & 1, abort))) break;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&b_full[s], kHalves * kLTile);
                    tma_load_2d(Bst + s * kHalves * kLTile, &mmap, 0, ii.pk_row0 + ii.k0 + mt * 128, &b_full[s]);
                    if (kHalves > 1)
                        tma_load_2d(Bst + (s * kHalves + 1) * kLTile, &mmap1, 0, ii.pk_row0 + ii.k0 + mt * 128,
                                    &b_full[s]);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && *abort) {
            for (int q = max(0, g - kLStages); q < g; ++q) ldrain(&b_full[q % kLStages], (q / kLStages) & 1);
            for (int q = max(0, ia - 2); q < ia; ++q) ldrain(&a_full[q & 1], (q >> 1) & 1);
        }
    } else if (warp == kLWarpMma) {
        // ------------------------------------------------ MMA issuer
        const uint64_t dA = desc_sw128(smem_u32(Ab), 16, 1024);
        const uint64_t dB = desc_sw128(smem_u32(Bst), 16, 1024);
        constexpr uint32_t id = idesc_bf16(128, 128, 0, 0);
        constexpr uint64_t kT = kLTile >> 4;
        int g = 0, ia = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const LbItem ii = map.item(item);
            const int nmt = (ii.K - ii.k0 + 127) / 128;
            if (nmt <= 0) continue;
            const int ab = ia & 1;
            if (!(ok = lwarp_wait(&a_full[ab], (ia >> 1) & 1, abort))) break;
            const uint64_t a = dA + (uint64_t)ab * kHalves * kT;
            for (int mt = 0; mt < nmt; ++mt, ++g) {
                const int s = g % kLStages, b = g % kLSBufs;
                if (!(ok = lwarp_wait(&b_full[s], (g / kLStages) & 1, abort))) break;
                if (g >= kLSBufs && !(ok = lwarp_wait(&s_empty[b], ((g / kLSBufs) - 1) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tS = tmem + b * 128;
#pragma unroll
                for (int hf = 0; hf < kHalves; ++hf) {
                    const uint64_t ah = a + (uint64_t)hf * kT;
                    const uint64_t bh = dB + (uint64_t)(s * kHalves + hf) * kT;
                    mma_bf16_warp(tS, ah, bh, id, hf == 0 ? 0u : 1u);  // Ph . Mh
                    mma_bf16_warp(tS, ah, bh + 2, id, 1);              // Ph . Mm
                    mma_bf16_warp(tS, ah + 2, bh, id, 1);              // Pm . Mh
                }
                mma_commit_warp(&s_full[b]);
                mma_commit_warp(&b_empty[s]);
            }
            if (!ok) break;
            mma_commit_warp(&a_empty[ab]);
            ++ia;
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[0]);
            ldrain(&aux[0], 0);
        }
    } else {
        // ------------------------------------------------ score readers
        const int q = warp & 3;                  // TMEM lane quadrant
        const int h = warp >> 2;                 // which 32 columns of a mode tile
        const int r = q * 32 + lane;             // pixel row of the tile
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int g = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x) {
            const LbItem ii = map.item(item);
            const int nmt = (ii.K - ii.k0 + 127) / 128;
            if (kMode != kLbLabel && nmt <= 0) continue;
            bool ok = true;
            float b1 = -INFINITY, b2 = -INFINITY;
            int i1 = -1;
            // merge rows: the candidate's rank, its frame's row base, and
            // whether it takes part (a candidate removed by an earlier mode
            // needs no conflict list)
            const int mi = ii.pt * 128 + r;
            const int64_t mbase = (kMode == kLbPairs && out.frames) ? out.frames[ii.frame].pix0 : 0;
            const bool mrow = kMode == kLbPairs && mi < ii.n && !out.removed_r[mbase + mi];
            int ma = -1;  // the row's candidate index, read when first needed
            for (int mt = 0; mt < nmt; ++mt, ++g) {
                const int b = g % kLSBufs;
                if (!(ok = lwarp_wait(&s_full[b], (g / kLSBufs) & 1, abort))) break;
                tc_fence_after();
                // A full slice of 32 columns gets its per-lane maximum from the
                // TMEM load itself; the last, partial slice of an item masks its
                // padding columns (scores of zero rows) and takes the maximum here.
                uint32_t v[32];
                float m;
                const int col0 = ii.k0 + mt * 128 + h * 32;
                const bool partial = col0 + 32 > ii.K;  // warp-uniform
                if (partial)
                    tmem_ld32(tmem + b * 128 + lane_base + h * 32, v);
                else
                    tmem_ld32_max(tmem + b * 128 + lane_base + h * 32, v, &m);
                tmem_ld_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_empty[b]);
                if (partial) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (col0 + j >= ii.K) v[j] = 0xFF800000u;  // -inf: past the last mode
                    m = __uint_as_float(v[0]);
#pragma unroll
                    for (int j = 1; j < 32; ++j) m = fmaxf(m, __uint_as_float(v[j]));
                }
                if (kCover) {
                    b1 = fmaxf(b1, m);
                    continue;
                }
                if constexpr (kMode == kLbPairs) {
                    const float lo = out.c_f - kDelta, hi = out.c_f + kDelta;
                    if (__any_sync(0xffffffffu, mrow && m >= lo) && mrow && m >= lo) {
                        uint32_t near = 0, sure = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float sc = __uint_as_float(v[j]);
                            near |= (uint32_t)(sc >= lo && col0 + j < mi) << j;
                            sure |= (uint32_t)(sc >= hi) << j;
                        }
                        float xr[kD];
                        bool have_x = false;
                        while (near) {
                            const int j = __ffs(near) - 1;
                            near &= near - 1;
                            const int col = col0 + j;
                            if (out.removed_r[mbase + col]) continue;
                            bool hit = (sure >> j) & 1u;
                            if (!hit) {
                                if (!have_x) {
#pragma unroll
                                    for (int k = 0; k < kD; ++k) xr[k] = out.Xr[(mbase + mi) * kD + k];
                                    have_x = true;
                                }
                                hit = cos_at_least<kD>(xr, out.Xr + (mbase + col) * kD, out.c_f, out.thr);
                            }
                            if (hit) {
                                if (ma < 0) ma = out.rank_cand[mbase + mi];
                                const int slot = atomicAdd(&out.conf_deg[mbase + ma], 1);
                                if (slot < kMergeCap) out.conf[(mbase + ma) * kMergeCap + slot] = out.rank_cand[mbase + col];
                            }
                        }
                    }
                    continue;
                }
                // A column can change the best two only if it beats the
                // second best; in increasing column order a tie keeps the
                // lower index as the best.
                if (__any_sync(0xffffffffu, m > b2)) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float sc = __uint_as_float(v[j]);
                        if (sc > b1) {
                            b2 = b1;
                            b1 = sc;
                            i1 = col0 + j;
                        } else if (sc > b2) {
                            b2 = sc;
                        }
                    }
                }
            }
            // Merge the four column slices of each pixel. The 16 score warps
            // meet at a named barrier that also ORs their failure flags, so
            // after a timeout they leave together and none waits there alone.
            xb1[h * 128 + r] = b1;
            xi1[h * 128 + r] = i1;
            xb2[h * 128 + r] = b2;
            uint32_t any_bad;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\t"
                "setp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, %2, p;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(any_bad)
                : "r"(ok ? 0u : 1u), "n"(kLEpi * 32)
                : "memory");
            if (any_bad) break;
            if (kMode == kLbOld && h == 0) {
                const float B1 = fmaxf(fmaxf(xb1[r], xb1[128 + r]), fmaxf(xb1[256 + r], xb1[384 + r]));
                const int i = ii.pt * 128 + r;
                const int64_t base = out.frames ? out.frames[ii.frame].pix0 : 0;
                if (i < ii.n && !out.removed_r[base + i]) {
                    if (B1 >= out.c_f + kDelta) {
                        out.removed_r[base + i] = 1;
                        out.cand_state[base + out.rank_cand[base + i]] = kRemoved;
                    } else if (B1 >= out.c_f - kDelta) {
                        const int slot = atomicAdd(out.fix_count, 1);
                        out.fix[slot] = make_int2(ii.frame, i);
                    }
                }
            } else if (kMode == kLbCover && h == 0) {
                const float B1 = fmaxf(fmaxf(xb1[r], xb1[128 + r]), fmaxf(xb1[256 + r], xb1[384 + r]));
                const int i = ii.pt * 128 + r;
                const int64_t base = out.frames ? out.frames[ii.frame].pix0 : 0;
                bool newly = false;
                if (i < ii.n && !out.covered[base + i]) {
                    if (B1 >= out.c_f + kEpsTc) {
                        out.covered[base + i] = 1;
                        newly = true;
                    } else if (B1 >= out.c_f - kEpsTc) {
                        const int slot = atomicAdd(out.fix_count, 1);
                        out.fix[slot] = make_int2(ii.frame, i);
                    }
                }
                const unsigned nb = __ballot_sync(0xffffffffu, newly);
                if (lane == 0 && nb)
                    atomicSub(out.states ? &out.states[ii.frame].dc.n_uncovered : out.n_uncovered, __popc(nb));
            } else if (kMode == kLbLabel && h == 0) {
                float B1 = xb1[r], B2 = xb2[r];
                int I1 = xi1[r];
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    const float c1 = xb1[k * 128 + r], c2 = xb2[k * 128 + r];
                    const int ci = xi1[k * 128 + r];
                    if (c1 > B1 || (c1 == B1 && ci >= 0 && (I1 < 0 || ci < I1))) {
                        B2 = fmaxf(B1, fmaxf(B2, c2));
                        B1 = c1;
                        I1 = ci;
                    } else {
                        B2 = fmaxf(B2, fmaxf(c1, c2));
                    }
                }
                const int i = ii.pt * 128 + r;
                if (i < ii.n) {
                    const int64_t base = out.frames ? out.frames[ii.frame].pix0 : 0;
                    int32_t* lab = out.labels ? out.labels[ii.frame] : out.labels1;
                    lab[out.pix[base + i]] = I1;
                    if (ii.K > 1 && !(B1 - B2 > 2.f * kEpsTc)) {
                        const int slot = atomicAdd(out.fix_count, 1);
                        out.fix[slot] = make_int2(ii.frame, i);
                    }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kLEpi * 32) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kLWarpMma) tmem_dealloc(tmem, kLTmemCols);
    if (threadIdx.x == 0 && *abort) atomicOr(status, 2);
}

// Near-ties: one warp per queued pixel re-decides its label as the FP32 form
// does. FP32 scores over all modes (lanes stride the modes), the best of
// them, then the FP64 cosine of the raw embedding for every mode within
// 2 * kEpsF32 of that best; the largest wins, the lowest index on ties.
template <int Dp>
__global__ void k_label_fix(const int2* __restrict__ fix, const int* __restrict__ fix_count,
                            const float* __restrict__ P32, const float* __restrict__ modes,
                            const BFrame* __restrict__ frames, const BState* __restrict__ states,
                            const int32_t* __restrict__ pix, const float* __restrict__ emb1, int K1, int d,
                            int32_t* const* __restrict__ labels, int32_t* __restrict__ labels1) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int cnt = *fix_count;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < cnt; e += gridDim.x * wpb) {
        const int2 fi = fix[e];
        const int f = fi.x, i = fi.y;
        const int64_t base = frames ? frames[f].pix0 : 0;
        const int K = states ? states[f].dc.n_kept : K1;
        const float* emb = frames ? frames[f].emb : emb1;
        int32_t* lab = labels ? labels[f] : labels1;
        const float* p = P32 + (base + i) * Dp;
        const float* M = modes + base * Dp;
        float pv[Dp];
#pragma unroll
        for (int k = 0; k < Dp; ++k) pv[k] = p[k];
        float b1 = -INFINITY;
        for (int j = lane; j < K; j += 32) b1 = fmaxf(b1, dot_seq<Dp>(pv, M + (int64_t)j * Dp));
        for (int o = 16; o > 0; o >>= 1) b1 = fmaxf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        const float* em = emb + (int64_t)pix[base + i] * d;
        double bc = -INFINITY;
        int best = K;
        for (int j = lane; j < K; j += 32) {
            const float* m = M + (int64_t)j * Dp;
            if (dot_seq<Dp>(pv, m) < b1 - 2.f * kEpsF32) continue;
            const double cs = cos64(em, m, d);
            if (cs > bc) {
                bc = cs;
                best = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, bc, o);
            const int oi = __shfl_xor_sync(0xffffffffu, best, o);
            if (ob > bc || (ob == bc && oi < best)) {
                bc = ob;
                best = oi;
            }
        }
        if (lane == 0 && best < K) lab[pix[base + i]] = best;
    }
}

// The same decision for one frame, with the mode reads shared: a block takes
// 64 queued pixels at a time and streams the modes through shared memory in
// tiles of 128, four threads per pixel each scoring a quarter of every tile
// (so a mode is read from L2 once per 64 pixels instead of once per pixel).
// Scores, thresholds and the FP64 tie-break are those of k_label_fix.
constexpr int kFixPix = 64, kFixQ = 4, kFixTile = 128;
template <int Dp>
__global__ void __launch_bounds__(kFixPix * kFixQ)
k_label_fix_tiled(const int2* __restrict__ fix, const int* __restrict__ fix_count, const float* __restrict__ P32,
                  const float* __restrict__ M, const int32_t* __restrict__ pix, const float* __restrict__ emb, int K,
                  int d, int32_t* __restrict__ labels) {
    __shared__ __align__(16) float tile[kFixTile * Dp];
    __shared__ float rb[kFixQ][kFixPix];
    __shared__ double rc[kFixQ][kFixPix];
    __shared__ int ri[kFixQ][kFixPix];
    const int cnt = *fix_count;
    const int pl = threadIdx.x % kFixPix, q = threadIdx.x / kFixPix;
    for (int g0 = blockIdx.x * kFixPix; g0 < cnt; g0 += gridDim.x * kFixPix) {
        const int e = g0 + pl;
        const bool live = e < cnt;
        const int i = live ? fix[e].y : 0;
        float pv[Dp];
#pragma unroll
        for (int k = 0; k < Dp; ++k) pv[k] = live ? P32[(int64_t)i * Dp + k] : 0.f;
        // pass 1: best FP32 score
        float b1 = -INFINITY;
        for (int j0 = 0; j0 < K; j0 += kFixTile) {
            const int nt = min(kFixTile, K - j0);
            __syncthreads();
            for (int t = threadIdx.x; t < nt * (Dp / 4); t += blockDim.x)
                reinterpret_cast<float4*>(tile)[t] = reinterpret_cast<const float4*>(M + (int64_t)j0 * Dp)[t];
            __syncthreads();
            for (int j = q; j < nt; j += kFixQ) b1 = fmaxf(b1, dot_seq<Dp>(pv, tile + j * Dp));
        }
        rb[q][pl] = b1;
        __syncthreads();
        b1 = fmaxf(fmaxf(rb[0][pl], rb[1][pl]), fmaxf(rb[2][pl], rb[3][pl]));
        // pass 2: FP64 cosine of the raw embedding for the modes near the best
        const float* em = emb + (int64_t)(live ? pix[i] : 0) * d;
        double bc = -INFINITY;
        int best = K;
        for (int j0 = 0; j0 < K; j0 += kFixTile) {
            const int nt = min(kFixTile, K - j0);
            __syncthreads();
            for (int t = threadIdx.x; t < nt * (Dp / 4); t += blockDim.x)
                reinterpret_cast<float4*>(tile)[t] = reinterpret_cast<const float4*>(M + (int64_t)j0 * Dp)[t];
            __syncthreads();
            if (!live) continue;
            for (int j = q; j < nt; j += kFixQ) {
                if (dot_seq<Dp>(pv, tile + j * Dp) < b1 - 2.f * kEpsF32) continue;
                const double cs = cos64(em, M + (int64_t)(j0 + j) * Dp, d);
                if (cs > bc) {  // j rises within a thread: '>' keeps the lowest index
                    bc = cs;
                    best = j0 + j;
                }
            }
        }
        rc[q][pl] = bc;
        ri[q][pl] = best;
        __syncthreads();
        if (q == 0 && live) {
            for (int o = 1; o < kFixQ; ++o)
                if (rc[o][pl] > bc || (rc[o][pl] == bc && ri[o][pl] < best)) {
                    bc = rc[o][pl];
                    best = ri[o][pl];
                }
            if (best < K) labels[pix[i]] = best;
        }
    }
}

// Mode row `mode` (Dp floats, or nullptr for a padding row) as BF16 split rows
// at row r of Mk: dimensions 0-15, and for Dp = 32 dimensions 16-31 in the
// second array, half_rows rows further (no ones there).
template <int Dp>
__device__ __forceinline__ void pack_mode(const float* mode, uint4* Mk, int64_t r, int64_t half_rows) {
    pack_split_row(mode, Mk + r * 8);
    if (Dp == 32) pack_split_row(mode ? mode + 16 : nullptr, Mk + (half_rows + r) * 8, false);
}

// Modes as BF16 split rows at the frame's Pk row offsets (padding rows hold
// the ones only; their columns are masked out by the score readers).
template <int Dp>
__global__ void k_pack_modes_single(const float* __restrict__ modes, int K, int K_pad, uint4* __restrict__ Mk,
                                    int64_t half_rows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= K_pad) return;
    pack_mode<Dp>(r < K ? modes + (int64_t)r * Dp : nullptr, Mk, r, half_rows);
}

template <int Dp>
__global__ void k_pack_modes_batch(const BFrame* __restrict__ frames, const BState* __restrict__ states,
                                   const float* __restrict__ modes, uint4* __restrict__ Mk, int64_t half_rows) {
    const BFrame& fr = frames[blockIdx.y];
    const int K = states[blockIdx.y].dc.n_kept;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (K + 127) / 128 * 128) return;
    pack_mode<Dp>(r < K ? modes + (fr.pix0 + r) * Dp : nullptr, Mk, fr.pk_row0 + r, half_rows);
}

// Modes [k0, k1) of one frame as BF16 split rows at their Mk rows.
template <int Dp>
__global__ void k_pack_modes_range(const float* __restrict__ modes, int k0, int k1, uint4* __restrict__ Mk,
                                   int64_t half_rows) {
    const int r = k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k1) return;
    pack_mode<Dp>(modes + (int64_t)r * Dp, Mk, r, half_rows);
}

// Coverage of the queued pixels (tensor-core score within kEpsTc of c),
// decided exactly as the FP32 form decides it: one warp per pixel, lanes over
// the new modes; a mode covers the pixel when its FP32 score clears c by
// kEpsF32, or is within kEpsF32 of c and the FP64 cosine of the raw embedding
// reaches c.
template <int Dp>
__global__ void k_cover_fix(const int2* __restrict__ fix, const int* __restrict__ fix_count,
                            const float* __restrict__ P32, const float* __restrict__ modes, int k0, int k1,
                            const int32_t* __restrict__ pix, const float* __restrict__ emb, int d, float c_f, double c,
                            uint8_t* __restrict__ covered, int* __restrict__ n_uncovered) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int cnt = *fix_count;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < cnt; e += gridDim.x * wpb) {
        const int i = fix[e].y;
        float pv[Dp];
#pragma unroll
        for (int k = 0; k < Dp; ++k) pv[k] = P32[(int64_t)i * Dp + k];
        const float* em = emb + (int64_t)pix[i] * d;
        bool cov = false;
        for (int j = k0 + lane; j < k1 && !cov; j += 32) {
            const float* m = modes + (int64_t)j * Dp;
            const float sc = dot_seq<Dp>(pv, m);
            cov = sc >= c_f + kEpsF32 || (sc >= c_f - kEpsF32 && cos64(em, m, d) >= c);
        }
        if (__any_sync(0xffffffffu, cov) && lane == 0) {
            covered[i] = 1;
            atomicSub(n_uncovered, 1);
        }
    }
}

// The batch form of k_pack_modes_range: every frame whose round ended packs
// its new modes [k0, n_kept) at its Mk rows; clears the recheck queue.
template <int Dp>
__global__ void k_pack_modes_new_batch(const BFrame* __restrict__ frames, const BState* __restrict__ states,
                                       const float* __restrict__ modes, uint4* __restrict__ Mk, int64_t half_rows,
                                       int* fix_count) {
    const BFrame& fr = frames[blockIdx.y];
    const BState& st = states[blockIdx.y];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *fix_count = 0;
    if (st.phase != kRoundDone) return;
    const int r = st.k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= st.dc.n_kept) return;
    pack_mode<Dp>(modes + (fr.pix0 + r) * Dp, Mk, fr.pk_row0 + r, half_rows);
}

// k_cover_fix for the batch: queued (frame, foreground index) pairs, each
// against its frame's new modes.
template <int Dp>
__global__ void k_cover_fix_batch(const int2* __restrict__ fix, const int* __restrict__ fix_count,
                                  const float* __restrict__ P32, const float* __restrict__ modes,
                                  const BFrame* __restrict__ frames, BState* states, const int32_t* __restrict__ pix,
                                  int d, float c_f, double c, uint8_t* __restrict__ covered) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int cnt = *fix_count;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < cnt; e += gridDim.x * wpb) {
        const int2 fi = fix[e];
        const int f = fi.x, i = fi.y;
        const BFrame& fr = frames[f];
        const int64_t base = fr.pix0;
        const int k0 = states[f].k0, k1 = states[f].dc.n_kept;
        float pv[Dp];
#pragma unroll
        for (int k = 0; k < Dp; ++k) pv[k] = P32[(base + i) * Dp + k];
        const float* em = fr.emb + (int64_t)pix[base + i] * d;
        bool cov = false;
        for (int j = k0 + lane; j < k1 && !cov; j += 32) {
            const float* m = modes + (base + j) * Dp;
            const float sc = dot_seq<Dp>(pv, m);
            cov = sc >= c_f + kEpsF32 || (sc >= c_f - kEpsF32 && cos64(em, m, d) >= c);
        }
        if (__any_sync(0xffffffffu, cov) && lane == 0) {
            covered[base + i] = 1;
            atomicSub(&states[f].dc.n_uncovered, 1);
        }
    }
}

// The candidates of every frame whose round ended, in rank order (Xr), as
// BF16 split rows at the frame's Pk row offsets; clears the recheck queue.
template <int Dp>
__global__ void k_pack_cands_batch(const BFrame* __restrict__ frames, const BState* __restrict__ states,
                                   const float* __restrict__ Xr, uint4* __restrict__ Ck, int64_t half_rows,
                                   int* fix_count) {
    const BFrame& fr = frames[blockIdx.y];
    const BState& st = states[blockIdx.y];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *fix_count = 0;
    if (st.phase != kRoundDone) return;
    const int k = st.dc.n_cand;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (k + 127) / 128 * 128) return;
    pack_mode<Dp>(r < k ? Xr + (fr.pix0 + r) * Dp : nullptr, Ck, fr.pk_row0 + r, half_rows);
}

// Candidates queued by the tensor-core test against earlier modes (score
// within kDelta of merge_cos), decided exactly as k_b_merge_old decides: one
// warp per candidate, lanes over the frame's earlier modes.
// One frame: frames and states are nullptr, the frame's earlier modes are K1.
template <int Dp>
__global__ void k_merge_old_fix_batch(const int2* __restrict__ fix, const int* __restrict__ fix_count,
                                      const float* __restrict__ Xr, const float* __restrict__ modes,
                                      const BFrame* __restrict__ frames, const BState* __restrict__ states, int K1,
                                      const int32_t* __restrict__ rank_cand, float thr_f, double thr,
                                      uint8_t* __restrict__ cand_state, uint8_t* __restrict__ removed_r) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int cnt = *fix_count;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < cnt; e += gridDim.x * wpb) {
        const int2 fi = fix[e];
        const int64_t base = frames ? frames[fi.x].pix0 : 0;
        const int K = states ? states[fi.x].dc.n_kept : K1;
        float x[Dp];
#pragma unroll
        for (int k = 0; k < Dp; ++k) x[k] = Xr[(base + fi.y) * Dp + k];
        bool hit = false;
        for (int j = lane; j < K && !hit; j += 32) hit = cos_at_least<Dp>(x, modes + (base + j) * Dp, thr_f, thr);
        if (__any_sync(0xffffffffu, hit) && lane == 0) {
            removed_r[base + fi.y] = 1;
            cand_state[base + rank_cand[base + fi.y]] = kRemoved;
        }
    }
}

// One frame's k candidates (rank order, Xr) as BF16 split rows [0, kp).
template <int Dp>
__global__ void k_pack_cands_single(const float* __restrict__ Xr, int k, int kp, uint4* __restrict__ Ck,
                                    int64_t half_rows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= kp) return;
    pack_mode<Dp>(r < k ? Xr + (int64_t)r * Dp : nullptr, Ck, r, half_rows);
}

// Per-frame offsets of the label items (128-pixel tiles); clears the queue.
__global__ void k_label_items(const BFrame* __restrict__ frames, int B, int32_t* __restrict__ off,
                              int* __restrict__ fix_count) {
    if (threadIdx.x != 0) return;
    int t = 0;
    for (int f = 0; f < B; ++f) {
        off[f] = t;
        t += (frames[f].n + 127) / 128;
    }
    off[B] = t;
    *fix_count = 0;
}

template <int D>
ms_status label_tc_setup_dim() {
    constexpr int smem = LbDim<D>::kSmemBytes;
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbSingle, kLbLabel, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbSingle, kLbCover, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbBatch, kLbLabel, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbBatchCover, kLbCover, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbBatchOld, kLbOld, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbBatchPairs, kLbPairs, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbSingleMerge, kLbOld, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    MS_CUDA(cudaFuncSetAttribute(k_label_tc<LbSingleMerge, kLbPairs, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    return MS_OK;
}

template <int Dp>
ms_status merge_tc_single(void* Ck, void* Mk, int64_t n_pad, int k, int K_old, const float* Xr, const float* modes,
                          const int32_t* rank_cand, uint8_t* cand_state, uint8_t* removed_r, int32_t* conf_deg,
                          int32_t* conf, float thr_f, double thr, LabelTcScratch sc, int grid, int* status,
                          cudaStream_t st) {
    MS_CUDA(cudaMemsetAsync(sc.fix_count, 0, sizeof(int), st));
    const int kp = (k + 127) / 128 * 128;
    k_pack_cands_single<Dp><<<(kp + 255) / 256, 256, 0, st>>>(Xr, k, kp, (uint4*)Ck, n_pad);
    MS_LAUNCH("k_pack_cands_single");
    CUtensorMap cmap, cmap1, mmap, mmap1;
    ms_status s = encode_pk_map(Ck, (int)n_pad, &cmap);
    if (s == MS_OK) s = encode_pk_map(Mk, (int)n_pad, &mmap);
    if (s != MS_OK) return s;
    cmap1 = cmap;
    mmap1 = mmap;
    if (Dp == 32 && (s = encode_pk_map((uint8_t*)Ck + n_pad * 128, (int)n_pad, &cmap1)) != MS_OK) return s;
    if (Dp == 32 && (s = encode_pk_map((uint8_t*)Mk + n_pad * 128, (int)n_pad, &mmap1)) != MS_OK) return s;
    LbOut out{};
    out.fix = sc.fix;
    out.fix_count = sc.fix_count;
    out.c_f = thr_f;
    out.Xr = Xr;
    out.removed_r = removed_r;
    out.rank_cand = rank_cand;
    out.cand_state = cand_state;
    out.conf_deg = conf_deg;
    out.conf = conf;
    out.thr = thr;
    if (K_old > 0) {
        LbSingleMerge om{k, K_old, 0};
        k_label_tc<LbSingleMerge, kLbOld, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(cmap, mmap, cmap1, mmap1,
                                                                                            om, out, status);
        MS_LAUNCH("k_label_tc(merge, earlier modes)");
        k_merge_old_fix_batch<Dp><<<grid, 256, 0, st>>>(sc.fix, sc.fix_count, Xr, modes, nullptr, nullptr, K_old,
                                                        rank_cand, thr_f, thr, cand_state, removed_r);
        MS_LAUNCH("k_merge_old_fix");
    }
    LbSingleMerge pm{k, 0, 1};
    k_label_tc<LbSingleMerge, kLbPairs, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(cmap, cmap, cmap1, cmap1,
                                                                                          pm, out, status);
    MS_LAUNCH("k_label_tc(merge, conflicts)");
    return MS_OK;
}

template <int Dp>
ms_status merge_tc_batch(const CUtensorMap& cmap, const CUtensorMap& cmap1, const CUtensorMap& mmap,
                         const CUtensorMap& mmap1, void* Ck, int64_t rows, const BFrame* frames, BState* states, int B,
                         int max_pk_rows, const float* Xr, const float* modes, const int32_t* rank_cand,
                         uint8_t* cand_state, uint8_t* removed_r, int32_t* conf_deg, int32_t* conf, float thr_f,
                         double thr, const int32_t* tile_off, LabelTcScratch sc, int grid, int* status,
                         cudaStream_t st) {
    const dim3 gp((unsigned)((max_pk_rows + 255) / 256), (unsigned)B);
    k_pack_cands_batch<Dp><<<gp, 256, 0, st>>>(frames, states, Xr, (uint4*)Ck, rows, sc.fix_count);
    MS_LAUNCH("k_pack_cands_batch");
    LbOut out{};
    out.frames = frames;
    out.fix = sc.fix;
    out.fix_count = sc.fix_count;
    out.c_f = thr_f;
    out.Xr = Xr;
    out.removed_r = removed_r;
    out.rank_cand = rank_cand;
    out.cand_state = cand_state;
    out.conf_deg = conf_deg;
    out.conf = conf;
    out.thr = thr;
    LbBatchOld om{frames, states, tile_off, B, 0};
    k_label_tc<LbBatchOld, kLbOld, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(cmap, mmap, cmap1, mmap1, om,
                                                                                     out, status);
    MS_LAUNCH("k_label_tc(merge, earlier modes)");
    k_merge_old_fix_batch<Dp><<<grid, 256, 0, st>>>(sc.fix, sc.fix_count, Xr, modes, frames, states, 0, rank_cand,
                                                    thr_f, thr, cand_state, removed_r);
    MS_LAUNCH("k_merge_old_fix_batch");
    LbBatchPairs pm{frames, states, tile_off, B, 0};
    k_label_tc<LbBatchPairs, kLbPairs, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(cmap, cmap, cmap1, cmap1,
                                                                                         pm, out, status);
    MS_LAUNCH("k_label_tc(merge, conflicts)");
    return MS_OK;
}

template <int Dp>
ms_status cover_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                         const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, const BFrame* frames, BState* states,
                         int B, int max_pk_rows, const float* modes, const float* P32, const int32_t* pix, int d,
                         double c, uint8_t* covered, const int32_t* tile_off, LabelTcScratch sc, int grid, int* status,
                         cudaStream_t st) {
    const dim3 gp((unsigned)((max_pk_rows + 255) / 256), (unsigned)B);
    k_pack_modes_new_batch<Dp><<<gp, 256, 0, st>>>(frames, states, modes, (uint4*)Mk, mk_rows, sc.fix_count);
    MS_LAUNCH("k_pack_modes_new_batch");
    const float c_f = (float)c;
    LbBatchCover map{frames, states, tile_off, B, 0};
    LbOut out{nullptr, nullptr, frames, pix, sc.fix, sc.fix_count, covered, nullptr, c_f, states};
    k_label_tc<LbBatchCover, kLbCover, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(pmap, mmap, pmap1, mmap1, map,
                                                                                       out, status);
    MS_LAUNCH("k_label_tc(cover, batch)");
    k_cover_fix_batch<Dp><<<grid, 256, 0, st>>>(sc.fix, sc.fix_count, P32, modes, frames, states, pix, d, c_f, c,
                                                covered);
    MS_LAUNCH("k_cover_fix_batch");
    return MS_OK;
}

template <int Dp>
ms_status cover_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad,
                          const float* modes, int k0, int k1, int n, const float* P32, const int32_t* pix,
                          const float* emb, int d, double c, uint8_t* covered, int* n_uncovered, LabelTcScratch sc,
                          int grid, int* status, cudaStream_t st) {
    MS_CUDA(cudaMemsetAsync(sc.fix_count, 0, sizeof(int), st));
    k_pack_modes_range<Dp><<<(k1 - k0 + 255) / 256, 256, 0, st>>>(modes, k0, k1, (uint4*)Mk, n_pad);
    MS_LAUNCH("k_pack_modes_range");
    CUtensorMap mmap, mmap1;
    ms_status s = encode_pk_map(Mk, (int)n_pad, &mmap);
    if (s != MS_OK) return s;
    mmap1 = mmap;
    if (Dp == 32 && (s = encode_pk_map((uint8_t*)Mk + n_pad * 128, (int)n_pad, &mmap1)) != MS_OK) return s;
    LbSingle map{n, k1};
    map.k0 = k0;
    const float c_f = (float)c;
    LbOut out{nullptr, nullptr, nullptr, pix, sc.fix, sc.fix_count, covered, n_uncovered, c_f, nullptr};
    k_label_tc<LbSingle, kLbCover, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(pmap, mmap, pmap1, mmap1, map, out,
                                                                                   status);
    MS_LAUNCH("k_label_tc(cover)");
    k_cover_fix<Dp><<<grid, 256, 0, st>>>(sc.fix, sc.fix_count, P32, modes, k0, k1, pix, emb, d, c_f, c, covered,
                                          n_uncovered);
    MS_LAUNCH("k_cover_fix");
    return MS_OK;
}

template <int Dp>
ms_status label_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad,
                          const float* modes, int K, int n, const float* P32, const int32_t* pix, const float* emb,
                          int d, int32_t* labels, LabelTcScratch sc, int grid, int* status, cudaStream_t st) {
    MS_CUDA(cudaMemsetAsync(sc.fix_count, 0, sizeof(int), st));
    if (K > 0) {
        const int K_pad = (K + 127) / 128 * 128;
        k_pack_modes_single<Dp><<<(K_pad + 255) / 256, 256, 0, st>>>(modes, K, K_pad, (uint4*)Mk, n_pad);
        MS_LAUNCH("k_pack_modes_single");
    }
    CUtensorMap mmap, mmap1;
    ms_status s = encode_pk_map(Mk, (int)n_pad, &mmap);
    if (s != MS_OK) return s;
    mmap1 = mmap;
    if (Dp == 32 && (s = encode_pk_map((uint8_t*)Mk + n_pad * 128, (int)n_pad, &mmap1)) != MS_OK) return s;
    LbSingle map{n, K};
    LbOut out{nullptr, labels, nullptr, pix, sc.fix, sc.fix_count, nullptr, nullptr, 0.f, nullptr};
    k_label_tc<LbSingle, kLbLabel, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(pmap, mmap, pmap1, mmap1, map,
                                                                                    out, status);
    MS_LAUNCH("k_label_tc");
    if (K > 1) {
        k_label_fix_tiled<Dp><<<2 * grid, kFixPix * kFixQ, 0, st>>>(sc.fix, sc.fix_count, P32, modes, pix, emb, K, d,
                                                                    labels);
        MS_LAUNCH("k_label_fix_tiled");
    }
    return MS_OK;
}

template <int Dp>
ms_status label_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                         const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, const BFrame* frames,
                         const BState* states, int B, int max_pk_rows, const float* modes, const float* P32,
                         const int32_t* pix, int d, int32_t* const* labels, LabelTcScratch sc, int grid, int* status,
                         cudaStream_t st) {
    const dim3 gp((unsigned)((max_pk_rows + 255) / 256), (unsigned)B);
    k_pack_modes_batch<Dp><<<gp, 256, 0, st>>>(frames, states, modes, (uint4*)Mk, mk_rows);
    MS_LAUNCH("k_pack_modes_batch");
    k_label_items<<<1, 32, 0, st>>>(frames, B, sc.off, sc.fix_count);
    MS_LAUNCH("k_label_items");
    LbBatch map{frames, states, sc.off, B, 0};
    LbOut out{labels, nullptr, frames, pix, sc.fix, sc.fix_count, nullptr, nullptr, 0.f, nullptr};
    k_label_tc<LbBatch, kLbLabel, Dp><<<grid, kLThreads, LbDim<Dp>::kSmemBytes, st>>>(pmap, mmap, pmap1, mmap1, map,
                                                                                   out, status);
    MS_LAUNCH("k_label_tc(batch)");
    k_label_fix<Dp><<<grid, 256, 0, st>>>(sc.fix, sc.fix_count, P32, modes, frames, states, pix, nullptr, 0, d, labels,
                                          nullptr);
    MS_LAUNCH("k_label_fix(batch)");
    return MS_OK;
}

}  // namespace

ms_status label_tc_setup() {
    ms_status s = label_tc_setup_dim<16>();
    return s == MS_OK ? label_tc_setup_dim<32>() : s;
}

ms_status launch_merge_tc_batch(const CUtensorMap& cmap, const CUtensorMap& cmap1, const CUtensorMap& mmap,
                                const CUtensorMap& mmap1, void* Ck, int64_t rows, int Dp, const BFrame* frames,
                                BState* states, int B, int max_pk_rows, const float* Xr, const float* modes,
                                const int32_t* rank_cand, uint8_t* cand_state, uint8_t* removed_r, int32_t* conf_deg,
                                int32_t* conf, float thr_f, double thr, const int32_t* tile_off, LabelTcScratch sc,
                                int grid, int* status, cudaStream_t st) {
    return Dp == 32 ? merge_tc_batch<32>(cmap, cmap1, mmap, mmap1, Ck, rows, frames, states, B, max_pk_rows, Xr, modes,
                                         rank_cand, cand_state, removed_r, conf_deg, conf, thr_f, thr, tile_off, sc,
                                         grid, status, st)
                    : merge_tc_batch<16>(cmap, cmap1, mmap, mmap1, Ck, rows, frames, states, B, max_pk_rows, Xr, modes,
                                         rank_cand, cand_state, removed_r, conf_deg, conf, thr_f, thr, tile_off, sc,
                                         grid, status, st);
}

ms_status launch_merge_tc_single(void* Ck, void* Mk, int64_t n_pad, int Dp, int k, int K_old, const float* Xr,
                                 const float* modes, const int32_t* rank_cand, uint8_t* cand_state, uint8_t* removed_r,
                                 int32_t* conf_deg, int32_t* conf, float thr_f, double thr, LabelTcScratch sc,
                                 int grid, int* status, cudaStream_t st) {
    if (k <= 0) return MS_OK;
    return Dp == 32 ? merge_tc_single<32>(Ck, Mk, n_pad, k, K_old, Xr, modes, rank_cand, cand_state, removed_r,
                                          conf_deg, conf, thr_f, thr, sc, grid, status, st)
                    : merge_tc_single<16>(Ck, Mk, n_pad, k, K_old, Xr, modes, rank_cand, cand_state, removed_r,
                                          conf_deg, conf, thr_f, thr, sc, grid, status, st);
}

ms_status launch_cover_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                                const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, int Dp, const BFrame* frames,
                                BState* states, int B, int max_pk_rows, const float* modes, const float* P32,
                                const int32_t* pix, int d, double c, uint8_t* covered, const int32_t* tile_off,
                                LabelTcScratch sc, int grid, int* status, cudaStream_t st) {
    return Dp == 32 ? cover_tc_batch<32>(pmap, mmap, pmap1, mmap1, Mk, mk_rows, frames, states, B, max_pk_rows, modes,
                                         P32, pix, d, c, covered, tile_off, sc, grid, status, st)
                    : cover_tc_batch<16>(pmap, mmap, pmap1, mmap1, Mk, mk_rows, frames, states, B, max_pk_rows, modes,
                                         P32, pix, d, c, covered, tile_off, sc, grid, status, st);
}

ms_status launch_cover_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad, int Dp,
                                 const float* modes, int k0, int k1, int n, const float* P32, const int32_t* pix,
                                 const float* emb, int d, double c, uint8_t* covered, int* n_uncovered,
                                 LabelTcScratch sc, int grid, int* status, cudaStream_t st) {
    if (n == 0 || k1 <= k0) return MS_OK;
    return Dp == 32 ? cover_tc_single<32>(pmap, pmap1, Mk, n_pad, modes, k0, k1, n, P32, pix, emb, d, c, covered,
                                          n_uncovered, sc, grid, status, st)
                    : cover_tc_single<16>(pmap, pmap1, Mk, n_pad, modes, k0, k1, n, P32, pix, emb, d, c, covered,
                                          n_uncovered, sc, grid, status, st);
}

ms_status launch_label_tc_single(const CUtensorMap& pmap, const CUtensorMap& pmap1, void* Mk, int64_t n_pad, int Dp,
                                 const float* modes, int K, int n, const float* P32, const int32_t* pix,
                                 const float* emb, int d, int32_t* labels, LabelTcScratch sc, int grid, int* status,
                                 cudaStream_t st) {
    if (n == 0) return MS_OK;
    return Dp == 32 ? label_tc_single<32>(pmap, pmap1, Mk, n_pad, modes, K, n, P32, pix, emb, d, labels, sc, grid,
                                          status, st)
                    : label_tc_single<16>(pmap, pmap1, Mk, n_pad, modes, K, n, P32, pix, emb, d, labels, sc, grid,
                                          status, st);
}

ms_status launch_label_tc_batch(const CUtensorMap& pmap, const CUtensorMap& mmap, const CUtensorMap& pmap1,
                                const CUtensorMap& mmap1, void* Mk, int64_t mk_rows, int Dp, const BFrame* frames,
                                const BState* states, int B, int max_pk_rows, const float* modes, const float* P32,
                                const int32_t* pix, int d, int32_t* const* labels, LabelTcScratch sc, int grid,
                                int* status, cudaStream_t st) {
    return Dp == 32 ? label_tc_batch<32>(pmap, mmap, pmap1, mmap1, Mk, mk_rows, frames, states, B, max_pk_rows, modes,
                                         P32, pix, d, labels, sc, grid, status, st)
                    : label_tc_batch<16>(pmap, mmap, pmap1, mmap1, Mk, mk_rows, frames, states, B, max_pk_rows, modes,
                                         P32, pix, d, labels, sc, grid, status, st);
}

}  // namespace ms
