// Shift iteration, BF16 tensor-core form (the shift loop of Algorithm 2; Eq. 6-8, 11).
//
// One work item = 128 seeds x a chunk of 128-pixel tiles. Per pixel tile:
//   GEMM1  S' = Xh.Ph + Xh.Pm + Xl.Ph - c       (4 tcgen05 MMAs, FP32 in TMEM)
//          x ~ Xh + Xl and p = Ph + Pm + Pl are round-to-nearest BF16 splits
//          of the FP32 vectors (p's exact) and -c is split into three BF16
//          terms against a ones column, so S' = x.p - c up to the dropped
//          terms (at most 3.04 * 2^-16 = 4.64e-5 for unit vectors: a BF16
//          residual is at most 2^-8 of what it splits) and the tensor cores'
//          FP32 accumulation (at most 51 * 2^-22 = 1.2e-5 even for an adder
//          that truncates; measured <= 6e-6): 5.9e-5 < kBand.
//   mask   a pair is in the window when S' >= 0 (sign bit clear). Pairs with
//          |S'| < kBand = 2^-14 are re-decided with the same sequential FP32
//          dot product as the FP32 form, against the pixel's exact FP32 value
//          rebuilt from its BF16 parts in the shared-memory tile, so every
//          decision equals the FP32 form's, whose dot product is within 1e-6
//          of x.p. Whether a warp holds such a pair comes with the TMEM load
//          of S' (tcgen05.ld.red min.abs: each lane's smallest |S'|), so the
//          mask costs a byte permute and a logic op per two pixels and nothing
//          else.
//   GEMM2  Y += Mask . [Ph | Pm | Pl | 1]    (8 tcgen05 MMAs, mask exact in BF16;
//          the ones column yields the window size)
// The seed-by-pixel matrix lives only in TMEM and registers. After the item's last tile the Y sums are added to the per-seed
// fixed-point accumulators shared with the FP32 form, and the same finalize
// kernel normalises the seeds and tests convergence in FP64.
//
// Warp roles (608 threads, one CTA per SM): warps 0-15 build the mask, four
// warps per 32-lane TMEM quadrant (warp w reaches lanes 32 * (w % 4) + 0..31),
// 32 pixels each, and store it to TMEM, where GEMM2 reads it as its A operand;
// warp 16 issues TMA loads of pixel tiles into an 11-stage ring; warp 17 owns
// TMEM (512 columns: two S, one Y and three mask buffers) and issues GEMM1,
// running ahead of the mask warps as far as the S buffers allow; warp 18
// issues GEMM2 as each mask tile lands. The issuing warps run their loops with
// all 32 lanes and let one elected lane issue each MMA and commit: a loop run
// by lane 0 alone issues the MMAs about 1.5x slower. Seed operands (A1) and S
// are double-buffered, masks triple-buffered (the mask warps would otherwise
// wait for GEMM2's commit round trip), Y single (one item at a time; the next
// item's first GEMM2 waits for the epilogue's read). All waits are bounded; a
// timeout raises the CTA's abort flag, drains what is in flight, frees TMEM
// and reports MS_ERR_TIMEOUT through the frame's status word.
#include <cudaTypedefs.h>

#include "ms_batch.cuh"
#include "ms_device.cuh"
#include "ms_tc.cuh"

#include <type_traits>

namespace ms {
namespace {

using namespace tc;

// Tile shape of a CTA (what the autotuner chooses among). Pixels arrive in
// 128-pixel stages; GEMM1 scores BN of them at a time (a unit: BN = 128, one
// unit per stage, two 128-column S buffers; BN = 64, two units per stage,
// four 64-column S buffers), and the mask of a unit takes BN / 2 TMEM columns
// (three or six mask buffers in 192 columns for d = 16, two or four in 128
// for d = 32). MW mask warps form G
// groups that take turns unit by unit (group k builds the masks of units u
// with u % G == k); each warp builds the mask of 4 * BN / (MW / G) pixels of
// its group's units. Then come the TMA producer, the GEMM1 issuer and NG2
// GEMM2 issuers (NG2 = 2: alternate units, on two sub-partitions).
template <int MW, int NG2, int G, int BN>
struct TcShape {
    static constexpr int kMaskWarps = MW;           // warps 0..MW-1 build the mask
    static constexpr int kGroups = G;
    static constexpr int kGroupWarps = MW / G;      // mask warps per unit
    static constexpr int kBN = BN;                  // pixels per unit
    static constexpr int kUPS = 128 / BN;           // units per 128-pixel stage
    static constexpr int kSBufs = 256 / BN;         // S buffers of BN columns
    static constexpr int kPxPerWarp = 4 * BN / kGroupWarps;  // pixels of a unit per mask warp
    static constexpr int kSub = kPxPerWarp / 32;    // 32-pixel TMEM loads per mask warp and unit
    static constexpr int kWarpTma = MW;
    static constexpr int kWarpG1 = MW + 1;
    static constexpr int kWarpG2 = MW + 2;          // first GEMM2 issuer
    static constexpr int kG2 = NG2;
    static constexpr int kThreads = (MW + 2 + NG2) * 32;
    static_assert(BN == 128 || BN == 64, "GEMM1 unit of 128 or 64 pixels");
    static_assert(MW % G == 0 && kGroupWarps % 4 == 0 && kPxPerWarp % 32 == 0 && kPxPerWarp >= 32,
                  "each group's mask warps cover the four TMEM quadrants evenly");
    static_assert(NG2 == 1 || NG2 == 2, "one or two GEMM2 issuers");
};
// Index = ms_config.tc_shape.
using TcShape0 = TcShape<16, 2, 1, 128>;
using TcShape1 = TcShape<16, 1, 1, 128>;
using TcShape2 = TcShape<8, 2, 1, 128>;
using TcShape3 = TcShape<8, 1, 1, 128>;
using TcShape4 = TcShape<16, 2, 2, 128>;
using TcShape5 = TcShape<16, 1, 2, 128>;
using TcShape6 = TcShape<16, 2, 2, 64>;
using TcShape7 = TcShape<16, 1, 2, 64>;
constexpr int kTileBytes = 128 * 128;  // 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxSBufs = 4, kMaxMBufs = 6;
constexpr uint32_t kColS = 0;          // S accumulators, 256 columns
constexpr uint32_t kColY = 256;        // Y accumulators: 64 columns per 16-dimensional half
constexpr float kBand = 6.103515625e-05f;    // 2^-14
constexpr float kFixScale = 68719476736.0f;  // 2^36

// Layout for embedding dimension D: 16, or 32 as two 16-dimensional halves,
// each with its own seed-operand tile, pixel tile (a second Pk array) and Y
// block; the mask buffers take the TMEM columns after Y.
template <int D>
struct TcDim {
    static_assert(D == 16 || D == 32, "embedding dimension 16 or 32");
    static constexpr int kHalves = D / 16;
    static constexpr int kStages = D == 16 ? 10 : 4;              // pixel-tile ring
    static constexpr int kStageBytes = kHalves * kTileBytes;
    static constexpr int kOffA1 = 0;                              // 2 items x kHalves x 16 KB
    static constexpr int kOffP = 2 * kHalves * kTileBytes;        // kStages stages
    static constexpr int kOffX = kOffP + kStages * kStageBytes;   // 2 x 128 x D floats: the item's seeds
    static constexpr int kOffBar = kOffX + 2 * 128 * D * 4;
    static constexpr int kNumBars = 2 * kStages + 2 * kMaxSBufs + 2 * kMaxMBufs + 2 + 2 + 3;  // aux: GEMM1 + two GEMM2
    static constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 32 + 1024;  // + TMEM slot, flags, alignment slack
    static constexpr uint32_t kColM = kColY + 64 * kHalves;       // mask buffers up to column 512
    static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

struct TcSplit {
    int tiles, chunks, tpc;  // seed tiles, pixel chunks, pixel tiles per chunk
};

__device__ __forceinline__ TcSplit tc_split(int n_active, int n_ptiles, int target, int grid) {
    TcSplit s;
    s.tiles = (n_active + 127) / 128;
    if (s.tiles == 0 || n_ptiles == 0) {
        s.chunks = 0;
        s.tpc = 1;
        return s;
    }
    s.tpc = tc_tiles_per_chunk(s.tiles, n_ptiles, target, grid);
    s.chunks = (n_ptiles + s.tpc - 1) / s.tpc;
    return s;
}

// Bounded wait that ignores the abort flag (used while draining).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

// Bytes {0,1} = sign of a, {2,3} = sign of b, replicated: 0xFFFF per negative half.
__device__ __forceinline__ uint32_t sign_halves(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Row r of one 16-dimensional half of a seed operand tile:
// [Xh | Xl | -c split | 0] for the first half, [Xh | Xl | 0 | 0] for the
// second (the -c column is added once), 128-byte swizzle.
__device__ __forceinline__ void write_a1_half(uint8_t* A1, int r, const float* x, float c_f, bool with_c) {
    uint32_t wh[8], wl[8];
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        const float h0 = bf16_round(x[k]), h1 = bf16_round(x[k + 1]);
        wh[k / 2] = pack_bf16(h0, h1);
        wl[k / 2] = pack_bf16(x[k] - h0, x[k + 1] - h1);
    }
    const float c_hi = bf16_round(c_f);
    const float c_mid = bf16_round(c_f - c_hi);
    const float c_lo = (c_f - c_hi) - c_mid;
    const uint32_t wc0 = with_c ? pack_bf16(-c_hi, -c_mid) : 0u, wc1 = with_c ? pack_bf16(-c_lo, 0.f) : 0u;
    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, 0)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, 1)) = make_uint4(wh[4], wh[5], wh[6], wh[7]);
    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, 2)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, 3)) = make_uint4(wl[4], wl[5], wl[6], wl[7]);
    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, 4)) = make_uint4(wc0, wc1, 0u, 0u);
#pragma unroll
    for (int cidx = 5; cidx < 8; ++cidx)
        *reinterpret_cast<uint4*>(A1 + sw128_offset(r, cidx)) = make_uint4(0u, 0u, 0u, 0u);
}

// Row r of an item's seed operand (one 16 KB tile per 16-dimensional half)
// and of its FP32 seed tile in shared memory, for seed slot `slot` of X
// (D components; a padding row, slot < 0: zeros), one half at a time.
template <int D>
__device__ __forceinline__ void write_seed_rows(uint8_t* A1, float* Xs, int r, const float* __restrict__ X, int slot,
                                                float c_f) {
#pragma unroll
    for (int hf = 0; hf < D / 16; ++hf) {
        float x[16];
#pragma unroll
        for (int k = 0; k < 16; k += 4) {
            const float4 v = slot >= 0 ? *reinterpret_cast<const float4*>(X + (int64_t)slot * D + 16 * hf + k)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
            *reinterpret_cast<float4*>(Xs + r * D + 16 * hf + k) = v;
        }
        write_a1_half(A1 + hf * kTileBytes, r, x, c_f, hf == 0);
    }
}

// What a work item covers, in the frame it belongs to.
struct TcItem {
    const int32_t* active;  // seed slots of the frame's active list
    int n_active;           // length of that list
    int seed0;              // list position of the item's first seed
    int pt0, pt1;           // the frame's 128-pixel tiles [pt0, pt1)
    int pk_row0;            // Pk row of the frame's pixel 0 (multiple of 128)
    int64_t pix0;           // P32 row of the frame's pixel 0
    int n;                  // the frame's pixel count
};

// Work items of one frame: seed tiles of 128 x chunks of 128-pixel tiles.
struct TcSingleMap {
    const int32_t* active;
    const DevCounters* dc;
    int n, n_ptiles, target;
    int n_active;
    TcSplit sp;
    __device__ __forceinline__ bool init() {
        if (dc->done) return false;
        n_active = dc->n_active;
        sp = tc_split(n_active, n_ptiles, target, (int)gridDim.x);
        return true;
    }
    __device__ __forceinline__ int total() const { return sp.tiles * sp.chunks; }
    __device__ __forceinline__ TcItem item(int i) const {
        const int t = i / sp.chunks, ch = i - t * sp.chunks;
        const int pt0 = ch * sp.tpc;
        TcItem it;
        it.active = active;
        it.n_active = n_active;
        it.seed0 = t * 128;
        it.pt0 = pt0;
        it.pt1 = min(n_ptiles, pt0 + sp.tpc);
        it.pk_row0 = 0;
        it.pix0 = 0;
        it.n = n;
        return it;
    }
};

// FP32 value of pixel row `row` of a 16-dimensional pixel stage, rebuilt
// exactly from its three BF16 parts (h + m) + l: the split of an FP32 value
// into three round-to-nearest BF16 terms is exact, and so is this sum.
__device__ __forceinline__ void stage_pixel16(const uint8_t* stage, int row, float (&p)[16]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint4 hv = *reinterpret_cast<const uint4*>(stage + sw128_offset(row, c));
        const uint4 mv = *reinterpret_cast<const uint4*>(stage + sw128_offset(row, c + 2));
        const uint4 lv = *reinterpret_cast<const uint4*>(stage + sw128_offset(row, c + 4));
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, mw[4] = {mv.x, mv.y, mv.z, mv.w},
                       lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            p[c * 8 + 2 * k] = __fadd_rn(__fadd_rn(__uint_as_float(hw[k] << 16), __uint_as_float(mw[k] << 16)),
                                         __uint_as_float(lw[k] << 16));
            p[c * 8 + 2 * k + 1] =
                __fadd_rn(__fadd_rn(__uint_as_float(hw[k] & 0xFFFF0000u), __uint_as_float(mw[k] & 0xFFFF0000u)),
                          __uint_as_float(lw[k] & 0xFFFF0000u));
        }
    }
}

// Dot product, in FP32 with one FMA per component in component order (the
// FP32 form's dot_seq, bit for bit), of seed x (D floats in shared memory)
// with pixel row `row` of a pixel stage (D / 16 tiles of 16 dimensions). The
// pixel is rebuilt exactly from its three BF16 parts (h + m) + l: the split of
// an FP32 value into three round-to-nearest BF16 terms is exact, and so is
// this sum.
template <int D>
__device__ __forceinline__ float stage_dot(const uint8_t* stage, int row, const float* x) {
    float acc = 0.f;
#pragma unroll
    for (int hf = 0; hf < D / 16; ++hf) {
        const uint8_t* t = stage + hf * kTileBytes;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint4 hv = *reinterpret_cast<const uint4*>(t + sw128_offset(row, c));
            const uint4 mv = *reinterpret_cast<const uint4*>(t + sw128_offset(row, c + 2));
            const uint4 lv = *reinterpret_cast<const uint4*>(t + sw128_offset(row, c + 4));
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, mw[4] = {mv.x, mv.y, mv.z, mv.w},
                           lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float p0 = __fadd_rn(__fadd_rn(__uint_as_float(hw[k] << 16), __uint_as_float(mw[k] << 16)),
                                           __uint_as_float(lw[k] << 16));
                const float p1 =
                    __fadd_rn(__fadd_rn(__uint_as_float(hw[k] & 0xFFFF0000u), __uint_as_float(mw[k] & 0xFFFF0000u)),
                              __uint_as_float(lw[k] & 0xFFFF0000u));
                acc = fmaf(x[16 * hf + c * 8 + 2 * k], p0, acc);
                acc = fmaf(x[16 * hf + c * 8 + 2 * k + 1], p1, acc);
            }
        }
    }
    return acc;
}

// Warp-uniform bounded wait: every lane polls, all lanes get the same answer.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

template <class Shape, int kD, bool kDebug, class Map>
__global__ void __launch_bounds__(Shape::kThreads, 1)
k_shift_tc(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap pmap1,
           const float* __restrict__ P32, const float* __restrict__ X, unsigned long long* __restrict__ acc, float c_f,
           Map map, int* status, unsigned long long* band_ctr, float* __restrict__ dbg_S, int64_t dbg_stride) {
    using L = TcDim<kD>;
    constexpr int kHalves = L::kHalves, kStages = L::kStages, kStageBytes = L::kStageBytes;
    constexpr uint32_t kColM = L::kColM;
    constexpr int kGroups = Shape::kGroups, kGroupWarps = Shape::kGroupWarps;
    constexpr int kBN = Shape::kBN, kUPS = Shape::kUPS, kSBufs = Shape::kSBufs;
    constexpr int kMBufs = (int)(kTmemCols - kColM) / (kBN / 2);  // mask buffers of BN / 2 columns
    static_assert(kMBufs >= 2 && kMBufs <= kMaxMBufs, "mask buffers");
    constexpr int kPxPerWarp = Shape::kPxPerWarp, kSub = Shape::kSub;
    constexpr int kWarpTma = Shape::kWarpTma, kWarpG1 = Shape::kWarpG1, kWarpG2 = Shape::kWarpG2, kG2 = Shape::kG2;
    // GEMM2 issuers commit a stage's release after their last unit of it.
    constexpr int kEmptyArrivals = kUPS < kG2 ? kUPS : kG2;
    if (!map.init()) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* A1 = smem + L::kOffA1;               // [item buffer][half] 16 KB tiles
    uint8_t* Pst = smem + L::kOffP;
    float* Xs = (float*)(smem + L::kOffX);        // [2][128][kD] seeds of an item (FP32 re-decisions)
    uint64_t* bars = (uint64_t*)(smem + L::kOffBar);
    uint64_t* full = bars;                        // [kStages] pixel tile landed
    uint64_t* empty = full + kStages;             // [kStages] pixel tile consumed by GEMM2
    uint64_t* s_full = empty + kStages;           // [kSBufs] GEMM1 of a unit done
    uint64_t* s_empty = s_full + kMaxSBufs;       // [kSBufs] S read by the mask warps of the unit's group
    uint64_t* m_full = s_empty + kMaxSBufs;       // [kMBufs] mask of a unit stored to TMEM by its group's warps
    uint64_t* m_empty = m_full + kMaxMBufs;       // [kMBufs] mask consumed by GEMM2
    uint64_t* a1_full = m_empty + kMaxMBufs;      // [2] seed operand written
    uint64_t* d_full = a1_full + 2;               // Y of an item complete
    uint64_t* d_empty = d_full + 1;               // Y read by the epilogue
    uint64_t* aux = d_empty + 1;                  // [1 + kG2] drain barriers of the MMA issuers
    uint32_t* tmem_slot = (uint32_t*)(bars + L::kNumBars);
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    volatile int* g2_next = (volatile int*)(tmem_slot + 2);  // the next unit whose GEMM2 may be issued

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kEmptyArrivals);
        }
        for (int b = 0; b < kSBufs; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_empty[b], kGroupWarps);
        }
        for (int b = 0; b < 2; ++b) mbar_init(&a1_full[b], 128);
        for (int b = 0; b < kMBufs; ++b) {
            mbar_init(&m_full[b], kGroupWarps);
            mbar_init(&m_empty[b], 1);
        }
        mbar_init(d_full, kG2);  // every GEMM2 issuer commits at an item's end
        mbar_init(d_empty, 128);
        for (int k = 0; k <= kG2; ++k) mbar_init(&aux[k], 1);
        *abort = 0;
        *g2_next = 0;
        fence_mbar_init();
    }
    if (warp == kWarpTma && lane == 0) {
        tma_prefetch_desc(&pmap);
        if (kHalves > 1) tma_prefetch_desc(&pmap1);
    }
    if (warp == kWarpG1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int items = map.total();

    if (warp == kWarpTma) {
        // ------------------------------------------------ TMA producer
        // The three issuing warps run their loops with all 32 lanes (waits
        // are warp-uniform) and one lane issues; see mma_bf16_warp.
        int g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const TcItem ii = map.item(item);
            for (int pt = ii.pt0; pt < ii.pt1; ++pt, ++g) {
                const int s = g % kStages;
                if (g >= kStages && !(ok = warp_wait(&empty[s], ((g / kStages) - 1) & 1, abort))) break;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], kStageBytes);
                    tma_load_2d(Pst + s * kStageBytes, &pmap, 0, ii.pk_row0 + pt * 128, &full[s]);
                    if (kHalves > 1)
                        tma_load_2d(Pst + s * kStageBytes + kTileBytes, &pmap1, 0, ii.pk_row0 + pt * 128, &full[s]);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && *abort)
            for (int q = max(0, g - kStages); q < g; ++q) drain_wait(&full[q % kStages], (q / kStages) & 1);
    } else if (warp == kWarpG1) {
        // ------------------------------------------------ GEMM1 issuer
        // Runs ahead of the mask warps as far as the S buffers allow.
        // Descriptors are built once; moving an operand by b bytes adds b >> 4
        // to the descriptor's start-address field (no carry: shared addresses
        // stay below 2^18).
        const uint64_t dA1 = desc_sw128(smem_u32(A1), 16, 1024);   // seed operand, K-major
        const uint64_t dP1 = desc_sw128(smem_u32(Pst), 16, 1024);  // pixel tile, K-major
        constexpr uint32_t id1 = idesc_bf16(128, kBN, 0, 0);
        constexpr uint64_t kT = kTileBytes >> 4;
        constexpr uint64_t kU = (kBN * 128) >> 4;  // one unit of pixel rows
        bool ok = true;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            const TcItem ii = map.item(item);
            if (!(ok = warp_wait(&a1_full[it & 1], (it >> 1) & 1, abort))) break;
            const uint64_t a = dA1 + (uint64_t)(it & 1) * kHalves * kT;
            for (int pt = ii.pt0; pt < ii.pt1 && ok; ++pt, ++g) {
                const int s = g % kStages;
                if (!(ok = warp_wait(&full[s], (g / kStages) & 1, abort))) break;
#pragma unroll
                for (int hh = 0; hh < kUPS; ++hh) {
                    const int u = g * kUPS + hh, b = u % kSBufs;
                    if (u >= kSBufs && !(ok = warp_wait(&s_empty[b], ((u / kSBufs) - 1) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t tS = tmem + kColS + b * kBN;
                    const uint64_t pb = dP1 + (uint64_t)s * kHalves * kT + hh * kU;
                    mma_bf16_warp(tS, a, pb, id1, 0);            // Xh . Ph
                    mma_bf16_warp(tS, a, pb + 2, id1, 1);        // Xh . Pm
                    mma_bf16_warp(tS, a + 2, pb, id1, 1);        // Xl . Ph
                    mma_bf16_warp(tS, a + 4, pb + 6, id1, 1);    // -c split . ones
                    if (kHalves > 1) {                           // dimensions 16..31
                        mma_bf16_warp(tS, a + kT, pb + kT, id1, 1);
                        mma_bf16_warp(tS, a + kT, pb + kT + 2, id1, 1);
                        mma_bf16_warp(tS, a + kT + 2, pb + kT, id1, 1);
                    }
                    mma_commit_warp(&s_full[b]);
                }
            }
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[0]);
            drain_wait(&aux[0], 0);
        }
    } else if (warp >= kWarpG2 && warp < kWarpG2 + kG2) {
        // ------------------------------------------------ GEMM2 issuers
        // Y += Mask . P as soon as a unit's mask is in TMEM; the pixel stage
        // is released when the MMAs of its units complete. With two issuers,
        // warps on different sub-partitions take alternate units, so neither
        // sub-partition's mask warps carry all of GEMM2's issue cost. Y
        // accumulates in unit order: a warp issues unit u only after unit u-1
        // was issued (g2_next, with tcgen05 fences around the hand-over).
        // Each warp commits the releases of the units it issued (a stage's
        // release after its last unit of that stage), and every issuer commits
        // d_full at an item's end (a commit covers only its own thread's MMAs).
        const int par = warp - kWarpG2;
        const uint64_t dP2 = desc_sw128(smem_u32(Pst), kTileBytes, 1024);  // pixel tile, MN-major
        constexpr uint32_t id2 = idesc_bf16(128, 64, 0, 1);
        constexpr uint64_t kT = kTileBytes >> 4;
        constexpr int kK2 = kBN / 16;  // K = 16 pixels per MMA
        bool ok = true;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            const TcItem ii = map.item(item);
            for (int pt = ii.pt0; pt < ii.pt1 && ok; ++pt, ++g) {
#pragma unroll
                for (int hh = 0; hh < kUPS; ++hh) {
                    const int u = g * kUPS + hh;
                    if (u % kG2 != par) continue;
                    const int s = g % kStages, mb = u % kMBufs;
                    const bool first = pt == ii.pt0 && hh == 0;
                    if (!(ok = warp_wait(&m_full[mb], (u / kMBufs) & 1, abort))) break;
                    if (!(ok = warp_wait(&full[s], (g / kStages) & 1, abort))) break;
                    if (first && it >= 1 && !(ok = warp_wait(d_empty, (it - 1) & 1, abort))) break;
                    if constexpr (kG2 > 1) {
                        const long long t0 = clock64();
                        bool turn = true;
                        while (*g2_next != u) {
                            if (*abort || clock64() - t0 > kWaitCycles) {
                                *abort = 1;
                                turn = false;
                                break;
                            }
                        }
                        if (!(ok = __all_sync(0xffffffffu, turn))) break;
                    }
                    tc_fence_after();
                    const uint32_t tM = tmem + kColM + mb * (kBN / 2);
#pragma unroll
                    for (int hf = 0; hf < kHalves; ++hf) {
                        const uint32_t tY = tmem + kColY + 64 * hf;
                        const uint64_t pb = dP2 + (uint64_t)(s * kHalves + hf) * kT + hh * kK2 * 128;
#pragma unroll
                        for (int k = 0; k < kK2; ++k)
                            mma_bf16_ts_warp(tY, tM + 8 * k, pb + k * 128, id2, (first && k == 0) ? 0u : 1u);
                    }
                    mma_commit_warp(&m_empty[mb]);
                    if (hh >= kUPS - kG2) mma_commit_warp(&empty[s]);
                    if constexpr (kG2 > 1) {  // one thread's MMAs execute in issue order: no hand-over
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) {
                            __threadfence_block();
                            *g2_next = u + 1;
                        }
                    }
                }
            }
            if (!ok) break;
            mma_commit_warp(d_full);
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[1 + par]);
            drain_wait(&aux[1 + par], 0);
        }
    } else {
        // ------------------------------------------------ mask warps
        // Group grp of kGroups takes the units u with u % kGroups == grp; in a
        // group, warp w reaches TMEM lanes 32 * (w % 4) + 0..31 (its seeds) and
        // builds the mask of kPxPerWarp pixels of the unit, 32 at a time.
        const int grp = warp / kGroupWarps;
        const int q = warp & 3;                         // TMEM lane quadrant
        const int h = (warp % kGroupWarps) >> 2;        // which kPxPerWarp pixels of a tile
        const bool lead = warp < 4;                     // writes the seed operand and reads Y
        const int r = q * 32 + lane;                    // seed row
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        // One group: the mask is stored once per tile. Two groups (64 pixels
        // per warp): each 32-pixel part of the mask is stored as soon as it
        // is built, which keeps fewer registers live.
        constexpr bool kEarlyStore = kGroups > 1;
        long long band_local = 0;
        int g = 0, it = 0;
        int mbn = 0, mphn = 0;  // mask buffer of tile g and its phase, kept without divisions
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
            if (__any_sync(0xffffffffu, *abort)) break;
            const TcItem ii = map.item(item);
            const int pt0 = ii.pt0, pt1 = ii.pt1;
            const int pos = ii.seed0 + r;
            const int slot = pos < ii.n_active ? ii.active[pos] : -1;
            if (lead) {
                // A1 for this item (first item only) and the next one; the next
                // one's buffer was last read by the GEMM1s of item it-1, which
                // completed before this warp observed s_full of that item's
                // last tile (a commit covers every earlier MMA of its thread).
                if (it == 0) {
                    write_seed_rows<kD>(A1, Xs, r, X, slot, c_f);
                    fence_proxy_async();
                    mbar_arrive(&a1_full[0]);
                }
                const int nitem = item + gridDim.x;
                if (nitem < items) {
                    const TcItem ni = map.item(nitem);
                    const int npos = ni.seed0 + r;
                    write_seed_rows<kD>(A1 + ((it + 1) & 1) * kHalves * kTileBytes, Xs + ((it + 1) & 1) * 128 * kD, r, X,
                                        npos < ni.n_active ? ni.active[npos] : -1, c_f);
                    fence_proxy_async();
                    mbar_arrive(&a1_full[(it + 1) & 1]);
                }
            }
            // The item's seeds in shared memory: written by the lead warps
            // before their a1_full arrival (at the start of the previous item,
            // after every mask warp had finished the item before it).
            bool ok = warp_wait(&a1_full[it & 1], (it >> 1) & 1, abort);
            const float* xs = Xs + (it & 1) * 128 * kD + r * kD;
            for (int pt = pt0; pt < pt1 && ok; ++pt, ++g) {
#pragma unroll
                for (int hh = 0; hh < kUPS; ++hh) {
                    const int u = g * kUPS + hh;  // unit: BN pixels of stage g
                    const int mb = mbn, mph = mphn;
                    if (++mbn == kMBufs) {
                        mbn = 0;
                        mphn ^= 1;
                    }
                    if (kGroups > 1 && u % kGroups != grp) continue;
                    const int b = u % kSBufs;
                    if (!(ok = warp_wait(&s_full[b], (u / kSBufs) & 1, abort))) break;
                    tc_fence_after();
                    uint32_t w[kEarlyStore ? 1 : kSub][16];
                    bool staged = false;  // pixel stage known to be complete (band path)
#pragma unroll
                    for (int j = 0; j < kSub; ++j) {
                        uint32_t (&wj)[16] = w[kEarlyStore ? 0 : j];
                        uint32_t v[32];
                        float mn;
                        tmem_ld32_minabs(tmem + kColS + b * kBN + lane_base + h * kPxPerWarp + j * 32, v, &mn);
                        tmem_ld_wait();
                        if (j == kSub - 1) {  // S read: hand the buffer back to GEMM1
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&s_empty[b]);
                        }
#pragma unroll
                        for (int i = 0; i < 16; ++i) wj[i] = ~sign_halves(v[2 * i], v[2 * i + 1]) & 0x3F803F80u;
                        if (__any_sync(0xffffffffu, mn < kBand)) {
                            // Re-decide near-boundary pairs with the FP32 form's dot
                            // product against the exact FP32 pixel rebuilt from the
                            // tile in shared memory. Bit masks keep register-array
                            // indices static.
                            const int s = g % kStages;
                            if (!staged && !(ok = warp_wait(&full[s], (g / kStages) & 1, abort))) break;
                            staged = true;
                            const uint8_t* stage = Pst + s * kStageBytes;
                            uint32_t bandm = 0;
#pragma unroll
                            for (int i = 0; i < 32; ++i) bandm |= (uint32_t)(fabsf(__uint_as_float(v[i])) < kBand) << i;
                            uint32_t inm = 0, todo = bandm;
                            while (todo) {
                                const int i = __ffs(todo) - 1;
                                todo &= todo - 1;
                                const int row = hh * kBN + h * kPxPerWarp + j * 32 + i;
                                if (pt * 128 + row < ii.n) {
                                    ++band_local;
                                    // xs: the seed (a padding row: zeros)
                                    float d;
                                    if constexpr (kD == 16) {
                                        float x[16], pv[16];
#pragma unroll
                                        for (int k = 0; k < 16; k += 4) {
                                            const float4 t4 = *reinterpret_cast<const float4*>(xs + k);
                                            x[k] = t4.x; x[k + 1] = t4.y; x[k + 2] = t4.z; x[k + 3] = t4.w;
                                        }
                                        stage_pixel16(stage, row, pv);
                                        d = dot_seq<16>(x, pv);
                                    } else {
                                        d = stage_dot<kD>(stage, row, xs);
                                    }
                                    if (d >= c_f) inm |= 1u << i;
                                }
                            }
#pragma unroll
                            for (int k = 0; k < 16; ++k) {
                                const uint32_t bm = (bandm >> (2 * k)) & 3u;
                                const uint32_t im = (inm >> (2 * k)) & 3u;
                                const uint32_t clear = ((bm & 1u) ? 0x3F80u : 0u) | ((bm & 2u) ? 0x3F800000u : 0u);
                                const uint32_t set = ((im & 1u) ? 0x3F80u : 0u) | ((im & 2u) ? 0x3F800000u : 0u);
                                wj[k] = (wj[k] & ~clear) | set;
                            }
                        }
                        if (kDebug) {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                dbg_S[(int64_t)r * dbg_stride + pt * 128 + hh * kBN + h * kPxPerWarp + j * 32 + i] =
                                    __uint_as_float(v[i]);
                        }
                        if constexpr (kEarlyStore) {
                            if (j == 0) {
                                if (u >= kMBufs && !(ok = warp_wait(&m_empty[mb], mph ^ 1, abort))) break;
                                tc_fence_after();
                            }
                            tmem_st16(tmem + kColM + mb * (kBN / 2) + lane_base + h * (kPxPerWarp / 2) + j * 16, wj);
                        }
                    }
                    if (!ok) break;
                    if constexpr (!kEarlyStore) {
                        if (u >= kMBufs && !(ok = warp_wait(&m_empty[mb], mph ^ 1, abort))) break;
                        tc_fence_after();
#pragma unroll
                        for (int j = 0; j < kSub; ++j)
                            tmem_st16(tmem + kColM + mb * (kBN / 2) + lane_base + h * (kPxPerWarp / 2) + j * 16, w[j]);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&m_full[mb]);
                }
            }
            if (!ok) break;
            if (lead) {
                if (!warp_wait(d_full, it & 1, abort)) break;
                tc_fence_after();
                // Y: per half [sum ph | sum pm | sum pl | count] (the count in
                // half 0); Y is handed back after the last half's load, the
                // sums go out as fixed-point reductions half by half
                const uint32_t ty = tmem + kColY + lane_base;
                bool live = false;
#pragma unroll
                for (int hf = 0; hf < kHalves; ++hf) {
                    uint32_t yh[16], ym[16], yl[16];
                    tmem_ld16(ty + 64 * hf, yh);
                    tmem_ld16(ty + 64 * hf + 16, ym);
                    tmem_ld16(ty + 64 * hf + 32, yl);
                    float cntf = 0.f;
                    if (hf == 0) {
                        uint32_t yc[16];
                        tmem_ld16(ty + 48, yc);
                        tmem_ld_wait();
                        cntf = __uint_as_float(yc[0]);
                        live = slot >= 0 && cntf > 0.f;
                    } else {
                        tmem_ld_wait();
                    }
                    if (hf == kHalves - 1) {
                        tc_fence_before();
                        mbar_arrive(d_empty);
                    }
                    if (live) {
                        unsigned long long* a = acc + (int64_t)slot * (kD + 1);
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const float y = __uint_as_float(yh[k]) + __uint_as_float(ym[k]) + __uint_as_float(yl[k]);
                            atomicAdd(a + 16 * hf + k, (unsigned long long)__float2ll_rn(y * kFixScale));
                        }
                        if (hf == 0) atomicAdd(a + kD, (unsigned long long)__float2ll_rn(cntf));
                    }
                }
            }
        }
        if (band_local) atomicAdd(band_ctr, (unsigned long long)band_local);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kWarpG1) tmem_dealloc(tmem, kTmemCols);
    if (threadIdx.x == 0 && *abort) atomicOr(status, 2);
}

// Pixels as BF16 splits for the tensor cores: row i = [Ph | Pm | Pl | 1 1 1 0..0]
// (64 values, 128 bytes) with p = Ph + Pm + Pl; rows from the foreground count
// n (read on the device) up to `rows` hold only the ones, so they score
// S' = -c and never enter a window. For D = 32 a second array of `rows` rows
// follows, holding dimensions 16..31 the same way without the ones.
__global__ void k_pack_bf16(const float* __restrict__ P32, const DevCounters* __restrict__ dc, int rows, int D,
                            uint4* __restrict__ Pk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const bool fg = i < dc->n_fg;
    pack_split_row(fg ? P32 + (int64_t)i * D : nullptr, Pk + (int64_t)i * 8);
    if (D == 32) pack_split_row(fg ? P32 + (int64_t)i * D + 16 : nullptr, Pk + ((int64_t)rows + i) * 8, false);
}

ms_status encode_pmap(void* Pk, int n_pad, CUtensorMap* map) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult qr;
        void* fn = nullptr;
        MS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr));
        if (qr != cudaDriverEntryPointSuccess || !fn)
            return set_error(MS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {64, (cuuint64_t)n_pad};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Pk, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MS_OK;
}

// Calls fn with a value of the shape type that `shape` (ms_config.tc_shape) names.
template <class Fn>
ms_status with_tc_shape(int shape, Fn&& fn) {
    switch (shape) {
        case 0: return fn(TcShape0{});
        case 1: return fn(TcShape1{});
        case 2: return fn(TcShape2{});
        case 3: return fn(TcShape3{});
        case 4: return fn(TcShape4{});
        case 5: return fn(TcShape5{});
        case 6: return fn(TcShape6{});
        case 7: return fn(TcShape7{});
        default: return set_error(MS_ERR_INVALID_ARG, "unknown tile shape %d", shape);
    }
}

template <class Map, int D>
ms_status allow_smem_all_shapes() {
    const auto f = [](auto sh) -> ms_status {
        using Sh = decltype(sh);
        MS_CUDA(cudaFuncSetAttribute(k_shift_tc<Sh, D, false, Map>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TcDim<D>::kSmemBytes));
        if constexpr (std::is_same_v<Map, TcSingleMap> && D == 16)  // the score dump is a d = 16 self-test
            MS_CUDA(cudaFuncSetAttribute(k_shift_tc<Sh, D, true, Map>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcDim<D>::kSmemBytes));
        return MS_OK;
    };
    for (int k = 0; k < kTcShapes; ++k)
        if (ms_status st = with_tc_shape(k, f); st != MS_OK) return st;
    return MS_OK;
}

}  // namespace

int tc_smem_bytes(int D) { return D == 32 ? TcDim<32>::kSmemBytes : TcDim<16>::kSmemBytes; }

ms_status tc_pack_async(ms_ctx* ctx) {
    const int rows = (int)((ctx->n_pixels + 127) / 128 * 128);
    if (rows == 0) return MS_OK;
    k_pack_bf16<<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(ctx->P32, ctx->dc, rows, (int)ctx->Dp,
                                                                         (uint4*)ctx->Pk);
    MS_LAUNCH("k_pack_bf16");
    ctx->launches += 1;
    return MS_OK;
}

ms_status tc_finish(ms_ctx* ctx) {
    ms_status st = ctx->Dp == 32 ? allow_smem_all_shapes<TcSingleMap, 32>() : allow_smem_all_shapes<TcSingleMap, 16>();
    if (st != MS_OK) return st;
    ctx->tc_grid = ctx->num_sms;  // one CTA per SM: it owns all 512 TMEM columns
    if (ctx->Mk)
        if (ms_status ls = label_tc_setup(); ls != MS_OK) return ls;
    // the packed rows use the padding of the workspace (n_pixels rounded up to 128)
    const int64_t rows = (ctx->n_pixels + 127) / 128 * 128;
    if ((st = encode_pmap(ctx->Pk, (int)ctx->n_pad, &ctx->pmap)) != MS_OK) return st;
    if (ctx->Dp == 32) return encode_pmap((uint8_t*)ctx->Pk + rows * 128, (int)ctx->n_pad, &ctx->pmap1);
    ctx->pmap1 = ctx->pmap;
    return MS_OK;
}

ms_status launch_shift_tc(ms_ctx* ctx, const int32_t* active, int grid, int target_items, float* dbg_S) {
    const float c = ceil_to_float(ctx->cfg.bandwidth_cos);
    TcSingleMap map;
    map.active = active;
    map.dc = ctx->dc;
    map.n = (int)ctx->n;
    map.n_ptiles = (int)(ctx->n_pad / 128);
    map.target = target_items;
    unsigned long long* band = (unsigned long long*)&ctx->dc->band_pairs;
    return with_tc_shape(ctx->cfg.tc_shape, [&](auto sh) -> ms_status {
        using Sh = decltype(sh);
        if (ctx->Dp == 32) {
            if (dbg_S) return set_error(MS_ERR_INVALID_ARG, "the score dump is for d <= 16");
            k_shift_tc<Sh, 32, false, TcSingleMap><<<grid, Sh::kThreads, TcDim<32>::kSmemBytes, ctx->stream>>>(
                ctx->pmap, ctx->pmap1, ctx->P32, ctx->X, ctx->acc, c, map, &ctx->dc->status, band, nullptr, 0);
        } else if (dbg_S) {
            k_shift_tc<Sh, 16, true, TcSingleMap><<<grid, Sh::kThreads, TcDim<16>::kSmemBytes, ctx->stream>>>(
                ctx->pmap, ctx->pmap1, ctx->P32, ctx->X, ctx->acc, c, map, &ctx->dc->status, band, dbg_S, ctx->n_pad);
        } else {
            k_shift_tc<Sh, 16, false, TcSingleMap><<<grid, Sh::kThreads, TcDim<16>::kSmemBytes, ctx->stream>>>(
                ctx->pmap, ctx->pmap1, ctx->P32, ctx->X, ctx->acc, c, map, &ctx->dc->status, band, nullptr, 0);
        }
        MS_LAUNCH("k_shift_tc");
        return MS_OK;
    });
}

// ------------------------------------------------------------ batched form
// Work items of every iterating frame: frame f contributes
// item_off[f+1] - item_off[f] items (seed tiles of 128 x chunks).
struct TcBatchMap {
    const BFrame* frames;
    const BState* states;
    BPlan plan;
    const int32_t* act0;
    const int32_t* act1;
    int nf;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = plan.item_off[nf];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ TcItem item(int i) const {
        const int f = locate(plan.item_off, nf, i);
        const int local = i - plan.item_off[f];
        const int chunks = plan.chunks[f], tpc = plan.tpc[f];
        const int t = local / chunks, ch = local - t * chunks;
        const BFrame& fr = frames[f];
        TcItem it;
        it.active = ((states[f].dc.iters & 1) ? act1 : act0) + fr.pix0;
        it.n_active = states[f].dc.n_active;
        it.seed0 = t * 128;
        it.pt0 = ch * tpc;
        it.pt1 = min(fr.n_ptiles, it.pt0 + tpc);
        it.pk_row0 = fr.pk_row0;
        it.pix0 = fr.pix0;
        it.n = fr.n;
        return it;
    }
};

ms_status tc_batch_setup(int D) {
    return D == 32 ? allow_smem_all_shapes<TcBatchMap, 32>() : allow_smem_all_shapes<TcBatchMap, 16>();
}

ms_status launch_shift_tc_batch(const CUtensorMap& pmap, const CUtensorMap& pmap1, int D, const float* P32,
                                const float* X, unsigned long long* acc, float c_f, const BFrame* frames,
                                const BState* states, BPlan plan, const int32_t* act0, const int32_t* act1, int nf,
                                int* status, unsigned long long* band, int grid, int shape, cudaStream_t st) {
    TcBatchMap map;
    map.frames = frames;
    map.states = states;
    map.plan = plan;
    map.act0 = act0;
    map.act1 = act1;
    map.nf = nf;
    map.total_ = 0;
    return with_tc_shape(shape, [&](auto sh) -> ms_status {
        using Sh = decltype(sh);
        if (D == 32)
            k_shift_tc<Sh, 32, false, TcBatchMap><<<grid, Sh::kThreads, TcDim<32>::kSmemBytes, st>>>(
                pmap, pmap1, P32, X, acc, c_f, map, status, band, nullptr, 0);
        else
            k_shift_tc<Sh, 16, false, TcBatchMap><<<grid, Sh::kThreads, TcDim<16>::kSmemBytes, st>>>(
                pmap, pmap1, P32, X, acc, c_f, map, status, band, nullptr, 0);
        MS_LAUNCH("k_shift_tc(batch)");
        return MS_OK;
    });
}

ms_status encode_pk_map(void* Pk, int rows, CUtensorMap* map) { return encode_pmap(Pk, rows, map); }

}  // namespace ms
