// Adjoint of the smooth-kernel (von Mises-Fisher) step on the tensor cores:
// the BF16 form of the two reverse passes that ms_vmf.cu runs in FP32.
//
// For one step x -> x' = y/|y| with y_m = sum_i w_mi p_i and
// w_mi = exp(kappa (x_m.p_i - 1)) (Eq. 2 with the exponential profile, the
// dense update of Sec. 3.2.1), and with gy_m = (g_m - x'_m (x'_m.g_m))/|y_m|
// from the upstream gradient g = dL/dx' (formed by k_vmf_adj_link):
//     a_mi  = gy_m . p_i,   ds_mi = kappa w_mi a_mi,
//     pass A   dL/dx_m  = sum_i ds_mi p_i                 rows: seeds,  columns: pixels
//     pass B   dL/dp_i += sum_m w_mi gy_m + ds_mi x_m      rows: pixels, columns: seeds
// Both passes are one kernel, k_vmf_adj_tc<kPassB>. A work item is a tile of
// 128 rows against a run of 64-column sub-tiles. Per sub-tile:
//   GEMM1  E = kappa log2(e) (x.p - 1) and A = gy.p (pass A: kappa gy.p),
//          128 x 64 each, FP32 in TMEM. Every operand is a three-term BF16
//          split (v = vh + vm + vl exactly) and six products per score (hh,
//          hm, mh, hl, mm, lh) leave out only terms below 2^-24 of |v||p|, as
//          in the forward kernel; -kappa log2(e) enters E as a seventh MMA, a
//          three-term split against the pixel rows' ones column.
//   weights  w = 2^E (one ex2.approx.ftz), and
//          pass A: ds = w (kappa a);  pass B: w and ds' = ds / (kappa log2(e))
//          = ln(2) w a, because pass B's seed operand is kappa log2(e) x
//          (ds' (kappa log2(e) x) = ds x; no division, and kappa = 0 is fine).
//          Each value becomes two BF16 terms, written over the warp's own
//          columns of E (and A): the buffers become GEMM2's A operands. The
//          arithmetic runs on FP32 pairs (f32x2 instructions).
//   GEMM2  pass A: Y += Dh.[Ph|Pm|Pl] + Dl.[Ph|Pm]            (8 MMAs)
//          pass B: Y += Wh.[Gh|Gm|Gl] + Wl.[Gh|Gm]
//                     + Dh'.[Vh|Vm|Vl] + Dl'.[Vh|Vm]          (16 MMAs)
//          with the column tile itself (MN-major) as the B operand; the low
//          weight terms are 2^-8 of the sum and need two data terms.
// Per item the epilogue writes Y's FP32 sums (h + m + l) to the item's slot of
// a partial buffer; pass B adds them to the slot instead from the second
// reverse step on (every slot belongs to one CTA per launch and launches are
// stream-ordered), so dL/dp is summed over the chunks once, after the last
// step. k_vmf_adj_link adds pass A's chunks, forms the next step's gy and
// packs that step's operands in one launch. Chunks are added in a fixed
// order, so results are deterministic. No seed-by-pixel matrix leaves TMEM.
//
// Roles (608 threads, one CTA per SM):
//   warps 0-15  weights: four per TMEM lane quadrant, 16 columns of each
//               sub-tile; warps 0-3 also read Y;
//   warp 16     TMA producer: the item's row operand(s) (double-buffered)
//               and a ring of column sub-tiles;
//   warp 17     GEMM1 issuer, up to three sub-tiles ahead (three E/A pairs);
//   warp 18     GEMM2 issuer.
// TMEM: three pairs (E 64 + A 64 columns) at 0, 128, 256 and Y at 384 (48).
// Every wait is bounded; a timeout raises the CTA's abort flag, drains the
// MMAs and TMA loads in flight, frees TMEM and sets *status.
#include <cudaTypedefs.h>

#include "ms_internal.cuh"
#include "ms_tc.cuh"

namespace ms {
namespace {

using namespace tc;

constexpr int kAdjThreads = 19 * 32;
constexpr int kAdjWarpTma = 16, kAdjWarpG1 = 17, kAdjWarpG2 = 18;
constexpr int kAdjWeightWarps = 16;
constexpr int kAdjStages = 8;
constexpr int kAdjTile = 128 * 128;       // one 128-row operand tile (128 bytes per row)
constexpr int kAdjSub = 64 * 128;         // one 64-row column operand
constexpr int kAdjPairs = 3;
constexpr uint32_t kAdjColY = 384;
constexpr int kAdjOffR = 0;                               // [2 items][2 tiles] row operands
constexpr int kAdjOffS = 4 * kAdjTile;                    // [kAdjStages] column stages of 16 KB
constexpr int kAdjOffBar = kAdjOffS + kAdjStages * kAdjTile;
// full, empty [kAdjStages]; r_full, r_empty [2]; s_full, w_full, w_empty
// [kAdjPairs]; d_full, d_empty; aux [2]
constexpr int kAdjNumBars = 2 * kAdjStages + 4 + 3 * kAdjPairs + 2 + 2;
constexpr int kAdjSmemBytes = kAdjOffBar + kAdjNumBars * 8 + 16 + 1024;
static_assert(kAdjSmemBytes <= 227 * 1024, "shared memory budget");
constexpr float kLn2 = 0.69314718055994531f;

struct AdjMap {
    int chunks, spc, n_sub, items;
    __device__ __forceinline__ void range(int item, int& t, int& c0, int& c1) const {
        t = item / chunks;
        c0 = (item - t * chunks) * spc;
        c1 = min(n_sub, c0 + spc);
    }
};

__device__ __forceinline__ float ex2_ftz(float e) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(e));
    return y;
}

__device__ __forceinline__ void adj_drain_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

__device__ __forceinline__ bool adj_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

// Elementwise products and differences of FP32 pairs, one instruction each.
__device__ __forceinline__ void mul2(float& r0, float& r1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void sub2(float& r0, float& r1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Two BF16 terms of a pair, packed: hi = RN(v), lo = RN(v - hi).
__device__ __forceinline__ void split2_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16(v0, v1);
    float r0, r1;
    sub2(r0, r1, v0, v1, __uint_as_float(hi << 16), __uint_as_float(hi & 0xFFFF0000u));
    lo = pack_bf16(r0, r1);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    uint16_t r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Six BF16 products of three-term splits into D (a, b: K-major descriptors of
// the [h | m | l] operand rows; +2 moves one 16-element K step).
__device__ __forceinline__ void six_products(uint32_t d, uint64_t a, uint64_t b, uint32_t id) {
    mma_bf16_warp(d, a, b, id, 0);          // h . h
    mma_bf16_warp(d, a, b + 2, id, 1);      // h . m
    mma_bf16_warp(d, a + 2, b, id, 1);      // m . h
    mma_bf16_warp(d, a, b + 4, id, 1);      // h . l
    mma_bf16_warp(d, a + 2, b + 2, id, 1);  // m . m
    mma_bf16_warp(d, a + 4, b, id, 1);      // l . h
}

// partial[item][r][k] (+)= the item's sum for row 128 t + r (pass A: dL/dx of
// a seed over a pixel chunk; pass B: dL/dp of a pixel over a seed chunk; `+=`
// when accumulate is set). Row maps: pass A rmap0 = Vk, rmap1 = Gak (kappa gy);
// pass B rmap0 = Pk. Column maps (64-row boxes): pass A cmap0 = Pk; pass B
// cmap0 = Vk, cmap1 = Gk. Vk rows hold -kappa log2(e) as a split in their
// fourth 16-element slot, Pk rows three ones there.
template <bool kPassB>
__global__ void __launch_bounds__(kAdjThreads, 1)
k_vmf_adj_tc(const __grid_constant__ CUtensorMap rmap0, const __grid_constant__ CUtensorMap rmap1,
             const __grid_constant__ CUtensorMap cmap0, const __grid_constant__ CUtensorMap cmap1, AdjMap map,
             float* __restrict__ partial, int accumulate, int* status) {
    constexpr int kRowBytes = kPassB ? kAdjTile : 2 * kAdjTile;
    constexpr int kStageBytes = kPassB ? 2 * kAdjSub : kAdjSub;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* R = smem + kAdjOffR;
    uint8_t* S = smem + kAdjOffS;
    uint64_t* bars = (uint64_t*)(smem + kAdjOffBar);
    uint64_t* full = bars;                      // [kAdjStages] column sub-tile landed
    uint64_t* empty = full + kAdjStages;        // [kAdjStages] consumed by GEMM2
    uint64_t* r_full = empty + kAdjStages;      // [2] row operand(s) of an item landed
    uint64_t* r_empty = r_full + 2;             // [2] last GEMM1 of that item done
    uint64_t* s_full = r_empty + 2;             // [kAdjPairs] GEMM1 of a sub-tile done
    uint64_t* w_full = s_full + kAdjPairs;      // [kAdjPairs] weights written over E/A
    uint64_t* w_empty = w_full + kAdjPairs;     // [kAdjPairs] GEMM2 done with the pair
    uint64_t* d_full = w_empty + kAdjPairs;     // Y of an item complete
    uint64_t* d_empty = d_full + 1;             // Y read by the epilogue
    uint64_t* aux = d_empty + 1;                // [2] drain of the MMA issuers
    uint32_t* tmem_slot = (uint32_t*)(bars + kAdjNumBars);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kAdjStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&r_full[b], 1);
            mbar_init(&r_empty[b], 1);
        }
        for (int b = 0; b < kAdjPairs; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&w_full[b], kAdjWeightWarps);
            mbar_init(&w_empty[b], 1);
        }
        mbar_init(d_full, 1);
        mbar_init(d_empty, 128);
        mbar_init(&aux[0], 1);
        mbar_init(&aux[1], 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == kAdjWarpTma && lane == 0) {
        tma_prefetch_desc(&rmap0);
        tma_prefetch_desc(&cmap0);
        if (!kPassB) tma_prefetch_desc(&rmap1);
        if (kPassB) tma_prefetch_desc(&cmap1);
    }
    if (warp == kAdjWarpG1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int items = map.items;

    if (warp == kAdjWarpTma) {
        // ------------------------------------------------ TMA producer
        int g = 0, it = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            int t, c0, c1;
            map.range(item, t, c0, c1);
            const int rb = it & 1;
            if (it >= 2 && !(ok = adj_wait(&r_empty[rb], ((it >> 1) - 1) & 1, abort))) break;
            if (lane == 0) {
                mbar_arrive_expect_tx(&r_full[rb], kRowBytes);
                tma_load_2d(R + rb * 2 * kAdjTile, &rmap0, 0, t * 128, &r_full[rb]);
                if (!kPassB) tma_load_2d(R + rb * 2 * kAdjTile + kAdjTile, &rmap1, 0, t * 128, &r_full[rb]);
            }
            __syncwarp();
            for (int c = c0; c < c1; ++c, ++g) {
                const int s = g % kAdjStages;
                if (g >= kAdjStages && !(ok = adj_wait(&empty[s], ((g / kAdjStages) - 1) & 1, abort))) break;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], kStageBytes);
                    tma_load_2d(S + s * kAdjTile, &cmap0, 0, c * 64, &full[s]);
                    if (kPassB) tma_load_2d(S + s * kAdjTile + kAdjSub, &cmap1, 0, c * 64, &full[s]);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && *abort) {
            for (int q = max(0, g - kAdjStages); q < g; ++q) adj_drain_wait(&full[q % kAdjStages], (q / kAdjStages) & 1);
            for (int q = max(0, it - 1); q <= it; ++q) adj_drain_wait(&r_full[q & 1], (q >> 1) & 1);
        }
    } else if (warp == kAdjWarpG1) {
        // ------------------------------------------------ GEMM1 issuer
        // Descriptors are built once; moving an operand by b bytes adds b >> 4.
        const uint64_t dR = desc_sw128(smem_u32(R), 16, 1024);  // row operands, K-major
        const uint64_t dS = desc_sw128(smem_u32(S), 16, 1024);  // column sub-tiles, K-major
        constexpr uint32_t id1 = idesc_bf16(128, 64, 0, 0);
        constexpr uint64_t kT = kAdjTile >> 4, kH = kAdjSub >> 4;
        bool ok = true;
        int g = 0, u = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            int t, c0, c1;
            map.range(item, t, c0, c1);
            const int rb = it & 1;
            if (!(ok = adj_wait(&r_full[rb], (it >> 1) & 1, abort))) break;
            const uint64_t a0 = dR + (uint64_t)rb * 2 * kT;        // pass A: V rows; pass B: P rows
            const uint64_t a1 = kPassB ? a0 : a0 + kT;            // pass A: G rows
            for (int c = c0; c < c1; ++c, ++g, ++u) {
                const int s = g % kAdjStages, b = u % kAdjPairs;
                if (!(ok = adj_wait(&full[s], (g / kAdjStages) & 1, abort))) break;
                if (u >= kAdjPairs && !(ok = adj_wait(&w_empty[b], ((u / kAdjPairs) - 1) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tE = tmem + b * 128, tA = tE + 64;
                const uint64_t b0 = dS + (uint64_t)s * kT;          // pass A: P; pass B: V
                const uint64_t b1 = kPassB ? b0 + kH : b0;          // pass B: G
                six_products(tE, a0, b0, id1);                      // E = kappa log2(e) x . p
                mma_bf16_warp(tE, a0 + 6, b0 + 6, id1, 1);          //   - kappa log2(e) (split . ones)
                six_products(tA, a1, b1, id1);                      // A = gy . p (pass A: kappa gy . p)
                mma_commit_warp(&s_full[b]);
            }
            if (!ok) break;
            mma_commit_warp(&r_empty[rb]);
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[0]);
            adj_drain_wait(&aux[0], 0);
        }
    } else if (warp == kAdjWarpG2) {
        // ------------------------------------------------ GEMM2 issuer
        // K step k of a sub-tile = its columns 16 k .. 16 k + 15 = weight warp
        // slice k: high terms at TMEM column 16 k of E (A), low terms 8 further.
        const uint64_t dC = desc_sw128(smem_u32(S), kAdjTile, 1024);  // column sub-tiles, MN-major
        constexpr uint32_t id48 = idesc_bf16(128, 48, 0, 1);
        constexpr uint32_t id32 = idesc_bf16(128, 32, 0, 1);
        constexpr uint64_t kT = kAdjTile >> 4, kH = kAdjSub >> 4;
        bool ok = true;
        int g = 0, u = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            int t, c0, c1;
            map.range(item, t, c0, c1);
            for (int c = c0; c < c1; ++c, ++g, ++u) {
                const int s = g % kAdjStages, b = u % kAdjPairs;
                const bool first = c == c0;
                if (!(ok = adj_wait(&w_full[b], (u / kAdjPairs) & 1, abort))) break;
                if (!(ok = adj_wait(&full[s], (g / kAdjStages) & 1, abort))) break;
                if (first && it >= 1 && !(ok = adj_wait(d_empty, (it - 1) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tE = tmem + b * 128, tA = tE + 64, tY = tmem + kAdjColY;
                const uint64_t st = dC + (uint64_t)s * kT;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t acc0 = (first && k == 0) ? 0u : 1u;
                    if constexpr (!kPassB) {
                        mma_bf16_ts_warp(tY, tE + 16 * k, st + k * 128, id48, acc0);      // Dh . [Ph|Pm|Pl]
                        mma_bf16_ts_warp(tY, tE + 16 * k + 8, st + k * 128, id32, 1u);    // Dl . [Ph|Pm]
                    } else {
                        mma_bf16_ts_warp(tY, tE + 16 * k, st + kH + k * 128, id48, acc0);  // Wh . [Gh|Gm|Gl]
                        mma_bf16_ts_warp(tY, tE + 16 * k + 8, st + kH + k * 128, id32, 1u); // Wl . [Gh|Gm]
                        mma_bf16_ts_warp(tY, tA + 16 * k, st + k * 128, id48, 1u);         // Dh' . [Vh|Vm|Vl]
                        mma_bf16_ts_warp(tY, tA + 16 * k + 8, st + k * 128, id32, 1u);     // Dl' . [Vh|Vm]
                    }
                }
                mma_commit_warp(&w_empty[b]);
                mma_commit_warp(&empty[s]);
                if (c == c1 - 1) mma_commit_warp(d_full);
            }
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[1]);
            adj_drain_wait(&aux[1], 0);
        }
    } else {
        // ------------------------------------------------ weight warps
        const int q = warp & 3;             // TMEM lane quadrant: rows 32 q .. 32 q + 31
        const int h = warp >> 2;            // columns 16 h .. 16 h + 15 of each sub-tile
        const int r = q * 32 + lane;        // row of the tile
        const bool lead = h == 0;           // reads Y
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int u = 0, it = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
            if (__any_sync(0xffffffffu, *abort)) break;
            int t, c0, c1;
            map.range(item, t, c0, c1);
            bool ok = true;
            for (int c = c0; c < c1; ++c, ++u) {
                const int b = u % kAdjPairs;
                if (!(ok = adj_wait(&s_full[b], (u / kAdjPairs) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tE = tmem + b * 128 + lane_base + 16 * h, tA = tE + 64;
                uint32_t e[16], a[16];
                tmem_ld16(tE, e);
                tmem_ld16(tA, a);
                tmem_ld_wait();
                uint32_t wh[8], wl[8], dh[8], dl[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float w0 = ex2_ftz(__uint_as_float(e[2 * i])), w1 = ex2_ftz(__uint_as_float(e[2 * i + 1]));
                    float d0, d1;
                    mul2(d0, d1, w0, w1, __uint_as_float(a[2 * i]), __uint_as_float(a[2 * i + 1]));
                    if constexpr (kPassB) {
                        mul2(d0, d1, d0, d1, kLn2, kLn2);
                        split2_pair(w0, w1, wh[i], wl[i]);
                    }
                    split2_pair(d0, d1, dh[i], dl[i]);
                }
                if constexpr (kPassB) {
                    tmem_st8(tE, wh);
                    tmem_st8(tE + 8, wl);
                    tmem_st8(tA, dh);
                    tmem_st8(tA + 8, dl);
                } else {
                    tmem_st8(tE, dh);
                    tmem_st8(tE + 8, dl);
                }
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&w_full[b]);
            }
            if (!ok) break;
            if (lead) {
                if (!adj_wait(d_full, it & 1, abort)) break;
                tc_fence_after();
                uint32_t yh[16], ym[16], yl[16];
                const uint32_t ty = tmem + kAdjColY + lane_base;
                tmem_ld16(ty, yh);
                tmem_ld16(ty + 16, ym);
                tmem_ld16(ty + 32, yl);
                tmem_ld_wait();
                tc_fence_before();
                mbar_arrive(d_empty);
                float* dst = partial + ((int64_t)item * 128 + r) * 16;
#pragma unroll
                for (int k = 0; k < 16; k += 4) {
                    float4 o;
                    o.x = (__uint_as_float(yh[k]) + __uint_as_float(ym[k])) + __uint_as_float(yl[k]);
                    o.y = (__uint_as_float(yh[k + 1]) + __uint_as_float(ym[k + 1])) + __uint_as_float(yl[k + 1]);
                    o.z = (__uint_as_float(yh[k + 2]) + __uint_as_float(ym[k + 2])) + __uint_as_float(yl[k + 2]);
                    o.w = (__uint_as_float(yh[k + 3]) + __uint_as_float(ym[k + 3])) + __uint_as_float(yl[k + 3]);
                    if (accumulate) {
                        const float4 p = *reinterpret_cast<const float4*>(dst + k);
                        o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
                    }
                    *reinterpret_cast<float4*>(dst + k) = o;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kAdjWarpG1) tmem_dealloc(tmem, 512);
    if (threadIdx.x == 0 && *abort) atomicOr(status, 2);
}

// out[m][k] (+)= sum over the chunks, in chunk order, of partial[t chunks + ch][r][k]
// for row m = 128 t + r < rows. Sixteen threads per row, one per component. A
// raised status poisons the outputs (NaN).
__global__ void k_vmf_adj_sum(const float* __restrict__ partial, int64_t rows, int chunks, const int* __restrict__ status,
                              float* __restrict__ out, int accumulate) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = gid >> 4;
    const int k = (int)(gid & 15);
    if (m >= rows) return;
    const int64_t t = m / 128, r = m % 128;
    const float* src = partial + ((t * chunks) * 128 + r) * 16 + k;
    float y = 0.f;
    for (int ch0 = 0; ch0 < chunks; ch0 += 8) {  // eight loads in flight, added in chunk order
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = ch0 + j < chunks ? src[(int64_t)(ch0 + j) * 128 * 16] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) y += v[j];
    }
    if (*status) y = __int_as_float(0x7fc00000);
    float* o = out + m * 16 + k;
    *o = accumulate ? *o + y : y;
}

// The link between two reverse steps, 16 threads per row (one per
// component) over the Mp padded rows, for the gradient g = dL/dx_s:
//   g = pass A's chunk sums for row m, added in chunk order (or g_in, the
//       upstream gradient, before the first step);
//   s = 0 (x_prev == nullptr): g_out = g, i.e. dL/dx_0;
//   else gy = (g - x_s (x_s . g)) / |y_(s-1)| and the operands of step s - 1:
//       Vk = split(kappa log2(e) x_(s-1)) with -kappa log2(e) split into its
//       fourth slot, Gk = split(gy), Gak = split(kappa gy).
// A split row is [h | m | l | slot 4] (16 BF16 values each), v = h + m + l
// exactly; rows >= M are zero (and carry the constant). A raised status
// poisons g (NaN).
__global__ void __launch_bounds__(256)
k_vmf_adj_link(const float* __restrict__ partial, int chunks, const float* __restrict__ g_in,
               const float* __restrict__ x_s, const float* __restrict__ x_prev, const float* __restrict__ yn_prev,
               int M, int Mp, float k2, float kappa, const int* __restrict__ status, float* __restrict__ g_out,
               uint16_t* __restrict__ Vk, uint16_t* __restrict__ Gk, uint16_t* __restrict__ Gak) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int m = (int)(gid >> 4), k = (int)(gid & 15);
    if (m >= Mp) return;  // never splits a row: Mp is a multiple of 128
    const bool live = m < M;
    float g = 0.f;
    if (live) {
        if (partial) {
            const int t = m / 128, r = m % 128;
            const float* src = partial + ((int64_t)t * chunks * 128 + r) * 16 + k;
            for (int ch0 = 0; ch0 < chunks; ch0 += 8) {  // eight loads in flight, added in chunk order
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = ch0 + j < chunks ? src[(int64_t)(ch0 + j) * 128 * 16] : 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) g += v[j];
            }
            if (*status) g = __int_as_float(0x7fc00000);
        } else {
            g = g_in[(int64_t)m * 16 + k];
        }
    }
    if (!x_prev) {
        if (live) g_out[(int64_t)m * 16 + k] = g;
        return;
    }
    const float xs = live ? x_s[(int64_t)m * 16 + k] : 0.f;
    float xg = xs * g;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) xg += __shfl_xor_sync(0xffffffffu, xg, o, 16);
    const float gy = live ? (g - xs * xg) * (1.f / yn_prev[m]) : 0.f;
    const float v = live ? k2 * x_prev[(int64_t)m * 16 + k] : 0.f;
    const float c_hi = bf16_value(bf16_bits(k2));
    const float c_mid = bf16_value(bf16_bits(k2 - c_hi));
    const float c_lo = (k2 - c_hi) - c_mid;
    const float c_k = k == 0 ? -c_hi : k == 1 ? -c_mid : k == 2 ? -c_lo : 0.f;
    const float vals[3] = {v, gy, kappa * gy};
    uint16_t* rows[3] = {Vk, Gk, Gak};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float x = vals[q];
        const uint16_t h = bf16_bits(x);
        const uint16_t mi = bf16_bits(x - bf16_value(h));
        const uint16_t l = bf16_bits((x - bf16_value(h)) - bf16_value(mi));
        uint16_t* row = rows[q] + (int64_t)m * 64;
        row[k] = h;
        row[16 + k] = mi;
        row[32 + k] = l;
        row[48 + k] = q == 0 ? bf16_bits(c_k) : (uint16_t)0;
    }
}

// Chunks of a row tile's column sub-tiles that keep the makespan smallest:
// ceil(items / grid) waves of (spc + 1) sub-tile times (the +1 stands for an
// item's fill, drain and epilogue); ties keep fewer chunks.
VmfAdjPlan adj_plan(int row_tiles, int n_sub, int grid) {
    VmfAdjPlan p;
    p.row_tiles = row_tiles;
    p.n_sub = n_sub;
    long long best = -1;
    for (int ch = 1; ch <= n_sub; ++ch) {
        const int spc = (n_sub + ch - 1) / ch;
        const int chn = (n_sub + spc - 1) / spc;
        const long long items = (long long)row_tiles * chn;
        const long long cost = ((items + grid - 1) / grid) * (long long)(spc + 1);
        if (best < 0 || cost < best) {
            best = cost;
            p.chunks = chn;
            p.spc = spc;
        }
    }
    p.items = row_tiles * p.chunks;
    p.grid = grid < p.items ? grid : p.items;
    return p;
}

ms_status encode_rows(void* base, int rows, int box_rows, CUtensorMap* map) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult qr;
        void* fn = nullptr;
        MS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr));
        if (qr != cudaDriverEntryPointSuccess || !fn)
            return set_error(MS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {64, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MS_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t vmf_adj_bytes(int32_t M, int64_t N, int grid) {
    const int Mp = (M + 127) / 128 * 128;
    const int64_t n_pad = (N + 127) / 128 * 128;
    const VmfAdjPlan pa = adj_plan(Mp / 128, (int)((N + 63) / 64), grid);
    const VmfAdjPlan pb = adj_plan((int)(n_pad / 128), (M + 63) / 64, grid);
    return 3 * align256((size_t)Mp * 128) + align256((size_t)pa.items * 128 * 16 * sizeof(float)) +
           align256((size_t)pb.items * 128 * 16 * sizeof(float));
}

ms_status vmf_adj_prepare(void* Pk, int64_t N, int32_t M, int grid, void* ws, VmfAdjWork* w) {
    // per call: the attribute belongs to the current device
    MS_CUDA(cudaFuncSetAttribute(k_vmf_adj_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmemBytes));
    MS_CUDA(cudaFuncSetAttribute(k_vmf_adj_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmemBytes));
    w->M = M;
    w->N = N;
    w->Mp = (M + 127) / 128 * 128;
    const int64_t n_pad = (N + 127) / 128 * 128;
    w->pa = adj_plan(w->Mp / 128, (int)((N + 63) / 64), grid);
    w->pb = adj_plan((int)(n_pad / 128), (M + 63) / 64, grid);
    char* b = (char*)ws;
    w->Vk = b;
    b += align256((size_t)w->Mp * 128);
    w->Gk = b;
    b += align256((size_t)w->Mp * 128);
    w->Gak = b;
    b += align256((size_t)w->Mp * 128);
    w->partial_a = (float*)b;
    b += align256((size_t)w->pa.items * 128 * 16 * sizeof(float));
    w->partial_b = (float*)b;
    ms_status s;
    if ((s = encode_rows(Pk, (int)n_pad, 128, &w->pk_rows)) != MS_OK) return s;
    if ((s = encode_rows(Pk, (int)n_pad, 64, &w->pk_cols)) != MS_OK) return s;
    if ((s = encode_rows(w->Vk, w->Mp, 128, &w->v_rows)) != MS_OK) return s;
    if ((s = encode_rows(w->Vk, w->Mp, 64, &w->v_cols)) != MS_OK) return s;
    if ((s = encode_rows(w->Gak, w->Mp, 128, &w->ga_rows)) != MS_OK) return s;
    return encode_rows(w->Gk, w->Mp, 64, &w->g_cols);
}

ms_status vmf_adj_backward(VmfAdjWork* w, const float* iters, const float* ynorm, int32_t T, float kappa,
                           const float* GT, int* status, float* dP, float* dX0, cudaStream_t st) {
    const float k2 = (float)((double)kappa * 1.4426950408889634);  // kappa log2(e)
    const int64_t MD = (int64_t)w->M * 16;
    const unsigned lblocks = (unsigned)(w->Mp * 16 / 256);
    if (T == 0) {  // x_T = x_0: dL/dx_0 = GT, and dP stays as the caller set it
        MS_CUDA(cudaMemcpyAsync(dX0, GT, sizeof(float) * (size_t)MD, cudaMemcpyDeviceToDevice, st));
        return MS_OK;
    }
    AdjMap ma, mb;
    ma.chunks = w->pa.chunks;
    ma.spc = w->pa.spc;
    ma.n_sub = w->pa.n_sub;
    ma.items = w->pa.items;
    mb.chunks = w->pb.chunks;
    mb.spc = w->pb.spc;
    mb.n_sub = w->pb.n_sub;
    mb.items = w->pb.items;
    // gy of step T-1 from the upstream gradient, and that step's operands
    k_vmf_adj_link<<<lblocks, 256, 0, st>>>(nullptr, 0, GT, iters + (size_t)T * MD, iters + (size_t)(T - 1) * MD,
                                          ynorm + (size_t)(T - 1) * w->M, w->M, w->Mp, k2, kappa, status, nullptr,
                                          (uint16_t*)w->Vk, (uint16_t*)w->Gk, (uint16_t*)w->Gak);
    MS_LAUNCH("k_vmf_adj_link");
    for (int t = T - 1; t >= 0; --t) {
        // pass B: dL/dp over every seed, added to the chunk slots
        k_vmf_adj_tc<true><<<(unsigned)w->pb.grid, kAdjThreads, kAdjSmemBytes, st>>>(
            w->pk_rows, w->pk_rows, w->v_cols, w->g_cols, mb, w->partial_b, t < T - 1 ? 1 : 0, status);
        MS_LAUNCH("k_vmf_adj_tc(pixels)");
        // pass A: dL/dx_t over every pixel
        k_vmf_adj_tc<false><<<(unsigned)w->pa.grid, kAdjThreads, kAdjSmemBytes, st>>>(
            w->v_rows, w->ga_rows, w->pk_cols, w->pk_cols, ma, w->partial_a, 0, status);
        MS_LAUNCH("k_vmf_adj_tc(seeds)");
        // dL/dx_t; then gy of step t-1 and its operands, or dL/dx_0
        k_vmf_adj_link<<<lblocks, 256, 0, st>>>(
            w->partial_a, ma.chunks, nullptr, iters + (size_t)t * MD, t > 0 ? iters + (size_t)(t - 1) * MD : nullptr,
            t > 0 ? ynorm + (size_t)(t - 1) * w->M : nullptr, w->M, w->Mp, k2, kappa, status, dX0, (uint16_t*)w->Vk,
            (uint16_t*)w->Gk, (uint16_t*)w->Gak);
        MS_LAUNCH("k_vmf_adj_link");
    }
    k_vmf_adj_sum<<<(unsigned)((w->N * 16 + 255) / 256), 256, 0, st>>>(w->partial_b, w->N, w->pb.chunks, status, dP,
                                                                       0);
    MS_LAUNCH("k_vmf_adj_sum");
    return MS_OK;
}

}  // namespace ms
