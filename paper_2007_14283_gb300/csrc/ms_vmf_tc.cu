// Smooth-kernel (von Mises-Fisher) mean-shift step on the tensor cores: the
// BF16 form of the dense update that ms_vmf.cu computes in FP32.
//
// One step (Eq. 2 with the exponential profile; the dense update of
// Sec. 3.2.1), for every seed m against every pixel i:
//     s_mi = x_m . p_i,   w_mi = exp(kappa (s_mi - 1)),   y_m = sum_i w_mi p_i,
//     x'_m = y_m / |y_m|.
// GEMM1 gives E = kappa log2(e) s in FP32 (TMEM) from BF16 splits: the seed
// operand holds kappa log2(e) x as three BF16 terms v = vh + vm + vl (exact)
// and the pixel rows p = ph + pm + pl; six products (vh.ph, vh.pm, vm.ph,
// vh.pl, vm.pm, vl.ph) leave out only terms below 2^-24 |v||p|. Weight warps
// read E, form w = 2^(E - kappa log2(e)) with one ex2.approx.ftz (relative
// error about 2^-22) and split it into two BF16 terms, w = wh + wl + O(2^-16 w).
// GEMM2 accumulates Y = Wh.[Ph | Pm | Pl] + Wl.[Ph | Pm] in TMEM (the Wl term
// is 2^-8 of the sum, so its pixel needs only the two leading BF16 terms). Per
// work item (128 seeds x a pixel chunk) the epilogue writes Y's FP32 sums to a
// partial buffer; a second kernel adds the chunks in a fixed order and
// renormalises, so results are deterministic.
//
// Roles (608 threads, one CTA per SM):
//   warps 0-15  weights: four per TMEM lane quadrant, 32 pixels of each tile;
//               warps 0-3 also write the seed operand and read Y;
//   warp 16     TMA producer: ring of 128-pixel tiles of Pk;
//   warp 17     GEMM1 issuer, up to three tiles ahead;
//   warp 18     GEMM2 issuer.
// TMEM: three tile buffers of 128 columns at 0, 128, 256 and Y at 384 (48
// columns). GEMM1 writes a tile's E into a buffer; each weight warp reads its
// 32 columns and writes its weights back over them (wh of its 32 pixels in
// the first 16 columns, wl in the next 16), so the buffer then holds GEMM2's A
// operand and is free again when GEMM2 completes: three tiles in flight.
// Every wait is bounded; a timeout raises the CTA's abort flag, drains the
// MMAs and TMA loads in flight, frees TMEM and sets *status.
#include <cudaTypedefs.h>

#include "ms_internal.cuh"
#include "ms_tc.cuh"

namespace ms {
namespace {

using namespace tc;

constexpr int kVWeightWarps = 16;
constexpr int kVWarpTma = 16, kVWarpG1 = 17, kVWarpG2 = 18;
constexpr int kVThreads = 19 * 32;
constexpr int kVStages = 8;
constexpr int kVTileBytes = 128 * 128;
constexpr int kVBufs = 3;
constexpr uint32_t kVColY = 384;
constexpr int kVOffA1 = 0;                              // 2 x 16 KB seed operand
constexpr int kVOffP = 2 * kVTileBytes;                 // kVStages x 16 KB
constexpr int kVOffBar = kVOffP + kVStages * kVTileBytes;
// full, empty [kVStages]; s_full, w_full, w_empty [kVBufs]; a1_full [2];
// d_full, d_empty; aux [2] (drain)
constexpr int kVNumBars = 2 * kVStages + 3 * kVBufs + 2 + 2 + 2;
constexpr int kVSmemBytes = kVOffBar + kVNumBars * 8 + 16 + 1024;
static_assert(kVSmemBytes <= 227 * 1024, "shared memory budget");

// Seed tile t of 128 seeds x pixel chunk ch: item t * chunks + ch.
struct VmfTcMap {
    int M, n_ptiles, chunks, tpc;
    __device__ __forceinline__ int items() const { return ((M + 127) / 128) * chunks; }
};

// Row r of the seed operand for seed x and k2 = kappa log2(e):
// [v_h | v_m | v_l | 0] with v = k2 x (FP32) split into three BF16 terms
// (v = v_h + v_m + v_l exactly), 128-byte swizzle.
__device__ __forceinline__ void write_seed_row(uint8_t* A1, int r, const float* __restrict__ x, float k2) {
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
        const float4 t = x ? *reinterpret_cast<const float4*>(x + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[k] = k2 * t.x; v[k + 1] = k2 * t.y; v[k + 2] = k2 * t.z; v[k + 3] = k2 * t.w;
    }
    uint32_t w[24];
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        const float h0 = bf16_round(v[k]), h1 = bf16_round(v[k + 1]);
        const float m0 = bf16_round(v[k] - h0), m1 = bf16_round(v[k + 1] - h1);
        w[k / 2] = pack_bf16(h0, h1);
        w[8 + k / 2] = pack_bf16(m0, m1);
        w[16 + k / 2] = pack_bf16((v[k] - h0) - m0, (v[k + 1] - h1) - m1);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
        *reinterpret_cast<uint4*>(A1 + sw128_offset(r, c)) = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
#pragma unroll
    for (int c = 6; c < 8; ++c) *reinterpret_cast<uint4*>(A1 + sw128_offset(r, c)) = make_uint4(0u, 0u, 0u, 0u);
}

// 2^e, one MUFU operation (results below 2^-126 flush to zero).
__device__ __forceinline__ float ex2_ftz(float e) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(e));
    return y;
}

__device__ __forceinline__ void vdrain_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

__device__ __forceinline__ bool vwarp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

// partial[item][r][k] = sum over the item's pixel chunk of w p_k for seed
// 128 t + r. k2 = kappa log2(e) (folded into the seed operand).
__global__ void __launch_bounds__(kVThreads, 1)
k_vmf_tc(const __grid_constant__ CUtensorMap pmap, const float* __restrict__ X, float k2, VmfTcMap map,
         float* __restrict__ partial, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* A1 = smem + kVOffA1;
    uint8_t* Pst = smem + kVOffP;
    uint64_t* bars = (uint64_t*)(smem + kVOffBar);
    uint64_t* full = bars;                  // [kVStages] pixel tile landed
    uint64_t* empty = full + kVStages;      // [kVStages] pixel tile consumed by GEMM2
    uint64_t* s_full = empty + kVStages;    // [kVBufs] GEMM1 of the buffer's tile done
    uint64_t* w_full = s_full + kVBufs;     // [kVBufs] weights written over it
    uint64_t* w_empty = w_full + kVBufs;    // [kVBufs] GEMM2 done with it
    uint64_t* a1_full = w_empty + kVBufs;   // [2] seed operand written
    uint64_t* d_full = a1_full + 2;         // Y of an item complete
    uint64_t* d_empty = d_full + 1;         // Y read by the epilogue
    uint64_t* aux = d_empty + 1;            // [2] drain of the two MMA issuers
    uint32_t* tmem_slot = (uint32_t*)(bars + kVNumBars);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kVStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kVBufs; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&w_full[b], kVWeightWarps);
            mbar_init(&w_empty[b], 1);
        }
        for (int b = 0; b < 2; ++b) mbar_init(&a1_full[b], 128);
        mbar_init(d_full, 1);
        mbar_init(d_empty, 128);
        mbar_init(&aux[0], 1);
        mbar_init(&aux[1], 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == kVWarpTma && lane == 0) tma_prefetch_desc(&pmap);
    if (warp == kVWarpG1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int items = map.items();

    if (warp == kVWarpTma) {
        // ------------------------------------------------ TMA producer
        int g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const int ch = item % map.chunks;
            const int pt0 = ch * map.tpc, pt1 = min(map.n_ptiles, pt0 + map.tpc);
            for (int pt = pt0; pt < pt1; ++pt, ++g) {
                const int s = g % kVStages;
                if (g >= kVStages && !(ok = vwarp_wait(&empty[s], ((g / kVStages) - 1) & 1, abort))) break;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], kVTileBytes);
                    tma_load_2d(Pst + s * kVTileBytes, &pmap, 0, pt * 128, &full[s]);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && *abort)
            for (int q = max(0, g - kVStages); q < g; ++q) vdrain_wait(&full[q % kVStages], (q / kVStages) & 1);
    } else if (warp == kVWarpG1) {
        // ------------------------------------------------ GEMM1 issuer
        // Scores up to three tiles ahead of the weight warps (the buffers).
        const uint64_t dA1 = desc_sw128(smem_u32(A1), 16, 1024);   // seed operand, K-major
        const uint64_t dP1 = desc_sw128(smem_u32(Pst), 16, 1024);  // pixel tile, K-major
        constexpr uint32_t id1 = idesc_bf16(128, 128, 0, 0);
        constexpr uint64_t kT = kVTileBytes >> 4;
        bool ok = true;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            const int ch = item % map.chunks;
            const int pt0 = ch * map.tpc, pt1 = min(map.n_ptiles, pt0 + map.tpc);
            if (!(ok = vwarp_wait(&a1_full[it & 1], (it >> 1) & 1, abort))) break;
            const uint64_t a = dA1 + (uint64_t)(it & 1) * kT;
            for (int pt = pt0; pt < pt1; ++pt, ++g) {
                const int s = g % kVStages, b = g % kVBufs;
                if (!(ok = vwarp_wait(&full[s], (g / kVStages) & 1, abort))) break;
                if (g >= kVBufs && !(ok = vwarp_wait(&w_empty[b], ((g / kVBufs) - 1) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tS = tmem + b * 128;
                const uint64_t pb = dP1 + (uint64_t)s * kT;
                mma_bf16_warp(tS, a, pb, id1, 0);          // vh . Ph
                mma_bf16_warp(tS, a, pb + 2, id1, 1);      // vh . Pm
                mma_bf16_warp(tS, a + 2, pb, id1, 1);      // vm . Ph
                mma_bf16_warp(tS, a, pb + 4, id1, 1);      // vh . Pl
                mma_bf16_warp(tS, a + 2, pb + 2, id1, 1);  // vm . Pm
                mma_bf16_warp(tS, a + 4, pb, id1, 1);      // vl . Ph
                mma_commit_warp(&s_full[b]);
            }
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[0]);
            vdrain_wait(&aux[0], 0);
        }
    } else if (warp == kVWarpG2) {
        // ------------------------------------------------ GEMM2 issuer
        // Y += Wh.[Ph | Pm | Pl] + Wl.[Ph | Pm] once a tile's weights are in
        // its buffer; completion frees the buffer (for GEMM1) and the stage.
        const uint64_t dP2 = desc_sw128(smem_u32(Pst), kVTileBytes, 1024);  // pixel tile, MN-major
        constexpr uint32_t id2h = idesc_bf16(128, 48, 0, 1);  // Wh . [Ph | Pm | Pl]
        constexpr uint32_t id2l = idesc_bf16(128, 32, 0, 1);  // Wl . [Ph | Pm]
        constexpr uint64_t kT = kVTileBytes >> 4;
        bool ok = true;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            const int ch = item % map.chunks;
            const int pt0 = ch * map.tpc, pt1 = min(map.n_ptiles, pt0 + map.tpc);
            for (int pt = pt0; pt < pt1; ++pt, ++g) {
                const int s = g % kVStages, b = g % kVBufs;
                const bool first = pt == pt0;
                if (!(ok = vwarp_wait(&w_full[b], (g / kVBufs) & 1, abort))) break;
                if (!(ok = vwarp_wait(&full[s], (g / kVStages) & 1, abort))) break;
                if (first && it >= 1 && !(ok = vwarp_wait(d_empty, (it - 1) & 1, abort))) break;
                tc_fence_after();
                const uint64_t pb = dP2 + (uint64_t)s * kT;
                // pixels 16 k .. 16 k + 15: weight warp slice k / 2, half k % 2;
                // its wh at columns 32 (k / 2) + 8 (k % 2), its wl 16 further
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    mma_bf16_ts_warp(tmem + kVColY, tmem + b * 128 + 32 * (k / 2) + 8 * (k % 2), pb + k * 128, id2h,
                                     (first && k == 0) ? 0u : 1u);
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    mma_bf16_ts_warp(tmem + kVColY, tmem + b * 128 + 32 * (k / 2) + 8 * (k % 2) + 16, pb + k * 128,
                                     id2l, 1u);
                mma_commit_warp(&w_empty[b]);
                mma_commit_warp(&empty[s]);
                if (pt == pt1 - 1) mma_commit_warp(d_full);
            }
        }
        if (__any_sync(0xffffffffu, *abort)) {
            mma_commit_warp(&aux[1]);
            vdrain_wait(&aux[1], 0);
        }
    } else {
        // ------------------------------------------------ weight warps
        const int q = warp & 3;           // TMEM lane quadrant: seeds 32 q .. 32 q + 31
        const int h = warp >> 2;          // pixels 32 h .. 32 h + 31 of each tile
        const int r = q * 32 + lane;      // seed row of the tile
        const bool lead = h == 0;         // writes the seed operand and reads Y
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
            if (__any_sync(0xffffffffu, *abort)) break;
            const int t = item / map.chunks, ch = item % map.chunks;
            const int pt0 = ch * map.tpc, pt1 = min(map.n_ptiles, pt0 + map.tpc);
            if (lead) {
                // this item's operand (first item) and the next one's; the
                // next one's buffer was last read by GEMM1s of item it-1, which
                // completed before this warp saw the E of that item's tiles
                if (it == 0) {
                    const int m = t * 128 + r;
                    write_seed_row(A1, r, m < map.M ? X + (int64_t)m * 16 : nullptr, k2);
                    fence_proxy_async();
                    mbar_arrive(&a1_full[0]);
                }
                const int nitem = item + gridDim.x;
                if (nitem < items) {
                    const int m = (nitem / map.chunks) * 128 + r;
                    write_seed_row(A1 + ((it + 1) & 1) * kVTileBytes, r, m < map.M ? X + (int64_t)m * 16 : nullptr,
                                   k2);
                    fence_proxy_async();
                    mbar_arrive(&a1_full[(it + 1) & 1]);
                }
            }
            bool ok = true;
            for (int pt = pt0; pt < pt1 && ok; ++pt, ++g) {
                const int b = g % kVBufs;
                if (!(ok = vwarp_wait(&s_full[b], (g / kVBufs) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tb = tmem + b * 128 + lane_base + h * 32;
                uint32_t v[32];
                tmem_ld32(tb, v);
                tmem_ld_wait();
                uint32_t wh[16], wl[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float w0 = ex2_ftz(__uint_as_float(v[2 * i]) - k2);
                    const float w1 = ex2_ftz(__uint_as_float(v[2 * i + 1]) - k2);
                    const uint32_t hp = pack_bf16(w0, w1);
                    wh[i] = hp;
                    wl[i] = pack_bf16(w0 - __uint_as_float(hp << 16), w1 - __uint_as_float(hp & 0xFFFF0000u));
                }
                // the weights go over this warp's own columns of E
                tmem_st16(tb, wh);
                tmem_st16(tb + 16, wl);
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&w_full[b]);
            }
            if (!ok) break;
            if (lead) {
                if (!vwarp_wait(d_full, it & 1, abort)) break;
                tc_fence_after();
                uint32_t yh[16], ym[16], yl[16];
                const uint32_t ty = tmem + kVColY + lane_base;
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
                    *reinterpret_cast<float4*>(dst + k) = o;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kVWarpG1) tmem_dealloc(tmem, 512);
    if (threadIdx.x == 0 && *abort) atomicOr(status, 2);
}

// x'_m = y_m / |y_m| with y_m the chunks' partial sums added in chunk order;
// |y_m| kept for the adjoint. Sixteen threads per seed, one per component. A
// raised status poisons the outputs (NaN).
__global__ void k_vmf_tc_reduce(const float* __restrict__ partial, VmfTcMap map, const int* __restrict__ status,
                                float* __restrict__ Xn, float* __restrict__ ynorm) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = gid >> 4, k = gid & 15;
    const bool live = m < map.M;
    const int t = m / 128, r = m % 128;
    float y = 0.f;
    if (live) {
        const float* src = partial + ((int64_t)t * map.chunks * 128 + r) * 16 + k;
        for (int ch0 = 0; ch0 < map.chunks; ch0 += 8) {  // eight loads in flight, added in chunk order
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = ch0 + j < map.chunks ? src[(int64_t)(ch0 + j) * 128 * 16] : 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) y += v[j];
        }
    }
    float ss = y * y;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o, 16);
    if (!live) return;
    const float yn = *status ? __int_as_float(0x7fc00000) : sqrtf(ss);
    Xn[(int64_t)m * 16 + k] = y / yn;
    if (ynorm && k == 0) ynorm[m] = yn;
}

__global__ void k_vmf_tc_pack(const float* __restrict__ P, int64_t n, int64_t rows, uint4* __restrict__ Pk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    pack_split_row(i < n ? P + i * 16 : nullptr, Pk + i * 8);
}

}  // namespace

VmfTcPlan vmf_tc_plan(int32_t M, int64_t N, int grid) {
    VmfTcPlan p;
    p.n_ptiles = (int)((N + 127) / 128);
    const int tiles = (M + 127) / 128;
    int chunks = (grid + tiles - 1) / tiles;
    chunks = chunks < 1 ? 1 : chunks > p.n_ptiles ? p.n_ptiles : chunks;
    p.tpc = (p.n_ptiles + chunks - 1) / chunks;
    p.chunks = (p.n_ptiles + p.tpc - 1) / p.tpc;
    p.items = tiles * p.chunks;
    p.grid = grid < p.items ? grid : p.items;
    return p;
}

size_t vmf_tc_pk_bytes(int64_t N) { return (size_t)((N + 127) / 128 * 128) * 128; }

ms_status vmf_tc_prepare(const float* P, int64_t N, void* Pk, CUtensorMap* map, cudaStream_t st) {
    // per call: the attribute belongs to the current device
    MS_CUDA(cudaFuncSetAttribute(k_vmf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kVSmemBytes));
    const int64_t rows = (N + 127) / 128 * 128;
    k_vmf_tc_pack<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(P, N, rows, (uint4*)Pk);
    MS_LAUNCH("k_vmf_tc_pack");
    return encode_pk_map(Pk, (int)rows, map);
}

ms_status vmf_tc_step(const CUtensorMap& map, const float* Xt, int32_t M, float kappa, const VmfTcPlan& plan,
                      float* partial, int* status, float* Xn, float* ynorm, cudaStream_t st) {
    VmfTcMap mp;
    mp.M = M;
    mp.n_ptiles = plan.n_ptiles;
    mp.chunks = plan.chunks;
    mp.tpc = plan.tpc;
    const float k2 = (float)((double)kappa * 1.4426950408889634);  // kappa log2(e)
    k_vmf_tc<<<(unsigned)plan.grid, kVThreads, kVSmemBytes, st>>>(map, Xt, k2, mp, partial, status);
    MS_LAUNCH("k_vmf_tc");
    k_vmf_tc_reduce<<<(unsigned)((M * 16 + 255) / 256), 256, 0, st>>>(partial, mp, status, Xn, ynorm);
    MS_LAUNCH("k_vmf_tc_reduce");
    return MS_OK;
}

}  // namespace ms
