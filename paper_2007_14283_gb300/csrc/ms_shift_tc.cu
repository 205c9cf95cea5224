// Shift iteration, BF16 tensor-core form (Algorithm 2, lines 4-9; Eq. 6-8, 11).
//
// One work item = 128 seeds x a chunk of 128-pixel tiles. Per pixel tile:
//   GEMM1  S = Xh.Ph^T + Xh.Pm^T + Xl.Ph^T   (tcgen05, BF16 in, FP32 in TMEM)
//          x = Xh + Xl and p = Ph + Pm + Pl are exact BF16 splits of the FP32
//          vectors, so |S - x.p| <= 3 * 2^-18 + 48 * 2^-24 < 1.4e-5 for unit
//          vectors.
//   mask   S' = S - c; a pair is in the window when S' >= 0. Pairs with
//          |S'| < kBand = 2^-15 are re-decided with the same sequential FP32
//          dot product as the FP32 form, so every decision equals the FP32
//          form's (the FP32 dot is itself within 1e-6 of x.p).
//   GEMM2  Y += Mask . [Ph | Pm | Pl | 0] (tcgen05, mask 0/1 exact in BF16)
// The seed-by-pixel matrix lives only in TMEM and registers. After the
// item's last tile Y = Ph + Pm + Pl sums are added to the per-seed fixed-point
// accumulators shared with the FP32 form, and the same finalize kernel
// normalises the seeds and tests convergence in FP64.
//
// Warp roles (192 threads, 2 CTAs per SM): warp 0 issues TMA loads of pixel
// tiles into a 3-stage ring; warp 1 owns TMEM (256 columns: S at 0, Y at 128)
// and issues the MMAs; warps 2-5 each own the 32 TMEM lanes (seeds) of their
// quadrant and compute the mask. All waits are bounded; a timeout raises the
// CTA's abort flag, drains what is in flight, frees TMEM and reports
// MS_ERR_TIMEOUT through the frame's status word.
#include <cudaTypedefs.h>

#include "ms_device.cuh"
#include "ms_tc.cuh"

namespace ms {
namespace {

using namespace tc;

constexpr int kTcThreads = 192;
constexpr int kStages = 3;
constexpr int kTileBytes = 128 * 128;        // 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColS = 0, kColY = 128;
constexpr float kBand = 3.0517578125e-05f;   // 2^-15
constexpr float kFixScale = 68719476736.0f;  // 2^36

constexpr int kOffA1 = 0;
constexpr int kOffP = kTileBytes;
constexpr int kOffM = kOffP + kStages * kTileBytes;
constexpr int kOffBar = kOffM + 2 * kTileBytes;
constexpr int kNumBars = 2 * kStages + 8;
constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16 + 1024;  // + alignment slack

struct TcSplit {
    int tiles, chunks, tpc;  // seed tiles, pixel chunks, pixel tiles per chunk
};

__device__ __forceinline__ TcSplit tc_split(int n_active, int n_ptiles, int target) {
    TcSplit s;
    s.tiles = (n_active + 127) / 128;
    if (s.tiles == 0 || n_ptiles == 0) {
        s.chunks = 0;
        s.tpc = 1;
        return s;
    }
    int ch = (target + s.tiles - 1) / s.tiles;
    ch = ch < 1 ? 1 : (ch > n_ptiles ? n_ptiles : ch);
    s.tpc = (n_ptiles + ch - 1) / ch;
    s.chunks = (n_ptiles + s.tpc - 1) / s.tpc;
    return s;
}

// Bounded wait that ignores the abort flag (used while draining).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

__global__ void __launch_bounds__(kTcThreads, 2)
k_shift_tc(const __grid_constant__ CUtensorMap pmap, const float* __restrict__ P32, int32_t n,
           int n_ptiles, const int32_t* __restrict__ active, const float* __restrict__ X,
           unsigned long long* __restrict__ acc, float c_f, int target_items, DevCounters* dc,
           float* __restrict__ dbg_S) {
    if (dc->done) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* A1 = smem + kOffA1;
    uint8_t* Pst = smem + kOffP;
    uint8_t* Mt = smem + kOffM;
    uint64_t* bars = (uint64_t*)(smem + kOffBar);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* s_full = bars + 2 * kStages + 0;
    uint64_t* s_empty = bars + 2 * kStages + 1;
    uint64_t* m_full = bars + 2 * kStages + 2;
    uint64_t* m_empty = bars + 2 * kStages + 3;
    uint64_t* a1_full = bars + 2 * kStages + 4;
    uint64_t* d_full = bars + 2 * kStages + 5;
    uint64_t* d_empty = bars + 2 * kStages + 6;
    uint64_t* aux = bars + 2 * kStages + 7;
    uint32_t* tmem_slot = (uint32_t*)(bars + kNumBars);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(s_full, 1);
        mbar_init(s_empty, 128);
        mbar_init(m_full, 128);
        mbar_init(m_empty, 1);
        mbar_init(a1_full, 128);
        mbar_init(d_full, 1);
        mbar_init(d_empty, 128);
        mbar_init(aux, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) tma_prefetch_desc(&pmap);
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_active = dc->n_active;
    const TcSplit sp = tc_split(n_active, n_ptiles, target_items);
    const int items = sp.tiles * sp.chunks;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int g = 0;
            for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x) {
                const int ch = item % sp.chunks;
                const int pt0 = ch * sp.tpc, pt1 = min(n_ptiles, pt0 + sp.tpc);
                for (int pt = pt0; pt < pt1; ++pt, ++g) {
                    const int s = g % kStages;
                    if (g >= kStages && !mbar_wait(&empty[s], ((g / kStages) - 1) & 1, abort)) break;
                    mbar_arrive_expect_tx(&full[s], kTileBytes);
                    tma_load_2d(Pst + s * kTileBytes, &pmap, 0, pt * 128, &full[s]);
                }
            }
            if (*abort)
                for (int q = max(0, g - kStages); q < g; ++q) drain_wait(&full[q % kStages], (q / kStages) & 1);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t tS = tmem + kColS, tY = tmem + kColY;
            const uint32_t a1 = smem_u32(A1), mt = smem_u32(Mt);
            constexpr uint32_t id1 = idesc_bf16(128, 128, 0, 0);
            constexpr uint32_t id2 = idesc_bf16(128, 64, 0, 1);  // [Ph|Pm|Pl|0]: one 128-byte atom
            int g = 0, it = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
                const int ch = item % sp.chunks;
                const int pt0 = ch * sp.tpc, pt1 = min(n_ptiles, pt0 + sp.tpc);
                if (!(ok = mbar_wait(a1_full, it & 1, abort))) break;
                for (int pt = pt0; pt < pt1; ++pt, ++g) {
                    const int s = g % kStages;
                    if (!(ok = mbar_wait(&full[s], (g / kStages) & 1, abort))) break;
                    if (g > 0 && !(ok = mbar_wait(s_empty, (g - 1) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t pb = smem_u32(Pst + s * kTileBytes);
                    mma_bf16(tS, desc_sw128(a1, 16, 1024), desc_sw128(pb, 16, 1024), id1, 0);
                    mma_bf16(tS, desc_sw128(a1, 16, 1024), desc_sw128(pb + 32, 16, 1024), id1, 1);
                    mma_bf16(tS, desc_sw128(a1 + 32, 16, 1024), desc_sw128(pb, 16, 1024), id1, 1);
                    mma_commit(s_full);
                    if (!(ok = mbar_wait(m_full, g & 1, abort))) break;
                    if (pt == pt0 && it > 0 && !(ok = mbar_wait(d_empty, (it - 1) & 1, abort))) break;
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint64_t ad = desc_sw128(mt + (k >> 2) * kTileBytes + (k & 3) * 32, 16, 1024);
                        const uint64_t bd = desc_sw128(pb + k * 2048, kTileBytes, 1024);
                        mma_bf16(tY, ad, bd, id2, (pt > pt0 || k > 0) ? 1u : 0u);
                    }
                    mma_commit(m_empty);
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(d_full);
            }
            if (*abort) {
                mma_commit(aux);
                drain_wait(aux, 0);
            }
        }
    } else {
        // ------------------------------------------------ mask / epilogue warps
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const uint32_t tS = tmem + kColS + lane_base, tY = tmem + kColY + lane_base;
        long long band_local = 0;
        int g = 0, it = 0;
        for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x, ++it) {
            const int t = item / sp.chunks, ch = item % sp.chunks;
            const int pt0 = ch * sp.tpc, pt1 = min(n_ptiles, pt0 + sp.tpc);
            const int pos = t * 128 + r;
            const int slot = pos < n_active ? active[pos] : -1;
            float x[16];
#pragma unroll
            for (int k = 0; k < 16; k += 4) {
                const float4 v = slot >= 0 ? *reinterpret_cast<const float4*>(X + (int64_t)slot * 16 + k)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
            }
            // A1 row r: [Xh (16) | Xl (16) | 0 (32)], 128-byte swizzle. The
            // previous item's MMAs are complete (d_full was awaited).
            {
                uint32_t wh[8], wl[8];
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const float h0 = bf16_round(x[k]), h1 = bf16_round(x[k + 1]);
                    wh[k / 2] = pack_bf16(h0, h1);
                    wl[k / 2] = pack_bf16(x[k] - h0, x[k + 1] - h1);
                }
#pragma unroll
                for (int cidx = 0; cidx < 8; ++cidx) {
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (cidx == 0) v = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                    if (cidx == 1) v = make_uint4(wh[4], wh[5], wh[6], wh[7]);
                    if (cidx == 2) v = make_uint4(wl[0], wl[1], wl[2], wl[3]);
                    if (cidx == 3) v = make_uint4(wl[4], wl[5], wl[6], wl[7]);
                    *reinterpret_cast<uint4*>(A1 + sw128_offset(r, cidx)) = v;
                }
            }
            fence_proxy_async();
            mbar_arrive(a1_full);
            int cnt = 0;
            for (int pt = pt0; pt < pt1; ++pt, ++g) {
                if (!mbar_wait(s_full, g & 1, abort)) break;
                if (g > 0 && !mbar_wait(m_empty, (g - 1) & 1, abort)) break;
                tc_fence_after();
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {
                    uint32_t v[32];
                    tmem_ld32(tS + cc * 32, v);
                    tmem_ld_wait();
                    uint32_t bits = 0;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float sv = __uint_as_float(v[i]);
                        const float sp_ = sv - c_f;
                        bool in = sp_ >= 0.f;
                        if (fabsf(sp_) < kBand) {
                            const int px = pt * 128 + cc * 32 + i;
                            if (px < n) {
                                ++band_local;
                                float pv[16];
#pragma unroll
                                for (int k = 0; k < 16; k += 4) {
                                    const float4 w = *reinterpret_cast<const float4*>(P32 + (int64_t)px * 16 + k);
                                    pv[k] = w.x; pv[k + 1] = w.y; pv[k + 2] = w.z; pv[k + 3] = w.w;
                                }
                                in = dot_seq<16>(x, pv) >= c_f;
                            } else {
                                in = false;
                            }
                        }
                        bits |= (in ? 1u : 0u) << i;
                        if (dbg_S) dbg_S[(int64_t)r * n_ptiles * 128 + pt * 128 + cc * 32 + i] = sv;
                    }
                    cnt += __popc(bits);
                    // 32 mask values -> 16 words -> 4 chunks of 16 bytes
                    const int blk = cc >> 1;
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        uint32_t w[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int b0 = c4 * 8 + h * 2;
                            w[h] = (((bits >> b0) & 1u) ? 0x3F80u : 0u) | (((bits >> (b0 + 1)) & 1u) ? 0x3F800000u : 0u);
                        }
                        const int cidx = (cc & 1) * 4 + c4;
                        *reinterpret_cast<uint4*>(Mt + blk * kTileBytes + sw128_offset(r, cidx)) =
                            make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                tc_fence_before();
                mbar_arrive(s_empty);
                fence_proxy_async();
                mbar_arrive(m_full);
            }
            if (*abort) break;
            if (!mbar_wait(d_full, it & 1, abort)) break;
            tc_fence_after();
            uint32_t h[16], m[16], l[16];
            tmem_ld16(tY, h);
            tmem_ld16(tY + 16, m);
            tmem_ld16(tY + 32, l);
            tmem_ld_wait();
            tc_fence_before();
            mbar_arrive(d_empty);
            if (slot >= 0 && cnt > 0) {
                unsigned long long* a = acc + (int64_t)slot * 17;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float y = __uint_as_float(h[k]) + __uint_as_float(m[k]) + __uint_as_float(l[k]);
                    atomicAdd(a + k, (unsigned long long)__float2ll_rn(y * kFixScale));
                }
                atomicAdd(a + 16, (unsigned long long)cnt);
            }
        }
        if (band_local) atomicAdd((unsigned long long*)&dc->band_pairs, (unsigned long long)band_local);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
    if (threadIdx.x == 0 && *abort) atomicOr(&dc->status, 2);
}

// Pixels as BF16 splits for the tensor cores: row i = [Ph | Pm | Pl | 0]
// (64 values, 128 bytes) with p = Ph + Pm + Pl; rows n..n_pad-1 are zero.
__global__ void k_pack_bf16(const float* __restrict__ P32, int n, int n_pad, uint4* __restrict__ Pk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    uint32_t w[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) w[k] = 0u;
    if (i < n) {
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            const float p0 = P32[(int64_t)i * 16 + k], p1 = P32[(int64_t)i * 16 + k + 1];
            const float h0 = bf16_round(p0), h1 = bf16_round(p1);
            const float m0 = bf16_round(p0 - h0), m1 = bf16_round(p1 - h1);
            w[k / 2] = pack_bf16(h0, h1);
            w[8 + k / 2] = pack_bf16(m0, m1);
            w[16 + k / 2] = pack_bf16((p0 - h0) - m0, (p1 - h1) - m1);
        }
    }
    uint4* row = Pk + (int64_t)i * 8;
#pragma unroll
    for (int c = 0; c < 8; ++c) row[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
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

}  // namespace

int tc_smem_bytes() { return kSmemBytes; }

ms_status tc_prepare(ms_ctx* ctx) {
    if (ctx->n_pad == 0) return MS_OK;
    k_pack_bf16<<<(unsigned)((ctx->n_pad + 255) / 256), 256, 0, ctx->stream>>>(ctx->P32, (int)ctx->n,
                                                                              (int)ctx->n_pad, (uint4*)ctx->Pk);
    MS_LAUNCH("k_pack_bf16");
    ctx->launches += 1;
    MS_CUDA(cudaFuncSetAttribute(k_shift_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    int per_sm = 0;
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_tc, kTcThreads, kSmemBytes));
    if (per_sm < 1) return set_error(MS_ERR_CUDA, "tensor-core shift kernel does not fit on an SM");
    ctx->tc_grid = ctx->num_sms * (per_sm > 2 ? 2 : per_sm);
    return encode_pmap(ctx->Pk, (int)ctx->n_pad, &ctx->pmap);
}

ms_status launch_shift_tc(ms_ctx* ctx, const int32_t* active, int grid, int target_items, float* dbg_S) {
    const float c = ceil_to_float(ctx->cfg.bandwidth_cos);
    k_shift_tc<<<grid, kTcThreads, kSmemBytes, ctx->stream>>>(ctx->pmap, ctx->P32, (int32_t)ctx->n,
                                                             (int)(ctx->n_pad / 128), active, ctx->X, ctx->acc,
                                                             c, target_items, ctx->dc, dbg_S);
    MS_LAUNCH("k_shift_tc");
    return MS_OK;
}

}  // namespace ms
