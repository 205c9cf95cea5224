// Ingest: compact the foreground in row-major order and normalise each vector
// to unit length in FP32 (cosine distance, Eq. 9, is scale invariant; the
// window mean of Eq. 8 is taken over the normalised vectors).
#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kIngestThreads = 1024;

__global__ void k_fg_count(const uint8_t* __restrict__ mask, int64_t n_pixels,
                           int32_t* __restrict__ block_counts) {
    int64_t i = (int64_t)blockIdx.x * kIngestThreads + threadIdx.x;
    bool fg = i < n_pixels && (mask == nullptr || mask[i] != 0);
    int c = __syncthreads_count(fg);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = c;
}

// Exclusive scan of block counts by one CTA; writes the total to dc->n_fg.
__global__ void k_scan_counts(int32_t* __restrict__ counts, int nb, DevCounters* dc) {
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += kIngestThreads) {
        int i = base + threadIdx.x;
        int v = i < nb ? counts[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = warp_sums[lane];
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_sums[lane] = wi - w;
        }
        __syncthreads();
        int excl = carry + warp_sums[wid] + incl - v;
        if (i < nb) counts[i] = excl;
        __syncthreads();
        if (threadIdx.x == kIngestThreads - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dc->n_fg = carry;
        dc->n_uncovered = carry;
    }
}

__global__ void k_compact_normalise(const float* __restrict__ emb, const uint8_t* __restrict__ mask,
                                    int64_t n_pixels, int d, int Dp,
                                    const int32_t* __restrict__ offsets, float* __restrict__ P32,
                                    int32_t* __restrict__ pix, DevCounters* dc) {
    __shared__ int32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t i = (int64_t)blockIdx.x * kIngestThreads + threadIdx.x;
    bool fg = i < n_pixels && (mask == nullptr || mask[i] != 0);
    unsigned bal = __ballot_sync(0xffffffffu, fg);
    if (lane == 0) warp_sums[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        int w = warp_sums[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - w;
    }
    __syncthreads();
    if (!fg) return;
    int pos = offsets[blockIdx.x] + warp_sums[wid] + __popc(bal & ((1u << lane) - 1u));
    const float* e = emb + i * d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(e[k], e[k], s);
    float nrm = sqrtf(s);
    if (!(nrm > 0.f) || !isfinite(nrm)) {
        atomicOr(&dc->status, 1);
        nrm = 1.f;
    }
    float* p = P32 + (int64_t)pos * Dp;
    for (int k = 0; k < d; ++k) p[k] = flush_tiny(e[k] / nrm);
    for (int k = d; k < Dp; ++k) p[k] = 0.f;
    pix[pos] = (int32_t)i;
}

}  // namespace

ms_status launch_ingest(ms_ctx* ctx) {
    int64_t nb = (ctx->n_pixels + kIngestThreads - 1) / kIngestThreads;
    if (nb == 0) nb = 1;
    k_fg_count<<<(unsigned)nb, kIngestThreads, 0, ctx->stream>>>(ctx->mask, ctx->n_pixels, ctx->block_tmp);
    MS_LAUNCH("k_fg_count");
    k_scan_counts<<<1, kIngestThreads, 0, ctx->stream>>>(ctx->block_tmp, (int)nb, ctx->dc);
    MS_LAUNCH("k_scan_counts");
    k_compact_normalise<<<(unsigned)nb, kIngestThreads, 0, ctx->stream>>>(
        ctx->emb, ctx->mask, ctx->n_pixels, ctx->d, ctx->Dp, ctx->block_tmp, ctx->P32, ctx->pix, ctx->dc);
    MS_LAUNCH("k_compact_normalise");
    ctx->launches += 3;
    return MS_OK;
}

}  // namespace ms
