// Labelling (the labelling step of Algorithm 2): every foreground vector takes the
// mode of highest cosine, lowest index on ties; background stays -1.
//
// FP32 form (the BF16 form labels on the tensor cores, ms_label_tc.cu, with
// the same result): a thread owns one pixel and scans the modes from shared
// memory in FP32, keeping the best and second-best scores. When the two are
// within 2*kEpsF32 the winner is re-decided in FP64 among the modes whose FP32
// score is within 2*kEpsF32 of the best, from the raw embedding: the FP64
// argmax always lies in that set, so the label is the exact FP64 argmax over
// the modes.
#include "ms_batch.cuh"
#include "ms_device.cuh"

namespace ms {
namespace {

constexpr int kLT = 256;
constexpr int kLV = 64;

template <int Dp>
__global__ void __launch_bounds__(kLT)
k_label(const float* __restrict__ P32, const float* __restrict__ emb, int d,
        const int32_t* __restrict__ pix, int n, const float* __restrict__ modes, int K,
        int32_t* __restrict__ labels) {
    __shared__ __align__(16) float tile[kLV * Dp];
    const int i = blockIdx.x * kLT + threadIdx.x;
    const bool act = i < n;
    float p[Dp];
    if (act) {
#pragma unroll
        for (int k = 0; k < Dp; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(P32 + (int64_t)i * Dp + k);
            p[k] = v.x; p[k + 1] = v.y; p[k + 2] = v.z; p[k + 3] = v.w;
        }
    }
    float b1 = -INFINITY, b2 = -INFINITY;
    int best = -1;
    for (int base = 0; base < K; base += kLV) {
        const int cnt = min(kLV, K - base);
        for (int q = threadIdx.x; q < cnt * Dp; q += kLT) tile[q] = modes[(int64_t)base * Dp + q];
        __syncthreads();
        if (act) {
            for (int j = 0; j < cnt; ++j) {
                const float s = dot_seq<Dp>(p, tile + j * Dp);
                if (s > b1) {
                    b2 = b1;
                    b1 = s;
                    best = base + j;
                } else if (s > b2) {
                    b2 = s;
                }
            }
        }
        __syncthreads();
    }
    if (!act) return;
    if (K > 1 && b1 - b2 <= 2.f * kEpsF32) {
        const float* e = emb + (int64_t)pix[i] * d;
        double bc = -INFINITY;
        for (int k = 0; k < K; ++k) {
            const float* m = modes + (int64_t)k * Dp;
            if (dot_seq<Dp>(p, m) < b1 - 2.f * kEpsF32) continue;
            const double cs = cos64(e, m, d);
            if (cs > bc) {
                bc = cs;
                best = k;
            }
        }
    }
    labels[pix[i]] = best;
}

}  // namespace

ms_status launch_label(ms_ctx* ctx, int32_t* d_labels) {
    MS_CUDA(cudaMemsetAsync(d_labels, 0xff, sizeof(int32_t) * (size_t)ctx->n_pixels, ctx->stream));
    if (ctx->n == 0) return MS_OK;
    if (ctx->Mk) {
        // BF16 form: the tensor-core kernel, same labels (exact FP64 argmax)
        LabelTcScratch sc{ctx->label_fix, (int*)(ctx->label_fix + ctx->n), nullptr};
        const ms_status s = launch_label_tc_single(ctx->pmap, ctx->pmap1, ctx->Mk, ctx->n_pad, ctx->Dp, ctx->modes,
                                                   ctx->n_kept, (int)ctx->n, ctx->P32, ctx->pix, ctx->emb, ctx->d,
                                                   d_labels, sc, ctx->num_sms, &ctx->dc->status, ctx->stream);
        ctx->launches += ctx->n_kept > 1 ? 3 : 2;
        return s;
    }
    const unsigned g = (unsigned)((ctx->n + kLT - 1) / kLT);
    if (ctx->Dp == 16)
        k_label<16><<<g, kLT, 0, ctx->stream>>>(ctx->P32, ctx->emb, ctx->d, ctx->pix, (int)ctx->n,
                                                ctx->modes, ctx->n_kept, d_labels);
    else
        k_label<32><<<g, kLT, 0, ctx->stream>>>(ctx->P32, ctx->emb, ctx->d, ctx->pix, (int)ctx->n,
                                                ctx->modes, ctx->n_kept, d_labels);
    MS_LAUNCH("k_label");
    ctx->launches += 1;
    return MS_OK;
}

}  // namespace ms
