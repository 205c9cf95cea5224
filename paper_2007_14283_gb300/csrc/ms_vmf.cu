// Smooth-kernel (von Mises-Fisher) mean-shift: T unrolled steps and their
// hand-written adjoint.
//
// The kernel family of Eq. 2 with the exponential profile instead of the flat
// kernel of Eq. 11. Each step moves every seed to the kernel-weighted mean of
// all pixels (the dense update of Sec. 3.2.1) and renormalises it:
//     s_mi = x_m . p_i,  w_mi = exp(kappa (s_mi - 1)),  y_m = sum_i w_mi p_i,
//     x'_m = y_m / |y_m|.
// (The factor exp(-kappa) cancels in the normalisation; it keeps w <= 1 in
// FP32.) Pixels are unconstrained inputs, seeds are not renormalised before
// the first step.
//
// Adjoint of one step, with g = dL/dx' given:
//     gy_m  = (g_m - x'_m (x'_m . g_m)) / |y_m|
//     a_mi  = gy_m . p_i,   ds_mi = kappa w_mi a_mi
//     dL/dx_m  = sum_i ds_mi p_i                      (pass A: seeds x pixel chunks)
//     dL/dp_i += sum_m (w_mi gy_m + ds_mi x_m)         (pass B: one thread per pixel)
// The backward call re-runs the forward to rebuild x_0..x_T and |y_t| (a few
// hundred KB) and recomputes every w_mi tile on the fly; no M x N matrix is
// ever stored. Reductions go through per-chunk partial sums added in a fixed
// order, so results are deterministic for a given GPU (the chunks fill one wave
// of resident blocks). The weights are evaluated as 2^(kappa log2(e) (s - 1))
// with exp2f. d = 16. The BF16 form runs the forward steps (ms_vmf_tc.cu) and
// both reverse passes (ms_vmf_tc_adj.cu) on the tensor cores instead.
#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kVPixTile = 128;    // pixels per shared-memory stage
constexpr int kVD = 16;
// Forward: 128 threads x 4 seeds = 512 seeds per work item. Adjoint pass A:
// 128 threads x 2 seeds = 256 seeds per item (three 16-vectors per seed).
// Adjoint pass B: 128 threads x 2 pixels.
constexpr int kFT = 128, kFS = 4, kFSeeds = kFT * kFS;
constexpr int kAT = 128, kAS = 2, kASeeds = kAT * kAS;
constexpr int kBT = 128, kBP = 2;

struct VSplit {
    int tiles, chunks, chunk_len, seeds;  // seed tiles of `seeds`, pixel chunks of chunk_len
};

// Seed tiles x pixel chunks filling one wave of `slots` resident blocks
// (chunks of any length: the stage loop handles a partial last stage).
inline VSplit vsplit(int M, int64_t N, int slots, int seeds) {
    VSplit s;
    s.seeds = seeds;
    s.tiles = (M + seeds - 1) / seeds;
    int ch = slots / s.tiles;
    ch = ch < 1 ? 1 : (int64_t)ch > N ? (int)N : ch;
    s.chunk_len = (int)((N + ch - 1) / ch);
    s.chunks = (int)((N + s.chunk_len - 1) / s.chunk_len);
    return s;
}

__device__ __forceinline__ void ld16(const float* src, float (&v)[16]) {
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
        const float4 a = *reinterpret_cast<const float4*>(src + k);
        v[k] = a.x; v[k + 1] = a.y; v[k + 2] = a.z; v[k + 3] = a.w;
    }
}

// Forward partial sums: for seed tile t and pixel chunk ch,
// partial[item][k][r] = sum over the chunk of w p_k for seed t*512 + r.
// Thread j holds seeds j, j+128, j+256, j+384 of the tile; every pixel of a
// stage is read once from shared memory for all four.
__global__ void __launch_bounds__(kFT)
k_vmf_fwd_partial(const float* __restrict__ P, int64_t N, const float* __restrict__ X, int M, float kappa,
                  VSplit sp, float* __restrict__ partial) {
    const float kl2 = kappa * 1.4426950408889634f;  // exp(kappa u) = 2^(kappa log2(e) u)
    __shared__ __align__(16) float tile[kVPixTile * kVD];
    const int item = blockIdx.x;
    const int t = item / sp.chunks, ch = item - t * sp.chunks;
    float x[kFS][16], y[kFS][16];
#pragma unroll
    for (int q = 0; q < kFS; ++q) {
        const int m = t * kFSeeds + q * kFT + threadIdx.x;
        if (m < M) ld16(X + (int64_t)m * kVD, x[q]);
        else
#pragma unroll
            for (int k = 0; k < 16; ++k) x[q][k] = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) y[q][k] = 0.f;
    }
    const int64_t p_begin = (int64_t)ch * sp.chunk_len;
    const int64_t p_end = min(N, p_begin + sp.chunk_len);
    for (int64_t pb = p_begin; pb < p_end; pb += kVPixTile) {
        const int cnt = (int)min((int64_t)kVPixTile, p_end - pb);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kFT)
            reinterpret_cast<float4*>(tile)[q] = reinterpret_cast<const float4*>(P + pb * kVD)[q];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float p[16];
            ld16(tile + j * kVD, p);
            float w[kFS];
#pragma unroll
            for (int q = 0; q < kFS; ++q) {
                float sc = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) sc = fmaf(x[q][k], p[k], sc);
                w[q] = exp2f(kl2 * (sc - 1.f));
            }
#pragma unroll
            for (int q = 0; q < kFS; ++q)
#pragma unroll
                for (int k = 0; k < 16; ++k) y[q][k] = fmaf(w[q], p[k], y[q][k]);
        }
    }
    float* out = partial + (size_t)item * kVD * kFSeeds;
#pragma unroll
    for (int q = 0; q < kFS; ++q)
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k * kFSeeds + q * kFT + threadIdx.x] = y[q][k];
}

// One warp per seed: sum the chunk partials in a fixed order (lane-strided,
// then a fixed shuffle tree). Forward mode writes x' = y/|y| and |y|.
// Adjoint mode writes g = dL/dx (the sum itself) and the next gy from it.
__device__ __forceinline__ void warp_sum16(const float* __restrict__ partial, VSplit sp, int m, float (&s)[16]) {
    const int lane = threadIdx.x & 31;
    const int t = m / sp.seeds, r = m - t * sp.seeds;
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = 0.f;
    for (int ch = lane; ch < sp.chunks; ch += 32) {
        const float* in = partial + (size_t)(t * sp.chunks + ch) * kVD * sp.seeds + r;
#pragma unroll
        for (int k = 0; k < 16; ++k) s[k] += in[k * sp.seeds];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
}

__global__ void k_vmf_fwd_reduce(const float* __restrict__ partial, VSplit sp, int M, float* __restrict__ Xn,
                                 float* __restrict__ ynorm) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (m >= M) return;
    float y[16];
    warp_sum16(partial, sp, m, y);
    if ((threadIdx.x & 31) == 0) {
        float ss = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) ss = fmaf(y[k], y[k], ss);
        const float yn = sqrtf(ss);
#pragma unroll
        for (int k = 0; k < 16; ++k) Xn[(int64_t)m * kVD + k] = y[k] / yn;
        if (ynorm) ynorm[m] = yn;
    }
}

// gy = (g - x (x . g)) / |y| for every seed.
__global__ void k_vmf_gy(const float* __restrict__ G, const float* __restrict__ Xn, const float* __restrict__ ynorm,
                         int M, float* __restrict__ GY) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float g[16], x[16];
    ld16(G + (int64_t)m * kVD, g);
    ld16(Xn + (int64_t)m * kVD, x);
    float xg = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) xg = fmaf(x[k], g[k], xg);
    const float inv = 1.f / ynorm[m];
#pragma unroll
    for (int k = 0; k < 16; ++k) GY[(int64_t)m * kVD + k] = (g[k] - x[k] * xg) * inv;
}

// Pass A: partial[item][k][r] = sum over the chunk of ds_mi p_ik, for seed
// t*256 + r (thread j holds seeds j and j+128).
__global__ void __launch_bounds__(kAT)
k_vmf_bwd_seeds(const float* __restrict__ P, int64_t N, const float* __restrict__ X, const float* __restrict__ GY,
                int M, float kappa, VSplit sp, float* __restrict__ partial) {
    const float kl2 = kappa * 1.4426950408889634f;  // exp(kappa u) = 2^(kappa log2(e) u)
    __shared__ __align__(16) float tile[kVPixTile * kVD];
    const int item = blockIdx.x;
    const int t = item / sp.chunks, ch = item - t * sp.chunks;
    float x[kAS][16], g[kAS][16], dd[kAS][16];
#pragma unroll
    for (int q = 0; q < kAS; ++q) {
        const int m = t * kASeeds + q * kAT + threadIdx.x;
        if (m < M) {
            ld16(X + (int64_t)m * kVD, x[q]);
            ld16(GY + (int64_t)m * kVD, g[q]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) x[q][k] = g[q][k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) dd[q][k] = 0.f;
    }
    const int64_t p_begin = (int64_t)ch * sp.chunk_len;
    const int64_t p_end = min(N, p_begin + sp.chunk_len);
    for (int64_t pb = p_begin; pb < p_end; pb += kVPixTile) {
        const int cnt = (int)min((int64_t)kVPixTile, p_end - pb);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kAT)
            reinterpret_cast<float4*>(tile)[q] = reinterpret_cast<const float4*>(P + pb * kVD)[q];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float p[16];
            ld16(tile + j * kVD, p);
            float e[kAS];
#pragma unroll
            for (int q = 0; q < kAS; ++q) {
                float sc = 0.f, a = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    sc = fmaf(x[q][k], p[k], sc);
                    a = fmaf(g[q][k], p[k], a);
                }
                e[q] = kappa * exp2f(kl2 * (sc - 1.f)) * a;
            }
#pragma unroll
            for (int q = 0; q < kAS; ++q)
#pragma unroll
                for (int k = 0; k < 16; ++k) dd[q][k] = fmaf(e[q], p[k], dd[q][k]);
        }
    }
    float* out = partial + (size_t)item * kVD * kASeeds;
#pragma unroll
    for (int q = 0; q < kAS; ++q)
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k * kASeeds + q * kAT + threadIdx.x] = dd[q][k];
}

__global__ void k_vmf_bwd_reduce(const float* __restrict__ partial, VSplit sp, int M, float* __restrict__ G) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (m >= M) return;
    float s[16];
    warp_sum16(partial, sp, m, s);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 16; ++k) G[(int64_t)m * kVD + k] = s[k];
}

// Pass B: two pixels per thread (i and i + 128 of the block's 256), all
// seeds from shared memory; each seed's x and gy are read once for both.
__global__ void __launch_bounds__(kBT)
k_vmf_bwd_pixels(const float* __restrict__ P, int64_t N, const float* __restrict__ X, const float* __restrict__ GY,
                 int M, float kappa, float* __restrict__ dP) {
    const float kl2 = kappa * 1.4426950408889634f;  // exp(kappa u) = 2^(kappa log2(e) u)
    __shared__ __align__(16) float sx[64 * kVD];
    __shared__ __align__(16) float sg[64 * kVD];
    float p[kBP][16], dp[kBP][16];
    int64_t idx[kBP];
    bool act[kBP];
#pragma unroll
    for (int u = 0; u < kBP; ++u) {
        idx[u] = (int64_t)blockIdx.x * (kBT * kBP) + u * kBT + threadIdx.x;
        act[u] = idx[u] < N;
        if (act[u]) {
            ld16(P + idx[u] * kVD, p[u]);
            ld16(dP + idx[u] * kVD, dp[u]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) p[u][k] = dp[u][k] = 0.f;
        }
    }
    for (int base = 0; base < M; base += 64) {
        const int cnt = min(64, M - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kBT) {
            reinterpret_cast<float4*>(sx)[q] = reinterpret_cast<const float4*>(X + (int64_t)base * kVD)[q];
            reinterpret_cast<float4*>(sg)[q] = reinterpret_cast<const float4*>(GY + (int64_t)base * kVD)[q];
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float x[16], g[16];
            ld16(sx + j * kVD, x);
            ld16(sg + j * kVD, g);
#pragma unroll
            for (int u = 0; u < kBP; ++u) {
                float sc = 0.f, a = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    sc = fmaf(x[k], p[u][k], sc);
                    a = fmaf(g[k], p[u][k], a);
                }
                const float w = exp2f(kl2 * (sc - 1.f));
                const float ds = kappa * w * a;
#pragma unroll
                for (int k = 0; k < 16; ++k) dp[u][k] = fmaf(w, g[k], fmaf(ds, x[k], dp[u][k]));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kBP; ++u)
        if (act[u])
#pragma unroll
            for (int k = 0; k < 16; ++k) dP[idx[u] * kVD + k] = dp[u][k];
}

struct VmfWork {
    bool tc;        // steps and adjoint passes on the tensor cores (BF16 splits)
    void* Pk;       // tc: BF16 split rows of P
    float* tc_partial;
    int* status;    // tc: raised by a bounded wait that gave up
    CUtensorMap pmap;
    VmfTcPlan plan;
    float* partial;
    float* iters;   // [T+1, M, 16]
    float* ynorm;   // [T, M]
    float* gy;      // [M, 16]
    float* g;       // [M, 16]
    VmfAdjWork adj; // tc backward: the tensor-core adjoint's plans, maps and buffers
    VSplit sp;      // forward items (512-seed tiles)
    VSplit spa;     // adjoint pass A items (256-seed tiles)
    void* adj_ws;   // tc backward: workspace of the tensor-core adjoint
    int sms;
};

// Resident blocks of a kernel over the whole GPU (blocks per SM x SMs).
template <class K>
int vmf_slots(K kernel, int threads) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess || per < 1) per = 1;
    return per * sms;
}

ms_status vmf_validate(const float* P, int64_t N, const float* X0, int32_t M, int32_t dim, double kappa, int32_t T) {
    if (!P || !X0) return set_error(MS_ERR_INVALID_ARG, "NULL input");
    if (dim != 16) return set_error(MS_ERR_INVALID_ARG, "the vMF form supports dim = 16");
    if (N < 1 || M < 1 || T < 0 || N >= (1LL << 31)) return set_error(MS_ERR_INVALID_ARG, "bad sizes");
    if (!(kappa >= 0.0 && kappa < 80.0)) return set_error(MS_ERR_INVALID_ARG, "kappa must be in [0, 80)");
    return MS_OK;
}

ms_status vmf_alloc(VmfWork* w, int64_t N, int32_t M, int32_t T, bool tc, bool adjoint, cudaStream_t st) {
    w->tc = tc;
    w->sp = vsplit(M, N, vmf_slots(k_vmf_fwd_partial, kFT), kFSeeds);
    w->spa = vsplit(M, N, vmf_slots(k_vmf_bwd_seeds, kAT), kASeeds);
    const size_t pf = (size_t)w->sp.tiles * w->sp.chunks * kFSeeds, pa = (size_t)w->spa.tiles * w->spa.chunks * kASeeds;
    const size_t pmax = pf > pa ? pf : pa;
    size_t tc_bytes = 0, adj_bytes = 0;
    w->sms = 1;
    if (tc) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, dev);
        w->plan = vmf_tc_plan(M, N, w->sms);
        tc_bytes = vmf_tc_pk_bytes(N) + (size_t)w->plan.items * 128 * kVD * sizeof(float) + 3 * 256;
        if (adjoint) adj_bytes = vmf_adj_bytes(M, N, w->sms) + 256;
    }
    const size_t bytes = pmax * kVD * sizeof(float) + (size_t)(T + 1) * M * kVD * sizeof(float) +
                         (size_t)(T > 0 ? T : 1) * M * sizeof(float) + 2 * (size_t)M * kVD * sizeof(float) + 4 * 256 +
                         tc_bytes + adj_bytes;
    char* b = nullptr;
    MS_CUDA(scratch_malloc_async((void**)&b, bytes, st));
    auto take = [&](size_t n) {
        char* p = b;
        b += (n + 255) / 256 * 256;
        return (float*)p;
    };
    w->partial = take(pmax * kVD * sizeof(float));
    w->iters = take((size_t)(T + 1) * M * kVD * sizeof(float));
    w->ynorm = take((size_t)(T > 0 ? T : 1) * M * sizeof(float));
    w->gy = take((size_t)M * kVD * sizeof(float));
    w->g = take((size_t)M * kVD * sizeof(float));
    w->Pk = nullptr;
    w->tc_partial = nullptr;
    w->status = nullptr;
    w->adj_ws = nullptr;
    if (tc) {
        w->Pk = take(vmf_tc_pk_bytes(N));
        w->tc_partial = take((size_t)w->plan.items * 128 * kVD * sizeof(float));
        w->status = (int*)take(sizeof(int));
        if (adjoint) w->adj_ws = take(adj_bytes - 256);
    }
    return MS_OK;
}

// Runs the T forward steps, keeping x_0..x_T in w->iters and |y_t| in w->ynorm.
ms_status vmf_forward_steps(const float* P, int64_t N, const float* X0, int32_t M, float kappa, int32_t T,
                            VmfWork* w, cudaStream_t st) {
    MS_CUDA(cudaMemcpyAsync(w->iters, X0, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st));
    if (w->tc) {
        MS_CUDA(cudaMemsetAsync(w->status, 0, sizeof(int), st));
        if (ms_status s = vmf_tc_prepare(P, N, w->Pk, &w->pmap, st); s != MS_OK) return s;
        for (int t = 0; t < T; ++t) {
            ms_status s = vmf_tc_step(w->pmap, w->iters + (size_t)t * M * kVD, M, kappa, w->plan, w->tc_partial,
                                      w->status, w->iters + (size_t)(t + 1) * M * kVD, w->ynorm + (size_t)t * M, st);
            if (s != MS_OK) return s;
        }
        // the tensor-core steps end in a status check (a bounded wait may have given up)
        int h_status = 0;
        MS_CUDA(cudaMemcpyAsync(&h_status, w->status, sizeof(int), cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
        if (h_status) return set_error(MS_ERR_TIMEOUT, "a bounded device wait in k_vmf_tc gave up");
        return MS_OK;
    }
    const unsigned items = (unsigned)(w->sp.tiles * w->sp.chunks);
    const unsigned rblocks = (unsigned)((M + 7) / 8);
    for (int t = 0; t < T; ++t) {
        const float* Xt = w->iters + (size_t)t * M * kVD;
        float* Xn = w->iters + (size_t)(t + 1) * M * kVD;
        k_vmf_fwd_partial<<<items, kFT, 0, st>>>(P, N, Xt, M, kappa, w->sp, w->partial);
        MS_LAUNCH("k_vmf_fwd_partial");
        k_vmf_fwd_reduce<<<rblocks, 256, 0, st>>>(w->partial, w->sp, M, Xn, w->ynorm + (size_t)t * M);
        MS_LAUNCH("k_vmf_fwd_reduce");
    }
    return MS_OK;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_vmf_forward_ex(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                       double kappa, int32_t T, int32_t precision, float* d_XT, void* stream) {
    ms_status s = vmf_validate(d_P, N, d_X0, M, dim, kappa, T);
    if (s != MS_OK) return s;
    if (!d_XT) return set_error(MS_ERR_INVALID_ARG, "d_XT is NULL");
    if (precision != MS_FP32 && precision != MS_BF16) return set_error(MS_ERR_INVALID_ARG, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    VmfWork w;
    s = vmf_alloc(&w, N, M, T, precision == MS_BF16, false, st);
    if (s != MS_OK) return s;
    char* base = (char*)w.partial;
    s = vmf_forward_steps(d_P, N, d_X0, M, (float)kappa, T, &w, st);
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(d_XT, w.iters + (size_t)T * M * kVD, sizeof(float) * (size_t)M * kVD,
                                       cudaMemcpyDeviceToDevice, st), "copy x_T");
    cudaFreeAsync(base, st);
    return s;
}

extern "C" ms_status ms_vmf_backward_ex(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                        double kappa, int32_t T, int32_t precision, const float* d_GT, float* d_dP,
                                        float* d_dX0, void* stream) {
    ms_status s = vmf_validate(d_P, N, d_X0, M, dim, kappa, T);
    if (s != MS_OK) return s;
    if (!d_GT || !d_dP || !d_dX0) return set_error(MS_ERR_INVALID_ARG, "NULL output or upstream gradient");
    if (precision != MS_FP32 && precision != MS_BF16) return set_error(MS_ERR_INVALID_ARG, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    VmfWork w;
    s = vmf_alloc(&w, N, M, T, precision == MS_BF16, true, st);
    if (s != MS_OK) return s;
    char* base = (char*)w.partial;
    const float kf = (float)kappa;
    s = vmf_forward_steps(d_P, N, d_X0, M, kf, T, &w, st);
    // BF16 form: the reverse passes on the tensor cores, over the split
    // pixel rows the forward steps packed
    if (s == MS_OK && w.tc) s = vmf_adj_prepare(w.Pk, N, M, w.sms, w.adj_ws, &w.adj);
    if (s == MS_OK) s = cuda_check(cudaMemsetAsync(d_dP, 0, sizeof(float) * (size_t)N * kVD, st), "memset dP");
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(w.g, d_GT, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st),
                       "copy g_T");
    if (s == MS_OK && w.tc) s = vmf_adj_backward(&w.adj, w.iters, w.ynorm, T, kf, d_GT, w.status, d_dP, d_dX0, st);
    const unsigned items = (unsigned)(w.spa.tiles * w.spa.chunks);
    const unsigned rblocks = (unsigned)((M + 7) / 8);
    for (int t = T - 1; t >= 0 && s == MS_OK && !w.tc; --t) {
        const float* Xt = w.iters + (size_t)t * M * kVD;
        const float* Xn = w.iters + (size_t)(t + 1) * M * kVD;
        k_vmf_gy<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(w.g, Xn, w.ynorm + (size_t)t * M, M, w.gy);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_gy")) != MS_OK) break;
        k_vmf_bwd_pixels<<<(unsigned)((N + kBT * kBP - 1) / (kBT * kBP)), kBT, 0, st>>>(d_P, N, Xt, w.gy, M, kf,
                                                                                    d_dP);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_bwd_pixels")) != MS_OK) break;
        k_vmf_bwd_seeds<<<items, kAT, 0, st>>>(d_P, N, Xt, w.gy, M, kf, w.spa, w.partial);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_bwd_seeds")) != MS_OK) break;
        k_vmf_bwd_reduce<<<rblocks, 256, 0, st>>>(w.partial, w.spa, M, w.g);
        s = cuda_check(cudaGetLastError(), "k_vmf_bwd_reduce");
    }
    if (s == MS_OK && !w.tc)
        s = cuda_check(cudaMemcpyAsync(d_dX0, w.g, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st),
                       "copy dX0");
    if (s == MS_OK && w.tc && T > 0) {  // a bounded wait in the tensor-core passes may have given up
        int h_status = 0;
        s = cuda_check(cudaMemcpyAsync(&h_status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
        if (s == MS_OK) s = cuda_check(cudaStreamSynchronize(st), "synchronise");
        if (s == MS_OK && h_status) s = set_error(MS_ERR_TIMEOUT, "a bounded device wait in k_vmf_adj_tc gave up");
    }
    cudaFreeAsync(base, st);
    return s;
}

extern "C" ms_status ms_vmf_forward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                    double kappa, int32_t T, float* d_XT, void* stream) {
    return ms_vmf_forward_ex(d_P, N, d_X0, M, dim, kappa, T, MS_FP32, d_XT, stream);
}

extern "C" ms_status ms_vmf_backward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                     double kappa, int32_t T, const float* d_GT, float* d_dP, float* d_dX0,
                                     void* stream) {
    return ms_vmf_backward_ex(d_P, N, d_X0, M, dim, kappa, T, MS_FP32, d_GT, d_dP, d_dX0, stream);
}
