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
// order, so results are deterministic. d = 16.
#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kVT = 128;          // threads per block
constexpr int kVSeeds = 256;      // seeds per work item (2 per thread)
constexpr int kVPixTile = 128;    // pixels per shared-memory stage
constexpr int kVD = 16;

struct VSplit {
    int tiles, chunks, chunk_len;
};

inline VSplit vsplit(int M, int64_t N, int target) {
    VSplit s;
    s.tiles = (M + kVSeeds - 1) / kVSeeds;
    const int max_chunks = (int)((N + kVPixTile - 1) / kVPixTile);
    int ch = (target + s.tiles - 1) / s.tiles;
    ch = ch < 1 ? 1 : (ch > max_chunks ? max_chunks : ch);
    int per = (int)((N + ch - 1) / ch);
    per = (per + kVPixTile - 1) / kVPixTile * kVPixTile;
    s.chunk_len = per;
    s.chunks = (int)((N + per - 1) / per);
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
// partial[item][k][r] = sum over the chunk of w p_k for seed t*256 + r.
__global__ void __launch_bounds__(kVT)
k_vmf_fwd_partial(const float* __restrict__ P, int64_t N, const float* __restrict__ X, int M, float kappa,
                  VSplit sp, float* __restrict__ partial) {
    __shared__ __align__(16) float tile[kVPixTile * kVD];
    const int item = blockIdx.x;
    const int t = item / sp.chunks, ch = item - t * sp.chunks;
    const int m0 = t * kVSeeds + threadIdx.x, m1 = m0 + kVT;
    float x0[16], x1[16], y0[16], y1[16];
    if (m0 < M) ld16(X + (int64_t)m0 * kVD, x0); else for (int k = 0; k < 16; ++k) x0[k] = 0.f;
    if (m1 < M) ld16(X + (int64_t)m1 * kVD, x1); else for (int k = 0; k < 16; ++k) x1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) y0[k] = y1[k] = 0.f;
    const int64_t p_begin = (int64_t)ch * sp.chunk_len;
    const int64_t p_end = min(N, p_begin + sp.chunk_len);
    for (int64_t pb = p_begin; pb < p_end; pb += kVPixTile) {
        const int cnt = (int)min((int64_t)kVPixTile, p_end - pb);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kVT)
            reinterpret_cast<float4*>(tile)[q] = reinterpret_cast<const float4*>(P + pb * kVD)[q];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float p[16];
            ld16(tile + j * kVD, p);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                s0 = fmaf(x0[k], p[k], s0);
                s1 = fmaf(x1[k], p[k], s1);
            }
            const float w0 = expf(kappa * (s0 - 1.f)), w1 = expf(kappa * (s1 - 1.f));
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                y0[k] = fmaf(w0, p[k], y0[k]);
                y1[k] = fmaf(w1, p[k], y1[k]);
            }
        }
    }
    float* out = partial + (size_t)item * kVD * kVSeeds;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        out[k * kVSeeds + threadIdx.x] = y0[k];
        out[k * kVSeeds + kVT + threadIdx.x] = y1[k];
    }
}

// One warp per seed: sum the chunk partials in a fixed order (lane-strided,
// then a fixed shuffle tree). Forward mode writes x' = y/|y| and |y|.
// Adjoint mode writes g = dL/dx (the sum itself) and the next gy from it.
__device__ __forceinline__ void warp_sum16(const float* __restrict__ partial, VSplit sp, int m, float (&s)[16]) {
    const int lane = threadIdx.x & 31;
    const int t = m / kVSeeds, r = m - t * kVSeeds;
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = 0.f;
    for (int ch = lane; ch < sp.chunks; ch += 32) {
        const float* in = partial + (size_t)(t * sp.chunks + ch) * kVD * kVSeeds + r;
#pragma unroll
        for (int k = 0; k < 16; ++k) s[k] += in[k * kVSeeds];
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

// Pass A: partial[item][k][r] = sum over the chunk of ds_mi p_ik.
__global__ void __launch_bounds__(kVT)
k_vmf_bwd_seeds(const float* __restrict__ P, int64_t N, const float* __restrict__ X, const float* __restrict__ GY,
                int M, float kappa, VSplit sp, float* __restrict__ partial) {
    __shared__ __align__(16) float tile[kVPixTile * kVD];
    const int item = blockIdx.x;
    const int t = item / sp.chunks, ch = item - t * sp.chunks;
    const int m0 = t * kVSeeds + threadIdx.x, m1 = m0 + kVT;
    float x0[16], x1[16], g0[16], g1[16], d0[16], d1[16];
    if (m0 < M) { ld16(X + (int64_t)m0 * kVD, x0); ld16(GY + (int64_t)m0 * kVD, g0); }
    else for (int k = 0; k < 16; ++k) x0[k] = g0[k] = 0.f;
    if (m1 < M) { ld16(X + (int64_t)m1 * kVD, x1); ld16(GY + (int64_t)m1 * kVD, g1); }
    else for (int k = 0; k < 16; ++k) x1[k] = g1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) d0[k] = d1[k] = 0.f;
    const int64_t p_begin = (int64_t)ch * sp.chunk_len;
    const int64_t p_end = min(N, p_begin + sp.chunk_len);
    for (int64_t pb = p_begin; pb < p_end; pb += kVPixTile) {
        const int cnt = (int)min((int64_t)kVPixTile, p_end - pb);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kVT)
            reinterpret_cast<float4*>(tile)[q] = reinterpret_cast<const float4*>(P + pb * kVD)[q];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float p[16];
            ld16(tile + j * kVD, p);
            float s0 = 0.f, s1 = 0.f, a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                s0 = fmaf(x0[k], p[k], s0);
                s1 = fmaf(x1[k], p[k], s1);
                a0 = fmaf(g0[k], p[k], a0);
                a1 = fmaf(g1[k], p[k], a1);
            }
            const float e0 = kappa * expf(kappa * (s0 - 1.f)) * a0;
            const float e1 = kappa * expf(kappa * (s1 - 1.f)) * a1;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                d0[k] = fmaf(e0, p[k], d0[k]);
                d1[k] = fmaf(e1, p[k], d1[k]);
            }
        }
    }
    float* out = partial + (size_t)item * kVD * kVSeeds;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        out[k * kVSeeds + threadIdx.x] = d0[k];
        out[k * kVSeeds + kVT + threadIdx.x] = d1[k];
    }
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

// Pass B: one thread per pixel, all seeds from shared memory.
__global__ void __launch_bounds__(kVT)
k_vmf_bwd_pixels(const float* __restrict__ P, int64_t N, const float* __restrict__ X, const float* __restrict__ GY,
                 int M, float kappa, float* __restrict__ dP) {
    __shared__ __align__(16) float sx[64 * kVD];
    __shared__ __align__(16) float sg[64 * kVD];
    const int64_t i = (int64_t)blockIdx.x * kVT + threadIdx.x;
    const bool act = i < N;
    float p[16], dp[16];
    if (act) { ld16(P + i * kVD, p); ld16(dP + i * kVD, dp); }
    else for (int k = 0; k < 16; ++k) p[k] = dp[k] = 0.f;
    for (int base = 0; base < M; base += 64) {
        const int cnt = min(64, M - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * 4; q += kVT) {
            reinterpret_cast<float4*>(sx)[q] = reinterpret_cast<const float4*>(X + (int64_t)base * kVD)[q];
            reinterpret_cast<float4*>(sg)[q] = reinterpret_cast<const float4*>(GY + (int64_t)base * kVD)[q];
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float x[16], g[16];
            ld16(sx + j * kVD, x);
            ld16(sg + j * kVD, g);
            float s = 0.f, a = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                s = fmaf(x[k], p[k], s);
                a = fmaf(g[k], p[k], a);
            }
            const float w = expf(kappa * (s - 1.f));
            const float ds = kappa * w * a;
#pragma unroll
            for (int k = 0; k < 16; ++k) dp[k] = fmaf(w, g[k], fmaf(ds, x[k], dp[k]));
        }
    }
    if (act)
#pragma unroll
        for (int k = 0; k < 16; ++k) dP[i * kVD + k] = dp[k];
}

struct VmfWork {
    float* partial;
    float* iters;   // [T+1, M, 16]
    float* ynorm;   // [T, M]
    float* gy;      // [M, 16]
    float* g;       // [M, 16]
    VSplit sp;
};

int vmf_target(int* sms_out) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *sms_out = sms;
    return 4 * sms;
}

ms_status vmf_validate(const float* P, int64_t N, const float* X0, int32_t M, int32_t dim, double kappa, int32_t T) {
    if (!P || !X0) return set_error(MS_ERR_INVALID_ARG, "NULL input");
    if (dim != 16) return set_error(MS_ERR_INVALID_ARG, "the vMF form supports dim = 16");
    if (N < 1 || M < 1 || T < 0 || N >= (1LL << 31)) return set_error(MS_ERR_INVALID_ARG, "bad sizes");
    if (!(kappa >= 0.0 && kappa < 80.0)) return set_error(MS_ERR_INVALID_ARG, "kappa must be in [0, 80)");
    return MS_OK;
}

ms_status vmf_alloc(VmfWork* w, int64_t N, int32_t M, int32_t T, cudaStream_t st) {
    int sms = 1;
    const int target = vmf_target(&sms);
    w->sp = vsplit(M, N, target);
    const size_t items = (size_t)w->sp.tiles * w->sp.chunks;
    const size_t bytes = items * kVD * kVSeeds * sizeof(float) + (size_t)(T + 1) * M * kVD * sizeof(float) +
                         (size_t)(T > 0 ? T : 1) * M * sizeof(float) + 2 * (size_t)M * kVD * sizeof(float) + 4 * 256;
    char* b = nullptr;
    MS_CUDA(cudaMallocAsync((void**)&b, bytes, st));
    auto take = [&](size_t n) {
        char* p = b;
        b += (n + 255) / 256 * 256;
        return (float*)p;
    };
    w->partial = take(items * kVD * kVSeeds * sizeof(float));
    w->iters = take((size_t)(T + 1) * M * kVD * sizeof(float));
    w->ynorm = take((size_t)(T > 0 ? T : 1) * M * sizeof(float));
    w->gy = take((size_t)M * kVD * sizeof(float));
    w->g = take((size_t)M * kVD * sizeof(float));
    return MS_OK;
}

// Runs the T forward steps, keeping x_0..x_T in w->iters and |y_t| in w->ynorm.
ms_status vmf_forward_steps(const float* P, int64_t N, const float* X0, int32_t M, float kappa, int32_t T,
                            VmfWork* w, cudaStream_t st) {
    MS_CUDA(cudaMemcpyAsync(w->iters, X0, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st));
    const unsigned items = (unsigned)(w->sp.tiles * w->sp.chunks);
    const unsigned rblocks = (unsigned)((M + 7) / 8);
    for (int t = 0; t < T; ++t) {
        const float* Xt = w->iters + (size_t)t * M * kVD;
        float* Xn = w->iters + (size_t)(t + 1) * M * kVD;
        k_vmf_fwd_partial<<<items, kVT, 0, st>>>(P, N, Xt, M, kappa, w->sp, w->partial);
        MS_LAUNCH("k_vmf_fwd_partial");
        k_vmf_fwd_reduce<<<rblocks, 256, 0, st>>>(w->partial, w->sp, M, Xn, w->ynorm + (size_t)t * M);
        MS_LAUNCH("k_vmf_fwd_reduce");
    }
    return MS_OK;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_vmf_forward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                    double kappa, int32_t T, float* d_XT, void* stream) {
    ms_status s = vmf_validate(d_P, N, d_X0, M, dim, kappa, T);
    if (s != MS_OK) return s;
    if (!d_XT) return set_error(MS_ERR_INVALID_ARG, "d_XT is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    VmfWork w;
    s = vmf_alloc(&w, N, M, T, st);
    if (s != MS_OK) return s;
    char* base = (char*)w.partial;
    s = vmf_forward_steps(d_P, N, d_X0, M, (float)kappa, T, &w, st);
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(d_XT, w.iters + (size_t)T * M * kVD, sizeof(float) * (size_t)M * kVD,
                                       cudaMemcpyDeviceToDevice, st), "copy x_T");
    cudaFreeAsync(base, st);
    return s;
}

extern "C" ms_status ms_vmf_backward(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                     double kappa, int32_t T, const float* d_GT, float* d_dP, float* d_dX0,
                                     void* stream) {
    ms_status s = vmf_validate(d_P, N, d_X0, M, dim, kappa, T);
    if (s != MS_OK) return s;
    if (!d_GT || !d_dP || !d_dX0) return set_error(MS_ERR_INVALID_ARG, "NULL output or upstream gradient");
    cudaStream_t st = (cudaStream_t)stream;
    VmfWork w;
    s = vmf_alloc(&w, N, M, T, st);
    if (s != MS_OK) return s;
    char* base = (char*)w.partial;
    const float kf = (float)kappa;
    s = vmf_forward_steps(d_P, N, d_X0, M, kf, T, &w, st);
    if (s == MS_OK) s = cuda_check(cudaMemsetAsync(d_dP, 0, sizeof(float) * (size_t)N * kVD, st), "memset dP");
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(w.g, d_GT, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st),
                       "copy g_T");
    const unsigned items = (unsigned)(w.sp.tiles * w.sp.chunks);
    const unsigned rblocks = (unsigned)((M + 7) / 8);
    for (int t = T - 1; t >= 0 && s == MS_OK; --t) {
        const float* Xt = w.iters + (size_t)t * M * kVD;
        const float* Xn = w.iters + (size_t)(t + 1) * M * kVD;
        k_vmf_gy<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(w.g, Xn, w.ynorm + (size_t)t * M, M, w.gy);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_gy")) != MS_OK) break;
        k_vmf_bwd_pixels<<<(unsigned)((N + kVT - 1) / kVT), kVT, 0, st>>>(d_P, N, Xt, w.gy, M, kf, d_dP);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_bwd_pixels")) != MS_OK) break;
        k_vmf_bwd_seeds<<<items, kVT, 0, st>>>(d_P, N, Xt, w.gy, M, kf, w.sp, w.partial);
        if ((s = cuda_check(cudaGetLastError(), "k_vmf_bwd_seeds")) != MS_OK) break;
        k_vmf_bwd_reduce<<<rblocks, 256, 0, st>>>(w.partial, w.sp, M, w.g);
        s = cuda_check(cudaGetLastError(), "k_vmf_bwd_reduce");
    }
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(d_dX0, w.g, sizeof(float) * (size_t)M * kVD, cudaMemcpyDeviceToDevice, st),
                       "copy dX0");
    cudaFreeAsync(base, st);
    return s;
}
