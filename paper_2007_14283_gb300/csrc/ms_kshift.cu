// Mean-shift with other distances and kernel profiles (Eq. 2-6; Eq. 3, 4, 9).
//
// T steps of the dense update (Sec. 3.2.1: every seed against every vector)
// with weights from a kernel profile of the scaled squared distance:
//     t_mi = (d(x_m, p_i) / h)^2,   w_mi = k(t_mi),
//     x'_m = sum_i w_mi p_i / sum_i w_mi            (Eq. 6 as an update)
// d is the Euclidean distance of Eq. 4 on the vectors as given, or the cosine
// distance 1 - cos of Eq. 9, for which vectors are normalised once and x' is
// renormalised to the unit sphere. k is flat [t <= 1] (Eq. 3), Epanechnikov
// max(0, 1 - t) or Gaussian exp(-t / 2). A seed whose weights are all zero
// stays where it is.
//
// Each step is one launch over (seed tile) x (vector chunk) items that fill a
// wave of resident blocks; every item writes its partial weighted sums, weight
// sum and nonzero-weight count, and a reduction adds the partials in a fixed
// order (deterministic results) and moves the seeds. Vectors stream through
// shared memory; seeds and their sums stay in registers. FP32 throughout;
// dimensions up to 32 (zero-padded to 16 or 32).
#include <cmath>

#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kKT = 128;        // threads per block
constexpr int kKPixTile = 128;  // vectors per shared-memory stage

template <int Dp>
struct KCfg {
    static constexpr int S = Dp == 16 ? 2 : 1;  // seeds per thread
    static constexpr int Seeds = kKT * S;       // seeds per item
    static constexpr int W = Dp + 2;            // partial words per seed: sums, weight sum, count
};

struct KSplit {
    int tiles, chunks, chunk_len;
};

inline KSplit ksplit(int M, int64_t N, int slots, int seeds) {
    KSplit s;
    s.tiles = (M + seeds - 1) / seeds;
    int ch = slots / s.tiles;
    ch = ch < 1 ? 1 : (int64_t)ch > N ? (int)N : ch;
    s.chunk_len = (int)((N + ch - 1) / ch);
    s.chunks = (int)((N + s.chunk_len - 1) / s.chunk_len);
    return s;
}

template <int Kind>
__device__ __forceinline__ float kprofile(float t) {
    if (Kind == MS_PROFILE_FLAT) return t <= 1.f ? 1.f : 0.f;
    if (Kind == MS_PROFILE_EPANECHNIKOV) return fmaxf(0.f, 1.f - t);
    return exp2f(-0.72134752044448170f * t);  // exp(-t / 2) = 2^(-t log2(e) / 2)
}

// Copy (and for the cosine distance normalise) rows of `dim` floats into
// zero-padded rows of Dp floats. A zero or non-finite norm raises *status.
__global__ void k_kprep(const float* __restrict__ src, int64_t rows, int dim, int Dp, int cosine,
                        float* __restrict__ dst, int* status) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* s = src + r * dim;
    float* o = dst + r * Dp;
    float scale = 1.f;
    if (cosine) {
        float ss = 0.f;
        for (int k = 0; k < dim; ++k) ss = fmaf(s[k], s[k], ss);
        const float nrm = sqrtf(ss);
        if (!(nrm > 0.f) || !isfinite(nrm)) {
            atomicOr(status, 1);
        } else {
            scale = 1.f / nrm;
        }
    }
    for (int k = 0; k < dim; ++k) {
        const float v = s[k];
        if (!isfinite(v)) atomicOr(status, 1);
        o[k] = cosine ? v * scale : v;
    }
    for (int k = dim; k < Dp; ++k) o[k] = 0.f;
}

// Partial sums of item (seed tile, vector chunk): partial[item][w][r] for
// seed r of the tile, w < Dp the weighted sums, Dp the weight sum, Dp+1 the
// count of nonzero weights.
template <int Dp, int Kind, bool Cosine>
__global__ void __launch_bounds__(kKT)
k_kshift_partial(const float* __restrict__ P, int64_t N, const float* __restrict__ X, int M, float inv_h,
                 KSplit sp, float* __restrict__ partial) {
    using C = KCfg<Dp>;
    __shared__ __align__(16) float tile[kKPixTile * Dp];
    const int item = blockIdx.x;
    const int t = item / sp.chunks, ch = item - t * sp.chunks;
    float x[C::S][Dp], y[C::S][Dp], ws[C::S], wc[C::S];
#pragma unroll
    for (int q = 0; q < C::S; ++q) {
        const int m = t * C::Seeds + q * kKT + threadIdx.x;
#pragma unroll
        for (int k = 0; k < Dp; ++k) {
            x[q][k] = m < M ? X[(int64_t)m * Dp + k] : 0.f;
            y[q][k] = 0.f;
        }
        ws[q] = wc[q] = 0.f;
    }
    const int64_t p_begin = (int64_t)ch * sp.chunk_len;
    const int64_t p_end = min(N, p_begin + sp.chunk_len);
    for (int64_t pb = p_begin; pb < p_end; pb += kKPixTile) {
        const int cnt = (int)min((int64_t)kKPixTile, p_end - pb);
        __syncthreads();
        for (int v = threadIdx.x; v < cnt * (Dp / 4); v += kKT)
            reinterpret_cast<float4*>(tile)[v] = reinterpret_cast<const float4*>(P + pb * Dp)[v];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            float p[Dp];
#pragma unroll
            for (int k = 0; k < Dp; k += 4) {
                const float4 a = *reinterpret_cast<const float4*>(tile + j * Dp + k);
                p[k] = a.x; p[k + 1] = a.y; p[k + 2] = a.z; p[k + 3] = a.w;
            }
            float w[C::S];
            bool any = false;
#pragma unroll
            for (int q = 0; q < C::S; ++q) {
                float u;
                if (Cosine) {
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < Dp; ++k) s = fmaf(x[q][k], p[k], s);
                    u = (1.f - s) * inv_h;
                    u = u * u;
                } else {
                    float d2 = 0.f;
#pragma unroll
                    for (int k = 0; k < Dp; ++k) {
                        const float e = x[q][k] - p[k];
                        d2 = fmaf(e, e, d2);
                    }
                    u = d2 * inv_h * inv_h;
                }
                w[q] = kprofile<Kind>(u);
                any |= w[q] > 0.f;
            }
            if (Kind == MS_PROFILE_GAUSSIAN || __any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int q = 0; q < C::S; ++q) {
#pragma unroll
                    for (int k = 0; k < Dp; ++k) y[q][k] = fmaf(w[q], p[k], y[q][k]);
                    ws[q] += w[q];
                    wc[q] += w[q] > 0.f ? 1.f : 0.f;
                }
            }
        }
    }
    float* out = partial + (size_t)item * C::W * C::Seeds;
#pragma unroll
    for (int q = 0; q < C::S; ++q) {
        const int r = q * kKT + threadIdx.x;
#pragma unroll
        for (int k = 0; k < Dp; ++k) out[k * C::Seeds + r] = y[q][k];
        out[Dp * C::Seeds + r] = ws[q];
        out[(Dp + 1) * C::Seeds + r] = wc[q];
    }
}

// One warp per seed: add its chunk partials in a fixed order, then move it.
template <int Dp>
__global__ void k_kshift_reduce(const float* __restrict__ partial, KSplit sp, int M, int cosine,
                                float* __restrict__ X, int32_t* __restrict__ counts) {
    using C = KCfg<Dp>;
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (m >= M) return;
    const int lane = threadIdx.x & 31;
    const int t = m / C::Seeds, r = m - t * C::Seeds;
    float s[Dp + 2];
#pragma unroll
    for (int k = 0; k < Dp + 2; ++k) s[k] = 0.f;
    for (int ch = lane; ch < sp.chunks; ch += 32) {
        const float* in = partial + (size_t)(t * sp.chunks + ch) * C::W * C::Seeds + r;
#pragma unroll
        for (int k = 0; k < Dp + 2; ++k) s[k] += in[k * C::Seeds];
    }
#pragma unroll
    for (int k = 0; k < Dp + 2; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (lane != 0) return;
    if (counts) counts[m] = (int32_t)s[Dp + 1];
    if (!(s[Dp] > 0.f)) return;  // no weight: the seed stays
    double scale;
    if (cosine) {
        double nn = 0.0;
#pragma unroll
        for (int k = 0; k < Dp; ++k) nn += (double)s[k] * (double)s[k];
        scale = 1.0 / sqrt(nn);
    } else {
        scale = 1.0 / (double)s[Dp];
    }
#pragma unroll
    for (int k = 0; k < Dp; ++k) X[(int64_t)m * Dp + k] = (float)((double)s[k] * scale);
}

__global__ void k_kunpad(const float* __restrict__ X, int M, int Dp, int dim, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * dim) return;
    out[i] = X[(i / dim) * Dp + (i % dim)];
}

template <class K>
int kslots(K kernel) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kKT, 0) != cudaSuccess || per < 1) per = 1;
    return per * sms;
}

template <int Dp, int Kind, bool Cosine>
ms_status kshift_steps(const float* Pw, int64_t N, float* X, int M, float inv_h, int T, int32_t* counts,
                       float* partial, KSplit sp, cudaStream_t st) {
    const unsigned items = (unsigned)(sp.tiles * sp.chunks);
    for (int t = 0; t < T; ++t) {
        k_kshift_partial<Dp, Kind, Cosine><<<items, kKT, 0, st>>>(Pw, N, X, M, inv_h, sp, partial);
        MS_LAUNCH("k_kshift_partial");
        k_kshift_reduce<Dp><<<(unsigned)((M + 7) / 8), 256, 0, st>>>(partial, sp, M, Cosine ? 1 : 0, X,
                                                                     t == T - 1 ? counts : nullptr);
        MS_LAUNCH("k_kshift_reduce");
    }
    return MS_OK;
}

template <int Dp>
ms_status kshift_dispatch(int distance, int profile, const float* Pw, int64_t N, float* X, int M, float inv_h, int T,
                          int32_t* counts, float* partial, KSplit sp, cudaStream_t st) {
#define MS_KS(KIND, COS) return kshift_steps<Dp, KIND, COS>(Pw, N, X, M, inv_h, T, counts, partial, sp, st)
    if (distance == MS_DIST_COSINE) {
        if (profile == MS_PROFILE_FLAT) MS_KS(MS_PROFILE_FLAT, true);
        if (profile == MS_PROFILE_EPANECHNIKOV) MS_KS(MS_PROFILE_EPANECHNIKOV, true);
        MS_KS(MS_PROFILE_GAUSSIAN, true);
    }
    if (profile == MS_PROFILE_FLAT) MS_KS(MS_PROFILE_FLAT, false);
    if (profile == MS_PROFILE_EPANECHNIKOV) MS_KS(MS_PROFILE_EPANECHNIKOV, false);
    MS_KS(MS_PROFILE_GAUSSIAN, false);
#undef MS_KS
}

template <int Dp>
int kshift_slots() {
    // the slowest instantiation bounds the occupancy of all of them
    return kslots(k_kshift_partial<Dp, MS_PROFILE_GAUSSIAN, false>);
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_kernel_shift(const float* d_P, int64_t N, const float* d_X0, int32_t M, int32_t dim,
                                     int32_t distance, int32_t profile, double h, int32_t T, float* d_XT,
                                     int32_t* d_counts, void* stream) {
    if (!d_P || !d_X0 || !d_XT) return set_error(MS_ERR_INVALID_ARG, "NULL buffer");
    if (N < 1 || N >= (1LL << 31) || M < 1 || T < 0) return set_error(MS_ERR_INVALID_ARG, "bad sizes");
    if (dim < 1 || dim > 32) return set_error(MS_ERR_INVALID_ARG, "dim must be in 1..32");
    if (distance != MS_DIST_COSINE && distance != MS_DIST_EUCLID)
        return set_error(MS_ERR_INVALID_ARG, "unknown distance");
    if (profile != MS_PROFILE_FLAT && profile != MS_PROFILE_EPANECHNIKOV && profile != MS_PROFILE_GAUSSIAN)
        return set_error(MS_ERR_INVALID_ARG, "unknown profile");
    if (!(h > 0.0) || !std::isfinite(h)) return set_error(MS_ERR_INVALID_ARG, "h must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int Dp = dim <= 16 ? 16 : 32;
    const int seeds = Dp == 16 ? KCfg<16>::Seeds : KCfg<32>::Seeds;
    const KSplit sp = ksplit(M, N, Dp == 16 ? kshift_slots<16>() : kshift_slots<32>(), seeds);
    const size_t pw_b = (size_t)N * Dp * sizeof(float), x_b = (size_t)M * Dp * sizeof(float);
    const size_t part_b = (size_t)sp.tiles * sp.chunks * (Dp + 2) * seeds * sizeof(float);
    char* b = nullptr;
    MS_CUDA(scratch_malloc_async((void**)&b, pw_b + x_b + part_b + 1024, st));
    float* Pw = (float*)b;
    float* X = (float*)(b + (pw_b + 255) / 256 * 256);
    float* partial = (float*)((char*)X + (x_b + 255) / 256 * 256);
    int* status = (int*)((char*)partial + (part_b + 255) / 256 * 256);
    const int cosine = distance == MS_DIST_COSINE;
    ms_status s = cuda_check(cudaMemsetAsync(status, 0, sizeof(int), st), "memset");
    if (s == MS_OK) {
        k_kprep<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(d_P, N, dim, Dp, cosine, Pw, status);
        s = cuda_check(cudaGetLastError(), "k_kprep");
    }
    if (s == MS_OK) {
        k_kprep<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(d_X0, M, dim, Dp, cosine, X, status);
        s = cuda_check(cudaGetLastError(), "k_kprep");
    }
    int h_status = 0;
    if (s == MS_OK) s = cuda_check(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    if (s == MS_OK) s = cuda_check(cudaStreamSynchronize(st), "sync");
    if (s == MS_OK && h_status) s = set_error(MS_ERR_INVALID_ARG, "a vector is non-finite or (cosine) of zero norm");
    if (s == MS_OK && d_counts && T == 0) s = cuda_check(cudaMemsetAsync(d_counts, 0, sizeof(int32_t) * M, st), "memset");
    const float inv_h = (float)(1.0 / h);
    if (s == MS_OK)
        s = Dp == 16 ? kshift_dispatch<16>(distance, profile, Pw, N, X, M, inv_h, T, d_counts, partial, sp, st)
                     : kshift_dispatch<32>(distance, profile, Pw, N, X, M, inv_h, T, d_counts, partial, sp, st);
    if (s == MS_OK) {
        k_kunpad<<<(unsigned)(((int64_t)M * dim + 255) / 256), 256, 0, st>>>(X, M, Dp, dim, d_XT);
        s = cuda_check(cudaGetLastError(), "k_kunpad");
    }
    cudaFreeAsync(b, st);
    return s;
}
