// Device helpers: FP32 dot products and thresholded cosine decisions whose
// outcome is exact in FP64.
#pragma once

#include "ms_internal.cuh"

namespace ms {

// Sequential FP32 dot product, k = 0..Dp-1, one fused multiply-add per term.
template <int Dp>
__device__ __forceinline__ float dot_seq(const float* a, const float* b) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < Dp; ++k) s = fmaf(a[k], b[k], s);
    return s;
}

// Cosine (Eq. 1) in FP64 of two FP32 vectors of length n.
__device__ __forceinline__ double cos64(const float* a, const float* b, int n) {
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int k = 0; k < n; ++k) {
        const double x = a[k], y = b[k];
        ab += x * y;
        aa += x * x;
        bb += y * y;
    }
    return ab / (sqrt(aa) * sqrt(bb));
}

// cos(a, b) >= thr for unit-length FP32 vectors: decided from the FP32 dot
// product when it clears thr by more than kEpsF32, else recomputed in FP64.
template <int Dp>
__device__ __forceinline__ bool cos_at_least(const float* a, const float* b, float thr_f, double thr) {
    const float s = dot_seq<Dp>(a, b);
    if (s >= thr_f + kEpsF32) return true;
    if (s < thr_f - kEpsF32) return false;
    return cos64(a, b, Dp) >= thr;
}

}  // namespace ms
