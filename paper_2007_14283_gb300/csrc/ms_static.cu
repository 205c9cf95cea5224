// Window sums with no device allocation: ms_window_sums_static.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena that owns the whole device, allocators that forbid
// cudaMalloc/cudaFree while a stream is being captured, or plugins whose host
// application hands them only the input and output buffers. For them this
// entry point runs the FP32 window-sum kernel with its scratch (normalised
// pixels, fixed-point accumulators, active list, counters) in one file-scope
// device array of fixed size. Every GPU that loads the library holds that
// array until the process exits; all calls on a device share it.
#include <cstddef>
#include <mutex>

#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kStaticMaxSeeds = 1024;
constexpr int kStaticMaxPixels = 16384;
constexpr int kStaticDim = 16;

constexpr size_t kOffPix = 0;
constexpr size_t kOffAcc = kOffPix + sizeof(float) * kStaticMaxPixels * kStaticDim;
constexpr size_t kOffActive = kOffAcc + sizeof(unsigned long long) * kStaticMaxSeeds * (kStaticDim + 1);
constexpr size_t kOffCounters = kOffActive + sizeof(int32_t) * kStaticMaxSeeds;
constexpr size_t kStaticBytes = kOffCounters + sizeof(DevCounters);

// The scratch. In host code its name is only a host-side stand-in, never a
// device address: host code takes the device address with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
ms_status scratch_address(void** out) {
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(MS_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        MS_CUDA(cudaGetSymbolAddress(&p, g_scratch));
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return MS_OK;
}

// Normalise the pixels into the scratch (same arithmetic as ingest), clear the
// accumulators of the m seeds, list seeds 0..m-1 as active, reset counters.
__global__ void k_static_prepare(const float* __restrict__ P, int n, int m, unsigned char* scratch) {
    float* P32 = reinterpret_cast<float*>(scratch + kOffPix);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(scratch + kOffAcc);
    int32_t* active = reinterpret_cast<int32_t*>(scratch + kOffActive);
    DevCounters* dc = reinterpret_cast<DevCounters*>(scratch + kOffCounters);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float* e = P + (int64_t)i * kStaticDim;
        float s = 0.f;
        for (int k = 0; k < kStaticDim; ++k) s = fmaf(e[k], e[k], s);
        const float nrm = sqrtf(s);
        float* p = P32 + (int64_t)i * kStaticDim;
        for (int k = 0; k < kStaticDim; ++k) p[k] = flush_tiny(e[k] / nrm);
        if (!(nrm > 0.f) || !isfinite(nrm)) atomicOr(&dc->status, 1);
    }
    if (i < m) {
        for (int k = 0; k <= kStaticDim; ++k) acc[(int64_t)i * (kStaticDim + 1) + k] = 0ull;
        active[i] = i;
    }
    if (i == 0) {
        dc->n_active = m;
        dc->done = 0;
    }
}

// Copy the accumulators out. When the prepare step met a pixel of zero or
// non-finite norm, every row instead reads sums 0 and count -1, so a caller
// that cannot synchronise inside the call still sees the error in its output.
__global__ void k_static_copy_out(int m, const unsigned char* scratch, int64_t* __restrict__ out) {
    const unsigned long long* acc = reinterpret_cast<const unsigned long long*>(scratch + kOffAcc);
    const DevCounters* dc = reinterpret_cast<const DevCounters*>(scratch + kOffCounters);
    const bool bad = dc->status != 0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m * (kStaticDim + 1))
        out[i] = bad ? ((i % (kStaticDim + 1)) == kStaticDim ? -1 : 0) : (int64_t)acc[i];
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_window_sums_static(const float* d_X, int32_t m, const float* d_P, int32_t n, double c,
                                           int64_t* d_acc_out, void* stream) {
    if (!d_X || !d_P || !d_acc_out) return set_error(MS_ERR_INVALID_ARG, "NULL buffer");
    if (m < 1 || m > kStaticMaxSeeds)
        return set_error(MS_ERR_INVALID_ARG, "m = %d seeds is outside 1..%d (the static scratch limit)", m,
                         kStaticMaxSeeds);
    if (n < 1 || n > kStaticMaxPixels)
        return set_error(MS_ERR_INVALID_ARG, "n = %d pixels is outside 1..%d (the static scratch limit)", n,
                         kStaticMaxPixels);
    if (!(c > -1.0 && c <= 1.0)) return set_error(MS_ERR_INVALID_ARG, "c must be in (-1, 1]");
    void* base = nullptr;
    ms_status s = scratch_address(&base);
    if (s != MS_OK) return s;
    unsigned char* scratch = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream;
    // the error flag starts clear on every call (the array keeps the last call's contents)
    MS_CUDA(cudaMemsetAsync(scratch + kOffCounters + offsetof(DevCounters, status), 0, sizeof(int32_t), st));
    const int threads = 256;
    const int items = n > m ? n : m;
    k_static_prepare<<<(items + threads - 1) / threads, threads, 0, st>>>(d_P, n, m, scratch);
    MS_LAUNCH("k_static_prepare");
    s = launch_window_sums_fp32(reinterpret_cast<const float*>(scratch + kOffPix), n,
                                reinterpret_cast<const int32_t*>(scratch + kOffActive), d_X,
                                reinterpret_cast<unsigned long long*>(scratch + kOffAcc), ceil_to_float(c),
                                reinterpret_cast<const DevCounters*>(scratch + kOffCounters), st);
    if (s != MS_OK) return s;
    const int total = m * (kStaticDim + 1);
    k_static_copy_out<<<(total + threads - 1) / threads, threads, 0, st>>>(m, scratch, d_acc_out);
    MS_LAUNCH("k_static_copy_out");
    return MS_OK;
}
