// Shift iteration, plain FP32 form (the shift loop of Algorithm 2; Eq. 6-8, 11).
//
// For every active seed x: y = sum of p_i over the window {i : x.p_i >= c},
// cnt = |window|; then x' = y / ||y|| and the FP64 norm ||x' - x|| decides
// convergence. Sec. 3.2.1's dense form is used (every pixel is tested against
// the kernel, no neighbour search), but the seed-by-pixel matrix is never
// materialised: pixels stream through shared memory and each thread keeps its
// seeds' sums in registers.
//
// Launch shape: a persistent grid. Each launch reads the active-seed count on
// the device and splits the work into (seed tile of 256) x (pixel chunk)
// items, so successive iterations can be queued without reading counts back.
// Each item adds its FP32 window sums into per-seed 64-bit fixed-point
// accumulators (units of 2^-36). Integer addition is associative, so the
// totals do not depend on the order in which items finish: runs are
// deterministic, and the finalize step reads one word per component.
#include "ms_batch.cuh"

namespace ms {
namespace {

constexpr float kFixScale = 68719476736.0f;      // 2^36
constexpr double kFixInv = 1.0 / 68719476736.0;  // 2^-36

// What a work item covers: a tile of the frame's active seeds and the pixel
// rows [p_begin, p_end) of P32.
struct F32Item {
    const int32_t* active;
    int n_active;
    int seed0;
    int64_t p_begin, p_end;
};

// Work items of one frame: seed tiles of 256 x pixel chunks.
struct F32SingleMap {
    const int32_t* active;
    const DevCounters* dc;
    int n, target;
    int n_active;
    ShiftSplit sp;
    __device__ __forceinline__ bool init() {
        if (dc->done) return false;
        n_active = dc->n_active;
        sp = shift_split(n_active, n, target);
        return true;
    }
    __device__ __forceinline__ int total() const { return sp.tiles * sp.chunks; }
    __device__ __forceinline__ F32Item item(int i) const {
        const int t = i / sp.chunks, ch = i - t * sp.chunks;
        F32Item it;
        it.active = active;
        it.n_active = n_active;
        it.seed0 = t * kSeedsPerTile;
        it.p_begin = (int64_t)ch * sp.chunk_len;
        it.p_end = min((int64_t)n, it.p_begin + sp.chunk_len);
        return it;
    }
};

template <int Dp, class Map>
__global__ void __launch_bounds__(kShiftThreads)
k_shift_fp32(const float* __restrict__ P32, const float* __restrict__ X, unsigned long long* __restrict__ acc,
             float c, Map map) {
    if (!map.init()) return;
    const int items = map.total();
    __shared__ __align__(16) float tile[kPixTile * Dp];
    const int tid = threadIdx.x;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const F32Item ii = map.item(item);
        const int pos0 = ii.seed0 + tid;
        const int pos1 = pos0 + kShiftThreads;
        const int s0 = pos0 < ii.n_active ? ii.active[pos0] : -1;
        const int s1 = pos1 < ii.n_active ? ii.active[pos1] : -1;
        float x0[Dp], x1[Dp], y0[Dp], y1[Dp];
        float c0 = 0.f, c1 = 0.f;
#pragma unroll
        for (int k = 0; k < Dp; k += 4) {
            float4 a = s0 >= 0 ? *reinterpret_cast<const float4*>(X + (int64_t)s0 * Dp + k)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 b = s1 >= 0 ? *reinterpret_cast<const float4*>(X + (int64_t)s1 * Dp + k)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
            x0[k] = a.x; x0[k + 1] = a.y; x0[k + 2] = a.z; x0[k + 3] = a.w;
            x1[k] = b.x; x1[k + 1] = b.y; x1[k + 2] = b.z; x1[k + 3] = b.w;
        }
#pragma unroll
        for (int k = 0; k < Dp; ++k) y0[k] = y1[k] = 0.f;
        const int64_t p_begin = ii.p_begin, p_end = ii.p_end;
        for (int64_t pb = p_begin; pb < p_end; pb += kPixTile) {
            const int cnt = (int)min((int64_t)kPixTile, p_end - pb);
            __syncthreads();
            const float4* src = reinterpret_cast<const float4*>(P32 + (int64_t)pb * Dp);
            float4* dst = reinterpret_cast<float4*>(tile);
            for (int q = tid; q < cnt * (Dp / 4); q += kShiftThreads) dst[q] = src[q];
            __syncthreads();
            for (int j = 0; j < cnt; ++j) {
                float p[Dp];
#pragma unroll
                for (int k = 0; k < Dp; k += 4) {
                    float4 v = *reinterpret_cast<const float4*>(tile + j * Dp + k);
                    p[k] = v.x; p[k + 1] = v.y; p[k + 2] = v.z; p[k + 3] = v.w;
                }
                float d0 = 0.f, d1 = 0.f;
#pragma unroll
                for (int k = 0; k < Dp; ++k) {
                    d0 = fmaf(x0[k], p[k], d0);
                    d1 = fmaf(x1[k], p[k], d1);
                }
                const bool in0 = d0 >= c, in1 = d1 >= c;
                if (__any_sync(0xffffffffu, in0 || in1)) {
                    if (in0) {
#pragma unroll
                        for (int k = 0; k < Dp; ++k) y0[k] += p[k];
                        c0 += 1.f;
                    }
                    if (in1) {
#pragma unroll
                        for (int k = 0; k < Dp; ++k) y1[k] += p[k];
                        c1 += 1.f;
                    }
                }
            }
        }
        if (s0 >= 0 && c0 > 0.f) {
            unsigned long long* a = acc + (int64_t)s0 * (Dp + 1);
#pragma unroll
            for (int k = 0; k < Dp; ++k) atomicAdd(a + k, (unsigned long long)__float2ll_rn(y0[k] * kFixScale));
            atomicAdd(a + Dp, (unsigned long long)c0);
        }
        if (s1 >= 0 && c1 > 0.f) {
            unsigned long long* a = acc + (int64_t)s1 * (Dp + 1);
#pragma unroll
            for (int k = 0; k < Dp; ++k) atomicAdd(a + k, (unsigned long long)__float2ll_rn(y1[k] * kFixScale));
            atomicAdd(a + Dp, (unsigned long long)c1);
        }
    }
}

// Reads and clears each active seed's accumulators, moves the seed to
// normalise(y) (FP32 state, computed from the exact sums in FP64) and tests
// ||x' - x|| < tol in FP64.
template <int Dp>
__global__ void __launch_bounds__(256)
k_finalize(unsigned long long* __restrict__ acc, const int32_t* __restrict__ active_in,
           int32_t* __restrict__ active_out, float* __restrict__ X, uint8_t* __restrict__ sstate,
           int32_t* __restrict__ support, double tol, DevCounters* dc) {
    if (dc->done) return;
    const int n_active = dc->n_active;
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    bool conv = false, fail = false, moving = false;
    int slot = -1;
    if (pos < n_active) {
        slot = active_in[pos];
        unsigned long long* a = acc + (int64_t)slot * (Dp + 1);
        const long long cnt = (long long)a[Dp];
        a[Dp] = 0ull;
        double y[Dp];
        double ss = 0.0;
#pragma unroll
        for (int k = 0; k < Dp; ++k) {
            y[k] = (double)(long long)a[k] * kFixInv;
            a[k] = 0ull;
            ss += y[k] * y[k];
        }
        if (cnt == 0) {
            fail = true;
            sstate[slot] = kFailed;
        } else {
            const double inv = 1.0 / sqrt(ss);
            float* x = X + (int64_t)slot * Dp;
            double dd = 0.0;
#pragma unroll
            for (int k = 0; k < Dp; ++k) {
                const float xn = (float)(y[k] * inv);
                const double diff = (double)xn - (double)x[k];
                dd += diff * diff;
                x[k] = xn;
            }
            support[slot] = (int32_t)cnt;
            if (sqrt(dd) < tol) {
                conv = true;
                sstate[slot] = kConverged;
            } else {
                moving = true;
            }
        }
    }
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mc = __ballot_sync(0xffffffffu, conv);
    const unsigned mf = __ballot_sync(0xffffffffu, fail);
    const unsigned mm = __ballot_sync(0xffffffffu, moving);
    int base = 0;
    if (lane == 0) {
        if (mc) atomicAdd(&dc->conv_new, __popc(mc));
        if (mf) atomicAdd(&dc->fail_total, __popc(mf));
        if (mm) base = atomicAdd(&dc->n_next, __popc(mm));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (moving) active_out[base + __popc(mm & ((1u << lane) - 1u))] = slot;
}

// Early stopping (Sec. 3.2.3): the round ends once more than gamma of its
// seeds have converged, when none is still moving, or at max_iter.
__global__ void k_round_check(DevCounters* dc, double gamma, int max_iter) {
    if (dc->done) return;
    dc->seed_iters += dc->n_active;
    dc->conv_total += dc->conv_new;
    dc->conv_new = 0;
    dc->n_active = dc->n_next;
    dc->n_next = 0;
    dc->iters += 1;
    if ((double)dc->conv_total > gamma * (double)dc->m_round || dc->n_active == 0 ||
        dc->iters >= max_iter)
        dc->done = 1;
}

template <int Dp>
ms_status shift_iteration_t(ms_ctx* ctx, int t, int max_iter, cudaEvent_t e0, cudaEvent_t e1) {
    const int32_t* a_in = ctx->active[t & 1];
    int32_t* a_out = ctx->active[(t + 1) & 1];
    const float c = ceil_to_float(ctx->cfg.bandwidth_cos);
    const double gamma = ctx->cfg.all_seeds ? 1.0 : ctx->cfg.gamma;
    const unsigned fin_blocks = (unsigned)((ctx->m_round + 255) / 256);
    if (e0) MS_CUDA(cudaEventRecord(e0, ctx->stream));
    if (ctx->cfg.precision == MS_BF16) {
        ms_status s = launch_shift_tc(ctx, a_in, ctx->tc_grid, 2 * ctx->tc_grid, nullptr);
        if (s != MS_OK) return s;
    } else {
        F32SingleMap map;
        map.active = a_in;
        map.dc = ctx->dc;
        map.n = (int)ctx->n;
        map.target = ctx->target_items;
        k_shift_fp32<Dp, F32SingleMap><<<ctx->shift_grid, kShiftThreads, 0, ctx->stream>>>(ctx->P32, ctx->X,
                                                                                         ctx->acc, c, map);
        MS_LAUNCH("k_shift_fp32");
    }
    if (e1) MS_CUDA(cudaEventRecord(e1, ctx->stream));
    k_finalize<Dp><<<fin_blocks, 256, 0, ctx->stream>>>(ctx->acc, a_in, a_out, ctx->X, ctx->sstate,
                                                        ctx->support, ctx->cfg.tol, ctx->dc);
    MS_LAUNCH("k_finalize");
    k_round_check<<<1, 1, 0, ctx->stream>>>(ctx->dc, gamma, max_iter);
    MS_LAUNCH("k_round_check");
    ctx->launches += 3;
    return MS_OK;
}

}  // namespace

float ceil_to_float(double c) {
    float f = (float)c;
    if ((double)f < c) f = nextafterf(f, 2.0f);
    return f;
}

int shift_blocks_per_sm() {
    int b16 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b16, k_shift_fp32<16, F32SingleMap>, kShiftThreads, 0);
    return b16 > 0 ? b16 : 1;
}

ms_status launch_window_sums_fp32(const float* P32, int32_t n, const int32_t* active, const float* X,
                                  unsigned long long* acc, float c, const DevCounters* dc,
                                  cudaStream_t stream) {
    int per_sm = shift_blocks_per_sm();
    int dev = 0, sms = 1;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * per_sm;
    F32SingleMap map;
    map.active = active;
    map.dc = dc;
    map.n = n;
    map.target = 2 * grid;
    k_shift_fp32<16, F32SingleMap><<<grid, kShiftThreads, 0, stream>>>(P32, X, acc, c, map);
    MS_LAUNCH("k_shift_fp32");
    return MS_OK;
}

// Work items of every iterating frame (batched form): frame f contributes
// item_off[f+1] - item_off[f] items, seed tiles of 256 x chunks of tpc[f] pixels.
struct F32BatchMap {
    const BFrame* frames;
    const BState* states;
    BPlan plan;
    const int32_t* act0;
    const int32_t* act1;
    int nf;
    int total_;
    __device__ __forceinline__ bool init() {
        total_ = plan.item_off[nf];
        return total_ > 0;
    }
    __device__ __forceinline__ int total() const { return total_; }
    __device__ __forceinline__ F32Item item(int i) const {
        const int f = locate(plan.item_off, nf, i);
        const int local = i - plan.item_off[f];
        const int chunks = plan.chunks[f];
        const int t = local / chunks, ch = local - t * chunks;
        const BFrame& fr = frames[f];
        F32Item it;
        it.active = ((states[f].dc.iters & 1) ? act1 : act0) + fr.pix0;
        it.n_active = states[f].dc.n_active;
        it.seed0 = t * kSeedsPerTile;
        const int64_t b = (int64_t)ch * plan.tpc[f];
        it.p_begin = fr.pix0 + b;
        it.p_end = fr.pix0 + min((int64_t)fr.n, b + plan.tpc[f]);
        return it;
    }
};

ms_status launch_shift_fp32_batch(const float* P32, const float* X, unsigned long long* acc, float c_f, int Dp,
                                  const BFrame* frames, const BState* states, BPlan plan, const int32_t* act0,
                                  const int32_t* act1, int nf, int grid, cudaStream_t st) {
    F32BatchMap map;
    map.frames = frames;
    map.states = states;
    map.plan = plan;
    map.act0 = act0;
    map.act1 = act1;
    map.nf = nf;
    map.total_ = 0;
    if (Dp == 16)
        k_shift_fp32<16, F32BatchMap><<<grid, kShiftThreads, 0, st>>>(P32, X, acc, c_f, map);
    else
        k_shift_fp32<32, F32BatchMap><<<grid, kShiftThreads, 0, st>>>(P32, X, acc, c_f, map);
    MS_LAUNCH("k_shift_fp32(batch)");
    return MS_OK;
}

ms_status launch_shift_iteration(ms_ctx* ctx, int t, int max_iter, cudaEvent_t e0, cudaEvent_t e1) {
    if (ctx->m_round <= 0) return MS_OK;
    return ctx->Dp == 16 ? shift_iteration_t<16>(ctx, t, max_iter, e0, e1)
                         : shift_iteration_t<32>(ctx, t, max_iter, e0, e1);
}

}  // namespace ms
