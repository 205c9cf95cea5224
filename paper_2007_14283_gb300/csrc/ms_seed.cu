// OSOP seed selection (the seed-selection step of Algorithm 2): the next `want` uncovered
// positions of the frame's fixed seed order pi(j) = (b + a j) mod n.
//
// One CTA walks the order 1024 positions at a time. Each thread tests one
// position; warp ballots and a block prefix count give every uncovered
// position its slot, so the batch is the first `want` uncovered positions in
// order, exactly as a sequential scan would take them.
#include "ms_internal.cuh"

namespace ms {
namespace {

constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads)
k_seed_select(int32_t n, uint64_t a, uint64_t b, int32_t want, int Dp,
              const float* __restrict__ P32, uint8_t* __restrict__ covered,
              float* __restrict__ X, int32_t* __restrict__ seed_pix,
              int32_t* __restrict__ seed_order, int32_t* __restrict__ active0,
              uint8_t* __restrict__ sstate, int32_t* __restrict__ seed_log,
              DevCounters* dc) {
    __shared__ int32_t warp_excl[32];
    __shared__ int32_t s_total;
    __shared__ int32_t s_cut;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int32_t cursor = dc->cursor;
    const int32_t drawn = dc->drawn;
    int32_t taken = 0;
    while (taken < want && cursor < n) {
        const int32_t pos = cursor + tid;
        int32_t p = -1;
        bool flag = false;
        if (pos < n) {
            p = (int32_t)((b + a * (uint64_t)pos) % (uint64_t)n);
            flag = covered[p] == 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_excl[wid] = __popc(bal);
        if (tid == 0) s_cut = n;
        __syncthreads();
        if (wid == 0) {
            int w = warp_excl[lane];
            int incl = w;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            warp_excl[lane] = incl - w;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        const int32_t r = warp_excl[wid] + __popc(bal & ((1u << lane) - 1u));
        if (flag && taken + r < want) {
            const int32_t slot = taken + r;
            covered[p] = 1;
            seed_pix[slot] = p;
            seed_order[slot] = drawn + slot;
            seed_log[drawn + slot] = p;
            active0[slot] = slot;
            sstate[slot] = kMoving;
            const float4* src = reinterpret_cast<const float4*>(P32 + (int64_t)p * Dp);
            float4* dst = reinterpret_cast<float4*>(X + (int64_t)slot * Dp);
            for (int k = 0; k < Dp / 4; ++k) dst[k] = src[k];
            if (taken + r == want - 1) s_cut = pos + 1;
        }
        __syncthreads();
        if (taken + s_total >= want) {
            cursor = s_cut;
            taken = want;
        } else {
            taken += s_total;
            cursor = min(n, cursor + kSelThreads);
        }
        __syncthreads();
    }
    if (tid == 0) {
        dc->cursor = cursor;
        dc->drawn = drawn + taken;
        dc->n_seeded = taken;
        dc->m_round = taken;
        dc->n_active = taken;
        dc->n_next = 0;
        dc->conv_new = 0;
        dc->conv_total = 0;
        dc->fail_total = 0;
        dc->iters = 0;
        dc->done = taken == 0;
        dc->n_uncovered -= taken;
    }
}

}  // namespace

ms_status launch_seed_select(ms_ctx* ctx, int32_t want) {
    k_seed_select<<<1, kSelThreads, 0, ctx->stream>>>(
        (int32_t)ctx->n, (uint64_t)ctx->perm_a, (uint64_t)ctx->perm_b, want, ctx->Dp, ctx->P32,
        ctx->covered, ctx->X, ctx->seed_pix, ctx->seed_order, ctx->active[0], ctx->sstate,
        ctx->seed_log, ctx->dc);
    MS_LAUNCH("k_seed_select");
    ctx->launches += 1;
    return MS_OK;
}

}  // namespace ms
