// Prune/merge of converged modes (the prune/merge step of Algorithm 2) and OSOP coverage.
//
// Merge rule: candidates (the round's converged seeds) are visited in order of
// support descending, then seed order ascending; a candidate is kept when its
// cosine to every mode kept so far is < merge_cos. Each decision is the FP64
// one: FP32 dot products decide pairs that clear the threshold by more than
// kEpsF32 and the rest are recomputed in FP64.
//
// The sequential greedy is evaluated in parallel as the lexicographically
// first independent set of the conflict graph: candidates that conflict with a
// previously kept mode are removed up front; then, sweep by sweep, a candidate
// is removed as soon as a higher-ranked conflicting candidate is kept, and kept
// as soon as every higher-ranked conflicting candidate is removed. This fixed
// point equals the sequential greedy result; a single-warp sequential pass
// finishes any candidates still undecided after a bounded number of sweeps.
#include "ms_batch.cuh"
#include "ms_device.cuh"

namespace ms {
namespace {

constexpr int kMT = 128;  // threads per merge block
constexpr int kVT = 64;   // vectors per shared-memory tile

__global__ void k_collect(const uint8_t* __restrict__ sstate, int m, int32_t* __restrict__ cand,
                          DevCounters* dc) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool c = s < m && sstate[s] == kConverged;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned b = __ballot_sync(0xffffffffu, c);
    int base = 0;
    if (lane == 0 && b) base = atomicAdd(&dc->n_cand, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (c) cand[base + __popc(b & ((1u << lane) - 1u))] = s;
}

// Rank of every candidate in (support desc, seed order asc): the count of
// candidates ahead of it. Block (x, y) counts candidate block x against slice y
// of all candidates and adds its partial count (ranks start at 0). A candidate
// is ahead of another exactly when its key support * 2^32 + (2^32 - 1 - order)
// is larger (seed orders are distinct within a frame).
__device__ __forceinline__ unsigned long long rank_key(int32_t support, int32_t order) {
    return ((unsigned long long)(uint32_t)support << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)order);
}

__global__ void k_rank(const int32_t* __restrict__ cand, int k, const int32_t* __restrict__ support,
                       const int32_t* __restrict__ order, int32_t* __restrict__ cand_rank) {
    __shared__ unsigned long long s_key[256];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long ka = a < k ? rank_key(support[cand[a]], order[cand[a]]) : 0ull;
    const int lo = (int)((int64_t)blockIdx.y * k / gridDim.y), hi = (int)((int64_t)(blockIdx.y + 1) * k / gridDim.y);
    int r = 0;
    for (int base = lo; base < hi; base += 256) {
        const int b = base + threadIdx.x;
        if (b < hi) s_key[threadIdx.x] = rank_key(support[cand[b]], order[cand[b]]);
        __syncthreads();
        const int lim = min(256, hi - base);
        for (int j = 0; j < lim; ++j) r += s_key[j] > ka;
        __syncthreads();
    }
    if (a < k && r) atomicAdd(&cand_rank[a], r);
}

__global__ void k_rank_invert(const int32_t* __restrict__ cand_rank, int k, int32_t* __restrict__ rank_cand) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < k) rank_cand[cand_rank[a]] = a;
}

// k_rank_invert that also copies each candidate's position to its rank's row
// of Xr (the BF16 form's tensor-core merge reads the candidates in rank order).
template <int Dp>
__global__ void k_rank_invert_xr(const int32_t* __restrict__ cand_rank, int k, const int32_t* __restrict__ cand,
                                 const float* __restrict__ X, int32_t* __restrict__ rank_cand, float* __restrict__ Xr) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= k) return;
    const int r = cand_rank[a];
    rank_cand[r] = a;
    const float4* src = reinterpret_cast<const float4*>(X + (int64_t)cand[a] * Dp);
    float4* dst = reinterpret_cast<float4*>(Xr + (int64_t)r * Dp);
#pragma unroll
    for (int q = 0; q < Dp / 4; ++q) dst[q] = src[q];
}

template <int Dp>
__device__ __forceinline__ void load_vec(float* dst, const float* src) {
#pragma unroll
    for (int k = 0; k < Dp; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(src + k);
        dst[k] = v.x; dst[k + 1] = v.y; dst[k + 2] = v.z; dst[k + 3] = v.w;
    }
}

// Candidates within merge_cos of a mode kept in an earlier round are removed
// (cand_state starts at kUndecided). Block (x, y): candidate block x against
// slice y of the old modes.
template <int Dp>
__global__ void __launch_bounds__(kMT)
k_merge_old(const float* __restrict__ X, const int32_t* __restrict__ cand, int k,
            const float* __restrict__ modes, int K_old, float thr_f, double thr,
            uint8_t* __restrict__ cand_state) {
    __shared__ __align__(16) float tile[kVT * Dp];
    const int a = blockIdx.x * kMT + threadIdx.x;
    float x[Dp];
    if (a < k) load_vec<Dp>(x, X + (int64_t)cand[a] * Dp);
    bool removed = false;
    const int lo = (int)((int64_t)blockIdx.y * K_old / gridDim.y);
    const int hi = (int)((int64_t)(blockIdx.y + 1) * K_old / gridDim.y);
    for (int base = lo; base < hi; base += kVT) {
        const int cnt = min(kVT, hi - base);
        for (int q = threadIdx.x; q < cnt * Dp; q += kMT) tile[q] = modes[(int64_t)base * Dp + q];
        __syncthreads();
        if (a < k && !removed) {
            for (int j = 0; j < cnt; ++j)
                if (cos_at_least<Dp>(x, tile + j * Dp, thr_f, thr)) {
                    removed = true;
                    break;
                }
        }
        __syncthreads();
    }
    if (a < k && removed) cand_state[a] = kRemoved;
}

// Higher-ranked conflicting candidates of each undecided candidate: the first
// kMergeCap found are stored (in no particular order; the resolve step treats
// them as a set), conf_deg (starting at 0) counts all of them. Block (x, y):
// candidate block x against slice y of all candidates.
template <int Dp>
__global__ void __launch_bounds__(kMT)
k_merge_pairs(const float* __restrict__ X, const int32_t* __restrict__ cand, int k,
              const int32_t* __restrict__ rank_cand, const uint8_t* __restrict__ cand_state,
              float thr_f, double thr, int32_t* __restrict__ conf_deg, int32_t* __restrict__ conf) {
    // Candidates in rank order: thread t of block x takes rank x*kMT + t and
    // compares it with the higher-priority candidates (lower ranks) of the
    // block's slice, so neighbouring lanes stop at neighbouring ranks and only
    // the k(k-1)/2 ordered pairs are tested.
    __shared__ __align__(16) float tile[kVT * Dp];
    __shared__ int32_t s_idx[kVT];
    __shared__ uint8_t s_state[kVT];
    const int r0 = blockIdx.x * kMT;
    const int r = r0 + threadIdx.x;
    const int a = r < k ? rank_cand[r] : -1;
    const bool act = a >= 0 && cand_state[a] == kUndecided;
    float x[Dp];
    if (act) load_vec<Dp>(x, X + (int64_t)cand[a] * Dp);
    const int lo = (int)((int64_t)blockIdx.y * k / gridDim.y);
    const int hi = min((int)((int64_t)(blockIdx.y + 1) * k / gridDim.y), r0 + kMT - 1);
    for (int base = lo; base < hi; base += kVT) {
        const int cnt = min(kVT, hi - base);
        for (int q = threadIdx.x; q < cnt * Dp; q += kMT) {
            const int j = q / Dp, kk = q - j * Dp;
            tile[q] = X[(int64_t)cand[rank_cand[base + j]] * Dp + kk];
        }
        for (int j = threadIdx.x; j < cnt; j += kMT) {
            const int cj = rank_cand[base + j];
            s_idx[j] = cj;
            s_state[j] = cand_state[cj];
        }
        __syncthreads();
        if (act) {
            const int jend = min(cnt, r - base);
            for (int j = 0; j < jend; ++j) {
                if (s_state[j] == kRemoved) continue;
                if (cos_at_least<Dp>(x, tile + j * Dp, thr_f, thr)) {
                    const int slot = atomicAdd(&conf_deg[a], 1);
                    if (slot < kMergeCap) conf[(int64_t)a * kMergeCap + slot] = s_idx[j];
                }
            }
        }
        __syncthreads();
    }
}

template <int Dp>
__global__ void __launch_bounds__(kMT)
k_merge_resolve(const float* __restrict__ X, const int32_t* __restrict__ cand, int k,
                const int32_t* __restrict__ cand_rank, const int32_t* __restrict__ rank_cand, uint8_t* cand_state,
                const int32_t* __restrict__ conf_deg, const int32_t* __restrict__ conf,
                float thr_f, double thr, DevCounters* dc) {
    const int a = blockIdx.x * kMT + threadIdx.x;
    if (a >= k) return;
    volatile uint8_t* st = cand_state;
    if (st[a] != kUndecided) return;
    const int deg = conf_deg[a];
    bool any_kept = false, all_removed = true;
    if (deg <= kMergeCap) {
        for (int j = 0; j < deg; ++j) {
            const uint8_t s = st[conf[(int64_t)a * kMergeCap + j]];
            if (s == kKept) {
                any_kept = true;
                break;
            }
            if (s == kUndecided) all_removed = false;
        }
    } else {
        // more conflicts than were stored: test the candidates ranked above
        // this one again, in rank order
        float x[Dp];
        load_vec<Dp>(x, X + (int64_t)cand[a] * Dp);
        const int ra = cand_rank[a];
        for (int rb = 0; rb < ra; ++rb) {
            const int b = rank_cand[rb];
            const uint8_t s = st[b];
            if (s == kRemoved) continue;
            if (!cos_at_least<Dp>(x, X + (int64_t)cand[b] * Dp, thr_f, thr)) continue;
            if (s == kKept) {
                any_kept = true;
                break;
            }
            all_removed = false;
        }
    }
    if (any_kept)
        st[a] = kRemoved;
    else if (all_removed)
        st[a] = kKept;
    else
        atomicAdd(&dc->undecided, 1);
}

// Exact sequential greedy for whatever is still undecided (one warp).
template <int Dp>
__global__ void k_merge_sequential(const float* __restrict__ X, const int32_t* __restrict__ cand,
                                   int k, const int32_t* __restrict__ rank_cand, uint8_t* cand_state,
                                   float thr_f, double thr) {
    volatile uint8_t* st = cand_state;
    const int lane = threadIdx.x;
    for (int r = 0; r < k; ++r) {
        const int a = rank_cand[r];
        if (st[a] != kUndecided) continue;
        const float* xa = X + (int64_t)cand[a] * Dp;
        bool hit = false;
        for (int rb = lane; rb < r && !hit; rb += 32) {
            const int b = rank_cand[rb];
            if (st[b] == kKept && cos_at_least<Dp>(xa, X + (int64_t)cand[b] * Dp, thr_f, thr)) hit = true;
        }
        const bool any = __any_sync(0xffffffffu, hit);
        if (lane == 0) st[a] = any ? kRemoved : kKept;
        __syncwarp();
    }
}

// Kept candidates are appended to the mode list in rank order.
template <int Dp>
__global__ void __launch_bounds__(1024)
k_merge_append(const float* __restrict__ X, const int32_t* __restrict__ cand,
               const int32_t* __restrict__ rank_cand, int k, const uint8_t* __restrict__ cand_state,
               const int32_t* __restrict__ support, float* __restrict__ modes,
               int32_t* __restrict__ mode_support, DevCounters* dc) {
    __shared__ int32_t warp_excl[32];
    __shared__ int32_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int base = dc->n_kept;
    int carry = 0;
    for (int r0 = 0; r0 < k; r0 += 1024) {
        const int r = r0 + tid;
        const int a = r < k ? rank_cand[r] : -1;
        const bool flag = a >= 0 && cand_state[a] == kKept;
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_excl[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            const int w = warp_excl[lane];
            int incl = w;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            warp_excl[lane] = incl - w;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (flag) {
            const int dst = base + carry + warp_excl[wid] + __popc(bal & ((1u << lane) - 1u));
            const int slot = cand[a];
            const float4* src = reinterpret_cast<const float4*>(X + (int64_t)slot * Dp);
            float4* out = reinterpret_cast<float4*>(modes + (int64_t)dst * Dp);
            for (int q = 0; q < Dp / 4; ++q) out[q] = src[q];
            mode_support[dst] = support[slot];
        }
        carry += s_total;
        __syncthreads();
    }
    if (tid == 0) dc->n_kept = base + carry;
}

// Coverage (OSOP stop rule): an uncovered pixel is covered once some new mode
// has cos >= c. FP32 decides pairs outside the band; inside it the cosine is
// recomputed in FP64 from the raw embedding.
// A block takes 256 * cover_per(Dp) consecutive pixels (1024 for d <= 16),
// compacts the uncovered ones into a shared list (warp ballots and a prefix
// over the block's warp-passes) and gives each thread up to cover_per of
// them, so every tile of new modes is read once for all of them.
__host__ __device__ constexpr int cover_per(int Dp) { return Dp <= 16 ? 4 : 2; }

template <int Dp>
__global__ void __launch_bounds__(256)
k_cover(const float* __restrict__ P32, const float* __restrict__ emb, int d,
        const int32_t* __restrict__ pix, int n, uint8_t* __restrict__ covered,
        const float* __restrict__ modes, int k0, int k1, float c_f, double c, DevCounters* dc) {
    constexpr int kPer = cover_per(Dp);
    constexpr int kNW = 256 / 32 * kPer;  // warp-passes of the block
    static_assert(kNW <= 32, "one warp scans the warp-pass counts");
    __shared__ __align__(16) float tile[kVT * Dp];
    __shared__ int32_t s_list[256 * kPer];
    __shared__ int32_t s_pos[kNW];
    __shared__ int s_nact;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * 256 * kPer;
    unsigned bal[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = i0 + u * 256 + threadIdx.x;
        bal[u] = __ballot_sync(0xffffffffu, i < n && covered[i] == 0);
        if (lane == 0) s_pos[u * 8 + warp] = __popc(bal[u]);
    }
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kNW ? s_pos[lane] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < kNW) s_pos[lane] = incl - v;
        if (lane == 31) s_nact = incl;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPer; ++u)
        if ((bal[u] >> lane) & 1u)
            s_list[s_pos[u * 8 + warp] + __popc(bal[u] & ((1u << lane) - 1u))] = i0 + u * 256 + threadIdx.x;
    __syncthreads();
    const int nact = s_nact;
    if (nact == 0) return;
    int idx[kPer];
    float p[kPer][Dp];
    bool cov[kPer], band[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * 256;
        idx[u] = e < nact ? s_list[e] : -1;
        if (idx[u] >= 0) load_vec<Dp>(p[u], P32 + (int64_t)idx[u] * Dp);
        cov[u] = band[u] = false;
    }
    for (int base = k0; base < k1; base += kVT) {
        const int cnt = min(kVT, k1 - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * Dp; q += 256) tile[q] = modes[(int64_t)base * Dp + q];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (idx[u] >= 0 && !cov[u])
                for (int j = 0; j < cnt; ++j) {
                    const float sc = dot_seq<Dp>(p[u], tile + j * Dp);
                    if (sc >= c_f + kEpsF32) {
                        cov[u] = true;
                        break;
                    }
                    if (sc >= c_f - kEpsF32) band[u] = true;
                }
    }
    int newly = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        if (idx[u] >= 0 && !cov[u] && band[u]) {
            const float* e = emb + (int64_t)pix[idx[u]] * d;
            for (int j = k0; j < k1 && !cov[u]; ++j) {
                const float* m = modes + (int64_t)j * Dp;
                if (dot_seq<Dp>(p[u], m) >= c_f - kEpsF32 && cos64(e, m, d) >= c) cov[u] = true;
            }
        }
        if (idx[u] >= 0 && cov[u]) {
            covered[idx[u]] = 1;
            ++newly;
        }
    }
    for (int o = 16; o > 0; o >>= 1) newly += __shfl_xor_sync(0xffffffffu, newly, o);
    if (lane == 0 && newly) atomicSub(&dc->n_uncovered, newly);
}

// Slices of an O(outer x inner) loop so that the grid fills about four waves
// of the GPU: the candidate blocks alone are often fewer than the SMs.
unsigned inner_slices(int outer_blocks, int inner, int num_sms) {
    int sl = (4 * num_sms + outer_blocks - 1) / outer_blocks;
    const int max_sl = (inner + kVT - 1) / kVT;
    sl = sl > max_sl ? max_sl : sl;
    sl = sl > 64 ? 64 : sl;
    return (unsigned)(sl < 1 ? 1 : sl);
}

template <int Dp>
ms_status merge_prepare_t(ms_ctx* ctx, int32_t k) {
    const float thr_f = (float)ctx->cfg.merge_cos;
    const double thr = ctx->cfg.merge_cos;
    const unsigned g256 = (unsigned)((k + 255) / 256), gm = (unsigned)((k + kMT - 1) / kMT);
    MS_CUDA(cudaMemsetAsync(ctx->cand_rank, 0, sizeof(int32_t) * (size_t)k, ctx->stream));
    MS_CUDA(cudaMemsetAsync(ctx->cand_state, kUndecided, (size_t)k, ctx->stream));
    MS_CUDA(cudaMemsetAsync(ctx->conf_deg, 0, sizeof(int32_t) * (size_t)k, ctx->stream));
    k_rank<<<dim3(g256, inner_slices((int)g256, k, ctx->num_sms)), 256, 0, ctx->stream>>>(
        ctx->cand, k, ctx->support, ctx->seed_order, ctx->cand_rank);
    MS_LAUNCH("k_rank");
    if (ctx->Ck) {  // BF16 form: both contractions of the merge on the tensor cores
        MS_CUDA(cudaMemsetAsync(ctx->removed_r, 0, (size_t)k, ctx->stream));
        k_rank_invert_xr<Dp><<<g256, 256, 0, ctx->stream>>>(ctx->cand_rank, k, ctx->cand, ctx->X, ctx->rank_cand,
                                                             ctx->Xr);
        MS_LAUNCH("k_rank_invert_xr");
        LabelTcScratch sc{ctx->label_fix, (int*)(ctx->label_fix + ctx->n), nullptr};
        const ms_status s = launch_merge_tc_single(ctx->Ck, ctx->Mk, ctx->n_pad, Dp, k, ctx->n_kept, ctx->Xr,
                                                   ctx->modes, ctx->rank_cand, ctx->cand_state, ctx->removed_r,
                                                   ctx->conf_deg, ctx->conf, thr_f, thr, sc, ctx->num_sms,
                                                   &ctx->dc->status, ctx->stream);
        ctx->launches += 4 + (ctx->n_kept > 0 ? 2 : 0);
        return s;
    }
    k_rank_invert<<<g256, 256, 0, ctx->stream>>>(ctx->cand_rank, k, ctx->rank_cand);
    MS_LAUNCH("k_rank_invert");
    if (ctx->n_kept > 0) {
        k_merge_old<Dp><<<dim3(gm, inner_slices((int)gm, ctx->n_kept, ctx->num_sms)), kMT, 0, ctx->stream>>>(
            ctx->X, ctx->cand, k, ctx->modes, ctx->n_kept, thr_f, thr, ctx->cand_state);
        MS_LAUNCH("k_merge_old");
    }
    k_merge_pairs<Dp><<<dim3(gm, inner_slices((int)gm, k, ctx->num_sms)), kMT, 0, ctx->stream>>>(
        ctx->X, ctx->cand, k, ctx->rank_cand, ctx->cand_state, thr_f, thr, ctx->conf_deg, ctx->conf);
    MS_LAUNCH("k_merge_pairs");
    ctx->launches += 4;
    return MS_OK;
}

}  // namespace

ms_status launch_collect(ms_ctx* ctx) {
    MS_CUDA(cudaMemsetAsync(&ctx->dc->n_cand, 0, sizeof(int32_t), ctx->stream));
    if (ctx->m_round <= 0) return MS_OK;
    k_collect<<<(unsigned)((ctx->m_round + 255) / 256), 256, 0, ctx->stream>>>(ctx->sstate, ctx->m_round,
                                                                             ctx->cand, ctx->dc);
    MS_LAUNCH("k_collect");
    ctx->launches += 1;
    return MS_OK;
}

ms_status launch_merge_prepare(ms_ctx* ctx, int32_t k) {
    if (k <= 0) return MS_OK;
    return ctx->Dp == 16 ? merge_prepare_t<16>(ctx, k) : merge_prepare_t<32>(ctx, k);
}

ms_status launch_merge_resolve(ms_ctx* ctx, int32_t k, int sweeps) {
    if (k <= 0) return MS_OK;
    const float thr_f = (float)ctx->cfg.merge_cos;
    const double thr = ctx->cfg.merge_cos;
    const unsigned gm = (unsigned)((k + kMT - 1) / kMT);
    for (int s = 0; s < sweeps; ++s) {
        MS_CUDA(cudaMemsetAsync(&ctx->dc->undecided, 0, sizeof(int32_t), ctx->stream));
        if (ctx->Dp == 16)
            k_merge_resolve<16><<<gm, kMT, 0, ctx->stream>>>(ctx->X, ctx->cand, k, ctx->cand_rank,
                                                             ctx->rank_cand, ctx->cand_state, ctx->conf_deg, ctx->conf,
                                                             thr_f, thr, ctx->dc);
        else
            k_merge_resolve<32><<<gm, kMT, 0, ctx->stream>>>(ctx->X, ctx->cand, k, ctx->cand_rank,
                                                             ctx->rank_cand, ctx->cand_state, ctx->conf_deg, ctx->conf,
                                                             thr_f, thr, ctx->dc);
        MS_LAUNCH("k_merge_resolve");
        ctx->launches += 1;
    }
    return MS_OK;
}

ms_status launch_merge_sequential(ms_ctx* ctx, int32_t k) {
    if (k <= 0) return MS_OK;
    const float thr_f = (float)ctx->cfg.merge_cos;
    const double thr = ctx->cfg.merge_cos;
    if (ctx->Dp == 16)
        k_merge_sequential<16><<<1, 32, 0, ctx->stream>>>(ctx->X, ctx->cand, k, ctx->rank_cand,
                                                          ctx->cand_state, thr_f, thr);
    else
        k_merge_sequential<32><<<1, 32, 0, ctx->stream>>>(ctx->X, ctx->cand, k, ctx->rank_cand,
                                                          ctx->cand_state, thr_f, thr);
    MS_LAUNCH("k_merge_sequential");
    ctx->launches += 1;
    return MS_OK;
}

ms_status launch_merge_append(ms_ctx* ctx, int32_t k) {
    if (k <= 0) return MS_OK;
    if (ctx->Dp == 16)
        k_merge_append<16><<<1, 1024, 0, ctx->stream>>>(ctx->X, ctx->cand, ctx->rank_cand, k,
                                                        ctx->cand_state, ctx->support, ctx->modes,
                                                        ctx->mode_support, ctx->dc);
    else
        k_merge_append<32><<<1, 1024, 0, ctx->stream>>>(ctx->X, ctx->cand, ctx->rank_cand, k,
                                                        ctx->cand_state, ctx->support, ctx->modes,
                                                        ctx->mode_support, ctx->dc);
    MS_LAUNCH("k_merge_append");
    ctx->launches += 1;
    return MS_OK;
}

ms_status launch_cover(ms_ctx* ctx, int32_t k0, int32_t k1) {
    if (k1 <= k0 || ctx->n == 0) return MS_OK;
    if (ctx->Mk) {  // BF16 form: the tensor cores score the pixels against the new modes
        LabelTcScratch sc{ctx->label_fix, (int*)(ctx->label_fix + ctx->n), nullptr};
        const ms_status s = launch_cover_tc_single(ctx->pmap, ctx->pmap1, ctx->Mk, ctx->n_pad, ctx->Dp, ctx->modes,
                                                   k0, k1, (int)ctx->n,
                                                   ctx->P32, ctx->pix, ctx->emb, ctx->d, ctx->cfg.bandwidth_cos,
                                                   ctx->covered, &ctx->dc->n_uncovered, sc, ctx->num_sms,
                                                   &ctx->dc->status, ctx->stream);
        ctx->launches += 3;
        return s;
    }
    const float c_f = (float)ctx->cfg.bandwidth_cos;
    const unsigned g = (unsigned)((ctx->n + 256 * cover_per(ctx->Dp) - 1) / (256 * cover_per(ctx->Dp)));
    if (ctx->Dp == 16)
        k_cover<16><<<g, 256, 0, ctx->stream>>>(ctx->P32, ctx->emb, ctx->d, ctx->pix, (int)ctx->n,
                                                ctx->covered, ctx->modes, k0, k1, c_f,
                                                ctx->cfg.bandwidth_cos, ctx->dc);
    else
        k_cover<32><<<g, 256, 0, ctx->stream>>>(ctx->P32, ctx->emb, ctx->d, ctx->pix, (int)ctx->n,
                                                ctx->covered, ctx->modes, k0, k1, c_f,
                                                ctx->cfg.bandwidth_cos, ctx->dc);
    MS_LAUNCH("k_cover");
    ctx->launches += 1;
    return MS_OK;
}

}  // namespace ms
