// Batched form: many frames of uneven size in one CUDA graph, with the whole
// OSOP control of every frame on the device.
//
// Each frame runs the same method as the single-frame path (Algorithm 2 with
// OSOP, Sec. 3.2): seed selection, lockstep shift iterations with early stop,
// merge, coverage, N schedule, labels. Here a per-frame state machine
// (need-seed -> iterating -> round-done -> need-seed ... -> finished) replaces
// the host loop. One graph holds: set-up (compaction, normalisation, BF16
// splits, state reset), a conditional WHILE node whose body advances every
// frame by one iteration (and runs seed selection and the merge chain only
// for frames in those phases), and labelling. The body's last kernel keeps
// the loop going while any frame is unfinished. The shift kernel of each
// iteration is one persistent launch over the work items of all iterating
// frames. Frames may be in different rounds at the same time. The host only
// launches the graph and synchronises once.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ms_batch.cuh"
#include "ms_device.cuh"
#include "ms_tc.cuh"

struct ms_batch {
    ms_config cfg;
    int B, d, Dp;
    bool tc;
    cudaStream_t stream;      // caller's stream (graph launches)
    cudaStream_t cap;         // private stream used only for capture
    int num_sms, grid, tc_grid, f32_grid;
    int64_t total_px, total_pk_rows, max_np, max_pk_rows, nblk_max;
    void* ws;
    size_t ws_bytes;
    ms::BFrame* frames;
    ms::BState* states;
    ms::BState* h_states;     // pinned copy for statistics
    ms::BPlan plan;
    int32_t* blk_off;         // [B + 2] block work list of the current merge/cover/label kernel
    int32_t* blk_split;       // [B + 2] block work list with the inner loop split (slices at [B + 1])
    int32_t* misc;            // [0] passes, [1] status, u64 at [2] band pairs, [4] tick, [6] shift ns, [8] shift
                              // launches, [14] last phase tick, [16..31] eight phase sums (ns)
    float* P32;
    int32_t* pix;
    uint8_t* covered;
    float* X;
    int32_t* seed_pix;
    int32_t* seed_order;
    uint8_t* sstate;
    int32_t* support;
    int32_t* act[2];
    unsigned long long* acc;
    float* modes;
    int32_t* cand;
    int32_t* cand_rank;
    int32_t* rank_cand;
    float* Xr;                // candidates' seed positions in rank order (merge)
    uint8_t* removed_r;       // candidates removed by a mode of an earlier round, in rank order
    uint8_t* cand_state;
    int32_t* conf_deg;
    int32_t* conf;
    int32_t* block_tmp;       // [B, nblk_max]
    void* Pk;
    void* Mk;                 // kept modes as BF16 split rows at the frames' Pk offsets (labelling)
    void* Ck;                 // merge candidates (rank order) as BF16 split rows at the frames' Pk offsets
    int32_t** label_ptrs;     // device array of B label buffers
    CUtensorMap pmap;
    CUtensorMap pmap1;        // d = 32: dimensions 16..31 (the second Pk array)
    CUtensorMap mmap;
    CUtensorMap mmap1;        // d = 32: the modes' dimensions 16..31 (the second Mk array)
    CUtensorMap cmap, cmap1;  // Ck, and its second array (d = 32)
    ms::LabelTcScratch lsc;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int64_t body_launches;    // kernels per pass of the loop body
    int split;                // 0: each frame split as on its own; 1: work items shared by load
    int target_mult;          // shift work items per launch = target_mult x shift grid
    int tc_shape;             // warp arrangement of the tensor-core shift kernel (ms_config.tc_shape)
    int64_t fixed_launches;   // set-up and labelling kernels
    bool prof;                // body brackets the shift launch with timer ticks
    bool prof_phases;         // ... and every phase of the graph with phase ticks (k_b_phase)
    int32_t h_misc[32];       // host copy of misc after the last synchronised run
    std::vector<ms::BFrame> hf;   // host copy of the frame table (device pointers of every frame)
    std::vector<int32_t*> h_labels;  // device label buffers
};

namespace ms {
namespace {

using tc::bf16_round;
using tc::pack_bf16;

constexpr int kIT = 1024;   // ingest / selection threads
constexpr int kMT = 128;    // merge threads
constexpr int kVT = 64;     // vectors per shared tile
constexpr int kPT = 256;    // pixel threads (cover, label)
constexpr int kDefaultMaxPasses = 200000;  // loop guard: far above any real run (rounds x iterations)

enum BlockSel { kSelDoneSeeds = 0, kSelDoneCands = 1, kSelDonePixels = 2, kSelAllPixels = 3 };
// Phase sums of profiling level 2 (ms_batch_phase_ms): set-up; per pass the
// loop's relaunch gap with seed selection and the work plan, the shift, its
// finalisation and early-stop check, the merge chain, coverage, the schedule
// with the loop condition; then labelling.
enum Phase { kPhSetup = 0, kPhSeed, kPhShift, kPhFinalize, kPhMerge, kPhCover, kPhSchedule, kPhLabel, kPhases };

// ------------------------------------------------------------ device math
__device__ uint64_t d_splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

__device__ int64_t d_gcd(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// The frame's fixed seed order pi(j) = (b + a j) mod n (see ms_api.cu).
__device__ void d_perm(int64_t n, uint64_t key, uint64_t* a, uint64_t* b) {
    if (n <= 1) {
        *a = 1;
        *b = 0;
        return;
    }
    const int64_t centre = (int64_t)floor(0.6180339887 * (double)n + 0.5);
    int64_t pick = 1;
    for (int64_t off = 0; off <= n; ++off) {
        const int64_t lo = centre - off;
        if (lo >= 1 && lo < n && d_gcd(lo, n) == 1) { pick = lo; break; }
        const int64_t hi = centre + off;
        if (hi >= 1 && hi < n && d_gcd(hi, n) == 1) { pick = hi; break; }
    }
    *a = (uint64_t)pick;
    *b = d_splitmix64(key) % (uint64_t)n;
}

// N schedule, Sec. 3.2.4 with Eq. 19 (r = 1).
__device__ int64_t d_schedule(int64_t N, int64_t I, double P, double L, double H, int64_t uncovered) {
    int64_t next = N;
    if (I > 0) {
        const double nmin = log(1.0 - exp(log(P) / (double)I)) / log(1.0 - 1.0 / (double)I);
        if ((double)N < L * nmin)
            next = 2 * N;
        else if ((double)N > H * nmin)
            next = N - (int64_t)ceil(nmin);
    }
    const int64_t cap = uncovered > 1 ? uncovered : 1;
    if (next > cap) next = cap;
    if (next < 1) next = 1;
    return next;
}

template <int Dp>
__device__ __forceinline__ void ldv(float* dst, const float* src) {
#pragma unroll
    for (int k = 0; k < Dp; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(src + k);
        dst[k] = v.x; dst[k + 1] = v.y; dst[k + 2] = v.z; dst[k + 3] = v.w;
    }
}

// Block-wide exclusive scan (blockDim.x a multiple of 32, at most 1024):
// returns the exclusive prefix of v and writes the block total to *total.
// Every thread of the block must call it; it may be called repeatedly.
__device__ int block_scan(int v, int* total) {
    __shared__ int ws[32];
    __shared__ int s_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? ws[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        ws[lane] = wi - w;
        if (lane == 31) s_tot = wi;
    }
    __syncthreads();
    const int excl = ws[wid] + incl - v;
    *total = s_tot;
    __syncthreads();
    return excl;
}

// ------------------------------------------------------------ set-up
__global__ void k_b_count(const BFrame* __restrict__ frames, int nblk_max, int32_t* __restrict__ bt) {
    const BFrame& fr = frames[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x;
    const bool fg = i < fr.n_pixels && (fr.mask == nullptr || fr.mask[i] != 0);
    const int c = __syncthreads_count(fg);
    if (threadIdx.x == 0) bt[(int64_t)blockIdx.y * nblk_max + blockIdx.x] = c;
}

__global__ void k_b_scan(BFrame* frames, BState* states, int nblk_max, int32_t* bt, uint64_t seed,
                         uint64_t frame_id0, int64_t n_initial) {
    const int f = blockIdx.x;
    BFrame& fr = frames[f];
    const int nb = (int)((fr.n_pixels + kIT - 1) / kIT);
    int32_t* c = bt + (int64_t)f * nblk_max;
    int carry = 0;
    for (int base = 0; base < nb; base += kIT) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? c[i] : 0;
        int tot;
        const int ex = block_scan(v, &tot);
        if (i < nb) c[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        fr.n = carry;
        fr.n_ptiles = (carry + 127) / 128;
        uint64_t a, b;
        d_perm(carry, seed ^ (frame_id0 + (uint64_t)f), &a, &b);
        fr.perm_a = a;
        fr.perm_b = b;
        BState& st = states[f];
        memset(&st, 0, sizeof(BState));
        st.dc.n_fg = carry;
        st.dc.n_uncovered = carry;
        st.N = n_initial;
        st.phase = carry > 0 ? kNeedSeed : kFinished;
    }
}

__global__ void k_b_compact(const BFrame* __restrict__ frames, int nblk_max, const int32_t* __restrict__ bt, int d,
                            int Dp, float* __restrict__ P32, int32_t* __restrict__ pix, int* status) {
    __shared__ int32_t ws[32];
    const int f = blockIdx.y;
    const BFrame& fr = frames[f];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x;
    const bool fg = i < fr.n_pixels && (fr.mask == nullptr || fr.mask[i] != 0);
    const unsigned bal = __ballot_sync(0xffffffffu, fg);
    if (lane == 0) ws[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        const int w = ws[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        ws[lane] = wi - w;
    }
    __syncthreads();
    if (!fg) return;
    const int64_t pos = fr.pix0 + bt[(int64_t)f * nblk_max + blockIdx.x] + ws[wid] + __popc(bal & ((1u << lane) - 1u));
    const float* e = fr.emb + i * d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(e[k], e[k], s);
    float nrm = sqrtf(s);
    if (!(nrm > 0.f) || !isfinite(nrm)) {
        atomicOr(status, 1);
        nrm = 1.f;
    }
    float* p = P32 + pos * Dp;
    for (int k = 0; k < d; ++k) p[k] = flush_tiny(e[k] / nrm);
    for (int k = d; k < Dp; ++k) p[k] = 0.f;
    pix[pos] = (int32_t)i;
}

// BF16 split rows of every frame's pixels at the frame's Pk rows; for d = 32
// a second array (after total_rows rows) holds dimensions 16..31.
__global__ void k_b_pack(const BFrame* __restrict__ frames, const float* __restrict__ P32, int Dp, int64_t total_rows,
                         uint4* __restrict__ Pk) {
    const BFrame& fr = frames[blockIdx.y];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= fr.n_ptiles * 128) return;
    const float* p = r < fr.n ? P32 + (fr.pix0 + r) * Dp : nullptr;
    tc::pack_split_row(p, Pk + (int64_t)(fr.pk_row0 + r) * 8);
    if (Dp == 32) tc::pack_split_row(p ? p + 16 : nullptr, Pk + (total_rows + fr.pk_row0 + r) * 8, false);
}

__global__ void k_b_labels_clear(const BFrame* __restrict__ frames, int32_t* const* __restrict__ labels) {
    const BFrame& fr = frames[blockIdx.y];
    int32_t* l = labels[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fr.n_pixels;
         i += (int64_t)gridDim.x * blockDim.x)
        l[i] = -1;
}

// ------------------------------------------------------------ seeds
__global__ void __launch_bounds__(kIT)
k_b_seed(const BFrame* __restrict__ frames, BState* states, const float* __restrict__ P32, int Dp,
         uint8_t* __restrict__ covered, float* __restrict__ X, int32_t* __restrict__ seed_pix,
         int32_t* __restrict__ seed_order, int32_t* __restrict__ act0, uint8_t* __restrict__ sstate, int max_rounds,
         int all_seeds) {
    __shared__ int32_t warp_excl[32];
    __shared__ int32_t s_total, s_cut;
    __shared__ int s_go;
    const int f = blockIdx.x;
    const BFrame& fr = frames[f];
    BState& st = states[f];
    if (threadIdx.x == 0) {
        s_go = 0;
        if (st.phase == kNeedSeed) {
            if (st.dc.n_uncovered <= 0 || st.rounds >= max_rounds)
                st.phase = kFinished;
            else
                s_go = 1;
        }
    }
    __syncthreads();
    if (!s_go) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t n = fr.n;
    int64_t wantl = all_seeds ? (int64_t)n : st.N;
    if (wantl > st.dc.n_uncovered) wantl = st.dc.n_uncovered;
    const int32_t want = (int32_t)wantl;
    const int64_t base = fr.pix0;
    int32_t cursor = st.dc.cursor;
    const int32_t drawn = st.dc.drawn;
    int32_t taken = 0;
    while (taken < want && cursor < n) {
        const int32_t pos = cursor + tid;
        int32_t p = -1;
        bool flag = false;
        if (pos < n) {
            p = (int32_t)((fr.perm_b + fr.perm_a * (uint64_t)pos) % (uint64_t)n);
            flag = covered[base + p] == 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_excl[wid] = __popc(bal);
        if (tid == 0) s_cut = n;
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
        const int32_t r = warp_excl[wid] + __popc(bal & ((1u << lane) - 1u));
        if (flag && taken + r < want) {
            const int64_t slot = base + taken + r;
            covered[base + p] = 1;
            seed_pix[slot] = p;
            seed_order[slot] = drawn + taken + r;
            act0[slot] = (int32_t)slot;
            sstate[slot] = kMoving;
            const float4* src = reinterpret_cast<const float4*>(P32 + (base + p) * Dp);
            float4* dst = reinterpret_cast<float4*>(X + slot * Dp);
            for (int k = 0; k < Dp / 4; ++k) dst[k] = src[k];
            if (taken + r == want - 1) s_cut = pos + 1;
        }
        __syncthreads();
        if (taken + s_total >= want) {
            cursor = s_cut;
            taken = want;
        } else {
            taken += s_total;
            cursor = min(n, cursor + kIT);
        }
        __syncthreads();
    }
    if (tid == 0) {
        DevCounters& dc = st.dc;
        dc.cursor = cursor;
        dc.drawn = drawn + taken;
        dc.n_seeded = taken;
        dc.m_round = taken;
        dc.n_active = taken;
        dc.n_next = 0;
        dc.conv_new = 0;
        dc.conv_total = 0;
        dc.fail_total = 0;
        dc.iters = 0;
        dc.done = 0;
        dc.n_cand = 0;
        dc.undecided = 0;
        dc.n_uncovered -= taken;
        st.seeds_total += taken;
        st.phase = taken > 0 ? kIterating : kFinished;
    }
}

// ------------------------------------------------------------ iteration
// Work split of this iteration over the iterating frames. Each frame is cut
// into seed tiles x pixel chunks by the single-frame rule (a target item count
// spread over the frame's seed tiles, chunks whole pixel tiles). With
// canon_target > 0 every frame gets that target, the one the single-frame path
// uses, so each frame's window sums, and with them all its results, are
// bit-identical to a single-frame run. With canon_target = 0 the batch target
// is shared out in proportion to each frame's seed-by-pixel work (exact
// integer totals, so the split is deterministic).
__global__ void k_b_plan(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B, BPlan plan,
                         int target, int canon_target, int tc, int grid) {
    __shared__ unsigned long long s_work;
    __shared__ int s_carry_items, s_carry_seeds;
    if (threadIdx.x == 0) {
        s_work = 0ull;
        s_carry_items = 0;
        s_carry_seeds = 0;
    }
    __syncthreads();
    if (canon_target <= 0)
        for (int f = threadIdx.x; f < B; f += blockDim.x)
            if (states[f].phase == kIterating)
                atomicAdd(&s_work, (unsigned long long)states[f].dc.n_active * (unsigned long long)frames[f].n);
    __syncthreads();
    const double total = s_work > 0ull ? (double)s_work : 1.0;
    for (int base = 0; base < B; base += kIT) {
        const int f = base + threadIdx.x;
        int items = 0, seeds = 0;
        if (f < B && states[f].phase == kIterating) {
            const BFrame& fr = frames[f];
            const int na = states[f].dc.n_active;
            int tf = canon_target;
            if (tf <= 0) {
                const double w = (double)((unsigned long long)na * (unsigned long long)fr.n);
                tf = (int)ceil((double)target * w / total);
                tf = tf < 1 ? 1 : tf;
            }
            if (tc) {
                // the canonical split fits the items to the grid exactly as a
                // single-frame launch on that grid does
                const int tiles = (na + 127) / 128;
                const int tpc = tc_tiles_per_chunk(tiles, fr.n_ptiles, tf, canon_target > 0 ? grid : 0);
                plan.tpc[f] = tpc;
                plan.chunks[f] = (fr.n_ptiles + tpc - 1) / tpc;
                items = tiles * plan.chunks[f];
            } else {
                const ShiftSplit sp = shift_split(na, fr.n, tf);
                plan.tpc[f] = sp.chunk_len;
                plan.chunks[f] = sp.chunks;
                items = sp.tiles * sp.chunks;
            }
            seeds = na;
        }
        int ti, ts;
        const int ei = block_scan(items, &ti);
        const int es = block_scan(seeds, &ts);
        if (f < B) {
            plan.item_off[f] = s_carry_items + ei;
            plan.seed_off[f] = s_carry_seeds + es;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry_items += ti;
            s_carry_seeds += ts;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        plan.item_off[B] = s_carry_items;
        plan.seed_off[B] = s_carry_seeds;
    }
}

// Warp-aggregated atomicAdd of 1 from every lane with flag set, grouped by
// key (lanes of one warp may belong to different frames). Returns the old
// value plus the lane's rank within its group.
__device__ __forceinline__ int agg_inc(int32_t* ctr, bool flag, int key) {
    const unsigned act = __ballot_sync(0xffffffffu, flag);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned grp = __match_any_sync(0xffffffffu, flag ? key : -1 - (int)lane) & act;
    int old = 0;
    if (flag && lane == (unsigned)(__ffs(grp) - 1)) old = atomicAdd(ctr, __popc(grp));
    old = __shfl_sync(0xffffffffu, old, flag ? __ffs(grp) - 1 : lane);
    return old + __popc(grp & ((1u << lane) - 1u));
}

// Mean-shift update of every active seed of every iterating frame (Eq. 5
// with the flat kernel): x <- normalise(window sum), converged when the FP64
// step norm is below tol; seeds still moving go to the frame's next list.
template <int Dp>
__global__ void __launch_bounds__(256)
k_b_finalize(const BFrame* __restrict__ frames, BState* states, int B, BPlan plan, int32_t* act0, int32_t* act1,
             unsigned long long* __restrict__ acc, float* __restrict__ X, uint8_t* __restrict__ sstate,
             int32_t* __restrict__ support, double tol) {
    const int total = plan.seed_off[B];
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < total; i0 += stride) {
        const int i = i0 + threadIdx.x;
        const bool in = i < total;
        int f = 0, slot = 0;
        bool fail = false, conv = false, moving = false;
        int32_t* a_out = nullptr;
        if (in) {
            f = locate(plan.seed_off, B, i);
            const int pos = i - plan.seed_off[f];
            const int64_t base = frames[f].pix0;
            const bool odd = states[f].dc.iters & 1;
            a_out = (odd ? act0 : act1) + base;
            slot = ((odd ? act1 : act0) + base)[pos];
            unsigned long long* a = acc + (int64_t)slot * (Dp + 1);
            const long long cnt = (long long)a[Dp];
            a[Dp] = 0ull;
            double y[Dp];
            double ss = 0.0;
#pragma unroll
            for (int k = 0; k < Dp; ++k) {
                y[k] = (double)(long long)a[k] * (1.0 / 68719476736.0);  // fixed point, 2^-36 units
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
        agg_inc(&states[f].dc.fail_total, fail, f);
        agg_inc(&states[f].dc.conv_new, conv, f);
        const int at = agg_inc(&states[f].dc.n_next, moving, f);
        if (moving) a_out[at] = slot;
    }
}

// Early stopping per frame (Sec. 3.2.3).
__global__ void k_b_check(BState* states, int B, double gamma, int max_iter) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    BState& st = states[f];
    if (st.phase != kIterating) return;
    DevCounters& dc = st.dc;
    dc.seed_iters += dc.n_active;
    dc.conv_total += dc.conv_new;
    dc.conv_new = 0;
    dc.n_active = dc.n_next;
    dc.n_next = 0;
    dc.iters += 1;
    if ((double)dc.conv_total > gamma * (double)dc.m_round || dc.n_active == 0 || dc.iters >= max_iter) {
        dc.done = 1;
        st.phase = kRoundDone;
        st.iters_total += dc.iters;
        st.cands_total += dc.conv_total;
        st.dropped_total += (int64_t)dc.m_round - dc.conv_total;
    }
}

// ------------------------------------------------------------ merge
// Block work list: frame f contributes ceil(count_f / per_block) blocks, times
// S slices of an inner loop when split_target > 0 (S chosen so the list holds
// about split_target blocks, 1..64; stored at off[B + 1]).
__global__ void k_b_blocks(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B, int sel,
                           int per_block, int split_target, int32_t* __restrict__ off) {
    if (threadIdx.x != 0) return;
    int outer = 0;
    for (int f = 0; f < B; ++f) {
        const BState& st = states[f];
        int cnt = 0;
        if (sel == kSelAllPixels) cnt = frames[f].n;
        else if (st.phase == kRoundDone) cnt = sel == kSelDoneSeeds ? st.dc.m_round
                                             : sel == kSelDoneCands ? st.dc.n_cand : frames[f].n;
        off[f] = outer;
        outer += (cnt + per_block - 1) / per_block;
    }
    int S = 1;
    if (split_target > 0 && outer > 0) {
        S = (split_target + outer - 1) / outer;
        S = S < 1 ? 1 : (S > 64 ? 64 : S);
    }
    for (int f = 0; f < B; ++f) off[f] *= S;
    off[B] = outer * S;
    off[B + 1] = S;
}

// Merge scratch of the frames whose round ended starts from zero ranks,
// undecided candidates and empty conflict lists.
__global__ void k_b_merge_zero(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
                               const int32_t* __restrict__ off, int32_t* __restrict__ cand_rank,
                               uint8_t* __restrict__ cand_state, int32_t* __restrict__ conf_deg,
                               uint8_t* __restrict__ removed_r) {
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int a = (bb - off[f]) * kMT + threadIdx.x;
        if (a < states[f].dc.n_cand) {
            const int64_t i = frames[f].pix0 + a;
            cand_rank[i] = 0;
            cand_state[i] = kUndecided;
            conf_deg[i] = 0;
            removed_r[i] = 0;  // rank a (ranks and candidates span the same range)
        }
    }
}

// rank_cand inverts cand_rank; each candidate's seed position is copied to
// its rank's row of Xr, so the conflict search reads contiguous rows.
template <int Dp>
__global__ void k_b_rank_invert(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
                                const int32_t* __restrict__ off, const int32_t* __restrict__ cand_rank,
                                const int32_t* __restrict__ cand, const float* __restrict__ X,
                                int32_t* __restrict__ rank_cand, float* __restrict__ Xr) {
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int a = (bb - off[f]) * kMT + threadIdx.x;
        if (a < states[f].dc.n_cand) {
            const int64_t base = frames[f].pix0;
            const int r = cand_rank[base + a];
            rank_cand[base + r] = a;
            const float4* src = reinterpret_cast<const float4*>(X + (int64_t)cand[base + a] * Dp);
            float4* dst = reinterpret_cast<float4*>(Xr + (base + r) * Dp);
#pragma unroll
            for (int q = 0; q < Dp / 4; ++q) dst[q] = src[q];
        }
    }
}

__global__ void k_b_collect(const BFrame* __restrict__ frames, BState* states, int B, const int32_t* __restrict__ off,
                            const uint8_t* __restrict__ sstate, int32_t* __restrict__ cand) {
    for (int b = blockIdx.x; b < off[B]; b += gridDim.x) {
        const int f = locate(off, B, b);
        const int lb = b - off[f];
        BState& st = states[f];
        const int64_t base = frames[f].pix0;
        const int s = lb * 256 + threadIdx.x;
        const bool c = s < st.dc.m_round && sstate[base + s] == kConverged;
        const unsigned lane = threadIdx.x & 31u;
        const unsigned bal = __ballot_sync(0xffffffffu, c);
        int w = 0;
        if (lane == 0 && bal) w = atomicAdd(&st.dc.n_cand, __popc(bal));
        w = __shfl_sync(0xffffffffu, w, 0);
        if (c) cand[base + w + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(base + s);
    }
}

// Rank in (support desc, seed order asc): block (candidate block, slice) adds
// its partial count of candidates ahead (ranks start at 0, k_b_merge_zero).
// A candidate is ahead of another exactly when its key support * 2^32 +
// (2^32 - 1 - order) is larger (seed orders are distinct within a frame).
__device__ __forceinline__ unsigned long long rank_key(int32_t support, int32_t order) {
    return ((unsigned long long)(uint32_t)support << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)order);
}

__global__ void k_b_rank(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
                         const int32_t* __restrict__ off, const int32_t* __restrict__ cand,
                         const int32_t* __restrict__ support, const int32_t* __restrict__ order,
                         int32_t* __restrict__ cand_rank) {
    __shared__ unsigned long long s_key[kMT];
    const int S = off[B + 1];
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f], sl = lb % S;
        const int64_t base = frames[f].pix0;
        const int k = states[f].dc.n_cand;
        const int a = (lb / S) * kMT + threadIdx.x;
        const int lo = (int)((int64_t)sl * k / S), hi = (int)((int64_t)(sl + 1) * k / S);
        const unsigned long long ka = a < k ? rank_key(support[cand[base + a]], order[cand[base + a]]) : 0ull;
        int r = 0;
        for (int t0 = lo; t0 < hi; t0 += kMT) {
            const int j = t0 + threadIdx.x;
            __syncthreads();
            if (j < hi) s_key[threadIdx.x] = rank_key(support[cand[base + j]], order[cand[base + j]]);
            __syncthreads();
            const int lim = min(kMT, hi - t0);
            for (int q = 0; q < lim; ++q) r += s_key[q] > ka;
        }
        if (a < k && r) atomicAdd(&cand_rank[base + a], r);
        __syncthreads();
    }
}

template <int Dp>
__global__ void __launch_bounds__(kMT)
k_b_merge_old(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
              const int32_t* __restrict__ off, const float* __restrict__ X, const int32_t* __restrict__ cand,
              const float* __restrict__ modes, float thr_f, double thr, uint8_t* __restrict__ cand_state,
              const int32_t* __restrict__ cand_rank, uint8_t* __restrict__ removed_r) {
    __shared__ __align__(16) float tile[kVT * Dp];
    const int S = off[B + 1];
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f], sl = lb % S;
        const int64_t base = frames[f].pix0;
        const int k = states[f].dc.n_cand;
        const int K_old = states[f].dc.n_kept;
        const int a = (lb / S) * kMT + threadIdx.x;
        const int lo = (int)((int64_t)sl * K_old / S), hi = (int)((int64_t)(sl + 1) * K_old / S);
        float x[Dp];
        if (a < k) ldv<Dp>(x, X + (int64_t)cand[base + a] * Dp);
        bool removed = false;
        for (int t0 = lo; t0 < hi; t0 += kVT) {
            const int cnt = min(kVT, hi - t0);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt * Dp; q += kMT) tile[q] = modes[(base + t0) * Dp + q];
            __syncthreads();
            if (a < k && !removed)
                for (int j = 0; j < cnt; ++j)
                    if (cos_at_least<Dp>(x, tile + j * Dp, thr_f, thr)) {
                        removed = true;
                        break;
                    }
        }
        if (a < k && removed) {
            cand_state[base + a] = kRemoved;
            removed_r[base + cand_rank[base + a]] = 1;
        }
        __syncthreads();
    }
}

template <int Dp>
__global__ void __launch_bounds__(kMT)
k_b_merge_pairs(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
                const int32_t* __restrict__ off, const float* __restrict__ Xr, const uint8_t* __restrict__ removed_r,
                const int32_t* __restrict__ rank_cand, float thr_f, double thr, int32_t* __restrict__ conf_deg,
                int32_t* __restrict__ conf) {
    // Candidates are visited in rank order: thread t of a block takes rank
    // r0 + t and compares it with every higher-priority candidate (rank < its
    // own) in the block's slice of ranks, so neighbouring lanes stop at
    // neighbouring ranks and only the k(k-1)/2 ordered pairs are tested. The
    // positions come from Xr (rank order), so a tile is one contiguous block
    // of rows, read as float4.
    constexpr int kQ = kVT * Dp / 4;  // float4 per tile
    __shared__ __align__(16) float tile[kVT * Dp];
    __shared__ int32_t s_idx[kVT];
    __shared__ uint8_t s_rem[kVT];
    const int S = off[B + 1];
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f], sl = lb % S;
        const int64_t base = frames[f].pix0;
        const int k = states[f].dc.n_cand;
        const int r0 = (lb / S) * kMT;
        const int r = r0 + threadIdx.x;
        const bool act = r < k && !removed_r[base + r];
        const int a = act ? rank_cand[base + r] : -1;
        const int lo = (int)((int64_t)sl * k / S);
        const int hi = min((int)((int64_t)(sl + 1) * k / S), r0 + kMT - 1);
        float x[Dp];
        if (act) ldv<Dp>(x, Xr + (base + r) * Dp);
        for (int t0 = lo; t0 < hi; t0 += kVT) {
            const int cnt = min(kVT, hi - t0);
            __syncthreads();
            const float4* src = reinterpret_cast<const float4*>(Xr + (base + t0) * Dp);
            for (int q = threadIdx.x; q < cnt * (Dp / 4) && q < kQ; q += kMT) reinterpret_cast<float4*>(tile)[q] = src[q];
            for (int j = threadIdx.x; j < cnt; j += kMT) {
                s_idx[j] = rank_cand[base + t0 + j];
                s_rem[j] = removed_r[base + t0 + j];
            }
            __syncthreads();
            if (act) {
                const int jend = min(cnt, r - t0);
                for (int j = 0; j < jend; ++j) {
                    if (s_rem[j]) continue;
                    if (cos_at_least<Dp>(x, tile + j * Dp, thr_f, thr)) {
                        const int slot = atomicAdd(&conf_deg[base + a], 1);
                        if (slot < kMergeCap) conf[(base + a) * kMergeCap + slot] = s_idx[j];
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int Dp>
__global__ void __launch_bounds__(kMT)
k_b_merge_resolve(const BFrame* __restrict__ frames, BState* states, int B, const int32_t* __restrict__ off,
                  const float* __restrict__ X, const int32_t* __restrict__ cand,
                  const int32_t* __restrict__ cand_rank, const int32_t* __restrict__ rank_cand, uint8_t* cand_state,
                  const int32_t* __restrict__ conf_deg, const int32_t* __restrict__ conf, float thr_f, double thr,
                  int count_left) {
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f];
        const int64_t base = frames[f].pix0;
        const int k = states[f].dc.n_cand;
        const int a = lb * kMT + threadIdx.x;
        if (a >= k) continue;
        volatile uint8_t* st = cand_state + base;
        if (st[a] != kUndecided) continue;
        const int deg = conf_deg[base + a];
        bool any_kept = false, all_removed = true;
        if (deg <= kMergeCap) {
            for (int j = 0; j < deg; ++j) {
                const uint8_t s = st[conf[(base + a) * kMergeCap + j]];
                if (s == kKept) { any_kept = true; break; }
                if (s == kUndecided) all_removed = false;
            }
        } else {
            // more conflicts than were stored: test the candidates ranked
            // above this one again, in rank order
            float x[Dp];
            ldv<Dp>(x, X + (int64_t)cand[base + a] * Dp);
            const int ra = cand_rank[base + a];
            for (int rb = 0; rb < ra; ++rb) {
                const int b2 = rank_cand[base + rb];
                const uint8_t s = st[b2];
                if (s == kRemoved) continue;
                if (!cos_at_least<Dp>(x, X + (int64_t)cand[base + b2] * Dp, thr_f, thr)) continue;
                if (s == kKept) { any_kept = true; break; }
                all_removed = false;
            }
        }
        if (any_kept)
            st[a] = kRemoved;
        else if (all_removed)
            st[a] = kKept;
        else if (count_left)
            atomicAdd(&states[f].dc.undecided, 1);
    }
}

template <int Dp>
__global__ void k_b_merge_sequential(const BFrame* __restrict__ frames, const BState* __restrict__ states,
                                     const float* __restrict__ X, const int32_t* __restrict__ cand,
                                     const int32_t* __restrict__ rank_cand, uint8_t* cand_state, float thr_f,
                                     double thr) {
    const int f = blockIdx.x;
    const BState& s0 = states[f];
    if (s0.phase != kRoundDone || s0.dc.undecided == 0) return;
    const int64_t base = frames[f].pix0;
    const int k = s0.dc.n_cand;
    volatile uint8_t* st = cand_state + base;
    const int lane = threadIdx.x;
    for (int r = 0; r < k; ++r) {
        const int a = rank_cand[base + r];
        if (st[a] != kUndecided) continue;
        const float* xa = X + (int64_t)cand[base + a] * Dp;
        bool hit = false;
        for (int rb = lane; rb < r && !hit; rb += 32) {
            const int b2 = rank_cand[base + rb];
            if (st[b2] == kKept && cos_at_least<Dp>(xa, X + (int64_t)cand[base + b2] * Dp, thr_f, thr)) hit = true;
        }
        const bool any = __any_sync(0xffffffffu, hit);
        if (lane == 0) st[a] = any ? kRemoved : kKept;
        __syncwarp();
    }
}

template <int Dp>
__global__ void __launch_bounds__(kIT)
k_b_merge_append(const BFrame* __restrict__ frames, BState* states, const float* __restrict__ X,
                 const int32_t* __restrict__ cand, const int32_t* __restrict__ rank_cand,
                 const uint8_t* __restrict__ cand_state, float* __restrict__ modes) {
    const int f = blockIdx.x;
    BState& st = states[f];
    if (st.phase != kRoundDone) return;
    const int64_t base = frames[f].pix0;
    const int k = st.dc.n_cand;
    const int kept0 = st.dc.n_kept;
    int carry = 0;
    for (int r0 = 0; r0 < k; r0 += kIT) {
        const int r = r0 + threadIdx.x;
        const int a = r < k ? rank_cand[base + r] : -1;
        const bool flag = a >= 0 && cand_state[base + a] == kKept;
        int tot;
        const int ex = block_scan(flag ? 1 : 0, &tot);
        if (flag) {
            const int64_t dst = base + kept0 + carry + ex;
            const int64_t slot = cand[base + a];
            for (int q = 0; q < Dp / 4; ++q)
                reinterpret_cast<float4*>(modes + dst * Dp)[q] = reinterpret_cast<const float4*>(X + slot * Dp)[q];
        }
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.k0 = kept0;
        st.dc.n_kept = kept0 + carry;
    }
}

// Coverage for the frames whose round ended: FP32 decides, FP64 inside the band.
// A block takes kPT * cov_per(Dp) consecutive pixels (1024 for d <= 16),
// compacts the uncovered ones into a shared list (warp ballots and a prefix
// over the block's warp-passes) and gives each thread up to cov_per of them,
// so every tile of new modes read from memory is tested against all the
// block's uncovered pixels at once.
__host__ __device__ constexpr int cov_per(int Dp) { return Dp <= 16 ? 4 : 2; }

template <int Dp>
__global__ void __launch_bounds__(kPT)
k_b_cover(const BFrame* __restrict__ frames, BState* states, int B, const int32_t* __restrict__ off, int d,
          const float* __restrict__ P32, const int32_t* __restrict__ pix, uint8_t* __restrict__ covered,
          const float* __restrict__ modes, float c_f, double c) {
    __shared__ __align__(16) float tile[kVT * Dp];
    constexpr int kCovPer = cov_per(Dp);
    constexpr int kNW = kPT / 32 * kCovPer;  // warp-passes of a block
    static_assert(kNW <= 32, "one warp scans the warp-pass counts");
    __shared__ int32_t s_list[kPT * kCovPer];
    __shared__ int32_t s_pos[kNW];
    __shared__ int s_nact;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f];
        const BFrame& fr = frames[f];
        BState& st = states[f];
        const int64_t base = fr.pix0;
        const int k0 = st.k0, k1 = st.dc.n_kept;
        const int i0 = lb * kPT * kCovPer;
        unsigned bal[kCovPer];
#pragma unroll
        for (int u = 0; u < kCovPer; ++u) {
            const int i = i0 + u * kPT + threadIdx.x;
            bal[u] = __ballot_sync(0xffffffffu, i < fr.n && covered[base + i] == 0);
            if (lane == 0) s_pos[u * (kPT / 32) + warp] = __popc(bal[u]);
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
        for (int u = 0; u < kCovPer; ++u)
            if ((bal[u] >> lane) & 1u)
                s_list[s_pos[u * (kPT / 32) + warp] + __popc(bal[u] & ((1u << lane) - 1u))] =
                    i0 + u * kPT + threadIdx.x;
        __syncthreads();
        const int nact = s_nact;
        if (nact == 0) continue;
        int idx[kCovPer];
        float p[kCovPer][Dp];
        bool cov[kCovPer], band[kCovPer];
#pragma unroll
        for (int u = 0; u < kCovPer; ++u) {
            const int e = threadIdx.x + u * kPT;
            idx[u] = e < nact ? s_list[e] : -1;
            if (idx[u] >= 0) ldv<Dp>(p[u], P32 + (base + idx[u]) * Dp);
            cov[u] = band[u] = false;
        }
        for (int t0 = k0; t0 < k1; t0 += kVT) {
            const int cnt = min(kVT, k1 - t0);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt * Dp; q += kPT) tile[q] = modes[(base + t0) * Dp + q];
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kCovPer; ++u)
                if (idx[u] >= 0 && !cov[u])
                    for (int j = 0; j < cnt; ++j) {
                        const float sc = dot_seq<Dp>(p[u], tile + j * Dp);
                        if (sc >= c_f + kEpsF32) { cov[u] = true; break; }
                        if (sc >= c_f - kEpsF32) band[u] = true;
                    }
        }
        int newly = 0;
#pragma unroll
        for (int u = 0; u < kCovPer; ++u) {
            if (idx[u] >= 0 && !cov[u] && band[u]) {
                const float* e = fr.emb + (int64_t)pix[base + idx[u]] * d;
                for (int j = k0; j < k1 && !cov[u]; ++j) {
                    const float* m = modes + (base + j) * Dp;
                    if (dot_seq<Dp>(p[u], m) >= c_f - kEpsF32 && cos64(e, m, d) >= c) cov[u] = true;
                }
            }
            if (idx[u] >= 0 && cov[u]) {
                covered[base + idx[u]] = 1;
                ++newly;
            }
        }
        // each warp's count of newly covered pixels
        for (int o = 16; o > 0; o >>= 1) newly += __shfl_xor_sync(0xffffffffu, newly, o);
        if (lane == 0 && newly) atomicSub(&st.dc.n_uncovered, newly);
        __syncthreads();
    }
}

__global__ void k_b_schedule(BState* states, int B, double P, double L, double H, int max_rounds, int all_seeds) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    BState& st = states[f];
    if (st.phase != kRoundDone) return;
    st.rounds += 1;
    st.N = d_schedule(st.N, st.dc.n_kept, P, L, H, st.dc.n_uncovered);
    const bool fin = st.dc.n_uncovered <= 0 || st.rounds >= max_rounds || all_seeds;
    st.phase = fin ? kFinished : kNeedSeed;
}

// Profiling ticks around the shift launch (kernels of one stream run in
// order, so stop - start spans the shift kernel plus one launch gap). The
// global timer counts nanoseconds.
__global__ void k_b_tick(int* misc, const int32_t* __restrict__ item_total, int stop) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    unsigned long long* m = reinterpret_cast<unsigned long long*>(misc);
    if (!stop) {
        m[2] = t;
    } else if (*item_total > 0) {
        m[3] += t - m[2];
        m[4] += 1ull;
    }
}

// Phase timer (profiling level 2): adds the global-timer time since the last
// phase tick to phase sum `slot` (u64 misc words 8..15); slot < 0 only starts
// the clock. Ticks sit between the phases in stream order, so a phase's sum
// includes the launch gaps inside it.
__global__ void k_b_phase(int* misc, int slot) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    unsigned long long* m = reinterpret_cast<unsigned long long*>(misc);
    if (slot >= 0) m[8 + slot] += t - m[7];
    m[7] = t;
}

__global__ void k_b_cond(const BState* __restrict__ states, int B, int* misc, int max_passes,
                         cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    int live = 0;
    for (int f = 0; f < B; ++f) live += states[f].phase != kFinished;
    const int passes = ++misc[0];
    if (passes >= max_passes && live) misc[1] |= 2;
    if (misc[1] != 0) live = 0;  // bad input or a bounded wait gave up: stop, the host reports it
    cudaGraphSetConditional(h, live ? 1u : 0u);
}

// ------------------------------------------------------------ labels
template <int Dp>
__global__ void __launch_bounds__(kPT)
k_b_label(const BFrame* __restrict__ frames, const BState* __restrict__ states, int B,
          const int32_t* __restrict__ off, int d, const float* __restrict__ P32, const int32_t* __restrict__ pix,
          const float* __restrict__ modes, int32_t* const* __restrict__ labels) {
    __shared__ __align__(16) float tile[kVT * Dp];
    for (int bb = blockIdx.x; bb < off[B]; bb += gridDim.x) {
        const int f = locate(off, B, bb);
        const int lb = bb - off[f];
        const BFrame& fr = frames[f];
        const int64_t base = fr.pix0;
        const int K = states[f].dc.n_kept;
        const int i = lb * kPT + threadIdx.x;
        const bool act = i < fr.n;
        float p[Dp];
        if (act) ldv<Dp>(p, P32 + (base + i) * Dp);
        float b1 = -INFINITY, b2 = -INFINITY;
        int best = -1;
        for (int t0 = 0; t0 < K; t0 += kVT) {
            const int cnt = min(kVT, K - t0);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt * Dp; q += kPT) tile[q] = modes[(base + t0) * Dp + q];
            __syncthreads();
            if (act)
                for (int j = 0; j < cnt; ++j) {
                    const float s = dot_seq<Dp>(p, tile + j * Dp);
                    if (s > b1) { b2 = b1; b1 = s; best = t0 + j; }
                    else if (s > b2) b2 = s;
                }
        }
        if (act) {
            if (K > 1 && b1 - b2 <= 2.f * kEpsF32) {
                const float* e = fr.emb + (int64_t)pix[base + i] * d;
                double bc = -INFINITY;
                for (int j = 0; j < K; ++j) {
                    const float* m = modes + (base + j) * Dp;
                    if (dot_seq<Dp>(p, m) < b1 - 2.f * kEpsF32) continue;
                    const double cs = cos64(e, m, d);
                    if (cs > bc) { bc = cs; best = j; }
                }
            }
            labels[f][pix[base + i]] = best;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ host
float ceil_f(double c) { return ceil_to_float(c); }

template <int Dp>
ms_status enqueue_body(ms_batch* b, cudaStream_t s, cudaGraphConditionalHandle h, bool with_cond, int64_t* nlaunch) {
    const int B = b->B;
    const float cf = ceil_f(b->cfg.bandwidth_cos);
    const float mf = (float)b->cfg.merge_cos;
    const double gamma = b->cfg.all_seeds ? 1.0 : b->cfg.gamma;
    const double L = b->cfg.L > 0.0 ? b->cfg.L : b->cfg.alpha / gamma;
    const int G = b->grid;
    int64_t nl = 0;
#define LAUNCHED(name) do { MS_LAUNCH(name); ++nl; } while (0)
    k_b_seed<<<B, kIT, 0, s>>>(b->frames, b->states, b->P32, Dp, b->covered, b->X, b->seed_pix, b->seed_order,
                               b->act[0], b->sstate, b->cfg.max_rounds, b->cfg.all_seeds);
    LAUNCHED("k_b_seed");
    // Split 0 gives every frame the single-frame target (2 x grid), so each
    // frame's results equal a single-frame run's; split 1 shares
    // target_mult x grid items across the iterating frames by their work.
    const int grid_shift = b->tc ? b->tc_grid : b->f32_grid;
    k_b_plan<<<1, kIT, 0, s>>>(b->frames, b->states, B, b->plan, b->target_mult * grid_shift,
                               b->split ? 0 : 2 * grid_shift, b->tc ? 1 : 0, grid_shift);
    LAUNCHED("k_b_plan");
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhSeed);
        LAUNCHED("k_b_phase");
    }
    if (b->prof) {
        k_b_tick<<<1, 1, 0, s>>>(b->misc, b->plan.item_off + B, 0);
        LAUNCHED("k_b_tick");
    }
    ms_status st;
    if (b->tc)
        st = launch_shift_tc_batch(b->pmap, b->pmap1, Dp, b->P32, b->X, b->acc, cf, b->frames, b->states, b->plan,
                                   b->act[0],
                                   b->act[1], B, b->misc + 1, (unsigned long long*)(b->misc + 2), b->tc_grid,
                                   b->tc_shape, s);
    else
        st = launch_shift_fp32_batch(b->P32, b->X, b->acc, cf, Dp, b->frames, b->states, b->plan, b->act[0],
                                     b->act[1], B, b->f32_grid, s);
    if (st != MS_OK) return st;
    ++nl;
    if (b->prof) {
        k_b_tick<<<1, 1, 0, s>>>(b->misc, b->plan.item_off + B, 1);
        LAUNCHED("k_b_tick");
    }
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhShift);
        LAUNCHED("k_b_phase");
    }
    k_b_finalize<Dp><<<G, 256, 0, s>>>(b->frames, b->states, B, b->plan, b->act[0], b->act[1], b->acc, b->X,
                                       b->sstate, b->support, b->cfg.tol);
    LAUNCHED("k_b_finalize");
    k_b_check<<<(B + 255) / 256, 256, 0, s>>>(b->states, B, gamma, b->cfg.max_iter);
    LAUNCHED("k_b_check");
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhFinalize);
        LAUNCHED("k_b_phase");
    }
    // merge chain for the frames whose round ended
    k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, B, kSelDoneSeeds, 256, 0, b->blk_off);
    LAUNCHED("k_b_blocks");
    k_b_collect<<<G, 256, 0, s>>>(b->frames, b->states, B, b->blk_off, b->sstate, b->cand);
    LAUNCHED("k_b_collect");
    k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, B, kSelDoneCands, kMT, 0, b->blk_off);
    LAUNCHED("k_b_blocks");
    k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, B, kSelDoneCands, kMT, 4 * b->num_sms, b->blk_split);
    LAUNCHED("k_b_blocks");
    k_b_merge_zero<<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_off, b->cand_rank, b->cand_state,
                                     b->conf_deg, b->removed_r);
    LAUNCHED("k_b_merge_zero");
    k_b_rank<<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_split, b->cand, b->support, b->seed_order,
                               b->cand_rank);
    LAUNCHED("k_b_rank");
    k_b_rank_invert<Dp><<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_off, b->cand_rank, b->cand, b->X,
                                          b->rank_cand, b->Xr);
    LAUNCHED("k_b_rank_invert");
    if (b->Ck) {  // BF16 form: both contractions of the merge on the tensor cores
        ms_status ms2 = launch_merge_tc_batch(b->cmap, b->cmap1, b->mmap, b->mmap1, b->Ck, b->total_pk_rows, Dp,
                                              b->frames, b->states, B, (int)b->max_pk_rows, b->Xr, b->modes,
                                              b->rank_cand, b->cand_state, b->removed_r, b->conf_deg, b->conf, mf,
                                              b->cfg.merge_cos, b->blk_off, b->lsc, b->num_sms, b->misc + 1, s);
        if (ms2 != MS_OK) return ms2;
        nl += 4;
    } else {
        k_b_merge_old<Dp><<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_split, b->X, b->cand, b->modes, mf,
                                            b->cfg.merge_cos, b->cand_state, b->cand_rank, b->removed_r);
        LAUNCHED("k_b_merge_old");
        k_b_merge_pairs<Dp><<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_split, b->Xr, b->removed_r,
                                              b->rank_cand, mf, b->cfg.merge_cos, b->conf_deg, b->conf);
        LAUNCHED("k_b_merge_pairs");
    }
    for (int sw = 0; sw < 8; ++sw) {
        k_b_merge_resolve<Dp><<<G, kMT, 0, s>>>(b->frames, b->states, B, b->blk_off, b->X, b->cand, b->cand_rank,
                                                b->rank_cand, b->cand_state, b->conf_deg, b->conf, mf,
                                                b->cfg.merge_cos, sw == 7);
        LAUNCHED("k_b_merge_resolve");
    }
    k_b_merge_sequential<Dp><<<B, 32, 0, s>>>(b->frames, b->states, b->X, b->cand, b->rank_cand, b->cand_state, mf,
                                              b->cfg.merge_cos);
    LAUNCHED("k_b_merge_sequential");
    k_b_merge_append<Dp><<<B, kIT, 0, s>>>(b->frames, b->states, b->X, b->cand, b->rank_cand, b->cand_state,
                                           b->modes);
    LAUNCHED("k_b_merge_append");
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhMerge);
        LAUNCHED("k_b_phase");
    }
    if (b->Mk) {  // BF16 form: the pixels against the new modes on the tensor cores
        k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, B, kSelDonePixels, 128, 0, b->blk_off);
        LAUNCHED("k_b_blocks");
        ms_status cs = launch_cover_tc_batch(b->pmap, b->mmap, b->pmap1, b->mmap1, b->Mk, b->total_pk_rows, Dp,
                                             b->frames, b->states, B, (int)b->max_pk_rows,
                                             b->modes, b->P32, b->pix, b->d, b->cfg.bandwidth_cos, b->covered,
                                             b->blk_off, b->lsc, b->num_sms, b->misc + 1, s);
        if (cs != MS_OK) return cs;
        nl += 3;
    } else {
        k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, B, kSelDonePixels, kPT * cov_per(Dp), 0, b->blk_off);
        LAUNCHED("k_b_blocks");
        k_b_cover<Dp><<<G, kPT, 0, s>>>(b->frames, b->states, B, b->blk_off, b->d, b->P32, b->pix, b->covered,
                                        b->modes, (float)b->cfg.bandwidth_cos, b->cfg.bandwidth_cos);
        LAUNCHED("k_b_cover");
    }
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhCover);
        LAUNCHED("k_b_phase");
    }
    k_b_schedule<<<(B + 255) / 256, 256, 0, s>>>(b->states, B, b->cfg.P_target, L, b->cfg.H, b->cfg.max_rounds,
                                                 b->cfg.all_seeds);
    LAUNCHED("k_b_schedule");
    if (with_cond) {
        k_b_cond<<<1, 32, 0, s>>>(b->states, B, b->misc,
                                  b->cfg.batch_max_passes > 0 ? b->cfg.batch_max_passes : kDefaultMaxPasses, h);
        LAUNCHED("k_b_cond");
    }
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhSchedule);
        LAUNCHED("k_b_phase");
    }
#undef LAUNCHED
    *nlaunch = nl;
    return MS_OK;
}

template <int Dp>
ms_status enqueue_setup(ms_batch* b, cudaStream_t s) {
    const int B = b->B;
    MS_CUDA(cudaMemsetAsync(b->covered, 0, (size_t)b->total_px, s));
    MS_CUDA(cudaMemsetAsync(b->acc, 0, sizeof(unsigned long long) * (size_t)b->total_px * (Dp + 1), s));
    MS_CUDA(cudaMemsetAsync(b->misc, 0, sizeof(b->h_misc), s));
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, -1);
        MS_LAUNCH("k_b_phase");
    }
    const dim3 gc((unsigned)b->nblk_max, (unsigned)B);
    k_b_count<<<gc, kIT, 0, s>>>(b->frames, (int)b->nblk_max, b->block_tmp);
    MS_LAUNCH("k_b_count");
    k_b_scan<<<B, kIT, 0, s>>>(b->frames, b->states, (int)b->nblk_max, b->block_tmp, b->cfg.seed,
                               b->cfg.frame_id, b->cfg.n_initial);
    MS_LAUNCH("k_b_scan");
    k_b_compact<<<gc, kIT, 0, s>>>(b->frames, (int)b->nblk_max, b->block_tmp, b->d, Dp, b->P32, b->pix, b->misc + 1);
    MS_LAUNCH("k_b_compact");
    if (b->tc) {
        const dim3 gp((unsigned)((b->max_pk_rows + 255) / 256), (unsigned)B);
        k_b_pack<<<gp, 256, 0, s>>>(b->frames, b->P32, Dp, (int64_t)b->total_pk_rows, (uint4*)b->Pk);
        MS_LAUNCH("k_b_pack");
    }
    const dim3 gl((unsigned)((b->max_np + 255) / 256 < 1024 ? (b->max_np + 255) / 256 : 1024), (unsigned)B);
    k_b_labels_clear<<<gl, 256, 0, s>>>(b->frames, b->label_ptrs);
    MS_LAUNCH("k_b_labels_clear");
    if (b->prof_phases) {
        k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhSetup);
        MS_LAUNCH("k_b_phase");
    }
    return MS_OK;
}

// The labelling phase's closing tick (profiling level 2).
ms_status enqueue_label_tick(ms_batch* b, cudaStream_t s) {
    if (!b->prof_phases) return MS_OK;
    k_b_phase<<<1, 1, 0, s>>>(b->misc, kPhLabel);
    MS_LAUNCH("k_b_phase");
    return MS_OK;
}

template <int Dp>
ms_status enqueue_label(ms_batch* b, cudaStream_t s) {
    if (b->Mk)  // BF16 form: the tensor-core kernel, same labels (exact FP64 argmax)
        return launch_label_tc_batch(b->pmap, b->mmap, b->pmap1, b->mmap1, b->Mk, b->total_pk_rows, Dp, b->frames,
                                     b->states, b->B, (int)b->max_pk_rows,
                                     b->modes, b->P32, b->pix, b->d, b->label_ptrs, b->lsc, b->num_sms, b->misc + 1,
                                     s);
    k_b_blocks<<<1, 32, 0, s>>>(b->frames, b->states, b->B, kSelAllPixels, kPT, 0, b->blk_off);
    MS_LAUNCH("k_b_blocks");
    k_b_label<Dp><<<b->grid, kPT, 0, s>>>(b->frames, b->states, b->B, b->blk_off, b->d, b->P32, b->pix, b->modes,
                                          b->label_ptrs);
    MS_LAUNCH("k_b_label");
    return MS_OK;
}

template <int Dp>
ms_status build_graph(ms_batch* b) {
    cudaGraph_t g = nullptr;
    MS_CUDA(cudaGraphCreate(&g, 0));
    b->graph = g;
    cudaStream_t s = b->cap;
    MS_CUDA(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ms_status st = enqueue_setup<Dp>(b, s);
    std::vector<cudaGraphNode_t> deps;
    if (st == MS_OK) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        st = cuda_check(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd), "capture info");
        if (st == MS_OK) deps.assign(d, d + nd);
    }
    cudaGraph_t tmp = nullptr;
    ms_status st2 = cuda_check(cudaStreamEndCapture(s, &tmp), "end capture (set-up)");
    if (st != MS_OK) return st;
    if (st2 != MS_OK) return st2;
    cudaGraphConditionalHandle h;
    MS_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    MS_CUDA(cudaGraphAddNode(&cnode, g, deps.data(), nullptr, deps.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MS_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int64_t nl = 0;
    st = enqueue_body<Dp>(b, s, h, true, &nl);
    st2 = cuda_check(cudaStreamEndCapture(s, &tmp), "end capture (body)");
    if (st != MS_OK) return st;
    if (st2 != MS_OK) return st2;
    MS_CUDA(cudaStreamBeginCaptureToGraph(s, g, &cnode, nullptr, 1, cudaStreamCaptureModeRelaxed));
    st = enqueue_label<Dp>(b, s);
    if (st == MS_OK) st = enqueue_label_tick(b, s);
    st2 = cuda_check(cudaStreamEndCapture(s, &tmp), "end capture (labels)");
    if (st != MS_OK) return st;
    if (st2 != MS_OK) return st2;
    MS_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->body_launches = nl;
    b->fixed_launches = (b->tc ? 5 : 4) + (b->Mk ? 4 : 2) + (b->prof_phases ? 3 : 0);  // set-up, then labelling
    return MS_OK;
}

// The graph's kernels as ordinary launches on the batch's stream: set-up,
// `passes` loop bodies (without the loop-control kernel) and labelling.
template <int Dp>
ms_status enqueue_eager(ms_batch* b, int passes) {
    ms_status st = enqueue_setup<Dp>(b, b->stream);
    for (int p = 0; st == MS_OK && p < passes; ++p) {
        int64_t nl = 0;
        st = enqueue_body<Dp>(b, b->stream, cudaGraphConditionalHandle{}, false, &nl);
    }
    if (st == MS_OK) st = enqueue_label<Dp>(b, b->stream);
    if (st == MS_OK) st = enqueue_label_tick(b, b->stream);
    return st;
}

ms_status rebuild_graph(ms_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return b->Dp == 16 ? build_graph<16>(b) : build_graph<32>(b);
}

void free_batch(ms_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ws) cudaFree(b->ws);
    if (b->h_states) cudaFreeHost(b->h_states);
    delete b;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" ms_status ms_batch_create(const ms_config* cfg, int32_t B, const float* const* d_embs,
                                     const uint8_t* const* d_masks, const int64_t* n_pixels,
                                     int32_t* const* d_labels, void* stream, ms_batch** out) {
    if (!out) return set_error(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return set_error(MS_ERR_INVALID_ARG, "config is NULL");
    if (B < 1 || B > 4096 || !d_embs || !n_pixels || !d_labels) return set_error(MS_ERR_INVALID_ARG, "bad batch");
    if (cfg->dim < 1 || cfg->dim > MS_MAX_DIM || cfg->kernel != MS_FLAT || !(cfg->tol > 0.0) || cfg->max_iter < 1 ||
        cfg->n_initial < 1 || !(cfg->gamma >= 0.0 && cfg->gamma <= 1.0) ||
        !(cfg->P_target > 0.0 && cfg->P_target < 1.0) || cfg->max_rounds < 1 ||
        (cfg->precision != MS_FP32 && cfg->precision != MS_BF16) ||
        (cfg->batch_split != 0 && cfg->batch_split != 1) || cfg->tc_shape < 0 || cfg->tc_shape >= ms::kTcShapes)
        return set_error(MS_ERR_INVALID_ARG, "invalid config");
    ms_batch* b = new (std::nothrow) ms_batch();
    if (!b) return set_error(MS_ERR_OOM, "host allocation failed");
    b->cfg = *cfg;
    b->B = B;
    b->d = cfg->dim;
    b->Dp = padded_dim(cfg->dim);
    b->tc = cfg->precision == MS_BF16;
    b->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = b->num_sms * 8;
    b->split = cfg->batch_split;
    b->target_mult = 2;
    b->tc_shape = cfg->tc_shape;
    b->tc_grid = b->num_sms;
    b->f32_grid = b->num_sms * shift_blocks_per_sm();
    std::vector<BFrame> hf((size_t)B);
    int64_t px = 0, rows = 0;
    b->max_np = 1;
    for (int f = 0; f < B; ++f) {
        if (n_pixels[f] < 0 || n_pixels[f] >= (1LL << 24) || (n_pixels[f] > 0 && (!d_embs[f] || !d_labels[f]))) {
            free_batch(b);
            return set_error(MS_ERR_INVALID_ARG, "frame %d: bad pixels or buffers", f);
        }
        memset(&hf[f], 0, sizeof(BFrame));
        hf[f].pix0 = px;
        hf[f].n_pixels = n_pixels[f];
        hf[f].pk_row0 = (int32_t)rows;
        hf[f].emb = d_embs[f];
        hf[f].mask = d_masks ? d_masks[f] : nullptr;
        px += n_pixels[f];
        rows += (n_pixels[f] + 127) / 128 * 128;
        if (n_pixels[f] > b->max_np) b->max_np = n_pixels[f];
    }
    if (px >= (1LL << 31) - 1) {
        free_batch(b);
        return set_error(MS_ERR_INVALID_ARG, "batch too large");
    }
    b->hf = hf;
    b->h_labels.assign(d_labels, d_labels + B);
    b->total_px = px > 0 ? px : 1;
    b->total_pk_rows = rows > 0 ? rows : 128;
    b->max_pk_rows = (b->max_np + 127) / 128 * 128;
    b->nblk_max = (b->max_np + kIT - 1) / kIT;
    const int Dp = b->Dp;
    const bool tcl = b->tc;  // labelling and coverage on the tensor cores
    const size_t n = (size_t)b->total_px;
    const size_t sizes[] = {
        sizeof(BFrame) * B, sizeof(BState) * B, sizeof(int32_t) * ((B + 1) * 4 + (B + 2) * 2), sizeof(b->h_misc),
        n * Dp * 4, n * 4, n, n * Dp * 4, n * 4, n * 4, n, n * 4, n * 4, n * 4,
        n * (Dp + 1) * 8, n * Dp * 4, n * 4, n * 4, n * 4, n, n * 4, n * kMergeCap * 4,
        (size_t)B * b->nblk_max * 4 + 4, b->tc ? (size_t)b->total_pk_rows * 128 * (Dp / 16) : 0, sizeof(int32_t*) * B,
        tcl ? (size_t)b->total_pk_rows * 128 * (Dp / 16) : 0, tcl ? n * sizeof(int2) : 0, sizeof(int32_t) * (B + 1) + 16,
        n * Dp * 4, n, tcl ? (size_t)b->total_pk_rows * 128 * (Dp / 16) : 0};
    const int NS = (int)(sizeof(sizes) / sizeof(sizes[0]));
    size_t offs[32], tot = 0;
    for (int i = 0; i < NS; ++i) {
        offs[i] = tot;
        tot += (sizes[i] + 255) / 256 * 256;
    }
    cudaError_t e = workspace_malloc(&b->ws, tot);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_check(e, "cudaMalloc(batch workspace)");
    }
    b->ws_bytes = tot;
    char* w = (char*)b->ws;
    b->frames = (BFrame*)(w + offs[0]);
    b->states = (BState*)(w + offs[1]);
    int32_t* planmem = (int32_t*)(w + offs[2]);
    b->plan.item_off = planmem;
    b->plan.seed_off = planmem + (B + 1);
    b->plan.chunks = planmem + 2 * (B + 1);
    b->plan.tpc = planmem + 3 * (B + 1);
    b->blk_off = planmem + 4 * (B + 1);
    b->blk_split = b->blk_off + (B + 2);
    b->misc = (int32_t*)(w + offs[3]);
    b->P32 = (float*)(w + offs[4]);
    b->pix = (int32_t*)(w + offs[5]);
    b->covered = (uint8_t*)(w + offs[6]);
    b->X = (float*)(w + offs[7]);
    b->seed_pix = (int32_t*)(w + offs[8]);
    b->seed_order = (int32_t*)(w + offs[9]);
    b->sstate = (uint8_t*)(w + offs[10]);
    b->support = (int32_t*)(w + offs[11]);
    b->act[0] = (int32_t*)(w + offs[12]);
    b->act[1] = (int32_t*)(w + offs[13]);
    b->acc = (unsigned long long*)(w + offs[14]);
    b->modes = (float*)(w + offs[15]);
    b->cand = (int32_t*)(w + offs[16]);
    b->cand_rank = (int32_t*)(w + offs[17]);
    b->rank_cand = (int32_t*)(w + offs[18]);
    b->cand_state = (uint8_t*)(w + offs[19]);
    b->conf_deg = (int32_t*)(w + offs[20]);
    b->conf = (int32_t*)(w + offs[21]);
    b->block_tmp = (int32_t*)(w + offs[22]);
    b->Pk = b->tc ? (void*)(w + offs[23]) : nullptr;
    b->label_ptrs = (int32_t**)(w + offs[24]);
    b->Mk = tcl ? (void*)(w + offs[25]) : nullptr;
    b->lsc.fix = tcl ? (int2*)(w + offs[26]) : nullptr;
    b->lsc.off = (int32_t*)(w + offs[27]);
    b->lsc.fix_count = b->lsc.off + (B + 1);
    b->Xr = (float*)(w + offs[28]);
    b->removed_r = (uint8_t*)(w + offs[29]);
    b->Ck = tcl ? (void*)(w + offs[30]) : nullptr;
    ms_status s = cuda_check(cudaMallocHost((void**)&b->h_states, sizeof(BState) * B), "cudaMallocHost");
    if (s == MS_OK) s = cuda_check(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(b->frames, hf.data(), sizeof(BFrame) * B, cudaMemcpyHostToDevice, b->stream),
                       "copy frames");
    if (s == MS_OK)
        s = cuda_check(cudaMemcpyAsync(b->label_ptrs, d_labels, sizeof(int32_t*) * B, cudaMemcpyHostToDevice,
                                       b->stream),
                       "copy label pointers");
    if (s == MS_OK) s = cuda_check(cudaStreamSynchronize(b->stream), "sync");
    if (s == MS_OK && b->tc) s = tc_batch_setup(Dp);
    if (s == MS_OK && b->tc) s = encode_pk_map(b->Pk, (int)b->total_pk_rows, &b->pmap);
    if (s == MS_OK && b->tc)
        s = encode_pk_map(Dp == 32 ? (uint8_t*)b->Pk + (size_t)b->total_pk_rows * 128 : b->Pk, (int)b->total_pk_rows,
                          &b->pmap1);
    if (s == MS_OK && tcl) s = encode_pk_map(b->Mk, (int)b->total_pk_rows, &b->mmap);
    if (s == MS_OK && tcl) b->mmap1 = b->mmap;
    if (s == MS_OK && tcl && Dp == 32)
        s = encode_pk_map((uint8_t*)b->Mk + (size_t)b->total_pk_rows * 128, (int)b->total_pk_rows, &b->mmap1);
    if (s == MS_OK && tcl) s = encode_pk_map(b->Ck, (int)b->total_pk_rows, &b->cmap);
    if (s == MS_OK && tcl) b->cmap1 = b->cmap;
    if (s == MS_OK && tcl && Dp == 32)
        s = encode_pk_map((uint8_t*)b->Ck + (size_t)b->total_pk_rows * 128, (int)b->total_pk_rows, &b->cmap1);
    if (s == MS_OK && tcl) s = label_tc_setup();
    if (s == MS_OK) s = rebuild_graph(b);
    if (s != MS_OK) {
        free_batch(b);
        return s;
    }
    *out = b;
    return MS_OK;
}

extern "C" ms_status ms_batch_run(ms_batch* b, int32_t sync) {
    if (!b) return set_error(MS_ERR_INVALID_ARG, "batch is NULL");
    MS_CUDA(cudaGraphLaunch(b->exec, b->stream));
    if (!sync) return MS_OK;
    MS_CUDA(cudaMemcpyAsync(b->h_states, b->states, sizeof(BState) * b->B, cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaMemcpyAsync(b->h_misc, b->misc, sizeof(b->h_misc), cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaStreamSynchronize(b->stream));
    const int32_t* misc = b->h_misc;
    if (misc[1] & 1) return set_error(MS_ERR_INVALID_ARG, "a foreground embedding has zero or non-finite norm");
    if (misc[1] & 2) return set_error(MS_ERR_TIMEOUT, "a bounded device wait or the pass limit was hit");
    return MS_OK;
}

extern "C" ms_status ms_batch_run_host(ms_batch* b, const float* const* h_embs, const uint8_t* const* h_masks,
                                      int32_t* const* h_labels) {
    if (!b || !h_embs || !h_labels) return set_error(MS_ERR_INVALID_ARG, "NULL argument");
    for (int f = 0; f < b->B; ++f) {
        const BFrame& fr = b->hf[f];
        if (fr.n_pixels == 0) continue;
        if (!h_embs[f] || !h_labels[f]) return set_error(MS_ERR_INVALID_ARG, "frame %d: NULL host buffer", f);
        if (fr.mask && (!h_masks || !h_masks[f]))
            return set_error(MS_ERR_INVALID_ARG, "frame %d is masked: its host mask is required", f);
    }
    for (int f = 0; f < b->B; ++f) {
        const BFrame& fr = b->hf[f];
        if (fr.n_pixels == 0) continue;
        MS_CUDA(cudaMemcpyAsync((void*)fr.emb, h_embs[f], sizeof(float) * (size_t)fr.n_pixels * b->d,
                                cudaMemcpyHostToDevice, b->stream));
        if (fr.mask)
            MS_CUDA(cudaMemcpyAsync((void*)fr.mask, h_masks[f], (size_t)fr.n_pixels, cudaMemcpyHostToDevice,
                                    b->stream));
    }
    MS_CUDA(cudaGraphLaunch(b->exec, b->stream));
    for (int f = 0; f < b->B; ++f) {
        const BFrame& fr = b->hf[f];
        if (fr.n_pixels == 0) continue;
        MS_CUDA(cudaMemcpyAsync(h_labels[f], b->h_labels[f], sizeof(int32_t) * (size_t)fr.n_pixels,
                                cudaMemcpyDeviceToHost, b->stream));
    }
    MS_CUDA(cudaMemcpyAsync(b->h_states, b->states, sizeof(BState) * b->B, cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaMemcpyAsync(b->h_misc, b->misc, sizeof(b->h_misc), cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaStreamSynchronize(b->stream));
    if (b->h_misc[1] & 1) return set_error(MS_ERR_INVALID_ARG, "a foreground embedding has zero or non-finite norm");
    if (b->h_misc[1] & 2) return set_error(MS_ERR_TIMEOUT, "a bounded device wait or the pass limit was hit");
    return MS_OK;
}

extern "C" ms_status ms_batch_run_eager(ms_batch* b, int32_t passes) {
    if (!b || passes < 0) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    ms_status st = b->Dp == 16 ? enqueue_eager<16>(b, passes) : enqueue_eager<32>(b, passes);
    if (st != MS_OK) return st;
    MS_CUDA(cudaMemcpyAsync(b->h_states, b->states, sizeof(BState) * b->B, cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaMemcpyAsync(b->h_misc, b->misc, sizeof(b->h_misc), cudaMemcpyDeviceToHost, b->stream));
    MS_CUDA(cudaStreamSynchronize(b->stream));
    b->h_misc[0] = passes;
    if (b->h_misc[1] & 1) return set_error(MS_ERR_INVALID_ARG, "a foreground embedding has zero or non-finite norm");
    if (b->h_misc[1] & 2) return set_error(MS_ERR_TIMEOUT, "a bounded device wait gave up");
    for (int f = 0; f < b->B; ++f)
        if (b->h_states[f].phase != kFinished) return set_error(MS_ERR_STATE, "frame %d unfinished after %d passes", f, passes);
    return MS_OK;
}

extern "C" ms_status ms_batch_configure(ms_batch* b, int32_t batch_split, int32_t target_mult, int32_t tc_shape) {
    if (!b || (batch_split != 0 && batch_split != 1) || target_mult < 1 || target_mult > 64 || tc_shape < 0 ||
        tc_shape >= ms::kTcShapes)
        return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    if (batch_split == b->split && target_mult == b->target_mult && tc_shape == b->tc_shape) return MS_OK;
    MS_CUDA(cudaStreamSynchronize(b->stream));
    b->split = batch_split;
    b->target_mult = target_mult;
    b->tc_shape = tc_shape;
    return rebuild_graph(b);
}

namespace {
// Median of `reps` graph launches of the batch as configured now, after one
// warm-up run (which also checks the batch's status).
ms_status time_graph(ms_batch* b, int reps, cudaEvent_t e0, cudaEvent_t e1, double* med) {
    ms_status st = ms_batch_run(b, 1);
    std::vector<float> t;
    for (int r = 0; st == MS_OK && r < reps; ++r) {
        st = cuda_check(cudaEventRecord(e0, b->stream), "cudaEventRecord");
        if (st == MS_OK) st = cuda_check(cudaGraphLaunch(b->exec, b->stream), "cudaGraphLaunch");
        if (st == MS_OK) st = cuda_check(cudaEventRecord(e1, b->stream), "cudaEventRecord");
        if (st == MS_OK) st = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms_ = 0.f;
        if (st == MS_OK) st = cuda_check(cudaEventElapsedTime(&ms_, e0, e1), "cudaEventElapsedTime");
        t.push_back(ms_);
    }
    if (st != MS_OK) return st;
    std::sort(t.begin(), t.end());
    *med = t[t.size() / 2];
    return MS_OK;
}
}  // namespace

extern "C" ms_status ms_batch_autotune(ms_batch* b, int32_t reps, ms_tune_result* results, int32_t cap,
                                       int32_t* n_results) {
    if (!b || reps < 1 || reps > 100 || cap < 0) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    static const int kSplits[][2] = {{0, 2}, {1, 1}, {1, 2}, {1, 4}, {1, 8}};
    const int ns = (int)(sizeof(kSplits) / sizeof(kSplits[0]));
    // Phase 1: the work splits on the default shape; phase 2: the other
    // shapes on the best split (tensor-core batches only).
    std::vector<ms_tune_result> cand;
    for (int c = 0; c < ns; ++c) cand.push_back({kSplits[c][0], kSplits[c][1], 0, 0, 0.0});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MS_CUDA(cudaEventCreate(&e0));
    ms_status st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
    int best = -1;
    for (size_t c = 0; st == MS_OK && c < cand.size(); ++c) {
        st = ms_batch_configure(b, cand[c].batch_split, cand[c].target_mult, cand[c].tc_shape);
        if (st == MS_OK) st = time_graph(b, reps, e0, e1, &cand[c].ms);
        if (st != MS_OK) break;
        if (best < 0 || cand[c].ms < cand[best].ms) best = (int)c;
        if ((int)c == ns - 1 && b->tc)
            for (int sh = 1; sh < ms::kTcShapes; ++sh)
                cand.push_back({cand[best].batch_split, cand[best].target_mult, sh, 0, 0.0});
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != MS_OK) return st;
    const int n = (int)cand.size() < cap ? (int)cand.size() : cap;
    if (results)
        for (int c = 0; c < n; ++c) results[c] = cand[c];
    if (n_results) *n_results = n;
    st = ms_batch_configure(b, cand[best].batch_split, cand[best].target_mult, cand[best].tc_shape);
    if (st == MS_OK) st = ms_batch_run(b, 1);  // leave the batch's outputs from the chosen configuration
    return st;
}

extern "C" ms_status ms_batch_stats(const ms_batch* b, int32_t frame, ms_stats* out) {
    if (!b || !out || frame < -1 || frame >= b->B) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    memset(out, 0, sizeof(*out));
    const int f0 = frame < 0 ? 0 : frame, f1 = frame < 0 ? b->B : frame + 1;
    for (int f = f0; f < f1; ++f) {
        const BState& st = b->h_states[f];
        out->rounds += st.rounds;
        out->n_modes += st.dc.n_kept;
        out->iters_total += st.iters_total;
        out->n_fg += st.dc.n_fg;
        out->seeds += st.seeds_total;
        out->seed_iters += st.dc.seed_iters;
        out->candidates += st.cands_total;
        out->dropped += st.dropped_total;
        out->uncovered += st.dc.n_uncovered;
    }
    out->workspace_bytes = (int64_t)b->ws_bytes;
    if (frame < 0) {
        const unsigned long long* m = reinterpret_cast<const unsigned long long*>(b->h_misc);
        out->launches = (int64_t)b->h_misc[0] * b->body_launches + b->fixed_launches;
        out->band_pairs = (int64_t)m[1];
        out->shift_ms = (double)m[3] * 1e-6;
        out->shift_launches = (int64_t)m[4];
        out->reserved0 = b->h_misc[0];  // loop passes
    }
    return MS_OK;
}

extern "C" ms_status ms_batch_profile(ms_batch* b, int32_t enable) {
    if (!b || enable < 0 || enable > 2) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    if ((enable != 0) == b->prof && (enable == 2) == b->prof_phases) return MS_OK;
    MS_CUDA(cudaStreamSynchronize(b->stream));
    b->prof = enable != 0;
    b->prof_phases = enable == 2;
    return rebuild_graph(b);
}

extern "C" ms_status ms_batch_phase_ms(const ms_batch* b, double* out, int32_t cap, int32_t* n_out) {
    if (!b || cap < 0 || (cap > 0 && !out)) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    const unsigned long long* m = reinterpret_cast<const unsigned long long*>(b->h_misc);
    const int n = cap < kPhases ? cap : kPhases;
    for (int i = 0; i < n; ++i) out[i] = b->prof_phases ? (double)m[8 + i] * 1e-6 : 0.0;
    if (n_out) *n_out = kPhases;
    return MS_OK;
}

extern "C" ms_status ms_batch_modes(const ms_batch* b, int32_t frame, float* h_out, int32_t cap,
                                    int32_t* n_modes_out) {
    if (!b || frame < 0 || frame >= b->B) return set_error(MS_ERR_INVALID_ARG, "bad arguments");
    const int K = b->h_states[frame].dc.n_kept;
    if (n_modes_out) *n_modes_out = K;
    if (!h_out || cap <= 0) return MS_OK;
    if (cap < K) return set_error(MS_ERR_INVALID_ARG, "cap %d < %d modes", cap, K);
    BFrame fr;
    MS_CUDA(cudaMemcpy(&fr, b->frames + frame, sizeof(BFrame), cudaMemcpyDeviceToHost));
    if (K > 0)
        MS_CUDA(cudaMemcpy2D(h_out, sizeof(float) * b->d, b->modes + fr.pix0 * b->Dp, sizeof(float) * b->Dp,
                             sizeof(float) * b->d, (size_t)K, cudaMemcpyDeviceToHost));
    return MS_OK;
}

extern "C" void ms_batch_destroy(ms_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
}
