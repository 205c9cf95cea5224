// Video form: the frames of one sequence clustered one after another, each as
// its own vector set (Algorithm 2), with the OSOP seed count N carried from
// each frame into the next (Sec. 3.2.4; Sec. 4.3 and Table 3, where N_initial
// matters only for the first frames of a sequence).
//
// Two workspaces alternate. While frame t runs its OSOP rounds on the video's
// stream, frame t+1 is bound to the other workspace on a second stream:
// foreground compaction, normalisation and (BF16 form) the split rows for the
// tensor cores. An event recorded after frame t-1's labelling keeps that bind
// from touching the workspace before frame t-1's last kernel has read it.
// Each frame's results are those of ms_create + ms_set_state(carried N) +
// ms_run on that frame with frame_id = cfg->frame_id + its index in the video.
#include <new>

#include "ms_internal.cuh"

struct ms_video {
    ms_config cfg;
    int64_t max_pixels;
    cudaStream_t stream;     // the caller's stream: OSOP rounds and labels
    cudaStream_t side;       // binds of the next frame
    ms_ctx* ctx[2];
    cudaEvent_t freed[2];    // recorded on `stream` after a frame's last kernel on ctx[i]
    int turn;                // ctx[turn] takes the next frame
    int64_t n_carry;         // N for the next frame
    int64_t frames;          // frames clustered so far
};

using namespace ms;

namespace {

void video_free(ms_video* v) {
    if (!v) return;
    if (v->stream) cudaStreamSynchronize(v->stream);
    if (v->side) {
        cudaStreamSynchronize(v->side);
        cudaStreamDestroy(v->side);
    }
    for (int i = 0; i < 2; ++i) {
        if (v->freed[i]) cudaEventDestroy(v->freed[i]);
        ctx_free(v->ctx[i]);
    }
    delete v;
}

}  // namespace

extern "C" ms_status ms_video_create(const ms_config* cfg, int64_t max_pixels, void* stream, ms_video** out) {
    if (!out) return set_error(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int64_t probe = 0;
    ms_status s = ms_workspace_bytes(cfg, max_pixels, &probe);  // validates cfg and max_pixels
    if (s != MS_OK) return s;
    if (cfg->all_seeds) return set_error(MS_ERR_INVALID_ARG, "the video form runs OSOP (all_seeds must be 0)");
    ms_video* v = new (std::nothrow) ms_video();
    if (!v) return set_error(MS_ERR_OOM, "host allocation failed");
    v->cfg = *cfg;
    v->max_pixels = max_pixels;
    v->stream = (cudaStream_t)stream;
    v->n_carry = cfg->n_initial;
    s = cuda_check(cudaStreamCreateWithFlags(&v->side, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int i = 0; i < 2 && s == MS_OK; ++i) {
        s = cuda_check(cudaEventCreateWithFlags(&v->freed[i], cudaEventDisableTiming), "cudaEventCreate");
        if (s == MS_OK) s = ctx_alloc(cfg, max_pixels, v->stream, &v->ctx[i]);
    }
    if (s != MS_OK) {
        video_free(v);
        return s;
    }
    *out = v;
    return MS_OK;
}

extern "C" ms_status ms_video_run(ms_video* v, int32_t T, const float* const* d_embs, const uint8_t* const* d_masks,
                                  const int64_t* n_pixels, int32_t* const* d_labels, int64_t* h_n_start,
                                  int32_t* h_n_modes) {
    if (!v) return set_error(MS_ERR_INVALID_ARG, "video is NULL");
    if (T < 0 || (T > 0 && (!d_embs || !n_pixels || !d_labels))) return set_error(MS_ERR_INVALID_ARG, "bad frame arrays");
    for (int t = 0; t < T; ++t) {
        if (n_pixels[t] < 0 || n_pixels[t] > v->max_pixels)
            return set_error(MS_ERR_INVALID_ARG, "frame %d: %lld pixels outside 0..%lld", t, (long long)n_pixels[t],
                             (long long)v->max_pixels);
        if (n_pixels[t] > 0 && (!d_embs[t] || !d_labels[t]))
            return set_error(MS_ERR_INVALID_ARG, "frame %d: NULL buffer", t);
    }
    if (T == 0) return MS_OK;
    auto mask_of = [&](int t) -> const uint8_t* { return d_masks ? d_masks[t] : nullptr; };
    // frame 0 binds on the side stream like every later frame; it waits for
    // the workspace's previous frame (an earlier call) to finish
    ms_ctx* first = v->ctx[v->turn];
    MS_CUDA(cudaStreamWaitEvent(v->side, v->freed[v->turn], 0));
    ms_status s = ctx_bind_async(first, d_embs[0], mask_of(0), n_pixels[0], v->side);
    for (int t = 0; t < T && s == MS_OK; ++t) {
        ms_ctx* cur = v->ctx[v->turn];
        const int nxt = v->turn ^ 1;
        const int64_t n_start = v->n_carry;
        s = ctx_bind_finish(cur, v->side, v->cfg.frame_id + (uint64_t)v->frames, n_start);
        if (s != MS_OK) break;
        cur->stream = v->stream;
        if (t + 1 < T) {
            // bind frame t+1 to the other workspace while frame t clusters
            s = cuda_check(cudaStreamWaitEvent(v->side, v->freed[nxt], 0), "cudaStreamWaitEvent");
            if (s == MS_OK) s = ctx_bind_async(v->ctx[nxt], d_embs[t + 1], mask_of(t + 1), n_pixels[t + 1], v->side);
            if (s != MS_OK) break;
        }
        int32_t k = 0;
        s = ms_run(cur, d_labels[t], nullptr, 0, &k);
        if (s != MS_OK) break;
        s = cuda_check(cudaEventRecord(v->freed[v->turn], v->stream), "cudaEventRecord");
        if (s != MS_OK) break;
        v->n_carry = v->cfg.video_restart ? v->cfg.n_initial : carried_n(cur);
        if (h_n_start) h_n_start[t] = n_start;
        if (h_n_modes) h_n_modes[t] = k;
        v->frames += 1;
        v->turn = nxt;
    }
    if (s != MS_OK) {
        // leave both streams idle so the video (or its destruction) can continue
        cudaStreamSynchronize(v->side);
        cudaStreamSynchronize(v->stream);
    }
    return s;
}

extern "C" ms_status ms_video_state(const ms_video* v, int64_t* n_carry_out, int64_t* frames_out) {
    if (!v) return set_error(MS_ERR_INVALID_ARG, "video is NULL");
    if (n_carry_out) *n_carry_out = v->n_carry;
    if (frames_out) *frames_out = v->frames;
    return MS_OK;
}

extern "C" ms_status ms_video_stats(const ms_video* v, int32_t which, ms_stats* out) {
    if (!v || !out || (which != 0 && which != 1)) return set_error(MS_ERR_INVALID_ARG, "bad argument");
    // which = 0: the last frame clustered; 1: the one before it
    const int i = v->turn ^ 1 ^ which;
    return ms_stats_get(v->ctx[i], out);
}

extern "C" void ms_video_destroy(ms_video* v) { video_free(v); }
