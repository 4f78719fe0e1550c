// ds_tune.cu -- autotuner of the tile kernels' launch parameters (host code
// over the public entry points).
//
// Coordinate search: starting from the context's current tuning, each knob
// in turn (tile shape, depth bits of the bin key, staging chunk, CTAs per
// SM) takes every candidate value with the others fixed; the fastest value
// is kept before the next knob.  A candidate's time is the median over
// `reps` timed repetitions (after one untimed run) of the forward pass, plus
// the backward pass when upstream gradients are given (or of the fused
// training pass when loss views are given), measured with CUDA events on the
// caller's stream.  Every candidate computes the same result
// (the tuning changes only the work decomposition), so the outputs of the
// last run are valid for the chosen tuning.
#include <algorithm>
#include <vector>

#include "ds_internal.h"

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" ds_status ds_autotune(ds_ctx* c, int32_t soup_id, const ds_camera* cams, const uint64_t* seeds,
                                 int32_t n_views, int32_t S, uint32_t mode, const float* bg, const ds_view_out* out,
                                 const ds_view_gin* gin, const ds_view_loss* lv, float scale, float* grad_verts,
                                 float* grad_tex, int32_t reps, ds_tuning* best, float* best_ms, void* stream) {
    if (!c || !best) {
        ds::report_error("NULL argument");
        return DS_ERR_INVALID_ARG;
    }
    if (reps < 1 || reps > 100) {
        ds::report_error("reps must be in [1, 100]");
        return DS_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ds_tuning cur{};
    ds_status rc = ds_get_tuning(c, &cur);
    if (rc != DS_OK) return rc;
    Timer tm;
    if (!tm.a || !tm.b) {
        ds::report_error("cudaEventCreate failed");
        return DS_ERR_CUDA;
    }
    const uint32_t gflags = DS_G_ALL | DS_REUSE_FORWARD | DS_OVERWRITE;

    auto run = [&](const ds_tuning& t, float* ms) -> ds_status {
        ds_status r = ds_set_tuning(c, &t);
        if (r != DS_OK) return r;
        std::vector<float> times;
        for (int k = 0; k <= reps; ++k) {
            if (cudaEventRecord(tm.a, st) != cudaSuccess) return DS_ERR_CUDA;
            if (lv) {
                r = ds_raster_train_l2(c, soup_id, cams, seeds, n_views, S, mode & 0xffu, bg, out, lv, scale, nullptr,
                                       DS_G_ALL | DS_OVERWRITE, grad_verts, grad_tex, stream);
                if (r != DS_OK) return r;
            } else {
                r = ds_raster_forward(c, soup_id, cams, seeds, n_views, S, mode & 0xffu, bg, out, stream);
                if (r != DS_OK) return r;
            }
            if (gin && !lv) {
                r = ds_raster_backward(c, soup_id, cams, n_views, S, out, gin, gflags, grad_verts, grad_tex, stream);
                if (r != DS_OK) return r;
            }
            if (cudaEventRecord(tm.b, st) != cudaSuccess || cudaEventSynchronize(tm.b) != cudaSuccess) {
                cudaGetLastError();
                ds::report_error("event timing failed");
                return DS_ERR_CUDA;
            }
            float e = 0.f;
            cudaEventElapsedTime(&e, tm.a, tm.b);
            if (k > 0) times.push_back(e);   // the first run sizes buffers
        }
        std::sort(times.begin(), times.end());
        *ms = times[times.size() / 2];
        return DS_OK;
    };

    float cur_ms = 0.f;
    rc = run(cur, &cur_ms);
    if (rc != DS_OK) return rc;
    const int tiles[] = {8, 16, 32};
    const int dbits[] = {-1, 8, 0};
    const int chunks[] = {64, 128, 256};
    const int blocks[] = {0, 2, 3};
    for (int knob = 0; knob < 4; ++knob) {
        const int* vals = knob == 0 ? tiles : knob == 1 ? dbits : knob == 2 ? chunks : blocks;
        for (int i = 0; i < 3; ++i) {
            ds_tuning t = cur;
            int& field = knob == 0 ? t.tile_w : knob == 1 ? t.depth_bits : knob == 2 ? t.chunk : t.blocks_per_sm;
            if (field == vals[i]) continue;
            field = vals[i];
            float ms = 0.f;
            rc = run(t, &ms);
            if (rc != DS_OK) return rc;
            if (ms < cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
    }
    // leave the outputs computed with the chosen tuning
    float ms = 0.f;
    rc = run(cur, &ms);
    if (rc != DS_OK) return rc;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return DS_OK;
}
