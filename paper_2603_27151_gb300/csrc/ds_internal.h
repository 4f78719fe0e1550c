// ds_internal.h -- host-side launchers shared by the library's translation
// units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ds_common.cuh"

namespace ds {

// Pipeline stages timed by the optional profiler (ds_profile_*).
enum Stage {
    kStActivate, kStSetup, kStScan, kStEmit, kStSort, kStRanges,
    kStRasterFwd, kStCount, kStGeom, kStRasterBwd, kStEdgeBwd, kStFinish, kStTrain, kNumStages
};
extern const char* const kStageNames[kNumStages];

// Set the message returned by ds_last_error on this thread.
void report_error(const std::string& msg);

// Argument checks and the view table shared by the forward entry points
// (ds_api.cu): a camera with finite parameters, a non-zero focal length, a
// positive near plane and a resolution in [1, DS_MAX_RESOLUTION]; non-NULL
// view outputs with a 16-byte aligned G-buffer (DS_ERR_INVALID_ARG with the
// message set otherwise); the table of tiles, work items and per-view
// pointers for tiles of tu.tile_w x (256 / tu.tile_w) pixels.
bool finite_cam(const ds_camera& c);
ds_status check_outputs(const ds_view_out* out, int32_t n_views);
void build_table(ViewTable& vt, const ds_tuning& tu, const ds_camera* cams, const uint64_t* seeds, int32_t n_views,
                 int32_t S, const ds_view_out* out, const ds_view_gin* gin);

// Library-wide count of kernel launches (every launch site adds to it).
void note_launches(int n);
long long launches_total();

// Scratch for the multi-level exclusive scan (one sum buffer per level).
struct ScanScratch {
    uint32_t* level[6] = {nullptr};
    uint32_t* level_out[6] = {nullptr};
    int64_t level_n[6] = {0};
    int levels = 0;
};

constexpr int kScanBlock = 4096;    // items per scan block (1024 threads x 4)
constexpr int kSortBlock = 4096;    // keys per radix-sort block (256 threads x 16)

// Number of level buffers (and their sizes) needed to scan n items.
int scan_levels(int64_t n, int64_t sizes[6]);

// out[i] = sum_{j<i} in[j]; *total = sum of all (device).  in != out.
cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                           const ScanScratch& sc, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on bits [0, nbits) with 8-bit
// digits.  The pair count is read on the device from *count; kcap bounds it
// (grid size).  Buffers ping-pong between (k0, v0) and (k1, v1); returns the
// index (0 or 1) of the pair holding the result.
int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                     const uint32_t* count, uint32_t kcap, int nbits, uint32_t* hist,
                     uint32_t* hist_scan, const ScanScratch& sc, cudaStream_t st,
                     cudaError_t* err);

// ---- set-up and binning (ds_setup.cu)
cudaError_t launch_activate(const SoupDev& s, cudaStream_t st);
// The views' soups (ViewDesc s_*, rec_base): one soup for every view, or
// soups[v] for view v (records of the views concatenated in view order);
// view_records = the number of set-up records of the table.
void set_view_soups(ViewTable& vt, const SoupDev& s);
void set_view_soups(ViewTable& vt, const SoupDev* const* soups);
long long view_records(const ViewTable& vt);
// One set-up record (and tile count, tile box, depth key) per (view,
// triangle of the view's soup), at rec_base + triangle.
cudaError_t launch_setup(const ViewTable& vt, SetupRec* recs, uint32_t* counts, int4* tbox, uint32_t* zkeys,
                         cudaStream_t st);
cudaError_t launch_emit(const ViewTable& vt, const SetupRec* recs, const uint32_t* counts, const uint32_t* offs,
                        const int4* tbox, const uint32_t* zkeys, int DB, uint32_t* keys, uint32_t* vals,
                        uint32_t cap, int* status, cudaStream_t st);
cudaError_t launch_tile_ranges(const uint32_t* keys, const uint32_t* count, uint32_t kcap, int DB,
                               uint2* ranges, cudaStream_t st);

// ---- forward rasteriser (ds_raster.cu)
// multi: every view reads its own soup (ViewDesc s_*, rec_base) instead of s
// (s then supplies N, C and V, which the views' soups share).
cudaError_t launch_raster_fwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs,
                              const uint32_t* keys, const uint32_t* vals, const uint2* ranges,
                              int DB, uint32_t mode, const Bg& bg, int* counter, int grid,
                              cudaStream_t st, bool with_loss = false, float scale = 0.f,
                              float* loss = nullptr, bool multi = false);
// mode 0: n_front into the views' n_front buffers; mode 1: add the number of
// covered fragments (one sample) to *total.
cudaError_t launch_raster_count(const ViewTable& vt, const SoupDev& s, const SetupRec* recs,
                                const uint32_t* keys, const uint32_t* vals, const uint2* ranges,
                                int DB, int mode, unsigned long long* total, int* counter,
                                int grid, cudaStream_t st);

// The scalars of Adam step t (t >= 1), bias corrections in FP64 on the host.
AdamDev make_adam(float lr, float b1, float b2, float eps, long long t);

// An Adam update fused into a gradient finish: the texture x and its moments
// m, v (device, the texture's layout) take the step instead of a gradient
// being written.
struct AdamTex {
    float* x;
    float* m;
    float* v;
    AdamDev a;
};

// ---- backward (ds_backward.cu)
cudaError_t launch_geom(const ViewTable& vt, const SoupDev& s, GeomRec* geom, cudaStream_t st);
cudaError_t launch_raster_bwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs,
                              const uint32_t* keys, const uint32_t* vals, const uint2* ranges,
                              int DB, uint32_t flags, const GeomRec* geom, double* acc_tex,
                              double* acc_verts, int* counter, int grid, cudaStream_t st);
// Fused training pass: forward + L2 loss + texture/score/interior gradients.
cudaError_t launch_raster_train(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const uint32_t* keys,
                                const uint32_t* vals, const uint2* ranges, int DB, uint32_t mode, const Bg& bg,
                                float scale, float* loss, uint32_t flags, const GeomRec* geom, double* acc_tex,
                                double* acc_verts, int* counter, int grid, cudaStream_t st);
cudaError_t launch_edge_bwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs,
                            const GeomRec* geom, double* acc_verts, int* counter, int grid,
                            cudaStream_t st);
// out[i] = (overwrite ? 0 : out[i]) + acc[i] (FP64 accumulators into FP32 gradients)
cudaError_t launch_grad_finish(const double* acc, float* out, long long n, bool overwrite,
                               cudaStream_t st);
// The texture finish with Adam fused: g = (float) acc[i] is the step's
// gradient of value i, applied to adam.x/m/v (no gradient is written).
cudaError_t launch_grad_finish_adam(const double* acc, const AdamTex& adam, long long n, cudaStream_t st);

// Multi-resolution grids (levels r_min..r_max, level R = [T][V_R][C], stored
// one after the other).  Composition of the finest grid's logits (act: the
// sigmoid activation, with the planar opacity copy if act_a is set), its adjoint
// from the FP64 gradient of the finest grid, and level resampling.
size_t level_floats(int T, int r_min, int r_max, int C);
cudaError_t launch_compose(const float* levels, int T, int r_min, int r_max, int C, float* out, bool act,
                           float* act_a, cudaStream_t st);
cudaError_t launch_restrict(const double* fine, int T, int r_min, int r_max, int C, float* out, bool overwrite,
                            cudaStream_t st);
// The adjoint with Adam fused: each level value's gradient is applied to
// adam.x/m/v (the levels' layout) instead of being written.
cudaError_t launch_restrict_adam(const double* fine, int T, int r_min, int r_max, int C, const AdamTex& adam,
                                 cudaStream_t st);
cudaError_t launch_resample(const float* src, int T, int r_src, int C, float* dst, int r_dst, cudaStream_t st);

// Adaptive control of primitives (ds_adapt.cu).
cudaError_t launch_coverage(const int4* const* gbufs, const long long* n, int n_views, int T, int* counts,
                            cudaStream_t st);
cudaError_t launch_edge_ratios(const float* verts, int T, const ds_camera* cams, int n_views, float* out,
                               cudaStream_t st);
cudaError_t launch_rebuild(const float* verts, const float* tex, int T, const int* grid_ns, int n_levels, int C,
                           const int* plan_dev, int n_out, float* verts_out, float* tex_out, cudaStream_t st);
int adapt_plan(const int32_t* counts, const float* ratios, int T, float threshold, long long budget, int32_t* plan);
int adapt_plan_fill(const int32_t* counts, const float* ratios, int T, long long target, int32_t* plan);

// Adam / VectorAdam step (ds_optim.cu): dim consecutive values share one
// second moment; t is the 1-based step count.
cudaError_t launch_adam(float* x, const float* g, float* m, float* v, long long n, int dim, float lr, float b1,
                        float b2, float eps, long long t, cudaStream_t st);

// lambda L1 + (1 - lambda) SSIM loss with its upstream gradients (ds_ssim.cu).
cudaError_t launch_loss_l1_ssim(int n_views, int S, int Co, const int* hw, const float* const* colors,
                                const float* const* targets, float* const* grad_colors, float* const* score_ws,
                                float lambda, float scale, float* loss, cudaStream_t st);

// One view of the deferred shading pass: feat [S][7][H][W], rgb [S][3][H][W],
// grad_rgb [S][3][H][W], grad_feat [S][7][H][W] (may be null), the pinhole
// intrinsics and the world-to-camera rotation (row-major).
struct ShadeView {
    const float* feat;
    float* rgb;
    const float* grad_rgb;
    float* grad_feat;
    int W, H, HW, blk0;
    float fx, fy, cx, cy;
    float R[9];
};
cudaError_t launch_shade_fwd(const ShadeView* views, int n, int S, const float* params, cudaStream_t st);
// The same forward on the tensor cores (tcgen05, TF32 split into hi + lo);
// a timed-out wait for the MMAs sets bit 1 of *status (device).  no_mma:
// the MMAs are never issued, so every wait runs out (tests the bounded wait).
cudaError_t launch_shade_fwd_tc(const ShadeView* views, int n, int S, const float* params, int* status,
                                cudaStream_t st, bool no_mma = false);
// Backward: writes one partial of the 595 parameter gradients per CTA into
// `partial` (shade_partial_floats(grid) floats) and, if grad_params is set,
// reduces them into it.
cudaError_t launch_shade_bwd(const ShadeView* views, int n, int S, const float* params, bool overwrite,
                             float* partial, int grid, float* grad_params, cudaStream_t st);
int shade_bwd_grid();
size_t shade_partial_floats(int grid);

// Persistent-grid size for the tile kernels on this device.
int persistent_grid(int n_items, int blocks_per_sm);

// Persistent grid of a tile kernel: every CTA the device can keep resident
// (SM count x occupancy of `kernel` at 256 threads), at most n_items.  A
// positive `grid` from the caller is used as given.
template <class Kernel>
inline int resident_grid(Kernel kernel, int n_items, int grid, size_t dyn_smem = 0) {
    if (grid > 0) return grid;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 256, dyn_smem) != cudaSuccess || blocks < 1) {
        cudaGetLastError();
        blocks = 1;
    }
    return persistent_grid(n_items, blocks);
}

}  // namespace ds
