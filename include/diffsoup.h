/*
 * diffsoup.h -- C ABI of the GB300 (sm_103a) library for the differentiable,
 * stochastically opacity-masked rasterisation of a textured triangle soup
 * (DiffSoup, arXiv 2603.27151) and its gradient.
 *
 * Conventions shared by every entry point
 *  - Pointers are DEVICE pointers unless the comment says "host".
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream) unless it says otherwise, and returns a
 *    ds_status.  Nothing aborts and no C++ exception crosses the ABI; the
 *    message of the last failure on the calling thread is ds_last_error().
 *  - Caller buffers must stay alive until the stream work that uses them has
 *    completed.  Gradients are accumulated (+=): the caller zeroes them.
 *  - Inputs are validated before any launch (sizes, counts, finiteness of
 *    cameras); a violation returns DS_ERR_INVALID_ARG and launches nothing.
 *  - The library owns its scratch memory (triangle set-up records, bin keys,
 *    sort buffers, activations); it grows it with cudaMalloc when a call
 *    needs more and frees it in ds_destroy.
 *
 * Notation (paper Sec. 3): T triangles; per-triangle mesh-colour grid with N
 * subdivisions per edge and V = (N+1)(N+2)/2 feature vertices (Sec. 3.3;
 * R = 5 gives N = 32, V = 561); C channels per feature vertex, the last one
 * being the opacity logit and the first C-1 the colour features (Sec. 3.3,
 * "Neural deferred shading"); S mask samples per pixel (independent draws of
 * the thresholds tau of Eq. 5).
 */
#ifndef DIFFSOUP_H
#define DIFFSOUP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DS_API __attribute__((visibility("default")))
#else
#define DS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ds_status;
typedef struct ds_ctx ds_ctx;   /* opaque library context (one CUDA device) */
#define DS_OK 0
#define DS_ERR_INVALID_ARG (-1) /* bad argument, nothing launched              */
#define DS_ERR_OOM (-2)         /* cudaMalloc of scratch or a soup copy failed */
#define DS_ERR_CUDA (-3)        /* a CUDA runtime call failed                  */
#define DS_ERR_CAPACITY (-4)    /* bin capacity exceeded (no-sync mode only)   */
#define DS_ERR_TIMEOUT (-5)     /* a bounded wait expired                      */
#define DS_ERR_NOT_FOUND (-6)   /* unknown soup id or request ticket           */
#define DS_ERR_BUSY (-7)        /* server queue full                           */

/* Limits (validated). */
#define DS_MAX_VIEWS 64          /* views per forward/backward call           */
#define DS_MAX_RESOLUTION 8192   /* width and height                          */
#define DS_MAX_TRIANGLES (1 << 24)
#define DS_MAX_GRID_N 32
#define DS_MAX_CHANNELS 16
#define DS_MAX_SAMPLES 64

/* Selection modes.  STOCHASTIC: Eq. 5 with tau ~ U[0,1) per fragment, drawn
 * by Philox4x32-10 (Salmon et al., SC'11) from counter (px, py, t, s / 4),
 * key (low, high 32 bits of the view's seed), word s % 4, tau = word>>8 * 2^-24.
 * THRESHOLD_HALF: Eq. 3, tau = 0.5 (the deployment render). */
#define DS_MODE_STOCHASTIC 0u
#define DS_MODE_THRESHOLD_HALF 1u
/* Forward option: skip the host synchronisation that sizes the bin buffers;
 * use the current capacity and report an overflow through ds_ctx_status. */
#define DS_NO_SYNC 0x100u

/* Gradient terms for ds_raster_backward (Algorithm A1 step 2; Sec. 3.2). */
#define DS_G_TEX 1u       /* 2(a): colour gradient of the selected fragment  */
#define DS_G_SCORE 2u     /* 2(b) with Eq. 9: opacity score gradient         */
#define DS_G_INTERIOR 4u  /* first term of Eq. 8 for the vertices            */
#define DS_G_EDGE 8u      /* edge gradients on all adjacent pixel pairs      */
#define DS_G_ALL 15u
/* The soup and cameras are the ones of the last ds_raster_forward on this
 * context and have not changed: reuse its set-up, bins and activations. */
#define DS_REUSE_FORWARD 0x100u
/* Overwrite instead of accumulate: zero grad_tex / grad_verts first
 * (cudaMemsetAsync on the stream). */
#define DS_OVERWRITE 0x200u

/* Soup upload flags. */
#define DS_COPY 0u    /* the library copies verts/tex and owns the copy       */
#define DS_BORROW 1u  /* the library keeps the caller's pointers (training)   */
#define DS_STATIC 2u  /* contents never change after upload: the sigmoid
                         activation is computed once and reused (serving)   */

/* Pinhole camera.  World -> camera: x_c = R x + t (R row-major); +z forward,
 * +x right, +y down; pixel (px, py) has its centre at (px + 0.5, py + 0.5);
 * screen x = fx * x_c / z_c + cx.  A triangle with a vertex at z_c <= near_z
 * is not drawn in that view. */
typedef struct ds_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_z;
} ds_camera;

/* One G-buffer texel (Algorithm A1 step 1: the stored fragment f*): selected
 * triangle (-1 = background), its barycentrics (b1, b2) -- weights of
 * vertices 1 and 2, perspective-correct -- and its view-space depth D
 * (+inf for the background). 16 bytes, stored as [S][H][W]. */
typedef struct ds_gbuf {
    int32_t tri_id;
    float b1, b2;
    float depth;
} ds_gbuf;

/* Per-view outputs of the forward pass. */
typedef struct ds_view_out {
    ds_gbuf* gbuf;     /* [S][H][W]                                          */
    float* color;      /* [S][C-1][H][W] decoded colour features, planar     */
    int32_t* n_front;  /* [S][H][W] or NULL: covered fragments in front of
                          the selected one (all covered ones if background)  */
} ds_view_out;

/* Per-view upstream gradients for the backward pass. */
typedef struct ds_view_gin {
    const float* grad_color;  /* [S][C-1][H][W]  dL/dC of every sample       */
    const float* score_w;     /* [S][H][W] or NULL: the per-sample loss value
                                 that multiplies the score of Eq. 9 (the
                                 L(C) of Algorithm A1 2(b)); NULL = zero     */
} ds_view_gin;

/* Library version (major * 10000 + minor * 100 + patch). Never fails. */
DS_API int32_t ds_version(void);

/* Message of the last failing call on this thread ("" if none). Host string
 * owned by the library, valid until the next call on this thread. */
DS_API const char* ds_last_error(void);

/* Create a context on CUDA device `device`.  Allocates nothing on the device
 * until a call needs scratch.  Errors: DS_ERR_INVALID_ARG (bad device),
 * DS_ERR_CUDA. */
DS_API ds_status ds_create(ds_ctx** out, int32_t device);

/* Destroy a context: waits for its work, frees its scratch and owned soups. */
DS_API void ds_destroy(ds_ctx* ctx);

/* Register a triangle soup (Sec. 3.1, "Triangle soup representation").
 *  verts: [T][3][3] float, vertex positions in world space.
 *  tex:   [T][V][C] float texture logits (the accumulated finest grid before
 *         the sigmoid of Sec. 3.3); channel C-1 is opacity.
 *  grid_n = N in [1, 32]; C in [2, 16]; T in [1, 2^24).
 *  flags: DS_COPY (asynchronous device-to-device copy on `stream` into
 *  library memory) or DS_BORROW (pointers kept; the caller keeps them valid
 *  and may change their contents between calls), optionally | DS_STATIC
 *  (the contents never change: activations are computed once).
 *  On success *soup_id receives a handle >= 0. */
DS_API ds_status ds_soup_upload(ds_ctx* ctx, const float* verts, const float* tex, int32_t T,
                         int32_t grid_n, int32_t C, uint32_t flags, int32_t* soup_id,
                         void* stream);

/* Release a soup (waits for the device, frees an owned copy). */
DS_API ds_status ds_soup_free(ds_ctx* ctx, int32_t soup_id);

/* Multi-resolution feature grids (Sec. 3.3, multi-resolution mesh colours).
 * Level R carries a mesh-colour grid with 2^R subdivisions per edge, V_R =
 * (2^R+1)(2^R+2)/2 feature vertices (level 0: the three triangle vertices).
 * tex_levels holds levels r_min..r_max one after the other, level R as
 * [T][V_R][C] logits.  The soup renders the finest grid (grid_n = 2^r_max)
 * whose logits are the sum over the levels of each level interpolated at the
 * finest grid's vertices (barycentric interpolation in the level's
 * micro-triangles), accumulated coarse to fine in FP32: z_(r_min) = level
 * r_min, z_R = P(z_(R-1)) + level R, with P the 2x prolongation (a vertex
 * that coincides with a coarser one takes its value, an edge midpoint
 * fmaf(0.5, z_q - z_p, z_p), p the endpoint of lower index); the sigmoid
 * follows (the composition runs inside the activation step).  Every other call treats the soup like one registered
 * with ds_soup_upload(grid_n = 2^r_max), except that grad_tex of the
 * backward passes has the layout of tex_levels: the gradient of each level
 * (the adjoint of the composition runs inside the gradient finish step).
 * 0 <= r_min <= r_max, 2^r_max <= DS_MAX_GRID_N.  Flags as ds_soup_upload. */
DS_API ds_status ds_soup_upload_levels(ds_ctx* ctx, const float* verts, const float* tex_levels, int32_t T,
                                       int32_t r_min, int32_t r_max, int32_t C, uint32_t flags, int32_t* soup_id,
                                       void* stream);

/* The composed finest grid [T][V_{r_max}][C] of tex_levels (as above):
 * logits, or their sigmoid if activate != 0 (the texture kept after
 * training, Sec. 3.3).  No context; allocates nothing. */
DS_API ds_status ds_levels_compose(const float* tex_levels, int32_t T, int32_t r_min, int32_t r_max, int32_t C,
                                   int32_t activate, float* out, void* stream);

/* One level's grid src [T][V_{r_src}][C] sampled at the vertices of level
 * r_dst: dst [T][V_{r_dst}][C] (a vertex that coincides with a src vertex
 * takes its value, else barycentric interpolation in src's micro-triangle).
 * The coarse-to-fine switch of the supplementary material copies the coarse
 * stage's features to the new r_min level this way.  No context; allocates
 * nothing. */
DS_API ds_status ds_levels_resample(const float* src, int32_t T, int32_t r_src, int32_t C, float* dst,
                                    int32_t r_dst, void* stream);

/* Forward pass (Eq. 5; Algorithm A1 step 1) for n_views views of one soup:
 * sigmoid activation of the texture (Sec. 3.3), triangle set-up, radix-sorted
 * binning of triangles into tiles of 256 pixels (8x32, 16x16 or 32x8: a
 * launch parameter of the context, see ds_set_tuning), then per pixel and sample the
 * foremost covered fragment whose interpolated opacity exceeds its threshold
 * (fixed tie-break: larger perspective-correct inverse depth first, then the
 * lower triangle index), and the mesh-colour decode of its C-1 colour
 * channels (background colour `bg` when nothing survives).
 *  cams  (host) [n_views]; seeds (host) [n_views]; bg (host) [C-1];
 *  out   (host) [n_views] per-view output pointers (device buffers).
 *  mode: DS_MODE_STOCHASTIC or DS_MODE_THRESHOLD_HALF, optionally | DS_NO_SYNC.
 * Without DS_NO_SYNC the call synchronises `stream` once to size its bin
 * buffers. */
DS_API ds_status ds_raster_forward(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                            const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode,
                            const float* bg, const ds_view_out* out, void* stream);

/* Backward pass (Algorithm A1 step 2, Eq. 8-9, Sec. 3.2) for the G-buffers
 * and colours `fwd` produced by ds_raster_forward with the same soup,
 * cameras and S.  Accumulates (+=) into
 *   grad_tex   [T][V][C] (gradient w.r.t. the logits) and
 *   grad_verts [T][3][3] (world space), either may be NULL,
 * the terms selected by grad_flags (DS_G_*), optionally | DS_REUSE_FORWARD.
 * Score term: for every sample with weight w = score_w, +w/alpha for the
 * selected fragment and -w/(1-alpha) for every covered fragment in front of
 * it (all covered fragments when the sample shows the background), chained
 * to the opacity logits.  Contributions are summed in FP64 scratch with
 * atomics (summation order varies from run to run) and added to the FP32
 * outputs at the end. */
DS_API ds_status ds_raster_backward(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                             int32_t n_views, int32_t S, const ds_view_out* fwd,
                             const ds_view_gin* gin, uint32_t grad_flags, float* grad_verts,
                             float* grad_tex, void* stream);

/* Adam state of a texture for ds_raster_backward_adam (Sec. 3.4; the
 * supplementary "Hyperparameters" train the texture features with Adam):
 *  m, v  (device) first and second moments, float32, one value per texture
 *        value in the soup's texture layout (levels back to back for a level
 *        soup), owned by the caller;
 *  n     the number of floats in each of m and v: must equal the soup's
 *        texture size (T V C, or the levels' total), else DS_ERR_INVALID_ARG;
 *  lr, beta1 in [0, 1), beta2 in [0, 1), eps >= 0; step t >= 1 (the bias
 *  corrections use 1 - beta^t). */
typedef struct ds_adam_args {
    float* m;
    float* v;
    int64_t n;
    float lr, beta1, beta2, eps;
    int64_t step;
} ds_adam_args;

/* ds_raster_backward with one Adam step of the soup's texture fused into
 * the gradient finish: the texture gradient of this call (the terms of
 * grad_flags, as ds_raster_backward would write with DS_OVERWRITE) is never
 * written; each value's gradient, rounded to FP32 exactly as written there,
 * updates the soup's texture in place together with m and v, with the
 * roundings of ds_adam_step at dim = 1, so that the result is bit-identical
 * to ds_raster_backward (DS_OVERWRITE) followed by ds_adam_step.  For a level
 * soup the update applies to the levels (in the adjoint's epilogue).  The
 * texture updated is the soup's own storage: the caller's tensor for a soup
 * uploaded with borrowing, the context's copy otherwise.  grad_verts as in
 * ds_raster_backward.  DS_ERR_INVALID_ARG for a NULL tex_adam, m or v, bad
 * hyperparameters, step < 1, no DS_G_TEX or DS_G_SCORE in grad_flags, a
 * static soup (DS_STATIC), or, for a level soup, C not a multiple of 4 or a
 * texture, m or v not 16-byte aligned (the update moves four values per
 * access). */
DS_API ds_status ds_raster_backward_adam(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                                         int32_t n_views, int32_t S, const ds_view_out* fwd,
                                         const ds_view_gin* gin, uint32_t grad_flags, float* grad_verts,
                                         const ds_adam_args* tex_adam, void* stream);

/* The two passes with the cameras and seeds in DEVICE memory (ds_camera[n]
 * and uint64[n], read by the kernels), the view sizes on the host
 * (wh [n][2] = width, height).  Otherwise as ds_raster_forward /
 * ds_raster_backward.  For a training step whose views are chosen at run time
 * inside a captured CUDA graph: the graph records the pointers, the caller
 * rewrites the camera and seed arrays before each replay.  The device values
 * are not validated (finite, fx, fy != 0, near_z > 0 are the caller's
 * contract).  DS_REUSE_FORWARD reuses the plan of the last device-camera
 * forward on this context with the same soup and view sizes. */
DS_API ds_status ds_raster_forward_devcam(ds_ctx* ctx, int32_t soup_id, const int32_t* wh,
                                          const ds_camera* cams, const uint64_t* seeds,
                                          int32_t n_views, int32_t S, uint32_t mode, const float* bg,
                                          const ds_view_out* out, void* stream);
DS_API ds_status ds_raster_backward_devcam(ds_ctx* ctx, int32_t soup_id, const int32_t* wh,
                                           const ds_camera* cams, int32_t n_views, int32_t S,
                                           const ds_view_out* fwd, const ds_view_gin* gin,
                                           uint32_t grad_flags, float* grad_verts, float* grad_tex,
                                           void* stream);

/* Loss inputs and outputs of one view for the fused training pass. */
typedef struct ds_view_loss {
    const float* target;  /* [C-1][H][W] target image                             */
    float* grad_color;    /* [S][C-1][H][W] written: dL/dC = 2 scale (C - target)  */
    float* score_w;       /* [S][H][W] written, or NULL: scale * l per sample       */
} ds_view_loss;

/* Fused training pass: ds_raster_forward, ds_loss_l2 and ds_raster_backward
 * in one call, with the forward, the per-pixel L2 loss and the texture,
 * score and interior gradients (Eq. 5; Algorithm A1 steps 1 and 2; first term
 * of Eq. 8) computed by one kernel per tile and sample group, and the edge
 * gradients (Sec. 3.2) by a second launch.  Results are those of the three
 * calls in sequence with DS_OVERWRITE semantics selected by grad_flags
 * (DS_G_* | optional DS_OVERWRITE): out receives the G-buffers and colours
 * (n_front must be NULL), lv[v] the upstream gradients and score weights,
 * *loss (device float, accumulated, may be NULL) scale * sum of l, and
 * grad_verts / grad_tex the gradients (either may be NULL).  The plan stays
 * valid for a later ds_raster_backward with DS_REUSE_FORWARD.  mode may
 * include DS_NO_SYNC.  The second form takes device cameras and seeds as
 * ds_raster_forward_devcam. */
DS_API ds_status ds_raster_train_l2(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                                    const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode,
                                    const float* bg, const ds_view_out* out, const ds_view_loss* lv,
                                    float scale, float* loss, uint32_t grad_flags, float* grad_verts,
                                    float* grad_tex, void* stream);
DS_API ds_status ds_raster_train_l2_devcam(ds_ctx* ctx, int32_t soup_id, const int32_t* wh,
                                           const ds_camera* cams, const uint64_t* seeds,
                                           int32_t n_views, int32_t S, uint32_t mode, const float* bg,
                                           const ds_view_out* out, const ds_view_loss* lv, float scale,
                                           float* loss, uint32_t grad_flags, float* grad_verts,
                                           float* grad_tex, void* stream);

/* Grow the context's bin buffers to hold `pairs` (tile, triangle) pairs, so
 * that DS_NO_SYNC forwards (which never allocate or synchronise) have that
 * capacity.  Synchronous (may call cudaMalloc). */
DS_API ds_status ds_reserve(ds_ctx* ctx, int64_t pairs);

/* Per-pixel L2 photometric loss of the rendered colour features against
 * target images, with its upstream gradients for ds_raster_backward (the
 * paper minimises L1 + SSIM, Eq. 10; the estimator of Eq. 8 takes any
 * per-pixel loss).  For every view v, sample s and pixel p:
 *   l = sum_c (color - target)^2,  grad_color = 2 * scale * (color - target),
 *   score_w = scale * l,            *loss += scale * sum of l over everything.
 *  hw (host) [n_views][2] = (width, height); colors, targets, grad_colors,
 *  score_ws (host arrays of device pointers): color [S][C-1][H][W], target
 *  [C-1][H][W], grad_color [S][C-1][H][W] (may be NULL), score_w [S][H][W]
 *  (may be NULL); loss: one device float, accumulated (may be NULL).
 *  scale is usually 1/S (the mean over mask samples).  Allocates nothing. */
DS_API ds_status ds_loss_l2(int32_t n_views, int32_t S, int32_t C, const int32_t* hw,
                            const float* const* colors, const float* const* targets,
                            float* const* grad_colors, float* const* score_ws, float scale,
                            float* loss, void* stream);

/* Adaptive control of primitives (Sec. 3.4): edges whose view-space length
 * exceeds a fraction of the image height are split; triangles with low pixel
 * coverage are pruned to hold a triangle budget.  Four calls make one round:
 *
 * ds_coverage_count: pixel coverage per triangle -- the number of
 *  pixel-samples of the given G-buffers (host array of device pointers, each
 *  [S][H][W] as written by a forward pass; hw host [n_views][2] = (W, H))
 *  whose selected triangle is t -- added to counts (device int32 [T]; ids
 *  outside [0, T) are ignored).  Allocates nothing. */
DS_API ds_status ds_coverage_count(const ds_gbuf* const* gbufs, const int32_t* hw, int32_t n_views, int32_t S,
                                   int32_t T, int32_t* counts, void* stream);

/* ds_edge_ratios: for every triangle and edge e = (v_e, v_(e+1)%3), the
 *  largest over the views (host cams, the paper samples 20 training views) of
 *  the edge's projected length divided by the image height, over the views
 *  where all three vertices lie in front of near_z and the projected
 *  triangle's bounding box meets the image; 0 if there is none.  verts
 *  device [T][3][3]; ratios device [T][3] (written).  FP32 with the
 *  projection of the set-up (x_c = R v + t by fused multiply-adds, screen =
 *  f x/z + c), length sqrt(dx^2 + dy^2).  Allocates nothing. */
DS_API ds_status ds_edge_ratios(const float* verts, int32_t T, const ds_camera* cams, int32_t n_views,
                                float* ratios, void* stream);

/* ds_adapt_plan (host only, no device work): one round's plan from host
 *  copies of counts [T] and ratios [T][3].  Every triangle whose largest
 *  ratio exceeds `threshold` (the paper: 1/5) splits that edge (the first of
 *  equal maxima); then, if budget >= 0 and the count after the splits
 *  exceeds it, triangles are removed in order of increasing coverage (lower
 *  index first among equal counts; removing a splitting triangle removes
 *  both children) until it does not.  plan (host, capacity 2T) receives one
 *  code per output triangle: parent << 3 | op, op 0 = copy, op 1 + 2e + c =
 *  child c of splitting edge e; survivors in index order, children in place
 *  of their parent.  *n_out = the new triangle count. */
DS_API ds_status ds_adapt_plan(const int32_t* counts, const float* ratios, int32_t T, float threshold,
                               int64_t budget, int32_t* plan, int32_t* n_out);

/* ds_adapt_plan_fill (host only): one round of the random-initialisation
 *  procedure (supplementary "Random Triangle Soup Initialization"): the
 *  triangles with no coverage in any training image (counts[t] <= 0) are
 *  removed; then, while fewer than `target` remain, the survivors whose
 *  longest edge has the largest ratio (lower index first among equal ones)
 *  split that edge, each at most once per round (repeat rounds, re-measuring,
 *  to grow further).  Plan codes and capacity as ds_adapt_plan. */
DS_API ds_status ds_adapt_plan_fill(const int32_t* counts, const float* ratios, int32_t T, int64_t target,
                                    int32_t* plan, int32_t* n_out);

/* ds_soup_rebuild: the soup after a plan.  verts [T][3][3] and tex (levels
 *  back to back, level l = [T][V_l][C] with V_l = (N_l+1)(N_l+2)/2, N_l =
 *  grid_ns[l] (host [n_levels]); one level for a plain soup) -> verts_out
 *  [n_out][3][3] and tex_out (same level layout with n_out triangles).  A
 *  child of edge e = (a, b) with opposite vertex o is (a, m, o) (c = 0) or
 *  (m, b, o) (c = 1), m = (a + b) * 0.5 in FP32 (the parent's winding); each
 *  level of its texture is the parent's level sampled at the child's grid
 *  vertices mapped into the parent (a point on a parent grid vertex takes its
 *  value, any other point -- a micro-edge midpoint -- is interpolated as the
 *  decode does).  plan is host memory, validated before any launch (parent in
 *  [0, T), op <= 6).  Uses a context scratch for the plan; returns with the
 *  rebuild complete (synchronises `stream`). */
DS_API ds_status ds_soup_rebuild(ds_ctx* ctx, const float* verts, const float* tex, int32_t T,
                                 const int32_t* grid_ns, int32_t n_levels, int32_t C, const int32_t* plan,
                                 int32_t n_out, float* verts_out, float* tex_out, void* stream);

/* One optimiser step (Sec. 3.4: VectorAdam for vertex positions, Adam for
 * everything else; supplementary "Hyperparameters": beta1 0.9, beta2 0.999,
 * eps 1e-8).  A vector is `dim` consecutive values of params (dim = 3 for
 * vertex positions [T][3][3]: VectorAdam; dim = 1: Adam) sharing one second
 * moment from the squared norm of its gradient:
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2)|g|^2,
 *   params <- params - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * params, grads, m: device [n]; v: device [n / dim]; step: 1-based count
 * (the caller keeps it; the bias corrections are computed on the host).
 * dim in [1, 4] dividing n.  FP32.  Allocates nothing. */
DS_API ds_status ds_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int32_t dim,
                              float lr, float beta1, float beta2, float eps, int64_t step, void* stream);

/* Neural deferred shading (Sec. 3.3, "Neural deferred shading"; supplementary
 * "MLP Architecture"): the per-pixel shading pass that turns the rasterised
 * colour features (C = 8: 7 features + opacity) into RGB.  For every view v,
 * mask sample s and pixel p the input is the 7 features f concatenated with
 * the real SH basis of degree <= 2 of the view direction (9 values: the unit
 * world-space ray R^T((x+0.5-cx)/fx, (y+0.5-cy)/fy, 1) normalised; the usual
 * graphics order and signs); a shared MLP 16 -> 16 (ReLU) -> 16 (ReLU) -> 3
 * (sigmoid) gives o, and the first four features, read as RGBA, are blended
 * with it:  rgb = A * f[0:3] + (1 - A) * o,  A = f[3].
 *  params: device [DS_SHADE_N_PARAMS] FP32 = W1 [16][16] (row = output; input
 *  columns 0..6 features, 7..15 SH), b1 [16], W2 [16][16], b2 [16], W3 [3][16],
 *  b3 [3].  cams (host [n_views]): only the size, intrinsics and R are read.
 *  feats, rgbs (host arrays of device pointers): feat [S][7][H][W], rgb
 *  [S][3][H][W] (written).  n_views = 0 is a no-op.  FP32 arithmetic on the
 *  CUDA cores.  Allocates nothing. */
#define DS_SHADE_N_PARAMS 595
DS_API ds_status ds_shade_forward(ds_ctx* ctx, int32_t n_views, int32_t S, const ds_camera* cams,
                                  const float* params, const float* const* feats, float* const* rgbs,
                                  void* stream);

/* Gradients of the deferred shading pass for the upstream gradients grad_rgb
 * [S][3][H][W] (host array of device pointers): grad_feat [S][7][H][W] (host
 * array of device pointers, or NULL for none) and grad_params
 * [DS_SHADE_N_PARAMS] (device, or NULL).  Both are accumulated (+=) unless
 * flags has DS_OVERWRITE (then written).  The parameter gradient is reduced
 * in a fixed order (one FP32 partial per CTA, summed in FP64): the result is
 * bit-reproducible for the same inputs on the same device.  Uses a context
 * scratch of about 1.5 MiB (grown with cudaMalloc on the first call). */
DS_API ds_status ds_shade_backward(ds_ctx* ctx, int32_t n_views, int32_t S, const ds_camera* cams,
                                   const float* params, const float* const* feats,
                                   const float* const* grad_rgbs, float* const* grad_feats,
                                   float* grad_params, uint32_t flags, void* stream);

/* Which kernel ds_shade_forward runs on this context (no paper counterpart:
 * two implementations of the same forward of Sec. 3.3's MLP):
 *  DS_SHADE_CUDA_CORES: FP32 fused multiply-adds on the CUDA cores;
 *  DS_SHADE_TENSOR_CORES: the three layers as tcgen05 MMAs of kind::tf32 on
 *    the 5th-generation tensor cores, every operand split into a TF32 high
 *    part and the remainder (x w ~ x_lo w_hi + x_hi w_lo + x_hi w_hi), FP32
 *    accumulation in tensor memory; about FP32 accuracy.  A launch whose wait
 *    for its MMAs runs out (about a second) stops, and the next
 *    ds_ctx_status returns DS_ERR_TIMEOUT.
 *  DS_SHADE_TENSOR_CORES_WAIT_TEST: diagnostic, for testing the bounded
 *    wait on a GPU: the tensor-core kernel with its MMAs never issued, so
 *    that every CTA's wait runs out (twice about 2^31 SM clocks, about 2 s
 *    in all); the output is left unwritten, the tensor memory is released,
 *    the next ds_ctx_status returns DS_ERR_TIMEOUT and the context stays
 *    usable.
 * A new context uses DS_SHADE_TENSOR_CORES (the faster of the two on
 * sm_103a).  Host calls; DS_ERR_INVALID_ARG for another value. */
#define DS_SHADE_CUDA_CORES 0
#define DS_SHADE_TENSOR_CORES 1
#define DS_SHADE_TENSOR_CORES_WAIT_TEST 2
DS_API ds_status ds_set_shade_path(ds_ctx* ctx, int32_t path);
DS_API ds_status ds_get_shade_path(ds_ctx* ctx, int32_t* path);

/* The paper's photometric loss lambda L1 + (1 - lambda) L_SSIM (Eq. 10, Sec.
 * 3.4; lambda = 0.8), per pixel, with its upstream gradients for
 * ds_raster_backward.  SSIM per channel with an 11 x 11 Gaussian window
 * (sigma 1.5, normalised), zero padding outside the image, C1 = 0.01^2,
 * C2 = 0.03^2.  For every view v, sample s and pixel p:
 *   ell = lambda mean_c |color - target| + (1 - lambda)(1 - mean_c ssim_c(p)),
 *   score_w = scale * ell,  *loss += scale * sum of ell over everything,
 *   grad_color = scale * d(sum_p ell_p)/d color  (non-local: the window).
 *  Arguments and layouts as ds_loss_l2 (C counts the opacity channel: C-1
 *  colour channels).  grad_colors, score_ws and loss may be NULL.  FP32; one
 *  fused pass per 32 x 16 tile.  Allocates nothing on the device. */
DS_API ds_status ds_loss_l1_ssim(int32_t n_views, int32_t S, int32_t C, const int32_t* hw,
                                 const float* const* colors, const float* const* targets,
                                 float* const* grad_colors, float* const* score_ws, float lambda, float scale,
                                 float* loss, void* stream);

/* Forward pass of views of different soups in one launch (Eq. 5; Algorithm
 * A1 step 1, as ds_raster_forward): view v renders soup soup_ids[v] (host
 * [n_views]) with camera cams[v] and seed seeds[v]; the set-up records of
 * all views are binned together and the persistent tile kernel serves every
 * view's tiles in one launch, each tile reading its view's soup.  Every
 * output (triangle ids index the view's own soup, barycentrics, depths,
 * colours, n_front) equals that of ds_raster_forward on the view alone: the
 * per-view arithmetic, mask thresholds and tie-breaks are the same.  The
 * soups must share grid_n and C (DS_ERR_INVALID_ARG otherwise).  The paper
 * has no counterpart: this serves the continuous-batching render server,
 * which batches queued requests for different resident soups.  Other
 * arguments, flags and errors as ds_raster_forward; the call leaves no plan
 * that a later ds_raster_backward can reuse. */
DS_API ds_status ds_raster_forward_multi(ds_ctx* ctx, const int32_t* soup_ids, const ds_camera* cams,
                                         const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode,
                                         const float* bg, const ds_view_out* out, void* stream);

/* Forward pass for callers that cannot allocate device memory: the same
 * computation and outputs as ds_raster_forward (Eq. 5, Algorithm A1 step 1),
 * on a soup passed directly (verts [T][3][3], tex [T][V][C] logits, as in
 * ds_soup_upload) instead of a registered one, and with no context.  The
 * paper has no counterpart: this serves embedding.  Some callers cannot call
 * cudaMalloc: engines and plug-in hosts that own every byte of device memory
 * through their own pool, programs under a hard device-memory budget, and
 * real-time loops that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may imply.  This entry point makes no cudaMalloc,
 * cudaFree or other allocating call.  Its scratch is one fixed device array
 * of about 21 MiB inside the library, which every GPU that loads the library
 * holds until the process exits.  Limits (checked before any launch,
 * DS_ERR_INVALID_ARG beyond them): T*V*C <= 2^20 texture values,
 * n_views*T <= 65536, at most 65536 16x16 tiles over all views.  The number
 * of (tile, triangle) pairs is known only after binning; the call reads it
 * back (one synchronisation of `stream`) and returns DS_ERR_CAPACITY above
 * 524288 pairs; every call therefore synchronises `stream` once.  The
 * first call on each device looks up the array's device address with that
 * device current.  Every
 * call in the process shares the one array and leaves its contents behind
 * (the call clears what must start at zero): calls whose work overlaps on the
 * GPU, from several streams or host threads, race and must be serialised by
 * the caller.  `mode` is DS_MODE_STOCHASTIC or DS_MODE_THRESHOLD_HALF without
 * flag bits (DS_NO_SYNC is rejected).  Inputs and outputs must be device (or
 * managed) memory of the current device, which the call checks with
 * cudaPointerGetAttributes; anything else returns DS_ERR_INVALID_ARG. */
DS_API ds_status ds_raster_forward_noalloc(const float* verts, const float* tex, int32_t T,
                                           int32_t grid_n, int32_t C, const ds_camera* cams,
                                           const uint64_t* seeds, int32_t n_views, int32_t S,
                                           uint32_t mode, const float* bg, const ds_view_out* out,
                                           void* stream);

/* Fragment statistics of Eq. 1 for n_views views: *n_cover_total (host)
 * receives the number of (pixel, covering triangle) pairs summed over the
 * views (|F|, one mask sample).  Synchronises `stream`. */
DS_API ds_status ds_fragment_count(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                            int32_t n_views, int64_t* n_cover_total, void* stream);

/* Sizes of the context's current binning plan (the last forward, backward or
 * fragment count): *pairs = (tile, triangle) pairs after binning, *tiles =
 * tiles (of the context's tile shape) over all views.  Host values; never
 * synchronises. */
DS_API ds_status ds_plan_stats(ds_ctx* ctx, int64_t* pairs, int64_t* tiles);

/* Read and clear the context's device status word (synchronises the
 * context's last stream): DS_ERR_CAPACITY after a DS_NO_SYNC forward whose
 * bins overflowed (its outputs are invalid), else DS_OK. */
DS_API ds_status ds_ctx_status(ds_ctx* ctx);

/* Launch parameters of the tile kernels (no paper counterpart: the work
 * decomposition of Eq. 5 and Algorithm A1; every setting computes the same
 * result).  tile_w: tile width in pixels, 8, 16 or 32 (tiles hold 256 pixels,
 * so 8x32, 16x16 or 32x8).  depth_bits: bits of quantised nearest depth in
 * the bin key that order each tile's list front to back for the early exit,
 * -1 = 16 (or fewer when the tile index needs the bits), 0 = unordered.
 * blocks_per_sm: CTAs per SM of the persistent tile kernels, 0 = each
 * kernel's occupancy limit.  chunk: triangles staged in shared memory per
 * round, a multiple of 32 in [32, 256].  Default {16, -1, 0, 256}. */
typedef struct ds_tuning {
    int32_t tile_w, depth_bits, blocks_per_sm, chunk;
} ds_tuning;

/* Set (validated; DS_ERR_INVALID_ARG otherwise) or read a context's tuning.
 * Setting it invalidates the context's binning plan. */
DS_API ds_status ds_set_tuning(ds_ctx* ctx, const ds_tuning* t);
DS_API ds_status ds_get_tuning(ds_ctx* ctx, ds_tuning* t);

/* Autotune the context's tuning on one workload: coordinate search over tile
 * shape {8x32, 16x16, 32x8}, depth bits {16, 8, 0}, chunk {64, 128, 256} and
 * CTAs per SM {occupancy, 2, 3}, each candidate timed (median of `reps` in
 * [1, 100] after one untimed run) with CUDA events on `stream` over
 * ds_raster_forward (mode) and, when gin is non-NULL, ds_raster_backward with
 * DS_G_ALL | DS_OVERWRITE into grad_verts / grad_tex; or, when lv is
 * non-NULL, over ds_raster_train_l2 with those loss views and scale.
 * Arguments as in those calls.  Synchronises `stream` after every run.
 * Sets the fastest tuning on the context and returns it in *best (host) with its time in *best_ms
 * (host, may be NULL); the outputs hold the results of a final run with it. */
DS_API ds_status ds_autotune(ds_ctx* ctx, int32_t soup_id, const ds_camera* cams,
                             const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode,
                             const float* bg, const ds_view_out* out, const ds_view_gin* gin,
                             const ds_view_loss* lv, float scale, float* grad_verts, float* grad_tex,
                             int32_t reps, ds_tuning* best, float* best_ms, void* stream);

/* ---------------------------------------------------------------------------
 * Render server: continuous batching of single-view forward requests over
 * resident soups (the inference use of Eq. 5 and Eq. 3; the paper measures
 * the rendering speed of the optimised soups, Sec. 4).  One scheduler thread
 * and n_streams workers, each a context with its own CUDA stream.  A free
 * worker takes the oldest queued request and every other queued request with
 * the same mode, background and texture shape (grid_n, C), whatever its soup
 * (up to max_batch views), into one ds_raster_forward_multi launch; requests
 * that arrive while batches run join the next one, and the
 * batches of different workers overlap on the device.  Admission by device
 * memory: a batch is launched only while the scratch estimate of all batches
 * in flight stays within mem_budget bytes (a batch of one request is always
 * admitted when nothing else runs).  Workers launch with DS_NO_SYNC after
 * ds_reserve(reserve_pairs); a batch whose bins overflow is rendered again
 * with synchronised sizing before its requests complete.  A request's output
 * is identical whichever batch it runs in (each view's pixels depend only on
 * its own soup, camera and seed).
 * ------------------------------------------------------------------------- */
typedef struct ds_server ds_server;   /* opaque */

typedef struct ds_request_stats {
    int64_t submit_ns, launch_ns, done_ns; /* steady-clock times (host, ns)         */
    int32_t batch;                         /* views in the launch that served it     */
    int32_t pad;
} ds_request_stats;

/* Create a server on `device`.  n_streams in [1, 32], max_batch in [1, 64],
 * reserve_pairs >= 0 (bin capacity per worker).  Starts the scheduler thread. */
DS_API ds_status ds_server_create(int32_t device, int32_t n_streams, size_t mem_budget,
                                  int32_t max_batch, int64_t reserve_pairs, ds_server** out);

/* Copy a soup (device pointers, layout as ds_soup_upload) into server memory
 * and register it with every worker as immutable (activations computed
 * once).  Synchronous.  *soup_id receives the server's handle. */
DS_API ds_status ds_server_add_soup(ds_server* srv, const float* verts, const float* tex, int32_t T,
                                    int32_t grid_n, int32_t C, int32_t* soup_id);

/* Queue one view for rendering; returns at once with *ticket (host).  cam,
 * bg [C-1] (NULL = zeros) are host values copied into the request; `out`
 * (host struct of device pointers, S = 1) must stay valid until the request
 * completes.  DS_ERR_BUSY when the queue is full or the server stops. */
DS_API ds_status ds_render_request(ds_server* srv, int32_t soup_id, const ds_camera* cam,
                                   uint64_t seed, uint32_t mode, const float* bg,
                                   const ds_view_out* out, uint64_t* ticket);

/* Wait for a request (timeout_ms < 0: no limit).  On return other than
 * DS_ERR_TIMEOUT the ticket is released; `stats` (host, may be NULL)
 * receives its timestamps.  The outputs are complete on the device when this
 * returns DS_OK. */
DS_API ds_status ds_request_wait(ds_server* srv, uint64_t ticket, int32_t timeout_ms,
                                 ds_request_stats* stats);

/* Hold (paused != 0) or resume the launching of queued requests. */
DS_API ds_status ds_server_pause(ds_server* srv, int32_t paused);

/* Cancel queued requests (their waits return DS_ERR_BUSY), let launched
 * batches finish, free everything. */
DS_API ds_status ds_server_destroy(ds_server* srv);

/* Profiling (off by default; no paper counterpart: instrumentation).  While
 * enabled, every pipeline stage that a call on this context launches
 * (activate, setup, scan, emit, sort, ranges, raster_fwd, count, geom,
 * raster_bwd, edge_bwd, finish) is bracketed by two CUDA events recorded on the caller's stream.
 * ds_profile_read waits for those events and returns, for stage index
 * `stage` in [0, ds_profile_stages()), its name (static host string), the
 * number of times it ran and its summed device time in ms since the last
 * ds_profile_reset. */
DS_API ds_status ds_profile_enable(ds_ctx* ctx, int32_t on);
DS_API int32_t ds_profile_stages(void);
DS_API ds_status ds_profile_read(ds_ctx* ctx, int32_t stage, const char** name, int64_t* runs,
                                 double* ms);
DS_API ds_status ds_profile_reset(ds_ctx* ctx);
/* Kernels launched by the library in this process so far (all contexts). */
DS_API int64_t ds_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* DIFFSOUP_H */
