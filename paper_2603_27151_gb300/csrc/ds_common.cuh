// ds_common.cuh -- internal definitions of the CUDA library (not installed).
//
// Pinned arithmetic: every floating-point step that decides an integer
// (coverage, the depth order, alpha > tau) uses explicit round-to-nearest
// intrinsics (__fmul_rn, __fadd_rn, __fmaf_rn, __fdiv_rn) so that neither the
// compiler's FMA contraction nor approximate division can change a result
// bit.  Gradient arithmetic is free-form FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/diffsoup.h"

namespace ds {

constexpr int kTilePix = 256;        // pixels per tile (one thread each); the
                                     // tile is tile_w x (256 / tile_w) pixels
constexpr int kChunk = 256;          // staging capacity of the tile kernels (triangles per round)
constexpr int kSampleGroup = 4;      // samples sharing one Philox block
constexpr float kGuard = 16384.0f;   // screen-space guard band (pixels)

// Camera as the kernels see it.
struct DevCam {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_z;
};

// Background colour (C-1 channels) of samples where no fragment survives.
struct Bg {
    float c[DS_MAX_CHANNELS];
};

// Per-view parameters, passed by value in the kernel parameter space.
struct ViewDesc {
    DevCam cam;
    int W, H, tiles_x, tiles_y;
    int tile_base;   // global index of this view's first tile
    int item_base;   // first work item (tiles x sample groups)
    uint32_t seed_lo, seed_hi;
    ds_gbuf* gbuf;
    float* color;
    int32_t* n_front;
    const float* grad_color;
    const float* score_w;
    const float* target;   // fused training pass: [C-1][H][W] target image
    // The view's soup and the index of its first set-up record: the call's
    // soup and v * T in a single-soup call; one soup per view in a
    // multi-soup forward (ds_raster_forward_multi), records concatenated.
    const float* s_verts;
    float* s_act;
    float* s_act_a;
    int s_T;
    long long rec_base;
};

struct ViewTable {
    int n;          // views
    int S;          // samples per pixel
    int n_groups;   // ceil(S / 4)
    int n_items;    // total work items
    int tile_w, tile_h;   // tile shape in pixels (8x32, 16x16 or 32x8)
    int chunk;      // triangles staged per round in the tile kernels (<= 256)
    // Optional device-resident cameras (ds_camera[n]) and seeds (uint64[n]):
    // when set they replace v[i].cam and v[i].seed_*, so that a captured
    // CUDA graph can render views chosen after capture.
    const ds_camera* dcam;
    const unsigned long long* dseed;
    ViewDesc v[DS_MAX_VIEWS];
};

// Camera and seed of view v (device table if present, else the parameters).
__device__ __forceinline__ const DevCam& view_cam(const ViewTable& vt, int v) {
    if (vt.dcam) return *reinterpret_cast<const DevCam*>(reinterpret_cast<const char*>(vt.dcam + v) + 8);
    return vt.v[v].cam;
}
__device__ __forceinline__ uint2 view_seed(const ViewTable& vt, int v) {
    if (vt.dseed) {
        const unsigned long long s = vt.dseed[v];
        return make_uint2((uint32_t)s, (uint32_t)(s >> 32));
    }
    return make_uint2(vt.v[v].seed_lo, vt.v[v].seed_hi);
}

// Triangle set-up of one (view, triangle), 64 bytes.  Edge i runs from vertex
// i+1 to vertex i+2; E_i(X, Y) = A_i X + B_i Y + C_i in 1/256-pixel units is
// oriented positive inside, with the fill-rule bias folded into C (a pixel
// centre is covered iff every biased E_i >= 0).  k_i = (1/w_i) / |2 area|.
struct __align__(16) SetupRec {
    int32_t A[3];
    int32_t B[3];
    long long C[3];
    float k[3];
    uint32_t bias;   // bit i set: edge i is not owned (bias 1 folded into C_i)
};
static_assert(sizeof(SetupRec) == 64, "SetupRec must be 64 bytes");

// Continuous (unsnapped) geometry of one (view, triangle) for the vertex
// gradients.  Computed once per backward pass in double-float arithmetic
// (about 2^-46 relative); quantities from which the per-pixel code later
// takes small differences of large values are kept as (hi, lo) float pairs,
// so that the per-pixel arithmetic stays FP32 with compensated steps.
// 208 bytes.
struct __align__(16) GeomRec {
    float2 sx[3], sy[3];   // screen position of each vertex (hi + lo)
    float jx[3][2];        // d sx / d(x_c, z_c): fx / z, -fx x / z^2
    float jy[3][2];        // d sy / d(y_c, z_c): fy / z, -fy y / z^2
    float2 n[3];           // e1 x e2 in camera space (hi + lo)
    float2 m1[3];          // e2 x V0
    float2 m2[3];          // V0 x e1
    float e1[3], e2[3], v0[3];
    float pad;
};
static_assert(sizeof(GeomRec) == 208, "GeomRec must be 208 bytes");

// Soup as the kernels see it.
struct SoupDev {
    const float* verts;   // [T][3][3]
    const float* tex;     // [T][V][C] logits
    float* act;           // [T][V][C] sigmoid(tex)
    float* act_a;         // [T][V]    opacity plane of act
    int T, N, C, V;
};

// ----------------------------------------------------------------- pinned math

// exp(x): Cody-Waite reduction x = k ln2 + r (ln2 = 16-bit head + float
// tail), degree-7 Taylor polynomial of e^r (coefficients 1/n! rounded to
// float) by Horner with fused multiply-adds, scaling by 2^k in two exact
// power-of-two factors.
__device__ __forceinline__ float pow2i(int k) { return __int_as_float((k + 127) << 23); }

__device__ __forceinline__ float pinned_exp(float x) {
    if (x != x) return x;
    if (x >= 0x1.62e430p+6f) return __int_as_float(0x7f800000);
    if (x < -0x1.9fe368p+6f) return 0.0f;
    const float kf = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fmaf_rn(-kf, 0x1.62e400p-1f, x);
    r = __fmaf_rn(-kf, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int k = (int)kf;
    const int k1 = k / 2, k2 = k - k1;
    return __fmul_rn(__fmul_rn(p, pow2i(k1)), pow2i(k2));
}

// Sigmoid of Sec. 3.3, applied per feature vertex before rasterisation.
__device__ __forceinline__ float pinned_sigmoid(float th) {
    return __fdiv_rn(1.0f, __fadd_rn(1.0f, pinned_exp(-th)));
}

// Philox4x32-10 block (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float word_to_tau(uint32_t w) {
    return __fmul_rn((float)(w >> 8), 0x1p-24f);   // exact: 24-bit integer times 2^-24
}

// Mesh-colour cell: the micro-triangle of the N-subdivided triangle that
// holds barycentrics (b1, b2).  Grid vertex (i, j), i + j <= N, sits at
// barycentrics (1 - (i+j)/N, i/N, j/N) and has index j(N+1) - j(j-1)/2 + i.
struct Cell {
    int k0, k1, k2;   // corner texel indices
    float wa, wb;     // value = a0 + wa (a1 - a0) + wb (a2 - a0)
    bool lower;       // lower (i,j),(i+1,j),(i,j+1) or upper micro-triangle
};

__device__ __forceinline__ int texel_index(int N, int i, int j) {
    return j * (N + 1) - ((j * (j - 1)) >> 1) + i;
}

__device__ __forceinline__ Cell find_cell(int N, float b1, float b2) {
    const float Nf = (float)N;
    const float u = __fmul_rn(Nf, b1), v = __fmul_rn(Nf, b2);
    const float fi = floorf(u), fj = floorf(v);
    const int i = fi < 0.0f ? 0 : (fi > (float)(N - 1) ? N - 1 : (int)fi);
    const int jmax = N - 1 - i;
    const int j = fj < 0.0f ? 0 : (fj > (float)jmax ? jmax : (int)fj);
    const float fu = __fsub_rn(u, (float)i), fv = __fsub_rn(v, (float)j);
    Cell c;
    c.lower = (__fadd_rn(fu, fv) <= 1.0f) || (i + j == N - 1);
    if (c.lower) {
        c.k0 = texel_index(N, i, j);
        c.k1 = texel_index(N, i + 1, j);
        c.k2 = texel_index(N, i, j + 1);
        c.wa = fu;
        c.wb = fv;
    } else {
        c.k0 = texel_index(N, i + 1, j + 1);
        c.k1 = texel_index(N, i, j + 1);
        c.k2 = texel_index(N, i + 1, j);
        c.wa = __fsub_rn(1.0f, fu);
        c.wb = __fsub_rn(1.0f, fv);
    }
    return c;
}

__device__ __forceinline__ float interp(float a0, float a1, float a2, float wa, float wb) {
    return __fmaf_rn(wb, __fsub_rn(a2, a0), __fmaf_rn(wa, __fsub_rn(a1, a0), a0));
}

// Pinned perspective-correct fragment from the three oriented (unbiased)
// edge values: q_i = E_i k_i, rho = (q0 + q1) + q2 (inverse depth).
struct Frag {
    float q1, q2, rho;
};

__device__ __forceinline__ Frag make_frag(long long e0, long long e1, long long e2, float k0, float k1, float k2) {
    Frag f;
    const float q0 = __fmul_rn(__ll2float_rn(e0), k0);
    f.q1 = __fmul_rn(__ll2float_rn(e1), k1);
    f.q2 = __fmul_rn(__ll2float_rn(e2), k2);
    f.rho = __fadd_rn(__fadd_rn(q0, f.q1), f.q2);
    return f;
}

// (rho, t) is in front of (rho2, t2): larger inverse depth, then lower index.
__device__ __forceinline__ bool in_front(float rho, int t, float rho2, int t2) {
    return rho > rho2 || (rho == rho2 && t < t2);
}

// Exact covered test and oriented edge values of one set-up record at a
// pixel (int64 arithmetic).
__device__ __forceinline__ bool cover_exact(const SetupRec& r, int px, int py, long long E[3]) {
    const long long X = 256LL * px + 128, Y = 256LL * py + 128;
    bool cov = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long eb = (long long)r.A[i] * X + (long long)r.B[i] * Y + r.C[i];
        cov = cov && (eb >= 0);
        E[i] = eb + ((r.bias >> i) & 1u);
    }
    return cov;
}

// ------------------------------------------------------------ compensated FP32
// TwoSum (Knuth): s + err == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    err = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    return s;
}

// a*b - c*d with one rounding error (Kahan's algorithm with fused multiply-add).
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Dot product of an exact FP32 vector with a (hi, lo) vector, evaluated as if
// in twice the working precision (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005: Dot2 with TwoProduct by FMA).
__device__ __forceinline__ float dot2(float x0, float x1, float x2, const float2* y) {
    float p = __fmul_rn(x0, y[0].x);
    float c = __fadd_rn(__fmaf_rn(x0, y[0].x, -p), __fmul_rn(x0, y[0].y));
    float s = p, t;
    p = __fmul_rn(x1, y[1].x);
    s = two_sum(s, p, t);
    c = __fadd_rn(c, __fadd_rn(t, __fadd_rn(__fmaf_rn(x1, y[1].x, -p), __fmul_rn(x1, y[1].y))));
    p = __fmul_rn(x2, y[2].x);
    s = two_sum(s, p, t);
    c = __fadd_rn(c, __fadd_rn(t, __fadd_rn(__fmaf_rn(x2, y[2].x, -p), __fmul_rn(x2, y[2].y))));
    return __fadd_rn(s, c);
}

// Pinned direction (z = 1) of the camera ray through screen point (x, y)
// (a pixel centre or the midpoint of two; both exact in FP32).
__device__ __forceinline__ void pinned_ray(const DevCam& c, float x, float y, float& dx, float& dy) {
    dx = __fdiv_rn(__fsub_rn(x, c.cx), c.fx);
    dy = __fdiv_rn(__fsub_rn(y, c.cy), c.fy);
}

__device__ __forceinline__ SetupRec load_rec(const SetupRec* p) {
    const int4* q = reinterpret_cast<const int4*>(p);
    SetupRec r;
    int4* d = reinterpret_cast<int4*>(&r);
    d[0] = __ldg(q);
    d[1] = __ldg(q + 1);
    d[2] = __ldg(q + 2);
    d[3] = __ldg(q + 3);
    return r;
}

// Adam (Sec. 3.4; supplementary "Hyperparameters"): the step's scalars, with
// the bias corrections c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t) formed on the host.
struct AdamDev {
    float lr, b1, b2, eps, c1, c2;
};

// One value's Adam step:
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   x <- x - lr (m c1) / (sqrt(v c2) + eps),
// every rounding fixed by an explicit intrinsic, so that each kernel that
// applies it (the optimiser step, the fused gradient finishes) gives the
// same bits for the same gradient.
__device__ __forceinline__ void adam_apply(float& x, float& m, float& v, float g, const AdamDev& a) {
    m = __fmaf_rn(a.b1, m, __fmul_rn(1.0f - a.b1, g));
    v = __fmaf_rn(a.b2, v, __fmul_rn(1.0f - a.b2, __fmul_rn(g, g)));
    const float u = __fdiv_rn(__fmul_rn(a.lr, __fmul_rn(m, a.c1)), __fadd_rn(__fsqrt_rn(__fmul_rn(v, a.c2)), a.eps));
    x = __fsub_rn(x, u);
}

}  // namespace ds
