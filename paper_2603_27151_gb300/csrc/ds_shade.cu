// ds_shade.cu -- neural deferred shading (Sec. 3.3 "Neural deferred shading";
// supplementary "MLP Architecture"): per pixel and mask sample, the 7 colour
// features of the rasterised G-buffer and the degree-2 real spherical-
// harmonic encoding of the view direction (9 values) feed a 16 -> 16 -> 16 -> 3
// MLP (ReLU, ReLU, sigmoid); the first four features, read as RGBA, are
// blended with the MLP colour: rgb = A * feat_rgb + (1 - A) * mlp.
//
// Two forwards: on the tensor cores (k_shade_fwd_tc, tcgen05 kind::tf32 with
// a hi/lo split, described further down; the faster one and the default)
// and in FP32 on the CUDA cores (k_shade_fwd); the backward runs on the
// CUDA cores.  On the CUDA cores the MLP is ALU-bound (560 multiply-adds per
// pixel-sample against 40 bytes of traffic), so those kernels are organised
// to issue few instructions besides the FFMAs:
//  - the SH half of the first layer does not depend on the mask sample: it is
//    evaluated once per pixel and reused for all S samples;
//  - the parameters sit in shared memory and are read as float4 broadcasts,
//    each load shared by two samples of the same pixel;
//  - the backward stages each round's activations and deltas in shared memory
//    and reduces the weight gradients as 4x4 outer-product blocks per thread
//    over the CTA's pixels, into one FP32 partial per CTA; a finish kernel
//    sums the partials in FP64 in a fixed order (deterministic gradients).
#include <string>

#include "ds_internal.h"

namespace ds {

namespace {

constexpr int kIn = 16, kHid = 16, kOut = 3, kFeat = 7, kSH = 9;
constexpr int oW1 = 0, oB1 = 256, oW2 = 272, oB2 = 528, oW3 = 544, oB3 = 592;
constexpr int kParams = DS_SHADE_N_PARAMS;   // 256 + 16 + 256 + 16 + 48 + 3
constexpr int kParamsPad = 596;   // shared copy padded to a float4 multiple
constexpr int kThreads = 256;

// Real SH basis of degree <= 2 (closed-form orthonormal harmonics, the usual
// graphics order and signs).
constexpr float kC0 = 0.28209479177387814f, kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f, kC2b = 0.31539156525252005f, kC2c = 0.5462742152960396f;

struct ShadeTable {
    int n, S, n_blocks, overwrite;
    ShadeView v[DS_MAX_VIEWS];
};

__device__ __forceinline__ int find_view(const ShadeTable& t, int blk) {
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.v[mid].blk0 <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_params(const float* __restrict__ g, float* sp) {
    for (int k = threadIdx.x; k < kParamsPad; k += blockDim.x) sp[k] = k < kParams ? __ldg(g + k) : 0.f;
}

// View direction of pixel (x, y) (unit world-space ray through the pixel
// centre) and its SH encoding.
__device__ __forceinline__ void sh_of_pixel(const ShadeView& V, int x, int y, float sh[kSH]) {
    const float dx = ((float)x + 0.5f - V.cx) / V.fx;
    const float dy = ((float)y + 0.5f - V.cy) / V.fy;
    float wx = fmaf(V.R[0], dx, fmaf(V.R[3], dy, V.R[6]));
    float wy = fmaf(V.R[1], dx, fmaf(V.R[4], dy, V.R[7]));
    float wz = fmaf(V.R[2], dx, fmaf(V.R[5], dy, V.R[8]));
    const float inv = 1.0f / sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    wx *= inv; wy *= inv; wz *= inv;
    sh[0] = kC0;
    sh[1] = -kC1 * wy;
    sh[2] = kC1 * wz;
    sh[3] = -kC1 * wx;
    sh[4] = kC2a * wx * wy;
    sh[5] = -kC2a * wy * wz;
    sh[6] = kC2b * (2.f * wz * wz - wx * wx - wy * wy);
    sh[7] = -kC2a * wx * wz;
    sh[8] = kC2c * (wx * wx - wy * wy);
}

// u = b1 + W1[:, 7:16] sh: the sample-independent part of the first layer.
__device__ __forceinline__ void first_layer_sh(const float* sp, const float sh[kSH], float u[kHid]) {
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        const float* w = sp + oW1 + i * kIn;
        float a = sp[oB1 + i];
#pragma unroll
        for (int k = 0; k < kSH; ++k) a = fmaf(w[kFeat + k], sh[k], a);
        u[i] = a;
    }
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// Forward of NS samples of one pixel: h1, h2 (post-ReLU) and o (sigmoid).
template <int NS>
__device__ __forceinline__ void mlp(const float* sp, const float u[kHid], const float f[NS][kFeat],
                                    float h1[NS][kHid], float h2[NS][kHid], float o[NS][kOut]) {
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        const float4 w0 = *reinterpret_cast<const float4*>(sp + oW1 + i * kIn);
        const float4 w1 = *reinterpret_cast<const float4*>(sp + oW1 + i * kIn + 4);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            float a = u[i];
            a = fmaf(w0.x, f[s][0], a); a = fmaf(w0.y, f[s][1], a);
            a = fmaf(w0.z, f[s][2], a); a = fmaf(w0.w, f[s][3], a);
            a = fmaf(w1.x, f[s][4], a); a = fmaf(w1.y, f[s][5], a);
            a = fmaf(w1.z, f[s][6], a);
            h1[s][i] = fmaxf(a, 0.f);
        }
    }
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        float a[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) a[s] = sp[oB2 + i];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 w = *reinterpret_cast<const float4*>(sp + oW2 + i * kHid + 4 * q);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                a[s] = fmaf(w.x, h1[s][4 * q + 0], a[s]); a[s] = fmaf(w.y, h1[s][4 * q + 1], a[s]);
                a[s] = fmaf(w.z, h1[s][4 * q + 2], a[s]); a[s] = fmaf(w.w, h1[s][4 * q + 3], a[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) h2[s][i] = fmaxf(a[s], 0.f);
    }
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        float a[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) a[s] = sp[oB3 + c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 w = *reinterpret_cast<const float4*>(sp + oW3 + c * kHid + 4 * q);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                a[s] = fmaf(w.x, h2[s][4 * q + 0], a[s]); a[s] = fmaf(w.y, h2[s][4 * q + 1], a[s]);
                a[s] = fmaf(w.z, h2[s][4 * q + 2], a[s]); a[s] = fmaf(w.w, h2[s][4 * q + 3], a[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) o[s][c] = sigmoidf_(a[s]);
    }
}

template <int NS>
__device__ __forceinline__ void shade_samples(const float* sp, const ShadeView& V, const float u[kHid], int s0,
                                              int p) {
    float f[NS][kFeat], h1[NS][kHid], h2[NS][kHid], o[NS][kOut];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int c = 0; c < kFeat; ++c) f[s][c] = __ldcs(V.feat + ((size_t)(s0 + s) * kFeat + c) * V.HW + p);
    mlp<NS>(sp, u, f, h1, h2, o);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const float A = f[s][3];
#pragma unroll
        for (int c = 0; c < kOut; ++c)
            __stcs(V.rgb + ((size_t)(s0 + s) * kOut + c) * V.HW + p, fmaf(A, f[s][c], (1.0f - A) * o[s][c]));
    }
}

// One thread per pixel, all S samples; blocks tile the concatenated pixels
// of all views.
__global__ void __launch_bounds__(kThreads) k_shade_fwd(const __grid_constant__ ShadeTable t,
                                                         const float* __restrict__ params) {
    __shared__ __align__(16) float sp[kParamsPad];
    load_params(params, sp);
    __syncthreads();
    const ShadeView& V = t.v[find_view(t, blockIdx.x)];
    const int p = (blockIdx.x - V.blk0) * kThreads + threadIdx.x;
    if (p >= V.HW) return;
    float sh[kSH], u[kHid];
    sh_of_pixel(V, p % V.W, p / V.W, sh);
    first_layer_sh(sp, sh, u);
    int s = 0;
    for (; s + 2 <= t.S; s += 2) shade_samples<2>(sp, V, u, s, p);
    if (s < t.S) shade_samples<1>(sp, V, u, s, p);
}

// ---------------------------------------------------------------------------
// Backward.
//
// Staging per round (one sample of the CTA's 256 pixels), row-major [p][20]:
// X (input: features, SH), H1, H2, D1 = dL/dz1, D2 = dL/dz2, D3 = dL/dz3
// (padded to 4).  Reduction: threads 0..251 = 7 pixel groups x 36 blocks;
// block b < 16 owns gW1[4(b/4)..][4(b%4)..] (+ gb1 if b%4 == 0), 16 <= b < 32
// the same of gW2, 32 <= b < 36 gW3[0..2][4(b-32)..] (+ gb3 if b == 32).
constexpr int kGroups = 7, kBlocks = 36;
constexpr int kRow = 20;   // 16 values + 4 pad: conflict-free float4 stores of the rows

// A warp of reducers reads one row of D1 and of D2 (and of X and of H1) at
// once: the 64-byte pads put those arrays on complementary shared-memory banks.
struct BwdSmem {
    float sp[kParamsPad];
    float X[kThreads][kRow];
    float pad0[16];
    float H1[kThreads][kRow], H2[kThreads][kRow], D1[kThreads][kRow];
    float pad1[16];
    float D2[kThreads][kRow];
    float D3[kThreads][4];
};
static_assert(sizeof(float) * kGroups * kParams <= sizeof(float) * (2 * kThreads * kRow + 16), "reduction buffer");

// The sample-independent part of the first layer (16 values per pixel) kept
// in the 4 pad columns of the thread's X, H1, H2 and D1 rows (the reducers
// read columns 0..15 only).
__device__ __forceinline__ float* upad(BwdSmem& sm, int tid, int q) {
    return q == 0 ? &sm.X[tid][16] : q == 1 ? &sm.H1[tid][16] : q == 2 ? &sm.H2[tid][16] : &sm.D1[tid][16];
}

__device__ __forceinline__ void store4(float* dst, const float* v) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(kThreads, 2) k_shade_bwd(const __grid_constant__ ShadeTable t,
                                                            const float* __restrict__ params,
                                                            float* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& sm = *reinterpret_cast<BwdSmem*>(smem_raw);
    const float* sp = sm.sp;
    load_params(params, sm.sp);

    const int tid = threadIdx.x;
    const int grp = tid / kBlocks, blk = tid % kBlocks;
    const bool reducer = tid < kGroups * kBlocks;
    const int layer = blk >> 4;                       // 0: W1, 1: W2, 2: W3
    const int ib = layer < 2 ? (blk >> 2) & 3 : 0;    // row block
    const int jb = layer < 2 ? blk & 3 : blk - 32;    // column block
    const int nrow = layer < 2 ? 4 : kOut;
    const bool bias_owner = (jb == 0);
    const float* Dsrc = layer == 0 ? &sm.D1[0][0] : layer == 1 ? &sm.D2[0][0] : &sm.D3[0][0];
    const float* Asrc = layer == 0 ? &sm.X[0][0] : layer == 1 ? &sm.H1[0][0] : &sm.H2[0][0];
    const int dstride = layer < 2 ? kRow : 4;
    float acc[4][4], accb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        accb[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    }
    __syncthreads();

    for (int b = blockIdx.x; b < t.n_blocks; b += gridDim.x) {
        const ShadeView& V = t.v[find_view(t, b)];
        const int p = (b - V.blk0) * kThreads + tid;
        const bool valid = p < V.HW;
        {
            // the SH columns 8..15 of the input row are the same for every
            // sample (column 7, the constant band, is stored with the features)
            float sh[kSH + 3] = {};
            float u[kHid];
            if (valid) {
                sh_of_pixel(V, p % V.W, p / V.W, sh);
                first_layer_sh(sp, sh, u);
#pragma unroll
                for (int q = 0; q < 4; ++q) store4(upad(sm, tid, q), u + 4 * q);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) store4(&sm.X[tid][8 + 4 * q], sh + 1 + 4 * q);
        }
        for (int s = 0; s < t.S; ++s) {
            // Rows are staged as soon as they are known; the ReLU masks of
            // the hidden layers stay in registers as bits.
            float d1[kHid], d3[4];
            if (valid) {
                float f[kFeat];
#pragma unroll
                for (int c = 0; c < kFeat; ++c) f[c] = __ldg(V.feat + ((size_t)s * kFeat + c) * V.HW + p);
                {
                    const float x4[4] = {f[4], f[5], f[6], kC0};
                    store4(&sm.X[tid][0], f);
                    store4(&sm.X[tid][4], x4);
                }
                // Forward.  h1 as in the forward kernel; then each h2 unit in
                // turn is staged and folded into the output accumulators, so
                // that h2 never sits in registers as a whole (the same FMA
                // order per output as the forward kernel).
                unsigned m1 = 0, m2 = 0;
                float h1[kHid];
#pragma unroll
                for (int i = 0; i < kHid; ++i) {
                    const float4 w0 = *reinterpret_cast<const float4*>(sp + oW1 + i * kIn);
                    const float4 w1 = *reinterpret_cast<const float4*>(sp + oW1 + i * kIn + 4);
                    float a = upad(sm, tid, i >> 2)[i & 3];
                    a = fmaf(w0.x, f[0], a); a = fmaf(w0.y, f[1], a);
                    a = fmaf(w0.z, f[2], a); a = fmaf(w0.w, f[3], a);
                    a = fmaf(w1.x, f[4], a); a = fmaf(w1.y, f[5], a);
                    a = fmaf(w1.z, f[6], a);
                    h1[i] = fmaxf(a, 0.f);
                    m1 |= (h1[i] > 0.f ? 1u : 0u) << i;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) store4(&sm.H1[tid][4 * q], h1 + 4 * q);
                float o[kOut];
#pragma unroll
                for (int c = 0; c < kOut; ++c) o[c] = sp[oB3 + c];
#pragma unroll
                for (int i = 0; i < kHid; ++i) {
                    float a = sp[oB2 + i];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 w = *reinterpret_cast<const float4*>(sp + oW2 + i * kHid + 4 * q);
                        a = fmaf(w.x, h1[4 * q + 0], a); a = fmaf(w.y, h1[4 * q + 1], a);
                        a = fmaf(w.z, h1[4 * q + 2], a); a = fmaf(w.w, h1[4 * q + 3], a);
                    }
                    const float h2 = fmaxf(a, 0.f);
                    m2 |= (h2 > 0.f ? 1u : 0u) << i;
                    sm.H2[tid][i] = h2;
#pragma unroll
                    for (int c = 0; c < kOut; ++c) o[c] = fmaf(sp[oW3 + c * kHid + i], h2, o[c]);
                }
#pragma unroll
                for (int c = 0; c < kOut; ++c) o[c] = sigmoidf_(o[c]);
                float g[kOut];
#pragma unroll
                for (int c = 0; c < kOut; ++c) g[c] = __ldcs(V.grad_rgb + ((size_t)s * kOut + c) * V.HW + p);
                const float A = f[3];
                float gA = 0.f;
#pragma unroll
                for (int c = 0; c < kOut; ++c) {
                    gA = fmaf(g[c], f[c] - o[c], gA);
                    const float go = (1.0f - A) * g[c];
                    d3[c] = go * o[c] * (1.0f - o[c]);
                }
                d3[3] = 0.f;
                // d2_j = (W3^T d3)_j [z2_j > 0], staged as soon as known and
                // folded into d1 = W2^T d2 (then masked by [z1 > 0])
#pragma unroll
                for (int k = 0; k < kHid; ++k) d1[k] = 0.f;
#pragma unroll
                for (int j = 0; j < kHid; ++j) {
                    float dj = 0.f;
#pragma unroll
                    for (int c = 0; c < kOut; ++c) dj = fmaf(sp[oW3 + c * kHid + j], d3[c], dj);
                    dj = (m2 >> j) & 1u ? dj : 0.f;
                    sm.D2[tid][j] = dj;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 w = *reinterpret_cast<const float4*>(sp + oW2 + j * kHid + 4 * q);
                        d1[4 * q + 0] = fmaf(w.x, dj, d1[4 * q + 0]); d1[4 * q + 1] = fmaf(w.y, dj, d1[4 * q + 1]);
                        d1[4 * q + 2] = fmaf(w.z, dj, d1[4 * q + 2]); d1[4 * q + 3] = fmaf(w.w, dj, d1[4 * q + 3]);
                    }
                }
#pragma unroll
                for (int k = 0; k < kHid; ++k) d1[k] = (m1 >> k) & 1u ? d1[k] : 0.f;
                // feature gradient: blend terms + (W1^T d1)[0:7]
                if (V.grad_feat) {
                    float gf[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) gf[m] = 0.f;
#pragma unroll
                    for (int k = 0; k < kHid; ++k) {
                        const float4 w0 = *reinterpret_cast<const float4*>(sp + oW1 + k * kIn);
                        const float4 w1 = *reinterpret_cast<const float4*>(sp + oW1 + k * kIn + 4);
                        gf[0] = fmaf(w0.x, d1[k], gf[0]); gf[1] = fmaf(w0.y, d1[k], gf[1]);
                        gf[2] = fmaf(w0.z, d1[k], gf[2]); gf[3] = fmaf(w0.w, d1[k], gf[3]);
                        gf[4] = fmaf(w1.x, d1[k], gf[4]); gf[5] = fmaf(w1.y, d1[k], gf[5]);
                        gf[6] = fmaf(w1.z, d1[k], gf[6]);
                    }
#pragma unroll
                    for (int c = 0; c < kOut; ++c) gf[c] = fmaf(A, g[c], gf[c]);
                    gf[3] += gA;
                    float* dst = V.grad_feat + (size_t)s * kFeat * V.HW + p;
                    if (t.overwrite) {
#pragma unroll
                        for (int c = 0; c < kFeat; ++c) dst[(size_t)c * V.HW] = gf[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < kFeat; ++c) dst[(size_t)c * V.HW] += gf[c];
                    }
                }
            } else {
                const float z4[4] = {0.f, 0.f, 0.f, 0.f};
                store4(&sm.X[tid][0], z4);
                store4(&sm.X[tid][4], z4);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    store4(&sm.H1[tid][4 * q], z4);
                    store4(&sm.H2[tid][4 * q], z4);
                }
#pragma unroll
                for (int k = 0; k < kHid; ++k) d1[k] = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) d3[c] = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) store4(&sm.D2[tid][4 * q], z4);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) store4(&sm.D1[tid][4 * q], d1 + 4 * q);
            store4(&sm.D3[tid][0], d3);
            __syncthreads();
            if (reducer) {
                for (int q = grp; q < kThreads; q += kGroups) {
                    const float4 d = *reinterpret_cast<const float4*>(Dsrc + q * dstride + 4 * ib);
                    const float4 a = *reinterpret_cast<const float4*>(Asrc + q * kRow + 4 * jb);
                    const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[i][0] = fmaf(dv[i], a.x, acc[i][0]); acc[i][1] = fmaf(dv[i], a.y, acc[i][1]);
                        acc[i][2] = fmaf(dv[i], a.z, acc[i][2]); acc[i][3] = fmaf(dv[i], a.w, acc[i][3]);
                        accb[i] += dv[i];
                    }
                }
            }
            __syncthreads();
        }
    }

    // Reduce the 7 pixel groups in shared memory, then one partial per CTA.
    float* red = &sm.X[0][0];   // [kGroups][kParams]
    for (int k = tid; k < kGroups * kParams; k += kThreads) red[k] = 0.f;
    __syncthreads();
    if (reducer) {
        float* r = red + grp * kParams;
        const int oW = layer == 0 ? oW1 : layer == 1 ? oW2 : oW3;
        const int oB = layer == 0 ? oB1 : layer == 1 ? oB2 : oB3;
        for (int i = 0; i < nrow; ++i) {
            const int row = 4 * ib + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) r[oW + row * kHid + 4 * jb + j] = acc[i][j];
            if (bias_owner) r[oB + row] = accb[i];
        }
    }
    __syncthreads();
    for (int k = tid; k < kParams; k += kThreads) {
        float a = 0.f;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) a += red[g * kParams + k];
        partial[(size_t)blockIdx.x * kParams + k] = a;
    }
}

// grad_params[k] (+)= sum over CTAs of partial[c][k], in FP64, CTA order.
__global__ void __launch_bounds__(kThreads) k_shade_finish(const float* __restrict__ partial, int n_cta,
                                                            float* __restrict__ out, int overwrite) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kParams) return;
    double a = 0.0;
    for (int c = 0; c < n_cta; ++c) a += (double)partial[(size_t)c * kParams + k];
    out[k] = overwrite ? (float)a : (float)((double)out[k] + a);
}

// ---------------------------------------------------------------------------
// Forward on the tensor cores: the three layers as tcgen05.mma of kind::tf32
// (Blackwell 5th-generation tensor cores).  A tile is 128 pixel-samples, one
// per thread and one tensor-memory lane each (M = 128); N = 16 hidden units
// (the 3 outputs padded to 16); K = 16 inputs in two MMAs of K = 8.  TF32
// keeps 10 mantissa bits, so every operand is split into hi = the TF32
// truncation and lo = the remainder (exact in FP32) and each product is taken
// as x_lo w_hi + x_hi w_lo + x_hi w_hi (the x_lo w_lo term, about 2^-21 of the
// product, is dropped): six MMAs per layer, and a seventh adds the bias (a
// constant K-chunk (1, 1, 0, ...) times the bias tile (b hi, b lo)), issued
// by one thread and completed on an mbarrier.
//
// The layer inputs (operand A) live in tensor memory beside the FP32
// accumulator: each thread writes its row with tcgen05.st and the MMAs read A
// from there, so shared memory carries only the weight and bias tiles (B, 9
// KB).  With A in shared memory every MMA re-read 4 KB of it, and the
// shared-memory bandwidth, not the tensor cores, set the kernel's speed.  Per
// layer the 128 threads read their accumulator row (tcgen05.ld), apply the
// activation and write the next layer's hi/lo row.
namespace tc {

constexpr int kRows = 128;   // pixel-samples per tile = TMEM lanes = M
// Tensor-memory columns of a CTA (one 32-bit value per column and lane): the
// accumulator D in 0..15, A hi in 16..31, A lo in 32..47, and in 48..55 the
// constant K-chunk (1, 1, 0, ..., 0) that adds the bias rows (b hi, b lo) of
// the bias tile.
constexpr uint32_t kTmemCols = 64;
constexpr uint32_t kColD = 0, kColAh = 16, kColAl = 32, kColOne = 48;
constexpr int kMaxCtasPerSm = 512 / (int)kTmemCols;   // the SM's 512 columns, none left waiting
// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// Byte offset of element (n, k) of a 16 x 16 K-major TF32 operand in shared
// memory in the canonical layout without swizzle: core matrices of 8 rows x
// 16 bytes (4 values), 128 bytes each; the two core matrices of one MMA's
// K = 8 are 128 bytes apart (leading-dimension offset), the two 8-row groups
// 512 bytes apart (stride-dimension offset).
__device__ __forceinline__ uint32_t op_off(int n, int k) {
    return (uint32_t)(((((n >> 3) << 2) + (k >> 2)) << 7) + ((n & 7) << 4) + ((k & 3) << 2));
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

struct Smem {
    uint8_t w[6][1024];   // W1 hi, W1 lo, W2 hi, W2 lo, W3 hi, W3 lo (N 16 x K 16)
    uint8_t b[3][1024];   // bias tiles of the three layers: K = 0 b hi, K = 1 b lo, else 0
    unsigned long long bar;
    uint32_t tmem;
};

// TF32 hi part (truncation to 10 mantissa bits) and FP32 remainder.
__device__ __forceinline__ void split(float x, uint32_t& h, uint32_t& l) {
    h = __float_as_uint(x) & 0xFFFFE000u;
    l = __float_as_uint(x - __uint_as_float(h));
}

// 16 columns of this thread's lane from column `col` on (warp w owns lanes
// 32w .. 32w + 31, the lane field sits in bits 16-31 of the address).
__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, uint32_t col) {
    return tmem + ((uint32_t)(threadIdx.x & ~31) << 16) + col;
}

__device__ __forceinline__ void st8(uint32_t ta, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(ta), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// Write eight values of this thread's operand row, K = 8 half .. 8 half + 7,
// as their hi and lo parts into tensor memory.
__device__ __forceinline__ void store_half(uint32_t tmem, int half, const uint32_t (&h)[8], const uint32_t (&l)[8]) {
    st8(lane_addr(tmem, kColAh + 8 * half), h);
    st8(lane_addr(tmem, kColAl + 8 * half), l);
}

__device__ __forceinline__ void split8(const float* x, uint32_t (&h)[8], uint32_t (&l)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) split(x[i], h[i], l[i]);
}

__device__ __forceinline__ void mma(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(accumulate));
}

// Layer L: D = A_lo W_hi + A_hi W_lo + A_hi W_hi (small terms first) + the
// bias, then the commit that arrives on the barrier when the MMAs are
// complete.  One thread.
__device__ __forceinline__ void issue_layer(Smem& sm, int L, uint32_t tmem) {
    const uint32_t b0 = saddr(sm.w[2 * L]), b1 = saddr(sm.w[2 * L + 1]);
    const uint32_t d = tmem + kColD;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        mma(d, tmem + kColAl + 8 * s, smem_desc(b0 + 256 * s), s);
        mma(d, tmem + kColAh + 8 * s, smem_desc(b1 + 256 * s), 1);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) mma(d, tmem + kColAh + 8 * s, smem_desc(b0 + 256 * s), 1);
    mma(d, tmem + kColOne, smem_desc(saddr(sm.b[L])), 1);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(&sm.bar))
                 : "memory");
}

// Wait for phase `parity` of the barrier, for at most about 2^31 SM clocks.
__device__ __forceinline__ bool wait_bar(const Smem& sm, uint32_t parity) {
    const uint32_t b = saddr(&sm.bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

// This thread's accumulator row, 16 columns.
__device__ __forceinline__ void load_row(uint32_t tmem, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(lane_addr(tmem, kColD)));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// This thread's tensor-memory stores complete, and they and its earlier
// tensor-memory loads ordered before the barrier that follows.
__device__ __forceinline__ void before_sync() {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

// Logistic function from the hardware exponential and the correctly rounded
// reciprocal (a few 1e-7 from the exact value on [0, 1]).
__device__ __forceinline__ float sigmoid(float z) { return __frcp_rn(1.0f + __expf(-z)); }

}  // namespace tc

// Per round a CTA takes one tile: 128 consecutive pixels of one view (tiles
// never straddle views: view v owns tiles blk0 .. blk0 + ceil(HW / 128) - 1)
// and all S mask samples of them in turn.  The SH encoding of the pixel and
// its hi/lo split are computed once per tile; per sample the thread writes
// its input row (7 features, then the 9 SH values) and the three layers
// run.  The next sample's features are loaded before the current sample's
// MMAs.  Persistent CTAs of 128 threads.  A wait for the MMAs that runs out
// (about a second) sets bit 1 of *status, and the CTA releases its tensor
// memory and returns.  kNoMma: the MMAs are never issued, so that every wait
// runs out (for testing the bounded wait on a GPU).
template <bool kNoMma>
__global__ void __launch_bounds__(tc::kRows, tc::kMaxCtasPerSm) k_shade_fwd_tc(const __grid_constant__ ShadeTable t,
                                                          const float* __restrict__ params, int* __restrict__ status) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u));
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights -> TF32 hi/lo operand tiles (W3's 3 rows padded with zeros)
    for (int q = tid; q < 3 * 256; q += kRows) {
        const int L = q >> 8, n = (q >> 4) & 15, k = q & 15;
        const int o = L == 0 ? oW1 : (L == 1 ? oW2 : oW3);
        const float w = (L < 2 || n < kOut) ? __ldg(params + o + n * 16 + k) : 0.f;
        uint32_t h, l;
        split(w, h, l);
        *reinterpret_cast<uint32_t*>(sm.w[2 * L] + op_off(n, k)) = h;
        *reinterpret_cast<uint32_t*>(sm.w[2 * L + 1] + op_off(n, k)) = l;
    }
    for (int q = tid; q < 3 * 256; q += kRows) {
        const int L = q >> 8, n = (q >> 4) & 15, k = q & 15;
        const int o = L == 0 ? oB1 : (L == 1 ? oB2 : oB3);
        const float b = (k < 2 && (L < 2 || n < kOut)) ? __ldg(params + o + n) : 0.f;
        uint32_t h, l;
        split(b, h, l);
        *reinterpret_cast<uint32_t*>(sm.b[L] + op_off(n, k)) = k == 0 ? h : (k == 1 ? l : 0u);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&sm.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&sm.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // the weight tiles (generic-proxy writes) visible to the MMAs
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    before_sync();
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem;
    {
        const uint32_t one = __float_as_uint(1.0f);
        const uint32_t r[8] = {one, one, 0u, 0u, 0u, 0u, 0u, 0u};
        st8(lane_addr(tmem, kColOne), r);
    }
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < t.n_blocks && ok; tile += gridDim.x) {
        const ShadeView& V = t.v[find_view(t, tile)];
        const int p = (tile - V.blk0) * kRows + tid;
        const bool valid = p < V.HW;
        const int py = valid ? p / V.W : 0, px = valid ? p - py * V.W : 0;
        // input columns 8..15 (SH bands 1..8), split once for all samples;
        // column 7 is the constant band
        uint32_t shh[8], shl[8];
        {
            float sh[kSH];
            sh_of_pixel(V, px, py, sh);
            split8(sh + 1, shh, shl);
        }
        const float* fp = V.feat + (valid ? p : 0);
        float fn[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) fn[c] = valid ? __ldcs(fp + (size_t)c * V.HW) : 0.f;
        for (int s = 0; s < t.S; ++s) {
            float f[kFeat];
#pragma unroll
            for (int c = 0; c < kFeat; ++c) f[c] = fn[c];
            if (s + 1 < t.S) {
#pragma unroll
                for (int c = 0; c < kFeat; ++c)
                    fn[c] = valid ? __ldcs(fp + ((size_t)(s + 1) * kFeat + c) * V.HW) : 0.f;
            }
            {
                const float x[8] = {f[0], f[1], f[2], f[3], f[4], f[5], f[6], kC0};
                uint32_t h[8], l[8];
                split8(x, h, l);
                store_half(tmem, 0, h, l);
                store_half(tmem, 1, shh, shl);
            }
            float o[kOut];
#pragma unroll
            for (int L = 0; L < 3; ++L) {
                // the rows are complete and every thread's reads of the
                // previous accumulator are done: the next MMAs may start
                before_sync();
                __syncthreads();
                if (tid == 0 && !kNoMma) issue_layer(sm, L, tmem);
                ok = __syncthreads_and(wait_bar(sm, phase));
                phase ^= 1u;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                float d[16];
                load_row(tmem, d);
                if (L < 2) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) d[i] = fmaxf(d[i], 0.f);
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        uint32_t h[8], l[8];
                        split8(d + 8 * half, h, l);
                        store_half(tmem, half, h, l);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < kOut; ++c) o[c] = sigmoid(d[c]);
                }
            }
            if (!ok) break;
            if (valid) {
                const float A = f[3];
#pragma unroll
                for (int c = 0; c < kOut; ++c)
                    __stcs(V.rgb + ((size_t)s * kOut + c) * V.HW + p, fmaf(A, f[c], (1.0f - A) * o[c]));
            }
        }
    }
    if (!ok) {
        // a layer's MMAs did not complete in time: record it, give them one
        // more bounded wait, then release the tensor memory and return
        if (tid == 0) atomicOr(status, 2);
        wait_bar(sm, phase ^ 1u);
    }
    before_sync();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

void fill_table(ShadeTable& t, const ShadeView* views, int n, int S, bool overwrite) {
    t.n = n;
    t.S = S;
    t.overwrite = overwrite ? 1 : 0;
    int blk = 0;
    for (int i = 0; i < n; ++i) {
        t.v[i] = views[i];
        t.v[i].HW = views[i].W * views[i].H;
        t.v[i].blk0 = blk;
        blk += (t.v[i].HW + kThreads - 1) / kThreads;
    }
    t.n_blocks = blk;
}

}  // namespace

int shade_bwd_grid() {
    static int cached = 0;
    if (cached > 0) return cached;
    int blocks = 0;
    const size_t smem = sizeof(BwdSmem);
    if (cudaFuncSetAttribute(k_shade_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_shade_bwd, kThreads, smem) != cudaSuccess ||
        blocks < 1) {
        cudaGetLastError();
        blocks = 1;
    }
    cached = persistent_grid(1 << 30, blocks);
    return cached;
}

size_t shade_partial_floats(int grid) { return (size_t)grid * kParams; }

cudaError_t launch_shade_fwd(const ShadeView* views, int n, int S, const float* params, cudaStream_t st) {
    ShadeTable t;
    fill_table(t, views, n, S, false);
    if (t.n_blocks == 0 || S == 0) return cudaSuccess;
    k_shade_fwd<<<t.n_blocks, kThreads, 0, st>>>(t, params);
    note_launches(1);
    return cudaGetLastError();
}

// Launch shape of k_shade_fwd_tc: dynamic shared memory and CTAs per SM.
// Each CTA holds kTmemCols of the SM's 512 tensor-memory columns, so at most
// kMaxCtasPerSm may be resident at once (a further CTA's allocation would
// wait for a CTA to finish); the shared-memory request is padded so that no
// more fit, and the residency is the least of what shared memory, registers
// and threads allow.  Computed here from the kernel's attributes: the
// runtime's occupancy query answers 1 for this kernel although more CTAs fit.
bool tc_launch_shape(size_t* dyn_smem, int* per_sm) {
    static size_t c_smem = 0;
    static int c_per_sm = 0;
    if (c_per_sm > 0) {
        *dyn_smem = c_smem;
        *per_sm = c_per_sm;
        return true;
    }
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, k_shade_fwd_tc<false>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t fixed = fa.sharedSizeBytes + (size_t)reserved;
    size_t smem = sizeof(tc::Smem) + 1024;   // + room to align the weight tiles to 1 KB
    const size_t at_least = (size_t)smem_sm / (tc::kMaxCtasPerSm + 1) + 1;   // kMaxCtasPerSm + 1 do not fit
    if (smem + fixed < at_least) smem = at_least - fixed;
    const int by_smem = (int)((size_t)smem_sm / (smem + fixed));
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;   // allocated per warp in units of 256
    const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * (tc::kRows / 32)) : tc::kMaxCtasPerSm;
    const int by_thr = thr_sm / tc::kRows;
    int n = by_smem < by_regs ? by_smem : by_regs;
    n = n < by_thr ? n : by_thr;
    if (n < 1 || n > tc::kMaxCtasPerSm) return false;
    c_smem = smem;
    c_per_sm = n;
    *dyn_smem = smem;
    *per_sm = n;
    return true;
}

cudaError_t launch_shade_fwd_tc(const ShadeView* views, int n, int S, const float* params, int* status,
                                cudaStream_t st, bool no_mma) {
    ShadeTable t;
    t.n = n;
    t.S = S;
    t.overwrite = 0;
    int blk = 0;
    for (int i = 0; i < n; ++i) {
        t.v[i] = views[i];
        t.v[i].HW = views[i].W * views[i].H;
        t.v[i].blk0 = blk;
        blk += (t.v[i].HW + tc::kRows - 1) / tc::kRows;
    }
    t.n_blocks = blk;
    if (t.n_blocks == 0) return cudaSuccess;
    size_t smem = 0;
    int per_sm = 0;
    if (!tc_launch_shape(&smem, &per_sm)) return cudaErrorInvalidConfiguration;
    // the diagnostic instantiation is launched with the production one's
    // shape (its shared-memory padding keeps the same residency cap)
    auto kernel = no_mma ? k_shade_fwd_tc<true> : k_shade_fwd_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<persistent_grid(t.n_blocks, per_sm), tc::kRows, smem, st>>>(t, params, status);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_shade_bwd(const ShadeView* views, int n, int S, const float* params, bool overwrite,
                             float* partial, int grid, float* grad_params, cudaStream_t st) {
    ShadeTable t;
    fill_table(t, views, n, S, overwrite);
    if (t.n_blocks > 0 && S > 0) {
        const size_t smem = sizeof(BwdSmem);
        cudaError_t e = cudaFuncSetAttribute(k_shade_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int g = grid < t.n_blocks ? grid : t.n_blocks;
        k_shade_bwd<<<g, kThreads, smem, st>>>(t, params, partial);
        note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (grad_params) {
            k_shade_finish<<<(kParams + kThreads - 1) / kThreads, kThreads, 0, st>>>(partial, g, grad_params,
                                                                                   overwrite ? 1 : 0);
            note_launches(1);
        }
    } else if (grad_params && overwrite) {
        return cudaMemsetAsync(grad_params, 0, sizeof(float) * kParams, st);
    }
    return cudaGetLastError();
}

}  // namespace ds
