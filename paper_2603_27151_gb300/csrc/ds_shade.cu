// ds_shade.cu -- neural deferred shading (Sec. 3.3 "Neural deferred shading";
// supplementary "MLP Architecture"): per pixel and mask sample, the 7 colour
// features of the rasterised G-buffer and the degree-2 real spherical-
// harmonic encoding of the view direction (9 values) feed a 16 -> 16 -> 16 -> 3
// MLP (ReLU, ReLU, sigmoid); the first four features, read as RGBA, are
// blended with the MLP colour: rgb = A * feat_rgb + (1 - A) * mlp.
//
// FP32 on the CUDA cores.  The MLP is ALU-bound (560 multiply-adds per
// pixel-sample against 40 bytes of traffic), so the kernels are organised to
// issue few instructions besides the FFMAs:
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
        float u[kHid];
        {
            // the SH columns 8..15 of the input row are the same for every
            // sample (column 7, the constant band, is stored with the features)
            float sh[kSH + 3] = {};
            if (valid) {
                sh_of_pixel(V, p % V.W, p / V.W, sh);
                first_layer_sh(sp, sh, u);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) store4(&sm.X[tid][8 + 4 * q], sh + 1 + 4 * q);
        }
        for (int s = 0; s < t.S; ++s) {
            // Rows are staged as soon as they are known; the ReLU masks of
            // the hidden layers stay in registers as bits.
            float d1[kHid], d2[kHid], d3[4];
            if (valid) {
                float f[1][kFeat], h1[1][kHid], h2[1][kHid], o[1][kOut];
#pragma unroll
                for (int c = 0; c < kFeat; ++c) f[0][c] = __ldg(V.feat + ((size_t)s * kFeat + c) * V.HW + p);
                {
                    const float x4[4] = {f[0][4], f[0][5], f[0][6], kC0};
                    store4(&sm.X[tid][0], f[0]);
                    store4(&sm.X[tid][4], x4);
                }
                mlp<1>(sp, u, f, h1, h2, o);
                unsigned m1 = 0, m2 = 0;
#pragma unroll
                for (int k = 0; k < kHid; ++k) {
                    m1 |= (h1[0][k] > 0.f ? 1u : 0u) << k;
                    m2 |= (h2[0][k] > 0.f ? 1u : 0u) << k;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    store4(&sm.H1[tid][4 * q], h1[0] + 4 * q);
                    store4(&sm.H2[tid][4 * q], h2[0] + 4 * q);
                }
                float g[kOut];
#pragma unroll
                for (int c = 0; c < kOut; ++c) g[c] = __ldcs(V.grad_rgb + ((size_t)s * kOut + c) * V.HW + p);
                const float A = f[0][3];
                float gA = 0.f;
#pragma unroll
                for (int c = 0; c < kOut; ++c) {
                    gA = fmaf(g[c], f[0][c] - o[0][c], gA);
                    const float go = (1.0f - A) * g[c];
                    d3[c] = go * o[0][c] * (1.0f - o[0][c]);
                }
                d3[3] = 0.f;
                // d2 = (W3^T d3) * [z2 > 0]
#pragma unroll
                for (int j = 0; j < kHid; ++j) d2[j] = 0.f;
#pragma unroll
                for (int c = 0; c < kOut; ++c)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 w = *reinterpret_cast<const float4*>(sp + oW3 + c * kHid + 4 * q);
                        d2[4 * q + 0] = fmaf(w.x, d3[c], d2[4 * q + 0]); d2[4 * q + 1] = fmaf(w.y, d3[c], d2[4 * q + 1]);
                        d2[4 * q + 2] = fmaf(w.z, d3[c], d2[4 * q + 2]); d2[4 * q + 3] = fmaf(w.w, d3[c], d2[4 * q + 3]);
                    }
#pragma unroll
                for (int j = 0; j < kHid; ++j) d2[j] = (m2 >> j) & 1u ? d2[j] : 0.f;
                // d1 = (W2^T d2) * [z1 > 0]
#pragma unroll
                for (int k = 0; k < kHid; ++k) d1[k] = 0.f;
#pragma unroll
                for (int j = 0; j < kHid; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 w = *reinterpret_cast<const float4*>(sp + oW2 + j * kHid + 4 * q);
                        d1[4 * q + 0] = fmaf(w.x, d2[j], d1[4 * q + 0]); d1[4 * q + 1] = fmaf(w.y, d2[j], d1[4 * q + 1]);
                        d1[4 * q + 2] = fmaf(w.z, d2[j], d1[4 * q + 2]); d1[4 * q + 3] = fmaf(w.w, d2[j], d1[4 * q + 3]);
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
#pragma unroll
                    for (int c = 0; c < kFeat; ++c) {
                        float* dst = V.grad_feat + ((size_t)s * kFeat + c) * V.HW + p;
                        *dst = t.overwrite ? gf[c] : *dst + gf[c];
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
                for (int k = 0; k < kHid; ++k) d1[k] = d2[k] = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) d3[c] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                store4(&sm.D1[tid][4 * q], d1 + 4 * q);
                store4(&sm.D2[tid][4 * q], d2 + 4 * q);
            }
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
