// ds_levels.cu -- multi-resolution feature grids (Sec. 3.3, multi-resolution
// mesh colours; supplementary "Coarse-to-Fine Optimization").
//
// Level R carries a mesh-colour grid with N_R = 2^R subdivisions per edge and
// V_R = (N_R+1)(N_R+2)/2 feature vertices; a soup's levels r_min..r_max are
// stored one after the other, level R as [T][V_R][C].  The texture that is
// rasterised is the finest grid (N = 2^r_max) whose logits are the sum of all
// levels evaluated at its vertices, then the sigmoid:
//  - k_compose (fused into the activation step): one CTA per triangle.  All
//    of the triangle's levels are staged in shared memory (vector loads, all
//    in flight together); each finest vertex then sums, coarsest level
//    first in FP32, the value of every level at its position (the
//    coinciding level vertex, or the decode's interpolation in the level's
//    micro-triangle), as the oracle does; the finest level adds its own
//    value, and the sum goes straight to the sigmoid;
//  - k_restrict (fused into the gradient finish step): the adjoint.  The
//    level-R function is piecewise linear on level R+1's mesh (same diagonal
//    orientation), so the composition is a chain of 2x prolongations and its
//    adjoint a chain of 2x restrictions: each coarse vertex gathers its fine
//    twin and, with weight 1/2, the midpoints of its six incident edges.  One
//    CTA per triangle, levels in shared memory, FP32 from the FP64
//    accumulator of the finest grid;
//  - k_restrict_staged: the same adjoint with all of a triangle's level
//    gradients staged in shared memory and written as float4 streams
//    (overwrite mode), or applied there as the levels' Adam step (the
//    backward with a fused texture optimiser);
//  - k_resample: one level's grid sampled at another level's vertices.
#include <cuda_fp16.h>

#include "ds_internal.h"

namespace ds {

namespace {

__host__ __device__ constexpr int level_V(int R) { return ((1 << R) + 1) * ((1 << R) + 2) / 2; }

// (i, j) of vertex v of the N-subdivided grid (rows of constant j).
__device__ __forceinline__ void texel_ij(int N, int v, int& i, int& j) {
    const float b = (float)(2 * N + 3);
    int jj = (int)floorf(0.5f * (b - sqrtf(b * b - 8.0f * (float)v)));
    jj = jj < 0 ? 0 : (jj > N ? N : jj);
    while (jj > 0 && texel_index(N, 0, jj) > v) --jj;
    while (jj < N && texel_index(N, 0, jj + 1) <= v) ++jj;
    j = jj;
    i = v - texel_index(N, 0, jj);
}

// Value of channel c of the level-R grid g ([V_R][C]) at vertex (i, j) of
// the grid with N = 2^k subdivisions.
__device__ __forceinline__ float level_value(const float* __restrict__ g, int R, int C, int c, int i, int j, int N) {
    const int NR = 1 << R;
    if (N <= NR) return __ldg(g + (size_t)texel_index(NR, i * (NR / N), j * (NR / N)) * C + c);
    const int s = N / NR;
    if (i % s == 0 && j % s == 0) return __ldg(g + (size_t)texel_index(NR, i / s, j / s) * C + c);
    const Cell cl = find_cell(NR, __fdiv_rn((float)i, (float)N), __fdiv_rn((float)j, (float)N));
    return interp(__ldg(g + (size_t)cl.k0 * C + c), __ldg(g + (size_t)cl.k1 * C + c), __ldg(g + (size_t)cl.k2 * C + c),
                  cl.wa, cl.wb);
}

// Value of the level-R grid zl ([V_R][C] in shared memory, channels c..c+3
// when kVec) at vertex (i, j) of the finest grid (Nf = 2^r_max
// subdivisions): the coinciding vertex, or the decode's interpolation in the
// micro-triangle that holds barycentrics (i / Nf, j / Nf) (exact: Nf is a
// power of two).
template <bool kVec>
__device__ __forceinline__ float4 level_at(const float* zl, int R, int C, int c, int i, int j, int Nf, int r_max) {
    const int NR = 1 << R, sh = r_max - R, m = (1 << sh) - 1;
    if (!(i & m) && !(j & m)) {
        const float* p = zl + (size_t)texel_index(NR, i >> sh, j >> sh) * C + c;
        return kVec ? *reinterpret_cast<const float4*>(p) : make_float4(*p, 0.f, 0.f, 0.f);
    }
    const float inv = __frcp_rn((float)Nf);   // exact power of two
    const Cell cl = find_cell(NR, __fmul_rn((float)i, inv), __fmul_rn((float)j, inv));
    const float* p0 = zl + (size_t)cl.k0 * C + c;
    const float* p1 = zl + (size_t)cl.k1 * C + c;
    const float* p2 = zl + (size_t)cl.k2 * C + c;
    if (kVec) {
        const float4 a0 = *reinterpret_cast<const float4*>(p0);
        const float4 a1 = *reinterpret_cast<const float4*>(p1);
        const float4 a2 = *reinterpret_cast<const float4*>(p2);
        return make_float4(interp(a0.x, a1.x, a2.x, cl.wa, cl.wb), interp(a0.y, a1.y, a2.y, cl.wa, cl.wb),
                           interp(a0.z, a1.z, a2.z, cl.wa, cl.wb), interp(a0.w, a1.w, a2.w, cl.wa, cl.wb));
    }
    return make_float4(interp(*p0, *p1, *p2, cl.wa, cl.wb), 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}

// Floats of one triangle's levels r_min..r_max (the shared-memory stage).
__host__ __device__ inline int stage_floats(int r_min, int r_max, int C) {
    int n = 0;
    for (int R = r_min; R <= r_max; ++R) n += level_V(R) * C;
    return n;
}

// Sigmoid of Sec. 3.3 with the reciprocal of (1 + e^-x) taken by the
// correctly rounded reciprocal: the same value as pinned_sigmoid's IEEE
// division 1 / (1 + e^-x) (both round 1/y to nearest; y >= 1).
__device__ __forceinline__ float sigmoid_rcp(float th) { return __frcp_rn(__fadd_rn(1.0f, pinned_exp(-th))); }

// Tap of one coarse level at one finest vertex, shared by every triangle:
// corner texel indices k0 | k1 << 10 | k2 << 20 (| 1 << 30 when the vertex
// coincides with level vertex k0) and the interpolation weights (wa, wb) of
// the decode (R3) as two halves: they are multiples of 2^-(r_max - R) in
// [0, 1] with r_max - R <= 5, exact in FP16.
__device__ __forceinline__ uint2 make_tap(int R, int i, int j, int Nf, int r_max) {
    const int NR = 1 << R, sh = r_max - R, m = (1 << sh) - 1;
    if (!(i & m) && !(j & m)) return make_uint2((uint32_t)texel_index(NR, i >> sh, j >> sh) | (1u << 30), 0u);
    const float inv = __frcp_rn((float)Nf);   // exact power of two
    const Cell cl = find_cell(NR, __fmul_rn((float)i, inv), __fmul_rn((float)j, inv));
    const __half2 w = __floats2half2_rn(cl.wa, cl.wb);
    return make_uint2((uint32_t)cl.k0 | ((uint32_t)cl.k1 << 10) | ((uint32_t)cl.k2 << 20),
                      *reinterpret_cast<const uint32_t*>(&w));
}

// Channels c..c+3 of level grid zl at a tap (the coinciding vertex, or the
// decode's interpolation in FP32 in the decode's order).
__device__ __forceinline__ float4 tap_value(const float* zl, uint2 tp, int C, int c) {
    const float4 a0 = *reinterpret_cast<const float4*>(zl + (size_t)(tp.x & 1023u) * C + c);
    if (tp.x >> 30) return a0;
    const float4 a1 = *reinterpret_cast<const float4*>(zl + (size_t)((tp.x >> 10) & 1023u) * C + c);
    const float4 a2 = *reinterpret_cast<const float4*>(zl + (size_t)((tp.x >> 20) & 1023u) * C + c);
    const float2 w = __half22float2(*reinterpret_cast<const __half2*>(&tp.y));
    return make_float4(interp(a0.x, a1.x, a2.x, w.x, w.y), interp(a0.y, a1.y, a2.y, w.x, w.y),
                       interp(a0.z, a1.z, a2.z, w.x, w.y), interp(a0.w, a1.w, a2.w, w.x, w.y));
}

// 16-byte asynchronous copy global -> shared (cp.async, completion by
// commit/wait groups: no spin loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the copies of triangle t's coarse levels r_min..r_max-1 into zs.
__device__ __forceinline__ void stage_coarse(float* zs, const float* __restrict__ levels, int t, int T, int r_min,
                                             int r_max, int C) {
    size_t off = 0;   // offset of level R in `levels`
    int so = 0;       // offset of level R in zs
    for (int R = r_min; R < r_max; ++R) {
        const int n = level_V(R) * C;
        const float* g = levels + off + (size_t)t * n;
        for (int k = threadIdx.x; k < n / 4; k += blockDim.x) cp_async16(zs + so + 4 * k, g + 4 * k);
        off += (size_t)T * n;
        so += n;
    }
}

// Persistent CTAs (grid-stride over triangles), C % 4 == 0 and 16-byte
// aligned levels and output.  Shared memory: the taps of the coarse levels
// at every finest vertex (computed once per CTA: they do not depend on the
// triangle), then two stages of one triangle's coarse levels, filled by
// asynchronous copies one triangle ahead.  Items are (finest vertex, group
// of four channels); an item's finest-level values stream from global
// memory (issued before the coarse levels are read), the coarse levels'
// values at the vertex come from the stage, and the sum runs from the
// coarsest level up (FP32, the oracle's order) before the sigmoid.  The
// small stages keep five CTAs resident per SM.
template <bool kAct>
__global__ void __launch_bounds__(256, 5) k_compose(const float* __restrict__ levels, int T, int r_min, int r_max,
                                                    int C, float* __restrict__ out, float* __restrict__ act_a) {
    extern __shared__ __align__(16) float smem[];
    const int Nf = 1 << r_max, Vf = level_V(r_max), L = r_max - r_min;   // L >= 1 coarse levels
    uint2* taps = reinterpret_cast<uint2*>(smem);                           // [L][Vf]
    const int tap_floats = (2 * L * Vf + 3) & ~3;
    const int sf = stage_floats(r_min, r_max - 1, C);                      // coarse levels of one triangle
    float* const stage0 = smem + tap_floats;                               // stage b at stage0 + b * sf
    size_t fine_off = 0;                                                   // the finest level in `levels`
    for (int R = r_min; R < r_max; ++R) fine_off += (size_t)T * level_V(R) * C;
    const int per = C / 4;
    int t = blockIdx.x;
    if (t < T) stage_coarse(stage0, levels, t, T, r_min, r_max, C);
    cp_async_commit();
    for (int q = threadIdx.x; q < L * Vf; q += blockDim.x) {
        const int l = q / Vf, v = q - l * Vf;
        int i, j;
        texel_ij(Nf, v, i, j);
        taps[q] = make_tap(r_min + l, i, j, Nf, r_max);
    }
    int buf = 0;
    for (; t < T; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tn < T) stage_coarse(stage0 + (buf ^ 1) * sf, levels, tn, T, r_min, r_max, C);
        cp_async_commit();
        cp_async_wait<1>();   // this thread's copies of triangle t have landed
        __syncthreads();      // everyone's (and the taps)
        const float* zs = stage0 + buf * sf;
        const float* fine = levels + fine_off + (size_t)t * Vf * C;
        for (int it = threadIdx.x; it < Vf * per; it += blockDim.x) {
            const int v = it / per, c = (it - v * per) * 4;
            const float4 y = __ldcs(reinterpret_cast<const float4*>(fine + (size_t)v * C + c));
            float4 z = tap_value(zs, taps[v], C, c);
            int so = level_V(r_min) * C;
            for (int l = 1; l < L; ++l) {
                z = add4(z, tap_value(zs + so, taps[l * Vf + v], C, c));
                so += level_V(r_min + l) * C;
            }
            z = add4(z, y);
            if (kAct) {
                z = make_float4(sigmoid_rcp(z.x), sigmoid_rcp(z.y), sigmoid_rcp(z.z), sigmoid_rcp(z.w));
                if (c + 4 == C && act_a) act_a[(size_t)t * Vf + v] = z.w;
            }
            __stcs(reinterpret_cast<float4*>(out + ((size_t)t * Vf + v) * C + c), z);
        }
        __syncthreads();      // stage[buf] is refilled next round
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// Any C or alignment: one CTA per triangle, the levels staged with plain
// loads, one (finest vertex, channel) per item; the same sum in the same
// order.
template <bool kAct>
__global__ void __launch_bounds__(256) k_compose_scalar(const float* __restrict__ levels, int T, int r_min, int r_max,
                                                        int C, float* __restrict__ out, float* __restrict__ act_a) {
    extern __shared__ __align__(16) float zs[];   // levels r_min..r_max of triangle t, one after the other
    const int t = blockIdx.x;
    {
        size_t off = 0;
        int so = 0;
        for (int R = r_min; R <= r_max; ++R) {
            const int n = level_V(R) * C;
            const float* g = levels + off + (size_t)t * n;
            for (int k = threadIdx.x; k < n; k += blockDim.x) zs[so + k] = __ldcs(g + k);
            off += (size_t)T * n;
            so += n;
        }
    }
    __syncthreads();
    const int Nf = 1 << r_max, Vf = level_V(r_max);
    for (int it = threadIdx.x; it < Vf * C; it += blockDim.x) {
        const int v = it / C, c = it - v * C;
        int i, j;
        texel_ij(Nf, v, i, j);
        float z = level_at<false>(zs, r_min, C, c, i, j, Nf, r_max).x;
        int so = level_V(r_min) * C;
        for (int R = r_min + 1; R <= r_max; ++R) {
            z = __fadd_rn(z, level_at<false>(zs + so, R, C, c, i, j, Nf, r_max).x);
            so += level_V(R) * C;
        }
        if (kAct) {
            z = pinned_sigmoid(z);
            if (c == C - 1 && act_a) act_a[(size_t)t * Vf + v] = z;
        }
        out[((size_t)t * Vf + v) * C + c] = z;
    }
}

// A single level (r_min == r_max): the level itself (or its sigmoid).
template <bool kAct>
__global__ void __launch_bounds__(256) k_compose_single(const float* __restrict__ g, long long n, int C,
                                                        float* __restrict__ out, float* __restrict__ act_a) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float z = __ldg(g + k);
        if (kAct) {
            z = pinned_sigmoid(z);
            if (act_a && k % C == C - 1) act_a[k / C] = z;
        }
        out[k] = z;
    }
}

// The adjoint's value k of level R (N = 2^R subdivisions) from the gradient
// G of level R + 1 ([V][C]): the hat function of the coarse vertex on the
// fine grid, weight 1 at the coincident vertex and 1/2 at its six
// neighbours.
__device__ __forceinline__ float restrict_value(const float* G, int N, int k, int C) {
    const int Nfine = 2 * N;
    const int u = k / C, c = k - u * C;
    int a, b;
    texel_ij(N, u, a, b);
    const int x = 2 * a, y = 2 * b;
    float acc = G[(size_t)texel_index(Nfine, x, y) * C + c];
    float half = 0.f;
    const int dx[6] = {1, -1, 0, 0, 1, -1}, dy[6] = {0, 0, 1, -1, -1, 1};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int xi = x + dx[e], yi = y + dy[e];
        if (xi >= 0 && yi >= 0 && xi + yi <= Nfine) half += G[(size_t)texel_index(Nfine, xi, yi) * C + c];
    }
    return fmaf(0.5f, half, acc);
}

// Adjoint of the composition for one triangle per CTA.  fine: FP64 gradient
// of the composed logits [T][V_f][C]; out: the level gradients (same layout
// as the levels), written or accumulated.
__global__ void __launch_bounds__(256) k_restrict(const double* __restrict__ fine, int T, int r_min, int r_max, int C,
                                                  float* __restrict__ out, int overwrite) {
    extern __shared__ float sm[];
    const int t = blockIdx.x;
    const int Vf = level_V(r_max);
    float* A = sm;                               // current (finer) level [V][C]
    float* B = sm + (size_t)Vf * C;              // next (coarser) level
    // level offsets in `out`
    size_t off[6];
    {
        size_t o = 0;
        for (int R = r_min; R <= r_max; ++R) {
            off[R - r_min] = o;
            o += (size_t)T * level_V(R) * C;
        }
    }
    {
        // the finest level: eight loads in flight per thread before they are used
        const double* src = fine + (size_t)t * Vf * C;
        float* dst = out + off[r_max - r_min] + (size_t)t * Vf * C;
        const int n = Vf * C;
        for (int k0 = threadIdx.x; k0 < n; k0 += 8 * blockDim.x) {
            double g[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * blockDim.x;
                g[u] = k < n ? __ldcs(src + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * blockDim.x;
                if (k < n) {
                    A[k] = (float)g[u];
                    dst[k] = overwrite ? (float)g[u] : (float)((double)dst[k] + g[u]);
                }
            }
        }
    }
    __syncthreads();
    for (int R = r_max - 1; R >= r_min; --R) {
        const int V = level_V(R);
        float* dst = out + off[R - r_min] + (size_t)t * V * C;
        for (int k = threadIdx.x; k < V * C; k += blockDim.x) {
            const float acc = restrict_value(A, 1 << R, k, C);
            B[k] = acc;
            dst[k] = overwrite ? acc : dst[k] + acc;
        }
        __syncthreads();
        float* tmp = A;
        A = B;
        B = tmp;
    }
}

// The adjoint staged in shared memory, one triangle per CTA: the gradients
// of all its levels (the FP32 values k_restrict writes with overwrite) are
// formed there level after level; then each level's block of the triangle --
// contiguous in the levels' layout -- leaves as a float4 stream: written to
// `out` (kAdam false), or, with the levels' Adam step fused (Sec. 3.4),
// applied to x, m and v so that the gradient never reaches memory.
template <bool kAdam>
__global__ void __launch_bounds__(256) k_restrict_staged(const double* __restrict__ fine, int T, int r_min, int r_max,
                                                         int C, float* __restrict__ out, AdamTex adam) {
    extern __shared__ float sm[];   // the levels' gradients of this triangle, finest first
    const int t = blockIdx.x;
    size_t off[6];
    int soff[6];
    {
        size_t o = 0;
        int so = 0;
        for (int R = r_min; R <= r_max; ++R) {
            off[R - r_min] = o;
            o += (size_t)T * level_V(R) * C;
        }
        for (int R = r_max; R >= r_min; --R) {
            soff[R - r_min] = so;
            so += level_V(R) * C;
        }
    }
    {
        const int n = level_V(r_max) * C;
        const double* src = fine + (size_t)t * n;
        float* G = sm + soff[r_max - r_min];
        for (int k0 = threadIdx.x; k0 < n; k0 += 8 * blockDim.x) {
            double g[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * blockDim.x;
                g[u] = k < n ? __ldcs(src + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * blockDim.x;
                if (k < n) G[k] = (float)g[u];
            }
        }
    }
    __syncthreads();
    for (int R = r_max - 1; R >= r_min; --R) {
        const float* Gf = sm + soff[R + 1 - r_min];
        float* G = sm + soff[R - r_min];
        const int n = level_V(R) * C;
        for (int k = threadIdx.x; k < n; k += blockDim.x) G[k] = restrict_value(Gf, 1 << R, k, C);
        __syncthreads();
    }
    // each level's block, four values per access (the block starts on a
    // 16-byte boundary: C and the level offsets are multiples of 4)
    for (int R = r_max; R >= r_min; --R) {
        const int n4 = level_V(R) * C / 4;
        const size_t base4 = (off[R - r_min] + (size_t)t * level_V(R) * C) / 4;
        const float4* G4 = reinterpret_cast<const float4*>(sm + soff[R - r_min]);
        if (!kAdam) {
            float4* O = reinterpret_cast<float4*>(out) + base4;
            for (int q = threadIdx.x; q < n4; q += blockDim.x) __stcs(O + q, G4[q]);
            continue;
        }
        float4* X = reinterpret_cast<float4*>(adam.x) + base4;
        float4* M = reinterpret_cast<float4*>(adam.m) + base4;
        float4* Vv = reinterpret_cast<float4*>(adam.v) + base4;
        for (int q = threadIdx.x; q < n4; q += blockDim.x) {
            const float4 g = G4[q];
            float4 x = X[q], m = __ldcs(M + q), v = __ldcs(Vv + q);
            adam_apply(x.x, m.x, v.x, g.x, adam.a);
            adam_apply(x.y, m.y, v.y, g.y, adam.a);
            adam_apply(x.z, m.z, v.z, g.z, adam.a);
            adam_apply(x.w, m.w, v.w, g.w, adam.a);
            X[q] = x;
            __stcs(M + q, m);
            __stcs(Vv + q, v);
        }
    }
}

__global__ void __launch_bounds__(256) k_resample(const float* __restrict__ src, int T, int r_src, int C,
                                                  float* __restrict__ dst, int r_dst) {
    const int Nd = 1 << r_dst, Vd = level_V(r_dst), Vs = level_V(r_src);
    const long long n = (long long)T * Vd;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += stride) {
        const int t = (int)(q / Vd), v = (int)(q - (long long)t * Vd);
        int i, j;
        texel_ij(Nd, v, i, j);
        const float* g = src + (size_t)t * Vs * C;
        for (int c = 0; c < C; ++c)
            dst[(size_t)q * C + c] = r_src == r_dst ? __ldg(g + (size_t)v * C + c) : level_value(g, r_src, C, c, i, j, Nd);
    }
}

int flat_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t level_floats(int T, int r_min, int r_max, int C) {
    size_t n = 0;
    for (int R = r_min; R <= r_max; ++R) n += (size_t)T * level_V(R) * C;
    return n;
}

cudaError_t launch_compose(const float* levels, int T, int r_min, int r_max, int C, float* out, bool act,
                           float* act_a, cudaStream_t st) {
    if (r_min == r_max) {
        const long long n = (long long)T * level_V(r_max) * C;
        if (act)
            k_compose_single<true><<<flat_grid(n), 256, 0, st>>>(levels, n, C, out, act_a);
        else
            k_compose_single<false><<<flat_grid(n), 256, 0, st>>>(levels, n, C, out, nullptr);
    } else if ((C % 4 == 0) && ((uintptr_t)levels % 16 == 0) && ((uintptr_t)out % 16 == 0)) {
        const int Vf = level_V(r_max), L = r_max - r_min;
        const size_t smem = sizeof(float) * ((size_t)((2 * L * Vf + 3) & ~3) + 2 * (size_t)stage_floats(r_min, r_max - 1, C));
        auto run = [&](auto kernel) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
            if (e != cudaSuccess) return e;
            const int grid = persistent_grid(T, per_sm < 1 ? 1 : per_sm);
            kernel<<<grid, 256, smem, st>>>(levels, T, r_min, r_max, C, out, act ? act_a : nullptr);
            return cudaSuccess;
        };
        cudaError_t e = act ? run(k_compose<true>) : run(k_compose<false>);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem = sizeof(float) * (size_t)stage_floats(r_min, r_max, C);
        auto run = [&](auto kernel) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            kernel<<<T, 256, smem, st>>>(levels, T, r_min, r_max, C, out, act ? act_a : nullptr);
            return cudaSuccess;
        };
        cudaError_t e = act ? run(k_compose_scalar<true>) : run(k_compose_scalar<false>);
        if (e != cudaSuccess) return e;
    }
    note_launches(1);
    return cudaGetLastError();
}

template <bool kAdam>
static cudaError_t run_staged(const double* fine, int T, int r_min, int r_max, int C, float* out, const AdamTex& adam,
                              cudaStream_t st) {
    size_t per_tri = 0;
    for (int R = r_min; R <= r_max; ++R) per_tri += (size_t)level_V(R) * C;
    const size_t smem = sizeof(float) * per_tri;
    cudaError_t e = cudaFuncSetAttribute(k_restrict_staged<kAdam>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_restrict_staged<kAdam><<<T, 256, smem, st>>>(fine, T, r_min, r_max, C, out, adam);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_restrict(const double* fine, int T, int r_min, int r_max, int C, float* out, bool overwrite,
                            cudaStream_t st) {
    // overwrite with a 16-byte-aligned output and C a multiple of 4: the
    // staged kernel (float4 stores); otherwise the per-level one
    if (overwrite && C % 4 == 0 && ((uintptr_t)out & 15) == 0)
        return run_staged<false>(fine, T, r_min, r_max, C, out, AdamTex{}, st);
    const size_t smem = sizeof(float) * (size_t)(level_V(r_max) + level_V(r_max > 0 ? r_max - 1 : 0)) * C;
    cudaError_t e = cudaFuncSetAttribute(k_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_restrict<<<T, 256, smem, st>>>(fine, T, r_min, r_max, C, out, overwrite ? 1 : 0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_restrict_adam(const double* fine, int T, int r_min, int r_max, int C, const AdamTex& adam,
                                 cudaStream_t st) {
    if (C % 4 != 0 || (((uintptr_t)adam.x | (uintptr_t)adam.m | (uintptr_t)adam.v) & 15) != 0)
        return cudaErrorInvalidValue;
    return run_staged<true>(fine, T, r_min, r_max, C, nullptr, adam, st);
}

cudaError_t launch_resample(const float* src, int T, int r_src, int C, float* dst, int r_dst, cudaStream_t st) {
    k_resample<<<flat_grid((long long)T * level_V(r_dst)), 256, 0, st>>>(src, T, r_src, C, dst, r_dst);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ds
