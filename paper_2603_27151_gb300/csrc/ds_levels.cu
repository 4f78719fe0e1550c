// ds_levels.cu -- multi-resolution feature grids (Sec. 3.3, multi-resolution
// mesh colours; supplementary "Coarse-to-Fine Optimization").
//
// Level R carries a mesh-colour grid with N_R = 2^R subdivisions per edge and
// V_R = (N_R+1)(N_R+2)/2 feature vertices; a soup's levels r_min..r_max are
// stored one after the other, level R as [T][V_R][C].  The texture that is
// rasterised is the finest grid (N = 2^r_max) whose logits are the sum of all
// levels evaluated at its vertices, then the sigmoid:
//  - k_compose (fused into the activation step): one CTA per triangle.  The
//    level-R function is piecewise linear on level R+1's mesh (same diagonal
//    orientation), so the levels are accumulated coarse to fine in shared
//    memory, z_R = P(z_(R-1)) + level R, P the 2x prolongation (the
//    coinciding vertex or a coarse edge's midpoint value), FP32 in the
//    oracle's order; the finest level goes straight to the sigmoid;
//  - k_restrict (fused into the gradient finish step): the adjoint.  The
//    level-R function is piecewise linear on level R+1's mesh (same diagonal
//    orientation), so the composition is a chain of 2x prolongations and its
//    adjoint a chain of 2x restrictions: each coarse vertex gathers its fine
//    twin and, with weight 1/2, the midpoints of its six incident edges.  One
//    CTA per triangle, levels in shared memory, FP32 from the FP64
//    accumulator of the finest grid;
//  - k_resample: one level's grid sampled at another level's vertices.
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

// Prolongation of channel c of the level grid z (N/2 subdivisions) to vertex
// (i, j) of the N-subdivided grid: the coinciding vertex, or the midpoint
// value fmaf(0.5, z_q - z_p, z_p) of the coarse edge the vertex bisects (p =
// the endpoint with the lower texel index).
__device__ __forceinline__ void prolong_taps(int Nc, int i, int j, int& p, int& q) {
    const int a = i >> 1, b = j >> 1;
    if (!(i & 1) && !(j & 1)) { p = q = texel_index(Nc, a, b); }
    else if ((i & 1) && !(j & 1)) { p = texel_index(Nc, a, b); q = texel_index(Nc, a + 1, b); }
    else if (!(i & 1)) { p = texel_index(Nc, a, b); q = texel_index(Nc, a, b + 1); }
    else { p = texel_index(Nc, a + 1, b); q = texel_index(Nc, a, b + 1); }
}

__device__ __forceinline__ float prolong(float zp, float zq, bool coincide) {
    return coincide ? zp : __fmaf_rn(0.5f, __fsub_rn(zq, zp), zp);
}

// One CTA per triangle.  The coarse levels are accumulated coarse to fine in
// shared memory (z_R = P(z_(R-1)) + level R, FP32 in the oracle's order); the
// finest level is formed on the fly and written as the composed logits, or
// their sigmoid with the planar opacity copy.  Items are (vertex, group of
// four channels) when vec (C % 4 == 0 and 16-byte aligned levels and
// output), else (vertex, channel).
template <bool kAct>
__global__ void __launch_bounds__(256) k_compose(const float* __restrict__ levels, int T, int r_min, int r_max, int C,
                                                 int vec, float* __restrict__ out, float* __restrict__ act_a) {
    extern __shared__ __align__(16) float zs[];   // two buffers of V_(r_max - 1) * C
    const int t = blockIdx.x;
    const int Vc = r_max > 0 ? level_V(r_max - 1) : 1;
    float* cur = zs;
    float* nxt = zs + (size_t)Vc * C;
    const int per = vec ? C / 4 : C;              // items per vertex
    size_t off = 0;
    // z_(r_min) = level r_min (only when a coarser level feeds a finer one)
    if (r_min < r_max) {
        const float* g = levels + (size_t)t * level_V(r_min) * C;
        for (int k = threadIdx.x; k < level_V(r_min) * C; k += blockDim.x) cur[k] = __ldg(g + k);
    }
    off += (size_t)T * level_V(r_min) * C;
    __syncthreads();
    for (int R = r_min + 1; R <= r_max; ++R) {
        const int N = 1 << R, V = level_V(R);
        const float* g = levels + off + (size_t)t * V * C;
        const bool last = R == r_max;
        for (int it = threadIdx.x; it < V * per; it += blockDim.x) {
            const int v = it / per, cg = it - v * per;
            int i, j, p, q;
            texel_ij(N, v, i, j);
            prolong_taps(N >> 1, i, j, p, q);
            const bool co = p == q;
            if (vec) {
                const int c = 4 * cg;
                const float4 zp = *reinterpret_cast<const float4*>(cur + (size_t)p * C + c);
                const float4 zq = *reinterpret_cast<const float4*>(cur + (size_t)q * C + c);
                const float4 th = __ldg(reinterpret_cast<const float4*>(g + (size_t)v * C + c));
                float4 z = make_float4(__fadd_rn(prolong(zp.x, zq.x, co), th.x), __fadd_rn(prolong(zp.y, zq.y, co), th.y),
                                       __fadd_rn(prolong(zp.z, zq.z, co), th.z), __fadd_rn(prolong(zp.w, zq.w, co), th.w));
                if (!last) {
                    *reinterpret_cast<float4*>(nxt + (size_t)v * C + c) = z;
                } else {
                    if (kAct) {
                        z = make_float4(pinned_sigmoid(z.x), pinned_sigmoid(z.y), pinned_sigmoid(z.z),
                                        pinned_sigmoid(z.w));
                        if (c + 4 == C && act_a) act_a[(size_t)t * V + v] = z.w;
                    }
                    *reinterpret_cast<float4*>(out + ((size_t)t * V + v) * C + c) = z;
                }
            } else {
                const int c = cg;
                float z = __fadd_rn(prolong(cur[(size_t)p * C + c], cur[(size_t)q * C + c], co),
                                    __ldg(g + (size_t)v * C + c));
                if (!last) {
                    nxt[(size_t)v * C + c] = z;
                } else {
                    if (kAct) {
                        z = pinned_sigmoid(z);
                        if (c == C - 1 && act_a) act_a[(size_t)t * V + v] = z;
                    }
                    out[((size_t)t * V + v) * C + c] = z;
                }
            }
        }
        off += (size_t)T * V * C;
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
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
        const int N = 1 << R, Nfine = 2 * N, V = level_V(R);
        float* dst = out + off[R - r_min] + (size_t)t * V * C;
        for (int k = threadIdx.x; k < V * C; k += blockDim.x) {
            const int u = k / C, c = k - u * C;
            int a, b;
            texel_ij(N, u, a, b);
            const int x = 2 * a, y = 2 * b;
            float acc = A[(size_t)texel_index(Nfine, x, y) * C + c];
            float half = 0.f;
            const int dx[6] = {1, -1, 0, 0, 1, -1}, dy[6] = {0, 0, 1, -1, -1, 1};
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const int xi = x + dx[e], yi = y + dy[e];
                if (xi >= 0 && yi >= 0 && xi + yi <= Nfine) half += A[(size_t)texel_index(Nfine, xi, yi) * C + c];
            }
            acc = fmaf(0.5f, half, acc);
            B[k] = acc;
            dst[k] = overwrite ? acc : dst[k] + acc;
        }
        __syncthreads();
        float* tmp = A;
        A = B;
        B = tmp;
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
    } else {
        const size_t smem = sizeof(float) * 2 * (size_t)level_V(r_max - 1) * C;
        const int vec = (C % 4 == 0) && ((uintptr_t)levels % 16 == 0) && ((uintptr_t)out % 16 == 0);
        if (act)
            k_compose<true><<<T, 256, smem, st>>>(levels, T, r_min, r_max, C, vec, out, act_a);
        else
            k_compose<false><<<T, 256, smem, st>>>(levels, T, r_min, r_max, C, vec, out, nullptr);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_restrict(const double* fine, int T, int r_min, int r_max, int C, float* out, bool overwrite,
                            cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)(level_V(r_max) + level_V(r_max > 0 ? r_max - 1 : 0)) * C;
    cudaError_t e = cudaFuncSetAttribute(k_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_restrict<<<T, 256, smem, st>>>(fine, T, r_min, r_max, C, out, overwrite ? 1 : 0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_resample(const float* src, int T, int r_src, int C, float* dst, int r_dst, cudaStream_t st) {
    k_resample<<<flat_grid((long long)T * level_V(r_dst)), 256, 0, st>>>(src, T, r_src, C, dst, r_dst);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ds
