// ds_levels.cu -- multi-resolution feature grids (Sec. 3.3, multi-resolution
// mesh colours; supplementary "Coarse-to-Fine Optimization").
//
// Level R carries a mesh-colour grid with N_R = 2^R subdivisions per edge and
// V_R = (N_R+1)(N_R+2)/2 feature vertices; a soup's levels r_min..r_max are
// stored one after the other, level R as [T][V_R][C].  The texture that is
// rasterised is the finest grid (N = 2^r_max) whose logits are the sum of all
// levels evaluated at its vertices, then the sigmoid:
//  - k_compose (fused into the activation step): one thread per (triangle,
//    finest vertex), all C channels; a vertex that coincides with a level
//    vertex takes its value, any other point is interpolated in the level's
//    micro-triangle containing it (the decode's cell and arithmetic), levels
//    summed in ascending order in FP32;
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

// Where the level-R grid is read for vertex (i, j) of the finest grid
// (N = 2^r_max > N_R): a coinciding vertex (direct) or a micro-triangle.
struct LevelTap {
    Cell cl;
    bool direct;
};

__device__ __forceinline__ LevelTap level_tap(int R, int i, int j, int N) {
    const int NR = 1 << R, s = N / NR;
    LevelTap tp;
    tp.direct = (i % s == 0) && (j % s == 0);
    if (tp.direct) {
        tp.cl.k0 = tp.cl.k1 = tp.cl.k2 = texel_index(NR, i / s, j / s);
        tp.cl.wa = tp.cl.wb = 0.f;
        tp.cl.lower = true;
    } else {
        // i / N by the exact power-of-two reciprocal: the same value as the division
        const float inv = __int_as_float((127 - __ffs(N) + 1) << 23);
        tp.cl = find_cell(NR, __fmul_rn((float)i, inv), __fmul_rn((float)j, inv));
    }
    return tp;
}

__device__ __forceinline__ float tap_value(const float* __restrict__ g, const LevelTap& tp, int C, int c) {
    const float a0 = __ldg(g + (size_t)tp.cl.k0 * C + c);
    if (tp.direct) return a0;
    return interp(a0, __ldg(g + (size_t)tp.cl.k1 * C + c), __ldg(g + (size_t)tp.cl.k2 * C + c), tp.cl.wa, tp.cl.wb);
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}

// Four consecutive channels c..c+3 of a level at a tap (same arithmetic as
// tap_value, channel by channel).
__device__ __forceinline__ float4 tap_value4(const float* __restrict__ g, const LevelTap& tp, int C, int c) {
    const float4 a0 = ld4(g + (size_t)tp.cl.k0 * C + c);
    if (tp.direct) return a0;
    const float4 a1 = ld4(g + (size_t)tp.cl.k1 * C + c), a2 = ld4(g + (size_t)tp.cl.k2 * C + c);
    const float wa = tp.cl.wa, wb = tp.cl.wb;
    return make_float4(interp(a0.x, a1.x, a2.x, wa, wb), interp(a0.y, a1.y, a2.y, wa, wb),
                       interp(a0.z, a1.z, a2.z, wa, wb), interp(a0.w, a1.w, a2.w, wa, wb));
}

// NL = r_max - r_min coarser levels below the finest.  kAct: act =
// sigmoid(composed logits) (+ the planar opacity copy); else the composed
// logits themselves.  kVec: C % 4 == 0 and 16-byte aligned levels and output:
// channels move as float4.
template <int NL, bool kAct, bool kVec>
__global__ void __launch_bounds__(256) k_compose(const float* __restrict__ levels, int T, int r_max, int C,
                                                 float* __restrict__ out, float* __restrict__ act_a) {
    const int r_min = r_max - NL;
    const int Nf = 1 << r_max, Vf = level_V(r_max);
    // (i, j) of every finest vertex, packed i | j << 8
    __shared__ unsigned short ij_of[level_V(5)];
    for (int v = threadIdx.x; v < Vf; v += blockDim.x) {
        int i, j;
        texel_ij(Nf, v, i, j);
        ij_of[v] = (unsigned short)(i | (j << 8));
    }
    __syncthreads();
    const long long n = (long long)T * Vf;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += stride) {
        const int t = (int)(q / Vf), v = (int)(q - (long long)t * Vf);
        const int i = ij_of[v] & 0xff, j = ij_of[v] >> 8;
        LevelTap tp[NL > 0 ? NL : 1];
        const float* g[NL + 1];
        size_t off = 0;
#pragma unroll
        for (int k = 0; k <= NL; ++k) {
            const int R = r_min + k;
            g[k] = levels + off + (size_t)t * level_V(R) * C;
            if (k < NL) tp[k] = level_tap(R, i, j, Nf);
            off += (size_t)T * level_V(R) * C;
        }
        float* o = out + (size_t)q * C;
        if (kVec) {
            for (int c = 0; c < C; c += 4) {
                float4 z = NL > 0 ? tap_value4(g[0], tp[0], C, c) : ld4(g[0] + (size_t)v * C + c);
#pragma unroll
                for (int k = 1; k < NL; ++k) z = add4(z, tap_value4(g[k], tp[k], C, c));
                if (NL > 0) z = add4(z, ld4(g[NL] + (size_t)v * C + c));
                if (kAct) {
                    z = make_float4(pinned_sigmoid(z.x), pinned_sigmoid(z.y), pinned_sigmoid(z.z), pinned_sigmoid(z.w));
                    if (c + 4 == C && act_a) act_a[q] = z.w;
                }
                *reinterpret_cast<float4*>(o + c) = z;
            }
        } else {
            for (int c = 0; c < C; ++c) {
                float z = NL > 0 ? tap_value(g[0], tp[0], C, c) : __ldg(g[0] + (size_t)v * C + c);
#pragma unroll
                for (int k = 1; k < NL; ++k) z = __fadd_rn(z, tap_value(g[k], tp[k], C, c));
                if (NL > 0) z = __fadd_rn(z, __ldg(g[NL] + (size_t)v * C + c));
                if (kAct) {
                    const float a = pinned_sigmoid(z);
                    o[c] = a;
                    if (c == C - 1 && act_a) act_a[q] = a;
                } else {
                    o[c] = z;
                }
            }
        }
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

template <int NL>
void compose_nl(const float* levels, int T, int r_max, int C, float* out, bool act, float* act_a, int g,
                cudaStream_t st) {
    const bool vec = C % 4 == 0 && (uintptr_t)levels % 16 == 0 && (uintptr_t)out % 16 == 0;
    if (act && vec)
        k_compose<NL, true, true><<<g, 256, 0, st>>>(levels, T, r_max, C, out, act_a);
    else if (act)
        k_compose<NL, true, false><<<g, 256, 0, st>>>(levels, T, r_max, C, out, act_a);
    else if (vec)
        k_compose<NL, false, true><<<g, 256, 0, st>>>(levels, T, r_max, C, out, nullptr);
    else
        k_compose<NL, false, false><<<g, 256, 0, st>>>(levels, T, r_max, C, out, nullptr);
}

cudaError_t launch_compose(const float* levels, int T, int r_min, int r_max, int C, float* out, bool act,
                           float* act_a, cudaStream_t st) {
    const int g = flat_grid((long long)T * level_V(r_max));
    switch (r_max - r_min) {
        case 0: compose_nl<0>(levels, T, r_max, C, out, act, act_a, g, st); break;
        case 1: compose_nl<1>(levels, T, r_max, C, out, act, act_a, g, st); break;
        case 2: compose_nl<2>(levels, T, r_max, C, out, act, act_a, g, st); break;
        case 3: compose_nl<3>(levels, T, r_max, C, out, act, act_a, g, st); break;
        case 4: compose_nl<4>(levels, T, r_max, C, out, act, act_a, g, st); break;
        default: compose_nl<5>(levels, T, r_max, C, out, act, act_a, g, st); break;
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
