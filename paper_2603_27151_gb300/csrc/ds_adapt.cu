// ds_adapt.cu -- adaptive control of primitives (Sec. 3.4 "Adaptive control
// of primitives"): the GPU measurements that drive it and the rebuild of the
// soup after a round of edge splits and prunes.
//  - k_coverage: pixel-samples won per triangle, from the G-buffers' triangle
//    ids; lanes holding the same id are merged with one match-any vote and
//    a single atomic per id and warp.
//  - k_edge_ratios: per triangle, each edge's largest projected length over
//    the views (those where the triangle lies in front of the near plane and
//    its projected bounding box meets the image), relative to the image
//    height; FP32 in the oracle's order, so that the split decision is the
//    same on both sides.
//  - the plan (host C++): split the longest edge above the threshold, then
//    remove the lowest-coverage triangles until the budget holds; or, for
//    the random initialisation of the supplementary material, remove the
//    uncovered triangles and split the longest edges up to a target count.
//  - k_rebuild_verts / k_rebuild_level: the new soup: copies, or the two
//    children of a split edge (midpoint in FP32), each child's grid sampled
//    from the parent's grid at the child's vertices mapped into the parent.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ds_internal.h"

namespace ds {

namespace {

struct CoverView {
    const int4* gbuf;   // [S][H][W] texels; .x = triangle id
    long long n;        // S * H * W
};
struct CoverTable {
    int n_views, T;
    CoverView v[DS_MAX_VIEWS];
};

__global__ void __launch_bounds__(256) k_coverage(const __grid_constant__ CoverTable ct, int* __restrict__ counts) {
    const CoverView& V = ct.v[blockIdx.y];
    for (long long base = (long long)blockIdx.x * blockDim.x; base < V.n; base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + threadIdx.x;
        int id = -1;
        if (k < V.n) id = __ldg(&V.gbuf[k].x);
        if (id >= ct.T) id = -1;
        const unsigned same = __match_any_sync(0xffffffffu, id);
        const int lead = __ffs(same) - 1;
        if (id >= 0 && (int)(threadIdx.x & 31) == lead) atomicAdd(counts + id, __popc(same));
    }
}

struct RatioCam {
    float fx, fy, cx, cy, R[9], t[3], near_z;
    int W, H;
};
struct RatioTable {
    int n_views;
    RatioCam c[DS_MAX_VIEWS];
};

__global__ void __launch_bounds__(256) k_edge_ratios(const __grid_constant__ RatioTable rt, const float* __restrict__ verts,
                                                     int T, float* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    float p[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = __ldg(verts + 9 * (size_t)t + k);
    float best[3] = {0.f, 0.f, 0.f};
    for (int v = 0; v < rt.n_views; ++v) {
        const RatioCam& c = rt.c[v];
        float sx[3], sy[3];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float* q = p + 3 * i;
            const float xc = __fmaf_rn(c.R[0], q[0], __fmaf_rn(c.R[1], q[1], __fmaf_rn(c.R[2], q[2], c.t[0])));
            const float yc = __fmaf_rn(c.R[3], q[0], __fmaf_rn(c.R[4], q[1], __fmaf_rn(c.R[5], q[2], c.t[1])));
            const float zc = __fmaf_rn(c.R[6], q[0], __fmaf_rn(c.R[7], q[1], __fmaf_rn(c.R[8], q[2], c.t[2])));
            ok = ok && (zc > c.near_z);
            sx[i] = __fmaf_rn(c.fx, __fdiv_rn(xc, zc), c.cx);
            sy[i] = __fmaf_rn(c.fy, __fdiv_rn(yc, zc), c.cy);
        }
        if (!ok) continue;
        const float x0 = fminf(sx[0], fminf(sx[1], sx[2])), x1 = fmaxf(sx[0], fmaxf(sx[1], sx[2]));
        const float y0 = fminf(sy[0], fminf(sy[1], sy[2])), y1 = fmaxf(sy[0], fmaxf(sy[1], sy[2]));
        if (x1 < 0.0f || x0 > (float)c.W || y1 < 0.0f || y0 > (float)c.H) continue;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = e, b = (e + 1) % 3;
            const float dx = __fsub_rn(sx[b], sx[a]), dy = __fsub_rn(sy[b], sy[a]);
            const float r = __fdiv_rn(__fsqrt_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))), (float)c.H);
            best[e] = r > best[e] ? r : best[e];
        }
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) out[3 * (size_t)t + e] = best[e];
}

// The child's corners in the parent's barycentrics, doubled (integers).
__device__ __forceinline__ void child_corners(int op, int P[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) P[i][q] = 2 * (i == q);
    if (op == 0) return;
    const int e = (op - 1) >> 1, c = (op - 1) & 1;
    const int a = e, b = (e + 1) % 3, o = (e + 2) % 3;
    int Q[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int pa = q == a ? 2 : 0, pb = q == b ? 2 : 0, pm = (q == a || q == b) ? 1 : 0, po = q == o ? 2 : 0;
        Q[0][q] = c == 0 ? pa : pm;
        Q[1][q] = c == 0 ? pm : pb;
        Q[2][q] = po;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) P[i][q] = Q[i][q];
}

__global__ void __launch_bounds__(256) k_rebuild_level(const float* __restrict__ gin, int N, int C,
                                                       const int* __restrict__ plan, int n_out,
                                                       float* __restrict__ gout) {
    const int V = (N + 1) * (N + 2) / 2;
    const long long n = (long long)n_out * V;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / V), v = (int)(q - (long long)k * V);
        int j = 0;
        while (j < N && texel_index(N, 0, j + 1) <= v) ++j;
        const int i = v - texel_index(N, 0, j);
        const int code = __ldg(plan + k), parent = code >> 3, op = code & 7;
        int P[3][3];
        child_corners(op, P);
        const int X = (N - i - j) * P[0][1] + i * P[1][1] + j * P[2][1];
        const int Y = (N - i - j) * P[0][2] + i * P[1][2] + j * P[2][2];
        const float* g = gin + (size_t)parent * V * C;
        float* d = gout + (size_t)q * C;
        if ((X & 1) == 0 && (Y & 1) == 0) {
            const float* s = g + (size_t)texel_index(N, X >> 1, Y >> 1) * C;
            for (int c = 0; c < C; ++c) d[c] = __ldg(s + c);
        } else {
            const Cell cl = find_cell(N, __fdiv_rn((float)X, (float)(2 * N)), __fdiv_rn((float)Y, (float)(2 * N)));
            for (int c = 0; c < C; ++c)
                d[c] = interp(__ldg(g + (size_t)cl.k0 * C + c), __ldg(g + (size_t)cl.k1 * C + c),
                              __ldg(g + (size_t)cl.k2 * C + c), cl.wa, cl.wb);
        }
    }
}

__global__ void __launch_bounds__(256) k_rebuild_verts(const float* __restrict__ vin, const int* __restrict__ plan,
                                                       int n_out, float* __restrict__ vout) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_out) return;
    const int code = __ldg(plan + k), parent = code >> 3, op = code & 7;
    const float* s = vin + 9 * (size_t)parent;
    float* d = vout + 9 * (size_t)k;
    if (op == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = __ldg(s + q);
        return;
    }
    const int e = (op - 1) >> 1, c = (op - 1) & 1;
    const int a = e, b = (e + 1) % 3, o = (e + 2) % 3;
    float m[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) m[q] = __fmul_rn(__fadd_rn(__ldg(s + 3 * a + q), __ldg(s + 3 * b + q)), 0.5f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        d[q] = c == 0 ? __ldg(s + 3 * a + q) : m[q];
        d[3 + q] = c == 0 ? m[q] : __ldg(s + 3 * b + q);
        d[6 + q] = __ldg(s + 3 * o + q);
    }
}

int flat_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_coverage(const int4* const* gbufs, const long long* n, int n_views, int T, int* counts,
                            cudaStream_t st) {
    CoverTable ct;
    ct.n_views = n_views;
    ct.T = T;
    long long most = 0;
    for (int v = 0; v < n_views; ++v) {
        ct.v[v].gbuf = gbufs[v];
        ct.v[v].n = n[v];
        most = std::max(most, n[v]);
    }
    if (most == 0) return cudaSuccess;
    const int gx = (int)std::min<long long>((most + 255) / 256, 2048);
    k_coverage<<<dim3(gx, n_views), 256, 0, st>>>(ct, counts);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_edge_ratios(const float* verts, int T, const ds_camera* cams, int n_views, float* out,
                               cudaStream_t st) {
    RatioTable rt;
    rt.n_views = n_views;
    for (int v = 0; v < n_views; ++v) {
        const ds_camera& c = cams[v];
        RatioCam& r = rt.c[v];
        r.fx = c.fx; r.fy = c.fy; r.cx = c.cx; r.cy = c.cy;
        for (int k = 0; k < 9; ++k) r.R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) r.t[k] = c.t[k];
        r.near_z = c.near_z;
        r.W = c.width;
        r.H = c.height;
    }
    k_edge_ratios<<<(T + 255) / 256, 256, 0, st>>>(rt, verts, T, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const float* verts, const float* tex, int T, const int* grid_ns, int n_levels, int C,
                           const int* plan_dev, int n_out, float* verts_out, float* tex_out, cudaStream_t st) {
    if (n_out == 0) return cudaSuccess;
    k_rebuild_verts<<<(n_out + 255) / 256, 256, 0, st>>>(verts, plan_dev, n_out, verts_out);
    note_launches(1);
    size_t off_in = 0, off_out = 0;
    for (int l = 0; l < n_levels; ++l) {
        const int N = grid_ns[l], V = (N + 1) * (N + 2) / 2;
        k_rebuild_level<<<flat_grid((long long)n_out * V), 256, 0, st>>>(tex + off_in, N, C, plan_dev, n_out,
                                                                          tex_out + off_out);
        note_launches(1);
        off_in += (size_t)T * V * C;
        off_out += (size_t)n_out * V * C;
    }
    return cudaGetLastError();
}

// One round of adaptive control on the host (the split/prune policy).
int adapt_plan(const int32_t* counts, const float* ratios, int T, float threshold, long long budget, int32_t* plan) {
    std::vector<int8_t> split(T, -1);
    long long n = T;
    for (int t = 0; t < T; ++t) {
        int e = 0;
        for (int k = 1; k < 3; ++k)
            if (ratios[3 * (size_t)t + k] > ratios[3 * (size_t)t + e]) e = k;
        if (ratios[3 * (size_t)t + e] > threshold) {
            split[t] = (int8_t)e;
            ++n;
        }
    }
    std::vector<char> removed(T, 0);
    if (budget >= 0 && n > budget) {
        std::vector<int> order(T);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return counts[a] < counts[b]; });
        for (int t : order) {
            if (n <= budget) break;
            removed[t] = 1;
            n -= split[t] >= 0 ? 2 : 1;
        }
    }
    int k = 0;
    for (int t = 0; t < T; ++t) {
        if (removed[t]) continue;
        if (split[t] < 0) {
            plan[k++] = t << 3;
        } else {
            plan[k++] = (t << 3) | (1 + 2 * split[t]);
            plan[k++] = (t << 3) | (2 + 2 * split[t]);
        }
    }
    return k;
}

// The random-initialisation round (host): remove the triangles no training
// image covers, then split the longest edges of the survivors with the
// largest ratios (each once) until the target count is reached.
int adapt_plan_fill(const int32_t* counts, const float* ratios, int T, long long target, int32_t* plan) {
    std::vector<int> keep;
    std::vector<int8_t> longest(T, 0);
    for (int t = 0; t < T; ++t) {
        if (counts[t] <= 0) continue;
        keep.push_back(t);
        int e = 0;
        for (int k = 1; k < 3; ++k)
            if (ratios[3 * (size_t)t + k] > ratios[3 * (size_t)t + e]) e = k;
        longest[t] = (int8_t)e;
    }
    long long want = target - (long long)keep.size();
    const size_t n_split = want <= 0 ? 0 : (size_t)std::min<long long>(want, (long long)keep.size());
    std::vector<int> order(keep);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return ratios[3 * (size_t)a + longest[a]] > ratios[3 * (size_t)b + longest[b]];
    });
    std::vector<char> split(T, 0);
    for (size_t k = 0; k < n_split; ++k) split[order[k]] = 1;
    int k = 0;
    for (int t : keep) {
        if (split[t]) {
            plan[k++] = (t << 3) | (1 + 2 * longest[t]);
            plan[k++] = (t << 3) | (2 + 2 * longest[t]);
        } else {
            plan[k++] = t << 3;
        }
    }
    return k;
}

}  // namespace ds
