// ds_backward.cu -- gradients of the stochastic rasteriser.
//
//  k_geom: per (view, triangle) double-float geometry for the vertex gradients.
//  k_raster_bwd: Algorithm A1 step 2 by G-buffer recomputation.  Every tile
//    list is walked again (front to back, stopping early) to find the covered
//    fragments in front of each stored winner: they get -w/(1-alpha) (Eq. 9);
//    the winner gets +w/alpha and the colour gradient (2(a)); the interior
//    vertex term (first term of Eq. 8) moves the winner's barycentrics.
//  k_edge_bwd: edge gradients on every horizontal and vertical pixel pair of
//    the sampled image (Sec. 3.2): silhouettes of the winning triangle and
//    mask-induced boundaries inside it.
//  k_grad_finish: adds the FP64 accumulators to the caller's FP32 gradients.
//
// Lane use: the walks are warp-synchronous (a warp steps through the tile's
// staged triangles, or through the samples of its pixels), and a small
// triangle covers few of a warp's 32 pixels.  The expensive work found on
// the way -- the opacity lookup and scatter of a fragment in front of a
// winner, the texture and interior terms of a pixel's distinct winners, an
// edge side -- is therefore queued per warp in shared memory and evaluated
// 32 jobs at a time, every lane busy.
//
// Scatter: lanes holding the same target (texel cell or triangle) in
// consecutive lanes are summed in registers first (warp_run_sum); only the
// first lane of each run issues the atomics, which accumulate in FP64 so that
// the summation order of the many opposite-signed score terms does not limit
// the result's accuracy.
#include "ds_internal.h"
#include "ds_tile.cuh"

namespace ds {


// ------------------------------------------------------------ small vectors
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// world-space gradient R^T g
__device__ __forceinline__ f3 to_world(const DevCam& c, f3 g) {
    return mk3(c.R[0] * g.x + c.R[3] * g.y + c.R[6] * g.z, c.R[1] * g.x + c.R[4] * g.y + c.R[7] * g.z,
               c.R[2] * g.x + c.R[5] * g.y + c.R[8] * g.z);
}

__device__ __forceinline__ float2 ld2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ f3 ld3(const float* p) { return mk3(__ldg(p), __ldg(p + 1), __ldg(p + 2)); }

// ------------------------------------------------------------ geometry record
// Double-float arithmetic (an unevaluated sum hi + lo of two floats, about
// 2^-46 relative): exact products of floats by FMA (Dekker/Kahan TwoProduct),
// exact sums by TwoSum (Knuth), renormalised after each operation.  This
// GPU's FP64 rate is a small fraction of its FP32 rate, and the record keeps
// (hi, lo) float pairs in any case.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df df_norm(float s, float e) {
    float e2;
    const float h = two_sum(s, e, e2);
    return df{h, e2};
}
__device__ __forceinline__ df df_prod(float a, float b) {   // exact a * b
    const float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    const df p = df_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return df_norm(p.hi, __fadd_rn(p.lo, t));
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const df p = df_prod(a.hi, b);
    return df_norm(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// 1 / a: float reciprocal refined by one Newton step in double-float
// (r + r (1 - a r)), which doubles the number of correct bits.
__device__ __forceinline__ df df_recip(df a) {
    const float r = __frcp_rn(a.hi);
    const df e = df_sub(df{1.0f, 0.0f}, df_mulf(a, r));
    return df_add(df{r, 0.0f}, df_mulf(e, r));
}
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ float2 df_split(df a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ df df_cross(df a1, df a2, df b1, df b2) { return df_sub(df_mul(a1, b2), df_mul(a2, b1)); }

// Camera-space positions and screen projection of every (view, triangle)
// (the oracle computes them in FP64 from the FP32 inputs), stored for
// compensated FP32 use (see GeomRec).
__global__ void k_geom(const __grid_constant__ ViewTable vt, const SoupDev s, GeomRec* __restrict__ out) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)vt.n * s.T) return;
    const int v = (int)(gid / s.T), t = (int)(gid - (long long)v * s.T);
    const DevCam& c = view_cam(vt, v);
    df V[3][3];
    const float* p = s.verts + 9LL * t;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float x = __ldg(p + 3 * m), y = __ldg(p + 3 * m + 1), z = __ldg(p + 3 * m + 2);
#pragma unroll
        for (int r = 0; r < 3; ++r)
            V[m][r] = df_add(df_add(df_prod(c.R[3 * r], x), df_prod(c.R[3 * r + 1], y)),
                             df_add(df_prod(c.R[3 * r + 2], z), df{c.t[r], 0.0f}));
    }
    GeomRec g;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const df iz = df_recip(V[m][2]);
        const df xz = df_mul(V[m][0], iz), yz = df_mul(V[m][1], iz);
        g.sx[m] = df_split(df_add(df_mulf(xz, c.fx), df{c.cx, 0.0f}));
        g.sy[m] = df_split(df_add(df_mulf(yz, c.fy), df{c.cy, 0.0f}));
        const float izf = df_f(iz);
        g.jx[m][0] = c.fx * izf;
        g.jx[m][1] = -c.fx * df_f(xz) * izf;
        g.jy[m][0] = c.fy * izf;
        g.jy[m][1] = -c.fy * df_f(yz) * izf;
    }
    df e1[3], e2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        e1[r] = df_sub(V[1][r], V[0][r]);
        e2[r] = df_sub(V[2][r], V[0][r]);
        g.e1[r] = df_f(e1[r]);
        g.e2[r] = df_f(e2[r]);
        g.v0[r] = df_f(V[0][r]);
    }
    const df* v0 = V[0];
    g.n[0] = df_split(df_cross(e1[1], e1[2], e2[1], e2[2]));
    g.n[1] = df_split(df_cross(e1[2], e1[0], e2[2], e2[0]));
    g.n[2] = df_split(df_cross(e1[0], e1[1], e2[0], e2[1]));
    g.m1[0] = df_split(df_cross(e2[1], e2[2], v0[1], v0[2]));
    g.m1[1] = df_split(df_cross(e2[2], e2[0], v0[2], v0[0]));
    g.m1[2] = df_split(df_cross(e2[0], e2[1], v0[0], v0[1]));
    g.m2[0] = df_split(df_cross(v0[1], v0[2], e1[1], e1[2]));
    g.m2[1] = df_split(df_cross(v0[2], v0[0], e1[2], e1[0]));
    g.m2[2] = df_split(df_cross(v0[0], v0[1], e1[0], e1[1]));
    g.pad = 0.f;
    const int4* src = reinterpret_cast<const int4*>(&g);
    int4* dst = reinterpret_cast<int4*>(out + gid);
#pragma unroll
    for (int k = 0; k < 13; ++k) dst[k] = src[k];
}

// Barycentrics (beta0, beta1, beta2) and 1/S of the hit of the pinned ray
// through screen point (x, y) with the plane of the triangle (Dot2 on the
// vectors of the geometry record: grazing triangles make S and the
// numerators small differences of O(1) terms).
__device__ __forceinline__ void ray_bary(const GeomRec* g, const DevCam& cam, float x, float y, float& dx, float& dy,
                                         float b[3], float& inv) {
    pinned_ray(cam, x, y, dx, dy);
    const float2 n[3] = {ld2(&g->n[0]), ld2(&g->n[1]), ld2(&g->n[2])};
    const float2 m1[3] = {ld2(&g->m1[0]), ld2(&g->m1[1]), ld2(&g->m1[2])};
    const float2 m2[3] = {ld2(&g->m2[0]), ld2(&g->m2[1]), ld2(&g->m2[2])};
    const float S = dot2(dx, dy, 1.0f, n);
    const float n1 = dot2(dx, dy, 1.0f, m1), n2 = dot2(dx, dy, 1.0f, m2);
    inv = 1.0f / S;
    b[0] = (S - n1 - n2) * inv;
    b[1] = n1 * inv;
    b[2] = n2 * inv;
}

// ------------------------------------------------------------ texture scatter
// Winner terms of one sample: colour gradient (C-1 channels) and the +w/alpha
// opacity score, merged into one pass over the corner texels, four channels
// at a time.  G receives dL/d(b1, b2) of the colour (for the interior term).
// The samples of one pixel whose winner is the same triangle have the same
// barycentrics, cell and weights, and every term is linear in the upstream
// gradient: the samples in `msk` (bit k: sample s0 + k, colour gradients at
// gcol0 + k * sstride) are handled in one pass with their upstream colour
// gradients summed; wscore is the sum of their score weights.
template <bool kInterior, int SG>
__device__ __forceinline__ void winner_texture(const SoupDev& s, double* acc_tex, bool act, int t, float b1, float b2,
                                               const float* gcol0, size_t sstride, int msk, size_t HW, float wscore,
                                               bool do_tex, bool do_score, float G[2]) {
    Cell cl;
    cl.k0 = cl.k1 = cl.k2 = 0;
    cl.wa = cl.wb = 0.f;
    cl.lower = true;
    if (act) cl = find_cell(s.N, b1, b2);
    const float w0 = 1.0f - cl.wa - cl.wb;
    const float sgnN = cl.lower ? (float)s.N : -(float)s.N;
    const int C = s.C;
    const float* base = s.act + (size_t)(act ? t : 0) * s.V * C;
    float alpha_g = 0.f;
    if (act && do_score && wscore != 0.0f) {
        const float* aa = s.act_a + (size_t)t * s.V;
        const float alpha = interp(__ldg(aa + cl.k0), __ldg(aa + cl.k1), __ldg(aa + cl.k2), cl.wa, cl.wb);
        alpha_g = wscore / alpha;
    }
    G[0] = G[1] = 0.f;
    const unsigned long long key =
        act ? (((unsigned long long)(unsigned)t << 20) | ((unsigned)cl.k0 << 1) | (cl.lower ? 1u : 0u)) : lane_sentinel();
    for (int c4 = 0; c4 < C; c4 += 4) {
        float v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = 0.f;
        if (act) {
            float A0[4], A1[4], A2[4];
            if ((C & 3) == 0) {   // 16-byte aligned texel rows: one vector load per corner
                const float4 x0 = __ldg(reinterpret_cast<const float4*>(base + (size_t)cl.k0 * C + c4));
                const float4 x1 = __ldg(reinterpret_cast<const float4*>(base + (size_t)cl.k1 * C + c4));
                const float4 x2 = __ldg(reinterpret_cast<const float4*>(base + (size_t)cl.k2 * C + c4));
                A0[0] = x0.x, A0[1] = x0.y, A0[2] = x0.z, A0[3] = x0.w;
                A1[0] = x1.x, A1[1] = x1.y, A1[2] = x1.z, A1[3] = x1.w;
                A2[0] = x2.x, A2[1] = x2.y, A2[2] = x2.z, A2[3] = x2.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = c4 + k < C ? c4 + k : C - 1;
                    A0[k] = __ldg(base + (size_t)cl.k0 * C + c);
                    A1[k] = __ldg(base + (size_t)cl.k1 * C + c);
                    A2[k] = __ldg(base + (size_t)cl.k2 * C + c);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c4 + k;
                if (c >= C) break;
                const float a0 = A0[k], a1 = A1[k], a2 = A2[k];
                float g = 0.f;
                if (c < C - 1) {
                    if (do_tex || kInterior) {
#pragma unroll
                        for (int q = 0; q < SG; ++q)
                            if (msk & (1 << q)) g += gcol0[q * sstride + c * HW];   // plain load: may be this kernel's own write
                    }
                    if (kInterior) {
                        G[0] += g * sgnN * (a1 - a0);
                        G[1] += g * sgnN * (a2 - a0);
                    }
                    if (!do_tex) g = 0.f;
                } else {
                    g = alpha_g;
                }
                v[k] = g * w0 * a0 * (1.0f - a0);
                v[4 + k] = g * cl.wa * a1 * (1.0f - a1);
                v[8 + k] = g * cl.wb * a2 * (1.0f - a2);
            }
        }
        bool any = false;
#pragma unroll
        for (int k = 0; k < 12; ++k) any = any || v[k] != 0.f;
        if (!__any_sync(kFullMask, act && any)) continue;
        const bool head = warp_run_sum<12>(key, v);
        if (act && head) {
            const int ks[3] = {cl.k0, cl.k1, cl.k2};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                double* gp = acc_tex + ((size_t)t * s.V + ks[m]) * C + c4;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (c4 + k >= C) break;
                    if (v[4 * m + k] != 0.f) atomicAdd(gp + k, (double)v[4 * m + k]);
                }
            }
        }
    }
}

// Nine-float vertex gradient of triangle t summed over runs of lanes.
__device__ __forceinline__ void scatter_verts_run(double* acc_verts, bool act, int t, float (&g)[9]) {
    if (!__any_sync(kFullMask, act)) return;
    const unsigned long long key = act ? (unsigned long long)(unsigned)t : lane_sentinel();
    const bool head = warp_run_sum<9>(key, g);
    if (act && head) {
        double* p = acc_verts + 9 * (size_t)t;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (g[k] != 0.f) atomicAdd(p + k, (double)g[k]);
    }
}

// Interior term at pixel (px, py).  With X = sum_i b_i V_i on the fixed ray
// d, moving vertex m gives e1 db1 + e2 db2 = dlambda d - b_m dV_m; crossing
// with d: db1/dV_m = -b_m (e2 x d) / S, db2/dV_m = -b_m (d x e1) / S with
// S = d.(e1 x e2).  So dL/dV_m = -(b_m / S) [G1 (e2 x d) + G2 (d x e1)].
__device__ __forceinline__ void interior_grad(const GeomRec* g, const DevCam& cam, int px, int py, const float G[2],
                                              float (&out)[9]) {
    float dx, dy, b[3], inv;
    ray_bary(g, cam, (float)px + 0.5f, (float)py + 0.5f, dx, dy, b, inv);
    const f3 d = mk3(dx, dy, 1.0f);
    const f3 c1 = cross3(ld3(g->e2), d), c2 = cross3(d, ld3(g->e1));
    const f3 u = mk3(G[0] * c1.x + G[1] * c2.x, G[0] * c1.y + G[1] * c2.y, G[0] * c1.z + G[1] * c2.z);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float k = -b[m] * inv;
        const f3 gw = to_world(cam, mk3(k * u.x, k * u.y, k * u.z));
        out[3 * m] = gw.x;
        out[3 * m + 1] = gw.y;
        out[3 * m + 2] = gw.z;
    }
}

// Winner terms of every sample: colour (Algorithm A1 2(a)), +w/alpha
// (2(b)) and the interior vertex term (first term of Eq. 8), once per
// distinct winner of a pixel's samples.  The warp's (pixel, distinct winner)
// jobs are compacted into a list in shared memory, sample by sample (the
// jobs of one sample index keep the pixels' lane order, so that runs of
// neighbouring pixels on the same triangle stay adjacent), and evaluated 32
// at a time: every lane of a round works on a job, instead of the warp
// stepping through every sample index with only the lanes whose sample
// holds a new winner active.
struct WinnerJob {
    int code;     // source lane | sample index << 5 | sample mask << 8
    int t;        // winner triangle
    float wsum;   // sum of the score weights of the samples in the mask
};
constexpr int kWinnerJobsPerWarp = kSampleGroup * 32;

// Per-warp scratch of the backward tile kernels: the score ring during the
// walk, then the winner jobs (the same warp uses them one after the other).
union WarpJobs {
    ScoreJob ring[kScoreRing];
    WinnerJob winners[kWinnerJobsPerWarp];
};

template <int SG, int TW>
__device__ __forceinline__ void winner_terms(const SoupDev& s, double* __restrict__ acc_tex,
                                             double* __restrict__ acc_verts, const GeomRec* __restrict__ vgeom,
                                             const DevCam& cam, const ViewDesc& V, const WorkItem& wi, int s0, int ns,
                                             size_t HW, bool valid, bool do_tex, bool do_score, bool do_int,
                                             const int (&wt)[SG], const float (&wsc)[SG], WinnerJob* jobs) {
    constexpr int TH = kTilePix / TW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int q = 0; q < SG; ++q) {
        bool first = valid && q < ns && wt[q] >= 0;
        int msk = 0;
        float wsum = 0.f;
#pragma unroll
        for (int r = 0; r < SG; ++r) {
            if (r < q && r < ns && wt[r] == wt[q]) first = false;   // handled with sample r
            if (r >= q && r < ns && wt[r] == wt[q]) {
                msk |= 1 << r;
                wsum += wsc[r];
            }
        }
        const unsigned bal = __ballot_sync(kFullMask, first);
        if (first) jobs[base + __popc(bal & lt)] = WinnerJob{lane | (q << 5) | (msk << 8), wt[q], wsum};
        base += __popc(bal);
    }
    __syncwarp();
    const size_t sstride = (size_t)(s.C - 1) * HW;
    for (int r0 = 0; r0 < base; r0 += 32) {
        const bool act = r0 + lane < base;
        // the round in triangle order (one run of interior atomics per triangle)
        unsigned skey = act ? (unsigned)jobs[r0 + lane].t : 0xffffffffu;
        int pos = lane;
        warp_sort32(skey, pos);
        WinnerJob jb{0, 0, 0.f};
        if (act) jb = jobs[r0 + pos];
        const int src = warp * 32 + (jb.code & 31), q = (jb.code >> 5) & 7, msk = jb.code >> 8;
        const int px = wi.tx * TW + (src & (TW - 1)), py = wi.ty * TH + src / TW;
        const size_t pix = (size_t)py * V.W + px;
        float b1 = 0.f, b2 = 0.f;
        if (act) {
            const int4 gb = reinterpret_cast<const int4*>(V.gbuf)[(s0 + q) * HW + pix];
            b1 = __int_as_float(gb.y);
            b2 = __int_as_float(gb.z);
        }
        const float* gcol0 = V.grad_color + (size_t)s0 * sstride + pix;
        float G[2];
        if (do_int)
            winner_texture<true, SG>(s, acc_tex, act, jb.t, b1, b2, gcol0, sstride, msk, HW, jb.wsum, do_tex,
                                     do_score, G);
        else if (do_tex || do_score)
            winner_texture<false, SG>(s, acc_tex, act, jb.t, b1, b2, gcol0, sstride, msk, HW, jb.wsum, do_tex,
                                      do_score, G);
        if (do_int) {
            float gv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) gv[k] = 0.f;
            if (act) interior_grad(vgeom + jb.t, cam, px, py, G, gv);
            scatter_verts_run(acc_verts, act, jb.t, gv);
        }
    }
    __syncwarp();   // the list is rewritten by the next work item
}

template <int SG, int TW>
__global__ void __launch_bounds__(kTilePix, DS_MINB_BWD)
    k_raster_bwd(const __grid_constant__ ViewTable vt, const SoupDev s, const SetupRec* __restrict__ recs,
                 const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                 const uint2* __restrict__ ranges, int DB, uint32_t flags, const GeomRec* __restrict__ geom,
                 double* __restrict__ acc_tex, double* __restrict__ acc_verts, int* __restrict__ counter) {
    __shared__ TileStage sm;
    __shared__ WarpJobs s_jobs[kTilePix / 32];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    constexpr int TH = kTilePix / TW;
    const int lx = tid & (TW - 1), ly = tid / TW, warp = tid >> 5;
    const bool do_tex = (flags & DS_G_TEX) && acc_tex;
    const bool do_score = (flags & DS_G_SCORE) && acc_tex;
    const bool do_int = (flags & DS_G_INTERIOR) && acc_verts;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= vt.n_items) break;
        const WorkItem wi = decode_item(vt, item);
        const ViewDesc& V = vt.v[wi.v];
        const int px = wi.tx * TW + lx, py = wi.ty * TH + ly;
        const bool valid = px < V.W && py < V.H;
        const int s0 = wi.g * kSampleGroup;
        const int ns = min(SG, vt.S - s0);
        const size_t HW = (size_t)V.H * V.W, pix = (size_t)py * V.W + px;
        const SetupRec* vrec = recs + (size_t)wi.v * s.T;

        int wt[SG];
        float wrho[SG], wsc[SG];
        bool any_score = false;
#pragma unroll
        for (int q = 0; q < SG; ++q) {
            wt[q] = -1;
            wrho[q] = wsc[q] = 0.f;
            if (valid && q < ns) {
                const int4 gb = reinterpret_cast<const int4*>(V.gbuf)[(s0 + q) * HW + pix];
                wt[q] = (gb.x >= 0 && gb.x < s.T) ? gb.x : -1;   // ids outside the soup read as background
                if (do_score && V.score_w) wsc[q] = V.score_w[(s0 + q) * HW + pix];
                if (wt[q] >= 0) {   // computed once per distinct winner of the pixel
                    bool seen = false;
                    float rr = 0.f;
#pragma unroll
                    for (int r = 0; r < SG; ++r)
                        if (r < q && !seen && wt[r] == wt[q]) {
                            seen = true;
                            rr = wrho[r];
                        }
                    wrho[q] = seen ? rr : winner_rho(vrec + wt[q], px, py);
                }
                any_score = any_score || wsc[q] != 0.f;
            }
        }

        const uint2 rg = ranges[V.tile_base + wi.ty * V.tiles_x + wi.tx];
        score_walk<SG, TW>(sm, recs, keys, vals, rg, DB, vt.chunk, (size_t)wi.v * s.T, wi, s, acc_tex, tid, lx, ly,
                           warp, false, any_score, wt, wrho, wsc, s_jobs[warp].ring);
        winner_terms<SG, TW>(s, acc_tex, acc_verts, geom + (size_t)wi.v * s.T, view_cam(vt, wi.v), V, wi, s0, ns, HW,
                             valid, do_tex, do_score, do_int, wt, wsc, s_jobs[warp].winners);
        __syncthreads();
    }
}

// ------------------------------------------------------------ fused training pass
// Forward (Eq. 5), per-pixel L2 loss, and the texture, score and interior
// gradients (Algorithm A1 step 2 without the edge terms) of one work item in
// one CTA: the masked z-test walk, then the G-buffer, colours, upstream
// gradients and score weights, then the score walk over the same staged list
// (still in shared memory when it fits one chunk) and the winner terms.  The
// winners' depths come from the forward walk instead of being recomputed.
template <int SG, int TW>
__global__ void __launch_bounds__(kTilePix, DS_MINB_TRAIN)
    k_raster_train(const __grid_constant__ ViewTable vt, const SoupDev s, const SetupRec* __restrict__ recs,
                   const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                   const uint2* __restrict__ ranges, int DB, uint32_t mode, const Bg bg, float scale,
                   float* __restrict__ loss, uint32_t flags, const GeomRec* __restrict__ geom,
                   double* __restrict__ acc_tex, double* __restrict__ acc_verts, int* __restrict__ counter) {
    __shared__ TileStage sm;
    __shared__ WarpJobs s_jobs[kTilePix / 32];
    __shared__ int s_item;
    __shared__ float s_loss[kTilePix / 32];
    const int tid = threadIdx.x;
    constexpr int TH = kTilePix / TW;
    const int lx = tid & (TW - 1), ly = tid / TW, warp = tid >> 5;
    const bool stochastic = mode == DS_MODE_STOCHASTIC;
    const bool do_tex = (flags & DS_G_TEX) && acc_tex;
    const bool do_score = (flags & DS_G_SCORE) && acc_tex;
    const bool do_int = (flags & DS_G_INTERIOR) && acc_verts;
    const float two_scale = 2.0f * scale;
    float lsum = 0.f;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= vt.n_items) break;
        const WorkItem wi = decode_item(vt, item);
        const ViewDesc& V = vt.v[wi.v];
        const int px = wi.tx * TW + lx, py = wi.ty * TH + ly;
        const bool valid = px < V.W && py < V.H;
        const int s0 = wi.g * kSampleGroup;
        const int ns = min(SG, vt.S - s0);
        const uint2 seed = view_seed(vt, wi.v);
        const size_t HW = (size_t)V.H * V.W, pix = (size_t)py * V.W + px;

        int bt[SG];
        float brho[SG], bb1[SG], bb2[SG], bD[SG];
#pragma unroll
        for (int q = 0; q < SG; ++q) {
            bt[q] = -1;
            brho[q] = 0.0f;
            bb1[q] = bb2[q] = 0.0f;
            bD[q] = __int_as_float(0x7f800000);
        }
        const uint2 rg = ranges[V.tile_base + wi.ty * V.tiles_x + wi.tx];
        const bool fits = forward_walk<SG, TW>(sm, recs, keys, vals, rg, DB, vt.chunk, (size_t)wi.v * s.T, wi, s, tid,
                                               lx, ly, warp, valid, px, py, ns, seed, stochastic, bt, brho, bb1, bb2,
                                               bD);

        // ---- G-buffer, colours, loss, upstream gradients, score weights
        float wsc[SG];
        bool any_score = false;
        const int Co = s.C - 1;
#pragma unroll
        for (int q = 0; q < SG; ++q) {
            wsc[q] = 0.f;
            if (!valid || q >= ns) continue;
            const int sg = s0 + q;
            reinterpret_cast<int4*>(V.gbuf)[sg * HW + pix] =
                make_int4(bt[q], __float_as_int(bb1[q]), __float_as_int(bb2[q]), __float_as_int(bD[q]));
            const float ell = color_loss_out(s, bt[q], bb1[q], bb2[q], bg, V.target + pix,
                                             V.color + (size_t)sg * Co * HW + pix,
                                             const_cast<float*>(V.grad_color) + (size_t)sg * Co * HW + pix, HW,
                                             two_scale);
            const float w = __fmul_rn(scale, ell);
            if (V.score_w) const_cast<float*>(V.score_w)[sg * HW + pix] = w;
            lsum += ell;
            if (do_score) wsc[q] = w;
            any_score = any_score || wsc[q] != 0.f;
        }

        // ---- Algorithm A1 step 2 (texture, score, interior)
        score_walk<SG, TW>(sm, recs, keys, vals, rg, DB, vt.chunk, (size_t)wi.v * s.T, wi, s, acc_tex, tid, lx, ly,
                           warp, fits, any_score, bt, brho, wsc, s_jobs[warp].ring);
        winner_terms<SG, TW>(s, acc_tex, acc_verts, geom + (size_t)wi.v * s.T, view_cam(vt, wi.v), V, wi, s0, ns, HW,
                             valid, do_tex, do_score, do_int, bt, wsc, s_jobs[warp].winners);
        __syncthreads();
    }
    // ---- the loss: one atomic per CTA
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) lsum += __shfl_down_sync(kFullMask, lsum, d);
    if ((tid & 31) == 0) s_loss[warp] = lsum;
    __syncthreads();
    if (tid == 0 && loss) {
        float t = 0.f;
        for (int w = 0; w < kTilePix / 32; ++w) t += s_loss[w];
        atomicAdd(loss, scale * t);
    }
}

// ------------------------------------------------------------ edge gradients
// Screen coordinate (hi + lo) relative to pixel coordinate x, compensated.
__device__ __forceinline__ float rel(float2 s, float x) {
    float e;
    const float d = two_sum(s.x, -x, e);
    return __fadd_rn(d, __fadd_rn(e, s.y));
}

__device__ __forceinline__ void add_world(const DevCam& cam, f3 gc, float* out) {
    const f3 gw = to_world(cam, gc);
    out[0] += gw.x;
    out[1] += gw.y;
    out[2] += gw.z;
}

// Contribution of side X of a pixel pair (X -> Y along unit axis e = (ex, ey))
// whose winner triangle is t: silhouette or mask-induced (implicit) boundary.
// phi = 1/2 sum_c (g_X + g_Y)(C_X - C_Y).  Returns false if X is not in front.
// Every array index is a compile-time constant (no local memory).
__device__ __forceinline__ bool edge_side(const DevCam& cam, const SetupRec* vrec, const GeomRec* g, int t, int xX,
                                          int yX, int xY, int yY, int tY, float phi, float (&out)[9]) {
    const SetupRec r = load_rec(vrec + t);
    long long E[3];
    const float ex = (float)(xY - xX), ey = (float)(yY - yX);
    if (cover_exact(r, xY, yY, E)) {
        const float rho = make_frag(E[0], E[1], E[2], r.k[0], r.k[1], r.k[2]).rho;
        if (tY >= 0 && !in_front(rho, t, winner_rho(vrec + tY, xY, yY), tY)) return false;   // occluded at Y
        // implicit boundary: the material point under the pair's midpoint
        // moves with the surface; weight 1 per pair axis
        float dx, dy, beta[3], inv;
        ray_bary(g, cam, 0.5f * (float)(xX + xY + 1), 0.5f * (float)(yX + yY + 1), dx, dy, beta, inv);
        const f3 e1 = ld3(g->e1), e2 = ld3(g->e2), v0 = ld3(g->v0);
        const f3 P = mk3(v0.x + beta[1] * e1.x + beta[2] * e2.x, v0.y + beta[1] * e1.y + beta[2] * e2.y,
                         v0.z + beta[1] * e1.z + beta[2] * e2.z);
        const float iz = 1.0f / P.z;
        // J^T e with J rows (fx/z, 0, -fx x/z^2), (0, fy/z, -fy y/z^2)
        const f3 je = mk3(ex * cam.fx * iz, ey * cam.fy * iz, -(ex * cam.fx * P.x + ey * cam.fy * P.y) * iz * iz);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float f = phi * beta[m];
            add_world(cam, mk3(f * je.x, f * je.y, f * je.z), out + 3 * m);
        }
        return true;
    }
    // silhouette: the first edge the segment X -> Y crosses; coordinates
    // relative to X's pixel centre
    const float cxX = (float)xX + 0.5f, cyX = (float)yX + 0.5f;
    float sx[3], sy[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        sx[m] = rel(ld2(&g->sx[m]), cxX);
        sy[m] = rel(ld2(&g->sy[m]), cyX);
    }
    const float area = diff_prod(sx[1] - sx[0], sy[2] - sy[0], sx[2] - sx[0], sy[1] - sy[0]);
    const float sg = area > 0.f ? 1.f : -1.f;
    int best = -1;
    float bs = 0.f, bfX = 0.f, bfY = 0.f, ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int a = (i + 1) % 3, b = (i + 2) % 3;
        const float fX = sg * diff_prod(sx[a], sy[b], sx[b], sy[a]);
        const float fY = sg * diff_prod(sx[a] - ex, sy[b] - ey, sx[b] - ex, sy[a] - ey);
        if (!(fY < 0.f && fX > fY)) continue;
        const float si = fX / (fX - fY);
        if (best < 0 || si < bs) {
            best = i;
            bs = si;
            bfX = fX;
            bfY = fY;
            ax = sx[a];
            ay = sy[a];
            bx = sx[b];
            by = sy[b];
        }
    }
    if (best < 0) return true;
    const float fX = bfX * sg, fY = bfY * sg;
    const float den = (fX - fY) * (fX - fY);
    const float ux = bx - ax, uy = by - ay;
    const float omega = (ex != 0.f ? uy * uy : ux * ux) / (ux * ux + uy * uy);
    const float k = omega * phi / den;
    // d f(x)/d a = (b_y - x_y, -(b_x - x_x)); d f(x)/d b = (-(a_y - x_y), a_x - x_x)
    const float gax = k * (fX * (by - ey) - fY * by), gay = k * (fX * (-(bx - ex)) - fY * (-bx));
    const float gbx = k * (fX * (-(ay - ey)) - fY * (-ay)), gby = k * (fX * (ax - ex) - fY * ax);
    const int ia = (best + 1) % 3, ib = (best + 2) % 3;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (m != ia && m != ib) continue;
        const float gx = m == ia ? gax : gbx;
        const float gy = m == ia ? gay : gby;
        const float j0 = __ldg(&g->jx[m][0]), j1 = __ldg(&g->jx[m][1]);
        const float k0 = __ldg(&g->jy[m][0]), k1 = __ldg(&g->jy[m][1]);
        add_world(cam, mk3(gx * j0, gy * k0, gx * j1 + gy * k1), out + 3 * m);
    }
    return true;
}

// One CTA per (view, tile, sample group); every pixel owns its pairs with
// the right and the lower neighbour.  A pair with different winners yields up
// to two side jobs (one per side with a triangle).  Each warp queues its jobs
// in a ring in shared memory (prefix over lanes) and evaluates them 32 at a
// time whenever 32 are waiting, across the samples of the work item, so that
// every lane works on a boundary instead of idling; only the last batch of a
// work item can be partial.  Consecutive jobs mostly share a triangle, and
// runs of equal triangles are summed before the atomics.
struct EdgeJob {
    int xy;      // X: x | (y << 16)
    int t;       // triangle of side X
    int tY;      // winner at Y (-1: background)
    float phi;   // 1/2 sum_c (g_X + g_Y)(C_X - C_Y) for side X
    int dir;     // Y = X + (1, 0) / (-1, 0) / (0, 1) / (0, -1): 0..3
};

// Ring capacity: up to 31 jobs left from earlier samples plus 4 per lane.
constexpr int kJobsPerWarp = 5 * 32;

template <int SG, int TW>
__global__ void __launch_bounds__(kTilePix, DS_MINB_EDGE)
    k_edge_bwd(const __grid_constant__ ViewTable vt, const SoupDev s, const SetupRec* __restrict__ recs,
               const GeomRec* __restrict__ geom, double* __restrict__ acc_verts, int* __restrict__ counter) {
    __shared__ int s_item;
    __shared__ EdgeJob s_jobs[kTilePix / 32][kJobsPerWarp];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int TH = kTilePix / TW;
    const int lx = tid & (TW - 1), ly = tid / TW;
    const int Co = s.C - 1;
    EdgeJob* jobs = s_jobs[warp];
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= vt.n_items) break;
        const WorkItem wi = decode_item(vt, item);
        const ViewDesc& V = vt.v[wi.v];
        const int px = wi.tx * TW + lx, py = wi.ty * TH + ly;
        const bool valid = px < V.W && py < V.H;
        const int s0 = wi.g * kSampleGroup;
        const int ns = min(SG, vt.S - s0);
        const size_t HW = (size_t)V.H * V.W, ip = (size_t)py * V.W + px;
        const SetupRec* vrec = recs + (size_t)wi.v * s.T;
        const GeomRec* vgeom = geom + (size_t)wi.v * s.T;
        const int4* gbuf = reinterpret_cast<const int4*>(V.gbuf);
        int head = 0, count = 0;   // the warp's job ring (same values in every lane)
#pragma unroll 1
        for (int q = 0; q < SG; ++q) {
            const bool qv = valid && q < ns;
            const int sq = s0 + (q < ns ? q : 0);
            int tp = qv ? gbuf[sq * HW + ip].x : -1;
            if (tp < 0 || tp >= s.T) tp = -1;
            const float* col = V.color + (size_t)sq * Co * HW;
            const float* gc = V.grad_color + (size_t)sq * Co * HW;
            // ---- this lane's jobs: slot dir for the pixel's own side, 2 + dir
            // for the neighbour's (the two own-side jobs share the pixel's
            // winner and sit next to each other: one run of atomics); fixed
            // slots keep the register arrays at constant indices
            EdgeJob sl[4];
            bool vl[4] = {false, false, false, false};
            // winners of the right and lower neighbours, and the pair terms
            // Phi of both directions in one pass over the channels (the
            // pixel's own colour and gradient are read once)
            int tqd[2] = {tp, tp};
            size_t iqd[2] = {ip, ip};
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int qx = px + (dir == 0), qy = py + (dir == 1);
                if (!qv || qx >= V.W || qy >= V.H) continue;
                iqd[dir] = (size_t)qy * V.W + qx;
                int tq = gbuf[sq * HW + iqd[dir]].x;
                tqd[dir] = (tq < 0 || tq >= s.T) ? -1 : tq;
            }
            const bool d0 = tqd[0] != tp, d1 = tqd[1] != tp;
            float phid[2] = {0.f, 0.f};
            if (d0 || d1) {
                for (int c = 0; c < Co; ++c) {
                    const float gp = __ldg(gc + c * HW + ip), cp = __ldg(col + c * HW + ip);
                    if (d0)
                        phid[0] += 0.5f * (gp + __ldg(gc + c * HW + iqd[0])) * (cp - __ldg(col + c * HW + iqd[0]));
                    if (d1)
                        phid[1] += 0.5f * (gp + __ldg(gc + c * HW + iqd[1])) * (cp - __ldg(col + c * HW + iqd[1]));
                }
            }
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int qx = px + (dir == 0), qy = py + (dir == 1);
                const int tq = tqd[dir];
                if (tq == tp) continue;
                const float phi = phid[dir];
                if (phi == 0.f) continue;
                if (tp >= 0) {
                    sl[dir] = EdgeJob{px | (py << 16), tp, tq, phi, dir == 0 ? 0 : 2};
                    vl[dir] = true;
                }
                if (tq >= 0) {
                    sl[2 + dir] = EdgeJob{qx | (qy << 16), tq, tp, -phi, dir == 0 ? 1 : 3};
                    vl[2 + dir] = true;
                }
            }
            const int nmine = (int)vl[0] + (int)vl[1] + (int)vl[2] + (int)vl[3];
            // ---- queue them (lane order, then slot order)
            int pre = nmine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(kFullMask, pre, d);
                if (lane >= d) pre += o;
            }
            const int total = __shfl_sync(kFullMask, pre, 31);
            pre -= nmine;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (vl[k]) jobs[(head + count + pre++) % kJobsPerWarp] = sl[k];
            count += total;
            __syncwarp();
            // ---- evaluate 32 at a time while a full batch waits (and the
            // remainder after the last sample)
            while (count >= 32 || (q == SG - 1 && count > 0)) {
                const int n = min(count, 32);
                float acc[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = 0.f;
                bool act = false;
                int t = -1;
                if (lane < n) {
                    const EdgeJob jb = jobs[(head + lane) % kJobsPerWarp];
                    const int xX = jb.xy & 0xffff, yX = jb.xy >> 16;
                    const int xY = xX + (jb.dir == 0) - (jb.dir == 1), yY = yX + (jb.dir == 2) - (jb.dir == 3);
                    t = jb.t;
                    act = edge_side(view_cam(vt, wi.v), vrec, vgeom + t, t, xX, yX, xY, yY, jb.tY, jb.phi, acc);
                }
                scatter_verts_run(acc_verts, act, t, acc);
                head = (head + n) % kJobsPerWarp;
                count -= n;
                __syncwarp();
            }
        }
    }
}

// Add (or write) the FP64 accumulators into the caller's FP32 gradients.
__global__ void k_grad_finish(const double* __restrict__ acc, float* __restrict__ out, long long n, int overwrite) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const double base = overwrite ? 0.0 : (double)out[i];
        out[i] = (float)(base + acc[i]);
    }
}

// The texture finish with Adam fused (Sec. 3.4): the step's gradient of value
// i, rounded to FP32 as the plain finish writes it, moves x, m, v at once.
__global__ void k_grad_finish_adam(const double* __restrict__ acc, float* __restrict__ x, float* __restrict__ m,
                                   float* __restrict__ v, long long n, AdamDev a) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float xi = x[i], mi = m[i], vi = v[i];
        adam_apply(xi, mi, vi, (float)(0.0 + __ldcs(acc + i)), a);
        x[i] = xi;
        m[i] = mi;
        v[i] = vi;
    }
}

cudaError_t launch_geom(const ViewTable& vt, const SoupDev& s, GeomRec* geom, cudaStream_t st) {
    const long long n = (long long)vt.n * s.T;
    k_geom<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(vt, s, geom);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const uint32_t* keys,
                              const uint32_t* vals, const uint2* ranges, int DB, uint32_t flags, const GeomRec* geom,
                              double* acc_tex, double* acc_verts, int* counter, int grid, cudaStream_t st) {
    dispatch_tile(vt.tile_w, vt.S == 1 ? 1 : (vt.S == 2 ? 2 : 4), [&](auto P) {
        constexpr int SG = decltype(P)::sg, TW = decltype(P)::tw;
        k_raster_bwd<SG, TW><<<resident_grid(k_raster_bwd<SG, TW>, vt.n_items, grid), kTilePix, 0, st>>>(
            vt, s, recs, keys, vals, ranges, DB, flags, geom, acc_tex, acc_verts, counter);
    });
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_raster_train(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const uint32_t* keys,
                                const uint32_t* vals, const uint2* ranges, int DB, uint32_t mode, const Bg& bg,
                                float scale, float* loss, uint32_t flags, const GeomRec* geom, double* acc_tex,
                                double* acc_verts, int* counter, int grid, cudaStream_t st) {
    dispatch_tile(vt.tile_w, vt.S == 1 ? 1 : (vt.S == 2 ? 2 : 4), [&](auto P) {
        constexpr int SG = decltype(P)::sg, TW = decltype(P)::tw;
        k_raster_train<SG, TW><<<resident_grid(k_raster_train<SG, TW>, vt.n_items, grid), kTilePix, 0, st>>>(
            vt, s, recs, keys, vals, ranges, DB, mode, bg, scale, loss, flags, geom, acc_tex, acc_verts, counter);
    });
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_edge_bwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const GeomRec* geom,
                            double* acc_verts, int* counter, int grid, cudaStream_t st) {
    dispatch_tile(vt.tile_w, vt.S == 1 ? 1 : (vt.S == 2 ? 2 : 4), [&](auto P) {
        constexpr int SG = decltype(P)::sg, TW = decltype(P)::tw;
        k_edge_bwd<SG, TW><<<resident_grid(k_edge_bwd<SG, TW>, vt.n_items, grid), kTilePix, 0, st>>>(
            vt, s, recs, geom, acc_verts, counter);
    });
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_grad_finish(const double* acc, float* out, long long n, bool overwrite, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    k_grad_finish<<<(unsigned)g, 256, 0, st>>>(acc, out, n, overwrite ? 1 : 0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_grad_finish_adam(const double* acc, const AdamTex& adam, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    k_grad_finish_adam<<<(unsigned)g, 256, 0, st>>>(acc, adam.x, adam.m, adam.v, n, adam.a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ds
