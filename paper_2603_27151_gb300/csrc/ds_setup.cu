// ds_setup.cu -- texture activation, per-(view, triangle) set-up and the
// emission of (tile, depth) keys for the radix-sorted binning.
#include "ds_internal.h"

namespace ds {

// ---------------------------------------------------------------- activation
// a = sigmoid(theta) on every feature-vertex channel (Sec. 3.3, applied to the
// finest grid before rasterisation); the opacity channel is also written to a
// planar [T][V] copy so that the per-fragment opacity lookups of the masked
// depth test touch 4 bytes per corner.
__global__ void k_activate(const float* __restrict__ tex, float* __restrict__ act,
                           float* __restrict__ act_a, long long n, int C) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float a = pinned_sigmoid(__ldg(tex + i));
        act[i] = a;
        const long long q = i / C;
        if (i - q * C == C - 1) act_a[q] = a;
    }
}

// Same with 16-byte vectors when C % 4 == 0 (the opacity channel is the last
// lane of every C/4-th vector).
__global__ void k_activate4(const float4* __restrict__ tex, float4* __restrict__ act,
                            float* __restrict__ act_a, long long n4, int C4) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 x = __ldg(tex + i);
        float4 a;
        a.x = pinned_sigmoid(x.x);
        a.y = pinned_sigmoid(x.y);
        a.z = pinned_sigmoid(x.z);
        a.w = pinned_sigmoid(x.w);
        act[i] = a;
        const long long q = i / C4;
        if (i - q * C4 == C4 - 1) act_a[q] = a.w;
    }
}

cudaError_t launch_activate(const SoupDev& s, cudaStream_t st) {
    const long long n = (long long)s.T * s.V * s.C;
    const bool vec = (s.C % 4 == 0) && ((uintptr_t)s.tex % 16 == 0) && ((uintptr_t)s.act % 16 == 0);
    const long long work = vec ? n / 4 : n;
    int grid = (int)((work + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    if (vec)
        k_activate4<<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(s.tex),
                                          reinterpret_cast<float4*>(s.act), s.act_a, n / 4, s.C / 4);
    else
        k_activate<<<grid, 256, 0, st>>>(s.tex, s.act, s.act_a, n, s.C);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- set-up
__device__ __forceinline__ int floordiv256(int x) { return x >> 8; }   // arithmetic shift = floor

// Upper bound of the biased edge value over the tw x th pixel centres of a
// tile: a linear function peaks at a corner of the centre grid.
__device__ __forceinline__ bool tile_may_cover(const SetupRec& r, int tx, int ty, int tw, int th) {
    const long long X0 = 256LL * (tw * tx) + 128, Y0 = 256LL * (th * ty) + 128;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long e0 = (long long)r.A[i] * X0 + (long long)r.B[i] * Y0 + r.C[i];
        const long long up = 256LL * ((long long)(tw - 1) * (r.A[i] > 0 ? r.A[i] : 0) +
                                      (long long)(th - 1) * (r.B[i] > 0 ? r.B[i] : 0));
        if (e0 + up < 0) return false;
    }
    return true;
}

constexpr int kExactTileLimit = 64;   // bbox tile counts above this skip the per-tile test

// One thread per (view, triangle): project, snap to 1/256 pixel, cull, build
// the oriented edge functions with the top-left fill rule (Eq. 1 fragments),
// the perspective factors k_i, the tile rectangle and the number of tiles
// whose pixel centres the triangle may cover.
// The view of set-up record `gid` (records of view v start at rec_base).
__device__ __forceinline__ int view_of_record(const ViewTable& vt, long long gid) {
    int v = 0;
    for (int i = 1; i < vt.n; ++i)
        if (vt.v[i].rec_base <= gid) v = i;
    return v;
}

__global__ void k_setup(const __grid_constant__ ViewTable vt, long long n_records,
                        SetupRec* __restrict__ recs, uint32_t* __restrict__ counts,
                        int4* __restrict__ tbox, uint32_t* __restrict__ zkeys) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= n_records) return;
    const int v = view_of_record(vt, gid), t = (int)(gid - vt.v[v].rec_base);
    const DevCam& cam = view_cam(vt, v);
    const int W = vt.v[v].W, H = vt.v[v].H;
    const float* p = vt.v[v].s_verts + 9LL * t;

    int X[3], Y[3];
    float w[3];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float px = __ldg(p + 3 * i), py = __ldg(p + 3 * i + 1), pz = __ldg(p + 3 * i + 2);
        const float xc = __fmaf_rn(cam.R[0], px, __fmaf_rn(cam.R[1], py, __fmaf_rn(cam.R[2], pz, cam.t[0])));
        const float yc = __fmaf_rn(cam.R[3], px, __fmaf_rn(cam.R[4], py, __fmaf_rn(cam.R[5], pz, cam.t[1])));
        const float zc = __fmaf_rn(cam.R[6], px, __fmaf_rn(cam.R[7], py, __fmaf_rn(cam.R[8], pz, cam.t[2])));
        ok = ok && (zc > cam.near_z);
        const float sx = __fmaf_rn(cam.fx, __fdiv_rn(xc, zc), cam.cx);
        const float sy = __fmaf_rn(cam.fy, __fdiv_rn(yc, zc), cam.cy);
        ok = ok && (fabsf(sx) <= kGuard) && (fabsf(sy) <= kGuard);
        X[i] = ok ? __float2int_rn(__fmul_rn(sx, 256.0f)) : 0;
        Y[i] = ok ? __float2int_rn(__fmul_rn(sy, 256.0f)) : 0;
        w[i] = zc;
    }
    const long long area = (long long)(X[1] - X[0]) * (Y[2] - Y[0]) - (long long)(X[2] - X[0]) * (Y[1] - Y[0]);
    ok = ok && (area != 0);

    SetupRec r;
    uint32_t cnt = 0;
    int4 box = make_int4(0, 0, -1, -1);
    uint32_t zk = 0;
    if (ok) {
        const int sg = area > 0 ? 1 : -1;
        r.bias = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            const int A = sg * (Y[j] - Y[k]);
            const int B = sg * (X[k] - X[j]);
            long long Cc = (long long)sg * ((long long)X[j] * Y[k] - (long long)X[k] * Y[j]);
            const bool owns = A > 0 || (A == 0 && B > 0);
            if (!owns) {
                Cc -= 1;
                r.bias |= 1u << i;
            }
            r.A[i] = A;
            r.B[i] = B;
            r.C[i] = Cc;
        }
        const float fa = __ll2float_rn(area > 0 ? area : -area);
#pragma unroll
        for (int i = 0; i < 3; ++i) r.k[i] = __fdiv_rn(__fdiv_rn(1.0f, w[i]), fa);

        // pixel centres 256 px + 128 inside [min, max] of the snapped vertices
        const int xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
        const int ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
        int px0 = floordiv256(xmin - 128 + 255), px1 = floordiv256(xmax - 128);
        int py0 = floordiv256(ymin - 128 + 255), py1 = floordiv256(ymax - 128);
        px0 = max(px0, 0);
        py0 = max(py0, 0);
        px1 = min(px1, W - 1);
        py1 = min(py1, H - 1);
        if (px0 <= px1 && py0 <= py1) {
            box = make_int4(px0 / vt.tile_w, py0 / vt.tile_h, px1 / vt.tile_w, py1 / vt.tile_h);
            const int nb = (box.z - box.x + 1) * (box.w - box.y + 1);
            if (nb > kExactTileLimit) {
                cnt = nb;
            } else {
                for (int ty = box.y; ty <= box.w; ++ty)
                    for (int tx = box.x; tx <= box.z; ++tx)
                        cnt += tile_may_cover(r, tx, ty, vt.tile_w, vt.tile_h) ? 1u : 0u;
            }
        }
        zk = __float_as_uint(fminf(w[0], fminf(w[1], w[2])));
    } else {
        r = SetupRec{};
        r.C[0] = r.C[1] = r.C[2] = -1;   // covers nothing
    }
    int4* dst = reinterpret_cast<int4*>(recs + gid);
    const int4* src = reinterpret_cast<const int4*>(&r);
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[2];
    dst[3] = src[3];
    counts[gid] = cnt;
    tbox[gid] = box;
    zkeys[gid] = zk;
}

long long view_records(const ViewTable& vt) {
    return vt.n > 0 ? vt.v[vt.n - 1].rec_base + vt.v[vt.n - 1].s_T : 0;
}

void set_view_soups(ViewTable& vt, const SoupDev* const* soups) {
    long long rb = 0;
    for (int v = 0; v < vt.n; ++v) {
        const SoupDev& s = *soups[v];
        ViewDesc& d = vt.v[v];
        d.s_verts = s.verts;
        d.s_act = s.act;
        d.s_act_a = s.act_a;
        d.s_T = s.T;
        d.rec_base = rb;
        rb += s.T;
    }
}

void set_view_soups(ViewTable& vt, const SoupDev& s) {
    const SoupDev* one[DS_MAX_VIEWS];
    for (int v = 0; v < vt.n; ++v) one[v] = &s;
    set_view_soups(vt, one);
}

cudaError_t launch_setup(const ViewTable& vt, SetupRec* recs, uint32_t* counts, int4* tbox, uint32_t* zkeys,
                         cudaStream_t st) {
    const long long n = view_records(vt);
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256);
    k_setup<<<grid, 256, 0, st>>>(vt, n, recs, counts, tbox, zkeys);
    note_launches(1);
    return cudaGetLastError();
}

__global__ void k_emit(const __grid_constant__ ViewTable vt, long long n_records, const SetupRec* __restrict__ recs,
                       const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offs,
                       const int4* __restrict__ tbox, const uint32_t* __restrict__ zkeys, int DB,
                       uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t cap,
                       int* __restrict__ status) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= n_records) return;
    const uint32_t cnt = counts[gid];
    if (cnt == 0) return;
    const int v = view_of_record(vt, gid), t = (int)(gid - vt.v[v].rec_base);
    const int4 box = tbox[gid];
    const SetupRec r = load_rec(recs + gid);
    const uint32_t dbits = DB > 0 ? ((zkeys[gid] & 0x7fffffffu) >> (31 - DB)) : 0u;
    const int nb = (box.z - box.x + 1) * (box.w - box.y + 1);
    const bool exact = nb <= kExactTileLimit;
    uint32_t o = offs[gid];
    const int tiles_x = vt.v[v].tiles_x, base = vt.v[v].tile_base;
    bool over = false;
    for (int ty = box.y; ty <= box.w; ++ty)
        for (int tx = box.x; tx <= box.z; ++tx) {
            if (exact && !tile_may_cover(r, tx, ty, vt.tile_w, vt.tile_h)) continue;
            if (o < cap) {
                keys[o] = ((uint32_t)(base + ty * tiles_x + tx) << DB) | dbits;
                vals[o] = (uint32_t)t;
            } else {
                over = true;
            }
            ++o;
        }
    if (over) atomicOr(status, 1);
}

cudaError_t launch_emit(const ViewTable& vt, const SetupRec* recs, const uint32_t* counts, const uint32_t* offs,
                        const int4* tbox, const uint32_t* zkeys, int DB, uint32_t* keys, uint32_t* vals,
                        uint32_t cap, int* status, cudaStream_t st) {
    const long long n = view_records(vt);
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256);
    k_emit<<<grid, 256, 0, st>>>(vt, n, recs, counts, offs, tbox, zkeys, DB, keys, vals, cap, status);
    note_launches(1);
    return cudaGetLastError();
}

// [begin, end) of every tile's run in the sorted keys (tiles with no pair
// keep the zero range written before the launch).
__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ count,
                              uint32_t kcap, int DB, uint2* __restrict__ ranges) {
    const uint32_t K = min(*count, kcap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t tile = keys[i] >> DB;
    if (i == 0 || (keys[i - 1] >> DB) != tile) ranges[tile].x = i;
    if (i == K - 1 || (keys[i + 1] >> DB) != tile) ranges[tile].y = i + 1;
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const uint32_t* count, uint32_t kcap, int DB,
                               uint2* ranges, cudaStream_t st) {
    if (kcap == 0) return cudaSuccess;
    const int grid = (int)((kcap + 255) / 256);
    k_tile_ranges<<<grid, 256, 0, st>>>(keys, count, kcap, DB, ranges);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ds
