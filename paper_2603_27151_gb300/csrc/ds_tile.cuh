// ds_tile.cuh -- device helpers shared by the tile kernels (forward, counts,
// backward): work-item decoding, per-tile staging of triangle set-up in
// shared memory, the tile-relative coverage test and the colour decode.
#pragma once

#include "ds_common.cuh"

namespace ds {

constexpr unsigned kFullMask = 0xffffffffu;

// Resident CTAs per SM requested from the compiler for the tile kernels
// (register budget 65536 / (256 x blocks)); set per kernel at build time.
// The backward and the fused training pass run at five (48 registers):
// their waits on gathers hide better with 40 warps than the spills cost;
// the edge kernel and the forward of 4-sample groups are faster at four,
// the forward of smaller groups (fewer registers per pixel) at five.
#ifndef DS_MINB_FWD
#define DS_MINB_FWD 4
#endif
#ifndef DS_MINB_FWD_SMALL
#define DS_MINB_FWD_SMALL 5
#endif
#ifndef DS_MINB_BWD
#define DS_MINB_BWD 5
#endif
#ifndef DS_MINB_EDGE
#define DS_MINB_EDGE 4
#endif
#ifndef DS_MINB_TRAIN
#define DS_MINB_TRAIN 5
#endif

// Per-tile staged set-up.  h0..h2 hold what the per-pixel coverage test reads
// for every triangle; eo/kk are read only for covered fragments.
struct TileStage {
    int4 h0[kChunk];         // A0, B0, thr0, A1
    int4 h1[kChunk];         // B1, thr1, A2, B2
    int4 h2[kChunk];         // thr2, triangle, rho bound (float bits), warp mask
    long long eo[kChunk][3]; // oriented (unbiased) edge values at the tile's first pixel centre
    float kk[kChunk][3];     // perspective factors k_i
};

struct WorkItem {
    int v, g, tx, ty;
};

// Work items are numbered view by view, then sample group, then tile.
__device__ __forceinline__ WorkItem decode_item(const ViewTable& vt, int item) {
    WorkItem w;
    w.v = 0;
    for (int i = 1; i < vt.n; ++i)
        if (vt.v[i].item_base <= item) w.v = i;
    const ViewDesc& V = vt.v[w.v];
    const int tiles = V.tiles_x * V.tiles_y;
    const int local = item - V.item_base;
    w.g = local / tiles;
    const int tile = local - w.g * tiles;
    w.ty = tile / V.tiles_x;
    w.tx = tile - w.ty * V.tiles_x;
    return w;
}

// Upper bound on the inverse depth of every triangle whose sort key is at
// least `key`: the key's depth bits are the top DB bits of the nearest
// vertex depth, so the float they encode is <= that depth.  The bound is
// widened by 2^-10 to cover the rounding of rho (a few ulps).
__device__ __forceinline__ float rho_bound(uint32_t key, int DB) {
    if (DB <= 0) return __int_as_float(0x7f800000);
    const uint32_t q = key & ((1u << DB) - 1u);
    const float zq = __uint_as_float(q << (31 - DB));
    if (!(zq > 0.0f)) return __int_as_float(0x7f800000);
    return __fmul_rn(__frcp_rn(zq), 1.0f + 0x1p-10f);
}

// Stage triangle t (set-up record in view base vbase) for the tile whose
// first pixel is (ox, oy).  For a pixel at local offset (lx, ly) the biased
// edge value is E'(origin) + 256 (A lx + B ly); it is >= 0 iff
// A lx + B ly >= thr with thr = ceil(-E'(origin) / 256).  Inside the guard
// band |A|, |B| < 2^23 and lx, ly < 32, so |A lx + B ly| < 2^29: thr is
// clamped to +-2^30 and the test runs in int32.
//
// h2.w receives a conservative mask of the tile's warps (bit w: the 32
// pixels of threads 32w..32w+31, rows w*R .. w*R+R-1 with R = 32 / TW) whose
// pixel centres the triangle may cover: for each edge the largest
// A lx + B ly over the warp's rectangle (at a corner) must reach thr.
template <int TW>
__device__ __forceinline__ void stage_triangle(TileStage& sm, int slot, const SetupRec* recs, size_t vbase,
                                               uint32_t key, uint32_t t, int DB, int ox, int oy) {
    const SetupRec r = load_rec(recs + vbase + t);
    const long long X0 = 256LL * ox + 128, Y0 = 256LL * oy + 128;
    int thr[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long eb = (long long)r.A[i] * X0 + (long long)r.B[i] * Y0 + r.C[i];
        long long th = -(eb >> 8);
        th = th < -(1LL << 30) ? -(1LL << 30) : (th > (1LL << 30) ? (1LL << 30) : th);
        thr[i] = (int)th;
        sm.eo[slot][i] = eb + ((r.bias >> i) & 1u);
        sm.kk[slot][i] = r.k[i];
    }
    constexpr int R = 32 / TW;   // rows per warp
    int wmask = 0;
#pragma unroll
    for (int w = 0; w < kTilePix / 32; ++w) {
        bool may = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int mx = r.A[i] > 0 ? r.A[i] * (TW - 1) : 0;
            const int my = r.B[i] * (r.B[i] > 0 ? w * R + R - 1 : w * R);
            may = may && (mx + my >= thr[i]);
        }
        wmask |= may ? 1 << w : 0;
    }
    sm.h0[slot] = make_int4(r.A[0], r.B[0], thr[0], r.A[1]);
    sm.h1[slot] = make_int4(r.B[1], thr[1], r.A[2], r.B[2]);
    sm.h2[slot] = make_int4(thr[2], (int)t, __float_as_int(rho_bound(key, DB)), wmask);
}

// Coverage of local pixel (lx, ly) by staged triangle j; on success E gets
// the exact oriented edge values (int64) at the pixel centre.
__device__ __forceinline__ bool tile_cover(const TileStage& sm, int j, int lx, int ly, long long E[3]) {
    const int4 h0 = sm.h0[j], h1 = sm.h1[j], h2 = sm.h2[j];
    const int a0 = h0.x * lx + h0.y * ly;
    const int a1 = h0.w * lx + h1.x * ly;
    const int a2 = h1.z * lx + h1.w * ly;
    if (((a0 - h0.z) | (a1 - h1.y) | (a2 - h2.x)) < 0) return false;
    E[0] = sm.eo[j][0] + 256LL * a0;
    E[1] = sm.eo[j][1] + 256LL * a1;
    E[2] = sm.eo[j][2] + 256LL * a2;
    return true;
}

// The masked z-test of one work item (Eq. 5): walk the tile's list (staged
// in shared memory chunk by chunk) and keep, per sample, the foremost
// covered fragment whose interpolated opacity exceeds its threshold.  Warps
// stop once every sample holds a fragment in front of the depth bound of the
// rest of the list.  Returns true when the whole list was staged in one chunk
// (it is then still in shared memory).
template <int SG, int TW>
__device__ __forceinline__ bool forward_walk(TileStage& sm, const SetupRec* __restrict__ recs,
                                             const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                             uint2 rg, int DB, int chunk, size_t vbase, const WorkItem& wi,
                                             const SoupDev& s, int tid, int lx, int ly, int warp, bool valid, int px,
                                             int py, int ns, uint2 seed, bool stochastic, int (&bt)[SG],
                                             float (&brho)[SG], float (&bb1)[SG], float (&bb2)[SG], float (&bD)[SG]) {
    constexpr int TH = kTilePix / TW;
    bool warp_done = !__any_sync(kFullMask, valid);
    for (uint32_t c0 = rg.x; c0 < rg.y; c0 += (uint32_t)chunk) {
        const int n = (int)min((uint32_t)chunk, rg.y - c0);
        __syncthreads();
        if (tid < n)
            stage_triangle<TW>(sm, tid, recs, vbase, keys[c0 + tid], vals[c0 + tid], DB, wi.tx * TW, wi.ty * TH);
        __syncthreads();
        if (!warp_done) {
            for (int j = 0; j < n; ++j) {
                const int4 h2 = sm.h2[j];
                if (!((h2.w >> warp) & 1)) continue;   // covers none of this warp's pixels
                // early exit: every sample already holds a fragment in
                // front of anything the rest of the (depth-sorted) list can
                // give (without depth bits in the key the bound is infinite)
                if (DB > 0) {
                    bool ldone = true;
                    if (valid) {
#pragma unroll
                        for (int q = 0; q < SG; ++q)
                            if (q < ns) ldone = ldone && bt[q] >= 0 && brho[q] > __int_as_float(h2.z);
                    }
                    if (__all_sync(kFullMask, ldone)) {
                        warp_done = true;
                        break;
                    }
                }
                if (!valid) continue;
                long long E[3];
                if (!tile_cover(sm, j, lx, ly, E)) continue;
                const int t = h2.y;
                const Frag f = make_frag(E[0], E[1], E[2], sm.kk[j][0], sm.kk[j][1], sm.kk[j][2]);
                bool need = false;
#pragma unroll
                for (int q = 0; q < SG; ++q)
                    need = need || (q < ns && (bt[q] < 0 || in_front(f.rho, t, brho[q], bt[q])));
                if (!need) continue;
                const float r = __frcp_rn(f.rho);
                const float b1 = __fmul_rn(f.q1, r), b2 = __fmul_rn(f.q2, r);
                const Cell cl = find_cell(s.N, b1, b2);
                const float* aa = s.act_a + (size_t)t * s.V;
                const float alpha = interp(__ldg(aa + cl.k0), __ldg(aa + cl.k1), __ldg(aa + cl.k2), cl.wa, cl.wb);
                float tau[4] = {0.5f, 0.5f, 0.5f, 0.5f};
                if (stochastic) {
                    const uint4 w = philox4x32_10(make_uint4((uint32_t)px, (uint32_t)py, (uint32_t)t, (uint32_t)wi.g),
                                                  seed.x, seed.y);
                    tau[0] = word_to_tau(w.x);
                    tau[1] = word_to_tau(w.y);
                    tau[2] = word_to_tau(w.z);
                    tau[3] = word_to_tau(w.w);
                }
#pragma unroll
                for (int q = 0; q < SG; ++q) {
                    if (q < ns && alpha > tau[q] && (bt[q] < 0 || in_front(f.rho, t, brho[q], bt[q]))) {
                        bt[q] = t;
                        brho[q] = f.rho;
                        bb1[q] = b1;
                        bb2[q] = b2;
                        bD[q] = r;
                    }
                }
            }
        }
        if (__syncthreads_and(warp_done)) break;
    }
    return rg.y - rg.x <= (uint32_t)chunk;
}

// Inverse depth of triangle `rec` at pixel (px, py) (the stored winner's
// key, recomputed bit for bit).  +inf if the record does not cover the pixel.
__device__ __forceinline__ float winner_rho(const SetupRec* rec, int px, int py) {
    const SetupRec r = load_rec(rec);
    long long E[3];
    if (!cover_exact(r, px, py, E)) return __int_as_float(0x7f800000);
    return make_frag(E[0], E[1], E[2], r.k[0], r.k[1], r.k[2]).rho;
}

// Decode the C-1 colour channels of triangle t at (b1, b2) into out[c * HW].
__device__ __forceinline__ void decode_color(const SoupDev& s, int t, float b1, float b2, float* out, size_t HW) {
    const Cell cl = find_cell(s.N, b1, b2);
    const int C = s.C;
    const float* base = s.act + (size_t)t * s.V * C;
    const float* p0 = base + (size_t)cl.k0 * C;
    const float* p1 = base + (size_t)cl.k1 * C;
    const float* p2 = base + (size_t)cl.k2 * C;
    if ((C & 3) == 0) {
        for (int c4 = 0; c4 < C; c4 += 4) {
            const float4 a0 = __ldg(reinterpret_cast<const float4*>(p0 + c4));
            const float4 a1 = __ldg(reinterpret_cast<const float4*>(p1 + c4));
            const float4 a2 = __ldg(reinterpret_cast<const float4*>(p2 + c4));
            const float v[4] = {interp(a0.x, a1.x, a2.x, cl.wa, cl.wb), interp(a0.y, a1.y, a2.y, cl.wa, cl.wb),
                                interp(a0.z, a1.z, a2.z, cl.wa, cl.wb), interp(a0.w, a1.w, a2.w, cl.wa, cl.wb)};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c4 + k < C - 1) out[(c4 + k) * HW] = v[k];
        }
    } else {
        for (int c = 0; c < C - 1; ++c)
            out[c * HW] = interp(__ldg(p0 + c), __ldg(p1 + c), __ldg(p2 + c), cl.wa, cl.wb);
    }
}

// Colour of the selected fragment (or the background), written to col[c*HW],
// with the per-pixel L2 loss against tgt[c*HW] and its upstream gradient
// gc[c*HW] = 2 scale (colour - target); returns l = sum_c (colour - target)^2.
// Same arithmetic, in the same order, as the forward's decode followed by
// ds_loss_l2.
__device__ __forceinline__ float color_loss_out(const SoupDev& s, int t, float b1, float b2, const Bg& bg,
                                                const float* __restrict__ tgt, float* __restrict__ col,
                                                float* __restrict__ gc, size_t HW, float two_scale) {
    const int Co = s.C - 1;
    float ell = 0.f;
    auto emit = [&](int c, float v) {
        col[c * HW] = v;
        const float d = __fsub_rn(v, __ldg(tgt + c * HW));
        ell = __fmaf_rn(d, d, ell);
        gc[c * HW] = __fmul_rn(two_scale, d);
    };
    if (t < 0) {
#pragma unroll
        for (int c = 0; c < DS_MAX_CHANNELS; ++c)   // constant indices into the parameter struct
            if (c < Co) emit(c, bg.c[c]);
        return ell;
    }
    const Cell cl = find_cell(s.N, b1, b2);
    const int C = s.C;
    const float* base = s.act + (size_t)t * s.V * C;
    const float* p0 = base + (size_t)cl.k0 * C;
    const float* p1 = base + (size_t)cl.k1 * C;
    const float* p2 = base + (size_t)cl.k2 * C;
    if ((C & 3) == 0) {
        for (int c4 = 0; c4 < C; c4 += 4) {
            const float4 a0 = __ldg(reinterpret_cast<const float4*>(p0 + c4));
            const float4 a1 = __ldg(reinterpret_cast<const float4*>(p1 + c4));
            const float4 a2 = __ldg(reinterpret_cast<const float4*>(p2 + c4));
            const float v[4] = {interp(a0.x, a1.x, a2.x, cl.wa, cl.wb), interp(a0.y, a1.y, a2.y, cl.wa, cl.wb),
                                interp(a0.z, a1.z, a2.z, cl.wa, cl.wb), interp(a0.w, a1.w, a2.w, cl.wa, cl.wb)};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c4 + k < Co) emit(c4 + k, v[k]);
        }
    } else {
        for (int c = 0; c < Co; ++c) emit(c, interp(__ldg(p0 + c), __ldg(p1 + c), __ldg(p2 + c), cl.wa, cl.wb));
    }
    return ell;
}

// Sum NV values over runs of consecutive lanes that hold the same key.  On
// return the first lane of every run holds the run's sums; the function
// returns true there.  All 32 lanes must call it; a lane with nothing to add
// passes a key no other lane uses (so it forms a run of its own).
template <int NV>
__device__ __forceinline__ bool warp_run_sum(unsigned long long key, float (&v)[NV]) {
    const int lane = threadIdx.x & 31;
    const unsigned long long prev = __shfl_up_sync(kFullMask, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(kFullMask, head);
    const unsigned above = heads & ~((2u << lane) - 1u);
    const int end = above ? __ffs(above) - 1 : 32;
    if (heads == kFullMask) return true;   // every run has one lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (!__any_sync(kFullMask, lane + d < end)) break;   // no run is longer than d
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const float o = __shfl_down_sync(kFullMask, v[q], d);
            if (lane + d < end) v[q] += o;
        }
    }
    return head;
}

// Sort (key, val) ascending over the 32 lanes of the warp (bitonic network,
// 15 compare-exchange steps by shuffles; equal keys never swap).  All 32
// lanes must call it.
__device__ __forceinline__ void warp_sort32(unsigned& key, int& val) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned ok = __shfl_xor_sync(kFullMask, key, j);
            const int ov = __shfl_xor_sync(kFullMask, val, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            if (lower == up ? ok < key : ok > key) {
                key = ok;
                val = ov;
            }
        }
}

// A key no other lane uses (for lanes with nothing to add in warp_run_sum).
__device__ __forceinline__ unsigned long long lane_sentinel() {
    return 0xffffffffffff0000ull | (threadIdx.x & 31);
}

// Eq. 9 for every covered fragment in front of the winner of each sample
// (Algorithm A1 2(b), G-buffer recomputation): walk the tile's list again and
// scatter -w/(1 - alpha) to the opacity texels of the fragments in front.
// `staged`: the whole list is already in shared memory (one chunk).
//
// The walk is warp-synchronous over the staged triangles, and a small
// triangle covers few of a warp's pixels, so the opacity lookup and the
// scatter of a fragment in front are not done where it is found: each lane
// appends (triangle, barycentrics, summed score weight) to the warp's ring
// in shared memory, and whenever 32 jobs wait the warp evaluates them with
// every lane busy (the rest after the walk).
struct ScoreJob {
    int t;
    float b1, b2;
    float gw;   // sum of the score weights of the samples whose winner lies behind
};
constexpr int kScoreRing = 64;   // up to 31 waiting jobs + 32 new ones

// Evaluate n <= 32 jobs of the ring from `head`: opacity at the fragment,
// g = -gw / (1 - alpha), chained through the interpolation weights and the
// sigmoid (a (1 - a) at each corner texel), summed over runs of lanes on
// the same cell, one FP64 atomic per corner and run.
__device__ __forceinline__ void score_batch(const SoupDev& s, double* __restrict__ acc_tex, const ScoreJob* ring,
                                            int head, int n) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < n;
    ScoreJob jb{0, 0.f, 0.f, 0.f};
    if (act) jb = ring[(head + lane) & (kScoreRing - 1)];
    Cell cl;
    cl.k0 = cl.k1 = cl.k2 = 0;
    cl.wa = cl.wb = 0.f;
    cl.lower = true;
    float v[3] = {0.f, 0.f, 0.f};
    unsigned long long key = lane_sentinel();
    if (act) {
        cl = find_cell(s.N, jb.b1, jb.b2);
        const float* aa = s.act_a + (size_t)jb.t * s.V;
        const float a0 = __ldg(aa + cl.k0), a1 = __ldg(aa + cl.k1), a2 = __ldg(aa + cl.k2);
        const float alpha = interp(a0, a1, a2, cl.wa, cl.wb);
        const float g = -jb.gw / (1.0f - alpha);
        v[0] = g * (1.0f - cl.wa - cl.wb) * (a0 * (1.0f - a0));
        v[1] = g * cl.wa * (a1 * (1.0f - a1));
        v[2] = g * cl.wb * (a2 * (1.0f - a2));
        key = ((unsigned long long)(unsigned)jb.t << 20) | ((unsigned)cl.k0 << 1) | (cl.lower ? 1u : 0u);
    }
    const bool head_lane = warp_run_sum<3>(key, v);
    if (act && head_lane) {
        const int ks[3] = {cl.k0, cl.k1, cl.k2};
#pragma unroll
        for (int m = 0; m < 3; ++m)
            atomicAdd(acc_tex + ((size_t)jb.t * s.V + ks[m]) * s.C + (s.C - 1), (double)v[m]);
    }
}

template <int SG, int TW>
__device__ __forceinline__ void score_walk(TileStage& sm, const SetupRec* __restrict__ recs,
                                           const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                           uint2 rg, int DB, int chunk, size_t vbase, const WorkItem& wi,
                                           const SoupDev& s, double* __restrict__ acc_tex, int tid, int lx, int ly,
                                           int warp, bool staged, bool any_score, const int (&wt)[SG],
                                           const float (&wrho)[SG], const float (&wsc)[SG], ScoreJob* ring) {
    constexpr int TH = kTilePix / TW;
    const unsigned lt = (1u << (tid & 31)) - 1u;
    int head = 0, count = 0;   // the warp's ring (same values in every lane)
    bool warp_done = !__any_sync(kFullMask, any_score);
    if (__syncthreads_or(!warp_done)) {
        for (uint32_t c0 = rg.x; c0 < rg.y; c0 += (uint32_t)chunk) {
            const int n = (int)min((uint32_t)chunk, rg.y - c0);
            __syncthreads();
            if (!staged) {
                if (tid < n)
                    stage_triangle<TW>(sm, tid, recs, vbase, keys[c0 + tid], vals[c0 + tid], DB, wi.tx * TW,
                                       wi.ty * TH);
                __syncthreads();
            }
            if (!warp_done) {
                for (int j = 0; j < n; ++j) {
                    const int4 h2 = sm.h2[j];
                    if (!((h2.w >> warp) & 1)) continue;   // covers none of this warp's pixels
                    if (DB > 0) {   // without depth bits the bound is infinite
                        bool ldone = true;
#pragma unroll
                        for (int q = 0; q < SG; ++q)
                            if (wsc[q] != 0.f) ldone = ldone && wt[q] >= 0 && wrho[q] > __int_as_float(h2.z);
                        if (__all_sync(kFullMask, ldone)) {
                            warp_done = true;
                            break;
                        }
                    }
                    const int t = h2.y;
                    bool need = false;
                    float gw = 0.f, b1 = 0.f, b2 = 0.f;
                    long long E[3];
                    if (any_score && tile_cover(sm, j, lx, ly, E)) {
                        const Frag f = make_frag(E[0], E[1], E[2], sm.kk[j][0], sm.kk[j][1], sm.kk[j][2]);
#pragma unroll
                        for (int q = 0; q < SG; ++q)
                            if (wsc[q] != 0.f && t != wt[q] && (wt[q] < 0 || in_front(f.rho, t, wrho[q], wt[q]))) {
                                need = true;
                                gw += wsc[q];
                            }
                        if (need) {
                            const float r = __frcp_rn(f.rho);
                            b1 = __fmul_rn(f.q1, r);
                            b2 = __fmul_rn(f.q2, r);
                        }
                    }
                    const unsigned bal = __ballot_sync(kFullMask, need);
                    if (bal) {
                        if (need) ring[(head + count + __popc(bal & lt)) & (kScoreRing - 1)] = ScoreJob{t, b1, b2, gw};
                        count += __popc(bal);
                        __syncwarp();
                        if (count >= 32) {
                            score_batch(s, acc_tex, ring, head, 32);
                            head = (head + 32) & (kScoreRing - 1);
                            count -= 32;
                            __syncwarp();
                        }
                    }
                }
            }
            if (__syncthreads_and(warp_done)) break;
        }
    }
    if (count > 0) score_batch(s, acc_tex, ring, head, count);
    __syncwarp();
}

// Tile-kernel dispatch on the sample group (1, 2 or 4 samples per CTA) and
// the tile width (8, 16 or 32 pixels): calls f(IntPair<SG, TW>{}).
template <int A, int B>
struct IntPair {
    static constexpr int sg = A, tw = B;
};
template <class F>
inline void dispatch_tile(int tw, int sg, F&& f) {
    if (tw == 8) {
        if (sg == 1) f(IntPair<1, 8>{});
        else if (sg == 2) f(IntPair<2, 8>{});
        else f(IntPair<4, 8>{});
    } else if (tw == 32) {
        if (sg == 1) f(IntPair<1, 32>{});
        else if (sg == 2) f(IntPair<2, 32>{});
        else f(IntPair<4, 32>{});
    } else {
        if (sg == 1) f(IntPair<1, 16>{});
        else if (sg == 2) f(IntPair<2, 16>{});
        else f(IntPair<4, 16>{});
    }
}

}  // namespace ds
