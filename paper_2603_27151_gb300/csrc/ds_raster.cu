// ds_raster.cu -- forward rasteriser: stochastic opacity masking (Eq. 5) by a
// z-buffer over each tile's depth-sorted triangle list, mesh-colour
// decode of the selected fragment, and the optional fragment counts.
#include <atomic>

#include "ds_internal.h"
#include "ds_tile.cuh"

namespace ds {

// One CTA (256 threads, one pixel each) per work item (view, tile, group of
// up to four samples), taken from a global counter until none is left.
// kLoss: the epilogue also evaluates the per-pixel L2 loss against the
// view's target and writes the upstream gradients and score weights (the
// first half of the fused training pass; same arithmetic as ds_loss_l2).
// kMulti: the views are of different soups (ViewDesc s_act, s_act_a,
// rec_base; the soups share N, C and V, given by s).
template <int SG, int TW, bool kLoss, bool kMulti>
__global__ void __launch_bounds__(kTilePix, SG == 4 ? DS_MINB_FWD : DS_MINB_FWD_SMALL)
    k_raster_fwd(const __grid_constant__ ViewTable vt, const SoupDev soup, const SetupRec* __restrict__ recs,
                 const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                 const uint2* __restrict__ ranges, int DB, uint32_t mode, const Bg bg, float scale,
                 float* __restrict__ loss, int* __restrict__ counter) {
    __shared__ TileStage sm;
    __shared__ int s_item;
    const int tid = threadIdx.x;
    constexpr int TH = kTilePix / TW;
    const int lx = tid & (TW - 1), ly = tid / TW, warp = tid >> 5;
    const bool stochastic = mode == DS_MODE_STOCHASTIC;
    float lsum = 0.f;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= vt.n_items) break;
        const WorkItem wi = decode_item(vt, item);
        const ViewDesc& V = vt.v[wi.v];
        SoupDev s = soup;
        size_t vbase = (size_t)wi.v * soup.T;
        if (kMulti) {
            s.act = V.s_act;
            s.act_a = V.s_act_a;
            s.T = V.s_T;
            vbase = (size_t)V.rec_base;
        }
        const int px = wi.tx * TW + lx, py = wi.ty * TH + ly;
        const bool valid = px < V.W && py < V.H;
        const int s0 = wi.g * kSampleGroup;
        const int ns = min(SG, vt.S - s0);
        const uint2 seed = view_seed(vt, wi.v);

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
        forward_walk<SG, TW>(sm, recs, keys, vals, rg, DB, vt.chunk, vbase, wi, s, tid, lx, ly, warp, valid,
                             px, py, ns, seed, stochastic, bt, brho, bb1, bb2, bD);

        if (valid) {
            const size_t HW = (size_t)V.H * V.W, pix = (size_t)py * V.W + px;
            const int Co = s.C - 1;
#pragma unroll
            for (int q = 0; q < SG; ++q) {
                if (q >= ns) continue;
                const int sg = s0 + q;
                reinterpret_cast<int4*>(V.gbuf)[sg * HW + pix] =
                    make_int4(bt[q], __float_as_int(bb1[q]), __float_as_int(bb2[q]), __float_as_int(bD[q]));
                float* out = V.color + (size_t)sg * Co * HW + pix;
                if (kLoss) {
                    const float ell = color_loss_out(s, bt[q], bb1[q], bb2[q], bg, V.target + pix, out,
                                                     const_cast<float*>(V.grad_color) + (size_t)sg * Co * HW + pix,
                                                     HW, 2.0f * scale);
                    if (V.score_w) const_cast<float*>(V.score_w)[sg * HW + pix] = __fmul_rn(scale, ell);
                    lsum += ell;
                } else if (bt[q] < 0) {
#pragma unroll
                    for (int c = 0; c < DS_MAX_CHANNELS; ++c)
                        if (c < Co) out[c * HW] = bg.c[c];
                } else {
                    decode_color(s, bt[q], bb1[q], bb2[q], out, HW);
                }
            }
        }
        __syncthreads();
    }
    if (kLoss) {
        __shared__ float s_loss[kTilePix / 32];
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
}

// Fragment counts.  mode 0: per sample, the covered fragments in front of
// the stored winner (all covered fragments for the background), written to
// n_front.  mode 1: covered fragments of the pixel (one sample), summed.
template <int SG, int TW>
__global__ void __launch_bounds__(kTilePix, DS_MINB_FWD)
    k_raster_count(const __grid_constant__ ViewTable vt, const SoupDev s, const SetupRec* __restrict__ recs,
                   const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                   const uint2* __restrict__ ranges, int DB, int mode, unsigned long long* __restrict__ total,
                   int* __restrict__ counter) {
    __shared__ TileStage sm;
    __shared__ int s_item;
    const int tid = threadIdx.x;
    constexpr int TH = kTilePix / TW;
    const int lx = tid & (TW - 1), ly = tid / TW, warp = tid >> 5;
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
        const int ns = mode == 0 ? min(SG, vt.S - s0) : 1;
        const size_t HW = (size_t)V.H * V.W, pix = (size_t)py * V.W + px;
        const size_t vbase = (size_t)V.rec_base;   // the view's records (per-view soups)

        int wt[SG], cnt[SG];
        float wrho[SG];
#pragma unroll
        for (int q = 0; q < SG; ++q) {
            wt[q] = -1;
            wrho[q] = 0.0f;
            cnt[q] = 0;
            if (mode == 0 && valid && q < ns) {
                wt[q] = reinterpret_cast<const int4*>(V.gbuf)[(s0 + q) * HW + pix].x;
                if (wt[q] < 0 || wt[q] >= V.s_T) wt[q] = -1;
                if (wt[q] >= 0) wrho[q] = winner_rho(recs + vbase + wt[q], px, py);
            }
        }
        const uint2 rg = ranges[V.tile_base + wi.ty * V.tiles_x + wi.tx];
        bool warp_done = !__any_sync(kFullMask, valid);
        for (uint32_t c0 = rg.x; c0 < rg.y; c0 += (uint32_t)vt.chunk) {
            const int n = (int)min((uint32_t)vt.chunk, rg.y - c0);
            __syncthreads();
            if (tid < n)
                stage_triangle<TW>(sm, tid, recs, vbase, keys[c0 + tid], vals[c0 + tid], DB, wi.tx * TW, wi.ty * TH);
            __syncthreads();
            if (!warp_done) {
                for (int j = 0; j < n; ++j) {
                    const int4 h2 = sm.h2[j];
                    if (!((h2.w >> warp) & 1)) continue;   // covers none of this warp's pixels
                    if (DB > 0) {   // without depth bits the bound is infinite
                        bool ldone = true;
                        if (valid && mode == 0) {
#pragma unroll
                            for (int q = 0; q < SG; ++q)
                                if (q < ns) ldone = ldone && wt[q] >= 0 && wrho[q] > __int_as_float(h2.z);
                        } else if (valid) {
                            ldone = false;
                        }
                        if (__all_sync(kFullMask, ldone)) {
                            warp_done = true;
                            break;
                        }
                    }
                    if (!valid) continue;
                    long long E[3];
                    if (!tile_cover(sm, j, lx, ly, E)) continue;
                    if (mode == 1) {
                        ++cnt[0];
                        continue;
                    }
                    const int t = h2.y;
                    const Frag f = make_frag(E[0], E[1], E[2], sm.kk[j][0], sm.kk[j][1], sm.kk[j][2]);
#pragma unroll
                    for (int q = 0; q < SG; ++q)
                        if (q < ns && (wt[q] < 0 || in_front(f.rho, t, wrho[q], wt[q]))) ++cnt[q];
                }
            }
            if (__syncthreads_and(warp_done)) break;
        }
        if (valid) {
            if (mode == 0) {
#pragma unroll
                for (int q = 0; q < SG; ++q)
                    if (q < ns) V.n_front[(s0 + q) * HW + pix] = cnt[q];
            }
        }
        if (mode == 1) {
            unsigned long long c = valid ? (unsigned long long)cnt[0] : 0ull;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(kFullMask, c, d);
            if ((tid & 31) == 0 && c) atomicAdd(total, c);
        }
        __syncthreads();
    }
}

cudaError_t launch_raster_fwd(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const uint32_t* keys,
                              const uint32_t* vals, const uint2* ranges, int DB, uint32_t mode, const Bg& bg,
                              int* counter, int grid, cudaStream_t st, bool with_loss, float scale, float* loss,
                              bool multi) {
    dispatch_tile(vt.tile_w, vt.S == 1 ? 1 : (vt.S == 2 ? 2 : 4), [&](auto P) {
        constexpr int SG = decltype(P)::sg, TW = decltype(P)::tw;
        if (with_loss)
            k_raster_fwd<SG, TW, true, false><<<resident_grid(k_raster_fwd<SG, TW, true, false>, vt.n_items, grid),
                                                kTilePix, 0, st>>>(vt, s, recs, keys, vals, ranges, DB, mode, bg, scale,
                                                                   loss, counter);
        else if (multi)
            k_raster_fwd<SG, TW, false, true><<<resident_grid(k_raster_fwd<SG, TW, false, true>, vt.n_items, grid),
                                                kTilePix, 0, st>>>(vt, s, recs, keys, vals, ranges, DB, mode, bg, scale,
                                                                   loss, counter);
        else
            k_raster_fwd<SG, TW, false, false><<<resident_grid(k_raster_fwd<SG, TW, false, false>, vt.n_items, grid),
                                                 kTilePix, 0, st>>>(vt, s, recs, keys, vals, ranges, DB, mode, bg, scale,
                                                                    loss, counter);
    });
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_raster_count(const ViewTable& vt, const SoupDev& s, const SetupRec* recs, const uint32_t* keys,
                                const uint32_t* vals, const uint2* ranges, int DB, int mode,
                                unsigned long long* total, int* counter, int grid, cudaStream_t st) {
    dispatch_tile(vt.tile_w, (mode == 1 || vt.S == 1) ? 1 : 4, [&](auto P) {
        constexpr int SG = decltype(P)::sg, TW = decltype(P)::tw;
        k_raster_count<SG, TW><<<resident_grid(k_raster_count<SG, TW>, vt.n_items, grid), kTilePix, 0, st>>>(
            vt, s, recs, keys, vals, ranges, DB, mode, total, counter);
    });
    note_launches(1);
    return cudaGetLastError();
}

const char* const kStageNames[kNumStages] = {"activate", "setup", "scan", "emit", "sort", "ranges",
                                             "raster_fwd", "count", "geom", "raster_bwd", "edge_bwd",
                                             "finish", "train"};

static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

int persistent_grid(int n_items, int blocks_per_sm) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = sms * blocks_per_sm;
    return n_items < g ? (n_items > 0 ? n_items : 1) : g;
}

}  // namespace ds
