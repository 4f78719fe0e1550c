// ds_ssim.cu -- the photometric loss lambda L1 + (1 - lambda) L_SSIM (Eq. 10,
// Sec. 3.4) per pixel, fused with its upstream gradients for the backward
// pass.  Per channel, SSIM uses an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2.  The
// per-pixel loss
//     ell_p = lambda mean_c |x - y| + (1 - lambda)(1 - mean_c ssim_c(p))
// is written as the score weight (scale * ell_p) and the colour gradient is
// that of scale * sum_p ell_p:
//     d/dx(q) = lambda sign(x - y)/C - (1 - lambda)/C [w*G1 + 2 x w*G2 + y w*G3](q),
// G1..G3 the derivatives of ssim with respect to the raw moments w*x, w*x^2,
// w*(xy) at each p (zero outside the image).
//
// One CTA per 64 x 16 output tile of one sample image: the inputs are staged
// with a 10-pixel halo, the five moments (separable blur) and ssim, G1..G3
// are formed on the tile plus a 5-pixel halo, and G1..G3 are blurred back
// onto the tile -- one pass, no intermediate maps in HBM.
//
// The blurs are issue-bound, so their operands are interleaved in shared
// memory as pairs that take the same weight -- (x, y), (x^2, y^2), (G1, G2)
// -- and each tap of a pair is one packed FP32 multiply-add (fma.rn.f32x2,
// the weight duplicated in both halves); x y and G3 stay scalar.  Every
// output keeps the order and rounding of its scalar FMA chain.
#include <cmath>
#include <new>

#include "ds_internal.h"

namespace ds {

namespace {

constexpr int kR = 5, kTaps = 2 * kR + 1;
constexpr int kTX = 64, kTY = 16;
constexpr int kIX = kTX + 4 * kR, kIY = kTY + 4 * kR;   // staged input 84 x 36
constexpr int kMX = kTX + 2 * kR, kMY = kTY + 2 * kR;   // moment region 74 x 26
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct SsimView {
    const float* color;    // [S][Co][H][W]
    const float* target;   // [Co][H][W]
    float* grad_color;     // [S][Co][H][W] or null
    float* score_w;        // [S][H][W] or null
    int W, H, tiles_x, tile0;   // first tile index of this view (all samples)
};

struct SsimTable {
    int n, S, Co, n_tiles;
    float lambda, scale;
    float w[kTaps];
    float2 wd[kTaps];   // (w, w)
    SsimView v[DS_MAX_VIEWS];
};

struct SsimSmem {
    float2 XY[kIY][kIX];            // (x, y)
    union {
        struct {
            float2 a[kIY][kMX];     // horizontal pass of (x, y)
            float2 b[kIY][kMX];     // of (x^2, y^2)
            float c[kIY][kMX];      // of x y
        } hm;
        struct {
            float2 a[kMY][kTX];     // horizontal pass of (G1, G2)
            float b[kMY][kTX];      // of G3
        } hg;
    };
    float2 Ga[kMY][kMX];            // (G1, G2)
    float Gb[kMY][kMX];             // G3
    float St[kTY][kTX];             // ssim of the tile's pixels (this channel)
};

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__global__ void __launch_bounds__(256) k_loss_l1_ssim(const __grid_constant__ SsimTable t, float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SsimSmem& sm = *reinterpret_cast<SsimSmem*>(smem_raw);
    // view, sample, tile of this CTA
    int item = blockIdx.x, vi = 0;
    while (vi + 1 < t.n && t.v[vi + 1].tile0 <= item) ++vi;
    const SsimView& V = t.v[vi];
    item -= V.tile0;
    const int tiles = V.tiles_x * ((V.H + kTY - 1) / kTY);
    const int s = item / tiles, tl = item - s * tiles;
    const int x0 = (tl % V.tiles_x) * kTX, y0 = (tl / V.tiles_x) * kTY;
    const size_t HW = (size_t)V.W * V.H;
    const int tid = threadIdx.x;

    float l1[4] = {0.f, 0.f, 0.f, 0.f}, ss[4] = {0.f, 0.f, 0.f, 0.f};
    // The staged inputs of channel c + 1 are loaded into registers while
    // channel c is processed (the loads' latency overlaps the blur passes).
    constexpr int kLoads = (kIX * kIY + 255) / 256;
    float px[kLoads], py[kLoads];
    auto load_regs = [&](int c) {
        const float* xs = V.color + ((size_t)s * t.Co + c) * HW;
        const float* ys = V.target + (size_t)c * HW;
#pragma unroll
        for (int i = 0; i < kLoads; ++i) {
            const int k = tid + 256 * i;
            const int r = k / kIX, q = k - r * kIX;
            const int gy = y0 - 2 * kR + r, gx = x0 - 2 * kR + q;
            const bool in = k < kIX * kIY && gx >= 0 && gx < V.W && gy >= 0 && gy < V.H;
            px[i] = in ? __ldg(xs + (size_t)gy * V.W + gx) : 0.f;
            py[i] = in ? __ldg(ys + (size_t)gy * V.W + gx) : 0.f;
        }
    };
    auto store_regs = [&]() {
#pragma unroll
        for (int i = 0; i < kLoads; ++i) {
            const int k = tid + 256 * i;
            if (k < kIX * kIY) {
                const int r = k / kIX, q = k - r * kIX;
                sm.XY[r][q] = make_float2(px[i], py[i]);
            }
        }
    };
    load_regs(0);
    store_regs();
    __syncthreads();
    for (int c = 0; c < t.Co; ++c) {
        if (c + 1 < t.Co) load_regs(c + 1);
        // 2. horizontal pass of the five moments, two neighbouring outputs
        //    per thread sharing their window (the pair starts at an even
        //    column: two input pairs per 16-byte read)
        for (int k = tid; k < kIY * (kMX / 2); k += 256) {
            const int r = k / (kMX / 2), q = 2 * (k - r * (kMX / 2));
            float2 A[2] = {}, B[2] = {};
            float Cxy[2] = {0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj <= kTaps; jj += 2) {
                const float4 in = *reinterpret_cast<const float4*>(&sm.XY[r][q + jj]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = jj + h;
                    const float2 v = h ? make_float2(in.z, in.w) : make_float2(in.x, in.y);
                    const float2 sq = __fmul2_rn(v, v);
                    const float xy = v.x * v.y;
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int tap = j - o;
                        if (tap < 0 || tap >= kTaps) continue;
                        A[o] = ffma2(t.wd[tap], v, A[o]);
                        B[o] = ffma2(t.wd[tap], sq, B[o]);
                        Cxy[o] = fmaf(t.w[tap], xy, Cxy[o]);
                    }
                }
            }
            *reinterpret_cast<float4*>(&sm.hm.a[r][q]) = make_float4(A[0].x, A[0].y, A[1].x, A[1].y);
            *reinterpret_cast<float4*>(&sm.hm.b[r][q]) = make_float4(B[0].x, B[0].y, B[1].x, B[1].y);
            *reinterpret_cast<float2*>(&sm.hm.c[r][q]) = make_float2(Cxy[0], Cxy[1]);
        }
        __syncthreads();
        // 3. vertical pass (two rows per thread), ssim and its derivatives
        //    w.r.t. the raw moments
        for (int k = tid; k < (kMY / 2) * kMX; k += 256) {
            const int rp = k / kMX, q = k - rp * kMX, r0 = 2 * rp;
            float2 A[2] = {}, B[2] = {};
            float Cxy[2] = {0.f, 0.f};
#pragma unroll
            for (int j = 0; j <= kTaps; ++j) {
                const float2 ha = sm.hm.a[r0 + j][q], hb = sm.hm.b[r0 + j][q];
                const float hc = sm.hm.c[r0 + j][q];
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int tap = j - o;
                    if (tap < 0 || tap >= kTaps) continue;
                    A[o] = ffma2(t.wd[tap], ha, A[o]);
                    B[o] = ffma2(t.wd[tap], hb, B[o]);
                    Cxy[o] = fmaf(t.w[tap], hc, Cxy[o]);
                }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int r = r0 + o;
                const int gy = y0 - kR + r, gx = x0 - kR + q;
                float g1 = 0.f, g2 = 0.f, g3 = 0.f;
                if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
                    const float mx = A[o].x, my = A[o].y;
                    const float A_ = 2.f * mx * my + kC1;
                    const float B_ = 2.f * (Cxy[o] - mx * my) + kC2;
                    const float Cc = mx * mx + my * my + kC1;
                    const float D = (B[o].x - mx * mx) + (B[o].y - my * my) + kC2;
                    // one reciprocal, 1/(Cc D)^2, gives ssim and its quotients by A, B, Cc, D
                    const float ab = A_ * B_, cd = Cc * D;
                    const float inv = 1.0f / (cd * cd);
                    const float ssim = ab * cd * inv;
                    const float sA = B_ * cd * inv, sB = A_ * cd * inv;   // ssim / A, ssim / B
                    const float sCc = ab * D * inv, sD = ab * Cc * inv;    // ssim / Cc, ssim / D
                    const float dmu = 2.f * my * sA - 2.f * mx * sCc;
                    const float dvar = -sD;
                    const float dcov = 2.f * sB;
                    g1 = dmu - 2.f * mx * dvar - my * dcov;
                    g2 = dvar;
                    g3 = dcov;
                    if (r >= kR && r < kR + kTY && q >= kR && q < kR + kTX) sm.St[r - kR][q - kR] = ssim;
                }
                sm.Ga[r][q] = make_float2(g1, g2);
                sm.Gb[r][q] = g3;
            }
        }
        __syncthreads();
        // 4. horizontal pass of G1..G3 (over the moments' buffer), two
        //    outputs per thread
        for (int k = tid; k < kMY * (kTX / 2); k += 256) {
            const int r = k / (kTX / 2), q = 2 * (k - r * (kTX / 2));
            float2 A[2] = {};
            float Bg[2] = {0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj <= kTaps; jj += 2) {
                const float4 ga = *reinterpret_cast<const float4*>(&sm.Ga[r][q + jj]);
                const float2 gb = *reinterpret_cast<const float2*>(&sm.Gb[r][q + jj]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = jj + h;
                    const float2 va = h ? make_float2(ga.z, ga.w) : make_float2(ga.x, ga.y);
                    const float vb = h ? gb.y : gb.x;
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int tap = j - o;
                        if (tap < 0 || tap >= kTaps) continue;
                        A[o] = ffma2(t.wd[tap], va, A[o]);
                        Bg[o] = fmaf(t.w[tap], vb, Bg[o]);
                    }
                }
            }
            *reinterpret_cast<float4*>(&sm.hg.a[r][q]) = make_float4(A[0].x, A[0].y, A[1].x, A[1].y);
            *reinterpret_cast<float2*>(&sm.hg.b[r][q]) = make_float2(Bg[0], Bg[1]);
        }
        __syncthreads();
        // 5. vertical pass onto the tile (four rows of one column per thread):
        //    gradient and the loss terms
        {
            const int q = tid % kTX, r0 = 4 * (tid / kTX);
            float2 A[4] = {};
            float Bg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kTaps + 3; ++j) {
                const float2 ha = sm.hg.a[r0 + j][q];
                const float hb = sm.hg.b[r0 + j][q];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int tap = j - o;
                    if (tap < 0 || tap >= kTaps) continue;
                    A[o] = ffma2(t.wd[tap], ha, A[o]);
                    Bg[o] = fmaf(t.w[tap], hb, Bg[o]);
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int r = r0 + o;
                const int gy = y0 + r, gx = x0 + q;
                if (gx >= V.W || gy >= V.H) continue;
                const float2 xy = sm.XY[r + 2 * kR][q + 2 * kR];
                const float x = xy.x, y = xy.y;
                const float d = x - y;
                l1[o] += fabsf(d);
                ss[o] += sm.St[r][q];
                if (V.grad_color) {
                    const float dsum = A[o].x + 2.f * x * A[o].y + y * Bg[o];
                    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    const float gval = (t.lambda * sg - (1.f - t.lambda) * dsum) / (float)t.Co;
                    V.grad_color[((size_t)s * t.Co + c) * HW + (size_t)gy * V.W + gx] = t.scale * gval;
                }
            }
        }
        __syncthreads();
        if (c + 1 < t.Co) {
            store_regs();
            __syncthreads();
        }
    }
    // per-pixel loss, score weight, total
    float acc = 0.f;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int q = tid % kTX, r = 4 * (tid / kTX) + h;
        const int gy = y0 + r, gx = x0 + q;
        if (gx >= V.W || gy >= V.H) continue;
        const float ell = t.lambda * l1[h] / (float)t.Co + (1.f - t.lambda) * (1.f - ss[h] / (float)t.Co);
        if (V.score_w) V.score_w[(size_t)s * HW + (size_t)gy * V.W + gx] = t.scale * ell;
        acc += ell;
    }
    if (loss) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        __shared__ float wsum[8];
        if ((tid & 31) == 0) wsum[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            float tot = 0.f;
            for (int u = 0; u < 8; ++u) tot += wsum[u];
            atomicAdd(loss, t.scale * tot);
        }
    }
}

}  // namespace

cudaError_t launch_loss_l1_ssim(int n_views, int S, int Co, const int* hw, const float* const* colors,
                                const float* const* targets, float* const* grad_colors, float* const* score_ws,
                                float lambda, float scale, float* loss, cudaStream_t st) {
    SsimTable* t = new (std::nothrow) SsimTable();
    if (!t) return cudaErrorMemoryAllocation;
    t->n = n_views;
    t->S = S;
    t->Co = Co;
    t->lambda = lambda;
    t->scale = scale;
    double w[kTaps], sum = 0.0;
    for (int j = 0; j < kTaps; ++j) {
        const double k = j - kR;
        w[j] = std::exp(-k * k / (2.0 * 1.5 * 1.5));
        sum += w[j];
    }
    for (int j = 0; j < kTaps; ++j) {
        t->w[j] = (float)(w[j] / sum);
        t->wd[j] = make_float2(t->w[j], t->w[j]);
    }
    int tile = 0;
    for (int v = 0; v < n_views; ++v) {
        SsimView& d = t->v[v];
        d.W = hw[2 * v];
        d.H = hw[2 * v + 1];
        d.color = colors[v];
        d.target = targets[v];
        d.grad_color = grad_colors ? grad_colors[v] : nullptr;
        d.score_w = score_ws ? score_ws[v] : nullptr;
        d.tiles_x = (d.W + kTX - 1) / kTX;
        d.tile0 = tile;
        tile += S * d.tiles_x * ((d.H + kTY - 1) / kTY);
    }
    t->n_tiles = tile;
    const size_t smem = sizeof(SsimSmem);
    cudaError_t e = cudaFuncSetAttribute(k_loss_l1_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && tile > 0) {
        k_loss_l1_ssim<<<tile, 256, smem, st>>>(*t, loss);
        note_launches(1);
        e = cudaGetLastError();
    }
    delete t;
    return e;
}

}  // namespace ds
