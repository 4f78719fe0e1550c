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
    SsimView v[DS_MAX_VIEWS];
};

struct SsimSmem {
    float X[kIY][kIX], Y[kIY][kIX];
    union {
        float HM[5][kIY][kMX];   // horizontal pass of x, y, x^2, y^2, xy
        float HG[3][kMY][kTX];   // horizontal pass of G1..G3
    };
    float G[3][kMY][kMX];
    float St[kTY][kTX];          // ssim of the tile's pixels (this channel)
};

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
                sm.X[r][q] = px[i];
                sm.Y[r][q] = py[i];
            }
        }
    };
    load_regs(0);
    store_regs();
    __syncthreads();
    for (int c = 0; c < t.Co; ++c) {
        if (c + 1 < t.Co) load_regs(c + 1);
        // 2. horizontal pass of the five moments, two neighbouring outputs
        //    per thread sharing their window (read and written as float2:
        //    the pair starts at an even column)
        for (int k = tid; k < kIY * (kMX / 2); k += 256) {
            const int r = k / (kMX / 2), q = 2 * (k - r * (kMX / 2));
            float a[2][5] = {};
#pragma unroll
            for (int jj = 0; jj <= kTaps; jj += 2) {
                const float2 x2 = *reinterpret_cast<const float2*>(&sm.X[r][q + jj]);
                const float2 y2 = *reinterpret_cast<const float2*>(&sm.Y[r][q + jj]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = jj + h;
                    const float x = h ? x2.y : x2.x, y = h ? y2.y : y2.x;
                    const float xx = x * x, yy = y * y, xy = x * y;
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int tap = j - o;
                        if (tap < 0 || tap >= kTaps) continue;
                        const float w = t.w[tap];
                        a[o][0] = fmaf(w, x, a[o][0]);
                        a[o][1] = fmaf(w, y, a[o][1]);
                        a[o][2] = fmaf(w, xx, a[o][2]);
                        a[o][3] = fmaf(w, yy, a[o][3]);
                        a[o][4] = fmaf(w, xy, a[o][4]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 5; ++u) *reinterpret_cast<float2*>(&sm.HM[u][r][q]) = make_float2(a[0][u], a[1][u]);
        }
        __syncthreads();
        // 3. vertical pass (two rows per thread), ssim and its derivatives
        //    w.r.t. the raw moments
        for (int k = tid; k < (kMY / 2) * kMX; k += 256) {
            const int rp = k / kMX, q = k - rp * kMX, r0 = 2 * rp;
            float m[2][5] = {};
#pragma unroll
            for (int j = 0; j <= kTaps; ++j) {
                float hv[5];
#pragma unroll
                for (int u = 0; u < 5; ++u) hv[u] = sm.HM[u][r0 + j][q];
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int tap = j - o;
                    if (tap < 0 || tap >= kTaps) continue;
                    const float w = t.w[tap];
#pragma unroll
                    for (int u = 0; u < 5; ++u) m[o][u] = fmaf(w, hv[u], m[o][u]);
                }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int r = r0 + o;
                const int gy = y0 - kR + r, gx = x0 - kR + q;
                float g1 = 0.f, g2 = 0.f, g3 = 0.f;
                if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
                    const float mx = m[o][0], my = m[o][1];
                    const float A = 2.f * mx * my + kC1;
                    const float B = 2.f * (m[o][4] - mx * my) + kC2;
                    const float Cc = mx * mx + my * my + kC1;
                    const float D = (m[o][2] - mx * mx) + (m[o][3] - my * my) + kC2;
                    // one reciprocal, 1/(Cc D)^2, gives ssim and its quotients by A, B, Cc, D
                    const float ab = A * B, cd = Cc * D;
                    const float inv = 1.0f / (cd * cd);
                    const float ssim = ab * cd * inv;
                    const float sA = B * cd * inv, sB = A * cd * inv;   // ssim / A, ssim / B
                    const float sCc = ab * D * inv, sD = ab * Cc * inv;  // ssim / Cc, ssim / D
                    const float dmu = 2.f * my * sA - 2.f * mx * sCc;
                    const float dvar = -sD;
                    const float dcov = 2.f * sB;
                    g1 = dmu - 2.f * mx * dvar - my * dcov;
                    g2 = dvar;
                    g3 = dcov;
                    if (r >= kR && r < kR + kTY && q >= kR && q < kR + kTX) sm.St[r - kR][q - kR] = ssim;
                }
                sm.G[0][r][q] = g1; sm.G[1][r][q] = g2; sm.G[2][r][q] = g3;
            }
        }
        __syncthreads();
        // 4. horizontal pass of G1..G3 (over the HM buffer), two outputs per
        //    thread (float2 reads and writes)
        for (int k = tid; k < kMY * (kTX / 2); k += 256) {
            const int r = k / (kTX / 2), q = 2 * (k - r * (kTX / 2));
            float a[2][3] = {};
#pragma unroll
            for (int jj = 0; jj <= kTaps; jj += 2) {
                float2 g2[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) g2[u] = *reinterpret_cast<const float2*>(&sm.G[u][r][q + jj]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = jj + h;
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int tap = j - o;
                        if (tap < 0 || tap >= kTaps) continue;
                        const float w = t.w[tap];
#pragma unroll
                        for (int u = 0; u < 3; ++u) a[o][u] = fmaf(w, h ? g2[u].y : g2[u].x, a[o][u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) *reinterpret_cast<float2*>(&sm.HG[u][r][q]) = make_float2(a[0][u], a[1][u]);
        }
        __syncthreads();
        // 5. vertical pass onto the tile (four rows of one column per thread):
        //    gradient and the loss terms
        {
            const int q = tid % kTX, r0 = 4 * (tid / kTX);
            float b[4][3] = {};
#pragma unroll
            for (int j = 0; j < kTaps + 3; ++j) {
                float hv[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) hv[u] = sm.HG[u][r0 + j][q];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int tap = j - o;
                    if (tap < 0 || tap >= kTaps) continue;
                    const float w = t.w[tap];
#pragma unroll
                    for (int u = 0; u < 3; ++u) b[o][u] = fmaf(w, hv[u], b[o][u]);
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int r = r0 + o;
                const int gy = y0 + r, gx = x0 + q;
                if (gx >= V.W || gy >= V.H) continue;
                const float x = sm.X[r + 2 * kR][q + 2 * kR], y = sm.Y[r + 2 * kR][q + 2 * kR];
                const float d = x - y;
                l1[o] += fabsf(d);
                ss[o] += sm.St[r][q];
                if (V.grad_color) {
                    const float dsum = b[o][0] + 2.f * x * b[o][1] + y * b[o][2];
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
    for (int j = 0; j < kTaps; ++j) t->w[j] = (float)(w[j] / sum);
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
