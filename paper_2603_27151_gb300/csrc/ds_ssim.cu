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
// One CTA per 32 x 16 output tile of one sample image: the inputs are staged
// with a 10-pixel halo, the five moments (separable blur) and ssim, G1..G3
// are formed on the tile plus a 5-pixel halo, and G1..G3 are blurred back
// onto the tile -- one pass, no intermediate maps in HBM.
#include <cmath>
#include <new>

#include "ds_internal.h"

namespace ds {

namespace {

constexpr int kR = 5, kTaps = 2 * kR + 1;
constexpr int kTX = 32, kTY = 16;
constexpr int kIX = kTX + 4 * kR, kIY = kTY + 4 * kR;   // staged input 52 x 36
constexpr int kMX = kTX + 2 * kR, kMY = kTY + 2 * kR;   // moment region 42 x 26
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

    float l1[2] = {0.f, 0.f}, ss[2] = {0.f, 0.f};
    for (int c = 0; c < t.Co; ++c) {
        const float* xs = V.color + ((size_t)s * t.Co + c) * HW;
        const float* ys = V.target + (size_t)c * HW;
        // 1. inputs with a 10-pixel halo (zero outside the image)
        for (int k = tid; k < kIX * kIY; k += 256) {
            const int r = k / kIX, q = k - r * kIX;
            const int gy = y0 - 2 * kR + r, gx = x0 - 2 * kR + q;
            const bool in = gx >= 0 && gx < V.W && gy >= 0 && gy < V.H;
            sm.X[r][q] = in ? __ldg(xs + (size_t)gy * V.W + gx) : 0.f;
            sm.Y[r][q] = in ? __ldg(ys + (size_t)gy * V.W + gx) : 0.f;
        }
        __syncthreads();
        // 2. horizontal pass of the five moments
        for (int k = tid; k < kIY * kMX; k += 256) {
            const int r = k / kMX, q = k - r * kMX;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
            for (int j = 0; j < kTaps; ++j) {
                const float w = t.w[j], x = sm.X[r][q + j], y = sm.Y[r][q + j];
                a0 = fmaf(w, x, a0);
                a1 = fmaf(w, y, a1);
                a2 = fmaf(w, x * x, a2);
                a3 = fmaf(w, y * y, a3);
                a4 = fmaf(w, x * y, a4);
            }
            sm.HM[0][r][q] = a0; sm.HM[1][r][q] = a1; sm.HM[2][r][q] = a2; sm.HM[3][r][q] = a3; sm.HM[4][r][q] = a4;
        }
        __syncthreads();
        // 3. vertical pass, ssim and its derivatives w.r.t. the raw moments
        for (int k = tid; k < kMY * kMX; k += 256) {
            const int r = k / kMX, q = k - r * kMX;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kTaps; ++j) {
                const float w = t.w[j];
#pragma unroll
                for (int u = 0; u < 5; ++u) m[u] = fmaf(w, sm.HM[u][r + j][q], m[u]);
            }
            const int gy = y0 - kR + r, gx = x0 - kR + q;
            float g1 = 0.f, g2 = 0.f, g3 = 0.f;
            if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
                const float mx = m[0], my = m[1];
                const float A = 2.f * mx * my + kC1;
                const float B = 2.f * (m[4] - mx * my) + kC2;
                const float Cc = mx * mx + my * my + kC1;
                const float D = (m[2] - mx * mx) + (m[3] - my * my) + kC2;
                const float sv = (A * B) / (Cc * D);
                const float dmu = sv * (2.f * my / A - 2.f * mx / Cc);
                const float dvar = -sv / D;
                const float dcov = 2.f * sv / B;
                g1 = dmu - 2.f * mx * dvar - my * dcov;
                g2 = dvar;
                g3 = dcov;
                if (r >= kR && r < kR + kTY && q >= kR && q < kR + kTX) sm.St[r - kR][q - kR] = sv;
            }
            sm.G[0][r][q] = g1; sm.G[1][r][q] = g2; sm.G[2][r][q] = g3;
        }
        __syncthreads();
        // 4. horizontal pass of G1..G3 (over the HM buffer)
        for (int k = tid; k < kMY * kTX; k += 256) {
            const int r = k / kTX, q = k - r * kTX;
            float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kTaps; ++j) {
                const float w = t.w[j];
#pragma unroll
                for (int u = 0; u < 3; ++u) a[u] = fmaf(w, sm.G[u][r][q + j], a[u]);
            }
            sm.HG[0][r][q] = a[0]; sm.HG[1][r][q] = a[1]; sm.HG[2][r][q] = a[2];
        }
        __syncthreads();
        // 5. vertical pass onto the tile: gradient and the loss terms
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = tid + 256 * h;
            const int r = k / kTX, q = k - r * kTX;
            const int gy = y0 + r, gx = x0 + q;
            if (gx >= V.W || gy >= V.H) continue;
            float b[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kTaps; ++j) {
                const float w = t.w[j];
#pragma unroll
                for (int u = 0; u < 3; ++u) b[u] = fmaf(w, sm.HG[u][r + j][q], b[u]);
            }
            const float x = sm.X[r + 2 * kR][q + 2 * kR], y = sm.Y[r + 2 * kR][q + 2 * kR];
            const float d = x - y;
            l1[h] += fabsf(d);
            ss[h] += sm.St[r][q];
            if (V.grad_color) {
                const float dsum = b[0] + 2.f * x * b[1] + y * b[2];
                const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                const float gval = (t.lambda * sg - (1.f - t.lambda) * dsum) / (float)t.Co;
                V.grad_color[((size_t)s * t.Co + c) * HW + (size_t)gy * V.W + gx] = t.scale * gval;
            }
        }
        __syncthreads();
    }
    // per-pixel loss, score weight, total
    float acc = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = tid + 256 * h;
        const int r = k / kTX, q = k - r * kTX;
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
