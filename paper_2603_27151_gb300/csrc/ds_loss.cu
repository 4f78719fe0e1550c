// ds_loss.cu -- fused per-pixel L2 photometric loss and its upstream
// gradients for the backward pass (one read of the rendered colours, one
// write of dL/dC and of the score weights).
#include <string>

#include "ds_internal.h"

namespace ds {

struct LossView {
    const float* color;    // [S][Co][H][W]
    const float* target;   // [Co][H][W]
    float* grad_color;     // [S][Co][H][W]
    float* score_w;        // [S][H][W]
    int HW;
};

struct LossTable {
    int n, S, Co;
    float scale;
    LossView v[DS_MAX_VIEWS];
};

// blockIdx.y = view; threads stride over the view's S*H*W pixel-samples.
__global__ void __launch_bounds__(256) k_loss_l2(const __grid_constant__ LossTable lt, float* __restrict__ loss) {
    const LossView& V = lt.v[blockIdx.y];
    const long long n = (long long)lt.S * V.HW;
    float acc = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / V.HW, p = i - s * V.HW;
        float ell = 0.f;
        for (int c = 0; c < lt.Co; ++c) {
            const long long ci = (s * lt.Co + c) * V.HW + p;
            const float d = V.color[ci] - __ldg(V.target + (long long)c * V.HW + p);
            ell += d * d;
            if (V.grad_color) V.grad_color[ci] = 2.0f * lt.scale * d;
        }
        if (V.score_w) V.score_w[i] = lt.scale * ell;
        acc += ell;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    __shared__ float wsum[8];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += wsum[w];
        atomicAdd(loss, lt.scale * t);
    }
}

}  // namespace ds

namespace {
thread_local std::string g_loss_err;
}

extern "C" DS_API ds_status ds_loss_l2(int32_t n_views, int32_t S, int32_t C, const int32_t* hw,
                                       const float* const* colors, const float* const* targets,
                                       float* const* grad_colors, float* const* score_ws, float scale,
                                       float* loss, void* stream) {
    if (n_views < 1 || n_views > DS_MAX_VIEWS || S < 1 || C < 2 || C > DS_MAX_CHANNELS || !hw || !colors ||
        !targets)
        return DS_ERR_INVALID_ARG;
    ds::LossTable* lt = new (std::nothrow) ds::LossTable();
    if (!lt) return DS_ERR_OOM;
    lt->n = n_views;
    lt->S = S;
    lt->Co = C - 1;
    lt->scale = scale;
    long long most = 0;
    for (int v = 0; v < n_views; ++v) {
        if (hw[2 * v] < 1 || hw[2 * v + 1] < 1 || !colors[v] || !targets[v]) {
            delete lt;
            return DS_ERR_INVALID_ARG;
        }
        lt->v[v].HW = hw[2 * v] * hw[2 * v + 1];
        lt->v[v].color = colors[v];
        lt->v[v].target = targets[v];
        lt->v[v].grad_color = grad_colors ? grad_colors[v] : nullptr;
        lt->v[v].score_w = score_ws ? score_ws[v] : nullptr;
        most = std::max(most, (long long)S * lt->v[v].HW);
    }
    const int gx = (int)std::min<long long>((most + 255) / 256, 2048);
    ds::k_loss_l2<<<dim3(gx, n_views), 256, 0, static_cast<cudaStream_t>(stream)>>>(*lt, loss);
    ds::note_launches(1);
    delete lt;
    return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ERR_CUDA;
}
