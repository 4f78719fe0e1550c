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

// blockIdx.y = view, blockIdx.z = sample; threads stride over the pixels.
__global__ void __launch_bounds__(256) k_loss_l2(const __grid_constant__ LossTable lt, float* __restrict__ loss) {
    const LossView& V = lt.v[blockIdx.y];
    const int s = blockIdx.z;
    const float* col = V.color + (size_t)s * lt.Co * V.HW;
    float* gc = V.grad_color ? V.grad_color + (size_t)s * lt.Co * V.HW : nullptr;
    float acc = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V.HW; p += gridDim.x * blockDim.x) {
        float ell = 0.f;
        for (int c = 0; c < lt.Co; ++c) {
            const float d = __fsub_rn(col[(size_t)c * V.HW + p], __ldg(V.target + (size_t)c * V.HW + p));
            ell = __fmaf_rn(d, d, ell);
            if (gc) gc[(size_t)c * V.HW + p] = __fmul_rn(2.0f * lt.scale, d);
        }
        if (V.score_w) V.score_w[(size_t)s * V.HW + p] = __fmul_rn(lt.scale, ell);
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
        most = std::max(most, (long long)lt->v[v].HW);
    }
    const int gx = (int)std::min<long long>((most + 1023) / 1024, 512);
    ds::k_loss_l2<<<dim3(gx, n_views, S), 256, 0, static_cast<cudaStream_t>(stream)>>>(*lt, loss);
    ds::note_launches(1);
    delete lt;
    return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ERR_CUDA;
}
