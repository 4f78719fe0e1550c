// ds_optim.cu -- the optimisers of Sec. 3.4 (supplementary "Hyperparameters"):
// Adam for textures and MLP weights, VectorAdam for vertex positions, as one
// fused step kernel.  A vector is `dim` consecutive values sharing one second
// moment from the squared norm of its gradient (dim = 1: Adam):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) |g|^2,
//   x <- x - lr (m c1) / (sqrt(v c2) + eps),  c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t).
// HBM-bound: one read of x, g, m, v and one write of x, m, v per value.
// Every value's update is adam_apply (ds_common.cuh), shared with the fused
// gradient finishes, so both give the same bits for the same gradient.
#include <cmath>

#include "ds_internal.h"

namespace ds {

namespace {

// dim = 1, four values per thread.
__global__ void __launch_bounds__(256) k_adam4(float4* __restrict__ x, const float4* __restrict__ g,
                                               float4* __restrict__ m, float4* __restrict__ v, long long n4,
                                               AdamDev a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 gi = __ldcs(g + i);
        float4 mi = m[i], vi = v[i], xi = x[i];
        adam_apply(xi.x, mi.x, vi.x, gi.x, a);
        adam_apply(xi.y, mi.y, vi.y, gi.y, a);
        adam_apply(xi.z, mi.z, vi.z, gi.z, a);
        adam_apply(xi.w, mi.w, vi.w, gi.w, a);
        m[i] = mi;
        v[i] = vi;
        x[i] = xi;
    }
}

// Any dim (1..4): one vector per thread; the second moment from the squared
// norm of the vector's gradient (VectorAdam), the same roundings as
// adam_apply (which it equals for dim = 1).
__global__ void __launch_bounds__(256) k_adam_vec(float* __restrict__ x, const float* __restrict__ g,
                                                  float* __restrict__ m, float* __restrict__ v, long long n_vec,
                                                  int dim, AdamDev a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_vec;
         i += (long long)gridDim.x * blockDim.x) {
        float gv[4], g2 = 0.f;
        for (int k = 0; k < dim; ++k) {
            gv[k] = __ldcs(g + i * dim + k);
            g2 = __fmaf_rn(gv[k], gv[k], g2);
        }
        const float vi = __fmaf_rn(a.b2, v[i], __fmul_rn(1.0f - a.b2, g2));
        v[i] = vi;
        const float den = __fadd_rn(__fsqrt_rn(__fmul_rn(vi, a.c2)), a.eps);
        for (int k = 0; k < dim; ++k) {
            const float mi = __fmaf_rn(a.b1, m[i * dim + k], __fmul_rn(1.0f - a.b1, gv[k]));
            m[i * dim + k] = mi;
            x[i * dim + k] = __fsub_rn(x[i * dim + k], __fdiv_rn(__fmul_rn(a.lr, __fmul_rn(mi, a.c1)), den));
        }
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

AdamDev make_adam(float lr, float b1, float b2, float eps, long long t) {
    AdamDev a;
    a.lr = lr;
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)t)));
    a.c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)t)));
    return a;
}

cudaError_t launch_adam(float* x, const float* g, float* m, float* v, long long n, int dim, float lr, float b1,
                        float b2, float eps, long long t, cudaStream_t st) {
    const AdamDev a = make_adam(lr, b1, b2, eps, t);
    if (n == 0) return cudaSuccess;
    const bool vec4 = dim == 1 && n % 4 == 0 && ((uintptr_t)x | (uintptr_t)g | (uintptr_t)m | (uintptr_t)v) % 16 == 0;
    if (vec4)
        k_adam4<<<grid_for(n / 4), 256, 0, st>>>(reinterpret_cast<float4*>(x), reinterpret_cast<const float4*>(g),
                                                 reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n / 4, a);
    else
        k_adam_vec<<<grid_for(n / dim), 256, 0, st>>>(x, g, m, v, n / dim, dim, a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ds
