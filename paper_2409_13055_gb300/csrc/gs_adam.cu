// gs_adam.cu -- A9 Adam (paper Sec. IV-A: the default 3DGS optimiser).
//
// One fused, HBM-bound pass over every parameter group: 16 bytes read
// (p, g, m, v) and 12 written (p, m, v) per float, float4-vectorised, grid
// sized to a multiple of the 152 SMs and striding over the buffer.  The step
// counter lives on the device and is advanced by a one-thread kernel first,
// so a captured CUDA graph replays correct bias corrections every iteration.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kAdamBlocks = 152 * 8;

struct Groups {
    long long off[GS_MAX_GROUPS + 1];
    float lr[GS_MAX_GROUPS];
    int n;
};

__global__ void k_step_inc(int32_t* step) { *step += 1; }

__device__ __forceinline__ float lr_of(const Groups& g, long long i) {
    float lr = g.lr[0];
#pragma unroll
    for (int k = 1; k < GS_MAX_GROUPS; ++k)
        if (k < g.n && i >= g.off[k]) lr = g.lr[k];
    return lr;
}

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                      float b2, float eps, float ibc1, float ibc2) {
    m = fmaf(b1, m, (1.0f - b1) * g);
    v = fmaf(b2, v, (1.0f - b2) * g * g);
    p -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

__global__ void __launch_bounds__(kAdamThreads)
k_adam(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
       float* __restrict__ v, long long n, Groups groups, float b1, float b2, float eps,
       const int32_t* __restrict__ step, int vec) {
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
        const int t = *step;
        s_bc[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
        s_bc[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
    }
    __syncthreads();
    const float ibc1 = s_bc[0], ibc2 = s_bc[1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = n >> 2;
        float4* P = reinterpret_cast<float4*>(params);
        const float4* G = reinterpret_cast<const float4*>(grads);
        float4* M = reinterpret_cast<float4*>(m);
        float4* V = reinterpret_cast<float4*>(v);
        for (long long i = tid; i < n4; i += stride) {
            float4 p4 = P[i], m4 = M[i], v4 = V[i];
            const float4 g4 = __ldcs(G + i);
            const long long e = i << 2;
            adam1(p4.x, g4.x, m4.x, v4.x, lr_of(groups, e), b1, b2, eps, ibc1, ibc2);
            adam1(p4.y, g4.y, m4.y, v4.y, lr_of(groups, e + 1), b1, b2, eps, ibc1, ibc2);
            adam1(p4.z, g4.z, m4.z, v4.z, lr_of(groups, e + 2), b1, b2, eps, ibc1, ibc2);
            adam1(p4.w, g4.w, m4.w, v4.w, lr_of(groups, e + 3), b1, b2, eps, ibc1, ibc2);
            P[i] = p4;
            M[i] = m4;
            V[i] = v4;
        }
        done = n4 << 2;
    }
    for (long long i = done + tid; i < n; i += stride) {
        float p = params[i], mm = m[i], vv = v[i];
        adam1(p, grads[i], mm, vv, lr_of(groups, i), b1, b2, eps, ibc1, ibc2);
        params[i] = p;
        m[i] = mm;
        v[i] = vv;
    }
}

}  // namespace

gs_status launch_adam(float* params, const float* grads, float* m, float* v, int64_t n,
                      int32_t n_groups, const int64_t* offs, const float* lrs, float b1, float b2,
                      float eps, int32_t* step_dev, cudaStream_t st) {
    Groups g;
    g.n = n_groups;
    for (int k = 0; k <= GS_MAX_GROUPS; ++k) g.off[k] = k <= n_groups ? offs[k] : n;
    for (int k = 0; k < GS_MAX_GROUPS; ++k) g.lr[k] = k < n_groups ? lrs[k] : 0.0f;
    const bool aligned = ((reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(grads) |
                           reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) &
                          15) == 0;
    long long work = aligned ? (n >> 2) : n;
    int blocks = (int)((work + kAdamThreads - 1) / kAdamThreads);
    if (blocks > kAdamBlocks) blocks = kAdamBlocks;
    if (blocks < 1) blocks = 1;
    k_step_inc<<<1, 1, 0, st>>>(step_dev);
    k_adam<<<blocks, kAdamThreads, 0, st>>>(params, grads, m, v, n, g, b1, b2, eps, step_dev,
                                            aligned ? 1 : 0);
    return launch_status();
}

}  // namespace gs
