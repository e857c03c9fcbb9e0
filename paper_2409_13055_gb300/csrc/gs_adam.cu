// gs_adam.cu -- A9 Adam (paper Sec. IV-A: the default 3DGS optimiser).
//
// One fused, HBM-bound pass over every parameter group: 16 bytes read
// (p, g, m, v) and 12 written (p, m, v) per float, float4-vectorised, grid
// sized to a multiple of the 152 SMs and striding over the buffer; the
// gradient is read with a streaming hint (used once).  At most 2^31 - 1
// floats per call.  The step
// counter lives on the device and is advanced by a one-thread kernel first,
// so a captured CUDA graph replays correct bias corrections every iteration.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kAdamBlocks = 152 * 8;

struct Groups {
    uint32_t off[GS_MAX_GROUPS + 1];  // element offsets (n < 2^31)
    float lr[GS_MAX_GROUPS];
    int n;
};

__global__ void k_step_inc(int32_t* step) { *step += 1; }

__device__ __forceinline__ float lr_of(const Groups& g, uint32_t i) {
    float lr = g.lr[0];
#pragma unroll
    for (int k = 1; k < GS_MAX_GROUPS; ++k)
        if (k < g.n && i >= g.off[k]) lr = g.lr[k];
    return lr;
}

// Learning rates of the four elements e..e+3; one lookup unless a group
// boundary falls inside the chunk.
__device__ __forceinline__ float4 lr4_of(const Groups& g, uint32_t e) {
    const float a = lr_of(g, e), d = lr_of(g, e + 3);
    if (a == d) return make_float4(a, a, a, a);
    return make_float4(a, lr_of(g, e + 1), lr_of(g, e + 2), d);
}

__device__ __forceinline__ void adam4(float4& p, const float4& g, float4& m, float4& v,
                                      const float4& lr, float b1, float b2, float eps, float ibc1,
                                      float ibc2) {
    adam1(p.x, g.x, m.x, v.x, lr.x, b1, b2, eps, ibc1, ibc2);
    adam1(p.y, g.y, m.y, v.y, lr.y, b1, b2, eps, ibc1, ibc2);
    adam1(p.z, g.z, m.z, v.z, lr.z, b1, b2, eps, ibc1, ibc2);
    adam1(p.w, g.w, m.w, v.w, lr.w, b1, b2, eps, ibc1, ibc2);
}

__global__ void __launch_bounds__(kAdamThreads)
k_adam(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
       float* __restrict__ v, long long n, Groups groups, float b1, float b2, float eps,
       const int32_t* __restrict__ step, int vec) {
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) adam_bias(b1, b2, *step, s_bc[0], s_bc[1]);
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
            float4 p0 = P[i], m0 = M[i], v0 = V[i];
            const float4 g0 = __ldcs(G + i);
            adam4(p0, g0, m0, v0, lr4_of(groups, (uint32_t)(i << 2)), b1, b2, eps, ibc1, ibc2);
            P[i] = p0;
            M[i] = m0;
            V[i] = v0;
        }
        done = n4 << 2;
    }
    for (long long i = done + tid; i < n; i += stride) {
        float p = params[i], mm = m[i], vv = v[i];
        adam1(p, grads[i], mm, vv, lr_of(groups, (uint32_t)i), b1, b2, eps, ibc1, ibc2);
        params[i] = p;
        m[i] = mm;
        v[i] = vv;
    }
}

}  // namespace

gs_status launch_step_inc(int32_t* step_dev, cudaStream_t st) {
    k_step_inc<<<1, 1, 0, st>>>(step_dev);
    return launch_status();
}

gs_status launch_adam(float* params, const float* grads, float* m, float* v, int64_t n,
                      int32_t n_groups, const int64_t* offs, const float* lrs, float b1, float b2,
                      float eps, int32_t* step_dev, cudaStream_t st) {
    if (n >= (int64_t(1) << 31)) return GS_ERR_UNSUPPORTED;
    Groups g;
    g.n = n_groups;
    for (int k = 0; k <= GS_MAX_GROUPS; ++k) g.off[k] = (uint32_t)(k <= n_groups ? offs[k] : n);
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
