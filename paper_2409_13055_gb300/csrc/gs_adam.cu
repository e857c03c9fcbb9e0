// gs_adam.cu -- A9 Adam (paper Sec. IV-A: the default 3DGS optimiser).
//
// One fused, HBM-bound pass over every parameter group: 16 bytes read
// (p, g, m, v) and 12 written (p, m, v) per float, float4-vectorised, grid
// sized to a multiple of the GPU's SM count and striding over the buffer; the
// gradient is read with a streaming hint (used once).  At most 2^31 - 1
// floats per call.  The step
// counter lives on the device and is advanced by a one-thread kernel first,
// so a captured CUDA graph replays correct bias corrections every iteration.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kAdamBlocksPerSm = 8;

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

// Visibility-masked variant: float j of a plane of s floats per Gaussian
// (means, log-scales and each SH plane: 3; quaternions: 4; opacities: 1)
// belongs to Gaussian j / s; floats of an invisible Gaussian are neither read
// nor written.  Grid: blockIdx.y = plane (planes listed on the host, each a
// contiguous run of s * n floats), each thread four consecutive floats of
// its plane, the owners found with divisions by the constants 1, 3 or 4.
// Memory traffic falls only where visible Gaussians are contiguous in index:
// a 32-byte sector is read whenever one of its floats is visible.
constexpr int kMaxPlanes = 64;
struct Planes {
    uint32_t start[kMaxPlanes];  // first float of the plane in the buffer
    uint8_t stride[kMaxPlanes];  // 1, 3 or 4 floats per Gaussian
    float lr[kMaxPlanes];
    int count;
};

template <int S>
__device__ __forceinline__ void sparse_scalar(float* __restrict__ params,
                                              const float* __restrict__ grads,
                                              float* __restrict__ m, float* __restrict__ v,
                                              uint32_t base, uint32_t j,
                                              const uint8_t* __restrict__ vis, float lr, float b1,
                                              float b2, float eps, float ibc1, float ibc2) {
    if (!vis[j / S]) return;
    const uint32_t i = base + j;
    float p = params[i], mm = m[i], vv = v[i];
    adam1(p, grads[i], mm, vv, lr, b1, b2, eps, ibc1, ibc2);
    params[i] = p;
    m[i] = mm;
    v[i] = vv;
}

// Aligned body of a plane in float4s: a float4 none of whose floats is
// visible is skipped without touching memory; otherwise the four floats are
// loaded as one vector and the visible ones updated (the others written back
// unchanged).
template <int S>
__device__ __forceinline__ void sparse_body(float* __restrict__ params,
                                            const float* __restrict__ grads,
                                            float* __restrict__ m, float* __restrict__ v,
                                            uint32_t base, uint32_t head, uint32_t n4,
                                            const uint8_t* __restrict__ vis, float lr, float b1,
                                            float b2, float eps, float ibc1, float ibc2) {
    for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < n4;
         f += gridDim.x * blockDim.x) {
        const uint32_t j = head + 4u * f;
        const bool o0 = vis[j / S], o1 = vis[(j + 1) / S], o2 = vis[(j + 2) / S],
                   o3 = vis[(j + 3) / S];
        if (!(o0 | o1 | o2 | o3)) continue;
        const uint32_t q = (base + j) >> 2;
        float4 p = reinterpret_cast<float4*>(params)[q];
        float4 mm = reinterpret_cast<float4*>(m)[q];
        float4 vv = reinterpret_cast<float4*>(v)[q];
        const float4 g = __ldcs(reinterpret_cast<const float4*>(grads) + q);
        if (o0) adam1(p.x, g.x, mm.x, vv.x, lr, b1, b2, eps, ibc1, ibc2);
        if (o1) adam1(p.y, g.y, mm.y, vv.y, lr, b1, b2, eps, ibc1, ibc2);
        if (o2) adam1(p.z, g.z, mm.z, vv.z, lr, b1, b2, eps, ibc1, ibc2);
        if (o3) adam1(p.w, g.w, mm.w, vv.w, lr, b1, b2, eps, ibc1, ibc2);
        reinterpret_cast<float4*>(params)[q] = p;
        reinterpret_cast<float4*>(m)[q] = mm;
        reinterpret_cast<float4*>(v)[q] = vv;
    }
}

// One plane per blockIdx.y: an unaligned head (< 4 floats up to the first
// 16-byte boundary of the buffer), the float4 body, a tail (< 4 floats).
// The buffers' base addresses are 16-byte aligned (checked on the host).
template <int S>
__device__ __forceinline__ void sparse_plane(float* params, const float* grads, float* m,
                                             float* v, uint32_t base, uint32_t len,
                                             const uint8_t* vis, float lr, float b1, float b2,
                                             float eps, float ibc1, float ibc2) {
    uint32_t head = (4u - (base & 3u)) & 3u;
    if (head > len) head = len;
    const uint32_t n4 = (len - head) >> 2, body_end = head + 4u * n4;
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const uint32_t t = threadIdx.x;
        const uint32_t j = t < 4 ? t : body_end + (t - 4);
        if ((t < 4 && j < head) || (t >= 4 && j < len))
            sparse_scalar<S>(params, grads, m, v, base, j, vis, lr, b1, b2, eps, ibc1, ibc2);
    }
    sparse_body<S>(params, grads, m, v, base, head, n4, vis, lr, b1, b2, eps, ibc1, ibc2);
}

__global__ void __launch_bounds__(kAdamThreads)
k_adam_sparse(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
              float* __restrict__ v, Planes planes, uint32_t n_gauss,
              const uint8_t* __restrict__ vis, float b1, float b2, float eps,
              const int32_t* __restrict__ step) {
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) adam_bias(b1, b2, *step, s_bc[0], s_bc[1]);
    __syncthreads();
    const int pl = blockIdx.y;
    const uint32_t S = planes.stride[pl], len = S * n_gauss, base = planes.start[pl];
    const float lr = planes.lr[pl];
    if (S == 3)
        sparse_plane<3>(params, grads, m, v, base, len, vis, lr, b1, b2, eps, s_bc[0], s_bc[1]);
    else if (S == 4)
        sparse_plane<4>(params, grads, m, v, base, len, vis, lr, b1, b2, eps, s_bc[0], s_bc[1]);
    else
        sparse_plane<1>(params, grads, m, v, base, len, vis, lr, b1, b2, eps, s_bc[0], s_bc[1]);
}

// Dense Adam with the gradient of whole groups of 32 consecutive Gaussians
// taken as zero and not read where group_vis[group] == 0 (groups that touch
// no tile, whose gradient the projection adjoint left unwritten): the update
// of k_adam, bit for bit, without the loads of known zeros.  Float j of a
// plane of S floats per Gaussian belongs to Gaussian j / S (S a compile-time
// 1, 3 or 4, so the division is a multiply); a grid-stride loop over the
// plane, a float4 per thread and trip (VEC) or a float.
template <int S, bool VEC>
__device__ __forceinline__ void groups_plane(float* __restrict__ params,
                                             const float* __restrict__ grads,
                                             float* __restrict__ m, float* __restrict__ v,
                                             uint32_t base, uint32_t len,
                                             const uint8_t* __restrict__ gvis, float lr,
                                             float b1, float b2, float eps, float ibc1,
                                             float ibc2, uint32_t t0, uint32_t stride) {
    auto scalar = [&](uint32_t j) {
        const uint32_t i = base + j;
        float p = params[i], mm = m[i], vv = v[i];
        const float g = gvis[(j / S) >> 5] ? grads[i] : 0.0f;
        adam1(p, g, mm, vv, lr, b1, b2, eps, ibc1, ibc2);
        params[i] = p;
        m[i] = mm;
        v[i] = vv;
    };
    if (VEC) {
        const uint32_t n4 = len >> 2;
        for (uint32_t f = t0; f < n4; f += stride) {
            const uint32_t j = 4u * f, q = (base + j) >> 2;
            float4 p = __ldcs(reinterpret_cast<float4*>(params) + q);
            float4 mm = __ldcs(reinterpret_cast<float4*>(m) + q);
            float4 vv = __ldcs(reinterpret_cast<float4*>(v) + q);
            const uint32_t ga = (j / S) >> 5, gb = ((j + 3) / S) >> 5;
            const bool va = gvis[ga] != 0, vb = ga == gb ? va : gvis[gb] != 0;
            float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (va && vb) {
                g = __ldcs(reinterpret_cast<const float4*>(grads) + q);
            } else if (va || vb) {  // the four floats straddle two groups
                const float* gp = grads + base + j;
                g.x = ((j / S) >> 5) == ga ? (va ? gp[0] : 0.0f) : (vb ? gp[0] : 0.0f);
                g.y = (((j + 1) / S) >> 5) == ga ? (va ? gp[1] : 0.0f) : (vb ? gp[1] : 0.0f);
                g.z = (((j + 2) / S) >> 5) == ga ? (va ? gp[2] : 0.0f) : (vb ? gp[2] : 0.0f);
                g.w = vb ? gp[3] : 0.0f;
            }
            adam1(p.x, g.x, mm.x, vv.x, lr, b1, b2, eps, ibc1, ibc2);
            adam1(p.y, g.y, mm.y, vv.y, lr, b1, b2, eps, ibc1, ibc2);
            adam1(p.z, g.z, mm.z, vv.z, lr, b1, b2, eps, ibc1, ibc2);
            adam1(p.w, g.w, mm.w, vv.w, lr, b1, b2, eps, ibc1, ibc2);
            __stcs(reinterpret_cast<float4*>(params) + q, p);
            __stcs(reinterpret_cast<float4*>(m) + q, mm);
            __stcs(reinterpret_cast<float4*>(v) + q, vv);
        }
        if (t0 < (len & 3u)) scalar(4u * n4 + t0);  // the last len % 4 floats
    } else {
        for (uint32_t j = t0; j < len; j += stride) scalar(j);
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kAdamThreads)
k_adam_groups(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
              float* __restrict__ v, Planes planes, uint32_t n_gauss,
              const uint8_t* __restrict__ gvis, float b1, float b2, float eps,
              const int32_t* __restrict__ step) {
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) adam_bias(b1, b2, *step, s_bc[0], s_bc[1]);
    __syncthreads();
    const float ibc1 = s_bc[0], ibc2 = s_bc[1];
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int pl = 0; pl < planes.count; ++pl) {
        const uint32_t S = planes.stride[pl], base = planes.start[pl];
        const float lr = planes.lr[pl];
        if (S == 3)
            groups_plane<3, VEC>(params, grads, m, v, base, 3u * n_gauss, gvis, lr, b1, b2, eps,
                                 ibc1, ibc2, t0, stride);
        else if (S == 4)
            groups_plane<4, VEC>(params, grads, m, v, base, 4u * n_gauss, gvis, lr, b1, b2, eps,
                                 ibc1, ibc2, t0, stride);
        else
            groups_plane<1, VEC>(params, grads, m, v, base, n_gauss, gvis, lr, b1, b2, eps, ibc1,
                                 ibc2, t0, stride);
    }
}

__global__ void k_visibility(int n, int n_views, const uint32_t* __restrict__ touched,
                             uint8_t* __restrict__ vis) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint8_t any = 0;
    for (int v = 0; v < n_views; ++v) any |= touched[(size_t)v * n + g] != 0u;
    vis[g] = any;
}

}  // namespace

gs_status launch_visibility(int n, int n_views, const uint32_t* touched, uint8_t* vis,
                            cudaStream_t st) {
    k_visibility<<<(n + 255) / 256, 256, 0, st>>>(n, n_views, touched, vis);
    return launch_status();
}

gs_status launch_adam_sparse(float* params, const float* grads, float* m, float* v, int64_t n,
                             int32_t n_groups, const int64_t* offs, const float* lrs,
                             const int32_t* strides, int32_t n_gauss, const uint8_t* vis,
                             float b1, float b2, float eps, int32_t* step_dev, cudaStream_t st) {
    if (n >= (int64_t(1) << 31)) return GS_ERR_UNSUPPORTED;
    Planes pl{};
    for (int k = 0; k < n_groups; ++k) {
        const int s = strides[k];
        if (s != 1 && s != 3 && s != 4) return GS_ERR_UNSUPPORTED;
        const int64_t plane = (int64_t)s * n_gauss;
        for (int64_t o = offs[k]; o + plane <= offs[k + 1]; o += plane) {
            if (pl.count == kMaxPlanes) return GS_ERR_UNSUPPORTED;
            pl.start[pl.count] = (uint32_t)o;
            pl.stride[pl.count] = (uint8_t)s;
            pl.lr[pl.count] = lrs[k];
            ++pl.count;
        }
    }
    if (pl.count == 0) return GS_ERR_INVALID;
    if (((reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(grads) |
          reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) != 0)
        return GS_ERR_INVALID;
    // a float4 per thread; enough CTAs along x to cover the largest plane
    // (4 n_gauss floats) with a few loop trips
    int bx = (int)((4LL * n_gauss + 4LL * kAdamThreads - 1) / (4LL * kAdamThreads));
    const int sms = sm_count();
    if (sms <= 0) return GS_ERR_CUDA;
    if (bx > sms * 4) bx = sms * 4;
    if (bx < 1) bx = 1;
    k_step_inc<<<1, 1, 0, st>>>(step_dev);
    k_adam_sparse<<<dim3(bx, pl.count), kAdamThreads, 0, st>>>(params, grads, m, v, pl,
                                                               (uint32_t)n_gauss, vis, b1, b2,
                                                               eps, step_dev);
    return launch_status();
}

gs_status launch_adam_groups(float* params, const float* grads, float* m, float* v, int64_t n,
                             int32_t n_groups, const int64_t* offs, const float* lrs,
                             const int32_t* strides, int32_t n_gauss, const uint8_t* group_vis,
                             float b1, float b2, float eps, int32_t* step_dev, cudaStream_t st) {
    if (n >= (int64_t(1) << 31)) return GS_ERR_UNSUPPORTED;
    Planes pl{};
    bool vec = ((reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(grads) |
                 reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    for (int k = 0; k < n_groups; ++k) {
        const int s = strides[k];
        if (s != 1 && s != 3 && s != 4) return GS_ERR_UNSUPPORTED;
        const int64_t plane = (int64_t)s * n_gauss;
        for (int64_t o = offs[k]; o + plane <= offs[k + 1]; o += plane) {
            if (pl.count == kMaxPlanes) return GS_ERR_UNSUPPORTED;
            pl.start[pl.count] = (uint32_t)o;
            pl.stride[pl.count] = (uint8_t)s;
            pl.lr[pl.count] = lrs[k];
            if (o & 3) vec = false;
            ++pl.count;
        }
    }
    if (pl.count == 0) return GS_ERR_INVALID;
    const int sms = sm_count();
    if (sms <= 0) return GS_ERR_CUDA;
    k_step_inc<<<1, 1, 0, st>>>(step_dev);
    auto* kern = vec ? k_adam_groups<true> : k_adam_groups<false>;
    kern<<<sms * kAdamBlocksPerSm, kAdamThreads, 0, st>>>(params, grads, m, v, pl, (uint32_t)n_gauss,
                                               group_vis, b1, b2, eps, step_dev);
    return launch_status();
}

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
    const int sms = sm_count();
    if (sms <= 0) return GS_ERR_CUDA;
    if (blocks > sms * kAdamBlocksPerSm) blocks = sms * kAdamBlocksPerSm;
    if (blocks < 1) blocks = 1;
    k_step_inc<<<1, 1, 0, st>>>(step_dev);
    k_adam<<<blocks, kAdamThreads, 0, st>>>(params, grads, m, v, n, g, b1, b2, eps, step_dev,
                                            aligned ? 1 : 0);
    return launch_status();
}

}  // namespace gs
