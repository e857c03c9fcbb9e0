// gs_densify.cu -- adaptive density control (paper Sec. III-B: periodic
// densification of Gaussians with a high homodirectional view-space position
// gradient, the AbsGS criterion -- clone small ones, split large ones with the
// original 3DGS parameters -- and pruning of low-opacity Gaussians).
//
// Three steps, all deterministic:
//   gs_densify_stats  per Gaussian, over the plan's views: the statistic of
//                     this iteration added to accum / denom (no atomics);
//   gs_densify_count  category per Gaussian, per-256-block counts, then one
//                     CTA turns them into exclusive offsets and totals;
//   gs_densify_apply  the new map and moments, every output slot computed from
//                     the block offsets and a block-local rank, so the order
//                     is by index within each section (kept, clones, children).
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kDensThreads = 256;
constexpr int kScanCta = 1024;
enum Category { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

__global__ void k_densify_stats(int n, ViewTable vt, const uint32_t* __restrict__ touched,
                                const float* __restrict__ absgrad, float* __restrict__ accum,
                                float* __restrict__ denom) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float a = accum[g], d = denom[g];
    for (int v = 0; v < vt.n_views; ++v) {
        const size_t vg = (size_t)v * n + g;
        if (touched[vg] == 0u) continue;
        // pixel units -> normalised device coordinates: d/dx_ndc = W/2 d/dx_px
        const float hx = absgrad[2 * vg] * (0.5f * (float)vt.v[v].width);
        const float hy = absgrad[2 * vg + 1] * (0.5f * (float)vt.v[v].height);
        a += sqrtf(hx * hx + hy * hy);
        d += 1.0f;
    }
    accum[g] = a;
    denom[g] = d;
}

__device__ __forceinline__ int category(const gs_map& m, const float* accum, const float* denom,
                                        const gs_densify_config& c, int g) {
    const float op = 1.0f / (1.0f + expf(-m.opacity_logits[g]));
    if (op < c.min_opacity) return kPrune;
    const float d = denom[g];
    if (d > 0.0f && accum[g] / d >= c.grad_threshold) {
        const float* ls = m.log_scales + 3 * (size_t)g;
        const float smax = expf(fmaxf(ls[0], fmaxf(ls[1], ls[2])));
        return smax <= c.percent_dense * c.extent ? kClone : kSplit;
    }
    return kKeep;
}

// scratch: cnt[3][nb] per-block counts, off[3][nb] their exclusive offsets
__global__ void __launch_bounds__(kDensThreads)
k_densify_count(gs_map m, const float* __restrict__ accum, const float* __restrict__ denom,
                gs_densify_config c, uint32_t* __restrict__ cnt, int nb) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int cat = g < m.n ? category(m, accum, denom, c, g) : kPrune;
    const int keep = __syncthreads_count(cat == kKeep || cat == kClone);
    const int clone = __syncthreads_count(cat == kClone);
    const int split = __syncthreads_count(cat == kSplit);
    if (threadIdx.x == 0) {
        cnt[blockIdx.x] = (uint32_t)keep;
        cnt[nb + blockIdx.x] = (uint32_t)clone;
        cnt[2 * nb + blockIdx.x] = (uint32_t)split;
    }
}

__global__ void __launch_bounds__(kScanCta)
k_densify_scan(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ off, int nb,
               int32_t* __restrict__ counts) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = 0; s < 3; ++s) {
        if (threadIdx.x == 0) carry = 0u;
        __syncthreads();
        for (int base = 0; base < nb; base += kScanCta) {
            const int i = base + threadIdx.x;
            const uint32_t x = i < nb ? cnt[(size_t)s * nb + i] : 0u;
            uint32_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) warp_sum[w] = inc;
            __syncthreads();
            if (w == 0) {
                const uint32_t t = warp_sum[lane];
                uint32_t ti = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
                    if (lane >= o) ti += y;
                }
                warp_sum[lane] = ti - t;
            }
            __syncthreads();
            const uint32_t c0 = carry;
            if (i < nb) off[(size_t)s * nb + i] = c0 + warp_sum[w] + inc - x;
            __syncthreads();
            if (threadIdx.x == kScanCta - 1) carry = c0 + warp_sum[w] + inc;
            __syncthreads();
        }
        if (threadIdx.x == 0) counts[s] = (int32_t)carry;
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[3] = 0;
}

// Exclusive rank of a predicate within the CTA (block order = index order).
__device__ __forceinline__ int block_rank(bool pred, int* warp_cnt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, pred);
    if (lane == 0) warp_cnt[w] = __popc(b);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_cnt[k];
    __syncthreads();
    return before + __popc(b & ((1u << lane) - 1u));
}

struct DenseOut {
    gs_map_grad p, m, v;
    int n_out, K;
};

// Copies Gaussian g of the source (parameters, and moments or zeros) to slot o.
__device__ __forceinline__ void copy_gaussian(const gs_map& src, const gs_map_grad& sm,
                                              const gs_map_grad& sv, int g, const DenseOut& d,
                                              int o, bool moments) {
    const size_t gs = (size_t)g, os = (size_t)o;
    for (int e = 0; e < 3; ++e) {
        d.p.means[3 * os + e] = src.means[3 * gs + e];
        d.p.log_scales[3 * os + e] = src.log_scales[3 * gs + e];
        d.m.means[3 * os + e] = moments ? sm.means[3 * gs + e] : 0.0f;
        d.v.means[3 * os + e] = moments ? sv.means[3 * gs + e] : 0.0f;
        d.m.log_scales[3 * os + e] = moments ? sm.log_scales[3 * gs + e] : 0.0f;
        d.v.log_scales[3 * os + e] = moments ? sv.log_scales[3 * gs + e] : 0.0f;
    }
    for (int e = 0; e < 4; ++e) {
        d.p.quats[4 * os + e] = src.quats[4 * gs + e];
        d.m.quats[4 * os + e] = moments ? sm.quats[4 * gs + e] : 0.0f;
        d.v.quats[4 * os + e] = moments ? sv.quats[4 * gs + e] : 0.0f;
    }
    d.p.opacity_logits[os] = src.opacity_logits[gs];
    d.m.opacity_logits[os] = moments ? sm.opacity_logits[gs] : 0.0f;
    d.v.opacity_logits[os] = moments ? sv.opacity_logits[gs] : 0.0f;
    for (int k = 0; k < d.K; ++k)
        for (int c = 0; c < 3; ++c) {
            const size_t si = ((size_t)k * src.n + gs) * 3 + c;
            const size_t di = ((size_t)k * d.n_out + os) * 3 + c;
            d.p.sh[di] = src.sh[si];
            d.m.sh[di] = moments ? sm.sh[si] : 0.0f;
            d.v.sh[di] = moments ? sv.sh[si] : 0.0f;
        }
}

__global__ void __launch_bounds__(kDensThreads)
k_densify_apply(gs_map src, gs_map_grad sm, gs_map_grad sv, const float* __restrict__ accum,
                const float* __restrict__ denom, const float* __restrict__ samples,
                gs_densify_config c, const uint32_t* __restrict__ off, int nb, DenseOut d,
                int32_t* counts) {
    __shared__ int warp_cnt[kDensThreads / 32];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int cat = g < src.n ? category(src, accum, denom, c, g) : kPrune;
    const int rk = block_rank(cat == kKeep || cat == kClone, warp_cnt);
    const int rc = block_rank(cat == kClone, warp_cnt);
    const int rs = block_rank(cat == kSplit, warp_cnt);
    const int K = counts[0], C = counts[1], S = counts[2];
    if (K + C + 2 * S != d.n_out) {
        if (g == 0) counts[3] = 1;
        return;
    }
    if (g >= src.n || cat == kPrune) return;
    if (cat == kKeep || cat == kClone) {
        const int o = (int)off[blockIdx.x] + rk;
        copy_gaussian(src, sm, sv, g, d, o, true);
        if (cat == kClone) copy_gaussian(src, sm, sv, g, d, K + (int)off[nb + blockIdx.x] + rc,
                                         false);
        return;
    }
    // split: two children, mean + R(q/|q|) (s * xi), log-scales - log(shrink)
    const float* q = src.quats + 4 * (size_t)g;
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    const float* ls = src.log_scales + 3 * (size_t)g;
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    const float shrink = logf(c.split_shrink);
    for (int ch = 0; ch < 2; ++ch) {
        const int o = K + C + 2 * ((int)off[2 * nb + blockIdx.x] + rs) + ch;
        copy_gaussian(src, sm, sv, g, d, o, false);
        const float* xi = samples + ((size_t)g * 2 + ch) * 3;
        const float t0 = s[0] * xi[0], t1 = s[1] * xi[1], t2 = s[2] * xi[2];
        for (int e = 0; e < 3; ++e) {
            d.p.means[3 * (size_t)o + e] =
                src.means[3 * (size_t)g + e] + (R[3 * e] * t0 + R[3 * e + 1] * t1 + R[3 * e + 2] * t2);
            d.p.log_scales[3 * (size_t)o + e] = ls[e] - shrink;
        }
    }
}

bool cfg_ok(const gs_densify_config* c) {
    return c && c->grad_threshold >= 0.0f && c->percent_dense >= 0.0f && c->min_opacity >= 0.0f &&
           c->split_shrink > 0.0f && c->extent >= 0.0f;
}

bool map_ok(const gs_map* m) {
    return m && m->n >= 1 && m->sh_degree >= 0 && m->sh_degree <= 3 && m->means &&
           m->log_scales && m->quats && m->opacity_logits && m->sh;
}

bool grad_ok(const gs_map_grad* g) {
    return g && g->means && g->log_scales && g->quats && g->opacity_logits && g->sh;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_densify_stats(const gs_plan* plan, int32_t n, const void* ws,
                                      float* accum, float* denom, void* stream) {
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!plan || p->magic != kPlanMagic || !ws || !accum || !denom) return GS_ERR_INVALID;
    if (n < 1 || n > p->n_capacity || !p->cfg.density_stats) return GS_ERR_INVALID;
    if (p->vt.n_views > p->ws_views) return GS_ERR_INVALID;  // a pass of a recompute plan
    k_densify_stats<<<(n + kDensThreads - 1) / kDensThreads, kDensThreads, 0,
                      (cudaStream_t)stream>>>(n, p->vt, cbuf<uint32_t>(p, ws, GS_BUF_TOUCHED),
                                              cbuf<float>(p, ws, GS_BUF_ABSGRAD), accum, denom);
    return launch_status();
}

extern "C" size_t gs_densify_scratch_bytes(int32_t n) {
    if (n < 1) return 0;
    const size_t nb = ((size_t)n + kDensThreads - 1) / kDensThreads;
    return 6 * nb * sizeof(uint32_t) + 256;
}

extern "C" gs_status gs_densify_count(const gs_map* map, const float* accum, const float* denom,
                                      const gs_densify_config* cfg, void* scratch,
                                      int32_t* counts_dev, void* stream) {
    if (!map_ok(map) || !accum || !denom || !cfg_ok(cfg) || !scratch || !counts_dev)
        return GS_ERR_INVALID;
    const int nb = (map->n + kDensThreads - 1) / kDensThreads;
    uint32_t* cnt = static_cast<uint32_t*>(scratch);
    uint32_t* off = cnt + 3 * (size_t)nb;
    cudaStream_t st = (cudaStream_t)stream;
    k_densify_count<<<nb, kDensThreads, 0, st>>>(*map, accum, denom, *cfg, cnt, nb);
    k_densify_scan<<<1, kScanCta, 0, st>>>(cnt, off, nb, counts_dev);
    return launch_status();
}

extern "C" gs_status gs_densify_apply(const gs_map* map, const gs_map_grad* src_m,
                                      const gs_map_grad* src_v, const float* accum,
                                      const float* denom, const float* samples,
                                      const gs_densify_config* cfg, const void* scratch,
                                      int32_t n_out, gs_map_grad* dst, gs_map_grad* dst_m,
                                      gs_map_grad* dst_v, int32_t* counts_dev, void* stream) {
    if (!map_ok(map) || !grad_ok(src_m) || !grad_ok(src_v) || !accum || !denom || !samples ||
        !cfg_ok(cfg) || !scratch || n_out < 0 || !grad_ok(dst) || !grad_ok(dst_m) ||
        !grad_ok(dst_v) || !counts_dev)
        return GS_ERR_INVALID;
    if (n_out == 0) return GS_OK;
    const int nb = (map->n + kDensThreads - 1) / kDensThreads;
    const uint32_t* off = static_cast<const uint32_t*>(scratch) + 3 * (size_t)nb;
    DenseOut d;
    d.p = *dst;
    d.m = *dst_m;
    d.v = *dst_v;
    d.n_out = n_out;
    d.K = (map->sh_degree + 1) * (map->sh_degree + 1);
    k_densify_apply<<<nb, kDensThreads, 0, (cudaStream_t)stream>>>(
        *map, *src_m, *src_v, accum, denom, samples, *cfg, off, nb, d, counts_dev);
    return launch_status();
}
