// gs_render.cu -- A5 forward compositing and A7 pixel adjoint.
//
// Front-to-back alpha blending of each pixel's depth-ordered tile list
// (paper Sec. II; the original 3DGS tile rasteriser of Sec. III-B), and its
// adjoint walking each list back to front.
//
// GB300 design:
//  * one CTA per 2D tile of one view, one thread per pixel; all views of a
//    batch share the launch (the CTA looks its view up from the tile id);
//  * each CTA streams its tile's Gaussians through shared memory in batches
//    of `smem_batch` records gathered with cp.async, double-buffered so the
//    gather of batch k+1 (L2-resident records, random order) overlaps the
//    blending of batch k;
//  * every Gaussian is evaluated in tile-local coordinates: the projected mean
//    arrives as a float pair and is reduced once per staging to an offset from
//    the tile origin, so FP32 keeps ~1e-6 px where a global FP32 coordinate
//    would keep only ~6e-5 px at x = 1000;
//  * the forward and the backward evaluate alpha with the same explicitly
//    rounded operations, so both take the same skip decisions;
//  * the backward reduces each Gaussian's nine gradient components over the
//    warp with xor shuffles (skipping Gaussians no lane touches) and issues
//    them as nine parallel atomics from lanes 0..8.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_one() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

struct TileCtx {
    int view, tile_local, tx0, ty0, width, height, channels;
    int64_t pix_base, val_base;
    uint32_t begin, end;
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewTable& vt, const uint32_t* ranges,
                                            int tile) {
    TileCtx c;
    c.view = view_of_tile(vt, tile);
    const ViewGeom& g = vt.v[c.view];
    c.tile_local = tile - g.tile_offset;
    c.tx0 = (c.tile_local % g.tiles_x) * vt.tile_w;
    c.ty0 = (c.tile_local / g.tiles_x) * vt.tile_h;
    c.width = g.width;
    c.height = g.height;
    c.channels = g.channels;
    c.pix_base = g.pixel_offset;
    c.val_base = g.value_offset;
    c.begin = ranges[2 * tile];
    c.end = ranges[2 * tile + 1];
    return c;
}

// Gather records [first, first+cnt) of the tile list into stage (3 float4
// each) and their (view*n + index) ids into ids.
__device__ __forceinline__ void issue_batch(float4* stage, uint32_t* ids,
                                            const uint32_t* __restrict__ ivals,
                                            const float4* __restrict__ rec, uint32_t first,
                                            int cnt) {
    for (int c = threadIdx.x; c < 3 * cnt; c += blockDim.x) {
        const int j = c / 3, part = c - 3 * j;
        const uint32_t vg = __ldg(ivals + first + j);
        cp_async16(stage + 3 * j + part, rec + (size_t)vg * 3 + part);
        if (part == 0 && ids) ids[j] = vg;
    }
}

// Replace the mean pair of each staged record by its tile-local offset:
// stage[3j] = {lx, ly, a, b}; stage[3j+1] = {a, b, c, o}; stage[3j+2] =
// {r, g, b, gray}.
__device__ __forceinline__ void localise_batch(float4* stage, int cnt, float tx0, float ty0) {
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        float4 m = stage[3 * j];
        const float4 q = stage[3 * j + 1];
        float4 col = stage[3 * j + 2];
        m.x = __fadd_rn(__fsub_rn(m.x, tx0), m.z);
        m.y = __fadd_rn(__fsub_rn(m.y, ty0), m.w);
        m.z = q.x;
        m.w = q.y;
        stage[3 * j] = m;
        col.w = (col.x + col.y + col.z) * (1.0f / 3.0f);
        stage[3 * j + 2] = col;
    }
}

__device__ __forceinline__ float alpha_of(float o, float power) {
    return fminf(kAlphaMax, __fmul_rn(o, __expf(power)));
}

template <int CH>
__device__ __forceinline__ void blend_batch(const float4* stage, int cnt, uint32_t pos0, float lx,
                                            float ly, float& T, float* C, int32_t& last,
                                            bool& done) {
    for (int j = 0; j < cnt; ++j) {
        const float4 g = stage[3 * j];
        const float4 q = stage[3 * j + 1];
        const float power = gauss_power(g.z, g.w, q.z, g.x - lx, g.y - ly);
        if (power > 0.0f) continue;
        const float alpha = alpha_of(q.w, power);
        if (alpha < kAlphaMin) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
        if (Tn < kTMin) {
            done = true;
            break;
        }
        const float4 col = stage[3 * j + 2];
        const float wgt = alpha * T;
        if (CH == 3) {
            C[0] = fmaf(wgt, col.x, C[0]);
            C[1] = fmaf(wgt, col.y, C[1]);
            C[2] = fmaf(wgt, col.z, C[2]);
        } else {
            C[0] = fmaf(wgt, col.w, C[0]);
        }
        T = Tn;
        last = (int32_t)(pos0 + j + 1);
    }
}

__global__ void k_render_fwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                             int batch, float bg0, float bg1, float bg2,
                             float* __restrict__ images, float* __restrict__ final_T,
                             int32_t* __restrict__ last_idx) {
    extern __shared__ float4 smem[];
    const TileCtx tc = tile_ctx(vt, ranges, blockIdx.x);
    const int lxi = threadIdx.x & (vt.tile_w - 1);
    const int lyi = threadIdx.x >> vt.log2_tw;
    const int px = tc.tx0 + lxi, py = tc.ty0 + lyi;
    const bool inside = px < tc.width && py < tc.height;
    const float lx = (float)lxi, ly = (float)lyi;
    float T = 1.0f, C[3] = {0.f, 0.f, 0.f};
    int32_t last = 0;
    bool done = !inside;
    const int total = (int)(tc.end - tc.begin);
    const int nb = (total + batch - 1) / batch;
    if (nb > 0) {
        issue_batch(smem, nullptr, ivals, rec, tc.begin, min(batch, total));
        cp_async_commit();
    }
    for (int b = 0; b < nb; ++b) {
        const int cnt = min(batch, total - b * batch);
        float4* cur = smem + (b & 1) * 3 * batch;
        if (b + 1 < nb) {
            issue_batch(smem + ((b + 1) & 1) * 3 * batch, nullptr, ivals, rec,
                        tc.begin + (b + 1) * batch, min(batch, total - (b + 1) * batch));
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        localise_batch(cur, cnt, (float)tc.tx0, (float)tc.ty0);
        __syncthreads();
        if (!done) {
            if (tc.channels == 3)
                blend_batch<3>(cur, cnt, (uint32_t)(b * batch), lx, ly, T, C, last, done);
            else
                blend_batch<1>(cur, cnt, (uint32_t)(b * batch), lx, ly, T, C, last, done);
        }
        if (__syncthreads_count(done) == (int)blockDim.x) {
            cp_async_wait_all();  // nothing may still be landing in shared memory
            break;
        }
    }
    if (!inside) return;
    const int64_t pix = (int64_t)py * tc.width + px;
    const int64_t plane = (int64_t)tc.width * tc.height;
    if (tc.channels == 3) {
        images[tc.val_base + pix] = fmaf(T, bg0, C[0]);
        images[tc.val_base + plane + pix] = fmaf(T, bg1, C[1]);
        images[tc.val_base + 2 * plane + pix] = fmaf(T, bg2, C[2]);
    } else {
        images[tc.val_base + pix] = fmaf(T, (bg0 + bg1 + bg2) * (1.0f / 3.0f), C[0]);
    }
    final_T[tc.pix_base + pix] = T;
    last_idx[tc.pix_base + pix] = last;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int CH>
__device__ __forceinline__ void adjoint_batch(const float4* stage, const uint32_t* ids, int lo_rel,
                                              int hi_rel, uint32_t pos0, float lx, float ly,
                                              int32_t last, const float* g, float& T, float* S,
                                              float* __restrict__ grad2d) {
    const int lane = threadIdx.x & 31;
    for (int j = hi_rel - 1; j >= lo_rel; --j) {
        const uint32_t pos = pos0 + (uint32_t)j;
        float v[kGrad2d];
#pragma unroll
        for (int k = 0; k < kGrad2d; ++k) v[k] = 0.0f;
        bool contrib = false;
        if ((int32_t)pos < last) {
            const float4 gm = stage[3 * j];
            const float4 q = stage[3 * j + 1];
            const float dx = gm.x - lx, dy = gm.y - ly;
            const float power = gauss_power(gm.z, gm.w, q.z, dx, dy);
            if (power <= 0.0f) {
                const float G = __expf(power);
                const float oG = __fmul_rn(q.w, G);
                const float alpha = fminf(kAlphaMax, oG);
                if (alpha >= kAlphaMin) {
                    contrib = true;
                    const float4 col = stage[3 * j + 2];
                    const float one_m = __fsub_rn(1.0f, alpha);
                    const float inv = 1.0f / one_m;
                    const float Ti = T * inv;
                    const float w = alpha * Ti;
                    float dal;
                    if (CH == 3) {
                        dal = g[0] * (Ti * col.x - S[0] * inv) + g[1] * (Ti * col.y - S[1] * inv) +
                              g[2] * (Ti * col.z - S[2] * inv);
                        S[0] = fmaf(w, col.x, S[0]);
                        S[1] = fmaf(w, col.y, S[1]);
                        S[2] = fmaf(w, col.z, S[2]);
                        v[6] = w * g[0];
                        v[7] = w * g[1];
                        v[8] = w * g[2];
                    } else {
                        dal = g[0] * (Ti * col.w - S[0] * inv);
                        S[0] = fmaf(w, col.w, S[0]);
                        v[6] = w * g[0];
                    }
                    T = Ti;
                    if (oG < kAlphaMax) {
                        const float dpow = oG * dal;
                        v[0] = -dpow * (gm.z * dx + gm.w * dy);
                        v[1] = -dpow * (gm.w * dx + q.z * dy);
                        v[2] = -0.5f * dpow * dx * dx;
                        v[3] = -dpow * dx * dy;
                        v[4] = -0.5f * dpow * dy * dy;
                        v[5] = G * dal;
                    }
                }
            }
        }
        if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
            for (int k = 0; k < kGrad2d; ++k) v[k] = warp_sum(v[k]);
            float mine = 0.0f;
#pragma unroll
            for (int k = 0; k < kGrad2d; ++k) mine = (lane == k) ? v[k] : mine;
            const int nval = CH == 3 ? kGrad2d : 7;
            if (lane < nval) atomicAdd(grad2d + (size_t)ids[j] * kGrad2d + lane, mine);
        }
    }
}

__global__ void k_render_bwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                             int batch, float bg0, float bg1, float bg2,
                             const float* __restrict__ final_T, const int32_t* __restrict__ last_idx,
                             const float* __restrict__ dL, float* __restrict__ grad2d) {
    extern __shared__ float4 smem[];
    uint32_t* const ids0 = reinterpret_cast<uint32_t*>(smem + 6 * batch);
    __shared__ int s_maxlast;
    const TileCtx tc = tile_ctx(vt, ranges, blockIdx.x);
    const int lxi = threadIdx.x & (vt.tile_w - 1);
    const int lyi = threadIdx.x >> vt.log2_tw;
    const int px = tc.tx0 + lxi, py = tc.ty0 + lyi;
    const bool inside = px < tc.width && py < tc.height;
    const float lx = (float)lxi, ly = (float)lyi;
    const int64_t pix = (int64_t)py * tc.width + px;
    const int64_t plane = (int64_t)tc.width * tc.height;
    int32_t last = 0;
    float T = 1.0f, g[3] = {0.f, 0.f, 0.f}, S[3] = {0.f, 0.f, 0.f};
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (inside) {
        last = last_idx[tc.pix_base + pix];
        T = final_T[tc.pix_base + pix];
        if (tc.channels == 3) {
            g[0] = dL[tc.val_base + pix];
            g[1] = dL[tc.val_base + plane + pix];
            g[2] = dL[tc.val_base + 2 * plane + pix];
            S[0] = T * bg0;
            S[1] = T * bg1;
            S[2] = T * bg2;
        } else {
            g[0] = dL[tc.val_base + pix];
            S[0] = T * ((bg0 + bg1 + bg2) * (1.0f / 3.0f));
        }
        atomicMax(&s_maxlast, last);
    }
    __syncthreads();
    const int maxlast = s_maxlast;
    const int nb = (maxlast + batch - 1) / batch;
    // batch k covers list positions [max(0, maxlast - (k+1) batch), maxlast - k batch)
    auto bounds = [&](int k, int& lo, int& hi) {
        hi = maxlast - k * batch;
        lo = max(0, hi - batch);
    };
    if (nb > 0) {
        int lo, hi;
        bounds(0, lo, hi);
        issue_batch(smem, ids0, ivals, rec, tc.begin + lo, hi - lo);
        cp_async_commit();
    }
    for (int k = 0; k < nb; ++k) {
        int lo, hi;
        bounds(k, lo, hi);
        float4* cur = smem + (k & 1) * 3 * batch;
        uint32_t* cur_ids = ids0 + (k & 1) * batch;
        if (k + 1 < nb) {
            int lo2, hi2;
            bounds(k + 1, lo2, hi2);
            issue_batch(smem + ((k + 1) & 1) * 3 * batch, ids0 + ((k + 1) & 1) * batch, ivals, rec,
                        tc.begin + lo2, hi2 - lo2);
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        localise_batch(cur, hi - lo, (float)tc.tx0, (float)tc.ty0);
        __syncthreads();
        if (tc.channels == 3)
            adjoint_batch<3>(cur, cur_ids, 0, hi - lo, (uint32_t)lo, lx, ly, last, g, T, S, grad2d);
        else
            adjoint_batch<1>(cur, cur_ids, 0, hi - lo, (uint32_t)lo, lx, ly, last, g, T, S, grad2d);
        __syncthreads();
    }
}

}  // namespace

gs_status launch_project_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                             void* ws, const gs_map_grad* grads, int accumulate, cudaStream_t st);

gs_status launch_render_fwd(const Plan* p, const void* ws, float* images, float* final_T,
                            int32_t* last_idx, cudaStream_t st) {
    const int batch = p->cfg.smem_batch;
    const size_t smem = (size_t)2 * 3 * batch * sizeof(float4);
    const int threads = p->cfg.tile_w * p->cfg.tile_h;
    k_render_fwd<<<p->total_tiles, threads, smem, st>>>(
        p->vt, cbuf<uint32_t>(p, ws, GS_BUF_RANGES),
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES),
        cbuf<float4>(p, ws, GS_BUF_PROJ), batch, p->cfg.bg[0], p->cfg.bg[1], p->cfg.bg[2], images,
        final_T, last_idx);
    return launch_status();
}

gs_status launch_render_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                            void* ws, const float* final_T, const int32_t* last_idx,
                            const float* dL, const gs_map_grad* grads, int32_t accumulate,
                            cudaStream_t st) {
    const int batch = p->cfg.smem_batch;
    const size_t smem = (size_t)2 * 3 * batch * sizeof(float4) + 2 * batch * sizeof(uint32_t);
    const int threads = p->cfg.tile_w * p->cfg.tile_h;
    float* grad2d = buf<float>(p, ws, GS_BUF_GRAD2D);
    const size_t g2bytes = (size_t)p->vt.n_views * map->n * kGrad2d * sizeof(float);
    if (cudaMemsetAsync(grad2d, 0, g2bytes, st) != cudaSuccess) return GS_ERR_CUDA;
    k_render_bwd<<<p->total_tiles, threads, smem, st>>>(
        p->vt, cbuf<uint32_t>(p, ws, GS_BUF_RANGES),
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES),
        cbuf<float4>(p, ws, GS_BUF_PROJ), batch, p->cfg.bg[0], p->cfg.bg[1], p->cfg.bg[2],
        final_T, last_idx, dL, grad2d);
    gs_status s = launch_status();
    if (s != GS_OK) return s;
    return launch_project_bwd(p, map, views_dev, ws, grads, accumulate, st);
}

}  // namespace gs
