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
//  * register blocking: each thread owns 1-8 consecutive pixels of a tile
//    row, so every staged Gaussian is read from shared memory once per
//    thread, not once per pixel;
//  * the backward sums each Gaussian's nine gradient components over the
//    thread's pixels, then over the warp with a recursive-halving
//    reduce-scatter (16 shuffles, skipped when no lane touches the
//    Gaussian), and issues them as nine parallel atomics.
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

// The threads that render one tile: the whole CTA (one tile per CTA), or a
// single warp (one tile per warp, several tiles per CTA), whose barriers,
// votes and reductions then stay inside the warp.  Warp teams lift the limit
// of 32 resident CTAs per SM when a tile needs only 32 threads.
template <bool WARP>
struct Team {
    int tid, size;
    __device__ __forceinline__ Team() {
        tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
        size = WARP ? 32 : (int)blockDim.x;
    }
    __device__ __forceinline__ void sync() const {
        if (WARP) __syncwarp(); else __syncthreads();
    }
    // predicate vote that is also a barrier (shared memory ordered across it)
    __device__ __forceinline__ bool any(bool p) const {
        if (WARP) {
            __syncwarp();
            return __any_sync(0xffffffffu, p);
        }
        return __syncthreads_or(p) != 0;
    }
    // max over the team; scratch: one shared int (CTA teams only)
    __device__ __forceinline__ int max(int v, int* scratch) const {
        if (WARP) return (int)__reduce_max_sync(0xffffffffu, (unsigned)v);
        if (threadIdx.x == 0) *scratch = 0;
        __syncthreads();
        atomicMax(scratch, v);
        __syncthreads();
        return *scratch;
    }
};

// Gather records [first, first+cnt) of the tile list into stage (3 float4
// each) and their (view*n + index) ids into ids.
template <class TM>
__device__ __forceinline__ void issue_batch(const TM& tm, float4* stage, uint32_t* ids,
                                            const uint32_t* __restrict__ ivals,
                                            const float4* __restrict__ rec, uint32_t first,
                                            int cnt) {
    for (int c = tm.tid; c < 3 * cnt; c += tm.size) {
        const int j = c / 3, part = c - 3 * j;
        const uint32_t vg = __ldg(ivals + first + j);
        cp_async16(stage + 3 * j + part, rec + (size_t)vg * 3 + part);
        if (part == 0 && ids) ids[j] = vg;
    }
}

// Replace the mean pair of each staged record by its tile-local offset:
// stage[3j] = {lx, ly, a, b}; stage[3j+1] = {a, b, c, o}; stage[3j+2] =
// {r, g, b, gray}; and record in wmask[j] which warps of the CTA the Gaussian
// can reach.  Warp w owns tile rows [w*rows, (w+1)*rows).  A warp is left out
// only if its pixel strip misses the bounding box of the Gaussian's
// alpha >= 1/255 ellipse, {d : d^T Q d <= 2 ln(255 o)}, whose half-extents
// are sqrt(2 ln(255 o) (Q^-1)_xx) and sqrt(2 ln(255 o) (Q^-1)_yy); the box is
// grown by 0.1% + 0.01 px, far beyond FP32 rounding, so every skipped
// evaluation would have been skipped by the alpha test itself.
template <class TM>
__device__ __forceinline__ void localise_batch(const TM& tm, float4* stage, uint32_t* wmask,
                                               int cnt, float tx0, float ty0, int tile_w, int rows,
                                               int nwarps) {
    for (int j = tm.tid; j < cnt; j += tm.size) {
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
        const uint32_t all = nwarps >= 32 ? 0xffffffffu : ((1u << nwarps) - 1u);
        uint32_t bits = 0u;
        const float tau = logf(255.0f * q.w);
        const float detq = q.x * q.z - q.y * q.y;
        if (tau > 0.0f) {
            if (!(detq > 0.0f)) {
                bits = all;
            } else {
                const float ex = sqrtf(2.0f * tau * q.z / detq) * 1.001f + 0.01f;
                const float ey = sqrtf(2.0f * tau * q.x / detq) * 1.001f + 0.01f;
                if (!(ex == ex) || !(ey == ey)) {
                    bits = all;
                } else if (m.x + ex >= 0.0f && m.x - ex <= (float)(tile_w - 1)) {
                    for (int w = 0; w < nwarps; ++w) {
                        const float r0 = (float)(w * rows), r1 = (float)(w * rows + rows - 1);
                        if (m.y + ey >= r0 && m.y - ey <= r1) bits |= 1u << w;
                    }
                }
            }
        }
        wmask[j] = bits;
    }
}

__device__ __forceinline__ float alpha_of(float o, float power) {
    return fminf(kAlphaMax, __fmul_rn(o, __expf(power)));
}

// Pixels a thread owns: PPT consecutive pixels of one tile row, starting at
// tile-local (lx0, ly).
struct PixelRun {
    int lx0, ly;
};

__device__ __forceinline__ PixelRun pixel_run(int tid, int ppt, int log2_tw, int tile_w) {
    const int p0 = tid * ppt;
    PixelRun r;
    r.lx0 = p0 & (tile_w - 1);
    r.ly = p0 >> log2_tw;
    return r;
}

// Front-to-back blending of one staged batch for the PPT pixels of a thread.
// live: bit k set while pixel k still accumulates.
template <int CH, int PPT>
__device__ __forceinline__ void blend_batch(int tid, const float4* stage, const uint32_t* wmask,
                                            int cnt, uint32_t pos0, int lx0, float ly, float* T,
                                            float (*C)[CH], int32_t* last, unsigned& live) {
    const uint32_t wbit = 1u << (tid >> 5);
    for (int j = 0; j < cnt && live; ++j) {
        if (!(wmask[j] & wbit)) continue;
        const float4 g = stage[3 * j];
        const float4 q = stage[3 * j + 1];
        const float4 col = stage[3 * j + 2];
        const float dy = g.y - ly;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            // predicated rather than branched: the same decisions as the
            // backward, without divergent control flow inside the warp
            const float power = gauss_power(g.z, g.w, q.z, g.x - (float)(lx0 + k), dy);
            const float alpha = alpha_of(q.w, power);
            const float Tn = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
            const bool hit = ((live >> k) & 1u) && power <= 0.0f && alpha >= kAlphaMin;
            const bool stop = hit && Tn < kTMin;
            const bool add = hit && !stop;
            const float wgt = add ? alpha * T[k] : 0.0f;
            if (CH == 3) {
                C[k][0] = fmaf(wgt, col.x, C[k][0]);
                C[k][1] = fmaf(wgt, col.y, C[k][1]);
                C[k][2] = fmaf(wgt, col.z, C[k][2]);
            } else {
                C[k][0] = fmaf(wgt, col.w, C[k][0]);
            }
            T[k] = add ? Tn : T[k];
            last[k] = add ? (int32_t)(pos0 + j + 1) : last[k];
            live = stop ? (live & ~(1u << k)) : live;
        }
    }
}

template <int CH, int PPT, class TM>
__device__ void render_fwd_tile(const TM& tm, const ViewTable& vt, const TileCtx& tc,
                                const uint32_t* __restrict__ ivals,
                                const float4* __restrict__ rec, float4* smem, int batch,
                                const float* bg, float* __restrict__ images,
                                float* __restrict__ final_T, int32_t* __restrict__ last_idx) {
    uint32_t* const mask0 = reinterpret_cast<uint32_t*>(smem + 6 * batch);
    const int nwarps = tm.size >> 5;
    const int rows = (32 * PPT) >> vt.log2_tw;
    const PixelRun pr = pixel_run(tm.tid, PPT, vt.log2_tw, vt.tile_w);
    const int py = tc.ty0 + pr.ly;
    float T[PPT], C[PPT][CH];
    int32_t last[PPT];
    unsigned live = 0u;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.0f;
        last[k] = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) C[k][c] = 0.0f;
        if (tc.tx0 + pr.lx0 + k < tc.width && py < tc.height) live |= 1u << k;
    }
    const int total = (int)(tc.end - tc.begin);
    const int nb = (total + batch - 1) / batch;
    if (nb > 0) {
        issue_batch(tm, smem, nullptr, ivals, rec, tc.begin, min(batch, total));
        cp_async_commit();
    }
    for (int b = 0; b < nb; ++b) {
        const int cnt = min(batch, total - b * batch);
        float4* cur = smem + (b & 1) * 3 * batch;
        if (b + 1 < nb) {
            issue_batch(tm, smem + ((b + 1) & 1) * 3 * batch, nullptr, ivals, rec,
                        tc.begin + (b + 1) * batch, min(batch, total - (b + 1) * batch));
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        tm.sync();
        uint32_t* cmask = mask0 + (b & 1) * batch;
        localise_batch(tm, cur, cmask, cnt, (float)tc.tx0, (float)tc.ty0, vt.tile_w, rows, nwarps);
        tm.sync();
        blend_batch<CH, PPT>(tm.tid, cur, cmask, cnt, (uint32_t)(b * batch), pr.lx0,
                             (float)pr.ly, T, C, last, live);
        if (!tm.any(live != 0u)) {
            cp_async_wait_all();  // nothing may still be landing in shared memory
            break;
        }
    }
    if (py >= tc.height) return;
    const int64_t plane = (int64_t)tc.width * tc.height;
    const float bgg = (bg[0] + bg[1] + bg[2]) * (1.0f / 3.0f);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = tc.tx0 + pr.lx0 + k;
        if (px >= tc.width) continue;
        const int64_t pix = (int64_t)py * tc.width + px;
        if (CH == 3) {
#pragma unroll
            for (int c = 0; c < CH; ++c)
                images[tc.val_base + c * plane + pix] = fmaf(T[k], bg[c], C[k][c]);
        } else {
            images[tc.val_base + pix] = fmaf(T[k], bgg, C[k][0]);
        }
        final_T[tc.pix_base + pix] = T[k];
        last_idx[tc.pix_base + pix] = last[k];
    }
}

template <int PPT>
__global__ void k_render_fwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ order,
                             const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                             int batch, float bg0, float bg1, float bg2,
                             float* __restrict__ images, float* __restrict__ final_T,
                             int32_t* __restrict__ last_idx) {
    extern __shared__ float4 smem[];
    const TileCtx tc = tile_ctx(vt, ranges, (int)order[blockIdx.x]);
    const float bg[3] = {bg0, bg1, bg2};
    const Team<false> tm;
    if (tc.channels == 3)
        render_fwd_tile<3, PPT>(tm, vt, tc, ivals, rec, smem, batch, bg, images, final_T, last_idx);
    else
        render_fwd_tile<1, PPT>(tm, vt, tc, ivals, rec, smem, batch, bg, images, final_T, last_idx);
}

// One tile per warp, blockDim.x / 32 tiles per CTA, each warp with its own
// slice of shared memory (team_f4 float4 per warp).
constexpr int kMaxWarpTeams = 4;
constexpr size_t kSmemDefault = 48 * 1024;  // dynamic shared memory without opt-in

template <int PPT>
__global__ void k_render_fwd_w(ViewTable vt, const uint32_t* __restrict__ ranges,
                               const uint32_t* __restrict__ order,
                               const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                               int batch, int team_f4, int total_tiles, float bg0, float bg1,
                               float bg2, float* __restrict__ images, float* __restrict__ final_T,
                               int32_t* __restrict__ last_idx) {
    extern __shared__ float4 smem[];
    const int w = threadIdx.x >> 5;
    const int slot = blockIdx.x * (blockDim.x >> 5) + w;
    if (slot >= total_tiles) return;
    const TileCtx tc = tile_ctx(vt, ranges, (int)order[slot]);
    const float bg[3] = {bg0, bg1, bg2};
    const Team<true> tm;
    float4* mine = smem + (size_t)w * team_f4;
    if (tc.channels == 3)
        render_fwd_tile<3, PPT>(tm, vt, tc, ivals, rec, mine, batch, bg, images, final_T, last_idx);
    else
        render_fwd_tile<1, PPT>(tm, vt, tc, ivals, rec, mine, batch, bg, images, final_T, last_idx);
}

// Warp reduce-scatter of 16 values by recursive halving: afterwards lane L
// holds the warp total of value L >> 1 (16 shuffles instead of 5 per value).
__device__ __forceinline__ float warp_reduce16(float* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int CH, int PPT, class TM>
__device__ void render_bwd_tile(const TM& tm, const ViewTable& vt, const TileCtx& tc,
                                const uint32_t* __restrict__ ivals,
                                const float4* __restrict__ rec, float4* smem, int* s_maxlast,
                                int batch, const float* bg, const float* __restrict__ final_T,
                                const int32_t* __restrict__ last_idx,
                                const float* __restrict__ dL, float* __restrict__ grad2d) {
    // shared memory: stage[2][3*batch] float4 | ids[2][batch] | masks[2][batch] |
    //                acc[batch][9] float (the batch's per-Gaussian gradient sums)
    uint32_t* const ids0 = reinterpret_cast<uint32_t*>(smem + 6 * batch);
    uint32_t* const mask0 = ids0 + 2 * batch;
    float* const acc = reinterpret_cast<float*>(mask0 + 2 * batch);
    const int nwarps = tm.size >> 5;
    const int rows = (32 * PPT) >> vt.log2_tw;
    const uint32_t wbit = 1u << (tm.tid >> 5);
    const PixelRun pr = pixel_run(tm.tid, PPT, vt.log2_tw, vt.tile_w);
    const int py = tc.ty0 + pr.ly;
    const float ly = (float)pr.ly;
    const int64_t plane = (int64_t)tc.width * tc.height;
    const float bgg = (bg[0] + bg[1] + bg[2]) * (1.0f / 3.0f);
    float T[PPT], g[PPT][CH], S[PPT][CH];
    int32_t last[PPT];
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = tc.tx0 + pr.lx0 + k;
        last[k] = 0;
        T[k] = 1.0f;
#pragma unroll
        for (int c = 0; c < CH; ++c) g[k][c] = S[k][c] = 0.0f;
        if (px < tc.width && py < tc.height) {
            const int64_t pix = (int64_t)py * tc.width + px;
            last[k] = last_idx[tc.pix_base + pix];
            T[k] = final_T[tc.pix_base + pix];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                g[k][c] = dL[tc.val_base + c * plane + pix];
                S[k][c] = T[k] * (CH == 3 ? bg[c] : bgg);
            }
            mylast = max(mylast, last[k]);
        }
    }
    for (int i = tm.tid; i < kGrad2d * batch; i += tm.size) acc[i] = 0.0f;
    const int maxlast = tm.max(mylast, s_maxlast);
    const int nb = (maxlast + batch - 1) / batch;
    const int lane = threadIdx.x & 31;
    const int ncomp = CH == 3 ? kGrad2d : 7;
    // batch k covers list positions [max(0, maxlast - (k+1) batch), maxlast - k batch)
    if (nb > 0) {
        const int lo = max(0, maxlast - batch);
        issue_batch(tm, smem, ids0, ivals, rec, tc.begin + lo, maxlast - lo);
        cp_async_commit();
    }
    for (int kb = 0; kb < nb; ++kb) {
        const int hi = maxlast - kb * batch, lo = max(0, hi - batch);
        const int cnt = hi - lo;
        float4* cur = smem + (kb & 1) * 3 * batch;
        const uint32_t* cur_ids = ids0 + (kb & 1) * batch;
        uint32_t* cmask = mask0 + (kb & 1) * batch;
        if (kb + 1 < nb) {
            const int hi2 = lo, lo2 = max(0, hi2 - batch);
            issue_batch(tm, smem + ((kb + 1) & 1) * 3 * batch, ids0 + ((kb + 1) & 1) * batch,
                        ivals, rec, tc.begin + lo2, hi2 - lo2);
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        tm.sync();
        localise_batch(tm, cur, cmask, cnt, (float)tc.tx0, (float)tc.ty0, vt.tile_w, rows, nwarps);
        tm.sync();
        for (int j = cnt - 1; j >= 0; --j) {
            if (!(cmask[j] & wbit)) continue;
            const int32_t pos = lo + j;
            const float4 gm = cur[3 * j];
            const float4 q = cur[3 * j + 1];
            const float4 col = cur[3 * j + 2];
            const float dy = gm.y - ly;
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.0f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                // predicated: every lane runs the same instructions; a lane
                // whose pixel is not blended here contributes zeros and
                // keeps its state
                const float dx = gm.x - (float)(pr.lx0 + k);
                const float power = gauss_power(gm.z, gm.w, q.z, dx, dy);
                const float G = __expf(power);
                const float oG = __fmul_rn(q.w, G);
                const float alpha = fminf(kAlphaMax, oG);
                const bool hit = pos < last[k] && power <= 0.0f && alpha >= kAlphaMin;
                contrib |= hit;
                const float inv = __frcp_rn(__fsub_rn(1.0f, alpha));
                const float Ti = T[k] * inv;
                const float w = hit ? alpha * Ti : 0.0f;
                float dal;
                if (CH == 3) {
                    dal = g[k][0] * (Ti * col.x - S[k][0] * inv) +
                          g[k][1] * (Ti * col.y - S[k][1] * inv) +
                          g[k][2] * (Ti * col.z - S[k][2] * inv);
                    S[k][0] = fmaf(w, col.x, S[k][0]);
                    S[k][1] = fmaf(w, col.y, S[k][1]);
                    S[k][2] = fmaf(w, col.z, S[k][2]);
                    v[6] = fmaf(w, g[k][0], v[6]);
                    v[7] = fmaf(w, g[k][1], v[7]);
                    v[8] = fmaf(w, g[k][2], v[8]);
                } else {
                    dal = g[k][0] * (Ti * col.w - S[k][0] * inv);
                    S[k][0] = fmaf(w, col.w, S[k][0]);
                    v[6] = fmaf(w, g[k][0], v[6]);
                }
                T[k] = hit ? Ti : T[k];
                // alpha = o G when unclamped; a clamped alpha passes no gradient
                const bool free_a = hit && oG < kAlphaMax;
                const float dpow = free_a ? oG * dal : 0.0f;
                v[0] -= dpow * (gm.z * dx + gm.w * dy);
                v[1] -= dpow * (gm.w * dx + q.z * dy);
                v[2] -= 0.5f * dpow * dx * dx;
                v[3] -= dpow * dx * dy;
                v[4] -= 0.5f * dpow * dy * dy;
                v[5] = fmaf(free_a ? G : 0.0f, dal, v[5]);
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float tot = warp_reduce16(v);
                const int comp = lane >> 1;
                if ((lane & 1) == 0 && comp < ncomp) atomicAdd(acc + j * kGrad2d + comp, tot);
            }
        }
        tm.sync();
        // flush this batch's sums: one global atomic per (Gaussian, component, tile)
        for (int i = tm.tid; i < kGrad2d * cnt; i += tm.size) {
            const float a = acc[i];
            if (a != 0.0f) {
                const int j = i / kGrad2d;
                atomicAdd(grad2d + (size_t)cur_ids[j] * kGrad2d + (i - j * kGrad2d), a);
                acc[i] = 0.0f;
            }
        }
        tm.sync();
    }
}

template <int PPT>
__global__ void k_render_bwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ order,
                             const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                             int batch, float bg0, float bg1, float bg2,
                             const float* __restrict__ final_T, const int32_t* __restrict__ last_idx,
                             const float* __restrict__ dL, float* __restrict__ grad2d) {
    extern __shared__ float4 smem[];
    __shared__ int s_maxlast;
    const TileCtx tc = tile_ctx(vt, ranges, (int)order[blockIdx.x]);
    const float bg[3] = {bg0, bg1, bg2};
    const Team<false> tm;
    if (tc.channels == 3)
        render_bwd_tile<3, PPT>(tm, vt, tc, ivals, rec, smem, &s_maxlast, batch, bg, final_T,
                                last_idx, dL, grad2d);
    else
        render_bwd_tile<1, PPT>(tm, vt, tc, ivals, rec, smem, &s_maxlast, batch, bg, final_T,
                                last_idx, dL, grad2d);
}

template <int PPT>
__global__ void k_render_bwd_w(ViewTable vt, const uint32_t* __restrict__ ranges,
                               const uint32_t* __restrict__ order,
                               const uint32_t* __restrict__ ivals, const float4* __restrict__ rec,
                               int batch, int team_f4, int total_tiles, float bg0, float bg1,
                               float bg2, const float* __restrict__ final_T,
                               const int32_t* __restrict__ last_idx, const float* __restrict__ dL,
                               float* __restrict__ grad2d) {
    extern __shared__ float4 smem[];
    const int w = threadIdx.x >> 5;
    const int slot = blockIdx.x * (blockDim.x >> 5) + w;
    if (slot >= total_tiles) return;
    const TileCtx tc = tile_ctx(vt, ranges, (int)order[slot]);
    const float bg[3] = {bg0, bg1, bg2};
    const Team<true> tm;
    float4* mine = smem + (size_t)w * team_f4;
    if (tc.channels == 3)
        render_bwd_tile<3, PPT>(tm, vt, tc, ivals, rec, mine, nullptr, batch, bg, final_T,
                                last_idx, dL, grad2d);
    else
        render_bwd_tile<1, PPT>(tm, vt, tc, ivals, rec, mine, nullptr, batch, bg, final_T,
                                last_idx, dL, grad2d);
}

}  // namespace

template <typename K1, typename K2, typename K4, typename K8>
static K1 pick(int ppt, K1 a, K2 b, K4 c, K8 d) {
    return ppt == 1 ? a : ppt == 2 ? b : ppt == 4 ? c : d;
}

// Shared memory of one tile team, in float4 units: the double-buffered
// stage (6 float4 per Gaussian slot) and the 32-bit arrays (2 per slot in the
// forward: masks; 4 plus the nine gradient sums in the backward).
static int team_f4(int batch, bool bwd) {
    const size_t words = bwd ? (size_t)(4 + kGrad2d) * batch : (size_t)2 * batch;
    return 6 * batch + (int)((words * 4 + 15) / 16);
}

// Warp teams per CTA: as many as fit the default dynamic shared memory, at
// most kMaxWarpTeams (the largest batch still fits one).
static int warp_teams(int tf4) {
    const int t = (int)(kSmemDefault / ((size_t)tf4 * sizeof(float4)));
    return t < 1 ? 1 : (t > kMaxWarpTeams ? kMaxWarpTeams : t);
}

gs_status launch_render_fwd(const Plan* p, const void* ws, float* images, float* final_T,
                            int32_t* last_idx, cudaStream_t st) {
    const int batch = p->cfg.smem_batch;
    const int ppt = p->cfg.pixels_per_thread;
    const int threads = p->cfg.tile_w * p->cfg.tile_h / ppt;
    const int tf4 = team_f4(batch, false);
    const uint32_t* ranges = cbuf<uint32_t>(p, ws, GS_BUF_RANGES);
    const uint32_t* order = cbuf<uint32_t>(p, ws, B_TILE_ORDER);
    const uint32_t* vals =
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES);
    const float4* rec = cbuf<float4>(p, ws, GS_BUF_PROJ);
    if (threads == 32) {
        auto kern = pick(ppt, k_render_fwd_w<1>, k_render_fwd_w<2>, k_render_fwd_w<4>,
                         k_render_fwd_w<8>);
        const int teams = warp_teams(tf4);
        const int blocks = (p->total_tiles + teams - 1) / teams;
        kern<<<blocks, 32 * teams, (size_t)teams * tf4 * sizeof(float4), st>>>(
            p->vt, ranges, order, vals, rec, batch, tf4, p->total_tiles, p->cfg.bg[0],
            p->cfg.bg[1], p->cfg.bg[2], images, final_T, last_idx);
        return launch_status();
    }
    auto kern = pick(ppt, k_render_fwd<1>, k_render_fwd<2>, k_render_fwd<4>, k_render_fwd<8>);
    kern<<<p->total_tiles, threads, (size_t)tf4 * sizeof(float4), st>>>(
        p->vt, ranges, order, vals, rec, batch, p->cfg.bg[0], p->cfg.bg[1], p->cfg.bg[2], images,
        final_T, last_idx);
    return launch_status();
}

gs_status launch_render_bwd_pixels(const Plan* p, void* ws, const float* final_T,
                                   const int32_t* last_idx, const float* dL, cudaStream_t st) {
    const int batch = p->cfg.smem_batch_bwd;
    const int ppt = p->cfg.pixels_per_thread_bwd;
    const int threads = p->cfg.tile_w * p->cfg.tile_h / ppt;
    const int tf4 = team_f4(batch, true);
    float* grad2d = buf<float>(p, ws, GS_BUF_GRAD2D);
    if (cudaMemsetAsync(grad2d, 0, p->len[GS_BUF_GRAD2D], st) != cudaSuccess) return GS_ERR_CUDA;
    const uint32_t* ranges = cbuf<uint32_t>(p, ws, GS_BUF_RANGES);
    const uint32_t* order = cbuf<uint32_t>(p, ws, B_TILE_ORDER);
    const uint32_t* vals =
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES);
    const float4* rec = cbuf<float4>(p, ws, GS_BUF_PROJ);
    if (threads == 32) {
        auto kern = pick(ppt, k_render_bwd_w<1>, k_render_bwd_w<2>, k_render_bwd_w<4>,
                         k_render_bwd_w<8>);
        const int teams = warp_teams(tf4);
        const int blocks = (p->total_tiles + teams - 1) / teams;
        kern<<<blocks, 32 * teams, (size_t)teams * tf4 * sizeof(float4), st>>>(
            p->vt, ranges, order, vals, rec, batch, tf4, p->total_tiles, p->cfg.bg[0],
            p->cfg.bg[1], p->cfg.bg[2], final_T, last_idx, dL, grad2d);
        return launch_status();
    }
    auto kern = pick(ppt, k_render_bwd<1>, k_render_bwd<2>, k_render_bwd<4>, k_render_bwd<8>);
    kern<<<p->total_tiles, threads, (size_t)tf4 * sizeof(float4), st>>>(
        p->vt, ranges, order, vals, rec, batch, p->cfg.bg[0], p->cfg.bg[1], p->cfg.bg[2],
        final_T, last_idx, dL, grad2d);
    return launch_status();
}

gs_status launch_render_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                            void* ws, const float* final_T, const int32_t* last_idx,
                            const float* dL, const gs_map_grad* grads, int32_t accumulate,
                            cudaStream_t st) {
    gs_status s = launch_render_bwd_pixels(p, ws, final_T, last_idx, dL, st);
    if (s != GS_OK) return s;
    return launch_project_bwd(p, map, views_dev, ws, grads, accumulate, st);
}

}  // namespace gs
