// gs_render.cu -- A5 forward compositing and A7 pixel adjoint.
//
// Front-to-back alpha blending of each pixel's depth-ordered tile list
// (paper Sec. II; the original 3DGS tile rasteriser of Sec. III-B), and its
// adjoint walking each list back to front.
//
// GB300 design:
//  * one CTA per 2D tile of one view, or one warp per tile (several tiles
//    per CTA) when a tile needs 32 threads; all views of a batch share the
//    launch (each tile looks its view up from the tile id); tiles are taken
//    heavy-first, by the length of their lists;
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
//  * the backward sums, per Gaussian, the moments of dL/dpower and the
//    colour weights (nine values, from which the screen-space gradient is
//    linear) over the thread's pixels, then over the warp with a split
//    reduce-scatter (12 shuffles, skipped when no lane touches the
//    Gaussian), into shared memory; once per batch they become the gradient
//    and leave as nine parallel atomics per Gaussian.
#include <mutex>

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
    // the next tile slot from the launch's queue counter (q), taken by one
    // thread; scratch: one shared int (CTA teams only)
    __device__ __forceinline__ int next(uint32_t* q, int* scratch) const {
        if (WARP) {
            int s = 0;
            if (tid == 0) s = (int)atomicAdd(q, 1u);
            return __shfl_sync(0xffffffffu, s, 0);
        }
        __syncthreads();  // every thread has read the previous slot
        if (threadIdx.x == 0) *scratch = (int)atomicAdd(q, 1u);
        __syncthreads();
        return *scratch;
    }
    // shared-memory accumulation: plain in a warp team, whose lanes write
    // distinct addresses; atomic when several warps share the sums
    __device__ __forceinline__ void add(float* a, float v) const {
        if (WARP) *a += v; else atomicAdd(a, v);
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
// each) and the list values into ids: the (view*n + index) id, or, in a
// deterministic plan (gid_of given), the emission position, whose id is
// gid_of[position].  A thread takes whole records, kR at a time, and loads
// their list values (then their ids) before the first copy: the copies'
// addresses wait for one round trip per kR records, not one per record.
template <class TM>
__device__ __forceinline__ void issue_batch(const TM& tm, float4* stage, uint32_t* ids,
                                            const uint32_t* __restrict__ ivals,
                                            const uint32_t* __restrict__ gid_of,
                                            const float4* __restrict__ rec, uint32_t first,
                                            int cnt) {
    constexpr int kR = 2;
    for (int j0 = 0; j0 < cnt; j0 += kR * tm.size) {
        uint32_t x[kR], vg[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int j = j0 + tm.tid + r * tm.size;
            x[r] = j < cnt ? __ldg(ivals + first + j) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int j = j0 + tm.tid + r * tm.size;
            vg[r] = (gid_of && j < cnt) ? __ldg(gid_of + x[r]) : x[r];
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int j = j0 + tm.tid + r * tm.size;
            if (j < cnt) {
                const float4* src = rec + (size_t)vg[r] * 3;
                cp_async16(stage + 3 * j, src);
                cp_async16(stage + 3 * j + 1, src + 1);
                cp_async16(stage + 3 * j + 2, src + 2);
                if (ids) ids[j] = x[r];
            }
        }
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
// With masks false the warp masks are neither formed nor written: for a team
// of one warp over tight tile sets, whose listed Gaussians all reach the
// tile's ellipse box up to the margins, the mask would leave the warp out of
// almost nothing.  Culling is only a shortcut: without it every listed
// Gaussian is evaluated and the alpha test decides.
template <class TM>
__device__ __forceinline__ void localise_batch(const TM& tm, float4* stage, uint32_t* wmask,
                                               int cnt, float tx0, float ty0, int tile_w, int rows,
                                               int nwarps, bool masks = true) {
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
        if (!masks) continue;
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

// The Gaussians j0 .. j0 + 31 of a batch of cnt that a warp evaluates, as a
// warp-uniform bitmask: all that exist, or with cull those whose warp mask
// names the warp (bit wbit).  The blend loops walk its set bits, so a
// Gaussian culled for the warp costs nothing.
__device__ __forceinline__ unsigned chunk_todo(int j0, int cnt, const uint32_t* wmask,
                                               uint32_t wbit, bool cull) {
    const int n = cnt - j0;
    if (!cull) return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    const int j = j0 + (int)(threadIdx.x & 31);
    return __ballot_sync(0xffffffffu, j < cnt && (wmask[j] & wbit) != 0u);
}

// Front-to-back blending of one staged batch for the PPT pixels of a thread.
// live: bit k set while pixel k still accumulates.  The loop is warp-uniform
// (a lane whose pixels are done runs predicated) so the warp can vote: a
// Gaussian that no pixel of the warp blends costs only its alpha evaluation,
// and the warp leaves the batch once none of its pixels is live.  That test
// runs only where no pixel blended the Gaussian: a pixel that is done
// blends nothing, so once all are done the next Gaussian lands there, and a
// blended Gaussian carries no second vote.
//
// With an even PPT the pixels go in pairs on packed FP32 pair operations,
// each half the scalar operation of the odd-PPT path on the same operands;
// -alpha, -o G and the colour (C holds -C) are kept negated so that no pair
// needs a sign flip: the decisions, T and the image are the same bits.
// nlx: the negated tile-local x of the pixel pairs; cull: test the warp masks.
template <int CH, int PPT>
__device__ __forceinline__ void blend_batch(int tid, const float4* stage, const uint32_t* wmask,
                                            int cnt, uint32_t pos0, int lx0, float ly, float* T,
                                            float (*C)[CH], int32_t* last, unsigned& live,
                                            const float2* nlx, bool cull) {
    const uint32_t wbit = 1u << (tid >> 5);
    if (!__any_sync(0xffffffffu, live != 0u)) return;
    if constexpr (PPT % 2 == 0) {
        constexpr int NP = PPT / 2;
        for (int j0 = 0; j0 < cnt; j0 += 32) {
            unsigned todo = chunk_todo(j0, cnt, wmask, wbit, cull);
            while (todo != 0u) {
                const int j = j0 + __ffs(todo) - 1;
                todo &= todo - 1u;
                const float4 g = stage[3 * j];
                const float4 q = stage[3 * j + 1];
                const float dy = g.y - ly;
                const float cdd = __fmul_rn(q.z, __fmul_rn(dy, dy));
                const float2 gx2 = make_float2(g.x, g.x), a2 = make_float2(g.z, g.z);
                const float2 cdd2 = make_float2(cdd, cdd), dy2 = make_float2(dy, dy);
                const float2 nb2 = make_float2(-g.w, -g.w), no2 = make_float2(-q.w, -q.w);
                float2 na[NP];
                unsigned hits = 0u;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float2 dx = add2(gx2, nlx[p]);
                    const float2 qq = fma2(a2, mul2(dx, dx), cdd2);
                    const float2 pw = fma2(make_float2(-0.5f, -0.5f), qq, mul2(nb2, mul2(dx, dy2)));
                    const float2 noG = mul2(no2, make_float2(__expf(pw.x), __expf(pw.y)));
                    na[p] = make_float2(fmaxf(-kAlphaMax, noG.x), fmaxf(-kAlphaMax, noG.y));
                    if (((live >> (2 * p)) & 1u) && pw.x <= 0.0f && na[p].x <= -kAlphaMin)
                        hits |= 1u << (2 * p);
                    if (((live >> (2 * p + 1)) & 1u) && pw.y <= 0.0f && na[p].y <= -kAlphaMin)
                        hits |= 1u << (2 * p + 1);
                }
                if (!__any_sync(0xffffffffu, hits != 0u)) {
                    if (!__any_sync(0xffffffffu, live != 0u)) return;
                    continue;
                }
                const float4 col = stage[3 * j + 2];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int k0 = 2 * p, k1 = 2 * p + 1;
                    const bool h0 = (hits >> k0) & 1u, h1 = (hits >> k1) & 1u;
                    const float2 T2 = make_float2(T[k0], T[k1]);
                    const float2 Tn = mul2(T2, add2(make_float2(1.0f, 1.0f), na[p]));
                    const bool s0 = h0 && Tn.x < kTMin, s1 = h1 && Tn.y < kTMin;
                    const bool a0 = h0 && !s0, a1 = h1 && !s1;
                    const float2 nwr = mul2(na[p], T2);
                    const float2 nw = make_float2(a0 ? nwr.x : 0.0f, a1 ? nwr.y : 0.0f);
                    if (CH == 3) {
                        const float2 c0 = fma2(nw, make_float2(col.x, col.x),
                                               make_float2(C[k0][0], C[k1][0]));
                        const float2 c1 = fma2(nw, make_float2(col.y, col.y),
                                               make_float2(C[k0][1], C[k1][1]));
                        const float2 c2 = fma2(nw, make_float2(col.z, col.z),
                                               make_float2(C[k0][2], C[k1][2]));
                        C[k0][0] = c0.x;
                        C[k1][0] = c0.y;
                        C[k0][1] = c1.x;
                        C[k1][1] = c1.y;
                        C[k0][2] = c2.x;
                        C[k1][2] = c2.y;
                    } else {
                        const float2 c0 = fma2(nw, make_float2(col.w, col.w),
                                               make_float2(C[k0][0], C[k1][0]));
                        C[k0][0] = c0.x;
                        C[k1][0] = c0.y;
                    }
                    T[k0] = a0 ? Tn.x : T[k0];
                    T[k1] = a1 ? Tn.y : T[k1];
                    last[k0] = a0 ? (int32_t)(pos0 + j + 1) : last[k0];
                    last[k1] = a1 ? (int32_t)(pos0 + j + 1) : last[k1];
                    live = s0 ? (live & ~(1u << k0)) : live;
                    live = s1 ? (live & ~(1u << k1)) : live;
                }
            }
        }
        return;
    }
    // the batch index of each pixel's last blended Gaussian (-1: none yet),
    // turned into the list position when the batch is left
    int lj[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) lj[k] = -1;
    for (int j0 = 0; j0 < cnt; j0 += 32) {
        unsigned todo = chunk_todo(j0, cnt, wmask, wbit, cull);
        while (todo != 0u) {
            const int j = j0 + __ffs(todo) - 1;
            todo &= todo - 1u;
            const float4 g = stage[3 * j];
            const float4 q = stage[3 * j + 1];
            const float dy = g.y - ly;
            float al[PPT];
            unsigned hits = 0u;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                // the same decisions as the backward, from the same rounded ops
                const float power = gauss_power(g.z, g.w, q.z, g.x - (float)(lx0 + k), dy);
                al[k] = alpha_of(q.w, power);
                if (((live >> k) & 1u) && power <= 0.0f && al[k] >= kAlphaMin) hits |= 1u << k;
            }
            if (!__any_sync(0xffffffffu, hits != 0u)) {
                if (!__any_sync(0xffffffffu, live != 0u)) goto done;
                continue;
            }
            const float4 col = stage[3 * j + 2];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const bool hit = (hits >> k) & 1u;
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.0f, al[k]));
                const bool stop = hit && Tn < kTMin;
                const bool add = hit && !stop;
                const float wgt = add ? al[k] * T[k] : 0.0f;
                if (CH == 3) {
                    C[k][0] = fmaf(wgt, col.x, C[k][0]);
                    C[k][1] = fmaf(wgt, col.y, C[k][1]);
                    C[k][2] = fmaf(wgt, col.z, C[k][2]);
                } else {
                    C[k][0] = fmaf(wgt, col.w, C[k][0]);
                }
                T[k] = add ? Tn : T[k];
                lj[k] = add ? j : lj[k];
                live = stop ? (live & ~(1u << k)) : live;
            }
        }
    }
done:
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        if (lj[k] >= 0) last[k] = (int32_t)(pos0 + (uint32_t)lj[k] + 1u);
}

template <int CH, int PPT, class TM>
__device__ void render_fwd_tile(const TM& tm, const ViewTable& vt, const TileCtx& tc,
                                const uint32_t* __restrict__ ivals,
                                const uint32_t* __restrict__ gid_of,
                                const float4* __restrict__ rec, float4* smem, int batch,
                                const float* bg, float* __restrict__ images,
                                float* __restrict__ final_T, int32_t* __restrict__ last_idx) {
    uint32_t* const mask0 = reinterpret_cast<uint32_t*>(smem + 6 * batch);
    const int nwarps = tm.size >> 5;
    const int rows = (32 * PPT) >> vt.log2_tw;
    const PixelRun pr = pixel_run(tm.tid, PPT, vt.log2_tw, vt.tile_w);
    const int py = tc.ty0 + pr.ly;
    // per-warp culling only where a warp covers part of the tile or the
    // tile lists are the square rects
    const bool cull = nwarps > 1 || !vt.tight_rect;
    // the negated tile-local x of the thread's pixels, in pairs (even PPT)
    float2 nlx[PPT / 2 > 0 ? PPT / 2 : 1];
#pragma unroll
    for (int p = 0; p < PPT / 2; ++p)
        nlx[p] = make_float2(-(float)(pr.lx0 + 2 * p), -(float)(pr.lx0 + 2 * p + 1));
    // C holds the accumulated colour, negated with an even PPT
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
        issue_batch(tm, smem, nullptr, ivals, gid_of, rec, tc.begin, min(batch, total));
        cp_async_commit();
    }
    for (int b = 0; b < nb; ++b) {
        const int cnt = min(batch, total - b * batch);
        float4* cur = smem + (b & 1) * 3 * batch;
        if (b + 1 < nb) {
            issue_batch(tm, smem + ((b + 1) & 1) * 3 * batch, nullptr, ivals, gid_of, rec,
                        tc.begin + (b + 1) * batch, min(batch, total - (b + 1) * batch));
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        tm.sync();
        uint32_t* cmask = mask0 + (b & 1) * batch;
        localise_batch(tm, cur, cmask, cnt, (float)tc.tx0, (float)tc.ty0, vt.tile_w, rows, nwarps,
                       cull);
        tm.sync();
        blend_batch<CH, PPT>(tm.tid, cur, cmask, cnt, (uint32_t)(b * batch), pr.lx0,
                             (float)pr.ly, T, C, last, live, nlx, cull);
        if (!tm.any(live != 0u)) {
            cp_async_wait_all();  // nothing may still be landing in shared memory
            break;
        }
    }
    if (py >= tc.height) return;
    const int64_t plane = (int64_t)tc.width * tc.height;
    const float bgg = (bg[0] + bg[1] + bg[2]) * (1.0f / 3.0f);
    constexpr float sC = PPT % 2 == 0 ? -1.0f : 1.0f;  // undo the negation (exact)
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = tc.tx0 + pr.lx0 + k;
        if (px >= tc.width) continue;
        const int64_t pix = (int64_t)py * tc.width + px;
        if (CH == 3) {
#pragma unroll
            for (int c = 0; c < CH; ++c)
                images[tc.val_base + c * plane + pix] = fmaf(T[k], bg[c], sC * C[k][c]);
        } else {
            images[tc.val_base + pix] = fmaf(T[k], bgg, sC * C[k][0]);
        }
        final_T[tc.pix_base + pix] = T[k];
        last_idx[tc.pix_base + pix] = last[k];
    }
}

// Persistent render kernels: each team (the CTA, or one warp of it) takes
// the next slot of the heavy-first tile order from a queue counter until the
// order is exhausted, so a team that drew a short list moves on at once
// (longest-first list scheduling).  A warp team owns team_f4 float4 of the
// CTA's dynamic shared memory.
template <int PPT, bool WARP>
__global__ void k_render_fwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ order,
                             const uint32_t* __restrict__ ivals,
                             const uint32_t* __restrict__ gid_of, const float4* __restrict__ rec,
                             int batch, int team_f4, int total_tiles, uint32_t* queue, float bg0,
                             float bg1, float bg2, float* __restrict__ images,
                             float* __restrict__ final_T, int32_t* __restrict__ last_idx) {
    extern __shared__ float4 smem[];
    __shared__ int s_slot;
    const Team<WARP> tm;
    float4* mine = smem + (WARP ? (size_t)(threadIdx.x >> 5) * team_f4 : 0);
    const float bg[3] = {bg0, bg1, bg2};
    for (;;) {
        const int slot = tm.next(queue, &s_slot);
        if (slot >= total_tiles) break;
        const TileCtx tc = tile_ctx(vt, ranges, (int)order[slot]);
        if (tc.channels == 3)
            render_fwd_tile<3, PPT>(tm, vt, tc, ivals, gid_of, rec, mine, batch, bg, images,
                                    final_T, last_idx);
        else
            render_fwd_tile<1, PPT>(tm, vt, tc, ivals, gid_of, rec, mine, batch, bg, images,
                                    final_T, last_idx);
    }
}

constexpr int kMaxWarpTeams = 4;
constexpr size_t kSmemDefault = 48 * 1024;  // dynamic shared memory without opt-in

// Warp reduce-scatter of N values (N = 9 or 7).  At the levels with lane
// offsets 16, 8, 4, 2 a lane holding S partial sums keeps the first
// ceil(S/2) (offset bit clear) or the rest (bit set, padded with a zero) and
// sends the other part to its partner; once one sum is left the remaining
// levels add it across lanes.  N = 9 takes 12 shuffles (a 16-wide
// reduce-scatter takes 16).  Returns the warp total of the component that
// reduce_component(lane) names.
template <int N, int O = 16>
__device__ __forceinline__ float warp_reduce_split(float* v) {
    constexpr int K = (N + 1) / 2;
    if (N == 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
    } else {
        const bool up = (threadIdx.x & O) != 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float lo = v[i];
            const float hi = i + K < N ? v[i + K] : 0.0f;
            v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, O);
        }
    }
    if constexpr (O > 1) return warp_reduce_split<(N == 1 ? 1 : K), O / 2>(v);
    return v[0];
}

// The component whose total warp_reduce_split<N> leaves in this lane, or -1
// when the lane holds padding or a copy that another lane reports.
template <int N>
__device__ __forceinline__ int reduce_component(int lane) {
    int sizes[5];
    for (int L = 0, s = N; L < 5; ++L, s = (s + 1) / 2) sizes[L] = s;
    int idx = 0;
    for (int L = 4; L >= 0; --L) {
        const int S = sizes[L], O = 16 >> L;
        if (S == 1) {
            if (lane & O) return -1;
            continue;
        }
        if (lane & O) idx += (S + 1) / 2;
        if (idx >= S) return -1;
    }
    return idx;
}

// Reciprocal by the hardware approximation (PTX rcp.approx.ftz.f32, within
// about one ulp); the argument 1 - alpha lies in [0.01, 1].
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The pixel adjoint's per-Gaussian work for a lane holding an even number of
// pixels, in pairs on packed FP32 pair operations: each half is the scalar
// operation of the one-pixel path in render_bwd_tile on the same operands,
// with the state kept negated (-gS; -alpha and -o G for the decisions; the
// sums negated) so that no pair needs a sign flip.  The decisions and the
// per-pixel T and gS are the same bits as the one-pixel path's.
template <int PPT>
struct PairEval {
    float2 dx[PPT / 2], noG[PPT / 2], na[PPT / 2];
    bool hk[PPT];
};

// Phase 1: alpha and the blend decision of every pixel of the lane; returns
// whether the lane blends the Gaussian at any of its pixels.
template <int PPT>
__device__ __forceinline__ bool pair_phase1(const float4& gm, const float4& q, float dy, int pos,
                                            const int32_t* last, const float2* nlx,
                                            PairEval<PPT>& e) {
    constexpr int NP = PPT / 2;
    const float cdd = __fmul_rn(q.z, __fmul_rn(dy, dy));
    const float2 gx2 = make_float2(gm.x, gm.x), a2 = make_float2(gm.z, gm.z);
    const float2 cdd2 = make_float2(cdd, cdd), dy2 = make_float2(dy, dy);
    const float2 nb2 = make_float2(-gm.w, -gm.w), no2 = make_float2(-q.w, -q.w);
    bool contrib = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        e.dx[p] = add2(gx2, nlx[p]);
        const float2 qq = fma2(a2, mul2(e.dx[p], e.dx[p]), cdd2);
        const float2 pw = fma2(make_float2(-0.5f, -0.5f), qq, mul2(nb2, mul2(e.dx[p], dy2)));
        e.noG[p] = mul2(no2, make_float2(__expf(pw.x), __expf(pw.y)));
        e.na[p] = make_float2(fmaxf(-kAlphaMax, e.noG[p].x), fmaxf(-kAlphaMax, e.noG[p].y));
        e.hk[2 * p] = pos < last[2 * p] && pw.x <= 0.0f && e.na[p].x <= -kAlphaMin;
        e.hk[2 * p + 1] = pos < last[2 * p + 1] && pw.y <= 0.0f && e.na[p].y <= -kAlphaMin;
        contrib |= e.hk[2 * p] | e.hk[2 * p + 1];
    }
    return contrib;
}

// Phase 2, predicated (a pixel not blended here contributes zeros and keeps
// its state): updates T and gS and writes the lane's NC values of the
// Gaussian (moments, colour weights, and with ABS the two magnitude sums).
template <int CH, int PPT, bool ABS>
__device__ __forceinline__ void pair_phase2(const PairEval<PPT>& e, const float4& gm,
                                            const float4& q, const float4& col, float dy,
                                            float* T, float (*g)[CH], float* gS, float* v) {
    constexpr int NP = PPT / 2;
    constexpr int NC0 = CH == 3 ? kGrad2d : 7;
    float2 nP0 = make_float2(0.f, 0.f), nP1 = nP0, nP3 = nP0, ncw[CH];
    float Hx = 0.0f, Hy = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; ++c) ncw[c] = nP0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int k0 = 2 * p, k1 = 2 * p + 1;
        const float2 inv = make_float2(rcp_approx(1.0f + e.na[p].x), rcp_approx(1.0f + e.na[p].y));
        const float2 Ti = mul2(make_float2(T[k0], T[k1]), inv);
        const float2 nwr = mul2(e.na[p], Ti);
        const float2 nw = make_float2(e.hk[k0] ? nwr.x : 0.0f, e.hk[k1] ? nwr.y : 0.0f);
        float2 gc;
        if (CH == 3)
            gc = fma2(make_float2(g[k0][2], g[k1][2]), make_float2(col.z, col.z),
                      fma2(make_float2(g[k0][1], g[k1][1]), make_float2(col.y, col.y),
                           mul2(make_float2(g[k0][0], g[k1][0]), make_float2(col.x, col.x))));
        else
            gc = mul2(make_float2(g[k0][0], g[k1][0]), make_float2(col.w, col.w));
        const float2 nS = make_float2(gS[k0], gS[k1]);
        const float2 dal = fma2(Ti, gc, mul2(inv, nS));
        const float2 nS1 = fma2(nw, gc, nS);
        gS[k0] = nS1.x;
        gS[k1] = nS1.y;
#pragma unroll
        for (int c = 0; c < CH; ++c) ncw[c] = fma2(nw, make_float2(g[k0][c], g[k1][c]), ncw[c]);
        T[k0] = e.hk[k0] ? Ti.x : T[k0];
        T[k1] = e.hk[k1] ? Ti.y : T[k1];
        // alpha = o G when unclamped; a clamped alpha passes no gradient
        const float2 ndr = mul2(e.noG[p], dal);
        const float2 ndp = make_float2((e.hk[k0] && e.noG[p].x > -kAlphaMax) ? ndr.x : 0.0f,
                                       (e.hk[k1] && e.noG[p].y > -kAlphaMax) ? ndr.y : 0.0f);
        const float2 nt = mul2(ndp, e.dx[p]);
        nP0 = add2(nP0, ndp);
        nP1 = add2(nP1, nt);
        nP3 = fma2(nt, e.dx[p], nP3);
        if (ABS) {
            // each pixel's own contribution to dL/dmean2d, by magnitude
            Hx += fabsf(ndp.x * fmaf(gm.z, e.dx[p].x, gm.w * dy));
            Hx += fabsf(ndp.y * fmaf(gm.z, e.dx[p].y, gm.w * dy));
            Hy += fabsf(ndp.x * fmaf(gm.w, e.dx[p].x, q.z * dy));
            Hy += fabsf(ndp.y * fmaf(gm.w, e.dx[p].y, q.z * dy));
        }
    }
    // the pixels of a run share dy: A2 = dy A0, A4 = dy A1, A5 = dy A2
    const float P0 = -(nP0.x + nP0.y), P1 = -(nP1.x + nP1.y);
    v[0] = P0;
    v[1] = P1;
    v[2] = dy * P0;
    v[3] = -(nP3.x + nP3.y);
    v[4] = dy * P1;
    v[5] = dy * v[2];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[6 + c] = -(ncw[c].x + ncw[c].y);
    if (ABS) {
        v[NC0] = Hx;
        v[NC0 + 1] = Hy;
    }
}

// Back-to-front adjoint of one tile (Eq. 1 differentiated; the transmittance
// before each Gaussian is recovered by dividing by 1 - alpha).  Per pixel the
// colour accumulated behind the current Gaussian enters only through its dot
// product with dL/dC, so one scalar gS = dL/dC . S is carried instead of S.
// Per Gaussian the lanes sum the moments of dL/dpower,
//   A0 = sum dp, A1 = sum dp dx, A2 = sum dp dy, A3 = sum dp dx^2,
//   A4 = sum dp dx dy, A5 = sum dp dy^2   (dx, dy = mean - pixel),
// and the colour weights; with power = -(a dx^2 + c dy^2)/2 - b dx dy the
// screen-space gradient is linear in them:
//   dL/dmean = -(a A1 + b A2, b A1 + c A2), dL/d(a, b, c) = (-A3/2, -A4, -A5/2),
//   dL/do = A0 / o   (dp = o G dL/dalpha wherever alpha = o G is unclamped),
// which is applied once per Gaussian and batch, before the global atomics.
template <int CH, int PPT, class TM, bool ABS>
__device__ void render_bwd_tile(const TM& tm, const ViewTable& vt, const TileCtx& tc,
                                const uint32_t* __restrict__ ivals,
                                const uint32_t* __restrict__ gid_of,
                                const float4* __restrict__ rec, float4* smem, int* s_maxlast,
                                int batch, const float* bg, const float* __restrict__ final_T,
                                const int32_t* __restrict__ last_idx,
                                const float* __restrict__ dL, float* __restrict__ grad2d,
                                float* __restrict__ absgrad, float* __restrict__ partial) {
    // shared memory: stage[2][3*batch] float4 | ids[2][batch] | masks[2][batch] |
    //                acc[batch][KA] float (the batch's per-Gaussian sums: 9, and
    //                with ABS the two homodirectional sums in slots 9, 10)
    constexpr int NC0 = CH == 3 ? kGrad2d : 7;  // moments + colour components
    constexpr int NC = NC0 + (ABS ? 2 : 0);      // values reduced per Gaussian
    constexpr int KA = kGrad2d + (ABS ? 2 : 0);  // shared slots per Gaussian
    uint32_t* const ids0 = reinterpret_cast<uint32_t*>(smem + 6 * batch);
    uint32_t* const mask0 = ids0 + 2 * batch;
    float* const acc = reinterpret_cast<float*>(mask0 + 2 * batch);
    const int nwarps = tm.size >> 5;
    const int rows = (32 * PPT) >> vt.log2_tw;
    const uint32_t wbit = 1u << (tm.tid >> 5);
    // per-warp culling only where a warp covers part of the tile or the
    // tile lists are the square rects
    const bool cull = nwarps > 1 || !vt.tight_rect;
    const PixelRun pr = pixel_run(tm.tid, PPT, vt.log2_tw, vt.tile_w);
    const int py = tc.ty0 + pr.ly;
    const float ly = (float)pr.ly;
    const int64_t plane = (int64_t)tc.width * tc.height;
    const float bgg = (bg[0] + bg[1] + bg[2]) * (1.0f / 3.0f);
    // gS holds -dL/dC . S (the colour behind the current Gaussian), negated
    float T[PPT], g[PPT][CH], gS[PPT];
    int32_t last[PPT];
    int mylast = 0;
    // the negated tile-local x of the lane's pixels, in pairs
    float2 nlx[PPT / 2 > 0 ? PPT / 2 : 1];
#pragma unroll
    for (int p = 0; p < PPT / 2; ++p)
        nlx[p] = make_float2(-(float)(pr.lx0 + 2 * p), -(float)(pr.lx0 + 2 * p + 1));
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = tc.tx0 + pr.lx0 + k;
        last[k] = 0;
        T[k] = 1.0f;
        gS[k] = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; ++c) g[k][c] = 0.0f;
        if (px < tc.width && py < tc.height) {
            const int64_t pix = (int64_t)py * tc.width + px;
            last[k] = last_idx[tc.pix_base + pix];
            T[k] = final_T[tc.pix_base + pix];
            float gb = 0.0f;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                g[k][c] = dL[tc.val_base + c * plane + pix];
                gb = fmaf(g[k][c], CH == 3 ? bg[c] : bgg, gb);
            }
            gS[k] = T[k] * -gb;  // minus the background seen through T_final
            mylast = max(mylast, last[k]);
        }
    }
    for (int i = tm.tid; i < KA * batch; i += tm.size) acc[i] = 0.0f;
    const int maxlast = tm.max(mylast, s_maxlast);
    const int nb = (maxlast + batch - 1) / batch;
    const int comp_r = reduce_component<NC>(threadIdx.x & 31);
    // the shared slot of the reduced value this lane holds
    const int comp = comp_r < NC0 ? comp_r : (comp_r < 0 ? -1 : kGrad2d + comp_r - NC0);
    // ... and of the joint reduction of two Gaussians' 2 NC values: the slot,
    // and whether it belongs to the second (front) Gaussian
    const int comp2_r = reduce_component<2 * NC>(threadIdx.x & 31);
    const int comp2_b = comp2_r >= NC ? 1 : 0;
    const int comp2_c = comp2_r - NC * comp2_b;
    const int comp2 =
        comp2_r < 0 ? -1 : (comp2_c < NC0 ? comp2_c : kGrad2d + comp2_c - NC0);
    // batch k covers list positions [max(0, maxlast - (k+1) batch), maxlast - k batch)
    if (nb > 0) {
        const int lo = max(0, maxlast - batch);
        issue_batch(tm, smem, ids0, ivals, gid_of, rec, tc.begin + lo, maxlast - lo);
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
                        ivals, gid_of, rec, tc.begin + lo2, hi2 - lo2);
            cp_async_commit();
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        tm.sync();
        localise_batch(tm, cur, cmask, cnt, (float)tc.tx0, (float)tc.ty0, vt.tile_w, rows, nwarps,
                       cull);
        tm.sync();
        if constexpr (PPT % 2 == 0) {
            // one Gaussian, its values reduced alone
            auto one = [&](int j) {
                const float4 gm = cur[3 * j], q = cur[3 * j + 1];
                const float dy = gm.y - ly;
                PairEval<PPT> e;
                if (!__any_sync(0xffffffffu, pair_phase1<PPT>(gm, q, dy, lo + j, last, nlx, e)))
                    return;
                float v[NC];
                pair_phase2<CH, PPT, ABS>(e, gm, q, cur[3 * j + 2], dy, T, g, gS, v);
                const float tot = warp_reduce_split<NC>(v);
                if (comp >= 0) tm.add(acc + j * KA + comp, tot);
            };
            if (cull) {
                for (int j = cnt - 1; j >= 0; --j)
                    if (cmask[j] & wbit) one(j);
            } else {
                // two Gaussians per step, j (behind) then j - 1, whose values
                // are reduced together when the warp blends both: one split
                // reduce-scatter of 2 NC values costs fewer shuffles and adds
                // than two of NC
                int j = cnt - 1;
                for (; j >= 1; j -= 2) {
                    const float4 gA = cur[3 * j], qA = cur[3 * j + 1];
                    const float4 gB = cur[3 * j - 3], qB = cur[3 * j - 2];
                    const float dyA = gA.y - ly, dyB = gB.y - ly;
                    PairEval<PPT> eA, eB;
                    const bool anyA = __any_sync(
                        0xffffffffu, pair_phase1<PPT>(gA, qA, dyA, lo + j, last, nlx, eA));
                    const bool anyB = __any_sync(
                        0xffffffffu, pair_phase1<PPT>(gB, qB, dyB, lo + j - 1, last, nlx, eB));
                    if (anyA && anyB) {
                        float v[2 * NC];
                        pair_phase2<CH, PPT, ABS>(eA, gA, qA, cur[3 * j + 2], dyA, T, g, gS, v);
                        pair_phase2<CH, PPT, ABS>(eB, gB, qB, cur[3 * j - 1], dyB, T, g, gS,
                                                  v + NC);
                        const float tot = warp_reduce_split<2 * NC>(v);
                        if (comp2 >= 0) tm.add(acc + (j - comp2_b) * KA + comp2, tot);
                    } else if (anyA) {
                        float v[NC];
                        pair_phase2<CH, PPT, ABS>(eA, gA, qA, cur[3 * j + 2], dyA, T, g, gS, v);
                        const float tot = warp_reduce_split<NC>(v);
                        if (comp >= 0) tm.add(acc + j * KA + comp, tot);
                    } else if (anyB) {
                        float v[NC];
                        pair_phase2<CH, PPT, ABS>(eB, gB, qB, cur[3 * j - 1], dyB, T, g, gS, v);
                        const float tot = warp_reduce_split<NC>(v);
                        if (comp >= 0) tm.add(acc + (j - 1) * KA + comp, tot);
                    }
                }
                if (j == 0) one(0);
            }
        } else {
            for (int j = cnt - 1; j >= 0; --j) {
                if (cull && !(cmask[j] & wbit)) continue;
                const int32_t pos = lo + j;
                const float4 gm = cur[3 * j];
                const float4 q = cur[3 * j + 1];
                const float4 col = cur[3 * j + 2];
                const float dy = gm.y - ly;
                float P0 = 0.0f, P1 = 0.0f, P3 = 0.0f, cw[CH], Hx = 0.0f, Hy = 0.0f;
                // phase 1: alpha and the blend decision of every pixel of the
                // lane; a Gaussian that no pixel of the warp blends is done here
                float dxk[PPT], oGk[PPT], alk[PPT];
                bool hk[PPT];
                bool contrib = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    dxk[k] = gm.x - (float)(pr.lx0 + k);
                    const float power = gauss_power(gm.z, gm.w, q.z, dxk[k], dy);
                    oGk[k] = __fmul_rn(q.w, __expf(power));
                    alk[k] = fminf(kAlphaMax, oGk[k]);
                    hk[k] = pos < last[k] && power <= 0.0f && alk[k] >= kAlphaMin;
                    contrib |= hk[k];
                }
                if (!__any_sync(0xffffffffu, contrib)) continue;
                // phase 2, predicated: a lane whose pixel is not blended here
                // contributes zeros and keeps its state (gS kept negated, as
                // in the paired path)
#pragma unroll
                for (int c = 0; c < CH; ++c) cw[c] = 0.0f;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float alpha = alk[k], oG = oGk[k], dx = dxk[k];
                    const bool hit = hk[k];
                    const float inv = rcp_approx(1.0f - alpha);
                    const float Ti = T[k] * inv;
                    const float w = hit ? alpha * Ti : 0.0f;
                    float gc;
                    if (CH == 3)
                        gc = fmaf(g[k][2], col.z, fmaf(g[k][1], col.y, g[k][0] * col.x));
                    else
                        gc = g[k][0] * col.w;
                    const float dal = fmaf(Ti, gc, inv * gS[k]);
                    gS[k] = fmaf(-w, gc, gS[k]);
#pragma unroll
                    for (int c = 0; c < CH; ++c) cw[c] = fmaf(w, g[k][c], cw[c]);
                    T[k] = hit ? Ti : T[k];
                    // alpha = o G when unclamped; a clamped alpha passes no gradient
                    const float dp = (hit && oG < kAlphaMax) ? oG * dal : 0.0f;
                    const float t = dp * dx;
                    P0 += dp;
                    P1 += t;
                    P3 = fmaf(t, dx, P3);
                    if (ABS) {
                        // this pixel's own contribution to dL/dmean2d, by magnitude
                        Hx += fabsf(dp * fmaf(gm.z, dx, gm.w * dy));
                        Hy += fabsf(dp * fmaf(gm.w, dx, q.z * dy));
                    }
                }
                // the pixels of a run share dy: A2 = dy A0, A4 = dy A1, A5 = dy A2
                float v[NC];
                v[0] = P0;
                v[1] = P1;
                v[2] = dy * P0;
                v[3] = P3;
                v[4] = dy * P1;
                v[5] = dy * v[2];
#pragma unroll
                for (int c = 0; c < CH; ++c) v[6 + c] = cw[c];
                if (ABS) {
                    v[NC0] = Hx;
                    v[NC0 + 1] = Hy;
                }
                const float tot = warp_reduce_split<NC>(v);
                if (comp >= 0) tm.add(acc + j * KA + comp, tot);
            }
        }
        tm.sync();
        // moments -> screen-space gradient (see above), one Gaussian per thread
        for (int j = tm.tid; j < cnt; j += tm.size) {
            float* a = acc + j * KA;
            const float A0 = a[0], A1 = a[1], A2 = a[2];
            if (A0 == 0.0f && A1 == 0.0f && A2 == 0.0f && a[3] == 0.0f && a[4] == 0.0f &&
                a[5] == 0.0f)
                continue;
            const float ca = cur[3 * j].z, cb = cur[3 * j].w;
            const float4 q = cur[3 * j + 1];
            a[0] = -fmaf(ca, A1, cb * A2);
            a[1] = -fmaf(cb, A1, q.z * A2);
            a[2] = -0.5f * a[3];
            a[3] = -a[4];
            a[4] = -0.5f * a[5];
            a[5] = A0 != 0.0f ? A0 / q.w : 0.0f;
        }
        tm.sync();
        // flush this batch's sums: one global atomic per (Gaussian, component, tile)
        if (partial) {
            // deterministic plan: every staged pair's sums go to its own slot
            // (cur_ids hold emission positions), zeros included
            for (int i = tm.tid; i < KA * cnt; i += tm.size) {
                const int j = i / KA, c = i - j * KA;
                partial[(size_t)cur_ids[j] * 11 + c] = acc[i];
                acc[i] = 0.0f;
            }
        } else {
            for (int i = tm.tid; i < KA * cnt; i += tm.size) {
                const float a = acc[i];
                if (a != 0.0f) {
                    const int j = i / KA, c = i - j * KA;
                    if (c < kGrad2d)
                        atomicAdd(grad2d + (size_t)cur_ids[j] * kGrad2d + c, a);
                    else
                        atomicAdd(absgrad + (size_t)cur_ids[j] * 2 + (c - kGrad2d), a);
                    acc[i] = 0.0f;
                }
            }
        }
        tm.sync();
    }
}

template <int PPT, bool WARP, bool ABS>
__global__ void k_render_bwd(ViewTable vt, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ order,
                             const uint32_t* __restrict__ ivals,
                             const uint32_t* __restrict__ gid_of, const float4* __restrict__ rec,
                             int batch, int team_f4, int total_tiles, uint32_t* queue, float bg0,
                             float bg1, float bg2, const float* __restrict__ final_T,
                             const int32_t* __restrict__ last_idx, const float* __restrict__ dL,
                             float* __restrict__ grad2d, float* __restrict__ absgrad,
                             float* __restrict__ partial) {
    extern __shared__ float4 smem[];
    __shared__ int s_slot, s_maxlast;
    const Team<WARP> tm;
    float4* mine = smem + (WARP ? (size_t)(threadIdx.x >> 5) * team_f4 : 0);
    const float bg[3] = {bg0, bg1, bg2};
    for (;;) {
        const int slot = tm.next(queue, &s_slot);
        if (slot >= total_tiles) break;
        const TileCtx tc = tile_ctx(vt, ranges, (int)order[slot]);
        if (tc.channels == 3)
            render_bwd_tile<3, PPT, Team<WARP>, ABS>(tm, vt, tc, ivals, gid_of, rec, mine,
                                                     &s_maxlast, batch, bg, final_T, last_idx, dL,
                                                     grad2d, absgrad, partial);
        else
            render_bwd_tile<1, PPT, Team<WARP>, ABS>(tm, vt, tc, ivals, gid_of, rec, mine,
                                                     &s_maxlast, batch, bg, final_T, last_idx, dL,
                                                     grad2d, absgrad, partial);
    }
}

// Deterministic plans: the screen-space gradient of each (view, Gaussian) is
// the sum of its (Gaussian, tile) partial sums in emission order -- the
// pairs of one (view, Gaussian) were emitted at consecutive positions
// [offs[k], offs[k+1]) of its depth-order rank k -- so every run adds the
// same numbers in the same order.
__global__ void k_partial_reduce(const uint32_t* __restrict__ depth_order,
                                 const uint32_t* __restrict__ offs,
                                 const DevCounters* __restrict__ ctr,
                                 const float* __restrict__ partial, int abs_stats,
                                 float* __restrict__ grad2d, float* __restrict__ absgrad) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ctr->vn) return;
    const uint32_t cnt = ctr->n_instances;
    const uint32_t vg = depth_order[k];
    const uint32_t a = min(offs[k], cnt), b = min(offs[k + 1], cnt);
    float s[11];
#pragma unroll
    for (int c = 0; c < 11; ++c) s[c] = 0.0f;
    for (uint32_t e = a; e < b; ++e)
#pragma unroll
        for (int c = 0; c < 11; ++c) s[c] += partial[(size_t)e * 11 + c];
#pragma unroll
    for (int c = 0; c < kGrad2d; ++c) grad2d[(size_t)vg * kGrad2d + c] = s[c];
    if (abs_stats) {
        absgrad[2 * (size_t)vg] = s[kGrad2d];
        absgrad[2 * (size_t)vg + 1] = s[kGrad2d + 1];
    }
}

}  // namespace

template <typename K>
static K pick(int ppt, K a, K b, K c, K d) {
    return ppt == 1 ? a : ppt == 2 ? b : ppt == 4 ? c : d;
}

// Shared memory of one tile team, in float4 units: the double-buffered
// stage (6 float4 per Gaussian slot) and the 32-bit arrays (2 per slot in the
// forward: masks; 4 plus the nine gradient sums in the backward).
static int team_f4(int batch, bool bwd, bool abs_stats = false) {
    const size_t words =
        bwd ? (size_t)(4 + kGrad2d + (abs_stats ? 2 : 0)) * batch : (size_t)2 * batch;
    return 6 * batch + (int)((words * 4 + 15) / 16);
}

// Warp teams per CTA: as many as fit the default dynamic shared memory, at
// most kMaxWarpTeams (the largest batch still fits one).
static int warp_teams(int tf4) {
    const int t = (int)(kSmemDefault / ((size_t)tf4 * sizeof(float4)));
    return t < 1 ? 1 : (t > kMaxWarpTeams ? kMaxWarpTeams : t);
}

// CTAs of a persistent launch: the resident CTAs of the whole GPU, no more
// than there are teams' worth of tiles.  The occupancy query runs once per
// (kernel, shape, device) and is cached.
static int persistent_blocks(const void* kern, int threads, size_t smem, int tiles_per_block,
                             int total_tiles) {
    struct Entry {
        const void* k;
        int threads, dev;
        size_t smem;
        int blocks;
    };
    static Entry cache[64];
    static int used = 0;
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < used; ++i)
            if (cache[i].k == kern && cache[i].threads == threads && cache[i].smem == smem &&
                cache[i].dev == dev)
                resident = cache[i].blocks;
        if (resident == 0) {
            int per_sm = 0, sms = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) !=
                    cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return -1;
            resident = per_sm * sms;
            if (resident < 1) return -1;
            if (used < 64) cache[used++] = Entry{kern, threads, dev, smem, resident};
        }
    }
    const int want = (total_tiles + tiles_per_block - 1) / tiles_per_block;
    return want < resident ? (want < 1 ? 1 : want) : resident;
}

// The launch shape of a render kernel: one warp per tile when a tile needs
// 32 threads, else one CTA per tile.
struct RenderShape {
    bool warp;
    int threads, tf4, teams;
    size_t smem;
};

static RenderShape render_shape(const Plan* p, int batch, int ppt, bool bwd) {
    RenderShape s;
    const int tile_threads = p->cfg.tile_w * p->cfg.tile_h / ppt;
    s.warp = tile_threads == 32;
    s.tf4 = team_f4(batch, bwd, bwd && p->cfg.density_stats != 0);
    s.teams = s.warp ? warp_teams(s.tf4) : 1;
    s.threads = s.warp ? 32 * s.teams : tile_threads;
    s.smem = (size_t)s.teams * s.tf4 * sizeof(float4);
    return s;
}

gs_status launch_render_fwd(const Plan* p, void* ws, float* images, float* final_T,
                            int32_t* last_idx, cudaStream_t st) {
    const int batch = p->cfg.smem_batch;
    const int ppt = p->cfg.pixels_per_thread;
    const RenderShape s = render_shape(p, batch, ppt, false);
    const uint32_t* ranges = cbuf<uint32_t>(p, ws, GS_BUF_RANGES);
    const uint32_t* order = cbuf<uint32_t>(p, ws, B_TILE_ORDER);
    const uint32_t* vals =
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES);
    const float4* rec = cbuf<float4>(p, ws, GS_BUF_PROJ);
    const uint32_t* gid_of = p->cfg.deterministic ? cbuf<uint32_t>(p, ws, B_GID_OF) : nullptr;
    uint32_t* queue = buf<uint32_t>(p, ws, B_TILE_QUEUE);
    auto kern = s.warp ? pick(ppt, k_render_fwd<1, true>, k_render_fwd<2, true>,
                              k_render_fwd<4, true>, k_render_fwd<8, true>)
                       : pick(ppt, k_render_fwd<1, false>, k_render_fwd<2, false>,
                              k_render_fwd<4, false>, k_render_fwd<8, false>);
    const int blocks = persistent_blocks((const void*)kern, s.threads, s.smem, s.teams,
                                         p->total_tiles);
    if (blocks < 0) return GS_ERR_CUDA;
    if (cudaMemsetAsync(queue, 0, sizeof(uint32_t), st) != cudaSuccess) return GS_ERR_CUDA;
    kern<<<blocks, s.threads, s.smem, st>>>(p->vt, ranges, order, vals, gid_of, rec, batch,
                                            s.tf4, p->total_tiles, queue, p->cfg.bg[0],
                                            p->cfg.bg[1], p->cfg.bg[2], images, final_T,
                                            last_idx);
    return launch_status();
}

gs_status launch_render_bwd_pixels(const Plan* p, void* ws, const float* final_T,
                                   const int32_t* last_idx, const float* dL, cudaStream_t st) {
    const int batch = p->cfg.smem_batch_bwd;
    const int ppt = p->cfg.pixels_per_thread_bwd;
    const RenderShape s = render_shape(p, batch, ppt, true);
    float* grad2d = buf<float>(p, ws, GS_BUF_GRAD2D);
    const uint32_t* ranges = cbuf<uint32_t>(p, ws, GS_BUF_RANGES);
    const uint32_t* order = cbuf<uint32_t>(p, ws, B_TILE_ORDER);
    const uint32_t* vals =
        cbuf<uint32_t>(p, ws, (p->tile_passes & 1) ? (int)B_IVAL_B : (int)GS_BUF_TILE_VALUES);
    const float4* rec = cbuf<float4>(p, ws, GS_BUF_PROJ);
    uint32_t* queue = buf<uint32_t>(p, ws, B_TILE_QUEUE) + 1;
    const bool abs_stats = p->cfg.density_stats != 0;
    float* absgrad = abs_stats ? buf<float>(p, ws, GS_BUF_ABSGRAD) : nullptr;
    const bool det = p->cfg.deterministic != 0;
    const uint32_t* gid_of = det ? cbuf<uint32_t>(p, ws, B_GID_OF) : nullptr;
    float* partial = det ? buf<float>(p, ws, B_PARTIAL) : nullptr;
    auto kern =
        abs_stats
            ? (s.warp ? pick(ppt, k_render_bwd<1, true, true>, k_render_bwd<2, true, true>,
                             k_render_bwd<4, true, true>, k_render_bwd<8, true, true>)
                      : pick(ppt, k_render_bwd<1, false, true>, k_render_bwd<2, false, true>,
                             k_render_bwd<4, false, true>, k_render_bwd<8, false, true>))
            : (s.warp ? pick(ppt, k_render_bwd<1, true, false>, k_render_bwd<2, true, false>,
                             k_render_bwd<4, true, false>, k_render_bwd<8, true, false>)
                      : pick(ppt, k_render_bwd<1, false, false>, k_render_bwd<2, false, false>,
                             k_render_bwd<4, false, false>, k_render_bwd<8, false, false>));
    const int blocks = persistent_blocks((const void*)kern, s.threads, s.smem, s.teams,
                                         p->total_tiles);
    if (blocks < 0) return GS_ERR_CUDA;
    if (cudaMemsetAsync(grad2d, 0, p->len[GS_BUF_GRAD2D], st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(queue, 0, sizeof(uint32_t), st) != cudaSuccess) return GS_ERR_CUDA;
    if (abs_stats &&
        cudaMemsetAsync(absgrad, 0, p->len[GS_BUF_ABSGRAD], st) != cudaSuccess)
        return GS_ERR_CUDA;
    if (det && cudaMemsetAsync(partial, 0, p->len[B_PARTIAL], st) != cudaSuccess)
        return GS_ERR_CUDA;
    kern<<<blocks, s.threads, s.smem, st>>>(p->vt, ranges, order, vals, gid_of, rec, batch,
                                            s.tf4, p->total_tiles, queue, p->cfg.bg[0],
                                            p->cfg.bg[1], p->cfg.bg[2], final_T, last_idx, dL,
                                            grad2d, absgrad, partial);
    if (det) {
        // grid over the plan's capacity; the pair count of the last binning
        // is read on the device
        const uint32_t VNcap = (uint32_t)p->vt.n_views * (uint32_t)p->n_capacity;
        k_partial_reduce<<<(VNcap + 255) / 256, 256, 0, st>>>(
            cbuf<uint32_t>(p, ws, GS_BUF_DEPTH_ORDER), cbuf<uint32_t>(p, ws, B_OFFSETS),
            cbuf<DevCounters>(p, ws, GS_BUF_COUNTERS), partial, abs_stats ? 1 : 0, grad2d,
            absgrad);
    }
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
