// gs_internal.cuh -- internal layout and device helpers of libgs_gb300.
//
// Not part of the C-ABI: the plan's private layout, the workspace carving and
// the small device functions shared by the kernels of this library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "../../include/gs.h"

namespace gs {

constexpr uint32_t kPlanMagic = 0x67733330u;  // "gs30"
constexpr int kOrderBuckets = 33;  // tile-order buckets: bit length of a list length
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;  // elements per sort block
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // elements per scan block
constexpr int kProjFloats = 12;                       // floats per projected record
constexpr int kLossTileW = 32, kLossTileH = 32;       // output tile of the loss kernels
constexpr int kGrad2d = 9;                            // floats per screen-space gradient

// Per-view geometry derived by gs_plan_init; passed to kernels by value.
struct ViewGeom {
    int32_t width, height, channels, tiles_x, tiles_y;
    int32_t tile_offset;   // first global tile id of this view
    int32_t loss_block_offset;  // first block of this view in the loss kernels
    int64_t pixel_offset;  // offset in per-pixel maps (H*W units)
    int64_t value_offset;  // offset in packed planar images (C*H*W units)
};

struct ViewTable {
    int32_t n_views;
    int32_t tile_w, tile_h, log2_tw, log2_th;
    int32_t tight_rect;  // gs_config.tight_rect
    ViewGeom v[GS_MAX_VIEWS];
};

// Workspace buffers (ids >= GS_BUF_COUNT are private).
enum PrivBuf {
    B_DKEY_A = GS_BUF_COUNT,  // [V*n] FP32 depth keys of the projection (0xFFFFFFFF: culled);
                              // the sort reads them and never overwrites them
    B_DKEY_B,
    B_DVAL_B,
    B_DKEY_C,
    B_SCAN_BLOCKS,
    B_HIST,
    B_IKEY_B,
    B_IVAL_B,
    B_LOSS_MAPS,
    B_LOSS_BLOCKS,
    B_GCOL,     // [V*n] x 3: colour gradient as it reaches the SH coefficients
    B_OFFSETS,  // [V*n + 1] instance offsets of the entries in depth order
    B_TILE_ORDER,  // [total_tiles] render order of the tiles, longest lists first;
                   // then 2 x kOrderBuckets words of scratch for building it
    B_TILE_QUEUE,  // [2] u32 next-tile counters of the forward and backward render
    B_GID_OF,      // [instance_capacity] u32 (view*n + index) of each emitted instance
                   // (deterministic plans: the sort then carries emission positions)
    B_PARTIAL,     // [instance_capacity] x 11 floats: per-(Gaussian, tile) partial sums
                   // of the pixel adjoint (deterministic plans)
    B_SPANS,       // [V*n] x kSpanRows u32: tight row spans, x0 | x1 << 16 per tile row
                   // (tight plans); a box of more than kSpanRows rows stores its spans
                   // in B_SPAN_POOL and the pool index of its first row in word 0
    B_SPAN_POOL,   // [span_pool_rows] u32: row spans of the taller boxes
    B_TOTAL
};

struct Plan {
    uint32_t magic;
    gs_config cfg;
    int32_t n_capacity;
    int64_t inst_capacity;
    int32_t total_tiles, tile_bits, tile_passes;
    int64_t total_pixels, total_values;
    int32_t depth_sort_blocks, inst_sort_blocks, scan_blocks, loss_blocks;
    uint32_t span_pool_rows;  // capacity of B_SPAN_POOL (tight plans)
    // Recompute plans (gs_config.recompute = views per pass): the workspace
    // holds the projection and binning of ws_views views; the plan itself
    // covers all n_views_full views, a pass plan (gs_plan_view_pass) the
    // views from view_index on (-1 in a plan made by gs_plan_init), with the
    // same layout.
    int32_t recompute, ws_views, n_views_full, view_index;
    size_t ws_bytes;
    size_t off[B_TOTAL];
    size_t len[B_TOTAL];
    ViewTable vt;
};
static_assert(sizeof(Plan) <= sizeof(gs_plan), "gs_plan too small for the private plan");

// Device counters at the head of the workspace.
struct DevCounters {
    uint32_t status;
    uint32_t n_instances;          // clamped to capacity
    unsigned long long n_raw;      // before clamping
    float loss;
    uint32_t loss_blocks_done;     // reserved (zero)
    uint32_t vn;                   // depth-order entries (visible pairs) of the last gs_bin_sort
    uint32_t n_sorted;             // visible pairs kept by the first depth pass
    uint32_t span_pool_used;       // rows of B_SPAN_POOL taken by the last gs_project
};

static_assert(offsetof(DevCounters, status) == 0, "gs_project keeps the leading status word");

inline const Plan* P(const gs_plan* p) { return reinterpret_cast<const Plan*>(p); }

template <typename T>
inline T* buf(const Plan* p, void* ws, int id) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + p->off[id]);
}
template <typename T>
inline const T* cbuf(const Plan* p, const void* ws, int id) {
    return reinterpret_cast<const T*>(static_cast<const char*>(ws) + p->off[id]);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Streaming multiprocessors of the current device, queried once per device
// and cached; 0 if the query fails.  Grid-stride kernels size their grids in
// multiples of it.
int sm_count();

inline gs_status launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// Programmatic dependent launch: the kernel may be scheduled while the kernel
// before it on the stream is still draining, so that chains of short kernels
// do not pay a full launch gap at every boundary.  Every kernel launched this
// way calls grid_dep_begin() before its first access to memory (the wait
// returns once the preceding grid has completed and its writes are visible),
// which also keeps the order transitive along the chain.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // checked by launch_status
}

// Start of a kernel launched by launch_pdl: wait for the preceding grid.  The
// next kernel of the chain is released when this grid's CTAs exit.  A plain
// launch makes the instruction a no-op.
__device__ __forceinline__ void grid_dep_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Let the next kernel of the chain launch once every CTA of this grid has
// called this (instead of once they have exited): its CTAs can then take the
// SMs this grid's last wave leaves idle and run up to their own
// grid_dep_begin(), which still waits for this whole grid.  A plain launch
// makes the instruction a no-op.
__device__ __forceinline__ void grid_dep_release() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------

// View of a global tile id: views are few (<= 64), a linear scan is uniform
// across the block.
__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int tile) {
    int v = 0;
    while (v + 1 < vt.n_views && tile >= vt.v[v + 1].tile_offset) ++v;
    return v;
}

// Error-free transformations on floats (Knuth's TwoSum, Dekker's FastTwoSum,
// and the fma-based exact product).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Compensated dot product r0*x0 + r1*x1 + r2*x2 + t (Ogita-Rump-Oishi Dot2),
// returned as a normalised (hi, lo) pair.
__device__ __forceinline__ void dot3_plus(float r0, float r1, float r2, float x0, float x1,
                                          float x2, float t, float& hi, float& lo) {
    float p, e, h, l, s, q;
    two_prod(r0, x0, p, e);
    two_prod(r1, x1, h, l);
    two_sum(p, h, s, q);
    e = __fadd_rn(e, __fadd_rn(q, l));
    two_prod(r2, x2, h, l);
    two_sum(s, h, p, q);
    e = __fadd_rn(e, __fadd_rn(q, l));
    two_sum(p, t, s, q);
    e = __fadd_rn(e, q);
    fast_two_sum(s, e, hi, lo);
}

// (xh + xl) / (zh + zl) as a (hi, lo) pair.
__device__ __forceinline__ void df_div(float xh, float xl, float zh, float zl, float& qh,
                                       float& ql) {
    float q1 = __fdiv_rn(xh, zh);
    // r = x - q1*z, with x - q1*zh exact through the fma
    float r = __fmaf_rn(-q1, zh, xh);
    r = __fadd_rn(r, __fmaf_rn(-q1, zl, xl));
    float q2 = __fdiv_rn(r, zh);
    fast_two_sum(q1, q2, qh, ql);
}

// f * (qh + ql) + c as a (hi, lo) pair.
__device__ __forceinline__ void df_affine(float f, float qh, float ql, float c, float& hi,
                                          float& lo) {
    float p, e, s, q;
    two_prod(f, qh, p, e);
    e = __fmaf_rn(f, ql, e);
    two_sum(p, c, s, q);
    fast_two_sum(s, __fadd_rn(e, q), hi, lo);
}

// floor((hi + lo) / t) for a power-of-two t, exact for a normalised pair.
__device__ __forceinline__ int df_floor_div(float hi, float lo, float inv_t) {
    float a = __fmul_rn(hi, inv_t);  // exact: power-of-two scaling
    float fa = floorf(a);
    if (fa == a && lo < 0.0f) fa -= 1.0f;
    return (int)fa;
}

// Tight tiles, row by row: the level of the widened ellipse q <= t outside
// which alpha = o exp(-q/2) < 1/255 with a margin (t = 1.01 * 2 ln(255 o) +
// 0.01), and the tiles of tile row ty (clipped to [rx0, rx1)) whose band of
// pixel rows meets it.  q = A dx^2 + 2 B dx dy + C dy^2 in the conic (A, B, C);
// for a fixed dy the ellipse spans dx = (-B dy +- sqrt(A t - D dy^2)) / A,
// D = AC - B^2; over the band the largest dx is sqrt(t C / D) when the row of
// the ellipse's rightmost point, dy* = -(B / C) sqrt(t C / D), lies in the band,
// else the larger band end; the smallest symmetrically at -dy*.  The
// projection computes the spans of every row of the box once and stores
// them for the emission to list: in the Gaussian's own kSpanRows slots
// (B_SPANS), or, for a taller box, in rows taken from the plan's span pool
// (B_SPAN_POOL), whose first index goes to slot 0.  A box that finds the
// pool full keeps all its tiles (kSpanNoPool in slot 0, GS_DEV_SPAN_POOL).
constexpr int kSpanRows = 16;
constexpr uint32_t kSpanNoPool = 0xFFFFFFFFu;
__device__ __forceinline__ float tight_level(float opacity) {
    return __fmaf_rn(1.01f, __fmul_rn(2.0f, logf(__fmul_rn(255.0f, opacity))), 0.01f);
}

struct TightEllipse {
    float mxh, mxl, myh, myl;  // mean as float pairs
    float X, Y;                // x- and y-half-extents of the widened ellipse
    float ds;                  // row of its rightmost point, relative to the mean
    float negB, invA, At, D;   // -B, 1/A, A t, AC - B^2
};

static __device__ __forceinline__ TightEllipse tight_ellipse(float mxh, float mxl, float myh,
                                                          float myl, float A, float B, float C,
                                                          float opacity) {
    TightEllipse E;
    const float t = tight_level(opacity);
    E.mxh = mxh; E.mxl = mxl; E.myh = myh; E.myl = myl;
    E.D = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    E.Y = __fsqrt_rn(__fdiv_rn(__fmul_rn(t, A), E.D));
    E.X = __fsqrt_rn(__fdiv_rn(__fmul_rn(t, C), E.D));
    E.ds = -__fmul_rn(__fdiv_rn(B, C), E.X);
    E.negB = -B;
    E.invA = __frcp_rn(A);
    E.At = __fmul_rn(A, t);
    return E;
}

static __device__ __forceinline__ int tight_row_span(const TightEllipse& E, int ty, int log2_tw,
                                                  int log2_th, int rx0, int rx1, int* x0,
                                                  int* x1) {
    const float th = (float)(1 << log2_th), tw = (float)(1 << log2_tw);
    float lo = __fsub_rn(__fsub_rn(__fmul_rn((float)ty, th), E.myh), E.myl);
    float hi = __fadd_rn(lo, __fsub_rn(th, 1.0f));
    *x0 = *x1 = rx0;
    if (lo > E.Y || hi < -E.Y) return 0;
    lo = fmaxf(lo, -E.Y);
    hi = fminf(hi, E.Y);
    auto half = [&](float dy) {
        return __fsqrt_rn(fmaxf(0.0f, __fsub_rn(E.At, __fmul_rn(E.D, __fmul_rn(dy, dy)))));
    };
    float xmax, xmin;
    if (lo <= E.ds && E.ds <= hi) {
        xmax = E.X;
    } else {
        xmax = fmaxf(__fmul_rn(__fadd_rn(__fmul_rn(E.negB, lo), half(lo)), E.invA),
                     __fmul_rn(__fadd_rn(__fmul_rn(E.negB, hi), half(hi)), E.invA));
    }
    if (lo <= -E.ds && -E.ds <= hi) {
        xmin = -E.X;
    } else {
        xmin = fminf(__fmul_rn(__fsub_rn(__fmul_rn(E.negB, lo), half(lo)), E.invA),
                     __fmul_rn(__fsub_rn(__fmul_rn(E.negB, hi), half(hi)), E.invA));
    }
    // tiles [ceil((mu + xmin - T + 1) / T), floor((mu + xmax) / T)], mu as a pair
    const float it = __frcp_rn(tw);  // exact: a power of two
    float s, e;
    two_sum(E.mxh, __fsub_rn(xmin, __fsub_rn(tw, 1.0f)), s, e);
    fast_two_sum(s, __fadd_rn(e, E.mxl), s, e);
    const int k0 = -df_floor_div(-s, -e, it);
    two_sum(E.mxh, xmax, s, e);
    fast_two_sum(s, __fadd_rn(e, E.mxl), s, e);
    const int k1 = df_floor_div(s, e, it) + 1;
    *x0 = min(max(k0, rx0), rx1);
    *x1 = max(min(k1, rx1), *x0);
    return *x1 - *x0;
}

// The Gaussian's weight at a pixel, evaluated identically by the forward and
// the backward kernels: power = -(a dx^2 + c dy^2)/2 - b dx dy.
// Packed FP32 pairs (PTX .f32x2, sm_100 and later): one instruction does the
// operation on both halves, each an IEEE round-to-nearest operation, so the
// results are bit-identical to fmaf / __fmul_rn / __fadd_rn on each half.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float gauss_power(float a, float b, float c, float dx, float dy) {
    float q = __fmaf_rn(a, __fmul_rn(dx, dx), __fmul_rn(c, __fmul_rn(dy, dy)));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(b, __fmul_rn(dx, dy)));
}

// One Adam update of one float (paper Sec. IV-A, the default 3DGS optimiser):
// m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr (m ibc1) / (sqrt(v ibc2) + eps),
// ibc = 1 / (1 - beta^t).  Shared by the stand-alone and the fused Adam so both
// produce the same bits.
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                      float b2, float eps, float ibc1, float ibc2) {
    m = fmaf(b1, m, (1.0f - b1) * g);
    v = fmaf(b2, v, (1.0f - b2) * g * g);
    p -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

// b^t for a step count t >= 0 by binary powering in FP64: at most 2 log2(t)
// roundings, a relative error below 1e-14 for any 32-bit t, and a few dozen
// dependent multiplications where a general FP64 pow costs thousands of
// cycles of the GPU's narrow FP64 pipe while every thread of the CTA waits.
__device__ __forceinline__ double pow_step(double b, int t) {
    double r = 1.0;
    for (; t > 0; t >>= 1) {
        if (t & 1) r *= b;
        b *= b;
    }
    return r;
}

// Bias corrections 1/(1 - b1^t), 1/(1 - b2^t) of step t.
__device__ __forceinline__ void adam_bias(float b1, float b2, int t, float& ibc1, float& ibc2) {
    ibc1 = (float)(1.0 / (1.0 - pow_step((double)b1, t)));
    ibc2 = (float)(1.0 / (1.0 - pow_step((double)b2, t)));
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// ---------------------------------------------------------------------------
// Host-side launch helpers implemented in the .cu files.
// ---------------------------------------------------------------------------
gs_status launch_project(const Plan* p, const gs_map* map, const gs_view* views_dev, void* ws,
                         cudaStream_t st);
gs_status launch_bin_sort(const Plan* p, int32_t n, void* ws, cudaStream_t st);
gs_status launch_render_fwd(const Plan* p, void* ws, float* images, float* final_T,
                            int32_t* last_idx, cudaStream_t st);
gs_status launch_loss(const Plan* p, const float* images, const float* targets, float lambda,
                      float view_weight, float* loss_dev, float* dL, void* ws, cudaStream_t st);
gs_status launch_render_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                            void* ws, const float* final_T, const int32_t* last_idx,
                            const float* dL, const gs_map_grad* grads, int32_t accumulate,
                            cudaStream_t st);
gs_status launch_render_bwd_pixels(const Plan* p, void* ws, const float* final_T,
                                   const int32_t* last_idx, const float* dL, cudaStream_t st);
gs_status launch_project_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                             void* ws, const gs_map_grad* grads, int accumulate, cudaStream_t st,
                             uint8_t* group_vis = nullptr);
gs_status launch_adam_groups(float* params, const float* grads, float* m, float* v, int64_t n,
                             int32_t n_groups, const int64_t* offs, const float* lrs,
                             const int32_t* strides, int32_t n_gauss, const uint8_t* group_vis,
                             float b1, float b2, float eps, int32_t* step_dev, cudaStream_t st);
gs_status launch_step_inc(int32_t* step_dev, cudaStream_t st);
gs_status launch_project_bwd_adam(const Plan* p, const gs_map* map, const gs_view* views_dev,
                                  void* ws, const gs_map_grad* params, const gs_map_grad* m,
                                  const gs_map_grad* v, const gs_map_grad* grads_acc,
                                  const gs_map_grad* grads_out, const float* lr6, float b1,
                                  float b2, float eps, int32_t* step_dev, cudaStream_t st);
gs_status launch_visibility(int n, int n_views, const uint32_t* touched, uint8_t* vis,
                            cudaStream_t st);
gs_status launch_adam_sparse(float* params, const float* grads, float* m, float* v, int64_t n,
                             int32_t n_groups, const int64_t* offs, const float* lrs,
                             const int32_t* strides, int32_t n_gauss, const uint8_t* vis,
                             float b1, float b2, float eps, int32_t* step_dev, cudaStream_t st);
gs_status launch_adam(float* params, const float* grads, float* m, float* v, int64_t n,
                      int32_t n_groups, const int64_t* offs, const float* lrs, float b1,
                      float b2, float eps, int32_t* step_dev, cudaStream_t st);

}  // namespace gs
