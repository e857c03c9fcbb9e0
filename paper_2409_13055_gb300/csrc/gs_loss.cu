// gs_loss.cu -- A6 photometric loss (paper Eq. 2) and its gradient.
//
// Eq. 2 as printed adds lambda * SSIM, which would reward dissimilarity, and
// has no mean; it is read as
//   L_v = (1 - lambda) mean|I - I_gt| + lambda (1 - mean SSIM(I, I_gt)),
// SSIM with an 11x11 Gaussian window (sigma 1.5, unit sum), zero padding,
// C1 = 0.01^2, C2 = 0.03^2, per channel, means over C*H*W of the view, and
// L = view_weight * sum over views (1/n_views: the mean).
//
// Two kernels, each over 32x32 output tiles of every channel plane of every
// view.  The forward stages the tile plus a 5-pixel halo of both images in
// shared memory and forms the window moments E[x], E[y], E[xy] and
// E[x^2 + y^2] with separable 11-tap passes (E[x^2] and E[y^2] enter SSIM
// only through the sum of the variances, and the derivative with respect to
// E[x^2] is the one with respect to that sum); per pixel it keeps the partial
// derivatives of SSIM with respect to E[x], E[x^2] and E[xy].  The backward
// correlates those three maps with the same window (the adjoint of a
// zero-padded symmetric correlation is itself) and adds the L1 term.  The
// loss is reduced deterministically: the forward's per-block partials,
// summed in block order by the backward's first CTA beside its own tile.
#include <math.h>


#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kTX = kLossTileW, kTY = kLossTileH, kHalo = 5, kWin = 11;
constexpr int kRows = kTY + 2 * kHalo;  // 42
constexpr int kCols = kTX + 2 * kHalo;  // 42
constexpr int kLossThreads = 256;       // 32 x 8
constexpr int kSeg = 4;                 // outputs per thread in the horizontal passes
constexpr int kOut = kTY / (kLossThreads / 32);  // output rows per thread in the vertical passes
static_assert(kTX == 32 && kTY % (kLossThreads / 32) == 0, "one warp per tile row band");

struct Win {
    float w[kWin];
};

struct BlockPos {
    int view, ch, x0, y0, width, height;
    int64_t plane;  // offset of the channel plane in packed images
};

__device__ __forceinline__ BlockPos block_pos(const ViewTable& vt, int b) {
    int v = 0;
    while (v + 1 < vt.n_views && b >= vt.v[v + 1].loss_block_offset) ++v;
    const ViewGeom& g = vt.v[v];
    const int bx = (g.width + kTX - 1) / kTX, by = (g.height + kTY - 1) / kTY;
    int r = b - g.loss_block_offset;
    BlockPos p;
    p.view = v;
    p.ch = r / (bx * by);
    r -= p.ch * bx * by;
    p.x0 = (r % bx) * kTX;
    p.y0 = (r / bx) * kTY;
    p.width = g.width;
    p.height = g.height;
    p.plane = g.value_offset + (int64_t)p.ch * g.width * g.height;
    return p;
}

__device__ __forceinline__ float block_sum(float x, float* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[w] = x;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;  // valid in thread 0
}

// The tile and its halo are loaded row by row: warp w takes rows w, w + 8,
// ... (kRowIters of them), lane l columns l and 32 + l (the latter for the
// 10 halo columns only); every load of a thread is issued before its stores.
constexpr int kWarpsL = kLossThreads / 32;
constexpr int kRowIters = (kRows + kWarpsL - 1) / kWarpsL;  // 6
static_assert(kCols - 32 <= 32, "two columns per lane");

struct RowLoader {
    int lane, warp;
    bool ok_a, ok_b;  // columns lane and 32 + lane inside the image (and the halo)
    int xa;
    __device__ __forceinline__ RowLoader(const BlockPos& bp) {
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        xa = bp.x0 - kHalo + lane;
        ok_a = xa >= 0 && xa < bp.width;
        ok_b = lane < kCols - 32 && xa + 32 >= 0 && xa + 32 < bp.width;
    }
    // global offset of tile row r's column lane (which may lie left of the
    // image: then ok_a is false); row_ok: the row is inside the halo and the image
    __device__ __forceinline__ int64_t row_base(const BlockPos& bp, int r, bool& row_ok) const {
        const int y = bp.y0 - kHalo + r;
        row_ok = r < kRows && y >= 0 && y < bp.height;
        return bp.plane + (int64_t)y * bp.width + xa;
    }
};

// Forward: the four window moments of every output value by two separable
// 11-tap passes (horizontal over the tile's 42 halo rows, then vertical),
// SSIM, and its partial derivatives with respect to E[x], E[x^2] and E[xy]
// (the maps the backward correlates).  x and y share one float2 of shared
// memory; the horizontal pass forms x^2 + y^2 and xy once per input value.
// The moments travel in pairs ({E[x], E[y]}, {E[x^2 + y^2], E[xy]}) through
// packed FP32 pair FMAs, each half the scalar fmaf of the same operands.
__global__ void __launch_bounds__(kLossThreads, 5)
k_ssim_fwd(ViewTable vt, Win win, const float* __restrict__ img, const float* __restrict__ tgt,
           float lambda, float inv_views, int64_t total_values, float* __restrict__ maps,
           float* __restrict__ partials, int nblocks, DevCounters* ctr,
           float* __restrict__ loss_dev) {
    __shared__ float2 sxy[kRows][kCols + 1];
    __shared__ float2 h[2][kRows][kTX + 1];
    __shared__ float red[32];
    grid_dep_begin();    // the rendered images are complete
    grid_dep_release();  // the backward's CTAs may take the SMs of the last wave
    const BlockPos bp = block_pos(vt, blockIdx.x);
    {
        const RowLoader ld(bp);
        float a[kRowIters], b[kRowIters], c[kRowIters], d[kRowIters];
#pragma unroll
        for (int k = 0; k < kRowIters; ++k) {
            bool row_ok;
            const int64_t base = ld.row_base(bp, ld.warp + kWarpsL * k, row_ok);
            a[k] = b[k] = c[k] = d[k] = 0.0f;
            if (row_ok && ld.ok_a) {
                a[k] = img[base];
                b[k] = tgt[base];
            }
            if (row_ok && ld.ok_b) {
                c[k] = img[base + 32];
                d[k] = tgt[base + 32];
            }
        }
#pragma unroll
        for (int k = 0; k < kRowIters; ++k) {
            const int r = ld.warp + kWarpsL * k;
            if (r < kRows) {
                sxy[r][ld.lane] = make_float2(a[k], b[k]);
                if (ld.lane < kCols - 32) sxy[r][32 + ld.lane] = make_float2(c[k], d[k]);
            }
        }
    }
    __syncthreads();
    // horizontal pass: a thread takes kSeg consecutive outputs of one row,
    // reading their kSeg + 10 inputs once; consecutive threads take
    // consecutive rows (conflict-free 8-byte shared accesses)
    for (int i = threadIdx.x; i < kRows * (kTX / kSeg); i += blockDim.x) {
        const int seg = i / kRows, r = i - seg * kRows, c0 = seg * kSeg;
        float2 xy[kSeg + kWin - 1], pq[kSeg + kWin - 1];  // {x, y}, {x^2 + y^2, x y}
#pragma unroll
        for (int k = 0; k < kSeg + kWin - 1; ++k) {
            const float2 p = sxy[r][c0 + k];
            xy[k] = p;
            pq[k] = make_float2(fmaf(p.x, p.x, p.y * p.y), p.x * p.y);
        }
#pragma unroll
        for (int o = 0; o < kSeg; ++o) {
            float2 m1 = make_float2(0.f, 0.f), m2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float2 w2 = make_float2(win.w[k], win.w[k]);
                m1 = fma2(w2, xy[o + k], m1);
                m2 = fma2(w2, pq[o + k], m2);
            }
            h[0][r][c0 + o] = m1;
            h[1][r][c0 + o] = m2;
        }
    }
    __syncthreads();
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float l1 = 0.0f, ss = 0.0f;
    // vertical pass: a thread takes kOut consecutive rows of one column,
    // reading their kOut + 10 rows of horizontal sums once
    const int r0 = kOut * ty;
    float2 m[kOut][2];
#pragma unroll
    for (int o = 0; o < kOut; ++o)
#pragma unroll
        for (int q = 0; q < 2; ++q) m[o][q] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < kWin + kOut - 1; ++k) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float2 hv = h[q][r0 + k][tx];
#pragma unroll
            for (int o = 0; o < kOut; ++o)
                if (k - o >= 0 && k - o < kWin)
                    m[o][q] = fma2(make_float2(win.w[k - o], win.w[k - o]), hv, m[o][q]);
        }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const int rr = r0 + o;
        const int x = bp.x0 + tx, y = bp.y0 + rr;
        if (x >= bp.width || y >= bp.height) continue;
        const float mx = m[o][0].x, my = m[o][0].y;
        const float mm = fmaf(mx, mx, my * my);
        const float vxy = m[o][1].x - mm, cxy = m[o][1].y - mx * my;  // sum of variances, covariance
        const float A = 2.0f * mx * my + C1, B = 2.0f * cxy + C2;
        const float Cd = mm + C1, D = vxy + C2;
        // one division: 1/Cd = D/(Cd D), 1/D = Cd/(Cd D) (Cd >= C1, D >= C2)
        const float iCD = 1.0f / (Cd * D);
        const float iC = D * iCD, iD = Cd * iCD;
        const float s = A * B * iCD;
        // dSSIM/dE[x], dSSIM/dE[x^2], dSSIM/dE[xy] (E[y], E[y^2] held fixed)
        const float ds_dm = 2.0f * my * (B - A) * iCD - 2.0f * mx * s * (iC - iD);
        const float ds_dxx = -s * iD;
        const float ds_dxy = 2.0f * A * iCD;
        const int64_t idx = bp.plane + (int64_t)y * bp.width + x;
        maps[idx] = ds_dm;
        maps[total_values + idx] = ds_dxx;
        maps[2 * total_values + idx] = ds_dxy;
        ss += s;
        const float2 p = sxy[rr + kHalo][tx + kHalo];
        l1 += fabsf(p.x - p.y);
    }
    const ViewGeom& g = vt.v[bp.view];
    const float invM = 1.0f / ((float)g.channels * (float)g.width * (float)g.height);
    const float part = inv_views * invM * ((1.0f - lambda) * l1 - lambda * ss);
    const float tot = block_sum(part, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// The loss: the forward's per-block partials summed in block order (one CTA).
__device__ __forceinline__ void loss_total(const ViewTable& vt, float lambda, float inv_views,
                                           const float* __restrict__ partials, int nblocks,
                                           DevCounters* ctr, float* __restrict__ loss_dev,
                                           float* red) {
    float acc = 0.0f;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[i];
    const float all = block_sum(acc, red);
    if (threadIdx.x == 0) {
        const float L = lambda * inv_views * (float)vt.n_views + all;
        *loss_dev = L;
        ctr->loss = L;
    }
}

// Backward: the three maps correlated with the window (two separable passes,
// as the forward), combined per value with x and y, plus the L1 term.
__global__ void __launch_bounds__(kLossThreads, 5)
k_ssim_bwd(ViewTable vt, Win win, const float* __restrict__ img, const float* __restrict__ tgt,
           float lambda, float inv_views, int64_t total_values, const float* __restrict__ maps,
           float* __restrict__ dL, const float* __restrict__ partials, int nblocks,
           DevCounters* ctr, float* __restrict__ loss_dev) {
    __shared__ float red[32];
    // maps 0 and 1 as pairs, map 2 alone (packed pair FMAs on the pairs)
    __shared__ float2 sm01[kRows][kCols + 1];
    __shared__ float sm2[kRows][kCols + 1];
    __shared__ float2 h01[kRows][kTX + 1];
    __shared__ float h2[kRows][kTX + 1];
    const BlockPos bp = block_pos(vt, blockIdx.x);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r0 = kOut * ty;
    // this thread's output values of both images, loaded with the maps
    float xo[kOut], yo[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const int x = bp.x0 + tx, y = bp.y0 + r0 + o;
        xo[o] = yo[o] = 0.0f;
        if (x < bp.width && y < bp.height) {
            xo[o] = img[bp.plane + (int64_t)y * bp.width + x];
            yo[o] = tgt[bp.plane + (int64_t)y * bp.width + x];
        }
    }
    // the images were complete before the forward's CTAs released this grid;
    // the maps and the loss partials are complete once the whole forward grid is
    grid_dep_begin();
    // CTA 0 also sums the loss (in block order), beside the other CTAs' work
    if (blockIdx.x == 0) loss_total(vt, lambda, inv_views, partials, nblocks, ctr, loss_dev, red);
    {
        // the three maps over the tile and its halo, in two halves of rows
        const RowLoader ld(bp);
        constexpr int kHalf = (kRowIters + 1) / 2;
#pragma unroll
        for (int h0 = 0; h0 < kRowIters; h0 += kHalf) {
            float a[kHalf][2], b[kHalf][2], d[kHalf][2];
#pragma unroll
            for (int k = 0; k < kHalf; ++k) {
                bool row_ok;
                const int64_t base = ld.row_base(bp, ld.warp + kWarpsL * (h0 + k), row_ok);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    a[k][s] = b[k][s] = d[k][s] = 0.0f;
                    if (row_ok && (s == 0 ? ld.ok_a : ld.ok_b)) {
                        const int64_t idx = base + 32 * s;
                        a[k][s] = maps[idx];
                        b[k][s] = maps[total_values + idx];
                        d[k][s] = maps[2 * total_values + idx];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kHalf; ++k) {
                const int r = ld.warp + kWarpsL * (h0 + k);
                if (r < kRows) {
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        if (s == 1 && ld.lane >= kCols - 32) continue;
                        sm01[r][32 * s + ld.lane] = make_float2(a[k][s], b[k][s]);
                        sm2[r][32 * s + ld.lane] = d[k][s];
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRows * (kTX / kSeg); i += blockDim.x) {
        const int seg = i / kRows, r = i - seg * kRows, c0 = seg * kSeg;
        float2 u01[kSeg + kWin - 1];
        float u2[kSeg + kWin - 1];
#pragma unroll
        for (int k = 0; k < kSeg + kWin - 1; ++k) {
            u01[k] = sm01[r][c0 + k];
            u2[k] = sm2[r][c0 + k];
        }
#pragma unroll
        for (int o = 0; o < kSeg; ++o) {
            float2 ab = make_float2(0.f, 0.f);
            float d = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float w = win.w[k];
                ab = fma2(make_float2(w, w), u01[o + k], ab);
                d = fmaf(w, u2[o + k], d);
            }
            h01[r][c0 + o] = ab;
            h2[r][c0 + o] = d;
        }
    }
    __syncthreads();
    const ViewGeom& g = vt.v[bp.view];
    const float scale = inv_views / ((float)g.channels * (float)g.width * (float)g.height);
    float2 m01[kOut];
    float m2[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        m01[o] = make_float2(0.0f, 0.0f);
        m2[o] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kWin + kOut - 1; ++k) {
        const float2 hv = h01[r0 + k][tx];
        const float hd = h2[r0 + k][tx];
#pragma unroll
        for (int o = 0; o < kOut; ++o)
            if (k - o >= 0 && k - o < kWin) {
                const float w = win.w[k - o];
                m01[o] = fma2(make_float2(w, w), hv, m01[o]);
                m2[o] = fmaf(w, hd, m2[o]);
            }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const int x = bp.x0 + tx, y = bp.y0 + r0 + o;
        if (x >= bp.width || y >= bp.height) continue;
        const int64_t idx = bp.plane + (int64_t)y * bp.width + x;
        const float xv = xo[o], yv = yo[o];
        const float diff = xv - yv;
        const float sgn = diff > 0.0f ? 1.0f : (diff < 0.0f ? -1.0f : 0.0f);
        const float dssim = m01[o].x + 2.0f * xv * m01[o].y + yv * m2[o];
        dL[idx] = scale * ((1.0f - lambda) * sgn - lambda * dssim);
    }
}

}  // namespace

// The 11-tap window: Gaussian of sigma 1.5 sampled at -5..5, normalised to
// unit sum (in double, then rounded once).
static Win loss_window() {
    Win win;
    double g[kWin], s = 0.0;
    for (int k = 0; k < kWin; ++k) {
        const double d = k - kHalo;
        g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k < kWin; ++k) win.w[k] = (float)(g[k] / s);
    return win;
}

gs_status launch_loss(const Plan* p, const float* images, const float* targets, float lambda,
                      float view_weight, float* loss_dev, float* dL, void* ws, cudaStream_t st) {
    const Win win = loss_window();
    float* maps = buf<float>(p, ws, B_LOSS_MAPS);
    float* partials = buf<float>(p, ws, B_LOSS_BLOCKS);
    DevCounters* ctr = buf<DevCounters>(p, ws, GS_BUF_COUNTERS);
    const float inv_views = view_weight;
    launch_pdl(k_ssim_fwd, p->loss_blocks, kLossThreads, 0, st, p->vt, win, images, targets,
               lambda, inv_views, p->total_values, maps, partials, p->loss_blocks, ctr, loss_dev);
    launch_pdl(k_ssim_bwd, p->loss_blocks, kLossThreads, 0, st, p->vt, win, images, targets,
               lambda, inv_views, p->total_values, (const float*)maps, dL,
               (const float*)partials, p->loss_blocks, ctr, loss_dev);
    return launch_status();
}

}  // namespace gs

// ---------------------------------------------------------------------------
// gs_loss_l1_ssim_noalloc: the same loss for callers that cannot allocate
// device memory, with its scratch in a fixed array compiled into this library.
// ---------------------------------------------------------------------------
namespace gs {
namespace {

constexpr size_t kNoAllocMaxValues = size_t(1) << 20;  // image values (C*H*W over all views)
constexpr int kNoAllocMaxBlocks = 8192;                // 32x32 loss tiles over all planes
constexpr size_t kNoAllocPartialsOffset = 256;         // after the counters
constexpr size_t kNoAllocMapsOffset =
    kNoAllocPartialsOffset + ((size_t(kNoAllocMaxBlocks + 1) * 2 * sizeof(float) + 255) & ~size_t(255));
constexpr size_t kNoAllocBytes = kNoAllocMapsOffset + 3 * kNoAllocMaxValues * sizeof(float);

// Scratch of gs_loss_l1_ssim_noalloc: counters (the loss) | per-block loss
// partials | the three SSIM partial-derivative maps.  About
// 12.6 MB, held on every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, with the device current.  It is looked up again
// on every call (a host-side table lookup once the module is loaded): an
// address kept from an earlier call could outlive its context (a device
// reset, a context destroyed and created again) and send the kernels to
// memory that is no longer the array.
gs_status noalloc_scratch(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
        return GS_ERR_CUDA;
    *out = p;
    return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_loss_l1_ssim_noalloc(const gs_plan* plan, const float* images,
                                             const float* targets, float lambda, float view_weight,
                                             float* loss_dev, float* dL_dimages, void* stream) {
    using namespace gs;
    if (!plan || P(plan)->magic != kPlanMagic || !images || !targets || !loss_dev || !dL_dimages)
        return GS_ERR_INVALID;
    if (!(lambda >= 0.0f && lambda <= 1.0f) || !(view_weight > 0.0f)) return GS_ERR_INVALID;
    const Plan* p = P(plan);
    // sizes are checked before anything touches the GPU
    if ((size_t)p->total_values > kNoAllocMaxValues || p->loss_blocks > kNoAllocMaxBlocks)
        return GS_ERR_CAPACITY;
    void* scratch = nullptr;
    gs_status s = noalloc_scratch(&scratch);
    if (s != GS_OK) return s;
    cudaStream_t st = S(stream);
    char* base = static_cast<char*>(scratch);
    DevCounters* ctr = reinterpret_cast<DevCounters*>(base);
    float* partials = reinterpret_cast<float*>(base + kNoAllocPartialsOffset);
    float* maps = reinterpret_cast<float*>(base + kNoAllocMapsOffset);
    const Win win = loss_window();
    k_ssim_fwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        view_weight, p->total_values, maps,
                                                        partials, p->loss_blocks, ctr, loss_dev);
    k_ssim_bwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        view_weight, p->total_values, maps,
                                                        dL_dimages, partials, p->loss_blocks, ctr,
                                                        loss_dev);
    return launch_status();
}
