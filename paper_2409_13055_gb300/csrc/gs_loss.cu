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
// shared memory and forms the five window moments (E[x], E[y], E[x^2],
// E[y^2], E[xy]) with separable 11-tap passes; per pixel it keeps the partial
// derivatives of SSIM with respect to E[x], E[x^2] and E[xy].  The backward
// correlates those three maps with the same window (the adjoint of a
// zero-padded symmetric correlation is itself) and adds the L1 term.  The
// loss is reduced deterministically: per-block partials, summed in block
// order by whichever block finishes last (a ticket counter, no waiting).
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

// Loads of the tile and its halo issued by every thread before any store.
constexpr int kLoads = (kRows * kCols + kLossThreads - 1) / kLossThreads;

// Forward: the five window moments of every output value by two separable
// 11-tap passes (horizontal over the tile's 42 halo rows, then vertical),
// SSIM, and its partial derivatives with respect to E[x], E[x^2] and E[xy]
// (the maps the backward correlates).  x and y share one float2 of shared
// memory; the horizontal pass forms x^2, y^2 and xy once per input value.
__global__ void __launch_bounds__(kLossThreads)
k_ssim_fwd(ViewTable vt, Win win, const float* __restrict__ img, const float* __restrict__ tgt,
           float lambda, float inv_views, int64_t total_values, float* __restrict__ maps,
           float* __restrict__ partials, int nblocks, DevCounters* ctr,
           float* __restrict__ loss_dev) {
    __shared__ float2 sxy[kRows][kCols + 1];
    __shared__ float h[5][kRows][kTX + 1];
    __shared__ float red[32];
    __shared__ bool is_last;
    const BlockPos bp = block_pos(vt, blockIdx.x);
    {
        float a[kLoads], b[kLoads];
#pragma unroll
        for (int it = 0; it < kLoads; ++it) {
            const int i = threadIdx.x + it * kLossThreads;
            const int r = i / kCols, c = i - r * kCols;
            const int y = bp.y0 - kHalo + r, x = bp.x0 - kHalo + c;
            a[it] = b[it] = 0.0f;
            if (i < kRows * kCols && x >= 0 && x < bp.width && y >= 0 && y < bp.height) {
                a[it] = img[bp.plane + (int64_t)y * bp.width + x];
                b[it] = tgt[bp.plane + (int64_t)y * bp.width + x];
            }
        }
#pragma unroll
        for (int it = 0; it < kLoads; ++it) {
            const int i = threadIdx.x + it * kLossThreads;
            if (i < kRows * kCols) {
                const int r = i / kCols, c = i - r * kCols;
                sxy[r][c] = make_float2(a[it], b[it]);
            }
        }
    }
    __syncthreads();
    // horizontal pass: a thread takes kSeg consecutive outputs of one row,
    // reading their kSeg + 10 inputs once
    for (int i = threadIdx.x; i < kRows * (kTX / kSeg); i += blockDim.x) {
        const int r = i / (kTX / kSeg), c0 = (i - r * (kTX / kSeg)) * kSeg;
        float u[kSeg + kWin - 1], v[kSeg + kWin - 1], uu[kSeg + kWin - 1], vv[kSeg + kWin - 1],
            uv[kSeg + kWin - 1];
#pragma unroll
        for (int k = 0; k < kSeg + kWin - 1; ++k) {
            const float2 p = sxy[r][c0 + k];
            u[k] = p.x;
            v[k] = p.y;
            uu[k] = p.x * p.x;
            vv[k] = p.y * p.y;
            uv[k] = p.x * p.y;
        }
#pragma unroll
        for (int o = 0; o < kSeg; ++o) {
            float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float w = win.w[k];
                mx = fmaf(w, u[o + k], mx);
                my = fmaf(w, v[o + k], my);
                xx = fmaf(w, uu[o + k], xx);
                yy = fmaf(w, vv[o + k], yy);
                xy = fmaf(w, uv[o + k], xy);
            }
            h[0][r][c0 + o] = mx;
            h[1][r][c0 + o] = my;
            h[2][r][c0 + o] = xx;
            h[3][r][c0 + o] = yy;
            h[4][r][c0 + o] = xy;
        }
    }
    __syncthreads();
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float l1 = 0.0f, ss = 0.0f;
    // vertical pass: a thread takes kOut consecutive rows of one column,
    // reading their kOut + 10 rows of horizontal sums once
    const int r0 = kOut * ty;
    float m[kOut][5];
#pragma unroll
    for (int o = 0; o < kOut; ++o)
#pragma unroll
        for (int q = 0; q < 5; ++q) m[o][q] = 0.0f;
#pragma unroll
    for (int k = 0; k < kWin + kOut - 1; ++k) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const float hv = h[q][r0 + k][tx];
#pragma unroll
            for (int o = 0; o < kOut; ++o)
                if (k - o >= 0 && k - o < kWin) m[o][q] = fmaf(win.w[k - o], hv, m[o][q]);
        }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const int rr = r0 + o;
        const int x = bp.x0 + tx, y = bp.y0 + rr;
        if (x >= bp.width || y >= bp.height) continue;
        const float mx = m[o][0], my = m[o][1];
        const float vx = m[o][2] - mx * mx, vy = m[o][3] - my * my, cxy = m[o][4] - mx * my;
        const float A = 2.0f * mx * my + C1, B = 2.0f * cxy + C2;
        const float Cd = mx * mx + my * my + C1, D = vx + vy + C2;
        const float iCD = 1.0f / (Cd * D);
        const float s = A * B * iCD;
        // dSSIM/dE[x], dSSIM/dE[x^2], dSSIM/dE[xy] (E[y], E[y^2] held fixed)
        const float ds_dm = (2.0f * my * B - 2.0f * my * A) * iCD - s * (2.0f * mx / Cd - 2.0f * mx / D);
        const float ds_dxx = -s / D;
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
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        const uint32_t ticket = atomicAdd(&ctr->loss_blocks_done, 1u);
        is_last = (ticket == (uint32_t)nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    float acc = 0.0f;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += ((volatile float*)partials)[i];
    const float all = block_sum(acc, red);
    if (threadIdx.x == 0) {
        const float L = lambda * inv_views * (float)vt.n_views + all;
        *loss_dev = L;
        ctr->loss = L;
        ctr->loss_blocks_done = 0u;
    }
}

// Backward: the three maps correlated with the window (two separable passes,
// as the forward), combined per value with x and y, plus the L1 term.
__global__ void __launch_bounds__(kLossThreads)
k_ssim_bwd(ViewTable vt, Win win, const float* __restrict__ img, const float* __restrict__ tgt,
           float lambda, float inv_views, int64_t total_values, const float* __restrict__ maps,
           float* __restrict__ dL) {
    __shared__ float sm[3][kRows][kCols + 1];
    __shared__ float h[3][kRows][kTX + 1];
    const BlockPos bp = block_pos(vt, blockIdx.x);
    {
        float a[kLoads], b[kLoads], d[kLoads];
#pragma unroll
        for (int it = 0; it < kLoads; ++it) {
            const int i = threadIdx.x + it * kLossThreads;
            const int r = i / kCols, c = i - r * kCols;
            const int y = bp.y0 - kHalo + r, x = bp.x0 - kHalo + c;
            a[it] = b[it] = d[it] = 0.0f;
            if (i < kRows * kCols && x >= 0 && x < bp.width && y >= 0 && y < bp.height) {
                const int64_t idx = bp.plane + (int64_t)y * bp.width + x;
                a[it] = maps[idx];
                b[it] = maps[total_values + idx];
                d[it] = maps[2 * total_values + idx];
            }
        }
#pragma unroll
        for (int it = 0; it < kLoads; ++it) {
            const int i = threadIdx.x + it * kLossThreads;
            if (i < kRows * kCols) {
                const int r = i / kCols, c = i - r * kCols;
                sm[0][r][c] = a[it];
                sm[1][r][c] = b[it];
                sm[2][r][c] = d[it];
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRows * (kTX / kSeg); i += blockDim.x) {
        const int r = i / (kTX / kSeg), c0 = (i - r * (kTX / kSeg)) * kSeg;
        float u[3][kSeg + kWin - 1];
#pragma unroll
        for (int k = 0; k < kSeg + kWin - 1; ++k) {
            u[0][k] = sm[0][r][c0 + k];
            u[1][k] = sm[1][r][c0 + k];
            u[2][k] = sm[2][r][c0 + k];
        }
#pragma unroll
        for (int o = 0; o < kSeg; ++o) {
            float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float w = win.w[k];
                a = fmaf(w, u[0][o + k], a);
                b = fmaf(w, u[1][o + k], b);
                d = fmaf(w, u[2][o + k], d);
            }
            h[0][r][c0 + o] = a;
            h[1][r][c0 + o] = b;
            h[2][r][c0 + o] = d;
        }
    }
    __syncthreads();
    const ViewGeom& g = vt.v[bp.view];
    const float scale = inv_views / ((float)g.channels * (float)g.width * (float)g.height);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r0 = kOut * ty;
    float m[kOut][3];
#pragma unroll
    for (int o = 0; o < kOut; ++o)
#pragma unroll
        for (int q = 0; q < 3; ++q) m[o][q] = 0.0f;
#pragma unroll
    for (int k = 0; k < kWin + kOut - 1; ++k) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float hv = h[q][r0 + k][tx];
#pragma unroll
            for (int o = 0; o < kOut; ++o)
                if (k - o >= 0 && k - o < kWin) m[o][q] = fmaf(win.w[k - o], hv, m[o][q]);
        }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const int x = bp.x0 + tx, y = bp.y0 + r0 + o;
        if (x >= bp.width || y >= bp.height) continue;
        const int64_t idx = bp.plane + (int64_t)y * bp.width + x;
        const float xv = img[idx], yv = tgt[idx];
        const float diff = xv - yv;
        const float sgn = diff > 0.0f ? 1.0f : (diff < 0.0f ? -1.0f : 0.0f);
        const float dssim = m[o][0] + 2.0f * xv * m[o][1] + yv * m[o][2];
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
    k_ssim_fwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        inv_views, p->total_values, maps,
                                                        partials, p->loss_blocks, ctr, loss_dev);
    k_ssim_bwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        inv_views, p->total_values, maps, dL);
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

// Scratch of gs_loss_l1_ssim_noalloc: counters (ticket of the loss reduction)
// | per-block loss partials | the three SSIM partial-derivative maps.  About
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
    // the array keeps whatever the last call left: the ticket must start at zero
    if (cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st) != cudaSuccess) return GS_ERR_CUDA;
    const Win win = loss_window();
    k_ssim_fwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        view_weight, p->total_values, maps,
                                                        partials, p->loss_blocks, ctr, loss_dev);
    k_ssim_bwd<<<p->loss_blocks, kLossThreads, 0, st>>>(p->vt, win, images, targets, lambda,
                                                        view_weight, p->total_values, maps,
                                                        dL_dimages);
    return launch_status();
}
