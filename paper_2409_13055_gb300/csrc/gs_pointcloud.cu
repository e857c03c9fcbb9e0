// gs_pointcloud.cu -- point-cloud densification on the GPU (paper Sec.
// III-A): DSO-style pixel selection and the mean-depth interpolation of flat
// pixels inside the Delaunay triangles of the tracked pixels (the
// triangulation itself is built on the host, gs_delaunay.cu).
//
//   k_grad_sq      squared central-difference gradient, zero on the border;
//   k_select_pass  one pass of the selection: a thread per block of
//                  block * 2^k pixels takes the first pixel of largest
//                  squared gradient, if the block holds no earlier selection
//                  and the pixel reaches the pass threshold;
//   k_tri_claim    a thread per triangle marks the grid pixels its closed
//                  triangle contains (integer edge functions) with atomicMin
//                  of its index, so the lowest-index triangle owns shared
//                  edges whatever the scheduling;
//   k_interp       each owned flat, unselected grid pixel gets the mean of its
//                  triangle's vertex depths.
#include "gs_internal.cuh"

namespace gs {
namespace {

__global__ void k_grad_sq(const float* __restrict__ gray, int H, int W, float* __restrict__ g2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    float v = 0.0f;
    if (x > 0 && x < W - 1 && y > 0 && y < H - 1) {
        const float gx = 0.5f * (gray[(size_t)y * W + x + 1] - gray[(size_t)y * W + x - 1]);
        const float gy = 0.5f * (gray[(size_t)(y + 1) * W + x] - gray[(size_t)(y - 1) * W + x]);
        v = fmaf(gx, gx, gy * gy);
    }
    g2[(size_t)y * W + x] = v;
}

__global__ void k_select_pass(const float* __restrict__ g2, int H, int W, int s, float thr,
                              int pass, int32_t* __restrict__ sel) {
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    const int x0 = bx * s, y0 = by * s;
    if (x0 >= W) return;
    const int x1 = min(x0 + s, W), y1 = min(y0 + s, H);
    float best = -1.0f;
    int bi = -1;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            const size_t i = (size_t)y * W + x;
            if (sel[i] != 0) return;  // an earlier pass chose a pixel here
            const float v = g2[i];
            if (v > best) {
                best = v;
                bi = (int)i;
            }
        }
    if (bi >= 0 && best >= thr) sel[bi] = pass + 1;
}

__global__ void k_tri_claim(const int32_t* __restrict__ tri, int n_tri,
                            const int32_t* __restrict__ xy, int H, int W, int grid,
                            int32_t* __restrict__ owner) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tri) return;
    const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    const long long ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1],
                    cx = xy[2 * c], cy = xy[2 * c + 1];
    const long long lox = min(ax, min(bx, cx)), hix = max(ax, max(bx, cx));
    const long long loy = min(ay, min(by, cy)), hiy = max(ay, max(by, cy));
    const int gw = (W + grid - 1) / grid, gh = (H + grid - 1) / grid;
    const int gx0 = (int)max(0LL, (lox + grid - 1) / grid), gx1 = (int)min((long long)gw - 1, hix / grid);
    const int gy0 = (int)max(0LL, (loy + grid - 1) / grid), gy1 = (int)min((long long)gh - 1, hiy / grid);
    for (int gy = gy0; gy <= gy1; ++gy)
        for (int gx = gx0; gx <= gx1; ++gx) {
            const long long x = (long long)gx * grid, y = (long long)gy * grid;
            const long long e0 = (bx - ax) * (y - ay) - (by - ay) * (x - ax);
            const long long e1 = (cx - bx) * (y - by) - (cy - by) * (x - bx);
            const long long e2 = (ax - cx) * (y - cy) - (ay - cy) * (x - cx);
            if (e0 >= 0 && e1 >= 0 && e2 >= 0) atomicMin(owner + (size_t)gy * gw + gx, t);
        }
}

__global__ void k_interp(const int32_t* __restrict__ tri, const float* __restrict__ depth,
                         const float* __restrict__ g2, const int32_t* __restrict__ sel, int H,
                         int W, int grid, float flat_sq, const int32_t* __restrict__ owner,
                         float* __restrict__ out) {
    const int gw = (W + grid - 1) / grid, gh = (H + grid - 1) / grid;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= gw || gy >= gh) return;
    const size_t o = (size_t)gy * gw + gx;
    const size_t p = (size_t)gy * grid * W + (size_t)gx * grid;
    const int t = owner[o];
    float d = 0.0f;
    if (t != 0x7fffffff && sel[p] == 0 && g2[p] < flat_sq)
        d = (depth[tri[3 * t]] + depth[tri[3 * t + 1]] + depth[tri[3 * t + 2]]) / 3.0f;
    out[o] = d;
}

__global__ void k_fill_i32(int32_t* __restrict__ a, size_t n, int32_t v) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_select_pixels(const float* gray, int32_t height, int32_t width,
                                      int32_t block, int32_t passes,
                                      const float* threshold_sq_host, float* grad_sq,
                                      int32_t* selected, void* stream) {
    if (!gray || !grad_sq || !selected || !threshold_sq_host || height < 1 || width < 1 ||
        block < 1 || passes < 1 || passes > 8 || (block << (passes - 1)) > (1 << 16))
        return GS_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    k_grad_sq<<<dim3((width + 255) / 256, height), 256, 0, st>>>(gray, height, width, grad_sq);
    if (cudaMemsetAsync(selected, 0, (size_t)height * width * sizeof(int32_t), st) != cudaSuccess)
        return GS_ERR_CUDA;
    for (int k = 0; k < passes; ++k) {
        const int s = block << k;
        const int nbx = (width + s - 1) / s, nby = (height + s - 1) / s;
        k_select_pass<<<dim3((nbx + 127) / 128, nby), 128, 0, st>>>(
            grad_sq, height, width, s, threshold_sq_host[k], k, selected);
    }
    return launch_status();
}

extern "C" gs_status gs_interp_depth(const int32_t* tri, int32_t n_tri, const int32_t* xy,
                                     const float* depth, const float* grad_sq,
                                     const int32_t* selected, int32_t height, int32_t width,
                                     int32_t grid, float flat_sq, int32_t* owner, float* out,
                                     void* stream) {
    if ((n_tri > 0 && (!tri || !xy || !depth)) || !grad_sq || !selected || !owner || !out ||
        n_tri < 0 || height < 1 || width < 1 || grid < 1)
        return GS_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int gw = (width + grid - 1) / grid, gh = (height + grid - 1) / grid;
    const size_t cells = (size_t)gw * gh;
    k_fill_i32<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(owner, cells, 0x7fffffff);
    if (n_tri > 0)
        k_tri_claim<<<(n_tri + 127) / 128, 128, 0, st>>>(tri, n_tri, xy, height, width, grid,
                                                          owner);
    k_interp<<<dim3((gw + 127) / 128, gh), 128, 0, st>>>(tri, depth, grad_sq, selected, height,
                                                         width, grid, flat_sq, owner, out);
    return launch_status();
}
