// gs_pyramid.cu -- one level of the Gaussian pyramid of a target image
// (paper Sec. III-B: the keyframe image is smoothed and down-sampled
// repeatedly, and training moves from the coarsest level to finer ones).
//
// Output pixel (r, c) of each channel plane is the 5x5 binomial
// ([1, 4, 6, 4, 1] / 16 along each axis) weighted sum around input pixel
// (2r, 2c), borders mirrored without repeating the edge pixel; the output
// is ceil(H/2) x ceil(W/2).  One thread per output value; the five row sums
// are formed first, then combined (separable order).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kPyrThreads = 256;

__device__ __forceinline__ int mirror(int i, int n) {
    if (n == 1) return 0;
    i = i < 0 ? -i : i;
    return i >= n ? 2 * n - 2 - i : i;
}

__global__ void __launch_bounds__(kPyrThreads)
k_pyr_down(const float* __restrict__ src, int C, int H, int W, float* __restrict__ dst, int Ho,
           int Wo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)C * Ho * Wo;
    if (idx >= total) return;
    const int c = (int)(idx % Wo);
    const long long t = idx / Wo;
    const int r = (int)(t % Ho);
    const int ch = (int)(t / Ho);
    const float w[5] = {1.0f / 16, 4.0f / 16, 6.0f / 16, 4.0f / 16, 1.0f / 16};
    const float* plane = src + (size_t)ch * H * W;
    int xs[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) xs[b] = mirror(2 * c + b - 2, W);
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        const float* row = plane + (size_t)mirror(2 * r + a - 2, H) * W;
        float h = 0.0f;
#pragma unroll
        for (int b = 0; b < 5; ++b) h = fmaf(w[b], row[xs[b]], h);
        acc = fmaf(w[a], h, acc);
    }
    dst[idx] = acc;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_pyr_down(const float* src, int32_t channels, int32_t height,
                                 int32_t width, float* dst, void* stream) {
    using namespace gs;
    if (!src || !dst || channels < 1 || height < 1 || width < 1) return GS_ERR_INVALID;
    const int Ho = (height + 1) / 2, Wo = (width + 1) / 2;
    const long long total = (long long)channels * Ho * Wo;
    const long long blocks = (total + kPyrThreads - 1) / kPyrThreads;
    if (blocks > 0x7fffffffLL) return GS_ERR_UNSUPPORTED;
    k_pyr_down<<<(unsigned)blocks, kPyrThreads, 0, (cudaStream_t)stream>>>(
        src, channels, height, width, dst, Ho, Wo);
    return launch_status();
}
