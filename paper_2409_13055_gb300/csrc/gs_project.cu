// gs_project.cu -- A1 projection and A8 projection adjoint.
//
// Projection follows the original 3DGS rasteriser the method renders with
// (paper Sec. III-B) and the projection step of Sec. II: per (view,
// Gaussian) the camera transform, EWA splatting of the 3D covariance into a
// dilated 2D covariance and its conic, a 3-sigma square extent and tile rect,
// a spherical-harmonics colour and a sigmoid opacity.
//
// GB300 layout decisions:
//  * one thread per Gaussian and per group of up to 4 views: the Gaussian's
//    parameters and its 3D covariance are loaded/computed once and reused for
//    every view of the group, so a 16-view batch reads the map 4 times, not 16;
//  * the camera transform, the perspective divide and the projected mean are
//    carried as float pairs (error-free transformations), so the projected
//    mean is exact to ~1e-12 relative and the FP32 depth key is the correctly
//    rounded depth; the renderers then evaluate every Gaussian in tile-local
//    coordinates, where FP32 keeps ~1e-6 px;
//  * the SH coefficients are stored coefficient-major ([K][N][3]), so each
//    coefficient plane is read by a warp as one contiguous 384-byte run.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kProjThreads = 256;
constexpr int kViewsPerThread = 4;

// Real spherical harmonics with the Condon-Shortley phase, degrees 0..3,
// ordered m = -l..l, as polynomials of a unit direction.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.4886025119029199f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.5462742152960396f;
constexpr float kY3a = 0.5900435899266435f;
constexpr float kY3b = 2.890611442640554f;
constexpr float kY3c = 0.4570457994644658f;
constexpr float kY3d = 0.3731763325901154f;
constexpr float kY3e = 1.445305721320277f;

// Every product and sum is an explicitly rounded intrinsic, so no FMA
// contraction is left to the compiler: the basis comes out bit-identical in
// every kernel that evaluates it (the fused and the two-pass adjoints form
// the SH gradient from it independently).
__device__ __forceinline__ void sh_eval(int degree, float x, float y, float z, float* Y) {
    Y[0] = kY0;
    if (degree < 1) return;
    Y[1] = __fmul_rn(-kY1, y);
    Y[2] = __fmul_rn(kY1, z);
    Y[3] = __fmul_rn(-kY1, x);
    if (degree < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xmy = __fsub_rn(xx, yy);                       // x^2 - y^2
    const float t2 = __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), xx), yy);  // 2z^2 - x^2 - y^2
    Y[4] = __fmul_rn(__fmul_rn(kY2a, x), y);
    Y[5] = __fmul_rn(__fmul_rn(-kY2a, y), z);
    Y[6] = __fmul_rn(kY2b, t2);
    Y[7] = __fmul_rn(__fmul_rn(-kY2a, x), z);
    Y[8] = __fmul_rn(kY2c, xmy);
    if (degree < 3) return;
    const float t4 = __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy);  // 4z^2 - x^2 - y^2
    Y[9] = __fmul_rn(__fmul_rn(-kY3a, y), __fsub_rn(__fmul_rn(3.0f, xx), yy));
    Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(kY3b, x), y), z);
    Y[11] = __fmul_rn(__fmul_rn(-kY3c, y), t4);
    Y[12] = __fmul_rn(__fmul_rn(kY3d, z),
                      __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), __fmul_rn(3.0f, xx)),
                                __fmul_rn(3.0f, yy)));
    Y[13] = __fmul_rn(__fmul_rn(-kY3c, x), t4);
    Y[14] = __fmul_rn(__fmul_rn(kY3e, z), xmy);
    Y[15] = __fmul_rn(__fmul_rn(-kY3a, x), __fsub_rn(xx, __fmul_rn(3.0f, yy)));
}

// d/d(x,y,z) of the polynomials above, accumulated as g += w * grad Y_k.
__device__ __forceinline__ void sh_grad_acc(int degree, float x, float y, float z,
                                            const float* w, float& gx, float& gy, float& gz) {
    if (degree < 1) return;
    gx += -kY1 * w[3];
    gy += -kY1 * w[1];
    gz += kY1 * w[2];
    if (degree < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += kY2a * y * w[4] - kY2a * z * w[7] - 2.0f * kY2b * x * w[6] + 2.0f * kY2c * x * w[8];
    gy += kY2a * x * w[4] - kY2a * z * w[5] - 2.0f * kY2b * y * w[6] - 2.0f * kY2c * y * w[8];
    gz += -kY2a * y * w[5] - kY2a * x * w[7] + 4.0f * kY2b * z * w[6];
    if (degree < 3) return;
    gx += -kY3a * 6.0f * x * y * w[9] + kY3b * y * z * w[10] + kY3c * 2.0f * x * y * w[11] -
          kY3d * 6.0f * x * z * w[12] - kY3c * (4.0f * zz - 3.0f * xx - yy) * w[13] +
          kY3e * 2.0f * x * z * w[14] - kY3a * (3.0f * xx - 3.0f * yy) * w[15];
    gy += -kY3a * (3.0f * xx - 3.0f * yy) * w[9] + kY3b * x * z * w[10] -
          kY3c * (4.0f * zz - xx - 3.0f * yy) * w[11] - kY3d * 6.0f * y * z * w[12] +
          kY3c * 2.0f * x * y * w[13] - kY3e * 2.0f * y * z * w[14] + kY3a * 6.0f * x * y * w[15];
    gz += kY3b * x * y * w[10] - kY3c * 8.0f * y * z * w[11] +
          kY3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12] - kY3c * 8.0f * x * z * w[13] +
          kY3e * (xx - yy) * w[14];
}

struct Cam {
    float R[9], t[3], fx, fy, cx, cy, cc[3];
    float ulo, uhi, vlo, vhi;
    int width, height;
};

__device__ void load_cam(const gs_view& vw, Cam& c) {
    for (int k = 0; k < 9; ++k) c.R[k] = vw.R[k];
    for (int k = 0; k < 3; ++k) c.t[k] = vw.t[k];
    c.fx = vw.fx;
    c.fy = vw.fy;
    c.cx = vw.cx;
    c.cy = vw.cy;
    // camera centre -R^T t
    for (int k = 0; k < 3; ++k)
        c.cc[k] = -(c.R[k] * c.t[0] + c.R[3 + k] * c.t[1] + c.R[6 + k] * c.t[2]);
    c.width = vw.width;
    c.height = vw.height;
    // Jacobian clamp: x/z in [-1.3 cx/fx, 1.3 (W - cx)/fx], same for y.
    c.ulo = -1.3f * c.cx / c.fx;
    c.uhi = 1.3f * ((float)vw.width - c.cx) / c.fx;
    c.vlo = -1.3f * c.cy / c.fy;
    c.vhi = 1.3f * ((float)vw.height - c.cy) / c.fy;
}

// View-independent part of a Gaussian: normalised rotation, scales, 3D covariance.
struct Shape {
    float qn[4], qnorm, Rq[9], s[3];
    float sig[6];  // 00 01 02 11 12 22
    bool finite;
};

__device__ __forceinline__ void make_shape(const float* ls, const float* q4, Shape& sh) {
    float w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    float nn = w * w + x * x + y * y + z * z;
    sh.finite = isfinite(nn) && nn > 0.0f && isfinite(ls[0]) && isfinite(ls[1]) &&
                isfinite(ls[2]);
    sh.qnorm = sqrtf(nn);
    float inv = 1.0f / sh.qnorm;
    w *= inv; x *= inv; y *= inv; z *= inv;
    sh.qn[0] = w; sh.qn[1] = x; sh.qn[2] = y; sh.qn[3] = z;
    float* R = sh.Rq;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    for (int k = 0; k < 3; ++k) sh.s[k] = expf(ls[k]);
    // Sigma = M M^T, M = Rq diag(s)
    float M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * sh.s[c];
    auto dot = [&](int a, int b) {
        return M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
    };
    sh.sig[0] = dot(0, 0); sh.sig[1] = dot(0, 1); sh.sig[2] = dot(0, 2);
    sh.sig[3] = dot(1, 1); sh.sig[4] = dot(1, 2); sh.sig[5] = dot(2, 2);
}

// Per-view projection of one Gaussian.
struct Proj {
    bool visible;
    float xc[3];              // camera-space mean (hi parts)
    float mxh, myh, mxl, myl; // projected mean as float pairs
    float u, v;               // clamped x/z, y/z
    bool uc, vc;              // clamp engaged
    float T[6];               // J W, row-major 2x3
    float a, b, c;            // dilated 2D covariance
    float det, ca, cb, cc;    // conic
    int radius;
    int rect[4];
    float dir[3], dist;
};

// Adam state for the fused projection adjoint: parameter, moment and optional
// gradient arrays in the gs_map layout; lr per group (means, log-scales,
// quaternions, opacity, SH DC, SH rest).
struct FusedAdam {
    float lr[6];
    float b1, b2, eps;
    const int32_t* step;
    float *p_means, *p_ls, *p_quats, *p_logit, *p_sh;
    float *m_means, *m_ls, *m_quats, *m_logit, *m_sh;
    float *v_means, *v_ls, *v_quats, *v_logit, *v_sh;
    const float *a_means, *a_ls, *a_quats, *a_logit, *a_sh;  // gradients to add, or null
    float *o_means, *o_ls, *o_quats, *o_logit, *o_sh;        // gradients out, or null
};

// Opacity below which no pixel can reach alpha >= 1/255 (alpha <= opacity),
// with a 0.1% margin: such a Gaussian gets no tile under tight rects.
constexpr float kTightMinOpacity = 0.999f / 255.0f;

__device__ __forceinline__ void project_one(const float* mean, const Shape& sh, const Cam& cam,
                                            float near_z, int log2_tw, int log2_th, int tiles_x,
                                            int tiles_y, float opacity, int tight, Proj& p) {
    p.visible = false;
    float xh, xl, yh, yl, zh, zl;
    dot3_plus(cam.R[0], cam.R[1], cam.R[2], mean[0], mean[1], mean[2], cam.t[0], xh, xl);
    dot3_plus(cam.R[3], cam.R[4], cam.R[5], mean[0], mean[1], mean[2], cam.t[1], yh, yl);
    dot3_plus(cam.R[6], cam.R[7], cam.R[8], mean[0], mean[1], mean[2], cam.t[2], zh, zl);
    p.xc[0] = xh; p.xc[1] = yh; p.xc[2] = zh;
    if (!(isfinite(xh) && isfinite(yh) && isfinite(zh)) || !sh.finite) return;
    if (!(zh > near_z)) return;
    float uh, ul, vh, vl;
    df_div(xh, xl, zh, zl, uh, ul);
    df_div(yh, yl, zh, zl, vh, vl);
    df_affine(cam.fx, uh, ul, cam.cx, p.mxh, p.mxl);
    df_affine(cam.fy, vh, vl, cam.cy, p.myh, p.myl);

    p.u = fminf(fmaxf(uh, cam.ulo), cam.uhi);
    p.v = fminf(fmaxf(vh, cam.vlo), cam.vhi);
    p.uc = (uh < cam.ulo) || (uh > cam.uhi);
    p.vc = (vh < cam.vlo) || (vh > cam.vhi);
    const float iz = 1.0f / zh;
    const float J00 = cam.fx * iz, J02 = -cam.fx * p.u * iz;
    const float J11 = cam.fy * iz, J12 = -cam.fy * p.v * iz;
    const float* W = cam.R;
    for (int k = 0; k < 3; ++k) {
        p.T[k] = J00 * W[k] + J02 * W[6 + k];
        p.T[3 + k] = J11 * W[3 + k] + J12 * W[6 + k];
    }
    const float* S = sh.sig;
    // Sigma T0^T and Sigma T1^T
    float s0[3], s1[3];
    s0[0] = S[0] * p.T[0] + S[1] * p.T[1] + S[2] * p.T[2];
    s0[1] = S[1] * p.T[0] + S[3] * p.T[1] + S[4] * p.T[2];
    s0[2] = S[2] * p.T[0] + S[4] * p.T[1] + S[5] * p.T[2];
    s1[0] = S[0] * p.T[3] + S[1] * p.T[4] + S[2] * p.T[5];
    s1[1] = S[1] * p.T[3] + S[3] * p.T[4] + S[4] * p.T[5];
    s1[2] = S[2] * p.T[3] + S[4] * p.T[4] + S[5] * p.T[5];
    p.a = p.T[0] * s0[0] + p.T[1] * s0[1] + p.T[2] * s0[2] + 0.3f;
    p.b = p.T[3] * s0[0] + p.T[4] * s0[1] + p.T[5] * s0[2];
    p.c = p.T[3] * s1[0] + p.T[4] * s1[1] + p.T[5] * s1[2] + 0.3f;
    // det = a c - b^2 with Kahan's fma-compensated 2x2 determinant
    const float w = __fmul_rn(p.b, p.b);
    const float e = __fmaf_rn(-p.b, p.b, w);
    const float f = __fmaf_rn(p.a, p.c, -w);
    p.det = __fadd_rn(f, e);
    if (!(p.det > 0.0f)) return;
    const float idet = 1.0f / p.det;
    p.ca = p.c * idet;
    p.cb = -p.b * idet;
    p.cc = p.a * idet;
    const float mid = 0.5f * (p.a + p.c);
    const float lam = mid + sqrtf(fmaxf(0.0f, mid * mid - p.det));
    p.radius = (int)ceilf(3.0f * sqrtf(lam));
    const float rr = (float)p.radius;
    const float itw = 1.0f / (float)(1 << log2_tw), ith = 1.0f / (float)(1 << log2_th);
    const float tw1 = (float)((1 << log2_tw) - 1), th1 = (float)((1 << log2_th) - 1);
    float sh_, sl;
    float e2;
    two_sum(p.mxh, -rr, sh_, e2);
    fast_two_sum(sh_, __fadd_rn(e2, p.mxl), sh_, sl);
    int x0 = df_floor_div(sh_, sl, itw);
    two_sum(p.myh, -rr, sh_, e2);
    fast_two_sum(sh_, __fadd_rn(e2, p.myl), sh_, sl);
    int y0 = df_floor_div(sh_, sl, ith);
    two_sum(p.mxh, rr + tw1, sh_, e2);
    fast_two_sum(sh_, __fadd_rn(e2, p.mxl), sh_, sl);
    int x1 = df_floor_div(sh_, sl, itw);
    two_sum(p.myh, rr + th1, sh_, e2);
    fast_two_sum(sh_, __fadd_rn(e2, p.myl), sh_, sl);
    int y1 = df_floor_div(sh_, sl, ith);
    p.rect[0] = min(max(x0, 0), tiles_x);
    p.rect[1] = min(max(y0, 0), tiles_y);
    p.rect[2] = min(max(x1, 0), tiles_x);
    p.rect[3] = min(max(y1, 0), tiles_y);
    if (tight) {
        // Cut to the tiles meeting the box of the ellipse q <= 1.01 t + 0.01,
        // t = 2 ln(255 o): outside it o exp(-q/2) < 1/255 with a margin no
        // FP32 evaluation of alpha can cross.  Tile k holds pixels
        // k T .. k T + T - 1, so tiles [ceil((mu - h - T + 1) / T),
        // floor((mu + h) / T)] meet [mu - h, mu + h].
        if (!(opacity >= kTightMinOpacity)) return;
        const float t = tight_level(opacity);
        const float hx = sqrtf(t * p.a), hy = sqrtf(t * p.c);
        two_sum(p.mxh, -(hx + tw1), sh_, e2);
        fast_two_sum(sh_, __fadd_rn(e2, p.mxl), sh_, sl);
        const int lx = -df_floor_div(-sh_, -sl, itw);  // ceil
        two_sum(p.myh, -(hy + th1), sh_, e2);
        fast_two_sum(sh_, __fadd_rn(e2, p.myl), sh_, sl);
        const int ly = -df_floor_div(-sh_, -sl, ith);
        two_sum(p.mxh, hx, sh_, e2);
        fast_two_sum(sh_, __fadd_rn(e2, p.mxl), sh_, sl);
        const int ux = df_floor_div(sh_, sl, itw) + 1;
        two_sum(p.myh, hy, sh_, e2);
        fast_two_sum(sh_, __fadd_rn(e2, p.myl), sh_, sl);
        const int uy = df_floor_div(sh_, sl, ith) + 1;
        p.rect[0] = max(p.rect[0], min(lx, tiles_x));
        p.rect[1] = max(p.rect[1], min(ly, tiles_y));
        p.rect[2] = min(p.rect[2], max(ux, 0));
        p.rect[3] = min(p.rect[3], max(uy, 0));
        if (p.rect[2] <= p.rect[0] || p.rect[3] <= p.rect[1]) return;
    }
    if ((p.rect[2] - p.rect[0]) * (p.rect[3] - p.rect[1]) <= 0) return;
    float d0 = mean[0] - cam.cc[0], d1 = mean[1] - cam.cc[1], d2 = mean[2] - cam.cc[2];
    p.dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float idist = p.dist > 0.0f ? 1.0f / p.dist : 0.0f;
    p.dir[0] = d0 * idist; p.dir[1] = d1 * idist; p.dir[2] = d2 * idist;
    p.visible = true;
}

// Ask the L2 for the cache lines of Gaussian g's K SH coefficients
// (coefficient-major, three floats each), so that the loads that come after
// the long arithmetic before them find them there.
template <int K>
__device__ __forceinline__ void prefetch_sh(const float* __restrict__ sh, int n, int g) {
#pragma unroll
    for (int k = 0; k < K; ++k)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(sh + ((size_t)k * n + g) * 3));
}

// ... and the lines of Gaussian g's mean, log-scales, quaternion and opacity
// logit.
__device__ __forceinline__ void prefetch_params(const float* __restrict__ means,
                                                const float* __restrict__ log_scales,
                                                const float* __restrict__ quats,
                                                const float* __restrict__ opacity_logits, int g) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(means + 3 * (size_t)g));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(log_scales + 3 * (size_t)g));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(quats + 4 * (size_t)g));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(opacity_logits + g));
}

template <int DEG>
__global__ void __launch_bounds__(kProjThreads, 4)
k_project(const float* __restrict__ means, const float* __restrict__ log_scales,
          const float* __restrict__ quats, const float* __restrict__ opacity_logits,
          const float* __restrict__ sh, int n, const gs_view* __restrict__ views,
          ViewTable vt, float near_z, float4* __restrict__ rec, uint16_t* __restrict__ rect_out,
          uint32_t* __restrict__ touched, int32_t* __restrict__ radius_out,
          uint32_t* __restrict__ dkey, DevCounters* counters,
          uint32_t* __restrict__ spans, uint32_t* __restrict__ pool, uint32_t pool_rows) {
    __shared__ Cam cams[kViewsPerThread];
    const int v0 = blockIdx.y * kViewsPerThread;
    const int nv = min(kViewsPerThread, vt.n_views - v0);
    if (threadIdx.x < nv) load_cam(views[v0 + threadIdx.x], cams[threadIdx.x]);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    // the map is streamed once per projection: evict-first loads, so that
    // the records written here stay in the L2 for the render kernels
    const float mean[3] = {__ldcs(means + 3 * g), __ldcs(means + 3 * g + 1),
                           __ldcs(means + 3 * g + 2)};
    const float ls[3] = {__ldcs(log_scales + 3 * g), __ldcs(log_scales + 3 * g + 1),
                         __ldcs(log_scales + 3 * g + 2)};
    const float4 q = __ldcs(reinterpret_cast<const float4*>(quats) + g);
    const float q4[4] = {q.x, q.y, q.z, q.w};
    Shape shp;
    make_shape(ls, q4, shp);
    const float logit = __ldcs(opacity_logits + g);
    const bool finite = shp.finite && isfinite(logit) && isfinite(mean[0]) &&
                        isfinite(mean[1]) && isfinite(mean[2]);
    if (!finite && v0 == 0) atomicOr(&counters->status, (uint32_t)GS_DEV_NONFINITE);
    const float opacity = 1.0f / (1.0f + expf(-logit));
    constexpr int K = (DEG + 1) * (DEG + 1);
    for (int j = 0; j < nv; ++j) {
        const int v = v0 + j;
        const size_t vg = (size_t)v * n + g;
        const ViewGeom& geo = vt.v[v];
        Proj p;
        project_one(mean, shp, cams[j], near_z, vt.log2_tw, vt.log2_th, geo.tiles_x,
                    geo.tiles_y, opacity, vt.tight_rect, p);
        bool vis = finite && p.visible;
        uint32_t area = 0u;
        if (vis) {
            prefetch_sh<K>(sh, n, g);
            area = (uint32_t)((p.rect[2] - p.rect[0]) * (p.rect[3] - p.rect[1]));
            if (vt.tight_rect) {
                // the row spans of the box, stored for the emission: in the
                // Gaussian's slots, or, for a tall box, in rows of the pool
                const int rows = p.rect[3] - p.rect[1];
                uint32_t* sp = spans + vg * kSpanRows;
                uint32_t* dst = sp;
                if (rows > kSpanRows) {
                    uint32_t base = kSpanNoPool;
                    if (counters->span_pool_used < pool_rows) {
                        base = atomicAdd(&counters->span_pool_used, (uint32_t)rows);
                        if ((uint64_t)base + (uint64_t)rows > (uint64_t)pool_rows)
                            base = kSpanNoPool;
                    }
                    sp[0] = base;
                    if (base == kSpanNoPool) {
                        atomicOr(&counters->status, (uint32_t)GS_DEV_SPAN_POOL);
                        dst = nullptr;  // the box keeps all its tiles
                    } else {
                        dst = pool + base;
                    }
                }
                if (dst) {
                    const TightEllipse E =
                        tight_ellipse(p.mxh, p.mxl, p.myh, p.myl, p.ca, p.cb, p.cc, opacity);
                    int a0, a1;
                    area = 0u;
                    for (int ty = p.rect[1]; ty < p.rect[3]; ++ty) {
                        area += (uint32_t)tight_row_span(E, ty, vt.log2_tw, vt.log2_th,
                                                         p.rect[0], p.rect[2], &a0, &a1);
                        dst[ty - p.rect[1]] = (uint32_t)a0 | ((uint32_t)a1 << 16);
                    }
                    vis = area > 0u;
                }
            }
        }
        if (!vis) {
            touched[vg] = 0u;
            dkey[vg] = 0xFFFFFFFFu;
            radius_out[vg] = 0;
            reinterpret_cast<uint2*>(rect_out)[vg] = make_uint2(0u, 0u);
            continue;
        }
        float Y[16];
        sh_eval(DEG, p.dir[0], p.dir[1], p.dir[2], Y);
        float col[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* c = sh + ((size_t)k * n + g) * 3;
            col[0] = fmaf(Y[k], __ldcs(c), col[0]);
            col[1] = fmaf(Y[k], __ldcs(c + 1), col[1]);
            col[2] = fmaf(Y[k], __ldcs(c + 2), col[2]);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(col[ch] + 0.5f, 0.0f);
        float4* r = rec + vg * 3;
        r[0] = make_float4(p.mxh, p.myh, p.mxl, p.myl);
        r[1] = make_float4(p.ca, p.cb, p.cc, opacity);
        r[2] = make_float4(col[0], col[1], col[2], p.xc[2]);
        touched[vg] = area;
        dkey[vg] = __float_as_uint(p.xc[2]);
        radius_out[vg] = p.radius;
        uint2 rc;
        rc.x = (uint32_t)p.rect[0] | ((uint32_t)p.rect[1] << 16);
        rc.y = (uint32_t)p.rect[2] | ((uint32_t)p.rect[3] << 16);
        reinterpret_cast<uint2*>(rect_out)[vg] = rc;
    }
}

// Whether any Gaussian of this warp's group of 32 touches a tile in any view
// (a warp-wide vote; every lane of the warp must call it).  Lane 0 records the
// answer in group_vis[g / 32] when given.
__device__ __forceinline__ bool group_touched(int g, int n, int n_views,
                                              const uint32_t* __restrict__ touched,
                                              uint8_t* __restrict__ group_vis) {
    bool mine = false;
    if (g < n)
        for (int v = 0; v < n_views; ++v) mine |= touched[(size_t)v * n + g] != 0u;
    const bool any = __any_sync(0xffffffffu, mine);
    if (group_vis && (threadIdx.x & 31) == 0 && g < n) group_vis[g >> 5] = any ? 1 : 0;
    return any;
}

// A8: chain rule of the projection for Gaussian g, summed over the views it
// is visible in: screen-space gradient -> gradients of the mean, log-scales,
// quaternion and opacity logit.  The colour gradient that reaches the SH
// coefficients (zero on clamped channels, a grayscale view's gradient spread
// over the three channels) goes, by MODE:
//   kShViaGcol  to gcol_out per (view, Gaussian), for k_sh_bwd;
//   kShStaged   into this Gaussian's SH gradient at once, sh_acc[k * sh_stride
//               + c] += Y_k(dir) gcol[c] view by view in view order (the sum
//               k_sh_bwd forms), sh_acc in shared memory;
//   kShDirect   (one view only) straight to the SH gradient array, sh_acc =
//               its row of this Gaussian, sh_stride = 3 n: Y_k(dir) gcol[c],
//               rounded as k_sh_bwd rounds it, written or (accumulate) added.
constexpr int kShViaGcol = 0, kShStaged = 1, kShDirect = 2;

template <int DEG, int MODE>
__device__ __forceinline__ void adjoint_one(
    int g, const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ opacity_logits,
    const float* __restrict__ sh, int n, const Cam* cam_all, const ViewTable& vt, float near_z,
    const uint32_t* __restrict__ touched, const float* __restrict__ grad2d,
    float* __restrict__ gcol_out, float* sh_acc, size_t sh_stride, int accumulate,
    float gm_out[3], float gls[3], float4& gq4, float& glog) {
    const float mean[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    const float ls[3] = {log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]};
    const float4 q = reinterpret_cast<const float4*>(quats)[g];
    const float q4[4] = {q.x, q.y, q.z, q.w};
    Shape shp;
    make_shape(ls, q4, shp);
    const float logit = opacity_logits[g];
    const float opacity = 1.0f / (1.0f + expf(-logit));
    constexpr int K = (DEG + 1) * (DEG + 1);

    float gm[3] = {0.f, 0.f, 0.f};
    float gsig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma as a symmetric matrix
    float gop = 0.0f;
    bool sh_written = false, sh_fetched = false;

    for (int v = 0; v < vt.n_views; ++v) {
        const size_t vg = (size_t)v * n + g;
        if (touched[vg] == 0u) continue;
        if (!sh_fetched) {
            // the SH coefficients are read after the projection below
            prefetch_sh<K>(sh, n, g);
            sh_fetched = true;
        }
        const float* g2 = grad2d + vg * kGrad2d;
        float gmx = g2[0], gmy = g2[1], gA = g2[2], gB = g2[3], gC = g2[4], gO = g2[5];
        float gcol[3] = {g2[6], g2[7], g2[8]};
        const ViewGeom& geo = vt.v[v];
        if (geo.channels == 1) gcol[0] = gcol[1] = gcol[2] = g2[6] * (1.0f / 3.0f);
        const Cam& cam = cam_all[v];
        Proj p;
        project_one(mean, shp, cam, near_z, vt.log2_tw, vt.log2_th, geo.tiles_x, geo.tiles_y,
                    opacity, vt.tight_rect, p);
        if (!p.visible) {
            if (MODE == kShViaGcol) {
                float* gc_out = gcol_out + vg * 3;
                gc_out[0] = gc_out[1] = gc_out[2] = 0.0f;
            }
            continue;
        }

        gop += gO;
        // colour -> SH coefficients and the viewing direction
        float Y[16];
        sh_eval(DEG, p.dir[0], p.dir[1], p.dir[2], Y);
        float col[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* c = sh + ((size_t)k * n + g) * 3;
            col[0] = fmaf(Y[k], c[0], col[0]);
            col[1] = fmaf(Y[k], c[1], col[1]);
            col[2] = fmaf(Y[k], c[2], col[2]);
        }
        // a clamped channel passes no gradient
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            if (col[ch] + 0.5f < 0.0f) gcol[ch] = 0.0f;
        // the SH coefficients' own gradient, Y_k(dir) gcol, from this masked
        // colour gradient
        if (MODE == kShStaged) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float* a = sh_acc + k * sh_stride;
                a[0] = fmaf(Y[k], gcol[0], a[0]);
                a[1] = fmaf(Y[k], gcol[1], a[1]);
                a[2] = fmaf(Y[k], gcol[2], a[2]);
            }
        } else if (MODE == kShDirect) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float* a = sh_acc + k * sh_stride;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float y = __fmul_rn(Y[k], gcol[c]);
                    a[c] = accumulate ? __fadd_rn(a[c], y) : y;
                }
            }
            sh_written = true;
        } else {
            float* gc_out = gcol_out + vg * 3;
            gc_out[0] = gcol[0];
            gc_out[1] = gcol[1];
            gc_out[2] = gcol[2];
        }
        float w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* c = sh + ((size_t)k * n + g) * 3;
            w[k] = gcol[0] * c[0] + gcol[1] * c[1] + gcol[2] * c[2];
        }
        float gd[3] = {0.f, 0.f, 0.f};
        sh_grad_acc(DEG, p.dir[0], p.dir[1], p.dir[2], w, gd[0], gd[1], gd[2]);
        if (p.dist > 0.0f) {
            const float dd = gd[0] * p.dir[0] + gd[1] * p.dir[1] + gd[2] * p.dir[2];
            const float id = 1.0f / p.dist;
            for (int e = 0; e < 3; ++e) gm[e] += (gd[e] - p.dir[e] * dd) * id;
        }
        // conic -> 2D covariance: dL/dCov = -Q G Q, G = [[gA, gB/2], [gB/2, gC]]
        const float A = p.ca, B = p.cb, C = p.cc;
        const float ga = -(A * A * gA + A * B * gB + B * B * gC);
        const float gc = -(B * B * gA + B * C * gB + C * C * gC);
        const float gb = -(2.0f * A * B * gA + (A * C + B * B) * gB + 2.0f * B * C * gC);
        // Cov = T Sigma T^T + 0.3 I:
        //   dSigma += T^T Gs T with Gs = [[ga, gb/2], [gb/2, gc]]
        //   dT = 2 Gs T Sigma
        const float* T = p.T;
        const float hb = 0.5f * gb;
        float GT[6];  // Gs T
        for (int k = 0; k < 3; ++k) {
            GT[k] = ga * T[k] + hb * T[3 + k];
            GT[3 + k] = hb * T[k] + gc * T[3 + k];
        }
        gsig[0] += T[0] * GT[0] + T[3] * GT[3];
        gsig[1] += T[0] * GT[1] + T[3] * GT[4];
        gsig[2] += T[0] * GT[2] + T[3] * GT[5];
        gsig[3] += T[1] * GT[1] + T[4] * GT[4];
        gsig[4] += T[1] * GT[2] + T[4] * GT[5];
        gsig[5] += T[2] * GT[2] + T[5] * GT[5];
        const float* S = shp.sig;
        float gT[6];
        for (int r = 0; r < 2; ++r) {
            const float* gr = GT + 3 * r;
            gT[3 * r + 0] = 2.0f * (gr[0] * S[0] + gr[1] * S[1] + gr[2] * S[2]);
            gT[3 * r + 1] = 2.0f * (gr[0] * S[1] + gr[1] * S[3] + gr[2] * S[4]);
            gT[3 * r + 2] = 2.0f * (gr[0] * S[2] + gr[1] * S[4] + gr[2] * S[5]);
        }
        // T = J W: dJ = dT W^T (only the non-constant entries of J)
        const float* W = cam.R;
        const float gJ00 = gT[0] * W[0] + gT[1] * W[1] + gT[2] * W[2];
        const float gJ02 = gT[0] * W[6] + gT[1] * W[7] + gT[2] * W[8];
        const float gJ11 = gT[3] * W[3] + gT[4] * W[4] + gT[5] * W[5];
        const float gJ12 = gT[3] * W[6] + gT[4] * W[7] + gT[5] * W[8];
        const float z = p.xc[2], iz = 1.0f / z, iz2 = iz * iz;
        float gxc[3];
        float gz = gJ00 * (-cam.fx * iz2) + gJ02 * (cam.fx * p.u * iz2) + gJ11 * (-cam.fy * iz2) +
                   gJ12 * (cam.fy * p.v * iz2);
        const float gu = gJ02 * (-cam.fx * iz), gv = gJ12 * (-cam.fy * iz);
        gxc[0] = gmx * cam.fx * iz;
        gxc[1] = gmy * cam.fy * iz;
        gz -= (gmx * cam.fx * p.xc[0] + gmy * cam.fy * p.xc[1]) * iz2;
        if (!p.uc) {
            gxc[0] += gu * iz;
            gz -= gu * p.xc[0] * iz2;
        }
        if (!p.vc) {
            gxc[1] += gv * iz;
            gz -= gv * p.xc[1] * iz2;
        }
        gxc[2] = gz;
        for (int e = 0; e < 3; ++e) gm[e] += W[e] * gxc[0] + W[3 + e] * gxc[1] + W[6 + e] * gxc[2];
    }

    // Sigma = M M^T, M = Rq diag(s): dM = 2 dSigma M (dSigma symmetric)
    const float* R = shp.Rq;
    float M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * shp.s[c];
    const float Gs[9] = {gsig[0], gsig[1], gsig[2], gsig[1], gsig[3], gsig[4],
                         gsig[2], gsig[4], gsig[5]};
    float gM[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            gM[3 * r + c] = 2.0f * (Gs[3 * r] * M[c] + Gs[3 * r + 1] * M[3 + c] +
                                    Gs[3 * r + 2] * M[6 + c]);
    float gR[9];
    for (int c = 0; c < 3; ++c) {
        const float gsc = gM[c] * R[c] + gM[3 + c] * R[3 + c] + gM[6 + c] * R[6 + c];
        gls[c] = gsc * shp.s[c];
        for (int r = 0; r < 3; ++r) gR[3 * r + c] = gM[3 * r + c] * shp.s[c];
    }
    // Rq(qn) -> qn
    const float w = shp.qn[0], x = shp.qn[1], y = shp.qn[2], z = shp.qn[3];
    float gq[4];
    gq[0] = 2.0f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.0f * (y * gR[1] + z * gR[2] + y * gR[3] - w * gR[5] + z * gR[6] + w * gR[7]) -
            4.0f * x * (gR[4] + gR[8]);
    gq[2] = 2.0f * (x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7]) -
            4.0f * y * (gR[0] + gR[8]);
    gq[3] = 2.0f * (-w * gR[1] + x * gR[2] + w * gR[3] + y * gR[5] + x * gR[6] + y * gR[7]) -
            4.0f * z * (gR[0] + gR[4]);
    // qn = q / |q|
    const float dq = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    const float iq = 1.0f / shp.qnorm;
    gq4 = make_float4((gq[0] - w * dq) * iq, (gq[1] - x * dq) * iq, (gq[2] - y * dq) * iq,
                      (gq[3] - z * dq) * iq);
    glog = gop * opacity * (1.0f - opacity);
#pragma unroll
    for (int e = 0; e < 3; ++e) gm_out[e] = gm[e];
    if (MODE == kShDirect && !sh_written && !accumulate) {
        // not visible in the view: a zero SH gradient
#pragma unroll
        for (int k = 0; k < K; ++k)
            sh_acc[k * sh_stride] = sh_acc[k * sh_stride + 1] = sh_acc[k * sh_stride + 2] = 0.0f;
    }
}


// DIRECT (single-view plans): the SH gradient is written here and k_sh_bwd
// is not launched.  With group_vis, a warp's 32 Gaussians form a group: a
// group none of whose Gaussians touches a tile in any view (all-zero
// gradient) writes nothing, and group_vis[group] records which groups wrote.
template <int DEG, bool DIRECT>
__global__ void __launch_bounds__(kProjThreads, 2)
k_project_bwd(const float* __restrict__ means, const float* __restrict__ log_scales,
              const float* __restrict__ quats, const float* __restrict__ opacity_logits,
              const float* __restrict__ sh, int n, const gs_view* __restrict__ views,
              ViewTable vt, float near_z, const uint32_t* __restrict__ touched,
              const float* __restrict__ grad2d, float* __restrict__ gcol_out,
              float* __restrict__ g_means, float* __restrict__ g_ls, float* __restrict__ g_quats,
              float* __restrict__ g_logit, float* __restrict__ g_sh, int accumulate,
              uint8_t* __restrict__ group_vis) {
    extern __shared__ Cam cam_all[];
    for (int v = threadIdx.x; v < vt.n_views; v += blockDim.x) load_cam(views[v], cam_all[v]);
    __syncthreads();
    // a grid of resident CTAs striding over the Gaussians (whole warps: the
    // group vote stays warp-wide); a thread's next Gaussian's touched words
    // and parameters go to the L2 while it works on this one
    const int stride = gridDim.x * blockDim.x;
    for (int g0 = blockIdx.x * blockDim.x; g0 < n; g0 += stride) {
        const int g = g0 + threadIdx.x;
        if (g + stride < n) {
            for (int v = 0; v < vt.n_views; ++v)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(touched + (size_t)v * n + g + stride));
            prefetch_params(means, log_scales, quats, opacity_logits, g + stride);
        }
        if (group_vis && !group_touched(g, n, vt.n_views, touched, group_vis)) continue;
        if (g >= n) continue;
        float gm[3], gls[3], glog;
        float4 gq4;
        adjoint_one<DEG, DIRECT ? kShDirect : kShViaGcol>(
            g, means, log_scales, quats, opacity_logits, sh, n, cam_all, vt, near_z, touched, grad2d,
            gcol_out, DIRECT ? g_sh + (size_t)g * 3 : nullptr, (size_t)3 * n, accumulate, gm, gls,
            gq4, glog);
        if (accumulate) {
            for (int e = 0; e < 3; ++e) {
                g_means[3 * g + e] += gm[e];
                g_ls[3 * g + e] += gls[e];
            }
            float4 o = reinterpret_cast<float4*>(g_quats)[g];
            o.x += gq4.x; o.y += gq4.y; o.z += gq4.z; o.w += gq4.w;
            reinterpret_cast<float4*>(g_quats)[g] = o;
            g_logit[g] += glog;
        } else {
            for (int e = 0; e < 3; ++e) {
                g_means[3 * g + e] = gm[e];
                g_ls[3 * g + e] = gls[e];
            }
            reinterpret_cast<float4*>(g_quats)[g] = gq4;
            g_logit[g] = glog;
        }
    }
}

// Gradient of the SH coefficients: sum over views of Y_k(dir_v) gcol_v, with
// gcol the colour gradient k_project_bwd left (zero on clamped channels, a
// grayscale view's gradient spread over the three channels).
template <int DEG>
__global__ void __launch_bounds__(kProjThreads)
k_sh_bwd(const float* means, int n, const gs_view* __restrict__ views, ViewTable vt,
         const uint32_t* __restrict__ touched, const float* __restrict__ gcol_in,
         float* __restrict__ g_sh, int accumulate, int groups) {
    extern __shared__ Cam cam_all[];
    for (int v = threadIdx.x; v < vt.n_views; v += blockDim.x) load_cam(views[v], cam_all[v]);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (groups && !group_touched(g, n, vt.n_views, touched, nullptr)) return;
    if (g >= n) return;
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float mean[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    float acc[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0f;
    for (int v = 0; v < vt.n_views; ++v) {
        const size_t vg = (size_t)v * n + g;
        if (touched[vg] == 0u) continue;
        const float* gc = gcol_in + vg * 3;
        const float c0 = gc[0], c1 = gc[1], c2 = gc[2];
        const Cam& cam = cam_all[v];
        const float d0 = mean[0] - cam.cc[0], d1 = mean[1] - cam.cc[1], d2 = mean[2] - cam.cc[2];
        const float dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        const float id = dist > 0.0f ? 1.0f / dist : 0.0f;
        float Y[16];
        sh_eval(DEG, d0 * id, d1 * id, d2 * id, Y);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            acc[k][0] = fmaf(Y[k], c0, acc[k][0]);
            acc[k][1] = fmaf(Y[k], c1, acc[k][1]);
            acc[k][2] = fmaf(Y[k], c2, acc[k][2]);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float* o = g_sh + ((size_t)k * n + g) * 3;
        if (accumulate) {
            o[0] += acc[k][0];
            o[1] += acc[k][1];
            o[2] += acc[k][2];
        } else {
            o[0] = acc[k][0];
            o[1] = acc[k][1];
            o[2] = acc[k][2];
        }
    }
}

// A8 + A9 in one pass over a chunk of kFuseThreads consecutive Gaussians.
//
// Phase 1 (a thread per Gaussian): the projection adjoint (adjoint_one) with
// the gradients staged in shared memory in the order of the parameter
// arrays: means [3c], log-scales [3c], quaternions [4c], logits [c], then one
// [3c] run per SH coefficient plane (the [K][N][3] layout), c = kFuseThreads.
// Phase 2 (a thread per float): Adam over those runs, each a contiguous
// range of a parameter array and of its two moments; every run is a multiple
// of kFuseThreads floats, so a warp always works inside one run and each of
// its loads and stores is one 128-byte line.  Up to six runs per thread are
// loaded before any is updated, for enough bytes in flight.  The gradients
// never go to global memory unless asked for (grads_out).
constexpr int kFuseThreads = 128;
constexpr int kFuseMinBlocks = 4;
constexpr int kShPlanes = 4;  // SH planes per Adam batch (3 runs each)
static_assert((11 + 3 * 16) * kFuseThreads * sizeof(float) + sizeof(Cam) * GS_MAX_VIEWS <=
                  48 * 1024,
              "the fused stage fits the default dynamic shared memory");

// Adam on NP planes x NR runs of kFuseThreads floats of one parameter array:
// run j of plane q starts at float off + q * plane_stride + j * kFuseThreads
// and holds the floats below `total` of its plane; its gradient is at
// g + (q * NR + j) * kFuseThreads in shared memory (plus add, if given).
// lr_first applies to plane 0, lr_rest to the others.  All NP * NR loads of
// a thread are issued before any update.
struct AdamRuns {
    float b1, b2, eps, ibc1, ibc2;
    int t;
    template <int NP, int NR>
    __device__ __forceinline__ void run(float* __restrict__ p, float* __restrict__ m,
                                        float* __restrict__ v, const float* __restrict__ add,
                                        float* __restrict__ out, size_t off, size_t plane_stride,
                                        int total, const float* g, float lr_first,
                                        float lr_rest) const {
        constexpr int U = NP * NR;
        float pp[U], mm[U], vv[U], gg[U];
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int u = q * NR + j;
                const size_t i = off + q * plane_stride + (size_t)j * kFuseThreads + t;
                if (j * kFuseThreads + t < total) {
                    gg[u] = g[u * kFuseThreads + t];
                    if (add) gg[u] += add[i];
                    pp[u] = p[i];
                    mm[u] = m[i];
                    vv[u] = v[i];
                }
            }
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int u = q * NR + j;
                const size_t i = off + q * plane_stride + (size_t)j * kFuseThreads + t;
                if (j * kFuseThreads + t < total) {
                    adam1(pp[u], gg[u], mm[u], vv[u], q == 0 ? lr_first : lr_rest, b1, b2, eps,
                          ibc1, ibc2);
                    p[i] = pp[u];
                    m[i] = mm[u];
                    v[i] = vv[u];
                    if (out) out[i] = gg[u];
                }
            }
    }
};

// Run r (of 11 + 3K) of the chunk of Gaussians [g0, g0 + cnt): its group
// (0 means, 1 log-scales, 2 quaternions, 3 logits, 4 SH), the offset of its
// first float in that group's array and the number of its floats in use.
template <int K>
__device__ __forceinline__ void run_of(int r, int g0, int cnt, int n, int& grp, size_t& off,
                                       int& len) {
    constexpr int C = kFuseThreads;
    if (r < 6) {
        grp = r / 3; off = (size_t)3 * g0 + (size_t)(r % 3) * C; len = 3 * cnt - (r % 3) * C;
    } else if (r < 10) {
        grp = 2; off = (size_t)4 * g0 + (size_t)(r - 6) * C; len = 4 * cnt - (r - 6) * C;
    } else if (r < 11) {
        grp = 3; off = (size_t)g0; len = cnt;
    } else {
        const int k = (r - 11) / 3, j = (r - 11) % 3;
        grp = 4; off = ((size_t)k * n + g0) * 3 + (size_t)j * C; len = 3 * cnt - j * C;
    }
}

// Parameter (a = 0), first moment (1) or second moment (2) array of group grp.
__device__ __forceinline__ const float* state_array(const FusedAdam& fa, int a, int grp) {
    auto pick = [grp](const float* g0, const float* g1, const float* g2, const float* g3,
                      const float* g4) {
        return grp == 0 ? g0 : grp == 1 ? g1 : grp == 2 ? g2 : grp == 3 ? g3 : g4;
    };
    return a == 0   ? pick(fa.p_means, fa.p_ls, fa.p_quats, fa.p_logit, fa.p_sh)
           : a == 1 ? pick(fa.m_means, fa.m_ls, fa.m_quats, fa.m_logit, fa.m_sh)
                    : pick(fa.v_means, fa.v_ls, fa.v_quats, fa.v_logit, fa.v_sh);
}

template <int DEG>
__global__ void __launch_bounds__(kFuseThreads, kFuseMinBlocks)
k_adjoint_adam(const float* __restrict__ means, const float* __restrict__ log_scales,
               const float* __restrict__ quats, const float* __restrict__ opacity_logits,
               const float* __restrict__ sh, int n, const gs_view* __restrict__ views,
               ViewTable vt, float near_z, const uint32_t* __restrict__ touched,
               const float* __restrict__ grad2d, FusedAdam fa) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int C = kFuseThreads;
    constexpr int kRuns = 11 + 3 * K;  // runs of C floats per chunk
    extern __shared__ float4 fuse_smem[];
    float* stage = reinterpret_cast<float*>(fuse_smem);  // kRuns * C floats
    Cam* cam_all = reinterpret_cast<Cam*>(stage + kRuns * C);
    __shared__ float s_bc[2];
    for (int v = threadIdx.x; v < vt.n_views; v += blockDim.x) load_cam(views[v], cam_all[v]);
    if (threadIdx.x == 0) adam_bias(fa.b1, fa.b2, *fa.step, s_bc[0], s_bc[1]);
    const int t = threadIdx.x;
    const int g0 = blockIdx.x * C;
    const int cnt = min(C, n - g0);
    // Ask L2 for the chunk's parameters and moments now, so that their DRAM
    // reads overlap the adjoint below: each of the kRuns runs of the three
    // arrays is C floats = 4 lines of 128 bytes; a thread takes every C-th
    // line, only lines that phase 2 will load.
    {
        constexpr int kLines = kRuns * 3 * (C / 32);
        for (int L = t; L < kLines; L += C) {
            const int r = L / (3 * (C / 32)), a = (L / (C / 32)) % 3, line = L % (C / 32);
            int grp, len;
            size_t off;
            run_of<K>(r, g0, cnt, n, grp, off, len);
            if (line * 32 < len)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(state_array(fa, a, grp) + off +
                                                              line * 32));
        }
    }
    float* sh_acc = stage + 11 * C + 3 * t;
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) sh_acc[(k / 3) * 3 * C + k % 3] = 0.0f;
    __syncthreads();
    if (t < cnt) {
        float gm[3], gls[3], glog;
        float4 gq4;
        adjoint_one<DEG, kShStaged>(g0 + t, means, log_scales, quats, opacity_logits, sh, n,
                                    cam_all, vt, near_z, touched, grad2d, nullptr, sh_acc, 3 * C,
                                    0, gm, gls, gq4, glog);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            stage[3 * t + e] = gm[e];
            stage[3 * C + 3 * t + e] = gls[e];
        }
        stage[6 * C + 4 * t + 0] = gq4.x;
        stage[6 * C + 4 * t + 1] = gq4.y;
        stage[6 * C + 4 * t + 2] = gq4.z;
        stage[6 * C + 4 * t + 3] = gq4.w;
        stage[10 * C + t] = glog;
    }
    __syncthreads();
    const AdamRuns ar{fa.b1, fa.b2, fa.eps, s_bc[0], s_bc[1], t};
    const size_t o3 = (size_t)3 * g0, o4 = (size_t)4 * g0;
    ar.run<1, 3>(fa.p_means, fa.m_means, fa.v_means, fa.a_means, fa.o_means, o3, 0, 3 * cnt,
                 stage, fa.lr[0], fa.lr[0]);
    ar.run<1, 3>(fa.p_ls, fa.m_ls, fa.v_ls, fa.a_ls, fa.o_ls, o3, 0, 3 * cnt, stage + 3 * C,
                 fa.lr[1], fa.lr[1]);
    ar.run<1, 4>(fa.p_quats, fa.m_quats, fa.v_quats, fa.a_quats, fa.o_quats, o4, 0, 4 * cnt,
                 stage + 6 * C, fa.lr[2], fa.lr[2]);
    ar.run<1, 1>(fa.p_logit, fa.m_logit, fa.v_logit, fa.a_logit, fa.o_logit, (size_t)g0, 0, cnt,
                 stage + 10 * C, fa.lr[3], fa.lr[3]);
    // SH: kShPlanes coefficient planes at a time; plane 0 takes the DC rate
    const size_t ps = (size_t)3 * n;
    int k = 0;
    for (; k + kShPlanes <= K; k += kShPlanes)
        ar.run<kShPlanes, 3>(fa.p_sh, fa.m_sh, fa.v_sh, fa.a_sh, fa.o_sh, k * ps + o3, ps,
                             3 * cnt, stage + (11 + 3 * k) * C, k == 0 ? fa.lr[4] : fa.lr[5],
                             fa.lr[5]);
    for (; k + 2 <= K; k += 2)
        ar.run<2, 3>(fa.p_sh, fa.m_sh, fa.v_sh, fa.a_sh, fa.o_sh, k * ps + o3, ps, 3 * cnt,
                     stage + (11 + 3 * k) * C, k == 0 ? fa.lr[4] : fa.lr[5], fa.lr[5]);
    if (k < K)
        ar.run<1, 3>(fa.p_sh, fa.m_sh, fa.v_sh, fa.a_sh, fa.o_sh, k * ps + o3, ps, 3 * cnt,
                     stage + (11 + 3 * k) * C, k == 0 ? fa.lr[4] : fa.lr[5], fa.lr[5]);
}

// The CTAs of a grid-stride kernel resident at once on this GPU (its
// occupancy per SM times the SMs), and no more than `needed`.
template <class K>
int resident_grid(K kernel, int threads, size_t smem, int needed) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int r = per_sm * sm_count();
    return needed < r ? needed : (r > 0 ? r : 1);
}

}  // namespace

gs_status launch_project(const Plan* p, const gs_map* map, const gs_view* views_dev, void* ws,
                         cudaStream_t st) {
    if (reinterpret_cast<uintptr_t>(map->quats) % 16) return GS_ERR_INVALID;
    const int n = map->n;
    DevCounters* ctr = buf<DevCounters>(p, ws, GS_BUF_COUNTERS);
    // the status word gathers the bits of all view passes of a recompute
    // plan: only the first pass (or a whole plan) clears it
    const size_t keep = p->view_index > 0 ? sizeof(uint32_t) : 0;
    if (cudaMemsetAsync(reinterpret_cast<char*>(ctr) + keep, 0, sizeof(DevCounters) - keep, st) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    auto* kern = map->sh_degree == 0   ? k_project<0>
                 : map->sh_degree == 1 ? k_project<1>
                 : map->sh_degree == 2 ? k_project<2>
                                       : k_project<3>;
    dim3 grid((n + kProjThreads - 1) / kProjThreads,
              (p->vt.n_views + kViewsPerThread - 1) / kViewsPerThread);
    kern<<<grid, kProjThreads, 0, st>>>(
        map->means, map->log_scales, map->quats, map->opacity_logits, map->sh, n, views_dev,
        p->vt, p->cfg.near_z, buf<float4>(p, ws, GS_BUF_PROJ), buf<uint16_t>(p, ws, GS_BUF_RECT),
        buf<uint32_t>(p, ws, GS_BUF_TOUCHED), buf<int32_t>(p, ws, GS_BUF_RADIUS),
        buf<uint32_t>(p, ws, B_DKEY_A), ctr,
        buf<uint32_t>(p, ws, B_SPANS), buf<uint32_t>(p, ws, B_SPAN_POOL), p->span_pool_rows);
    return launch_status();
}

static gs_status launch_project_adjoint(const Plan* p, const gs_map* map,
                                        const gs_view* views_dev, void* ws,
                                        const gs_map_grad* grads, int accumulate,
                                        uint8_t* group_vis, cudaStream_t st) {
    const int n = map->n;
    const size_t smem = sizeof(Cam) * p->vt.n_views;
    const bool direct = p->vt.n_views == 1;
    auto* kern = direct ? (map->sh_degree == 0   ? k_project_bwd<0, true>
                           : map->sh_degree == 1 ? k_project_bwd<1, true>
                           : map->sh_degree == 2 ? k_project_bwd<2, true>
                                                 : k_project_bwd<3, true>)
                        : (map->sh_degree == 0   ? k_project_bwd<0, false>
                           : map->sh_degree == 1 ? k_project_bwd<1, false>
                           : map->sh_degree == 2 ? k_project_bwd<2, false>
                                                 : k_project_bwd<3, false>);
    const int blocks =
        resident_grid(kern, kProjThreads, smem, (n + kProjThreads - 1) / kProjThreads);
    kern<<<blocks, kProjThreads, smem, st>>>(
        map->means, map->log_scales, map->quats, map->opacity_logits, map->sh, n, views_dev,
        p->vt, p->cfg.near_z, buf<uint32_t>(p, ws, GS_BUF_TOUCHED),
        buf<float>(p, ws, GS_BUF_GRAD2D), buf<float>(p, ws, B_GCOL), grads->means,
        grads->log_scales, grads->quats, grads->opacity_logits, grads->sh, accumulate, group_vis);
    return launch_status();
}

gs_status launch_project_bwd(const Plan* p, const gs_map* map, const gs_view* views_dev,
                             void* ws, const gs_map_grad* grads, int accumulate,
                             cudaStream_t st, uint8_t* group_vis) {
    if (reinterpret_cast<uintptr_t>(grads->quats) % 16) return GS_ERR_INVALID;
    gs_status s = launch_project_adjoint(p, map, views_dev, ws, grads, accumulate, group_vis, st);
    if (s != GS_OK || p->vt.n_views == 1) return s;  // one view: SH gradient already written
    const int n = map->n;
    auto* kern_sh = map->sh_degree == 0   ? k_sh_bwd<0>
                    : map->sh_degree == 1 ? k_sh_bwd<1>
                    : map->sh_degree == 2 ? k_sh_bwd<2>
                                          : k_sh_bwd<3>;
    kern_sh<<<(n + kProjThreads - 1) / kProjThreads, kProjThreads, sizeof(Cam) * p->vt.n_views,
              st>>>(map->means, n, views_dev, p->vt, buf<uint32_t>(p, ws, GS_BUF_TOUCHED),
                    buf<float>(p, ws, B_GCOL), grads->sh, accumulate, group_vis ? 1 : 0);
    return launch_status();
}

gs_status launch_project_bwd_adam(const Plan* p, const gs_map* map, const gs_view* views_dev,
                                  void* ws, const gs_map_grad* params, const gs_map_grad* m,
                                  const gs_map_grad* v, const gs_map_grad* grads_acc,
                                  const gs_map_grad* grads_out, const float* lr6, float b1,
                                  float b2, float eps, int32_t* step_dev, cudaStream_t st) {
    auto misaligned = [](const gs_map_grad* g) {
        return g && (reinterpret_cast<uintptr_t>(g->quats) % 16) != 0;
    };
    if (misaligned(params) || misaligned(m) || misaligned(v) || misaligned(grads_acc) ||
        misaligned(grads_out) || reinterpret_cast<uintptr_t>(map->quats) % 16)
        return GS_ERR_INVALID;
    FusedAdam fa{};
    for (int k = 0; k < 6; ++k) fa.lr[k] = lr6[k];
    fa.b1 = b1;
    fa.b2 = b2;
    fa.eps = eps;
    fa.step = step_dev;
    fa.p_means = params->means; fa.p_ls = params->log_scales; fa.p_quats = params->quats;
    fa.p_logit = params->opacity_logits; fa.p_sh = params->sh;
    fa.m_means = m->means; fa.m_ls = m->log_scales; fa.m_quats = m->quats;
    fa.m_logit = m->opacity_logits; fa.m_sh = m->sh;
    fa.v_means = v->means; fa.v_ls = v->log_scales; fa.v_quats = v->quats;
    fa.v_logit = v->opacity_logits; fa.v_sh = v->sh;
    if (grads_acc) {
        fa.a_means = grads_acc->means; fa.a_ls = grads_acc->log_scales;
        fa.a_quats = grads_acc->quats; fa.a_logit = grads_acc->opacity_logits;
        fa.a_sh = grads_acc->sh;
    }
    if (grads_out) {
        fa.o_means = grads_out->means; fa.o_ls = grads_out->log_scales;
        fa.o_quats = grads_out->quats; fa.o_logit = grads_out->opacity_logits;
        fa.o_sh = grads_out->sh;
    }
    gs_status s = launch_step_inc(step_dev, st);
    if (s != GS_OK) return s;
    const int n = map->n;
    const int K = (map->sh_degree + 1) * (map->sh_degree + 1);
    const size_t smem =
        (size_t)(11 + 3 * K) * kFuseThreads * sizeof(float) + sizeof(Cam) * p->vt.n_views;
    auto* kern = map->sh_degree == 0   ? k_adjoint_adam<0>
                 : map->sh_degree == 1 ? k_adjoint_adam<1>
                 : map->sh_degree == 2 ? k_adjoint_adam<2>
                                       : k_adjoint_adam<3>;
    kern<<<(n + kFuseThreads - 1) / kFuseThreads, kFuseThreads, smem, st>>>(
        map->means, map->log_scales, map->quats, map->opacity_logits, map->sh, n, views_dev,
        p->vt, p->cfg.near_z, buf<uint32_t>(p, ws, GS_BUF_TOUCHED),
        buf<float>(p, ws, GS_BUF_GRAD2D), fa);
    return launch_status();
}

}  // namespace gs
