/*
 * gs_oracle.c -- FP64 CPU oracle for the 3D Gaussian Splatting mapping step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, double-precision
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant with the CUDA library; every constant below is
 * derived here from its mathematical definition.
 *
 * What is computed, and where the method states it:
 *   - The map is a set of anisotropic 3D Gaussians, each with an opacity, a
 *     rotation, a location, a scale and a colour, rendered with the original
 *     differentiable tile-based rasteriser of 3DGS (paper Sec. III-B, "Dense
 *     Reconstruction").
 *   - Rendering projects the Gaussians onto the camera plane, sorts them by
 *     depth and blends them front to back (paper Sec. II, "Related Work",
 *     paragraph on 3DGS).
 *   - The parameters are optimised by gradient descent on the photometric loss
 *     of Eq. 2, an L1 term plus an SSIM term weighted by lambda (paper
 *     Sec. III-B); the optimiser is the default 3DGS configuration, i.e. Adam
 *     (paper Sec. IV-A, "Experimental Setup").
 * The paper gives no rasteriser formulas; the readings used where it is
 * silent (near plane, pixel centre, Jacobian clamp, 3-sigma tile extent,
 * 0.3 px^2 dilation, alpha/transmittance thresholds, SH basis, grayscale,
 * the garbled form of Eq. 2, Adam constants) are stated next to each step.
 *
 * Data layout (all arrays row-major, double):
 *   means[n][3], log_scales[n][3], quats[n][4] as (w,x,y,z), opacity_logits[n],
 *   sh[K][n][3] with K = (degree+1)^2 (coefficient-major), camera
 *   cam[16] = R[9] (world->camera, row-major), t[3], fx, fy, cx, cy.
 *   Images are planar [channels][H][W]; per-pixel maps are [H][W].
 *
 * Threads: oracle_set_threads(k) lets the loops over independent Gaussians,
 * pixel rows and parameters run on k host threads (OpenMP).  The default is
 * one thread, which the tests use; with more, only the order in which the
 * adjoint's per-pixel terms are added into a Gaussian's gradient (and the
 * loss's per-row sums) can change, i.e. the last bits of the result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of the parallel loops (1 unless set). */
void oracle_set_threads(int k) {
#ifdef _OPENMP
    omp_set_num_threads(k > 0 ? k : 1);
#else
    (void)k;
#endif
}

/* ------------------------------------------------------------------------ */
/* Readings of points where the paper is silent.                            */
/* ------------------------------------------------------------------------ */
#define OR_ALPHA_MIN (1.0 / 255.0) /* skip a Gaussian whose alpha < 1/255 */
#define OR_ALPHA_MAX 0.99          /* clamp alpha from above */
#define OR_T_MIN 1e-4              /* stop before T would drop below 1e-4 */
#define OR_DILATION 0.3            /* low-pass filter added to the 2D cov */
#define OR_CLIP 1.3                /* Jacobian clamp as a multiple of the image half-extent */
#define OR_SIGMAS 3.0              /* tile extent: 3 standard deviations */

/* Guard-band margins: a decision whose FP64 margin is below these can be
 * taken the other way by an FP32 evaluation of the same formula. */
#define OR_G_TILE 1e-9   /* rect edges, in tile units */
#define OR_G_RADIUS 1e-5 /* 3 sqrt(lambda_max) vs an integer, relative */
#define OR_G_NEAR 1e-6   /* depth vs near plane, relative */
#define OR_G_ALPHA 5e-5  /* o*G vs 1/255, relative */
#define OR_G_TRANS 1e-3  /* T*(1-alpha) vs 1e-4, relative */
#define OR_G_POWER 1e-6  /* power vs 0 */
#define OR_G_CLAMP 1e-6  /* colour vs 0, alpha vs 0.99, Jacobian clamp (gradient kinks) */
#define OR_G_DEPTH 1e-12 /* relative distance of the depth to an FP32 rounding midpoint */

/* Guard bits reported per Gaussian by oracle_project. */
#define OR_GUARD_RECT 1
#define OR_GUARD_NEAR 2
#define OR_GUARD_DET 4
#define OR_GUARD_KINK 8 /* colour clamp or Jacobian clamp close to switching */
#define OR_GUARD_DEPTH 16 /* FP32 depth key ambiguous (depth next to a rounding midpoint) */
/* a tight-rect edge (reading C19) or its opacity cut close to switching: the
 * tile it adds or drops has alpha < 1/255 at every pixel, so the lists may
 * differ there but no pixel value can */
#define OR_GUARD_TIGHT 32
/* 3 sqrt(lambda_max) close to an integer: the radius may differ by one */
#define OR_GUARD_RADIUS 64

/* Guard bits reported per pixel by oracle_render. */
#define OR_GPX_ALPHA 1
#define OR_GPX_TRANS 2
#define OR_GPX_POWER 4
#define OR_GPX_KINK 16 /* alpha near its 0.99 clamp (gradient kink only) */

static int near_int(double v, double margin) {
    double r = floor(v + 0.5);
    return fabs(v - r) < margin;
}

/*
 * Tile rect of one projected Gaussian, [x0,y0,x1,y1) clamped to the grid, and
 * its radius r; returns the area (0: the Gaussian draws into no tile).
 *
 * Square rect (reading C4): [floor((mu-r)/t), floor((mu+r+t-1)/t)) with
 * r = ceil(3 sqrt(lambda_max)) of the dilated 2D covariance.
 *
 * tight = 1 (reading C19): the square rect intersected with the tiles that
 * meet the axis-aligned box of the ellipse outside which alpha < 1/255.
 * alpha = min(0.99, o exp(-q/2)) with q = d^T cov^-1 d, so alpha >= 1/255
 * needs q <= t_a = 2 ln(255 o), and the ellipse q <= t_a has half-widths
 * sqrt(t_a cov_xx), sqrt(t_a cov_yy).  A tile left out has no pixel that
 * the renderer would blend: the rect shrinks, the image does not.  The level
 * is widened to t = 1.01 t_a + 0.01 so that no FP32 evaluation of alpha near
 * the ellipse can reach 1/255 in a dropped tile; with o < 0.999/255 no pixel
 * reaches it at all and the rect is empty.  Pixel x of tile k satisfies
 * k t <= x <= k t + t - 1, so tiles [ceil((mu - h - t + 1)/t), floor((mu + h)/t)]
 * meet [mu - h, mu + h].  Within that box, every tile row keeps only the
 * tiles whose pixel rectangle meets the widened ellipse (row_span below):
 * the kept tiles are exactly the tiles of the square rect that meet the
 * ellipse, a purely geometric set, whatever the box's shape.
 */
#define OR_TIGHT_MIN_OPACITY (0.999 / 255.0)
#define OR_G_TIGHT 1e-5 /* tight rect edges in tile units, relative to 1 + h / t */

/* Square rect of radius r: rc = [floor((mu-r)/t), floor((mu+r+t-1)/t)) clamped
 * to the grid; ex[k] the unfloored edge values. */
static void square_rect(const double mean2d[2], int r, int tile_w, int tile_h, int tiles_x,
                        int tiles_y, int rc[4], double ex[4]) {
    ex[0] = (mean2d[0] - r) / tile_w;
    ex[1] = (mean2d[1] - r) / tile_h;
    ex[2] = (mean2d[0] + r + tile_w - 1) / tile_w;
    ex[3] = (mean2d[1] + r + tile_h - 1) / tile_h;
    int lim[4] = {tiles_x, tiles_y, tiles_x, tiles_y};
    for (int k = 0; k < 4; k++) {
        double f = floor(ex[k]);
        rc[k] = f < 0.0 ? 0 : (f > lim[k] ? lim[k] : (int)f);
    }
}

/* Tiles of tile row ty that meet the widened ellipse d^T cov^-1 d <= t
 * (reading C19, per row): the band of pixel rows ty*th .. ty*th+th-1 cuts
 * the ellipse in a convex set whose x-extent is [xmin, xmax]; tiles
 * [ceil((mu_x + xmin - tw + 1)/tw), floor((mu_x + xmax)/tw)] meet it, clipped
 * to [rx0, rx1).  For fixed dy the ellipse spans x = (b/c) dy +- sqrt(det
 * (t c - dy^2))/c; over the band, x is largest at dy* = b sqrt(t/a) (x =
 * sqrt(t a)) when dy* lies in the band, else at a band end (the upper edge
 * is concave in dy); symmetrically for the smallest x at -dy*.  Returns the
 * number of tiles; decisions within the tight margin are flagged. */
static int row_span(const double mean2d[2], const double cov[3], double t, int ty, int tile_w,
                    int tile_h, int rx0, int rx1, int *x0, int *x1, int *guard) {
    const double a = cov[0], b = cov[1], c = cov[2], det = a * c - b * b;
    const double Y = sqrt(t * c), X = sqrt(t * a);
    double lo = ty * (double)tile_h - mean2d[1], hi = lo + tile_h - 1.0;
    const double my = 1e-5 * (1.0 + Y);
    if (fabs(lo - Y) < my || fabs(hi + Y) < my) *guard |= OR_GUARD_TIGHT;
    if (lo > Y || hi < -Y) return 0;
    if (lo < -Y) lo = -Y;
    if (hi > Y) hi = Y;
    const double ds = b * sqrt(t / a);
    double xmax, xmin;
    if (lo <= ds && ds <= hi) {
        xmax = X;
    } else {
        const double e0 = (b / c) * lo + sqrt(fmax(0.0, det * (t * c - lo * lo))) / c;
        const double e1 = (b / c) * hi + sqrt(fmax(0.0, det * (t * c - hi * hi))) / c;
        xmax = e0 > e1 ? e0 : e1;
    }
    if (lo <= -ds && -ds <= hi) {
        xmin = -X;
    } else {
        const double e0 = (b / c) * lo - sqrt(fmax(0.0, det * (t * c - lo * lo))) / c;
        const double e1 = (b / c) * hi - sqrt(fmax(0.0, det * (t * c - hi * hi))) / c;
        xmin = e0 < e1 ? e0 : e1;
    }
    const double el = (mean2d[0] + xmin - tile_w + 1.0) / tile_w, eh = (mean2d[0] + xmax) / tile_w;
    const double m = OR_G_TIGHT * (1.0 + X / tile_w);
    if (near_int(el, m) || near_int(eh, m)) *guard |= OR_GUARD_TIGHT;
    double klo = ceil(el), khi = floor(eh) + 1.0;
    int k0 = klo < rx0 ? rx0 : (klo > rx1 ? rx1 : (int)klo);
    int k1 = khi > rx1 ? rx1 : (khi < rx0 ? rx0 : (int)khi);
    *x0 = k0;
    *x1 = k1;
    return k1 > k0 ? k1 - k0 : 0;
}

static double tight_level(double opacity) { return 1.01 * (2.0 * log(255.0 * opacity)) + 0.01; }

/* The tight cut (reading C19) applied to rc in place; returns the number of
 * tiles (the box of the widened ellipse, then its row spans). */
static int cut_rect(const double mean2d[2], const double cov[3], double opacity, int tile_w,
                    int tile_h, int tiles_x, int tiles_y, int tight, int rc[4], int *guard) {
    if (tight) {
        int lim[2] = {tiles_x, tiles_y};
        if (fabs(opacity - OR_TIGHT_MIN_OPACITY) < 1e-6 * OR_TIGHT_MIN_OPACITY)
            *guard |= OR_GUARD_TIGHT;
        if (!(opacity >= OR_TIGHT_MIN_OPACITY)) return 0;
        double t = tight_level(opacity);
        double h[2] = {sqrt(t * cov[0]), sqrt(t * cov[2])};
        double tl[2] = {tile_w, tile_h};
        for (int a = 0; a < 2; a++) {
            double lo = (mean2d[a] - h[a] - tl[a] + 1.0) / tl[a];
            double hi = (mean2d[a] + h[a]) / tl[a];
            double margin = OR_G_TIGHT * (1.0 + h[a] / tl[a]);
            if (near_int(lo, margin) || near_int(hi, margin)) *guard |= OR_GUARD_TIGHT;
            double klo = ceil(lo), khi = floor(hi) + 1.0;
            if (klo > rc[a]) rc[a] = klo > lim[a] ? lim[a] : (int)klo;
            if (khi < rc[a + 2]) rc[a + 2] = khi < 0.0 ? 0 : (int)khi;
        }
        if (rc[2] <= rc[0] || rc[3] <= rc[1]) return 0;
        int total = 0, x0, x1;
        for (int ty = rc[1]; ty < rc[3]; ty++)
            total += row_span(mean2d, cov, t, ty, tile_w, tile_h, rc[0], rc[2], &x0, &x1, guard);
        return total;
    }
    int w = rc[2] - rc[0], hgt = rc[3] - rc[1];
    return (w > 0 && hgt > 0) ? w * hgt : 0;
}

static int same_rect(const int a[4], int area_a, const int b[4], int area_b) {
    if (area_a == 0 || area_b == 0) return area_a == area_b;
    return a[0] == b[0] && a[1] == b[1] && a[2] == b[2] && a[3] == b[3];
}

/* Guards: OR_GUARD_RADIUS when 3 sqrt(lambda_max) is close to an integer
 * (the radius itself may differ in FP32); OR_GUARD_RECT only when that, or
 * a square edge close to a tile boundary, could change the final rect
 * (checked by computing the rect with the other choice). */
static int tile_rect(const double mean2d[2], const double cov[3], double det, double opacity,
                     int tile_w, int tile_h, int tiles_x, int tiles_y, int tight, int rc[4],
                     int *r_out, int *guard) {
    double mid = 0.5 * (cov[0] + cov[2]);
    double lam = mid + sqrt(fmax(0.0, mid * mid - det));
    double ext = OR_SIGMAS * sqrt(lam);
    int r = (int)ceil(ext);
    *r_out = r;
    double ex[4];
    int sq[4];
    square_rect(mean2d, r, tile_w, tile_h, tiles_x, tiles_y, sq, ex);
    for (int k = 0; k < 4; k++) rc[k] = sq[k];
    int area = cut_rect(mean2d, cov, opacity, tile_w, tile_h, tiles_x, tiles_y, tight, rc, guard);
    int alt[4], scratch = 0;
    double ex2[4];
    if (near_int(ext, OR_G_RADIUS * fmax(1.0, ext))) {
        *guard |= OR_GUARD_RADIUS;
        int k0 = (int)floor(ext + 0.5);
        square_rect(mean2d, r == k0 ? k0 + 1 : k0, tile_w, tile_h, tiles_x, tiles_y, alt, ex2);
        int a2 = cut_rect(mean2d, cov, opacity, tile_w, tile_h, tiles_x, tiles_y, tight, alt,
                          &scratch);
        if (!same_rect(rc, area, alt, a2)) *guard |= OR_GUARD_RECT;
    }
    int lim[4] = {tiles_x, tiles_y, tiles_x, tiles_y};
    for (int k = 0; k < 4; k++) {
        if (!near_int(ex[k], OR_G_TILE)) continue;
        double m = floor(ex[k] + 0.5), f = floor(ex[k]);
        double g = f == m ? m - 1.0 : m; /* the other floor */
        for (int j = 0; j < 4; j++) alt[j] = sq[j];
        alt[k] = g < 0.0 ? 0 : (g > lim[k] ? lim[k] : (int)g);
        int a2 = cut_rect(mean2d, cov, opacity, tile_w, tile_h, tiles_x, tiles_y, tight, alt,
                          &scratch);
        if (!same_rect(rc, area, alt, a2)) *guard |= OR_GUARD_RECT;
    }
    return area;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degrees 0..3.                                  */
/* Reading of the colour model: the paper renders plain RGB (Sec. III-B,   */
/* following MonoGS); the workloads also use SH degree 3.  The basis is the */
/* real SH basis with the Condon-Shortley phase, ordered m = -l..l within   */
/* each degree, evaluated at a unit direction (x,y,z):                       */
/*   Y_{l,m} = sqrt(2) Im Y_l^{|m|}  (m<0),  Y_l^0 (m=0),  sqrt(2) Re Y_l^m  */
/* with the complex Y_l^m of the usual physics normalisation.  Each real    */
/* function is written as a polynomial in x,y,z and its normalisation      */
/* constant is computed from its closed form.                               */
/* ------------------------------------------------------------------------ */
static void sh_basis(int degree, double x, double y, double z, double *Y) {
    const double pi = acos(-1.0);
    Y[0] = sqrt(1.0 / (4.0 * pi));
    if (degree < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    if (degree < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (3.0 * z * z - (x * x + y * y + z * z));
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (x * x - y * y);
    if (degree < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    const double r2 = x * x + y * y + z * z;
    Y[9] = -k3a * y * (3.0 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (5.0 * z * z - r2);
    Y[12] = k3d * z * (5.0 * z * z - 3.0 * r2);
    Y[13] = -k3c * x * (5.0 * z * z - r2);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* Gradient of each basis polynomial above with respect to (x,y,z):
 * dY[k][0..2].  Differentiated term by term from sh_basis. */
static void sh_basis_grad(int degree, double x, double y, double z, double dY[16][3]) {
    const double pi = acos(-1.0);
    memset(dY, 0, sizeof(double) * 16 * 3);
    if (degree < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    dY[1][1] = -k1;
    dY[2][2] = k1;
    dY[3][0] = -k1;
    if (degree < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    /* Y4 = k2a x y */
    dY[4][0] = k2a * y; dY[4][1] = k2a * x;
    /* Y5 = -k2a y z */
    dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    /* Y6 = k2b (2 z^2 - x^2 - y^2) */
    dY[6][0] = -2.0 * k2b * x; dY[6][1] = -2.0 * k2b * y; dY[6][2] = 4.0 * k2b * z;
    /* Y7 = -k2a x z */
    dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
    /* Y8 = k2c (x^2 - y^2) */
    dY[8][0] = 2.0 * k2c * x; dY[8][1] = -2.0 * k2c * y;
    if (degree < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    /* Y9 = -k3a (3 x^2 y - y^3) */
    dY[9][0] = -k3a * 6.0 * x * y; dY[9][1] = -k3a * (3.0 * x * x - 3.0 * y * y);
    /* Y10 = k3b x y z */
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    /* Y11 = -k3c y (4 z^2 - x^2 - y^2) = -k3c (4 y z^2 - x^2 y - y^3) */
    dY[11][0] = -k3c * (-2.0 * x * y);
    dY[11][1] = -k3c * (4.0 * z * z - x * x - 3.0 * y * y);
    dY[11][2] = -k3c * (8.0 * y * z);
    /* Y12 = k3d z (2 z^2 - 3 x^2 - 3 y^2) = k3d (2 z^3 - 3 x^2 z - 3 y^2 z) */
    dY[12][0] = k3d * (-6.0 * x * z);
    dY[12][1] = k3d * (-6.0 * y * z);
    dY[12][2] = k3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    /* Y13 = -k3c x (4 z^2 - x^2 - y^2) = -k3c (4 x z^2 - x^3 - x y^2) */
    dY[13][0] = -k3c * (4.0 * z * z - 3.0 * x * x - y * y);
    dY[13][1] = -k3c * (-2.0 * x * y);
    dY[13][2] = -k3c * (8.0 * x * z);
    /* Y14 = k3e z (x^2 - y^2) */
    dY[14][0] = k3e * 2.0 * x * z; dY[14][1] = -k3e * 2.0 * y * z; dY[14][2] = k3e * (x * x - y * y);
    /* Y15 = -k3a (x^3 - 3 x y^2) */
    dY[15][0] = -k3a * (3.0 * x * x - 3.0 * y * y); dY[15][1] = -k3a * (-6.0 * x * y);
}

/* Rotation matrix of a unit quaternion (w,x,y,z). */
static void quat_to_rot(const double q[4], double Rq[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    Rq[0][0] = 1.0 - 2.0 * (y * y + z * z);
    Rq[0][1] = 2.0 * (x * y - w * z);
    Rq[0][2] = 2.0 * (x * z + w * y);
    Rq[1][0] = 2.0 * (x * y + w * z);
    Rq[1][1] = 1.0 - 2.0 * (x * x + z * z);
    Rq[1][2] = 2.0 * (y * z - w * x);
    Rq[2][0] = 2.0 * (x * z - w * y);
    Rq[2][1] = 2.0 * (y * z + w * x);
    Rq[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* dRq[i][j][c] = d Rq_ij / d q_c, c over (w,x,y,z), for the formula above. */
static void quat_to_rot_jac(const double q[4], double dR[3][3][4]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    memset(dR, 0, sizeof(double) * 36);
    /* R00 = 1 - 2(y^2+z^2) */
    dR[0][0][2] = -4.0 * y; dR[0][0][3] = -4.0 * z;
    /* R01 = 2(xy - wz) */
    dR[0][1][0] = -2.0 * z; dR[0][1][1] = 2.0 * y; dR[0][1][2] = 2.0 * x; dR[0][1][3] = -2.0 * w;
    /* R02 = 2(xz + wy) */
    dR[0][2][0] = 2.0 * y; dR[0][2][1] = 2.0 * z; dR[0][2][2] = 2.0 * w; dR[0][2][3] = 2.0 * x;
    /* R10 = 2(xy + wz) */
    dR[1][0][0] = 2.0 * z; dR[1][0][1] = 2.0 * y; dR[1][0][2] = 2.0 * x; dR[1][0][3] = 2.0 * w;
    /* R11 = 1 - 2(x^2+z^2) */
    dR[1][1][1] = -4.0 * x; dR[1][1][3] = -4.0 * z;
    /* R12 = 2(yz - wx) */
    dR[1][2][0] = -2.0 * x; dR[1][2][1] = -2.0 * w; dR[1][2][2] = 2.0 * z; dR[1][2][3] = 2.0 * y;
    /* R20 = 2(xz - wy) */
    dR[2][0][0] = -2.0 * y; dR[2][0][1] = 2.0 * z; dR[2][0][2] = -2.0 * w; dR[2][0][3] = 2.0 * x;
    /* R21 = 2(yz + wx) */
    dR[2][1][0] = 2.0 * x; dR[2][1][1] = 2.0 * w; dR[2][1][2] = 2.0 * z; dR[2][1][3] = 2.0 * y;
    /* R22 = 1 - 2(x^2+y^2) */
    dR[2][2][1] = -4.0 * x; dR[2][2][2] = -4.0 * y;
}

/* Exported for the tests: the SH basis at one direction. */
void oracle_sh_basis(int degree, const double *dir, double *out) {
    sh_basis(degree, dir[0], dir[1], dir[2], out);
}

/* Per-Gaussian intermediate quantities of the projection, kept so that the
 * backward can walk the same chain in reverse. */
typedef struct {
    int visible;
    double xc[3];    /* camera-space mean */
    double qn[4];    /* normalised quaternion */
    double qnorm;    /* |q| */
    double Rq[3][3]; /* rotation of the Gaussian */
    double s[3];     /* exp(log_scale) */
    double M[3][3];  /* Rq diag(s) */
    double Sig[3][3];/* 3D covariance M M^T */
    double u, v;     /* x/z, y/z after the Jacobian clamp */
    int u_clamped, v_clamped;
    double J[2][3];
    double T[2][3];  /* J W, W the camera rotation */
    double cov[3];   /* a, b, c of the dilated 2D covariance */
    double det;
    double conic[3];
    double dir[3], dist; /* unit view direction and distance to the camera centre */
    double rgb[3];
    int clamped[3];
    double opacity;
    double mean2d[2];
} proj_t;

static int project_one(int i, int n, int degree, const double *means, const double *log_scales,
                       const double *quats, const double *opacity_logits, const double *sh,
                       const double *cam, int W, int H, double near_z, proj_t *P, int *guard) {
    const double *R = cam, *t = cam + 9;
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const double *x = means + 3 * i;
    memset(P, 0, sizeof(*P));
    *guard = 0;
    for (int r = 0; r < 3; r++)
        P->xc[r] = R[3 * r + 0] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];
    double z = P->xc[2];
    int finite = isfinite(P->xc[0]) && isfinite(P->xc[1]) && isfinite(z);
    for (int k = 0; k < 3; k++) finite = finite && isfinite(log_scales[3 * i + k]);
    for (int k = 0; k < 4; k++) finite = finite && isfinite(quats[4 * i + k]);
    finite = finite && isfinite(opacity_logits[i]);
    if (!finite) return 0;
    if (fabs(z - near_z) < OR_G_NEAR * fmax(1.0, fabs(z))) *guard |= OR_GUARD_NEAR;
    {
        /* The sort key is the FP32 value nearest to z; flag z when it lies
         * next to the midpoint between two FP32 neighbours. */
        float zf = (float)z;
        double up = 0.5 * ((double)zf + (double)nextafterf(zf, INFINITY));
        double dn = 0.5 * ((double)zf + (double)nextafterf(zf, -INFINITY));
        if (fabs(z - up) < OR_G_DEPTH * fabs(z) || fabs(z - dn) < OR_G_DEPTH * fabs(z))
            *guard |= OR_GUARD_DEPTH;
    }
    /* Reading: cull a Gaussian whose centre is not beyond the near plane. */
    if (!(z > near_z)) return 0;

    /* Rotation and scale -> 3D covariance Sigma = Rq S S^T Rq^T. */
    const double *q = quats + 4 * i;
    double qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(qn2 > 0.0)) return 0;
    P->qnorm = sqrt(qn2);
    for (int k = 0; k < 4; k++) P->qn[k] = q[k] / P->qnorm;
    quat_to_rot(P->qn, P->Rq);
    for (int k = 0; k < 3; k++) P->s[k] = exp(log_scales[3 * i + k]);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) P->M[r][c] = P->Rq[r][c] * P->s[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += P->M[r][k] * P->M[c][k];
            P->Sig[r][c] = acc;
        }

    /* Local affine approximation of the perspective projection (EWA
     * splatting).  Reading: x/z and y/z are clamped to 1.3 times the image
     * extent on each side of the principal point before forming J. */
    double u0 = P->xc[0] / z, v0 = P->xc[1] / z;
    double ulo = -OR_CLIP * cx / fx, uhi = OR_CLIP * (W - cx) / fx;
    double vlo = -OR_CLIP * cy / fy, vhi = OR_CLIP * (H - cy) / fy;
    P->u = u0; P->v = v0;
    if (u0 < ulo) { P->u = ulo; P->u_clamped = 1; }
    if (u0 > uhi) { P->u = uhi; P->u_clamped = 1; }
    if (v0 < vlo) { P->v = vlo; P->v_clamped = 1; }
    if (v0 > vhi) { P->v = vhi; P->v_clamped = 1; }
    if (fabs(u0 - ulo) < OR_G_CLAMP || fabs(u0 - uhi) < OR_G_CLAMP || fabs(v0 - vlo) < OR_G_CLAMP ||
        fabs(v0 - vhi) < OR_G_CLAMP)
        *guard |= OR_GUARD_KINK;
    P->J[0][0] = fx / z; P->J[0][1] = 0.0; P->J[0][2] = -fx * P->u / z;
    P->J[1][0] = 0.0; P->J[1][1] = fy / z; P->J[1][2] = -fy * P->v / z;
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += P->J[r][k] * R[3 * k + c];
            P->T[r][c] = acc;
        }
    /* 2D covariance T Sigma T^T, plus the 0.3 px^2 low-pass dilation. */
    double C2[2][2];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += P->T[r][k] * P->Sig[k][l] * P->T[c][l];
            C2[r][c] = acc;
        }
    P->cov[0] = C2[0][0] + OR_DILATION;
    P->cov[1] = C2[0][1];
    P->cov[2] = C2[1][1] + OR_DILATION;
    P->det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (P->det < OR_G_NEAR * P->cov[0] * P->cov[2]) *guard |= OR_GUARD_DET;
    if (!(P->det > 0.0)) return 0;
    P->conic[0] = P->cov[2] / P->det;
    P->conic[1] = -P->cov[1] / P->det;
    P->conic[2] = P->cov[0] / P->det;

    P->mean2d[0] = fx * P->xc[0] / z + cx;
    P->mean2d[1] = fy * P->xc[1] / z + cy;

    /* Colour: SH evaluated along the unit direction from the camera centre
     * to the mean; colour = max(0, sum + 0.5). */
    double cc[3];
    for (int k = 0; k < 3; k++) cc[k] = -(R[0 + k] * t[0] + R[3 + k] * t[1] + R[6 + k] * t[2]);
    double d[3] = {x[0] - cc[0], x[1] - cc[1], x[2] - cc[2]};
    P->dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; k++) P->dir[k] = P->dist > 0.0 ? d[k] / P->dist : 0.0;
    int K = (degree + 1) * (degree + 1);
    double Y[16];
    sh_basis(degree, P->dir[0], P->dir[1], P->dir[2], Y);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += Y[k] * sh[((size_t)k * n + i) * 3 + ch];
        acc += 0.5;
        if (fabs(acc) < OR_G_CLAMP) *guard |= OR_GUARD_KINK;
        P->clamped[ch] = acc < 0.0;
        P->rgb[ch] = acc < 0.0 ? 0.0 : acc;
    }
    P->opacity = 1.0 / (1.0 + exp(-opacity_logits[i]));
    P->visible = 1;
    return 1;
}

/*
 * Projection of every Gaussian into one view (paper Sec. II: the Gaussians
 * are mapped onto the image plane; Sec. III-B: original 3DGS rasteriser).
 * Outputs per Gaussian: mean2d, depth (camera z), cov2d (a,b,c dilated),
 * conic (inverse of cov2d), opacity, rgb, colour-clamp mask, radius
 * r = ceil(3 sqrt(lambda_max)), tile rect [x0,y0,x1,y1) and tiles_touched.
 * A culled Gaussian has tiles_touched = 0 and rect 0; one culled only
 * because its rect is empty keeps its other outputs.
 * Returns the number of visible Gaussians.
 */
int oracle_project(int n, int degree, const double *means, const double *log_scales,
                   const double *quats, const double *opacity_logits, const double *sh,
                   const double *cam, int W, int H, int tile_w, int tile_h, double near_z,
                   double *mean2d, double *depth, double *cov2d, double *conic, double *opacity,
                   double *rgb, int *clamped, int *radius, int *rect, int *tiles_touched,
                   int *guard, int tight) {
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    int nvis = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : nvis)
    for (int i = 0; i < n; i++) {
        proj_t P;
        int g = 0;
        int ok = project_one(i, n, degree, means, log_scales, quats, opacity_logits, sh, cam, W, H,
                             near_z, &P, &g);
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0;
        depth[i] = P.xc[2];
        for (int k = 0; k < 3; k++) {
            cov2d[3 * i + k] = conic[3 * i + k] = rgb[3 * i + k] = 0.0;
            clamped[3 * i + k] = 0;
        }
        opacity[i] = 0.0;
        radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        tiles_touched[i] = 0;
        if (ok) {
            int rc[4], r;
            int area = tile_rect(P.mean2d, P.cov, P.det, P.opacity, tile_w, tile_h, tiles_x,
                                 tiles_y, tight, rc, &r, &g);
            /* Screen-space quantities are reported for every Gaussian that
             * survives the near-plane and determinant tests, so that callers
             * can locate one whose rect came out empty. */
            mean2d[2 * i] = P.mean2d[0];
            mean2d[2 * i + 1] = P.mean2d[1];
            for (int k = 0; k < 3; k++) {
                cov2d[3 * i + k] = P.cov[k];
                conic[3 * i + k] = P.conic[k];
                rgb[3 * i + k] = P.rgb[k];
                clamped[3 * i + k] = P.clamped[k];
            }
            opacity[i] = P.opacity;
            radius[i] = r;
            if (area > 0) {
                for (int k = 0; k < 4; k++) rect[4 * i + k] = rc[k];
                tiles_touched[i] = area;
                nvis++;
            }
        }
        guard[i] = g;
    }
    return nvis;
}

/* ------------------------------------------------------------------------ */
/* Binning: the per-tile list of Gaussians in (depth, index) order.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t tile;
    float depth;
    int32_t idx;
} inst_t;

static int inst_cmp(const void *pa, const void *pb) {
    const inst_t *a = (const inst_t *)pa, *b = (const inst_t *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/*
 * For each tile of the grid (tile id = ty * tiles_x + tx), the Gaussians
 * whose rect contains it, ordered by the FP32 depth value and then by
 * Gaussian index (paper Sec. II: depth sorting; ties by index is the
 * reading that makes the order unique).  Gaussians with tiles_touched = 0
 * are absent.  tile_start has tiles_x*tiles_y+1 entries; list receives the
 * Gaussian indices (capacity given by list_cap).  Returns the total number
 * of instances, or -1 when list_cap is too small.
 */
int64_t oracle_bin(int n, const float *depth_key, const int *rect, const int *tiles_touched,
                   int tiles_x, int tiles_y, int64_t *tile_start, int32_t *list,
                   int64_t list_cap) {
    int64_t total = 0;
    for (int i = 0; i < n; i++) {
        total += tiles_touched[i];
        if (tiles_touched[i] > 0 &&
            tiles_touched[i] != (rect[4 * i + 2] - rect[4 * i + 0]) * (rect[4 * i + 3] - rect[4 * i + 1]))
            return -2; /* counts that are not the rect areas: not this function's lists */
    }
    if (total > list_cap) return -1;
    inst_t *buf = (inst_t *)malloc(sizeof(inst_t) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int i = 0; i < n; i++) {
        if (tiles_touched[i] <= 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ty++)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; tx++) {
                buf[k].tile = (int64_t)ty * tiles_x + tx;
                buf[k].depth = depth_key[i];
                buf[k].idx = i;
                k++;
            }
    }
    qsort(buf, (size_t)total, sizeof(inst_t), inst_cmp);
    int64_t T = (int64_t)tiles_x * tiles_y;
    int64_t p = 0;
    for (int64_t t = 0; t < T; t++) {
        tile_start[t] = p;
        while (p < total && buf[p].tile == t) {
            list[p] = buf[p].idx;
            p++;
        }
    }
    tile_start[T] = total;
    free(buf);
    return total;
}

/* The same with tight rects (reading C19): each Gaussian's tiles are the row
 * spans of its rect (row_span), from its projected mean, 2D covariance and
 * opacity. */
int64_t oracle_bin_spans(int n, const float *depth_key, const int *rect, const int *tiles_touched,
                         const double *mean2d, const double *cov2d, const double *opacity,
                         int tile_w, int tile_h, int tiles_x, int tiles_y, int64_t *tile_start,
                         int32_t *list, int64_t list_cap) {
    int64_t total = 0;
    for (int i = 0; i < n; i++) total += tiles_touched[i];
    if (total > list_cap) return -1;
    inst_t *buf = (inst_t *)malloc(sizeof(inst_t) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int i = 0; i < n; i++) {
        if (tiles_touched[i] <= 0) continue;
        const double t = tight_level(opacity[i]);
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ty++) {
            int x0 = rect[4 * i + 0], x1 = rect[4 * i + 2], g = 0;
            row_span(mean2d + 2 * i, cov2d + 3 * i, t, ty, tile_w, tile_h, rect[4 * i + 0],
                     rect[4 * i + 2], &x0, &x1, &g);
            for (int tx = x0; tx < x1; tx++) {
                if (k == total) { free(buf); return -2; } /* spans disagree with the count */
                buf[k].tile = (int64_t)ty * tiles_x + tx;
                buf[k].depth = depth_key[i];
                buf[k].idx = i;
                k++;
            }
        }
    }
    if (k != total) { free(buf); return -2; }
    qsort(buf, (size_t)total, sizeof(inst_t), inst_cmp);
    int64_t T = (int64_t)tiles_x * tiles_y;
    int64_t p = 0;
    for (int64_t tt = 0; tt < T; tt++) {
        tile_start[tt] = p;
        while (p < total && buf[p].tile == tt) {
            list[p] = buf[p].idx;
            p++;
        }
    }
    tile_start[T] = total;
    free(buf);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Front-to-back compositing of one pixel.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int idx;       /* Gaussian index */
    double alpha;  /* alpha after clamping */
    double T;      /* transmittance in front of this Gaussian */
    double G;      /* exp(power) */
    double dx, dy; /* mean2d - pixel */
    int clamped;   /* alpha hit the 0.99 clamp */
} contrib_t;

/*
 * Composite the list entries [0, len) of one pixel at integer coordinates
 * (px, py) (reading: a pixel is sampled at its integer coordinates, in the
 * frame where mean2d = (fx x/z + cx, fy y/z + cy)).  For each entry in
 * order: power = -(a dx^2 + c dy^2)/2 - b dx dy; skip when power > 0;
 * alpha = min(0.99, o e^power); skip when alpha < 1/255; stop before the
 * Gaussian whose inclusion would take T below 1e-4; otherwise add
 * alpha T rgb and multiply T by (1 - alpha).
 * Fills cs[] with the included Gaussians and returns their count; *last is
 * one past the list position of the last included one (0 if none), *neval
 * the number of entries examined, *gpx the guard bits of the pixel.  When
 * gguard is given, each guard bit is also set on the Gaussian whose own
 * decision it is (gguard[index]), so that the Gaussians whose inclusion at
 * some pixel FP32 may decide the other way can be named.
 */
static int composite_pixel(const int32_t *ids, int64_t len, double px, double py,
                           const double *mean2d, const double *conic, const double *opacity,
                           contrib_t *cs, double *T_out, int *last, int *neval, int *gpx,
                           int32_t *gguard) {
    double T = 1.0;
    int nc = 0;
    *last = 0;
    *gpx = 0;
    int64_t j;
    for (j = 0; j < len; j++) {
        int g = ids[j];
        double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
        double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        int gb = 0;
        if (fabs(power) < OR_G_POWER) gb |= OR_GPX_POWER;
        if (power > 0.0) {
            *gpx |= gb;
            if (gguard && gb) {
#pragma omp atomic update
                gguard[g] |= gb;
            }
            continue;
        }
        double G = exp(power);
        double oG = opacity[g] * G;
        if (fabs(oG * 255.0 - 1.0) < OR_G_ALPHA) gb |= OR_GPX_ALPHA;
        if (fabs(oG / OR_ALPHA_MAX - 1.0) < OR_G_CLAMP) gb |= OR_GPX_KINK;
        double alpha = oG < OR_ALPHA_MAX ? oG : OR_ALPHA_MAX;
        double Tn = T * (1.0 - alpha);
        if (alpha >= OR_ALPHA_MIN && fabs(Tn / OR_T_MIN - 1.0) < OR_G_TRANS) gb |= OR_GPX_TRANS;
        *gpx |= gb;
        if (gguard && gb) {
#pragma omp atomic update
            gguard[g] |= gb;
        }
        if (alpha < OR_ALPHA_MIN) continue;
        if (Tn < OR_T_MIN) { j++; break; }
        cs[nc].idx = g;
        cs[nc].alpha = alpha;
        cs[nc].T = T;
        cs[nc].G = G;
        cs[nc].dx = dx;
        cs[nc].dy = dy;
        cs[nc].clamped = !(oG < OR_ALPHA_MAX);
        nc++;
        T = Tn;
        *last = (int)(j + 1);
    }
    *neval = (int)j;
    *T_out = T;
    return nc;
}

/*
 * Render one view from per-tile lists (tile_start/list as produced by
 * oracle_bin).  channels = 3 writes RGB; channels = 1 writes the mean of the
 * three composited channels (reading for grayscale views: compositing is
 * linear, so this equals compositing the per-Gaussian mean colour).  The
 * background bg[3] enters as T_final * bg.  Outputs image[channels][H][W], final_T[H][W],
 * last_idx[H][W], n_eval[H][W], n_included[H][W] and guard_px[H][W]; and, if
 * guard_g is given, guard_g[n]: the OR over pixels of the guard bits of each
 * Gaussian's own decisions (zeroed first).
 */
void oracle_render(int n, const double *mean2d, const double *conic, const double *opacity,
                   const double *rgb, const int64_t *tile_start,
                   const int32_t *list, int W, int H, int tile_w, int tile_h, int channels,
                   const double *bg, double *image, double *final_T, int32_t *last_idx,
                   int32_t *n_eval, int32_t *n_included, int32_t *guard_px, int32_t *guard_g) {
    if (guard_g)
        for (int i = 0; i < n; i++) guard_g[i] = 0;
    const int tiles_x = (W + tile_w - 1) / tile_w;
    int64_t maxlen = 0;
    int64_t T_tiles = (int64_t)tiles_x * ((H + tile_h - 1) / tile_h);
    for (int64_t t = 0; t < T_tiles; t++)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
#pragma omp parallel
    {
    contrib_t *cs = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(maxlen + 1));
#pragma omp for schedule(dynamic, 1)
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int64_t t = (int64_t)(py / tile_h) * tiles_x + px / tile_w;
            const int32_t *ids = list + tile_start[t];
            int64_t len = tile_start[t + 1] - tile_start[t];
            double T;
            int last, ne, gp;
            int nc = composite_pixel(ids, len, px, py, mean2d, conic, opacity, cs, &T, &last,
                                     &ne, &gp, guard_g);
            double C[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < nc; k++)
                for (int ch = 0; ch < 3; ch++) C[ch] += cs[k].alpha * cs[k].T * rgb[3 * cs[k].idx + ch];
            for (int ch = 0; ch < 3; ch++) C[ch] += T * bg[ch];
            size_t p = (size_t)py * W + px;
            if (channels == 3) {
                for (int ch = 0; ch < 3; ch++) image[(size_t)ch * W * H + p] = C[ch];
            } else {
                image[p] = (C[0] + C[1] + C[2]) / 3.0;
            }
            final_T[p] = T;
            last_idx[p] = last;
            n_eval[p] = ne;
            n_included[p] = nc;
            guard_px[p] = gp;
        }
    free(cs);
    }
}

/* Sort helper for the brute-force renderer: (depth key, index). */
typedef struct {
    float depth;
    int32_t idx;
} dk_t;
static int dk_cmp(const void *pa, const void *pb) {
    const dk_t *a = (const dk_t *)pa, *b = (const dk_t *)pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/*
 * Brute-force renderer: no tile lists and no radix sort.  Every visible
 * Gaussian is sorted once by (FP32 depth, index); each pixel then walks that
 * whole order and admits a Gaussian iff rect is NULL or the pixel's tile
 * lies inside the Gaussian's rect.  With rect given, it must equal
 * oracle_render; with rect NULL it is the tile-free reference.
 */
void oracle_render_brute(int n, const double *mean2d, const double *conic, const double *opacity,
                         const double *rgb, const float *depth_key, const int *tiles_touched,
                         const int *rect, int W, int H, int tile_w, int tile_h, int channels,
                         const double *bg, double *image, double *final_T, int32_t *n_included) {
    dk_t *ord = (dk_t *)malloc(sizeof(dk_t) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; i++)
        if (tiles_touched[i] > 0) {
            ord[m].depth = depth_key[i];
            ord[m].idx = i;
            m++;
        }
    qsort(ord, (size_t)m, sizeof(dk_t), dk_cmp);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    contrib_t *cs = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(m + 1));
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int tx = px / tile_w, ty = py / tile_h;
            int len = 0;
            for (int k = 0; k < m; k++) {
                int g = ord[k].idx;
                if (rect && !(tx >= rect[4 * g] && tx < rect[4 * g + 2] && ty >= rect[4 * g + 1] &&
                              ty < rect[4 * g + 3]))
                    continue;
                ids[len++] = g;
            }
            double T;
            int last, ne, gp;
            int nc = composite_pixel(ids, len, px, py, mean2d, conic, opacity, cs, &T, &last,
                                     &ne, &gp, NULL);
            double C[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < nc; k++)
                for (int ch = 0; ch < 3; ch++) C[ch] += cs[k].alpha * cs[k].T * rgb[3 * cs[k].idx + ch];
            for (int ch = 0; ch < 3; ch++) C[ch] += T * bg[ch];
            size_t p = (size_t)py * W + px;
            if (channels == 3) {
                for (int ch = 0; ch < 3; ch++) image[(size_t)ch * W * H + p] = C[ch];
            } else {
                image[p] = (C[0] + C[1] + C[2]) / 3.0;
            }
            final_T[p] = T;
            n_included[p] = nc;
        }
    free(cs);
    free(ids);
    free(ord);
}

/*
 * Adjoint of oracle_render.  For every pixel the forward is re-run and every
 * included Gaussian's transmittance T_i is kept exactly.  With the output
 * C = sum_i alpha_i T_i c_i + T_final bg and g = dL/dC:
 *   dL/dc_i     = alpha_i T_i g
 *   dL/dalpha_i = g . (T_i c_i - S_i / (1 - alpha_i)),
 *                 S_i = sum_{j>i} alpha_j T_j c_j + T_final bg
 * alpha = min(0.99, o G), G = exp(power): when unclamped, dL/do = G dL/dalpha
 * and dL/dpower = o G dL/dalpha; a clamped alpha passes no gradient.
 * power = -(a dx^2 + c dy^2)/2 - b dx dy with d = mean2d - pixel gives the
 * mean2d and conic gradients.  A grayscale view spreads g/3 to each channel.
 * Gradients are accumulated (+=) into dmean2d[n][2], dconic[n][3],
 * dopacity[n], drgb[n][3].
 */
void oracle_render_bwd(int n, const double *mean2d, const double *conic, const double *opacity,
                       const double *rgb, const int64_t *tile_start, const int32_t *list, int W,
                       int H, int tile_w, int tile_h, int channels, const double *bg,
                       const double *dL_dimg, double *dmean2d, double *dconic, double *dopacity,
                       double *drgb, double *dmean2d_abs) {
    (void)n;
    const int tiles_x = (W + tile_w - 1) / tile_w;
    int64_t maxlen = 0;
    int64_t T_tiles = (int64_t)tiles_x * ((H + tile_h - 1) / tile_h);
    for (int64_t t = 0; t < T_tiles; t++)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
#pragma omp parallel
    {
    contrib_t *cs = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(maxlen + 1));
#pragma omp for schedule(dynamic, 1)
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int64_t t = (int64_t)(py / tile_h) * tiles_x + px / tile_w;
            const int32_t *ids = list + tile_start[t];
            int64_t len = tile_start[t + 1] - tile_start[t];
            double T;
            int last, ne, gp;
            int nc = composite_pixel(ids, len, px, py, mean2d, conic, opacity, cs, &T, &last,
                                     &ne, &gp, NULL);
            size_t p = (size_t)py * W + px;
            double g[3];
            if (channels == 3) {
                for (int ch = 0; ch < 3; ch++) g[ch] = dL_dimg[(size_t)ch * W * H + p];
            } else {
                for (int ch = 0; ch < 3; ch++) g[ch] = dL_dimg[p] / 3.0;
            }
            double S[3] = {T * bg[0], T * bg[1], T * bg[2]};
            for (int k = nc - 1; k >= 0; k--) {
                int gi = cs[k].idx;
                const double *c = rgb + 3 * gi;
                double al = cs[k].alpha, Ti = cs[k].T;
                double dal = 0.0;
                /* (the adds into a Gaussian's gradient are atomic only so
                 * that several threads may run; one thread adds in order) */
                for (int ch = 0; ch < 3; ch++) {
#pragma omp atomic update
                    drgb[3 * gi + ch] += al * Ti * g[ch];
                    dal += g[ch] * (Ti * c[ch] - S[ch] / (1.0 - al));
                }
                for (int ch = 0; ch < 3; ch++) S[ch] += al * Ti * c[ch];
                if (cs[k].clamped) continue;
                double o = opacity[gi];
#pragma omp atomic update
                dopacity[gi] += cs[k].G * dal;
                double dpow = o * cs[k].G * dal;
                double a = conic[3 * gi], b = conic[3 * gi + 1], cc = conic[3 * gi + 2];
                double dx = cs[k].dx, dy = cs[k].dy;
                const double gx = dpow * (-(a * dx + b * dy));
                const double gy = dpow * (-(b * dx + cc * dy));
#pragma omp atomic update
                dmean2d[2 * gi] += gx;
#pragma omp atomic update
                dmean2d[2 * gi + 1] += gy;
                /* Homodirectional view-space gradient (AbsGS, the density
                 * control of paper Sec. III-B): the per-pixel contributions
                 * summed by absolute value, component by component, so that
                 * contributions of opposite sign do not cancel. */
                if (dmean2d_abs) {
#pragma omp atomic update
                    dmean2d_abs[2 * gi] += fabs(gx);
#pragma omp atomic update
                    dmean2d_abs[2 * gi + 1] += fabs(gy);
                }
#pragma omp atomic update
                dconic[3 * gi] += dpow * (-0.5 * dx * dx);
#pragma omp atomic update
                dconic[3 * gi + 1] += dpow * (-dx * dy);
#pragma omp atomic update
                dconic[3 * gi + 2] += dpow * (-0.5 * dy * dy);
            }
        }
    free(cs);
    }
}

/*
 * Adjoint of oracle_project for one view: from the screen-space gradients
 * (dmean2d, dconic, dopacity, drgb) to the parameter gradients, accumulated
 * (+=) into gmeans[n][3], glog_scales[n][3], gquats[n][4],
 * gopacity_logits[n], gsh[K][n][3].  Each step is the chain rule of the
 * corresponding forward step, written out scalar by scalar.
 */
void oracle_project_bwd(int n, int degree, const double *means, const double *log_scales,
                        const double *quats, const double *opacity_logits, const double *sh,
                        const double *cam, int W, int H, int tile_w, int tile_h, double near_z,
                        const double *dmean2d, const double *dconic, const double *dopacity,
                        const double *drgb, double *gmeans, double *glog_scales, double *gquats,
                        double *gopacity_logits, double *gsh, int tight) {
    const double *R = cam;
    const double fx = cam[12], fy = cam[13];
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    const int K = (degree + 1) * (degree + 1);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int i = 0; i < n; i++) {
        proj_t P;
        int gd;
        if (!project_one(i, n, degree, means, log_scales, quats, opacity_logits, sh, cam, W, H,
                         near_z, &P, &gd))
            continue;
        /* Same visibility test as oracle_project: non-empty rect. */
        int rc[4], r, gr = 0;
        if (tile_rect(P.mean2d, P.cov, P.det, P.opacity, tile_w, tile_h, tiles_x, tiles_y, tight,
                      rc, &r, &gr) == 0)
            continue;

        const double z = P.xc[2];
        double gxc[3] = {0.0, 0.0, 0.0};
        double gx_world[3] = {0.0, 0.0, 0.0};

        /* Opacity: o = sigmoid(logit). */
        gopacity_logits[i] += dopacity[i] * P.opacity * (1.0 - P.opacity);

        /* Colour -> SH coefficients and view direction. */
        double Y[16], dY[16][3];
        sh_basis(degree, P.dir[0], P.dir[1], P.dir[2], Y);
        sh_basis_grad(degree, P.dir[0], P.dir[1], P.dir[2], dY);
        double gdir[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 3; ch++) {
            if (P.clamped[ch]) continue;
            double gc = drgb[3 * i + ch];
            for (int k = 0; k < K; k++) {
                gsh[((size_t)k * n + i) * 3 + ch] += Y[k] * gc;
                double shv = sh[((size_t)k * n + i) * 3 + ch];
                for (int e = 0; e < 3; e++) gdir[e] += gc * shv * dY[k][e];
            }
        }
        if (P.dist > 0.0) {
            /* dir = d/|d|: d(dir)/dd = (I - dir dir^T)/|d| */
            double dd = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
            for (int e = 0; e < 3; e++) gx_world[e] += (gdir[e] - P.dir[e] * dd) / P.dist;
        }

        /* mean2d = (fx x/z + cx, fy y/z + cy). */
        gxc[0] += dmean2d[2 * i] * fx / z;
        gxc[1] += dmean2d[2 * i + 1] * fy / z;
        gxc[2] += -dmean2d[2 * i] * fx * P.xc[0] / (z * z) - dmean2d[2 * i + 1] * fy * P.xc[1] / (z * z);

        /* conic = (c, -b, a)/det with det = a c - b^2 over cov = (a, b, c). */
        double a = P.cov[0], b = P.cov[1], c = P.cov[2], det = P.det, det2 = det * det;
        double gA = dconic[3 * i], gB = dconic[3 * i + 1], gC = dconic[3 * i + 2];
        double ga = gA * (-c * c / det2) + gB * (b * c / det2) + gC * (-b * b / det2);
        double gb = gA * (2.0 * b * c / det2) + gB * (-(a * c + b * b) / det2) + gC * (2.0 * a * b / det2);
        double gc2 = gA * (-b * b / det2) + gB * (a * b / det2) + gC * (-a * a / det2);

        /* cov = (T0 Sig T0^T + 0.3, T0 Sig T1^T, T1 Sig T1^T + 0.3). */
        double gSig[3][3];
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++)
                gSig[k][l] = ga * P.T[0][k] * P.T[0][l] + gb * P.T[0][k] * P.T[1][l] +
                             gc2 * P.T[1][k] * P.T[1][l];
        double gT[2][3];
        for (int k = 0; k < 3; k++) {
            double S0 = 0.0, S1 = 0.0; /* (Sig T0^T)_k, (Sig T1^T)_k, Sig symmetric */
            for (int l = 0; l < 3; l++) {
                S0 += P.Sig[k][l] * P.T[0][l];
                S1 += P.Sig[k][l] * P.T[1][l];
            }
            gT[0][k] = 2.0 * ga * S0 + gb * S1;
            gT[1][k] = gb * S0 + 2.0 * gc2 * S1;
        }
        /* T = J W: dJ_rk = sum_c dT_rc W_kc. */
        double gJ[2][3];
        for (int r2 = 0; r2 < 2; r2++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int cc2 = 0; cc2 < 3; cc2++) acc += gT[r2][cc2] * R[3 * k + cc2];
                gJ[r2][k] = acc;
            }
        /* J = [[fx/z, 0, -fx u/z], [0, fy/z, -fy v/z]] with u, v the clamped x/z, y/z. */
        double gz = gJ[0][0] * (-fx / (z * z)) + gJ[0][2] * (fx * P.u / (z * z)) +
                    gJ[1][1] * (-fy / (z * z)) + gJ[1][2] * (fy * P.v / (z * z));
        double gu = gJ[0][2] * (-fx / z), gv = gJ[1][2] * (-fy / z);
        if (!P.u_clamped) {
            gxc[0] += gu / z;
            gz += -gu * P.xc[0] / (z * z);
        }
        if (!P.v_clamped) {
            gxc[1] += gv / z;
            gz += -gv * P.xc[1] / (z * z);
        }
        gxc[2] += gz;

        /* x_c = W x + t: dx = W^T dx_c. */
        for (int e = 0; e < 3; e++)
            gx_world[e] += R[e] * gxc[0] + R[3 + e] * gxc[1] + R[6 + e] * gxc[2];
        for (int e = 0; e < 3; e++) gmeans[3 * i + e] += gx_world[e];

        /* Sig_kl = sum_m M_km M_lm (each entry a function of M). */
        double gM[3][3];
        for (int k = 0; k < 3; k++)
            for (int m = 0; m < 3; m++) {
                double acc = 0.0;
                for (int l = 0; l < 3; l++) acc += (gSig[k][l] + gSig[l][k]) * P.M[l][m];
                gM[k][m] = acc;
            }
        /* M_km = Rq_km s_m. */
        double gRq[3][3];
        for (int m = 0; m < 3; m++) {
            double gs = 0.0;
            for (int k = 0; k < 3; k++) {
                gs += gM[k][m] * P.Rq[k][m];
                gRq[k][m] = gM[k][m] * P.s[m];
            }
            glog_scales[3 * i + m] += gs * P.s[m];
        }
        /* Rq(qn), qn = q/|q|. */
        double dR[3][3][4];
        quat_to_rot_jac(P.qn, dR);
        double gqn[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 3; k++)
            for (int m = 0; m < 3; m++)
                for (int e = 0; e < 4; e++) gqn[e] += gRq[k][m] * dR[k][m][e];
        double dotq = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
        for (int e = 0; e < 4; e++) gquats[4 * i + e] += (gqn[e] - P.qn[e] * dotq) / P.qnorm;
    }
}

/* ------------------------------------------------------------------------ */
/* Photometric loss, Eq. 2.                                                  */
/* Reading: as printed, Eq. 2 adds lambda * SSIM, which would reward a     */
/* dissimilar render, and it has no mean.  It is read as                   */
/*   L = (1 - lambda) mean|I - I_gt| + lambda (1 - mean SSIM(I, I_gt))      */
/* with SSIM of Wang et al.: an 11x11 Gaussian window of sigma 1.5,         */
/* normalised to unit sum, zero padding outside the image, C1 = 0.01^2,     */
/* C2 = 0.03^2, computed per channel and averaged over C*H*W.               */
/* d|x|/dx is taken as 0 at x = 0.                                          */
/* ------------------------------------------------------------------------ */
static void ssim_window(double w[11][11]) {
    double g[11], s = 0.0;
    for (int k = 0; k < 11; k++) {
        double d = k - 5;
        g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k < 11; k++) g[k] /= s;
    for (int a = 0; a < 11; a++)
        for (int b = 0; b < 11; b++) w[a][b] = g[a] * g[b];
}

/* Exported for tests: the 11x11 window. */
void oracle_ssim_window(double *out) {
    double w[11][11];
    ssim_window(w);
    memcpy(out, w, sizeof(w));
}

/*
 * Loss and gradient for one image pair of `channels` planes of H x W.
 * Returns L; writes dL/dimg (may be NULL).  ssim_map (nullable) receives
 * the per-pixel SSIM values.  Every windowed mean is a direct 121-term sum.
 */
double oracle_loss_l1_ssim(const double *img, const double *tgt, int channels, int H, int W,
                           double lambda, double *dimg, double *ssim_map) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double w[11][11];
    ssim_window(w);
    const size_t HW = (size_t)H * W;
    const double M = (double)channels * HW;
    double l1 = 0.0, ssum = 0.0;
    /* Per-pixel partial derivatives of SSIM with respect to the window
     * moments mu_x, E[x^2], E[xy]. */
    double *dm = (double *)calloc(HW, sizeof(double));
    double *dxx = (double *)calloc(HW, sizeof(double));
    double *dxy = (double *)calloc(HW, sizeof(double));
    double *rows = (double *)calloc((size_t)H, sizeof(double)); /* SSIM sum per row */
    for (int ch = 0; ch < channels; ch++) {
        const double *x = img + ch * HW, *y = tgt + ch * HW;
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < H; i++) {
            rows[i] = 0.0;
            for (int j = 0; j < W; j++) {
                double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
                for (int a = -5; a <= 5; a++)
                    for (int b = -5; b <= 5; b++) {
                        int ii = i + a, jj = j + b;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        double wt = w[a + 5][b + 5];
                        double xv = x[(size_t)ii * W + jj], yv = y[(size_t)ii * W + jj];
                        mx += wt * xv;
                        my += wt * yv;
                        sxx += wt * xv * xv;
                        syy += wt * yv * yv;
                        sxy += wt * xv * yv;
                    }
                double vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
                double A = 2.0 * mx * my + C1, B = 2.0 * cxy + C2;
                double Cd = mx * mx + my * my + C1, D = vx + vy + C2;
                double s = A * B / (Cd * D);
                rows[i] += s;
                if (ssim_map) ssim_map[ch * HW + (size_t)i * W + j] = s;
                /* partials with respect to (mx, sxx, sxy), my/syy fixed */
                double dA_dmx = 2.0 * my;
                double dB_dmx = -2.0 * my, dB_dsxy = 2.0;
                double dC_dmx = 2.0 * mx;
                double dD_dmx = -2.0 * mx, dD_dsxx = 1.0;
                double ds_dmx = (dA_dmx * B + A * dB_dmx) / (Cd * D) -
                                s * (dC_dmx / Cd + dD_dmx / D);
                double ds_dsxx = -s * dD_dsxx / D;
                double ds_dsxy = A * dB_dsxy / (Cd * D);
                size_t p = (size_t)i * W + j;
                dm[p] = ds_dmx;
                dxx[p] = ds_dsxx;
                dxy[p] = ds_dsxy;
            }
        }
        for (int i = 0; i < H; i++) ssum += rows[i];
        for (size_t p = 0; p < HW; p++) l1 += fabs(x[p] - y[p]);
        if (dimg) {
            /* dSSIM_sum/dx_q = sum_p w(p-q) [dm_p + 2 x_q dxx_p + y_q dxy_p] */
#pragma omp parallel for schedule(dynamic, 1)
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++) {
                    double acc_m = 0, acc_xx = 0, acc_xy = 0;
                    for (int a = -5; a <= 5; a++)
                        for (int b = -5; b <= 5; b++) {
                            int ii = i + a, jj = j + b;
                            if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                            double wt = w[a + 5][b + 5];
                            size_t p = (size_t)ii * W + jj;
                            acc_m += wt * dm[p];
                            acc_xx += wt * dxx[p];
                            acc_xy += wt * dxy[p];
                        }
                    size_t q = (size_t)i * W + j;
                    double dssim = acc_m + 2.0 * x[q] * acc_xx + y[q] * acc_xy;
                    double diff = x[q] - y[q];
                    double sgn = diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0);
                    dimg[ch * HW + q] = (1.0 - lambda) * sgn / M - lambda * dssim / M;
                }
        }
    }
    free(dm);
    free(dxx);
    free(dxy);
    free(rows);
    return (1.0 - lambda) * l1 / M + lambda * (1.0 - ssum / M);
}

/* ------------------------------------------------------------------------ */
/* Adam (paper Sec. IV-A: the default 3DGS optimiser configuration).        */
/* One step t (1-based) over n elements:                                    */
/*   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;                           */
/*   p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)              */
/* ------------------------------------------------------------------------ */
void oracle_adam(int64_t n, double *p, const double *g, double *m, double *v, double lr,
                 double b1, double b2, double eps, int t) {
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);
    }
}
