/*
 * gsta_oracle.c -- a plain, slow FP64 CPU statement of one GSta training step
 * (3-D Gaussian splatting with gradient-norm freezing).
 *
 * TEST INFRASTRUCTURE. This library is the parity reference for the CUDA
 * path. Only the test-suite, the package smoke check and the benchmark's
 * CPU-baseline leg load it; the product never does. It shares no code,
 * header, table or constant generator with the CUDA sources.
 *
 * Paper: "GSta: Efficient Training Scheme with Siestaed Gaussians for
 * Monocular 3D Scene Reconstruction" (arXiv 2504.06716).
 *
 *   Sec. 3.1, Eq. 1   projected 2-D Gaussian (EWA splatting)   or_project
 *   Sec. 3.1          SH view-dependent colour                 or_sh_basis
 *   Sec. 3.1          blending "in a sorted order"             or_sort
 *   Sec. 3.1, Eq. 2   front-to-back alpha compositing          or_render, or_render_brute
 *   Sec. 3.1, Eq. 3   L = (1 - 0.2) L1 + 0.2 D-SSIM            or_loss
 *   Sec. 3.2.4        backward skips frozen Gaussians          or_render_bwd, or_project_bwd
 *   Sec. 3.2.1, Eq. 4-6  per-Gaussian freeze decision          or_freeze_update
 *   Sec. 3.2.4        optimiser updates unfrozen Gaussians     or_adam
 *   Sec. 3.2.2, Eq. 7 PSNR on a training subset                or_psnr
 *
 * The paper cites EWA splatting and 3DGS for the renderer and does not write
 * its internals out. The readings taken here (camera model, dilation,
 * 3-sigma radius, tile rule, alpha and transmittance cut-offs, SH offset and
 * clamp, SSIM window) are stated at each function and are shared with the
 * CUDA path only through their written statement.
 *
 * Loops over independent Gaussians, pixels or tiles run on all host cores
 * (OpenMP); every sum is taken in an order that does not depend on the
 * number of threads, so results are the same with one core or many.
 *
 * Every computation is a direct loop in double precision. Where a floating
 * point value decides an integer that the CUDA path must reproduce bit for
 * bit (the tile rectangle of a Gaussian, the sort key, the freeze test) the
 * decision is taken in single precision, the precision of the kernels.
 *
 * Layouts (all row-major, caller-allocated):
 *   params  [n][59]  0-2 mean, 3-5 log-scale, 6-9 quaternion (w,x,y,z),
 *                    10 opacity logit, 11+3c+ch SH coefficient c, channel ch
 *   mean2d  [n][2], conic [n][3] (a, b, c of [[a,b],[b,c]]), rgb [n][3]
 *   rect    [n][4]   x0, y0, x1, y1 tile rectangle, half-open
 *   image   [3][H][W]
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NP 59

/* Planted mistakes, for the test that shows the pins catch them
 * (tests/test_oracle_mutants.py): a build with -DORACLE_PLANT=k, k >= 1,
 * changes the one step marked PLANTED(k) below. Every normal build has
 * ORACLE_PLANT 0, where each PLANTED(k) is the constant 0. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#define PLANTED(k) (ORACLE_PLANT == (k))

typedef struct {
    int32_t width, height, tile, pad0;
    double fx, fy, cx, cy;
    double R[9];      /* world -> camera rotation, row-major */
    double t[3];      /* world -> camera translation */
    double campos[3]; /* camera centre, world space */
    double znear;     /* Gaussians with camera-space z <= znear are culled */
    double dilation;  /* added to both diagonal entries of the 2-D covariance */
    double bg[3];     /* background colour */
} or_camera;

static const double PI = 3.14159265358979323846;

/* Host threads the parallel loops use (the baseline timing reports them). */
void or_set_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : 1); }
int32_t or_max_threads(void) { return (int32_t)omp_get_max_threads(); }

/* ------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3 (Sec. 3.1: "a set of spherical
 * harmonics (SH) coefficients (up to 3 bands)").
 *
 * Textbook definition, built here from Legendre polynomials:
 *   Y_l^0   = K_l^0 P_l(z)
 *   Y_l^{m} = sqrt2 K_l^m cos(m phi) P_l^m(z)        m > 0
 *   Y_l^{-m}= sqrt2 K_l^m sin(m phi) P_l^m(z)        m > 0
 *   K_l^m   = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
 *   P_l^m(z)= (-1)^m (1-z^2)^{m/2} d^m/dz^m P_l(z)   (Condon-Shortley phase)
 * With sin^m(theta) e^{i m phi} = (x + i y)^m this is a polynomial in the
 * unit direction (x, y, z). Coefficient index c = l^2 + l + m.
 * ------------------------------------------------------------------ */

/* Coefficients of P_l (l <= 3) by Bonnet's recurrence. */
static void legendre_coeffs(double P[4][4]) {
    memset(P, 0, sizeof(double) * 16);
    P[0][0] = 1.0;
    P[1][1] = 1.0;
    for (int n = 1; n < 3; ++n) {
        for (int k = 0; k < 4; ++k) {
            double v = -n * P[n - 1][k];
            if (k > 0) v += (2 * n + 1) * P[n][k - 1];
            P[n + 1][k] = v / (n + 1);
        }
    }
}

static double poly_eval(const double *c, int deg, double z) {
    double r = 0.0;
    for (int k = deg; k >= 0; --k) r = r * z + c[k];
    return r;
}

static void poly_deriv(const double *c, double *d) {
    for (int k = 0; k < 3; ++k) d[k] = (k + 1) * c[k + 1];
    d[3] = 0.0;
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* Y[16] and, if dY != NULL, dY[16][3]: the gradient of the polynomial
 * extension above with respect to (x, y, z). */
static void sh_eval(const double dir[3], double *Y, double *dY) {
    double P[4][4];
    legendre_coeffs(P);
    double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= 3; ++l) {
        double Q[4], dQ[4];
        memcpy(Q, P[l], sizeof(Q));
        for (int m = 0; m <= l; ++m) {
            /* Q = d^m P_l / dz^m, dQ = its derivative */
            poly_deriv(Q, dQ);
            double K = sqrt((2 * l + 1) / (4.0 * PI) * (PLANTED(4) ? 1.0 : factorial(l - m) / factorial(l + m)));
            double q = poly_eval(Q, 3, z), dq = poly_eval(dQ, 3, z);
            if (m == 0) {
                int c = l * l + l;
                Y[c] = K * q;
                if (dY) { dY[3 * c] = 0; dY[3 * c + 1] = 0; dY[3 * c + 2] = K * dq; }
            } else {
                /* (x+iy)^m and m (x+iy)^(m-1) */
                double re = 1, im = 0, pre = 1, pim = 0;
                for (int k = 0; k < m; ++k) {
                    if (k == m - 1) { pre = m * re; pim = m * im; }
                    double nre = re * x - im * y, nim = re * y + im * x;
                    re = nre; im = nim;
                }
                double A = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
                int cp = l * l + l + m, cn = l * l + l - m;
                Y[cp] = A * re * q;
                Y[cn] = A * im * q;
                if (dY) {
                    /* d/dx Re = Re(m w^(m-1)), d/dy Re = -Im(m w^(m-1));
                       d/dx Im = Im(m w^(m-1)), d/dy Im =  Re(m w^(m-1)) */
                    dY[3 * cp] = A * pre * q;
                    dY[3 * cp + 1] = -A * pim * q;
                    dY[3 * cp + 2] = A * re * dq;
                    dY[3 * cn] = A * pim * q;
                    dY[3 * cn + 1] = A * pre * q;
                    dY[3 * cn + 2] = A * im * dq;
                }
            }
            memcpy(Q, dQ, sizeof(Q));
        }
    }
}

void or_sh_basis(const double *dir, double *Y) { sh_eval(dir, Y, NULL); }
void or_sh_basis_grad(const double *dir, double *dY) {
    double Y[16];
    sh_eval(dir, Y, dY);
}

/* ------------------------------------------------------------------ */
/* Small dense helpers.                                                */
/* ------------------------------------------------------------------ */
static void matmul(const double *A, const double *B, double *C, int n, int k, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0;
            for (int r = 0; r < k; ++r) s += A[i * k + r] * B[r * m + j];
            C[i * m + j] = s;
        }
}
static void transpose(const double *A, double *T, int n, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dw, dR/dx, dR/dy, dR/dz of the matrix above. */
static void quat_to_rot_grad(const double *q, double dR[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double a[4][9] = {
        {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
        {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
        {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
        {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0},
    };
    memcpy(dR, a, sizeof(a));
}

/* ------------------------------------------------------------------ */
/* Projection (Sec. 3.1, Eq. 1).                                        */
/* ------------------------------------------------------------------ */

/* Tile rectangle of a splat, decided in single precision:
 *   x0 = floor((mx - r) / T), x1 = floor((mx + r) / T), same for y,
 * clipped to the grid; half-open output. Returns the tile count. */
static int32_t tile_rect(float mx, float my, int32_t r, int32_t tile, int32_t tx, int32_t ty, int32_t *rect) {
    float inv = 1.0f / (float)tile; /* exact: the tile size is a power of two */
    float fr = (float)r;
    float x0 = floorf((mx - fr) * inv), x1 = floorf((mx + fr) * inv);
    float y0 = floorf((my - fr) * inv), y1 = floorf((my + fr) * inv);
    if (x0 < 0.0f) x0 = 0.0f;
    if (y0 < 0.0f) y0 = 0.0f;
    if (x1 > (float)(tx - 1)) x1 = (float)(tx - 1);
    if (y1 > (float)(ty - 1)) y1 = (float)(ty - 1);
    if (x0 > x1 || y0 > y1) { rect[0] = rect[1] = rect[2] = rect[3] = 0; return 0; }
    rect[0] = (int32_t)x0; rect[1] = (int32_t)y0;
    rect[2] = (int32_t)x1 + 1; rect[3] = (int32_t)y1 + 1;
    return (rect[2] - rect[0]) * (rect[3] - rect[1]);
}

/* Reading of the tile lists (Sec. 3.1, Eq. 2; 3DGS, which the paper builds
 * on, lists a splat in every tile of its 3-sigma rectangle): a tile of the
 * rectangle lists the splat only if one of its pixel centres inside the image
 * has alpha = o exp(-q/2) >= (1 - LIST_SLACK) / 255, q = d^T Q d with d =
 * pixel - mean and Q the conic. At every other pixel of the rectangle the
 * compositing floor of Eq. 2 skips the splat, so the image and every gradient
 * are those of the full rectangle. The slack lists the splats whose alpha
 * lies just below the floor, where single precision may take the other
 * decision: compositing skips them, but it evaluates them and records how
 * close each decision came (the parity tests' margins). Brute force over the
 * tile's pixels in double precision; the alpha test is taken in the
 * equivalent form q <= 2 ln(255 o / (1 - LIST_SLACK)). */
#define LIST_SLACK 3e-4
static int tile_lists(double mx, double my, double a, double b, double c, double o, int32_t tile, int32_t x,
                      int32_t y, int32_t W, int32_t H) {
    double floor_alpha = (PLANTED(44) ? 1.0 / 128.0 : 1.0 / 255.0) * (1.0 - LIST_SLACK);
    if (!(o >= floor_alpha)) return 0;
    double tau = 2.0 * log(o / floor_alpha);
    int32_t px1 = x * tile + tile < W ? x * tile + tile : W;
    int32_t py1 = y * tile + tile < H ? y * tile + tile : H;
    for (int32_t py = y * tile; py < py1; ++py)
        for (int32_t px = x * tile; px < px1; ++px) {
            double dx = px - mx, dy = py - my;
            if (a * dx * dx + 2.0 * b * dx * dy + c * dy * dy <= tau) return 1;
        }
    return 0;
}

static double frac_dist(double v) { /* distance of v to the nearest integer */
    return fabs(v - floor(v + 0.5));
}

typedef struct {
    int visible;
    double tc[3], s[3], qn[4], qlen, Rq[9], Sigma[9], J[6], Tm[6], cov[4], det, Q[4];
    double mean2d[2];
    int clampx, clampy;
    double cux, cuy;
    double dir[3], dist, Y[16], dY[48], rgb_raw[3], rgb[3], opacity;
    int32_t radius, rect[4];
    double margin;
} gauss_fwd;

/* One Gaussian through the projection.
 * Readings (the paper names EWA splatting and 3DGS without their formulas):
 *  - camera space t = R mu + t_c, culled when t_z <= znear;
 *  - Sigma = R(q/|q|) diag(exp(2 s)) R^T;
 *  - J = [[fx/tz, 0, -fx u/tz], [0, fy/tz, -fy v/tz]] with u = tx/tz and
 *    v = ty/tz clamped to +-1.3 * (W/2)/fx and +-1.3 * (H/2)/fy;
 *  - 2-D covariance J R_c Sigma R_c^T J^T + dilation * I, culled when det <= 0;
 *  - 2-D mean (fx tx/tz + cx, fy ty/tz + cy), pixel (i, j) sits at (i, j);
 *  - radius = ceil(3 sqrt(largest eigenvalue)), tile rectangle as tile_rect;
 *  - opacity = sigmoid(logit); opacity_act = 1 takes |x| instead (the
 *    absolute-value activation of the finetuning stage, Sec. 4.1);
 *  - colour = max(0, sum_c k_c Y_c(d) + 1/2), d = (mu - campos)/|mu - campos|.
 * smooth != 0 drops every cut-off except the near plane (for finite
 * differences): no radius, all tiles, no colour clamp. */
/* Volume mask (Sec. 3.3): hard mask 1[sigmoid(m) > 0.01], decided on the
 * float32 logit against logit(0.01) rounded to float32. */
static int mask_on(double m) { return (float)m > (float)(PLANTED(45) ? -2.1972245773362196 : -4.595119850134589); }

static void project_one(const double *p, const or_camera *cam, int sh_degree, int smooth, int opacity_act,
                        const double *mask, gauss_fwd *g) {
    memset(g, 0, sizeof(*g));
    g->margin = INFINITY;
    if (mask && !mask_on(*mask)) return; /* mask 0: opacity and scales 0, culled */
    const double *mu = p;
    for (int i = 0; i < 3; ++i)
        g->tc[i] = PLANTED(3) ? cam->R[i] * mu[0] + cam->R[3 + i] * mu[1] + cam->R[6 + i] * mu[2] + cam->t[i]
                              : cam->R[3 * i] * mu[0] + cam->R[3 * i + 1] * mu[1] + cam->R[3 * i + 2] * mu[2] + cam->t[i];
    if (!smooth) g->margin = fabs(g->tc[2] - cam->znear);
    if (g->tc[2] <= cam->znear) return;
    double tz = g->tc[2];

    for (int i = 0; i < 3; ++i) g->s[i] = exp(p[3 + i]);
    double qq = 0;
    for (int i = 0; i < 4; ++i) qq += p[6 + i] * p[6 + i];
    g->qlen = sqrt(qq);
    for (int i = 0; i < 4; ++i) g->qn[i] = p[6 + i] / g->qlen;
    quat_to_rot(g->qn, g->Rq);
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = g->Rq[3 * i + j] * g->s[j];
    double Mt[9];
    transpose(M, Mt, 3, 3);
    matmul(M, Mt, g->Sigma, 3, 3, 3);

    double limx = 1.3 * 0.5 * cam->width / cam->fx, limy = 1.3 * 0.5 * cam->height / cam->fy;
    double u = g->tc[0] / tz, v = g->tc[1] / tz;
    g->cux = u; g->cuy = v;
    if (u > limx) { g->cux = limx; g->clampx = 1; }
    if (u < -limx) { g->cux = -limx; g->clampx = 1; }
    if (v > limy) { g->cuy = limy; g->clampy = 1; }
    if (v < -limy) { g->cuy = -limy; g->clampy = 1; }
    if (!smooth) { /* distance (pixels) of the screen position to the clamp, a decision of the gradient */
        double mx = cam->fx * fmin(fabs(u - limx), fabs(u + limx)), my = cam->fy * fmin(fabs(v - limy), fabs(v + limy));
        if (mx < g->margin) g->margin = mx;
        if (my < g->margin) g->margin = my;
    }
    double *J = g->J;
    J[0] = cam->fx / tz; J[1] = 0; J[2] = PLANTED(2) ? 0.0 : -cam->fx * g->cux / tz;
    J[3] = 0; J[4] = cam->fy / tz; J[5] = -cam->fy * g->cuy / tz;
    matmul(J, cam->R, g->Tm, 2, 3, 3);
    double TS[6], Tt[6];
    matmul(g->Tm, g->Sigma, TS, 2, 3, 3);
    transpose(g->Tm, Tt, 2, 3);
    matmul(TS, Tt, g->cov, 2, 3, 2);
    if (!PLANTED(1)) {
        g->cov[0] += cam->dilation;
        g->cov[3] += cam->dilation;
    }
    g->det = g->cov[0] * g->cov[3] - g->cov[1] * g->cov[2];
    if (g->det <= 0) return;
    g->Q[0] = g->cov[3] / g->det; g->Q[1] = -g->cov[1] / g->det;
    g->Q[2] = -g->cov[2] / g->det; g->Q[3] = g->cov[0] / g->det;
    g->mean2d[0] = cam->fx * u + cam->cx;
    g->mean2d[1] = cam->fy * v + cam->cy;

    int32_t tx = (cam->width + cam->tile - 1) / cam->tile, ty = (cam->height + cam->tile - 1) / cam->tile;
    if (smooth) {
        g->radius = 1;
        g->rect[0] = 0; g->rect[1] = 0; g->rect[2] = tx; g->rect[3] = ty;
    } else {
        double half = 0.5 * (g->cov[0] + g->cov[3]);
        double dif = 0.5 * (g->cov[0] - g->cov[3]);
        double lam = half + sqrt(dif * dif + g->cov[1] * g->cov[1]);
        double r3 = 3.0 * sqrt(lam);
        g->radius = (int32_t)ceil(r3);
        double m = frac_dist(r3);
        if (m < g->margin) g->margin = m;
        if (g->radius <= 0) { g->radius = 0; return; }
        if (tile_rect((float)g->mean2d[0], (float)g->mean2d[1], g->radius, cam->tile, tx, ty, g->rect) == 0) {
            g->radius = 0;
            return;
        }
        double e[4] = {(g->mean2d[0] - g->radius) / cam->tile, (g->mean2d[0] + g->radius) / cam->tile,
                       (g->mean2d[1] - g->radius) / cam->tile, (g->mean2d[1] + g->radius) / cam->tile};
        for (int i = 0; i < 4; ++i) {
            double dm = frac_dist(e[i]) * cam->tile;
            if (dm < g->margin) g->margin = dm;
        }
    }

    g->opacity = opacity_act ? fabs(p[10]) : 1.0 / (1.0 + exp(-p[10]));
    double dv[3] = {mu[0] - cam->campos[0], mu[1] - cam->campos[1], mu[2] - cam->campos[2]};
    g->dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int i = 0; i < 3; ++i) g->dir[i] = dv[i] / g->dist;
    sh_eval(g->dir, g->Y, g->dY);
    int nc = (sh_degree + 1) * (sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double c = 0.5;
        for (int k = 0; k < nc; ++k) c += p[11 + 3 * k + ch] * g->Y[k];
        g->rgb_raw[ch] = c;
        g->rgb[ch] = (smooth || c > 0) ? c : 0.0;
    }
    g->visible = 1;
}

/* Per-Gaussian projection. margin[i] is the smallest distance (pixels, or
 * world units for the near plane) of a value that decides an integer
 * (radius, tile rectangle, culling) to its threshold. */
void or_project_act(int64_t n, const double *P, const or_camera *cam, int32_t sh_degree, int32_t smooth,
                    int32_t opacity_act, const double *mask, double *mean2d, double *conic, double *depth,
                    double *opacity, double *rgb, int32_t *radius, int32_t *rect, double *margin) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        gauss_fwd g;
        project_one(P + NP * i, cam, sh_degree, smooth, opacity_act, mask ? mask + i : NULL, &g);
        if (margin) margin[i] = g.margin;
        if (!g.visible) {
            mean2d[2 * i] = mean2d[2 * i + 1] = 0;
            conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
            depth[i] = 0; opacity[i] = 0;
            rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0;
            radius[i] = 0;
            rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
            continue;
        }
        mean2d[2 * i] = g.mean2d[0]; mean2d[2 * i + 1] = g.mean2d[1];
        conic[3 * i] = g.Q[0]; conic[3 * i + 1] = g.Q[1]; conic[3 * i + 2] = g.Q[3];
        depth[i] = g.tc[2];
        opacity[i] = g.opacity;
        for (int c = 0; c < 3; ++c) rgb[3 * i + c] = g.rgb[c];
        radius[i] = g.radius;
        for (int c = 0; c < 4; ++c) rect[4 * i + c] = g.rect[c];
    }
}

void or_project(int64_t n, const double *P, const or_camera *cam, int32_t sh_degree, int32_t smooth,
                double *mean2d, double *conic, double *depth, double *opacity, double *rgb,
                int32_t *radius, int32_t *rect, double *margin) {
    or_project_act(n, P, cam, sh_degree, smooth, 0, NULL, mean2d, conic, depth, opacity, rgb, radius, rect, margin);
}

/* ------------------------------------------------------------------ */
/* Depth order per tile (Sec. 3.1: colours "blended in a sorted order"). */
/* Every (Gaussian, tile of its rectangle) pair becomes one entry with
 * key = (tile id << 32) | bits(float32 depth); entries are generated in
 * Gaussian-index order, tiles row-major inside a rectangle, and sorted
 * stably by key, so equal keys keep ascending Gaussian index.
 * ------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int64_t order;
    uint32_t val;
} sort_entry;

static int cmp_entry(const void *a, const void *b) {
    const sort_entry *x = (const sort_entry *)a, *y = (const sort_entry *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (PLANTED(13)) return x->order > y->order ? -1 : (x->order < y->order);
    return x->order < y->order ? -1 : (x->order > y->order);
}

/* Whether tile (x, y) lists splat i (rectangle already known to hold it). */
static int lists(const float *mean2d, const float *conic, const float *opacity, int64_t i, int32_t tile, int32_t x,
                 int32_t y, int32_t W, int32_t H) {
    return tile_lists(mean2d[2 * i], mean2d[2 * i + 1], conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], opacity[i],
                      tile, x, y, W, H);
}

/* Returns P, the number of entries (tiles of each splat's rectangle that
 * list it, see tile_lists). Writes vals[P] and ranges[tiles][2] (start, end;
 * (0, 0) for an empty tile) when P <= capacity; otherwise writes nothing and
 * returns -P. mean2d, conic, opacity, depth are the splats' single-precision
 * values. smooth != 0: every Gaussian with radius > 0 covers every tile. */
int64_t or_sort(int64_t n, const float *mean2d, const float *conic, const float *opacity, const int32_t *radius,
                const float *depth, int32_t W, int32_t H, int32_t tile, int32_t smooth, int64_t capacity,
                uint32_t *vals, uint32_t *ranges) {
    int32_t tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1)); /* entries of Gaussians before i */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        int32_t rect[4];
        if (radius[i] > 0) {
            if (smooth) c = (int64_t)tx * ty;
            else if (tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], tile, tx, ty, rect) > 0)
                for (int32_t y = rect[1]; y < rect[3]; ++y)
                    for (int32_t x = rect[0]; x < rect[2]; ++x) c += lists(mean2d, conic, opacity, i, tile, x, y, W, H);
        }
        first[i + 1] = c;
    }
    first[0] = 0;
    for (int64_t i = 0; i < n; ++i) first[i + 1] += first[i];
    int64_t P = first[n];
    if (P > capacity) { free(first); return -P; }
    sort_entry *e = (sort_entry *)malloc(sizeof(sort_entry) * (P > 0 ? P : 1));
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        if (first[i + 1] == first[i]) continue;
        int32_t rect[4];
        if (smooth) { rect[0] = 0; rect[1] = 0; rect[2] = tx; rect[3] = ty; }
        else tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], tile, tx, ty, rect);
        uint32_t dbits;
        memcpy(&dbits, &depth[i], 4);
        int64_t k = first[i]; /* entries in (Gaussian index, tile row-major) order */
        for (int32_t y = rect[1]; y < rect[3]; ++y)
            for (int32_t x = rect[0]; x < rect[2]; ++x) {
                if (!smooth && !lists(mean2d, conic, opacity, i, tile, x, y, W, H)) continue;
                e[k].key = ((uint64_t)(uint32_t)(y * tx + x) << 32) | dbits;
                e[k].order = k;
                e[k].val = (uint32_t)i;
                ++k;
            }
    }
    free(first);
    qsort(e, (size_t)P, sizeof(sort_entry), cmp_entry);
    for (int64_t t = 0; t < (int64_t)tx * ty; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t j = 0; j < P; ++j) {
        vals[j] = e[j].val;
        uint32_t t = (uint32_t)(e[j].key >> 32);
        if (j == 0 || (uint32_t)(e[j - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)j;
        if (j == P - 1 || (uint32_t)(e[j + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(e);
    return P;
}

/* ------------------------------------------------------------------ */
/* Compositing (Sec. 3.1, Eq. 2): C = sum_i c_i a_i prod_{j<i} (1 - a_j).  */
/* Readings: a_i = min(0.99, o_i exp(-0.5 d^T Q d)), d = mean2d - pixel;
 * a Gaussian with a positive exponent or a_i < 1/255 is skipped; the ray
 * stops before the Gaussian that would take the transmittance below 1e-4;
 * the remaining transmittance shows the background. smooth != 0 removes
 * every cut-off. n_last = number of list entries up to and including the
 * last one that contributed.                                              */
/* ------------------------------------------------------------------ */
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4

typedef struct {
    int skip, stop;
    double alpha, G, power, dx, dy, rel_margin;
    int capped;
} blend_eval;

static void eval_entry(const double *mean2d, const double *conic, const double *opacity, uint32_t g, double px,
                       double py, double T, int smooth, blend_eval *e) {
    e->dx = mean2d[2 * g] - px;
    e->dy = mean2d[2 * g + 1] - py;
    double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
    e->power = -0.5 * (a * e->dx * e->dx + c * e->dy * e->dy) - b * e->dx * e->dy;
    double scale = 0.5 * (fabs(a) * e->dx * e->dx + fabs(c) * e->dy * e->dy) + fabs(b * e->dx * e->dy) + 1e-300;
    e->rel_margin = fabs(e->power) / scale;
    e->skip = e->stop = e->capped = 0;
    if (!smooth && e->power > 0) { e->skip = 1; return; }
    e->G = exp(e->power);
    double oG = opacity[g] * e->G;
    e->alpha = oG;
    if (!smooth) {
        double m = fabs(oG - ALPHA_MAX) / ALPHA_MAX;
        if (m < e->rel_margin) e->rel_margin = m;
        if (oG > ALPHA_MAX && !PLANTED(14)) { e->alpha = ALPHA_MAX; e->capped = 1; }
        m = fabs(e->alpha - ALPHA_MIN) / ALPHA_MIN;
        if (m < e->rel_margin) e->rel_margin = m;
        if (e->alpha < ALPHA_MIN) { e->skip = 1; return; }
        double tn = T * (1.0 - e->alpha);
        m = fabs(tn - T_MIN) / T_MIN;
        if (m < e->rel_margin) e->rel_margin = m;
        if (tn < (PLANTED(11) ? 1e-3 : T_MIN)) e->stop = 1;
    }
}

/* Tiled render over the sorted lists. margin[H][W] (may be NULL): the
 * smallest relative distance of a per-pixel decision (exponent sign, alpha
 * cap, alpha floor, transmittance floor) to its threshold. */
void or_render(int32_t W, int32_t H, int32_t tile, const double *bg, int32_t smooth, const double *mean2d,
               const double *conic, const double *opacity, const double *rgb, const uint32_t *vals,
               const uint32_t *ranges, double *image, double *t_final, int32_t *n_last, double *margin) {
    int32_t tx = (W + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            int32_t t = (py / tile) * tx + (px / tile);
            uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
            double T = 1.0, C[3] = {0, 0, 0}, mg = INFINITY;
            int32_t last = 0;
            for (uint32_t k = s; k < e; ++k) {
                uint32_t g = vals[k];
                blend_eval ev;
                eval_entry(mean2d, conic, opacity, g, px, py, T, smooth, &ev);
                if (ev.rel_margin < mg) mg = ev.rel_margin;
                if (ev.skip) continue;
                if (ev.stop) break;
                if (PLANTED(5)) T *= 1.0 - ev.alpha;
                for (int c = 0; c < 3; ++c) C[c] += rgb[3 * g + c] * ev.alpha * T;
                if (!PLANTED(5)) T *= 1.0 - ev.alpha;
                last = (int32_t)(k - s + 1);
            }
            int64_t pix = (int64_t)py * W + px;
            for (int c = 0; c < 3; ++c) image[(int64_t)c * H * W + pix] = C[c] + T * bg[c];
            t_final[pix] = T;
            n_last[pix] = last;
            if (margin) margin[pix] = mg;
        }
}

/* The tiled render of Eq. 2 at a list of pixels only (same rules as
 * or_render); out [3][npix], t_final [npix], n_last [npix]. */
void or_render_pixels(int64_t npix, const int32_t *pxs, const int32_t *pys, int32_t W, int32_t tile, const double *bg,
                      const double *mean2d, const double *conic, const double *opacity, const double *rgb,
                      const uint32_t *vals, const uint32_t *ranges, double *out, double *t_final, int32_t *n_last,
                      double *margin) {
    int32_t tx = (W + tile - 1) / tile;
    for (int64_t q = 0; q < npix; ++q) {
        int32_t px = pxs[q], py = pys[q];
        int32_t t = (py / tile) * tx + (px / tile);
        double T = 1.0, C[3] = {0, 0, 0}, mg = INFINITY;
        int32_t last = 0;
        for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) {
            blend_eval ev;
            eval_entry(mean2d, conic, opacity, vals[k], px, py, T, 0, &ev);
            if (ev.rel_margin < mg) mg = ev.rel_margin;
            if (ev.skip) continue;
            if (ev.stop) break;
            for (int c = 0; c < 3; ++c) C[c] += rgb[3 * vals[k] + c] * ev.alpha * T;
            T *= 1.0 - ev.alpha;
            last = (int32_t)(k - ranges[2 * t] + 1);
        }
        for (int c = 0; c < 3; ++c) out[c * npix + q] = C[c] + T * bg[c];
        t_final[q] = T;
        n_last[q] = last;
        if (margin) margin[q] = mg;
    }
}

/* Test support for finite differences of the piecewise-smooth loss: the
 * render of or_render_pixels with every discrete decision held fixed.
 * mode 0 (record) renders as or_render_pixels and writes, for pixel q and
 * position k of its tile's list, dec[q * stride + k] = 0 skipped, 1 blended,
 * 2 blended at the alpha cap, 3 the ray stopped before this entry (later
 * positions are not visited). mode 1 (replay) takes those decisions instead
 * of making them, on the same lists, so the result is a smooth function of
 * the per-Gaussian values near the recorded point: its derivative is the one
 * the analytic backward computes. stride >= the longest visited list. */
void or_render_pixels_locked(int64_t npix, const int32_t *pxs, const int32_t *pys, int32_t W, int32_t tile,
                             const double *bg, const double *mean2d, const double *conic, const double *opacity,
                             const double *rgb, const uint32_t *vals, const uint32_t *ranges, int32_t mode,
                             int64_t stride, uint8_t *dec, double *out) {
    int32_t tx = (W + tile - 1) / tile;
    for (int64_t q = 0; q < npix; ++q) {
        int32_t px = pxs[q], py = pys[q];
        int32_t t = (py / tile) * tx + (px / tile);
        uint8_t *d = dec + q * stride;
        double T = 1.0, C[3] = {0, 0, 0};
        for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) {
            int64_t pos = k - ranges[2 * t];
            uint32_t g = vals[k];
            double alpha;
            if (mode == 0) {
                blend_eval ev;
                eval_entry(mean2d, conic, opacity, g, px, py, T, 0, &ev);
                if (ev.skip) { d[pos] = 0; continue; }
                if (ev.stop) { d[pos] = 3; break; }
                d[pos] = ev.capped ? 2 : 1;
                alpha = ev.alpha;
            } else {
                if (d[pos] == 0) continue;
                if (d[pos] == 3) break;
                if (d[pos] == 2) {
                    alpha = ALPHA_MAX;
                } else {
                    double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                    double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
                    alpha = opacity[g] * exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy);
                }
            }
            for (int c = 0; c < 3; ++c) C[c] += rgb[3 * g + c] * alpha * T;
            T *= 1.0 - alpha;
        }
        for (int c = 0; c < 3; ++c) out[c * npix + q] = C[c] + T * bg[c];
    }
}

/* Contributors of one pixel in blending order: list position, alpha and
 * the transmittance in front of each. Returns their number (at most cap). */
int32_t or_pixel_trace(int32_t px, int32_t py, int32_t W, int32_t tile, const double *mean2d, const double *conic,
                       const double *opacity, const uint32_t *vals, const uint32_t *ranges, int32_t cap,
                       int32_t *pos, double *alpha, double *trans) {
    int32_t tx = (W + tile - 1) / tile;
    int32_t t = (py / tile) * tx + (px / tile);
    double T = 1.0;
    int32_t k = 0;
    for (uint32_t j = ranges[2 * t]; j < ranges[2 * t + 1] && k < cap; ++j) {
        blend_eval ev;
        eval_entry(mean2d, conic, opacity, vals[j], px, py, T, 0, &ev);
        if (ev.skip) continue;
        if (ev.stop) break;
        pos[k] = (int32_t)(j - ranges[2 * t]);
        alpha[k] = ev.alpha;
        trans[k] = T;
        ++k;
        T *= 1.0 - ev.alpha;
    }
    return k;
}

/* The same image by brute force: for every pixel, all Gaussians whose
 * tile rectangle holds the pixel's tile, in ascending (float32 depth,
 * index) order, composited by Eq. 2 with the same cut-offs. */
typedef struct { float d; int64_t i; } depth_idx;
static int cmp_depth(const void *a, const void *b) {
    const depth_idx *x = (const depth_idx *)a, *y = (const depth_idx *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return x->i < y->i ? -1 : (x->i > y->i);
}

void or_render_brute(int64_t n, int32_t W, int32_t H, int32_t tile, const double *bg, const double *mean2d,
                     const double *conic, const double *opacity, const double *rgb, const int32_t *radius,
                     const int32_t *rect, const float *depth, double *image) {
    depth_idx *ord = (depth_idx *)malloc(sizeof(depth_idx) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (radius[i] > 0) { ord[m].d = depth[i]; ord[m].i = i; ++m; }
    qsort(ord, (size_t)m, sizeof(depth_idx), cmp_depth);
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            int32_t tcx = px / tile, tcy = py / tile;
            double T = 1.0, C[3] = {0, 0, 0};
            for (int64_t k = 0; k < m; ++k) {
                int64_t g = ord[k].i;
                const int32_t *r = rect + 4 * g;
                if (tcx < r[0] || tcx >= r[2] || tcy < r[1] || tcy >= r[3]) continue;
                double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                double pw = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
                if (pw > 0) continue;
                double a = opacity[g] * exp(pw);
                if (a > ALPHA_MAX) a = ALPHA_MAX;
                if (a < ALPHA_MIN) continue;
                if (T * (1 - a) < T_MIN) break;
                for (int c = 0; c < 3; ++c) C[c] += rgb[3 * g + c] * a * T;
                T *= 1 - a;
            }
            for (int c = 0; c < 3; ++c) image[(int64_t)c * H * W + (int64_t)py * W + px] = C[c] + T * bg[c];
        }
    free(ord);
}

/* ------------------------------------------------------------------ */
/* Loss (Sec. 3.1, Eq. 3): L = (1 - l) L1 + l (1 - SSIM), l = 0.2.        */
/* Readings: L1 and SSIM are means over all 3 H W values; SSIM per channel
 * with an 11x11 Gaussian window (sigma 1.5, normalised to sum 1), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2 (the usual SSIM constants for a unit
 * dynamic range). The gradient of |x - y| at x = y is taken as 0.
 * Direct 2-D windows, no separable shortcut.                              */
/* ------------------------------------------------------------------ */
static void ssim_window(double w[11][11]) {
    double g[11], s = 0;
    for (int i = 0; i < 11; ++i) { g[i] = exp(-((i - 5) * (i - 5)) / (2 * 1.5 * 1.5)); s += g[i]; }
    for (int i = 0; i < 11; ++i)
        for (int j = 0; j < 11; ++j) w[i][j] = g[i] * g[j] / (s * s);
}

/* SSIM map value of one channel at pixel (i, j): Gaussian-weighted window
 * means of x, y, x^2, y^2, xy over the 11x11 neighbourhood inside the image
 * (zero padding), then the usual luminance x contrast-structure ratio. */
typedef struct { double m, mx, my, n1, n2, d1, d2; } ssim_px;

static ssim_px ssim_at(const double *x, const double *y, int32_t H, int32_t W, int32_t i, int32_t j,
                       double w[11][11]) {
    const double C1 = 0.01 * 0.01, C2 = PLANTED(8) ? 0.02 * 0.02 : 0.03 * 0.03;
    double mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
    for (int di = -5; di <= 5; ++di)
        for (int dj = -5; dj <= 5; ++dj) {
            int32_t a = i + di, b = j + dj;
            if (a < 0 || a >= H || b < 0 || b >= W) continue;
            double wt = w[di + 5][dj + 5], xv = x[(int64_t)a * W + b], yv = y[(int64_t)a * W + b];
            mx += wt * xv; my += wt * yv; xx += wt * xv * xv; yy += wt * yv * yv; xy += wt * xv * yv;
        }
    double sx = xx - mx * mx, sy = yy - my * my, sxy = xy - mx * my;
    ssim_px r;
    r.mx = mx; r.my = my;
    r.n1 = 2 * mx * my + C1; r.n2 = 2 * sxy + C2;
    r.d1 = mx * mx + my * my + C1; r.d2 = sx + sy + C2;
    r.m = r.n1 * r.n2 / (r.d1 * r.d2);
    return r;
}

double or_loss(int32_t H, int32_t W, const double *image, const double *gt, double lambda, double *dl_dimage) {
    double w[11][11];
    ssim_window(w);
    int64_t HW = (int64_t)H * W, N = 3 * HW;
    double l1 = 0, ssim = 0;
    double *A = (double *)malloc(sizeof(double) * HW), *B = (double *)malloc(sizeof(double) * HW),
           *Cm = (double *)malloc(sizeof(double) * HW);
    double *row_ssim = (double *)malloc(sizeof(double) * (size_t)H), *row_l1 = (double *)malloc(sizeof(double) * H);
    for (int ch = 0; ch < 3; ++ch) {
        const double *x = image + ch * HW, *y = gt + ch * HW;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < H; ++i) {
            row_ssim[i] = 0;
            for (int32_t j = 0; j < W; ++j) {
                ssim_px r = ssim_at(x, y, H, W, i, j, w);
                double m = r.m, mx = r.mx, my = r.my, n1 = r.n1, n2 = r.n2, d1 = r.d1, d2 = r.d2;
                row_ssim[i] += m;
                /* partial derivatives of the map value with respect to the
                   window mean of x, of x^2 and of x*y */
                int64_t p = (int64_t)i * W + j;
                /* m / n1 = n2 / (d1 d2) and m / n2 = n1 / (d1 d2): no division
                   by n1 or n2, which can be zero (d1 >= C1, d2 >= C2) */
                A[p] = 2 * my * (n2 - n1) / (d1 * d2) - 2 * mx * m / d1 + 2 * mx * m / d2;
                B[p] = -m / d2;
                Cm[p] = 2 * n1 / (d1 * d2);
            }
        }
        for (int32_t i = 0; i < H; ++i) ssim += row_ssim[i];
        if (dl_dimage) {
#pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < H; ++i)
                for (int32_t j = 0; j < W; ++j) {
                    double ga = 0, gb = 0, gc = 0;
                    for (int di = -5; di <= 5; ++di)
                        for (int dj = -5; dj <= 5; ++dj) {
                            int32_t a = i + di, b = j + dj;
                            if (a < 0 || a >= H || b < 0 || b >= W) continue;
                            double wt = w[di + 5][dj + 5];
                            int64_t q = (int64_t)a * W + b;
                            ga += wt * A[q]; gb += wt * B[q]; gc += wt * Cm[q];
                        }
                    int64_t p = (int64_t)i * W + j;
                    double dssim = (ga + 2 * x[p] * gb + y[p] * gc) / N;
                    double d = x[p] - y[p];
                    double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
                    dl_dimage[ch * HW + p] = (1 - lambda) * sg / N - lambda * dssim;
                }
        }
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < H; ++i) {
            row_l1[i] = 0;
            for (int32_t j = 0; j < W; ++j) row_l1[i] += fabs(x[(int64_t)i * W + j] - y[(int64_t)i * W + j]);
        }
        for (int32_t i = 0; i < H; ++i) l1 += row_l1[i];
    }
    free(A); free(B); free(Cm); free(row_ssim); free(row_l1);
    return (1 - lambda) * l1 / N + lambda * (1 - ssim / N);
}

/* The part of the Eq. 3 loss owed to the pixels of the window
 * [x0, x1) x [y0, y1) of an H x W image, all three channels:
 *   (1 - lambda)/N sum |x - y|  -  lambda/N sum SSIM(p),   N = 3 H W,
 * so that or_loss = lambda + the sum of this over any partition of the image
 * into windows. The SSIM value of a window pixel reads the image up to 5
 * pixels around it (zero padding at the image border); a change confined to
 * a region changes only the window terms of the pixels within 5 of it. */
double or_loss_window(int32_t H, int32_t W, const double *image, const double *gt, double lambda, int32_t x0,
                      int32_t y0, int32_t x1, int32_t y1) {
    double w[11][11];
    ssim_window(w);
    int64_t HW = (int64_t)H * W, N = 3 * HW;
    double l1 = 0, ssim = 0;
    for (int ch = 0; ch < 3; ++ch) {
        const double *x = image + ch * HW, *y = gt + ch * HW;
        for (int32_t i = y0; i < y1; ++i)
            for (int32_t j = x0; j < x1; ++j) {
                ssim += ssim_at(x, y, H, W, i, j, w).m;
                l1 += fabs(x[(int64_t)i * W + j] - y[(int64_t)i * W + j]);
            }
    }
    return (1 - lambda) * l1 / N - lambda * ssim / N;
}

/* ------------------------------------------------------------------ */
/* Rasteriser backward. Sec. 3.2.4: the gradient is not computed for a   */
/* frozen Gaussian; frozen Gaussians still occlude and so still enter the */
/* transmittance of the others.                                           */
/* For every pixel the forward pass is rerun and its contributors kept;
 * with suffix sums S_k = sum_{i>k} c_i a_i T_i the derivative of Eq. 2 is
 *   dC/da_k = c_k T_k - (S_k + T_final bg) / (1 - a_k),   dC/dc_k = a_k T_k.
 * Outputs are accumulated over pixels for unfrozen Gaussians only:
 *   d_mean2d[n][2], d_conic[n][3] (a, b, c), d_opacity[n], d_rgb[n][3].
 * amb[H][W] (optional): pixels whose forward decisions are ambiguous;
 * tainted[n] (optional) is set for every Gaussian evaluated at one;
 * amb_abs[n][9] (optional) sums, over ambiguous pixels, the absolute value of
 * each of a Gaussian's nine per-pixel gradient terms (mean x, y; conic a, b,
 * c; opacity; r, g, b): a decision that flips at such a pixel changes a
 * Gaussian's gradient by no more than its terms there.
 * tile_mask[tiles] (optional): only pixels of tiles with a non-zero entry
 * are processed; the gradient of a Gaussian is complete when every tile of
 * its rectangle is in the mask.                                           */
/* ------------------------------------------------------------------ */
void or_render_bwd(int64_t n, int32_t W, int32_t H, int32_t tile, const double *bg, int32_t smooth,
                   const double *mean2d, const double *conic, const double *opacity, const double *rgb,
                   const uint32_t *vals, const uint32_t *ranges, const double *dl_dimage, const uint8_t *frozen,
                   const uint8_t *amb, const uint8_t *tile_mask, double *d_mean2d, double *d_conic,
                   double *d_opacity, double *d_rgb, uint8_t *tainted, double *amb_abs) {
    int32_t tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t ntiles = (int64_t)tx * ty, HW = (int64_t)H * W;
    memset(d_mean2d, 0, sizeof(double) * 2 * n);
    memset(d_conic, 0, sizeof(double) * 3 * n);
    memset(d_opacity, 0, sizeof(double) * n);
    memset(d_rgb, 0, sizeof(double) * 3 * n);
    if (tainted) memset(tainted, 0, (size_t)n);
    if (amb_abs) memset(amb_abs, 0, sizeof(double) * 9 * n);
    int32_t cap = 0;
    int64_t P = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        int32_t len = (int32_t)(ranges[2 * t + 1] - ranges[2 * t]);
        if (len > cap) cap = len;
        if ((int64_t)ranges[2 * t + 1] > P) P = ranges[2 * t + 1];
    }
    /* Each tile's pixels add into per-entry partial sums (an entry belongs to
     * one tile); the partials are then added into the per-Gaussian gradients
     * in entry order, so the summation order is the same on any number of
     * threads. Per entry: d_mean2d (2), d_conic (3), d_opacity, d_rgb (3). */
    double *part = (double *)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
    double *part_amb = amb_abs ? (double *)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double)) : NULL;
    uint8_t *part_taint = tainted ? (uint8_t *)calloc((size_t)(P > 0 ? P : 1), 1) : NULL;
#pragma omp parallel
    {
        blend_eval *ev = (blend_eval *)malloc(sizeof(blend_eval) * (cap > 0 ? cap : 1));
        uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * (cap > 0 ? cap : 1));
        double *Tk = (double *)malloc(sizeof(double) * (cap > 0 ? cap : 1));
        double *S = (double *)malloc(sizeof(double) * 3 * (cap > 0 ? cap : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < ntiles; ++t) {
            if (tile_mask && !tile_mask[t]) continue;
            uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
            int32_t x0 = (int32_t)(t % tx) * tile, y0 = (int32_t)(t / tx) * tile;
            for (int32_t py = y0; py < y0 + tile && py < H; ++py)
                for (int32_t px = x0; px < x0 + tile && px < W; ++px) {
                    int64_t pix = (int64_t)py * W + px;
                    int ambiguous = amb ? amb[pix] : 0;
                    double T = 1.0;
                    int nc = 0;
                    for (uint32_t k = s; k < e; ++k) {
                        blend_eval b;
                        eval_entry(mean2d, conic, opacity, vals[k], px, py, T, smooth, &b);
                        if (ambiguous && part_taint) part_taint[k] = 1;
                        if (b.skip) continue;
                        if (b.stop) break;
                        ev[nc] = b; pos[nc] = k; Tk[nc] = T; ++nc;
                        T *= 1.0 - b.alpha;
                    }
                    double Tf = T;
                    double acc[3] = {0, 0, 0};
                    for (int k = nc - 1; k >= 0; --k) {
                        uint32_t g = vals[pos[k]];
                        for (int c = 0; c < 3; ++c) S[3 * k + c] = acc[c];
                        for (int c = 0; c < 3; ++c) acc[c] += rgb[3 * g + c] * ev[k].alpha * Tk[k];
                    }
                    double dC[3];
                    for (int c = 0; c < 3; ++c) dC[c] = dl_dimage[c * HW + pix];
                    for (int k = 0; k < nc; ++k) {
                        uint32_t g = vals[pos[k]];
                        if (frozen && frozen[g]) continue;
                        double *pt = part + 9 * (int64_t)pos[k];
                        double a = ev[k].alpha, dA = 0;
                        double *ab = (ambiguous && part_amb) ? part_amb + 9 * (int64_t)pos[k] : NULL;
                        for (int c = 0; c < 3; ++c) {
                            double dCda = rgb[3 * g + c] * Tk[k] - (S[3 * k + c] + (PLANTED(7) ? 0.0 : Tf * bg[c])) / (1.0 - a);
                            dA += dC[c] * dCda;
                            pt[6 + c] += a * Tk[k] * dC[c];
                            if (ab) ab[6 + c] += fabs(a * Tk[k] * dC[c]);
                        }
                        if (ev[k].capped) continue; /* alpha = 0.99 does not depend on o or G */
                        double o = opacity[g], G = ev[k].G;
                        pt[5] += dA * G;
                        double dpow = dA * o * G;
                        double dx = ev[k].dx, dy = ev[k].dy;
                        double qa = conic[3 * g], qb = conic[3 * g + 1], qc = conic[3 * g + 2];
                        pt[2] += -0.5 * dx * dx * dpow;
                        pt[3] += (PLANTED(43) ? -0.5 : -1.0) * dx * dy * dpow;
                        pt[4] += -0.5 * dy * dy * dpow;
                        pt[0] += (PLANTED(6) ? 1.0 : -1.0) * (qa * dx + qb * dy) * dpow;
                        pt[1] += -(qb * dx + qc * dy) * dpow;
                        if (ab) {
                            ab[0] += fabs((qa * dx + qb * dy) * dpow);
                            ab[1] += fabs((qb * dx + qc * dy) * dpow);
                            ab[2] += fabs(0.5 * dx * dx * dpow);
                            ab[3] += fabs(dx * dy * dpow);
                            ab[4] += fabs(0.5 * dy * dy * dpow);
                            ab[5] += fabs(dA * G);
                        }
                    }
                }
        }
        free(ev); free(pos); free(Tk); free(S);
    }
    for (int64_t k = 0; k < P; ++k) {
        uint32_t g = vals[k];
        const double *pt = part + 9 * k;
        d_mean2d[2 * g] += pt[0]; d_mean2d[2 * g + 1] += pt[1];
        d_conic[3 * g] += pt[2]; d_conic[3 * g + 1] += pt[3]; d_conic[3 * g + 2] += pt[4];
        d_opacity[g] += pt[5];
        d_rgb[3 * g] += pt[6]; d_rgb[3 * g + 1] += pt[7]; d_rgb[3 * g + 2] += pt[8];
        if (part_amb) {
            const double *pa = part_amb + 9 * k;
            double *ab = amb_abs + 9 * (int64_t)g;
            for (int c = 0; c < 9; ++c) ab[c] += pa[c];
        }
        if (part_taint && part_taint[k]) tainted[g] = 1;
    }
    free(part);
    free(part_amb);
    free(part_taint);
}

/* ------------------------------------------------------------------ */
/* Projection backward: chain rule from the 2-D quantities to the 59     */
/* parameters, for unfrozen visible Gaussians (Sec. 3.2.4). Also returns  */
/* the two quantities of the freeze test (Sec. 3.2.1):                    */
/*   xyz_norm = |dL/d mean2d| in normalised device units, i.e. with the   */
/*              pixel gradient scaled by (W/2, H/2) (the positional        */
/*              gradient that 3DGS densification thresholds);              */
/*   rgb_norm = |dL/d k_0| over the 3 channels (the diffuse colour).       */
/* G is [n][59]; rows of frozen or culled Gaussians are zero.             */
/* ------------------------------------------------------------------ */
/* mask (n or NULL): volume-mask logits; then G_mask [n] receives the
 * straight-through gradient of each logit, (dL/dM + mask_loss) sigmoid'(m)
 * with dL/dM = dL/dopacity * opacity + sum_b dL/dlog s_b for a visible
 * Gaussian and 0 otherwise (mask_loss = lambda_m / N, the mask term's
 * derivative), 0 for frozen ones. */
void or_project_bwd_act(int64_t n, const double *P, const or_camera *cam, int32_t sh_degree, int32_t smooth,
                        int32_t opacity_act, const double *mask, double mask_loss, const uint8_t *frozen,
                        const double *d_mean2d, const double *d_conic, const double *d_opacity, const double *d_rgb,
                        double *G, double *G_mask, double *xyz_norm, double *rgb_norm) {
    memset(G, 0, sizeof(double) * NP * n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (xyz_norm) xyz_norm[i] = 0;
        if (rgb_norm) rgb_norm[i] = 0;
        if (G_mask) G_mask[i] = 0;
        if (frozen && frozen[i]) continue;
        const double *p = P + NP * i;
        double *gp = G + NP * i;
        double mslope = 0;
        if (mask) {
            double sm = 1.0 / (1.0 + exp(-mask[i]));
            mslope = sm * (1.0 - sm);
            if (G_mask) G_mask[i] = mask_loss * mslope;
        }
        gauss_fwd g;
        project_one(p, cam, sh_degree, smooth, opacity_act, mask ? mask + i : NULL, &g);
        if (!g.visible) continue;
        const double *dm = d_mean2d + 2 * i, *dq = d_conic + 3 * i, *dc = d_rgb + 3 * i;

        /* colour: c = max(0, sum_k k_c Y_c(d) + 1/2) */
        int nc = (sh_degree + 1) * (sh_degree + 1);
        double gc[3], ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) gc[ch] = (smooth || g.rgb_raw[ch] > 0) ? dc[ch] : 0.0;
        for (int k = 0; k < nc; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                gp[11 + 3 * k + ch] = g.Y[k] * gc[ch];
                for (int a = 0; a < 3; ++a) ddir[a] += p[11 + 3 * k + ch] * gc[ch] * g.dY[3 * k + a];
            }
        double dmu[3], dd = ddir[0] * g.dir[0] + ddir[1] * g.dir[1] + ddir[2] * g.dir[2];
        for (int a = 0; a < 3; ++a) dmu[a] = PLANTED(15) ? 0.0 : (ddir[a] - g.dir[a] * dd) / g.dist;

        /* opacity = sigmoid(x): d/dx = o (1 - o); opacity = |x|: d/dx = sign(x) */
        if (opacity_act)
            gp[10] = d_opacity[i] * (PLANTED(42) ? 1.0 : (p[10] > 0 ? 1.0 : (p[10] < 0 ? -1.0 : 0.0)));
        else
            gp[10] = d_opacity[i] * g.opacity * (1 - g.opacity);

        /* conic = inverse of the 2-D covariance: dL/dcov = -Q dL/dQ Q */
        double GQ[4] = {dq[0], 0.5 * dq[1], 0.5 * dq[1], dq[2]}, tmp[4], Gcov[4];
        matmul(g.Q, GQ, tmp, 2, 2, 2);
        matmul(tmp, g.Q, Gcov, 2, 2, 2);
        for (int a = 0; a < 4; ++a) Gcov[a] = -Gcov[a];

        /* cov = Tm Sigma Tm^T (+ dilation): dSigma = Tm^T Gcov Tm, dTm = 2 Gcov Tm Sigma */
        double Tt[6], t1[6], GSig[9], t2[6], GTm[6];
        transpose(g.Tm, Tt, 2, 3);
        matmul(Tt, Gcov, t1, 3, 2, 2);
        matmul(t1, g.Tm, GSig, 3, 2, 3);
        matmul(Gcov, g.Tm, t2, 2, 2, 3);
        matmul(t2, g.Sigma, GTm, 2, 3, 3);
        for (int a = 0; a < 6; ++a) GTm[a] *= PLANTED(17) ? 1 : 2;

        /* Tm = J R_c */
        double Rct[9], GJ[6];
        transpose(cam->R, Rct, 3, 3);
        matmul(GTm, Rct, GJ, 2, 3, 3);
        double tx = g.tc[0], ty = g.tc[1], tz = g.tc[2];
        double dtz = GJ[0] * (-cam->fx / (tz * tz)) + GJ[4] * (-cam->fy / (tz * tz)) +
                     GJ[2] * (cam->fx * g.cux / (tz * tz)) + GJ[5] * (cam->fy * g.cuy / (tz * tz));
        double dcu = GJ[2] * (-cam->fx / tz), dcv = GJ[5] * (-cam->fy / tz);
        double du = ((g.clampx && !PLANTED(18)) ? 0.0 : dcu) + cam->fx * dm[0];
        double dv = (g.clampy ? 0.0 : dcv) + cam->fy * dm[1];
        double dtc[3] = {du / tz, dv / tz, dtz - du * tx / (tz * tz) - dv * ty / (tz * tz)};
        for (int a = 0; a < 3; ++a)
            dmu[a] += cam->R[a] * dtc[0] + cam->R[3 + a] * dtc[1] + cam->R[6 + a] * dtc[2];
        for (int a = 0; a < 3; ++a) gp[a] = dmu[a];

        /* Sigma = M M^T, M = R_q diag(s) */
        double M[9], GM[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[3 * a + b] = g.Rq[3 * a + b] * g.s[b];
        matmul(GSig, M, GM, 3, 3, 3);
        for (int a = 0; a < 9; ++a) GM[a] *= 2;
        double GR[9];
        for (int b = 0; b < 3; ++b) {
            double ds = 0;
            for (int a = 0; a < 3; ++a) {
                ds += GM[3 * a + b] * g.Rq[3 * a + b];
                GR[3 * a + b] = GM[3 * a + b] * g.s[b];
            }
            gp[3 + b] = ds * g.s[b];
        }
        double dR[4][9], dqn[4], qd = 0;
        quat_to_rot_grad(g.qn, dR);
        for (int k = 0; k < 4; ++k) {
            dqn[k] = 0;
            for (int a = 0; a < 9; ++a) dqn[k] += GR[a] * dR[k][a];
            qd += dqn[k] * g.qn[k];
        }
        for (int k = 0; k < 4; ++k) gp[6 + k] = (dqn[k] - (PLANTED(16) ? 0.0 : g.qn[k] * qd)) / g.qlen;

        if (xyz_norm) {
            double ex = dm[0] * (PLANTED(19) ? 1.0 : 0.5 * cam->width), ey = dm[1] * (PLANTED(19) ? 1.0 : 0.5 * cam->height);
            xyz_norm[i] = sqrt(ex * ex + ey * ey);
        }
        if (rgb_norm) rgb_norm[i] = sqrt(gp[11] * gp[11] + gp[12] * gp[12] + gp[13] * gp[13]);
        if (mask && G_mask) {
            /* o' = M o and s' = M s at M = 1: dL/dM = dL/do' o + sum_b dL/ds'_b s_b */
            double dM = d_opacity[i] * g.opacity + gp[3] + gp[4] + gp[5];
            G_mask[i] = (dM + mask_loss) * mslope;
        }
    }
}

void or_project_bwd(int64_t n, const double *P, const or_camera *cam, int32_t sh_degree, int32_t smooth,
                    const uint8_t *frozen, const double *d_mean2d, const double *d_conic, const double *d_opacity,
                    const double *d_rgb, double *G, double *xyz_norm, double *rgb_norm) {
    or_project_bwd_act(n, P, cam, sh_degree, smooth, 0, NULL, 0.0, frozen, d_mean2d, d_conic, d_opacity, d_rgb, G,
                       NULL, xyz_norm, rgb_norm);
}

/* ------------------------------------------------------------------ */
/* Adam restricted to unfrozen Gaussians (Sec. 3.2.4: the optimiser only  */
/* updates Gaussians whose gradients were computed). Textbook Adam with   */
/* bias correction at the global step `step` (>= 1); lr has one entry per  */
/* parameter group: xyz, scale, rotation, opacity, SH DC, SH rest.         */
/* Frozen rows of P, M and V are not touched.                             */
/* ------------------------------------------------------------------ */
static int param_group(int r) {
    if (r < 3) return 0;
    if (r < 6) return 1;
    if (r < 10) return 2;
    if (r < 11) return 3;
    if (r < 14) return 4;
    return 5;
}

void or_adam(int64_t n, double *P, const double *G, double *M, double *V, const uint8_t *frozen, const double *lr,
             double b1, double b2, double eps, int64_t step) {
    double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (frozen && frozen[i] && !PLANTED(12)) continue;
        for (int r = 0; r < NP; ++r) {
            int64_t k = NP * i + r;
            double g = G[k];
            M[k] = b1 * M[k] + (1 - b1) * g;
            V[k] = b2 * V[k] + (1 - b2) * g * g;
            double mh = M[k] / bc1, vh = PLANTED(9) ? V[k] : V[k] / bc2;
            P[k] -= lr[param_group(r)] * mh / (sqrt(vh) + eps);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Freeze map update (Sec. 3.2.1, Eqs. 4-6; cadence in Sec. 4.1).          */
/* The gradient norms of each Gaussian are summed over the iterations      */
/* since the last update in which it was visible (acc_*, cnt). mode:       */
/*   0 update: freeze_i |= cnt>0 && acc_xyz/cnt < eps_xyz                  */
/*                               && acc_rgb/cnt < eps_rgb   (Eqs. 4, 6)    */
/*             (a frozen Gaussian stays frozen: the map accumulates);      */
/*   1 reset : every Gaussian unfrozen;                                    */
/*   2 clear : the map is kept;                                            */
/*   3 list  : the map and the statistics are kept (after densification    */
/*             moved the Gaussians).                                       */
/* Modes 0-2 then zero the statistics; every mode lists the unfrozen       */
/* Gaussians in ascending order in act. The average and the comparison are */
/* taken in single precision. Returns the number of unfrozen Gaussians.    */
/* ------------------------------------------------------------------ */
int64_t or_freeze_update(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen, float eps_xyz,
                         float eps_rgb, int32_t mode, int32_t *act) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (mode == 1) frozen[i] = 0;
        if (mode == 0 && cnt[i] > 0) {
            volatile float c = (float)cnt[i];
            volatile float ax = acc_xyz[i] / c, ar = acc_rgb[i] / c;
            if (PLANTED(10) ? (ax < eps_xyz || ar < eps_rgb) : (ax < eps_xyz && ar < eps_rgb)) frozen[i] = 1;
        }
        if (mode != 3) { acc_xyz[i] = 0; acc_rgb[i] = 0; cnt[i] = 0; }
        if (!frozen[i]) act[k++] = (int32_t)i;
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* PSNR (Sec. 3.2.2, Eq. 7 uses it): 10 log10(1 / MSE) with the rendered   */
/* image clamped to [0, 1], MSE over all 3 H W values; an MSE below 1e-10   */
/* reads as 1e-10 (100 dB).                                                */
/* ------------------------------------------------------------------ */
void or_psnr(int32_t S, int32_t H, int32_t W, const double *images, const double *gts, double *psnr) {
    int64_t N = 3 * (int64_t)H * W;
    for (int32_t s = 0; s < S; ++s) {
        double se = 0;
        for (int64_t k = 0; k < N; ++k) {
            double x = images[s * N + k];
            x = x < 0 ? 0 : (x > 1 ? 1 : x);
            double d = x - gts[s * N + k];
            se += d * d;
        }
        double mse = se / N;
        if (mse < 1e-10) mse = 1e-10;
        psnr[s] = 10.0 * log10(1.0 / mse);
    }
}

/* ------------------------------------------------------------------ */
/* Learned freeze predictor. The paper has no learned component: this is */
/* the plain statement of the predictor the CUDA path builds (features,  */
/* 16 -> 64 -> 64 -> 1 MLP, weighted BCE, Adam), used as its reference.  */
/* ------------------------------------------------------------------ */
#define MLP_IN 16
#define MLP_H 64
#define OFF_W1 0                      /* [16][64], input-major */
#define OFF_B1 (OFF_W1 + MLP_IN * MLP_H)
#define OFF_W2 (OFF_B1 + MLP_H)       /* [64][64], input-major */
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)       /* [64] */
#define OFF_B3 (OFF_W3 + MLP_H)
#define MLP_NPARAM (OFF_B3 + 1)       /* 5313 */

int32_t or_mlp_nparams(void) { return MLP_NPARAM; }

/* Round to bfloat16 (8-bit mantissa) by round-to-nearest-even on the
 * float32 value: add 0x7fff plus the lowest kept bit, drop 16 bits. */
double or_bf16(double x) {
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, 4);
    if (!PLANTED(22)) b += 0x7fffu + ((b >> 16) & 1u);
    b &= 0xffff0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* Per-Gaussian predictor state, [n][12]: 0-3 history of the xyz norm EMA
 * (most recent first), 4-7 the same for rgb, 8 xyz EMA, 9 rgb EMA,
 * 10 visible iterations so far, 11 boundaries spent frozen.
 * At every statistics boundary (every 250 iterations, before the statistics
 * are cleared): if the Gaussian was visible (cnt > 0) each EMA becomes
 * 0.5 EMA + 0.5 (acc / cnt) and views += cnt; frozen += frozen[i]; then each
 * history shifts by one and takes the EMA at its front. */
void or_pred_history(int64_t n, const float *acc_xyz, const float *acc_rgb, const int32_t *cnt, const uint8_t *frozen,
                     double *state) {
    for (int64_t i = 0; i < n; ++i) {
        double *s = state + 12 * i;
        if (cnt[i] > 0) {
            s[8] = 0.5 * s[8] + 0.5 * ((double)acc_xyz[i] / cnt[i]);
            s[9] = 0.5 * s[9] + 0.5 * ((double)acc_rgb[i] / cnt[i]);
            s[10] += PLANTED(23) ? 1 : cnt[i];
        }
        if (frozen && frozen[i]) s[11] += 1;
        for (int j = 3; j > 0; --j) { s[j] = s[j - 1]; s[4 + j] = s[4 + j - 1]; }
        s[0] = s[8];
        s[4] = s[9];
    }
}

static double log_ratio(double v, double eps) {
    double r = log10((v > 1e-30 ? v : 1e-30) / eps);
    return r < -8 ? -8 : (r > 8 ? 8 : r);
}

/* The 16 features of Gaussian i at iteration k of K, with thresholds
 * eps_xyz, eps_rgb: 0-3 log10(history_xyz / eps_xyz), 4-7 the same for rgb
 * (each clamped to [-8, 8], norms below 1e-30 read as 1e-30), 8 opacity
 * sigmoid(logit), 9 largest and 10 smallest log-scale, 11 ln(1 + views),
 * 12 k / K, 13-14 log10 of the current window's average norm over its
 * threshold (0 visible iterations read as a norm of 0), 15 min(frozen
 * boundaries, 8) / 8. */
void or_pred_features(int64_t n, const double *P, const float *acc_xyz, const float *acc_rgb, const int32_t *cnt,
                      const double *state, int32_t k, int32_t K, double eps_xyz, double eps_rgb, double *X) {
    for (int64_t i = 0; i < n; ++i) {
        const double *s = state + 12 * i, *p = P + NP * i;
        double *x = X + MLP_IN * i;
        for (int j = 0; j < 4; ++j) {
            x[j] = log_ratio(s[j], eps_xyz);
            x[4 + j] = log_ratio(s[4 + j], eps_rgb);
        }
        x[8] = PLANTED(24) ? p[10] : 1.0 / (1.0 + exp(-p[10]));
        double mx = p[3], mn = p[3];
        for (int j = 4; j < 6; ++j) { if (p[j] > mx) mx = p[j]; if (p[j] < mn) mn = p[j]; }
        x[9] = mx;
        x[10] = mn;
        x[11] = log(1.0 + s[10]);
        x[12] = (double)k / K;
        double ax = cnt[i] > 0 ? (double)acc_xyz[i] / cnt[i] : 0.0, ar = cnt[i] > 0 ? (double)acc_rgb[i] / cnt[i] : 0.0;
        x[13] = log_ratio(ax, eps_xyz);
        x[14] = log_ratio(ar, eps_rgb);
        x[15] = (s[11] < 8 ? s[11] : 8) / 8.0;
    }
}

/* Forward of one row: a1 = X W1 + b1, h1 = relu(a1), a2 = h1 W2 + b2,
 * h2 = relu(a2), z = h2 . W3 + b3. With round != 0 the inputs X, the
 * weights W1, W2, W3 and h1 (the second layer's input) are rounded to
 * bfloat16 first; biases are not. */
static double mlp_row(const double *xin, const double *prm, int round, double *xr, double *a1, double *h1r, double *a2,
                      double *h2) {
    for (int c = 0; c < MLP_IN; ++c) xr[c] = round ? or_bf16(xin[c]) : xin[c];
    for (int j = 0; j < MLP_H; ++j) {
        double s = prm[OFF_B1 + j];
        for (int c = 0; c < MLP_IN; ++c) {
            double w = prm[OFF_W1 + c * MLP_H + j];
            s += xr[c] * (round ? or_bf16(w) : w);
        }
        a1[j] = s;
        double h = (s > 0 || PLANTED(20)) ? s : 0;
        h1r[j] = round ? or_bf16(h) : h;
    }
    double z = prm[OFF_B3];
    for (int j = 0; j < MLP_H; ++j) {
        double s = prm[OFF_B2 + j];
        for (int c = 0; c < MLP_H; ++c) {
            double w = prm[OFF_W2 + c * MLP_H + j];
            s += h1r[c] * (round ? or_bf16(w) : w);
        }
        a2[j] = s;
        h2[j] = s > 0 ? s : 0;
        double w3 = prm[OFF_W3 + j];
        z += h2[j] * (round ? or_bf16(w3) : w3);
    }
    return z;
}

/* p[i] = sigmoid(z) of every row. */
void or_mlp_forward(int64_t n, const double *X, const double *prm, int32_t round, double *p) {
    double xr[MLP_IN], a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H];
    for (int64_t i = 0; i < n; ++i) {
        double z = mlp_row(X + MLP_IN * i, prm, round, xr, a1, h1, a2, h2);
        p[i] = 1.0 / (1.0 + exp(-z));
    }
}

/* Weighted binary cross-entropy L = sum_i w_i (softplus(z_i) - y_i z_i) /
 * sum_i w_i (w = NULL: all 1) and its gradient over the 5313 parameters
 * (added into grad). The gradient passes through the bfloat16 roundings as
 * the identity. abs_grad (optional) receives the sum of the absolute values
 * of the per-row terms of each gradient entry (the scale of its rounding
 * error in finite precision). Returns L. */
#define ADDG(k, v) do { double v_ = (v); grad[k] += v_; if (abs_grad) abs_grad[k] += fabs(v_); } while (0)
double or_mlp_loss_grad(int64_t n, const double *X, const double *y, const double *w, const double *prm,
                        int32_t round, double *grad, double *abs_grad) {
    double xr[MLP_IN], a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H], dh2[MLP_H], dh1[MLP_H];
    double wsum = 0, L = 0;
    for (int64_t i = 0; i < n; ++i) wsum += w ? w[i] : 1.0;
    for (int64_t i = 0; i < n; ++i) {
        double wi = (w ? w[i] : 1.0) / wsum;
        double z = mlp_row(X + MLP_IN * i, prm, round, xr, a1, h1, a2, h2);
        double sp = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
        L += wi * (sp - y[i] * z);
        double dz = wi * (1.0 / (1.0 + exp(-z)) - y[i]);
        ADDG(OFF_B3, dz);
        for (int j = 0; j < MLP_H; ++j) {
            double w3 = prm[OFF_W3 + j];
            ADDG(OFF_W3 + j, dz * h2[j]);
            dh2[j] = (a2[j] > 0 || PLANTED(21)) ? dz * (round ? or_bf16(w3) : w3) : 0.0;
            ADDG(OFF_B2 + j, dh2[j]);
        }
        for (int c = 0; c < MLP_H; ++c) {
            double s = 0;
            for (int j = 0; j < MLP_H; ++j) {
                double w2 = prm[OFF_W2 + c * MLP_H + j];
                ADDG(OFF_W2 + c * MLP_H + j, h1[c] * dh2[j]);
                s += dh2[j] * (round ? or_bf16(w2) : w2);
            }
            dh1[c] = a1[c] > 0 ? s : 0.0;
            ADDG(OFF_B1 + c, dh1[c]);
        }
        for (int c = 0; c < MLP_IN; ++c)
            for (int j = 0; j < MLP_H; ++j) ADDG(OFF_W1 + c * MLP_H + j, xr[c] * dh1[j]);
    }
    return L;
}
#undef ADDG

/* One Adam step on the predictor's parameters (textbook, bias-corrected). */
void or_mlp_adam(double *prm, const double *grad, double *m, double *v, double lr, double b1, double b2, double eps,
                 int64_t step) {
    double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
    for (int k = 0; k < MLP_NPARAM; ++k) {
        m[k] = b1 * m[k] + (1 - b1) * grad[k];
        v[k] = b2 * v[k] + (1 - b2) * grad[k] * grad[k];
        prm[k] -= lr * (m[k] / (PLANTED(26) ? 1.0 : bc1)) / (sqrt(v[k] / bc2) + eps);
    }
}

/* Predicted freezing: frozen |= prob > tau; the unfrozen indices in
 * ascending order go to act. Statistics are not touched. Returns their count. */
int64_t or_freeze_apply(int64_t n, const float *prob, float tau, uint8_t *frozen, int32_t *act) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (prob[i] > tau) frozen[i] = 1;
        else if (PLANTED(25)) frozen[i] = 0;
        if (!frozen[i]) act[k++] = (int32_t)i;
    }
    return k;
}
