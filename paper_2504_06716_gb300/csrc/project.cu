// Projection of 3-D Gaussians to 2-D splats (Sec. 3.1, Eq. 1) with SH colour,
// and its backward (Sec. 3.2.4) over the list of unfrozen Gaussians.
//
// One thread per Gaussian. A parameter row is 256 contiguous bytes read as
// 16-byte vectors, so a Gaussian that is not on screen costs one 48-byte
// read (mean, scales, rotation, opacity) and its 192 bytes of SH are never
// fetched. The backward runs over the compacted active list, so a frozen
// Gaussian is never read or written.
#include <algorithm>

#include "common.cuh"

namespace gs {
namespace {

// Real SH basis, degree <= 3, Condon-Shortley phase, coefficient c = l^2 + l + m.
// Constants are the normalisations sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), times
// sqrt(2) for m != 0, folded into the Cartesian polynomials.
constexpr float kY00 = 0.28209479177387814f;  // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15/(16 pi))
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35/(32 pi))
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105/(4 pi))
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21/(32 pi))
constexpr float kY3d = 0.37317633259011540f;  // sqrt(7/(16 pi))
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105/(16 pi))

__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = kY00;
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (3.f * zz - 1.f);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (xx - yy);
    Y[9] = -kY3a * y * (3.f * xx - yy);
    Y[10] = kY3b * x * y * z;
    Y[11] = -kY3c * y * (5.f * zz - 1.f);
    Y[12] = kY3d * z * (5.f * zz - 3.f);
    Y[13] = -kY3c * x * (5.f * zz - 1.f);
    Y[14] = kY3e * z * (xx - yy);
    Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// d Y_c / d(x, y, z) of the polynomials above, accumulated with weight w_c.
__device__ __forceinline__ void sh_basis_grad_acc(float x, float y, float z, const float *w, float &gx, float &gy,
                                                  float &gz) {
    float xx = x * x, yy = y * y, zz = z * z;
    gy += -kY1 * w[1];
    gz += kY1 * w[2];
    gx += -kY1 * w[3];
    gx += kY2a * y * w[4];
    gy += kY2a * x * w[4];
    gy += -kY2a * z * w[5];
    gz += -kY2a * y * w[5];
    gz += 6.f * kY2b * z * w[6];
    gx += -kY2a * z * w[7];
    gz += -kY2a * x * w[7];
    gx += 2.f * kY2c * x * w[8];
    gy += -2.f * kY2c * y * w[8];
    gx += -6.f * kY3a * x * y * w[9];
    gy += -3.f * kY3a * (xx - yy) * w[9];
    gx += kY3b * y * z * w[10];
    gy += kY3b * x * z * w[10];
    gz += kY3b * x * y * w[10];
    gy += -kY3c * (5.f * zz - 1.f) * w[11];
    gz += -10.f * kY3c * y * z * w[11];
    gz += kY3d * (15.f * zz - 3.f) * w[12];
    gx += -kY3c * (5.f * zz - 1.f) * w[13];
    gz += -10.f * kY3c * x * z * w[13];
    gx += 2.f * kY3e * x * z * w[14];
    gy += -2.f * kY3e * y * z * w[14];
    gz += kY3e * (xx - yy) * w[14];
    gx += -3.f * kY3a * (xx - yy) * w[15];
    gy += 6.f * kY3a * x * y * w[15];
}

// Geometry of one Gaussian in one view, shared by forward and backward.
struct Geo {
    float tx, ty, tz;         // camera-space mean
    float s[3];               // scales
    float qw, qx, qy, qz;     // unit quaternion
    float qinv;               // 1 / |q|
    float R[9];               // rotation of the Gaussian
    float S00, S01, S02, S11, S12, S22;  // 3-D covariance
    float T0[3], T1[3];       // rows of J W
    float cu, cv;             // clamped tan-space coordinates
    bool clampx, clampy;
    float A, B, C;            // 2-D covariance incl. dilation
    float det;
};

// Returns false if the Gaussian is culled by the near plane or a degenerate
// 2-D covariance.
__device__ __forceinline__ bool geometry(const float4 r0, const float4 r1, const float4 r2, const DevCam &cam, Geo &g) {
    const float mx = r0.x, my = r0.y, mz = r0.z;
    g.tx = cam.R[0] * mx + cam.R[1] * my + cam.R[2] * mz + cam.t[0];
    g.ty = cam.R[3] * mx + cam.R[4] * my + cam.R[5] * mz + cam.t[1];
    g.tz = cam.R[6] * mx + cam.R[7] * my + cam.R[8] * mz + cam.t[2];
    if (!(g.tz > cam.znear)) return false;

    g.s[0] = expf(r0.w);
    g.s[1] = expf(r1.x);
    g.s[2] = expf(r1.y);
    float qw = r1.z, qx = r1.w, qy = r2.x, qz = r2.y;
    float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    g.qinv = rsqrtf(qn2);
    qw *= g.qinv; qx *= g.qinv; qy *= g.qinv; qz *= g.qinv;
    g.qw = qw; g.qx = qx; g.qy = qy; g.qz = qz;
    float *R = g.R;
    R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
    // Sigma = (R S)(R S)^T
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * g.s[j];
    g.S00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    g.S01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    g.S02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    g.S11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    g.S12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    g.S22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];

    float iz = 1.f / g.tz;
    float u = g.tx * iz, v = g.ty * iz;
    g.clampx = (u > cam.limx) || (u < -cam.limx);
    g.clampy = (v > cam.limy) || (v < -cam.limy);
    g.cu = fminf(fmaxf(u, -cam.limx), cam.limx);
    g.cv = fminf(fmaxf(v, -cam.limy), cam.limy);
    // J = [[fx/z, 0, -fx cu/z], [0, fy/z, -fy cv/z]]; T = J W
    float j00 = cam.fx * iz, j02 = -cam.fx * g.cu * iz, j11 = cam.fy * iz, j12 = -cam.fy * g.cv * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.T0[k] = j00 * cam.R[k] + j02 * cam.R[6 + k];
        g.T1[k] = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
    }
    // U = T Sigma
    float U0[3], U1[3];
    U0[0] = g.T0[0] * g.S00 + g.T0[1] * g.S01 + g.T0[2] * g.S02;
    U0[1] = g.T0[0] * g.S01 + g.T0[1] * g.S11 + g.T0[2] * g.S12;
    U0[2] = g.T0[0] * g.S02 + g.T0[1] * g.S12 + g.T0[2] * g.S22;
    U1[0] = g.T1[0] * g.S00 + g.T1[1] * g.S01 + g.T1[2] * g.S02;
    U1[1] = g.T1[0] * g.S01 + g.T1[1] * g.S11 + g.T1[2] * g.S12;
    U1[2] = g.T1[0] * g.S02 + g.T1[1] * g.S12 + g.T1[2] * g.S22;
    g.A = U0[0] * g.T0[0] + U0[1] * g.T0[1] + U0[2] * g.T0[2] + cam.dilation;
    g.B = U0[0] * g.T1[0] + U0[1] * g.T1[1] + U0[2] * g.T1[2];
    g.C = U1[0] * g.T1[0] + U1[1] * g.T1[1] + U1[2] * g.T1[2] + cam.dilation;
    g.det = g.A * g.C - g.B * g.B;
    return g.det > 0.f;
}

__device__ __forceinline__ void write_culled(float *out, int64_t i) {
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 *o = reinterpret_cast<float4 *>(out + i * kSplat);
    o[0] = z;
    o[1] = z;
    o[2] = z;
}

// Opacity from its parameter x: sigmoid(x), or |x| under the absolute-value
// activation of the finetuning stage (Sec. 4.1); and d opacity / dx.
__device__ __forceinline__ float opacity_of(float x, int abs_act) {
    return abs_act ? fabsf(x) : opacity_sigmoid(x);
}

__device__ __forceinline__ float opacity_slope(float x, int abs_act) {
    if (abs_act) return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f);
    const float o = opacity_sigmoid(x);
    return o * (1.f - o);
}

// Volume mask (Sec. 3.3, "Pruning with Volume Masking"): float 59 of a row is
// the mask logit m; the hard mask is 1[sigmoid(m) > 0.01], i.e. m > logit(0.01).
// A Gaussian whose mask is 0 has zero opacity and zero scale: it is culled.
constexpr float kMaskLogitMin = -4.59511985f;  // logit(0.01) in float32

__device__ __forceinline__ bool masked_off(const float *__restrict__ P, int64_t i, int flags) {
    return (flags & GS_VOLUME_MASK) && !(__ldg(P + i * kRow + 59) > kMaskLogitMin);
}

__global__ void __launch_bounds__(256) k_project_fwd(const float *__restrict__ P, int64_t n, int deg, int flags,
                                                     DevCam cam, float *__restrict__ out) {
    wait_prior_grid();
    const int abs_act = flags & GS_OPACITY_ABS;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 *row = reinterpret_cast<const float4 *>(P + i * kRow);
    float4 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2);
    Geo g;
    if (masked_off(P, i, flags) || !geometry(r0, r1, r2, cam, g)) { write_culled(out, i); return; }
    float iz = 1.f / g.tz;
    float mean_x = cam.fx * g.tx * iz + cam.cx;
    float mean_y = cam.fy * g.ty * iz + cam.cy;
    float half = 0.5f * (g.A + g.C), dif = 0.5f * (g.A - g.C);
    float lam = half + sqrtf(dif * dif + g.B * g.B);
    int radius = (int)ceilf(3.f * sqrtf(lam));
    int x0, y0, x1, y1;
    int tiles = radius > 0 ? tile_rect(mean_x, mean_y, radius, cam.tile, cam.tiles_x, cam.tiles_y, x0, y0, x1, y1) : 0;
    if (tiles == 0) { write_culled(out, i); return; }
    float idet = 1.f / g.det;
    float ca = g.C * idet, cb = -g.B * idet, cc = g.A * idet;
    float opacity = opacity_of(r2.z, abs_act);

    // SH colour at the view direction; SH rows are fetched only here.
    float dx = r0.x - cam.campos[0], dy = r0.y - cam.campos[1], dz = r0.z - cam.campos[2];
    float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_basis(dx * il, dy * il, dz * il, Y);
    float sh[48];
    sh[0] = r2.w;
#pragma unroll
    for (int c = 3; c < 15; ++c) {
        float4 v = __ldg(row + c);
        int f = 4 * c - 11;
        sh[f] = v.x;
        sh[f + 1] = v.y;
        sh[f + 2] = v.z;
        if (f + 3 < 48) sh[f + 3] = v.w;
    }
    int nc = (deg + 1) * (deg + 1);
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < nc) acc += sh[3 * c + ch] * Y[c];
        rgb[ch] = fmaxf(acc, 0.f);
    }
    float4 *o = reinterpret_cast<float4 *>(out + i * kSplat);
    o[0] = make_float4(mean_x, mean_y, ca, cb);
    o[1] = make_float4(cc, opacity, rgb[0], rgb[1]);
    o[2] = make_float4(rgb[2], g.tz, __int_as_float(radius), __int_as_float(tiles));
}

// Up to two statistics windows updated by the backward (e.g. freezing and
// densification), passed by value.
struct StatSets {
    float *ax[2], *ar[2];
    int32_t *cnt[2], *maxr[2];
    int n;
};

// Backward of the projection for act[0 .. *n_active). See gs_project_bwd;
// with ACC the gradient rows are added to G instead of written.
// One instance for both modes (ACC a run-time flag), so that the row added
// under ACC is bit for bit the row written without it.
__device__ __forceinline__ void project_bwd_one(int64_t k, const float *__restrict__ P, int deg, int flags,
                                                float mask_loss, const DevCam &cam, const float *__restrict__ splats,
                                                const int32_t *__restrict__ act, float *__restrict__ grad2d,
                                                float *__restrict__ G, const StatSets &st, int ACC) {
    const int abs_act = flags & GS_OPACITY_ABS;
    const int64_t i = act[k];
    float4 *gout = reinterpret_cast<float4 *>(G + i * kRow);
    const int radius = __float_as_int(__ldg(splats + i * kSplat + 10));
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // volume mask: sigmoid'(m), the straight-through derivative of the hard mask
    float mslope = 0.f;
    if (flags & GS_VOLUME_MASK) {
        const float sm = opacity_sigmoid(__ldg(P + i * kRow + 59));
        mslope = sm * (1.f - sm);
    }
    if (radius <= 0) {
        if (!ACC) {
#pragma unroll
            for (int c = 0; c < 16; ++c) gout[c] = z4;
        }
        if (mslope != 0.f) {  // only the mask term of the loss reaches it
            float *g59 = G + i * kRow + 59;
            const float gm = mask_loss * mslope;
            *g59 = ACC ? __fadd_rn(*g59, gm) : gm;
        }
        return;
    }
    float4 *g2p = reinterpret_cast<float4 *>(grad2d + i * kG2d);
    const float4 ga = g2p[0], gb = g2p[1], gc4 = g2p[2];
    g2p[0] = z4; g2p[1] = z4; g2p[2] = z4;
    const float dmx = ga.x, dmy = ga.y, dca = ga.z, dcb = ga.w, dcc = gb.x, dop = gb.y;
    float drgb[3] = {gb.z, gb.w, gc4.x};

    const float4 *row = reinterpret_cast<const float4 *>(P + i * kRow);
    const float4 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2);
    Geo g;
    geometry(r0, r1, r2, cam, g);  // visible in this view, so not culled

    // ---- colour: c = max(0, sum_c k_c Y_c(d) + 1/2) ----
    float vx = r0.x - cam.campos[0], vy = r0.y - cam.campos[1], vz = r0.z - cam.campos[2];
    float il = rsqrtf(vx * vx + vy * vy + vz * vz);
    float x = vx * il, y = vy * il, z = vz * il;
    float Y[16];
    sh_basis(x, y, z, Y);
    float sh[48];
    sh[0] = r2.w;
#pragma unroll
    for (int c = 3; c < 15; ++c) {
        float4 v = __ldg(row + c);
        int f = 4 * c - 11;
        sh[f] = v.x;
        sh[f + 1] = v.y;
        sh[f + 2] = v.z;
        if (f + 3 < 48) sh[f + 3] = v.w;
    }
    const int nc = (deg + 1) * (deg + 1);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float raw = 0.5f;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < nc) raw += sh[3 * c + ch] * Y[c];
        if (!(raw > 0.f)) drgb[ch] = 0.f;
    }
    float w[16];
    float gsh[48];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        bool on = c < nc;
        w[c] = on ? sh[3 * c] * drgb[0] + sh[3 * c + 1] * drgb[1] + sh[3 * c + 2] * drgb[2] : 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gsh[3 * c + ch] = on ? Y[c] * drgb[ch] : 0.f;
    }
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
    sh_basis_grad_acc(x, y, z, w, gdx, gdy, gdz);
    float dd = gdx * x + gdy * y + gdz * z;
    float dmu0 = (gdx - x * dd) * il, dmu1 = (gdy - y * dd) * il, dmu2 = (gdz - z * dd) * il;

    // ---- opacity = sigmoid(x) or |x| ----
    float dlogit = dop * opacity_slope(r2.z, abs_act);

    // ---- conic = inverse of [[A, B], [B, C]] ----
    float id2 = 1.f / (g.det * g.det);
    float dA = (-g.C * g.C * dca + g.B * g.C * dcb - g.B * g.B * dcc) * id2;
    float dC = (-g.B * g.B * dca + g.A * g.B * dcb - g.A * g.A * dcc) * id2;
    float dB = (2.f * g.B * g.C * dca - (g.det + 2.f * g.B * g.B) * dcb + 2.f * g.A * g.B * dcc) * id2;

    // ---- 2-D covariance = T Sigma T^T: dSigma and dT ----
    // dSigma = dA T0 T0^T + dB (T0 T1^T + T1 T0^T)/2 + dC T1 T1^T
    const float *T0 = g.T0, *T1 = g.T1;
    float hB = 0.5f * dB;
    float G00 = dA * T0[0] * T0[0] + 2.f * hB * T0[0] * T1[0] + dC * T1[0] * T1[0];
    float G11 = dA * T0[1] * T0[1] + 2.f * hB * T0[1] * T1[1] + dC * T1[1] * T1[1];
    float G22 = dA * T0[2] * T0[2] + 2.f * hB * T0[2] * T1[2] + dC * T1[2] * T1[2];
    float G01 = dA * T0[0] * T0[1] + hB * (T0[0] * T1[1] + T1[0] * T0[1]) + dC * T1[0] * T1[1];
    float G02 = dA * T0[0] * T0[2] + hB * (T0[0] * T1[2] + T1[0] * T0[2]) + dC * T1[0] * T1[2];
    float G12 = dA * T0[1] * T0[2] + hB * (T0[1] * T1[2] + T1[1] * T0[2]) + dC * T1[1] * T1[2];
    // U = T Sigma; dT0 = 2 dA U0 + dB U1, dT1 = dB U0 + 2 dC U1
    float U0[3], U1[3];
    U0[0] = T0[0] * g.S00 + T0[1] * g.S01 + T0[2] * g.S02;
    U0[1] = T0[0] * g.S01 + T0[1] * g.S11 + T0[2] * g.S12;
    U0[2] = T0[0] * g.S02 + T0[1] * g.S12 + T0[2] * g.S22;
    U1[0] = T1[0] * g.S00 + T1[1] * g.S01 + T1[2] * g.S02;
    U1[1] = T1[0] * g.S01 + T1[1] * g.S11 + T1[2] * g.S12;
    U1[2] = T1[0] * g.S02 + T1[1] * g.S12 + T1[2] * g.S22;
    float dT0[3], dT1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dT0[a] = 2.f * dA * U0[a] + dB * U1[a];
        dT1[a] = dB * U0[a] + 2.f * dC * U1[a];
    }
    // ---- T = J W: only J00, J02, J11, J12 vary ----
    const float *W = cam.R;
    float dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
    float dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
    float dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
    float dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
    float iz = 1.f / g.tz, iz2 = iz * iz;
    float dtz = -cam.fx * iz2 * dJ00 - cam.fy * iz2 * dJ11 + cam.fx * g.cu * iz2 * dJ02 + cam.fy * g.cv * iz2 * dJ12;
    float du = (g.clampx ? 0.f : -cam.fx * iz * dJ02) + cam.fx * dmx;
    float dv = (g.clampy ? 0.f : -cam.fy * iz * dJ12) + cam.fy * dmy;
    float dtx = du * iz, dty = dv * iz;
    dtz -= (du * g.tx + dv * g.ty) * iz2;
    dmu0 += W[0] * dtx + W[3] * dty + W[6] * dtz;
    dmu1 += W[1] * dtx + W[4] * dty + W[7] * dtz;
    dmu2 += W[2] * dtx + W[5] * dty + W[8] * dtz;

    // ---- Sigma = M M^T, M = R diag(s): dM = 2 dSigma M ----
    const float *R = g.R;
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[3 * a + b] = R[3 * a + b] * g.s[b];
    float Gs[9] = {G00, G01, G02, G01, G11, G12, G02, G12, G22};
    float dR[9], dls[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float ds = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float dM = 2.f * (Gs[3 * a] * M[b] + Gs[3 * a + 1] * M[3 + b] + Gs[3 * a + 2] * M[6 + b]);
            ds += dM * R[3 * a + b];
            dR[3 * a + b] = dM * g.s[b];
        }
        dls[b] = ds * g.s[b];
    }
    // ---- R(q) for a unit quaternion, then through q / |q| ----
    const float qw = g.qw, qx = g.qx, qy = g.qy, qz = g.qz;
    float dqw = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    float dqx = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] +
                       qw * dR[7] - 2.f * qx * dR[8]);
    float dqy = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] +
                       qz * dR[7] - 2.f * qy * dR[8]);
    float dqz = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] + qy * dR[5] +
                       qx * dR[6] + qy * dR[7]);
    float qd = dqw * qw + dqx * qx + dqy * qy + dqz * qz;
    dqw = (dqw - qw * qd) * g.qinv;
    dqx = (dqx - qx * qd) * g.qinv;
    dqy = (dqy - qy * qd) * g.qinv;
    dqz = (dqz - qz * qd) * g.qinv;

    // ---- write the 64-float gradient row ----
    float grow[64];
    grow[0] = dmu0; grow[1] = dmu1; grow[2] = dmu2;
    grow[3] = dls[0]; grow[4] = dls[1]; grow[5] = dls[2];
    grow[6] = dqw; grow[7] = dqx; grow[8] = dqy; grow[9] = dqz;
    grow[10] = dlogit;
#pragma unroll
    for (int f = 0; f < 48; ++f) grow[11 + f] = gsh[f];
#pragma unroll
    for (int f = 59; f < 64; ++f) grow[f] = 0.f;
    if (flags & GS_VOLUME_MASK) {
        // o' = M o and s' = M s with the hard mask M = 1 here: dL/dM =
        // dL/do' o + sum_b dL/ds'_b s_b = dop o + sum_b dL/dlog s_b
        const float dM = dop * opacity_of(r2.z, abs_act) + dls[0] + dls[1] + dls[2];
        grow[59] = (dM + mask_loss) * mslope;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        float4 v = make_float4(grow[4 * c], grow[4 * c + 1], grow[4 * c + 2], grow[4 * c + 3]);
        if (ACC) {
            const float4 o = gout[c];  // a plain add, never fused with the product before it
            v.x = __fadd_rn(v.x, o.x); v.y = __fadd_rn(v.y, o.y);
            v.z = __fadd_rn(v.z, o.z); v.w = __fadd_rn(v.w, o.w);
        }
        gout[c] = v;
    }

    if (st.n) {
        const float ex = dmx * 0.5f * (float)cam.W, ey = dmy * 0.5f * (float)cam.H;
        const float nx = sqrtf(ex * ex + ey * ey), nr = sqrtf(gsh[0] * gsh[0] + gsh[1] * gsh[1] + gsh[2] * gsh[2]);
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {  // constant indices: st stays in parameter space
            if (k2 >= st.n) break;
            st.ax[k2][i] += nx;
            st.ar[k2][i] += nr;
            st.cnt[k2][i] += 1;
            if (st.maxr[k2] && radius > st.maxr[k2][i]) st.maxr[k2][i] = radius;
        }
    }
}

// A grid sized for the device, each thread walking the active list with a
// stride: the list's length is known only on the device.
__global__ void __launch_bounds__(128, 4) k_project_bwd(const float *__restrict__ P, int deg, int flags, float mask_loss,
                                                     DevCam cam, const float *__restrict__ splats,
                                                     const int32_t *__restrict__ act,
                                                     const int32_t *__restrict__ n_active, float *__restrict__ grad2d,
                                                     float *__restrict__ G, StatSets st, int ACC) {
    wait_prior_grid();
    const int64_t na = *n_active;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < na; k += (int64_t)gridDim.x * blockDim.x)
        project_bwd_one(k, P, deg, flags, mask_loss, cam, splats, act, grad2d, G, st, ACC);
}

}  // namespace
}  // namespace gs

using namespace gs;

static bool flags_ok(int32_t flags) { return (flags & ~(GS_OPACITY_ABS | GS_VOLUME_MASK)) == 0; }

extern "C" int gs_project_ex(const float *P, int64_t n, int32_t sh_degree, int32_t opacity_act,
                             const gs_camera *cam, float *splats, gs_stream_t stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !camera_ok(cam)) return GS_ERR_INVALID_ARG;
    if (!flags_ok(opacity_act)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !splats) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(splats)) & 15) return GS_ERR_INVALID_ARG;
    launch_chained(k_project_fwd, grid_for(n, 256), 256, as_stream(stream), P, n, sh_degree, opacity_act, make_cam(cam),
                   splats);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_project(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, float *splats,
                          gs_stream_t stream) {
    return gs_project_ex(P, n, sh_degree, GS_OPACITY_SIGMOID, cam, splats, stream);
}

static int project_bwd(bool acc, const float *P, int64_t n, int32_t sh_degree, int32_t opacity_act,
                       float mask_loss, const gs_camera *cam, const float *splats, const int32_t *act,
                       const int32_t *n_active_dev, float *grad2d, float *G, const gs_grad_stats *sets,
                       int32_t n_sets, gs_stream_t stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !camera_ok(cam) || n_sets < 0 || n_sets > 2 ||
        (n_sets > 0 && !sets) || !flags_ok(opacity_act) || !(mask_loss >= 0.f))
        return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !splats || !act || !n_active_dev || !grad2d || !G) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(splats) | reinterpret_cast<uintptr_t>(grad2d) |
         reinterpret_cast<uintptr_t>(G)) & 15)
        return GS_ERR_INVALID_ARG;
    StatSets st{};
    st.n = n_sets;
    for (int k = 0; k < n_sets; ++k) {
        if (!sets[k].acc_xyz || !sets[k].acc_rgb || !sets[k].cnt) return GS_ERR_INVALID_ARG;
        st.ax[k] = sets[k].acc_xyz;
        st.ar[k] = sets[k].acc_rgb;
        st.cnt[k] = sets[k].cnt;
        st.maxr[k] = sets[k].max_radius;
    }
    const DevCam dc = make_cam(cam);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // as many blocks as are resident at once: the grid-stride loop then runs in
    // one wave, every block with the same share of the active list
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_project_bwd, 128, 0) != cudaSuccess || v < 1) v = 2;
        per_sm = v;
    }
    const unsigned grid = std::min<unsigned>(grid_for(n, 128), (unsigned)(sms > 0 ? sms : 152) * (unsigned)per_sm);
    launch_chained(k_project_bwd, grid, 128, as_stream(stream), P, sh_degree, opacity_act, mask_loss, dc, splats, act,
                   n_active_dev, grad2d, G, st, acc ? 1 : 0);
    note_launches(1);
    return launch_status();
}

static int project_bwd_one(bool acc, const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam,
                           const float *splats, const int32_t *act, const int32_t *n_active_dev, float *grad2d,
                           float *G, float *acc_xyz, float *acc_rgb, int32_t *cnt, gs_stream_t stream) {
    const bool any_stat = acc_xyz || acc_rgb || cnt, all_stat = acc_xyz && acc_rgb && cnt;
    if (any_stat && !all_stat) return GS_ERR_INVALID_ARG;
    const gs_grad_stats one{acc_xyz, acc_rgb, cnt, nullptr};
    return project_bwd(acc, P, n, sh_degree, GS_OPACITY_SIGMOID, 0.f, cam, splats, act, n_active_dev, grad2d, G,
                       all_stat ? &one : nullptr, all_stat ? 1 : 0, stream);
}

extern "C" int gs_project_bwd(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam,
                              const float *splats, const int32_t *act, const int32_t *n_active_dev, float *grad2d,
                              float *G, float *acc_xyz, float *acc_rgb, int32_t *cnt, gs_stream_t stream) {
    return project_bwd_one(false, P, n, sh_degree, cam, splats, act, n_active_dev, grad2d, G, acc_xyz, acc_rgb, cnt,
                           stream);
}

extern "C" int gs_project_bwd_accum(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam,
                                    const float *splats, const int32_t *act, const int32_t *n_active_dev,
                                    float *grad2d, float *G, float *acc_xyz, float *acc_rgb, int32_t *cnt,
                                    gs_stream_t stream) {
    return project_bwd_one(true, P, n, sh_degree, cam, splats, act, n_active_dev, grad2d, G, acc_xyz, acc_rgb, cnt,
                           stream);
}

extern "C" int gs_project_bwd_stats(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam,
                                    const float *splats, const int32_t *act, const int32_t *n_active_dev,
                                    float *grad2d, float *G, int32_t accumulate, const gs_grad_stats *sets,
                                    int32_t n_sets, gs_stream_t stream) {
    return project_bwd(accumulate != 0, P, n, sh_degree, GS_OPACITY_SIGMOID, 0.f, cam, splats, act, n_active_dev,
                       grad2d, G, sets, n_sets, stream);
}

extern "C" int gs_project_bwd_ex(const float *P, int64_t n, int32_t sh_degree, int32_t opacity_act,
                                 float mask_loss, const gs_camera *cam, const float *splats, const int32_t *act,
                                 const int32_t *n_active_dev, float *grad2d, float *G, int32_t accumulate,
                                 const gs_grad_stats *sets, int32_t n_sets, gs_stream_t stream) {
    return project_bwd(accumulate != 0, P, n, sh_degree, opacity_act, mask_loss, cam, splats, act, n_active_dev,
                       grad2d, G, sets, n_sets, stream);
}
