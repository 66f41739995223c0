// SH + SG view-dependent colour (Eq. 4-9) on the device, forward and gradient.
//
// Real SH basis Y_lm, index l*l + l + m, Condon-Shortley phase, written as polynomials of
// the unit direction d = (x, y, z).  The constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0) multiplied into the
// Legendre-derivative factors:
//   l=0: 1/(2 sqrt(pi))
//   l=1: sqrt(3/(4 pi)) {-y, z, -x}
//   l=2: 1/2 sqrt(15/pi) {xy, -yz, -xz}, 1/4 sqrt(5/pi) (3z^2-1), 1/4 sqrt(15/pi) (x^2-y^2)
//   l=3: -1/4 sqrt(35/(2pi)) {y(3x^2-y^2), x(x^2-3y^2)}, 1/2 sqrt(105/pi) xyz,
//        -1/4 sqrt(21/(2pi)) {y, x}(5z^2-1), 1/4 sqrt(7/pi) z(5z^2-3),
//        1/4 sqrt(105/pi) z(x^2-y^2)
// SG lobe (Eq. 5): a_k exp(lambda_k (mu_k . d - 1)), mu_k normalised (free axes) or the
// world axis e_k (Eq. 7-8 with the axes of Sec. "Implementation").
// colour = max(0, SH(d) + 0.5 + sum_k SG_k(d)) per channel (Eq. 9 with the diffuse term
// being the l = 0 SH band).
#pragma once
#include "sgs.h"

namespace sgs {

constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.4886025119029199f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.5462742152960396f;
constexpr float kY3a = -0.5900435899266435f;
constexpr float kY3b = 2.890611442640554f;
constexpr float kY3c = -0.4570457994644658f;
constexpr float kY3d = 0.3731763325901154f;
constexpr float kY3e = 1.445305721320277f;

template <int L>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kY0;
    if (L >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (L >= 2) {
        const float z2 = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (3.0f * z2 - 1.0f);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (x * x - y * y);
    }
    if (L >= 3) {
        const float x2 = x * x, y2 = y * y, z2 = z * z;
        Y[9] = kY3a * y * (3.0f * x2 - y2);
        Y[10] = kY3b * x * y * z;
        Y[11] = kY3c * y * (5.0f * z2 - 1.0f);
        Y[12] = kY3d * z * (5.0f * z2 - 3.0f);
        Y[13] = kY3c * x * (5.0f * z2 - 1.0f);
        Y[14] = kY3e * z * (x2 - y2);
        Y[15] = kY3a * x * (x2 - 3.0f * y2);
    }
}

// Accumulates g_k * grad(Y_k) (ambient gradient of the polynomial forms above).
template <int L>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float* g, float& gx,
                                             float& gy, float& gz) {
    if (L >= 1) {
        gx += -kY1 * g[3];
        gy += -kY1 * g[1];
        gz += kY1 * g[2];
    }
    if (L >= 2) {
        gx += kY2a * y * g[4] - kY2a * z * g[7] + 2.0f * kY2c * x * g[8];
        gy += kY2a * x * g[4] - kY2a * z * g[5] - 2.0f * kY2c * y * g[8];
        gz += -kY2a * y * g[5] + 6.0f * kY2b * z * g[6] - kY2a * x * g[7];
    }
    if (L >= 3) {
        const float x2 = x * x, y2 = y * y, z2 = z * z;
        gx += 6.0f * kY3a * x * y * g[9] + kY3b * y * z * g[10] + kY3c * (5.0f * z2 - 1.0f) * g[13] +
              2.0f * kY3e * x * z * g[14] + kY3a * (3.0f * x2 - 3.0f * y2) * g[15];
        gy += kY3a * (3.0f * x2 - 3.0f * y2) * g[9] + kY3b * x * z * g[10] +
              kY3c * (5.0f * z2 - 1.0f) * g[11] - 2.0f * kY3e * y * z * g[14] - 6.0f * kY3a * x * y * g[15];
        gz += kY3b * x * y * g[10] + 10.0f * kY3c * y * z * g[11] + kY3d * (15.0f * z2 - 3.0f) * g[12] +
              10.0f * kY3c * x * z * g[13] + kY3e * (x2 - y2) * g[14];
    }
}

// |m| of a lobe axis, in one written-out operation order (the forward and the backward
// pass must normalise an axis to the same bits).
__device__ __forceinline__ float axis_length(const float m[3]) {
    return sqrtf(fmaf(m[0], m[0], fmaf(m[1], m[1], m[2] * m[2])));
}

// Lobe-axis layouts (sgs_axis_mode): 0 free unit axes, 1 the world axes, 2 the columns of
// a per-Gaussian rotation given by 3 parameters.
constexpr int kAxFree = 0, kAxWorld = 1, kAxFrame = 2;

// Rotation matrix of the unit quaternion q = (w, x, y, z) (the covariance rotation of Eq. 3
// and the lobe frame use the same map).
__device__ __forceinline__ void quat_to_matrix(const float q[4], float R[3][3]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
}

// dL/dq of R(q) for a unit q, given dL/dR (the unnormalised-quaternion chain is separate).
__device__ __forceinline__ void quat_to_matrix_vjp(const float q[4], const float gR[3][3], float gq[4]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    gq[0] = 2.0f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    gq[1] = 2.0f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.0f * x * gR[1][1] - w * gR[1][2] +
                    z * gR[2][0] + w * gR[2][1] - 2.0f * x * gR[2][2]);
    gq[2] = 2.0f * (-2.0f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                    w * gR[2][0] + z * gR[2][1] - 2.0f * y * gR[2][2]);
    gq[3] = 2.0f * (-2.0f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.0f * z * gR[1][1] +
                    y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
}

// The orthonormal lobe frame of 3 parameters f (Sec. "Multi-Axis Orthogonal Gaussians": 3
// parameters fix the orthogonal directions): q = (1, f0, f1, f2) / |(1, f0, f1, f2)|, the
// lobe axes are the columns of R(q).  f = 0 is the world frame.  Returns |(1, f)|.
__device__ __forceinline__ float frame_axes(const float f[3], float q[4], float R[3][3]) {
    const float n = sqrtf(fmaf(f[0], f[0], fmaf(f[1], f[1], fmaf(f[2], f[2], 1.0f))));
    const float inv = 1.0f / n;
    q[0] = inv;
    q[1] = f[0] * inv;
    q[2] = f[1] * inv;
    q[3] = f[2] * inv;
    quat_to_matrix(q, R);
    return n;
}

// Pre-clamp colour at unit direction d from the first nsh SH coefficients and the K lobes
// (Eq. 4, 5, 7, 9).  P provides csh(k, c), camp(k, c), caxis(k, c) (unit axes) and
// csharp(k).  The lobe's exponential is the hardware's (__expf, a few 1e-7 relative at
// the sharpness range's exponents): colour is not a binning decision, and the backward pass
// takes the forward's colour-clamp decisions from the record's flags, not from its own
// evaluation.
template <int L, int K, int AX, class P>
__device__ __forceinline__ void colour_eval(const P& p, const float* d, float* pre, int nsh) {
    constexpr int NSH = (L + 1) * (L + 1);
    float Y[NSH];
    sh_basis<L>(d[0], d[1], d[2], Y);
#pragma unroll
    for (int c = 0; c < 3; ++c) pre[c] = 0.5f;
#pragma unroll
    for (int k = 0; k < NSH; ++k)
        if (k < nsh) {
#pragma unroll
            for (int c = 0; c < 3; ++c) pre[c] = fmaf(p.csh(k, c), Y[k], pre[c]);
        }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float cosv =
            AX == kAxWorld ? d[k] : fmaf(p.caxis(k, 0), d[0], fmaf(p.caxis(k, 1), d[1], p.caxis(k, 2) * d[2]));
        const float e = __expf(p.csharp(k) * (cosv - 1.0f));
#pragma unroll
        for (int c = 0; c < 3; ++c) pre[c] = fmaf(p.camp(k, c), e, pre[c]);
    }
}

// Number of SH coefficients a record sums: (D+1)^2 with D = sh_degree, or with adaptive
// degrees D = 0 / 1 / 2 as the record's integer pixel radius is below sh_radius[0] /
// below sh_radius[1] / not (capped at the stored degree L).
template <int L>
__device__ __forceinline__ int record_sh_degree(const sgs_gaussians& g, float radius) {
    int D = L;
    if (g.sh_adaptive) {
        D = radius < g.sh_radius[0] ? 0 : (radius < g.sh_radius[1] ? 1 : 2);
        D = D < L ? D : L;
    }
    return D;
}
template <int L>
__device__ __forceinline__ int record_sh_coeffs(const sgs_gaussians& g, float radius) {
    const int D = record_sh_degree<L>(g, radius);
    return (D + 1) * (D + 1);
}

// Gradient accumulators of the colour parameters (summed over views).
template <int L, int K, int AX>
struct ColourGrads {
    static constexpr int NSH = (L + 1) * (L + 1);
    float sh[NSH][3];
    float amp[K > 0 ? K : 1][3];
    float axis[(K > 0 && AX != kAxWorld) ? K : 1][3];  // w.r.t. the unit axis
    float sharp[K > 0 ? K : 1];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < NSH; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) sh[k][c] = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                amp[k][c] = 0.0f;
                if (AX != kAxWorld) axis[k][c] = 0.0f;
            }
            sharp[k] = 0.0f;
        }
    }

    // g_pre: dL/d(pre-clamp colour) at direction d for a record that sums the first
    // `nsh` SH coefficients; accumulates into this and returns dL/dd (ambient) in gd.
    template <class P>
    __device__ __forceinline__ void accumulate(const P& p, const float* d, const float* g_pre, float* gd,
                                               int nsh) {
        float Y[NSH];
        sh_basis<L>(d[0], d[1], d[2], Y);
        float gY[NSH];
#pragma unroll
        for (int k = 0; k < NSH; ++k) {
            const float on = k < nsh ? 1.0f : 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) sh[k][c] = fmaf(g_pre[c] * on, Y[k], sh[k][c]);
            gY[k] = on * (g_pre[0] * p.csh(k, 0) + g_pre[1] * p.csh(k, 1) + g_pre[2] * p.csh(k, 2));
        }
        gd[0] = gd[1] = gd[2] = 0.0f;
        sh_basis_vjp<L>(d[0], d[1], d[2], gY, gd[0], gd[1], gd[2]);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float cs =
                AX == kAxWorld ? d[k] : fmaf(p.caxis(k, 0), d[0], fmaf(p.caxis(k, 1), d[1], p.caxis(k, 2) * d[2]));
            const float e = __expf(p.csharp(k) * (cs - 1.0f));
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                amp[k][c] = fmaf(g_pre[c], e, amp[k][c]);
                s = fmaf(g_pre[c] * p.camp(k, c), e, s);
            }
            sharp[k] = fmaf(s, cs - 1.0f, sharp[k]);
            const float gcos = s * p.csharp(k);
            if (AX == kAxWorld) {
                gd[k] += gcos;
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gd[c] = fmaf(gcos, p.caxis(k, c), gd[c]);
                    axis[k][c] = fmaf(gcos, d[c], axis[k][c]);
                }
            }
        }
    }

    // P: the colour parameters' accessors (csh, camp, caxis, csharp, caxis_norm, cframe_q,
    // cframe_norm; ColourShared of the preprocess)
    template <class P>
    __device__ __forceinline__ void store(const P& p, const sgs_grads& out, int64_t S, int64_t i) const {
#pragma unroll
        for (int k = 0; k < NSH; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) out.sh[(k * 3 + c) * S + i] = sh[k][c];
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) out.sg_amp[(k * 3 + c) * S + i] = amp[k][c];
            out.sg_sharp[k * S + i] = sharp[k];
            if constexpr (AX == kAxFree) {
                // mu = m/|m|:  dL/dm = (g - mu (mu . g)) / |m|
                const float dot =
                    axis[k][0] * p.caxis(k, 0) + axis[k][1] * p.caxis(k, 1) + axis[k][2] * p.caxis(k, 2);
                const float inv = 1.0f / p.caxis_norm(k);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    out.sg_axis[(k * 3 + c) * S + i] = (axis[k][c] - p.caxis(k, c) * dot) * inv;
            }
        }
        if constexpr (AX == kAxFrame && K > 0) {
            // mu_k = column k of R(q): dL/dR[c][k] = dL/dmu_k[c]; then q = v/|v|, v = (1, f)
            float gR[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < 3; ++k) gR[c][k] = k < K ? axis[k < K ? k : 0][c] : 0.0f;
            float gq[4];
            const float fq[4] = {p.cframe_q(0), p.cframe_q(1), p.cframe_q(2), p.cframe_q(3)};
            quat_to_matrix_vjp(fq, gR, gq);
            const float dot = gq[0] * fq[0] + gq[1] * fq[1] + gq[2] * fq[2] + gq[3] * fq[3];
            const float inv = 1.0f / p.cframe_norm();
#pragma unroll
            for (int j = 0; j < 3; ++j) out.sg_axis[j * S + i] = (gq[1 + j] - fq[1 + j] * dot) * inv;
        }
    }
};

}  // namespace sgs
