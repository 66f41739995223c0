// FP64 adjoint of forward64.cpp -- test infrastructure (see oracle.h).
//
// L = sum over the listed pixels of dL_drgb[p] . pixel[p].  The reverse mode is written
// by hand, step by step against the forward definition:
//   pixel = sum_k c_k a_k T_k + T_{n+1} bg,   T_k = prod_{j<k} (1 - a_j)
//   dL/dc_k = a_k T_k g
//   dL/da_k = g . (c_k T_k - (sum_{j>k} c_j a_j T_j + T_{n+1} bg) / (1 - a_k))
//   a_k = min(0.99, o G),  G = exp(power)   (the clamped branch passes no gradient)
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy,  dx = px - (x + 1/2),  dy = py - (y + 1/2)
// then per Gaussian: conic = inverse(Sigma2D) -> Sigma2D = T Sigma T^T + 0.3 I ->
// T = J W and J(t) (with the frustum clamp) -> t = W X + t_v; Sigma = M M^T, M = R S ->
// R(q/|q|) (Eq. 3); colour rgb = max(0, SH + 1/2 + sum SG) (Eq. 4, 5, 7, 9) -> SH
// coefficients, lobe amplitudes, sharpness and axes, and the direction d -> X.
// Where a clamp is active the derivative of the taken branch is used.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "oracle_internal.h"

using namespace orc64;

namespace {

struct Contrib {
    int64_t i;
    double g[9];  // d/d(px, py, A, B, C, opacity, r, g, b)
};

// Per-Gaussian chain from the 2D quantities to the scene parameters.
void chain_to_params(const orc_scene* s, const Cam64& k, const Pre64& p, const double* g2,
                     int64_t i, orc_grads* out) {
    const int64_t S = s->stride;
    const double gpx = g2[0], gpy = g2[1], gA = g2[2], gB = g2[3], gC = g2[4];
    double gX[3] = {0.0, 0.0, 0.0};
    double gt[3] = {0.0, 0.0, 0.0};

    // colour -> SH, SG and the direction
    double gpre[3];
    for (int ch = 0; ch < 3; ++ch) gpre[ch] = p.pre[ch] < 0.0 ? 0.0 : g2[6 + ch];
    double gdir[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l <= p.sh_top; ++l)  // bands above the record's degree get nothing
        for (int m = -l; m <= l; ++m) {
            const int kk = l * l + l + m;
            const double Y = sh_basis(l, m, p.dir);
            double gY[3];
            sh_basis_grad(l, m, p.dir, gY);
            double wsum = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                out->sh[(kk * 3 + ch) * S + i] += gpre[ch] * Y;
                wsum += gpre[ch] * s->sh[(kk * 3 + ch) * S + i];
            }
            for (int j = 0; j < 3; ++j) gdir[j] += wsum * gY[j];
        }
    double gF[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};  // frame mode: dL/dR
    for (int lobe = 0; lobe < s->num_lobes; ++lobe) {
        double mu[3], mun = 1.0;
        lobe_axis(s, i, lobe, mu);
        if (s->axis_mode == 0) {
            double muraw[3];
            for (int j = 0; j < 3; ++j) muraw[j] = s->sg_axis[(lobe * 3 + j) * S + i];
            mun = std::sqrt(muraw[0] * muraw[0] + muraw[1] * muraw[1] + muraw[2] * muraw[2]);
        }
        const double lam = s->sg_sharp[lobe * S + i];
        const double cosang = mu[0] * p.dir[0] + mu[1] * p.dir[1] + mu[2] * p.dir[2];
        const double e = std::exp(lam * (cosang - 1.0));
        double sacc = 0.0;  // sum_ch g_ch a_ch e
        for (int ch = 0; ch < 3; ++ch) {
            out->sg_amp[(lobe * 3 + ch) * S + i] += gpre[ch] * e;
            sacc += gpre[ch] * s->sg_amp[(lobe * 3 + ch) * S + i] * e;
        }
        out->sg_sharp[lobe * S + i] += sacc * (cosang - 1.0);
        const double gcos = sacc * lam;
        for (int j = 0; j < 3; ++j) gdir[j] += gcos * mu[j];
        if (s->axis_mode == 0) {
            // mu = muraw / |muraw|:  d mu/d muraw = (I - mu mu^T) / |muraw|
            double gmu[3], dotp = 0.0;
            for (int j = 0; j < 3; ++j) {
                gmu[j] = gcos * p.dir[j];
                dotp += gmu[j] * mu[j];
            }
            for (int j = 0; j < 3; ++j)
                out->sg_axis[(lobe * 3 + j) * S + i] += (gmu[j] - mu[j] * dotp) / mun;
        } else if (s->axis_mode == 2) {
            for (int j = 0; j < 3; ++j) gF[j][lobe] += gcos * p.dir[j];  // mu = column `lobe` of R
        }
    }
    if (s->axis_mode == 2 && s->num_lobes > 0) {
        // R(q) entry by entry, differentiated w.r.t. (w, x, y, z); then q = v / |v|, v = (1, f)
        const double f[3] = {s->sg_axis[i], s->sg_axis[S + i], s->sg_axis[2 * S + i]};
        double q[4], R[3][3];
        const double n = lobe_frame(f, q, R);
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        const double dR[3][3][4] = {
            {{0, 0, -4 * y, -4 * z}, {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x}},
            {{2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z}, {-2 * x, -2 * w, 2 * z, 2 * y}},
            {{-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}}};
        double gq[4] = {0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 4; ++k) gq[k] += gF[r][c] * dR[r][c][k];
        const double dotq = gq[0] * q[0] + gq[1] * q[1] + gq[2] * q[2] + gq[3] * q[3];
        for (int j = 0; j < 3; ++j) out->sg_axis[j * S + i] += (gq[1 + j] - q[1 + j] * dotq) / n;
    }
    {  // d = dvec / |dvec|, dvec = X - campos
        double dotp = 0.0;
        for (int j = 0; j < 3; ++j) dotp += gdir[j] * p.dir[j];
        for (int j = 0; j < 3; ++j) gX[j] += (gdir[j] - p.dir[j] * dotp) / p.dlen;
    }

    // conic (A, B, C) = (c, -b, a) / det, det = a c - b^2
    const double a = p.a, b = p.b, c = p.c, d2 = p.det * p.det;
    const double ga = gA * (-c * c / d2) + gB * (b * c / d2) + gC * (-b * b / d2);
    const double gb = gA * (2 * b * c / d2) + gB * (-(a * c + b * b) / d2) + gC * (2 * a * b / d2);
    const double gc = gA * (-b * b / d2) + gB * (a * b / d2) + gC * (-a * a / d2);
    // Sigma2D entries s00 = a - 0.3, s01 = b, s11 = c - 0.3; Sigma2D = T Sigma T^T
    double gSig[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l)
            gSig[j][l] = ga * p.Tm[0][j] * p.Tm[0][l] + gb * p.Tm[0][j] * p.Tm[1][l] +
                         gc * p.Tm[1][j] * p.Tm[1][l];
    double ST0[3], ST1[3];  // Sigma T0^T, Sigma T1^T
    for (int j = 0; j < 3; ++j) {
        ST0[j] = ST1[j] = 0.0;
        for (int l = 0; l < 3; ++l) {
            ST0[j] += p.Sig[j][l] * p.Tm[0][l];
            ST1[j] += p.Sig[j][l] * p.Tm[1][l];
        }
    }
    double gT[2][3];
    for (int j = 0; j < 3; ++j) {
        gT[0][j] = 2.0 * ga * ST0[j] + gb * ST1[j];
        gT[1][j] = gb * ST0[j] + 2.0 * gc * ST1[j];
    }
    // T = J W:  T0c = J00 W0c + J02 W2c,  T1c = J11 W1c + J12 W2c
    double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
    for (int cc = 0; cc < 3; ++cc) {
        gJ00 += gT[0][cc] * k.V[cc];
        gJ02 += gT[0][cc] * k.V[8 + cc];
        gJ11 += gT[1][cc] * k.V[4 + cc];
        gJ12 += gT[1][cc] * k.V[8 + cc];
    }
    // J00 = fx/tz, J02 = -fx tx/tz^2, J11 = fy/tz, J12 = -fy ty/tz^2,
    // tx = t.x (unclamped) or u tz with u = +-limx (clamped); same for y.
    const double tz = p.t[2];
    const double tx = p.u * tz, ty = p.v * tz;
    gt[2] += -k.fx / (tz * tz) * gJ00 - k.fy / (tz * tz) * gJ11 +
             2.0 * k.fx * tx / (tz * tz * tz) * gJ02 + 2.0 * k.fy * ty / (tz * tz * tz) * gJ12;
    const double gtx = -k.fx / (tz * tz) * gJ02, gty = -k.fy / (tz * tz) * gJ12;
    if (p.clampx) gt[2] += gtx * p.u; else gt[0] += gtx;
    if (p.clampy) gt[2] += gty * p.v; else gt[1] += gty;
    // screen mean px = fx t.x/t.z + cx, py = fy t.y/t.z + cy
    gt[0] += k.fx / tz * gpx;
    gt[2] += -k.fx * p.t[0] / (tz * tz) * gpx;
    gt[1] += k.fy / tz * gpy;
    gt[2] += -k.fy * p.t[1] / (tz * tz) * gpy;
    // t = W X + t_v
    for (int j = 0; j < 3; ++j)
        for (int r = 0; r < 3; ++r) gX[j] += k.V[4 * r + j] * gt[r];
    for (int j = 0; j < 3; ++j) out->mean[j * S + i] += gX[j];

    // Sigma = M M^T:  dL/dM = (G + G^T) M;  M = R diag(s)
    double gM[3][3];
    for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += (gSig[r][l] + gSig[l][r]) * p.M[l][cc];
            gM[r][cc] = acc;
        }
    double gR[3][3];
    for (int cc = 0; cc < 3; ++cc) {
        double gs = 0.0;
        for (int r = 0; r < 3; ++r) {
            gR[r][cc] = gM[r][cc] * p.s[cc];
            gs += gM[r][cc] * p.R[r][cc];
        }
        out->scale[cc * S + i] += gs;
    }
    // R(w, x, y, z) for the unit quaternion (Eq. 3)
    const double w = p.q[0], x = p.q[1], y = p.q[2], z = p.q[3];
    double gq[4];
    gq[0] = -2 * z * gR[0][1] + 2 * y * gR[0][2] + 2 * z * gR[1][0] - 2 * x * gR[1][2] -
            2 * y * gR[2][0] + 2 * x * gR[2][1];
    gq[1] = 2 * y * gR[0][1] + 2 * z * gR[0][2] + 2 * y * gR[1][0] - 4 * x * gR[1][1] -
            2 * w * gR[1][2] + 2 * z * gR[2][0] + 2 * w * gR[2][1] - 4 * x * gR[2][2];
    gq[2] = -4 * y * gR[0][0] + 2 * x * gR[0][1] + 2 * w * gR[0][2] + 2 * x * gR[1][0] +
            2 * z * gR[1][2] - 2 * w * gR[2][0] + 2 * z * gR[2][1] - 4 * y * gR[2][2];
    gq[3] = -4 * z * gR[0][0] - 2 * w * gR[0][1] + 2 * x * gR[0][2] + 2 * w * gR[1][0] -
            4 * z * gR[1][1] + 2 * y * gR[1][2] + 2 * x * gR[2][0] + 2 * y * gR[2][1];
    // q = qraw / |qraw|
    double dotp = 0.0;
    for (int j = 0; j < 4; ++j) dotp += gq[j] * p.q[j];
    for (int j = 0; j < 4; ++j) out->rot[j * S + i] += (gq[j] - p.q[j] * dotp) / p.qnorm;

    out->opacity[i] += g2[5];
}

}  // namespace

extern "C" {

void orc_adjoint_pixels(const orc_scene* s, const float* cams, int32_t B, const double* bg,
                        const int32_t* pix, int64_t P, const double* dL_drgb, orc_grads* out,
                        int32_t threads) {
    const int64_t S = s->stride;
    const int nsh = (s->sh_degree + 1) * (s->sh_degree + 1);
    std::fill(out->mean, out->mean + 3 * S, 0.0);
    std::fill(out->scale, out->scale + 3 * S, 0.0);
    std::fill(out->rot, out->rot + 4 * S, 0.0);
    std::fill(out->opacity, out->opacity + S, 0.0);
    std::fill(out->sh, out->sh + nsh * 3 * S, 0.0);
    if (s->num_lobes) {
        std::fill(out->sg_amp, out->sg_amp + s->num_lobes * 3 * S, 0.0);
        std::fill(out->sg_sharp, out->sg_sharp + s->num_lobes * S, 0.0);
        if (s->axis_mode == 0) std::fill(out->sg_axis, out->sg_axis + s->num_lobes * 3 * S, 0.0);
        if (s->axis_mode == 2) std::fill(out->sg_axis, out->sg_axis + 3 * S, 0.0);
    }
    for (int v = 0; v < B; ++v) {
        std::vector<int64_t> mine;
        for (int64_t p = 0; p < P; ++p)
            if (pix[3 * p] == v) mine.push_back(p);
        if (mine.empty()) continue;
        const float* cam = cams + 22 * v;
        const Cam64 k = cam64(cam);
        std::vector<Pre64> pre(s->n);
        parallel_for(s->n, threads, [&](int64_t i) { pre[i] = preprocess(s, i, cam); });
        std::vector<std::vector<Contrib>> per_pixel(mine.size());
        parallel_for((int64_t)mine.size(), threads, [&](int64_t jj) {
            const int64_t p = mine[jj];
            const int x = pix[3 * p + 1], y = pix[3 * p + 2];
            const double* gout = dL_drgb + 3 * p;
            const std::vector<Hit> hits = support_list(pre, x, y);
            struct Step { int64_t i; double alpha, T, G, oG; };
            std::vector<Step> steps;
            double T = 1.0;
            for (const Hit& h : hits) {
                const Pre64& g = pre[h.i];
                const double G = std::exp(power64(g, x, y));
                const double oG = g.opacity * G;
                const double alpha = std::min(0.99, oG);
                if (alpha < 1.0 / 255.0) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < 1e-4) break;
                steps.push_back({h.i, alpha, T, G, oG});
                T = Tn;
            }
            const double Tfinal = T;
            // behind[k] = sum_{j>k} c_j a_j T_j + T_{n+1} bg, built from the back
            double behind[3];
            for (int ch = 0; ch < 3; ++ch) behind[ch] = Tfinal * bg[ch];
            std::vector<Contrib>& outc = per_pixel[jj];
            for (int64_t kk = (int64_t)steps.size() - 1; kk >= 0; --kk) {
                const Step& st = steps[kk];
                const Pre64& g = pre[st.i];
                Contrib cb;
                cb.i = st.i;
                double galpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    cb.g[6 + ch] = st.alpha * st.T * gout[ch];
                    galpha += gout[ch] * (g.rgb[ch] * st.T - behind[ch] / (1.0 - st.alpha));
                }
                for (int ch = 0; ch < 3; ++ch) behind[ch] += g.rgb[ch] * st.alpha * st.T;
                const bool clamped = st.oG > 0.99;
                const double go = clamped ? 0.0 : galpha * st.G;
                const double gG = clamped ? 0.0 : galpha * g.opacity;
                const double gpow = gG * st.G;
                const double dx = g.px - (x + 0.5), dy = g.py - (y + 0.5);
                cb.g[0] = gpow * (-(g.A * dx + g.B * dy));
                cb.g[1] = gpow * (-(g.C * dy + g.B * dx));
                cb.g[2] = gpow * (-0.5 * dx * dx);
                cb.g[3] = gpow * (-dx * dy);
                cb.g[4] = gpow * (-0.5 * dy * dy);
                cb.g[5] = go;
                outc.push_back(cb);
            }
        });
        // serial, deterministic accumulation of the 2D gradients per Gaussian
        std::vector<std::array<double, 9>> g2(s->n);
        std::vector<uint8_t> touched(s->n, 0);
        for (auto& a : g2) a.fill(0.0);
        for (const auto& list : per_pixel)
            for (const Contrib& cb : list) {
                touched[cb.i] = 1;
                for (int j = 0; j < 9; ++j) g2[cb.i][j] += cb.g[j];
            }
        for (int64_t i = 0; i < s->n; ++i)
            if (touched[i]) chain_to_params(s, k, pre[i], g2[i].data(), i, out);
    }
}

}  // extern "C"
