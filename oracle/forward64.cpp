// FP64 brute-force forward renderer -- test infrastructure (see oracle.h).
//
// Definition followed (no tiles, no blocking): for each pixel, take every Gaussian that
// survives the cull and whose 3-sigma support holds the pixel centre, order them by
// (FP32 view-depth bits, Gaussian index), and alpha-blend them front to back.
//
//   Eq. 2-3   G(x) = exp(-1/2 (x-X)^T Sigma^-1 (x-X)),  Sigma = R S S^T R^T.
//   EWA       Sigma2D = J W Sigma W^T J^T + 0.3 I (the projection the paper cites,
//             Zwicker et al. 2002, with the 3D-GS low-pass), conic = Sigma2D^-1.
//   Eq. 4     SH term  sum_{l<=L} sum_m c_lm Y_lm(d), real Y_lm with the Condon-Shortley
//             phase, evaluated from the associated-Legendre definition.
//   Eq. 5-9   SG lobes  sum_k a_k exp(lambda_k (mu_k . d - 1)), mu_k normalised (free
//             axes) or the world axes (1,0,0), (0,1,0), (0,0,1) (Sec. "Implementation").
//   colour    rgb = max(0, SH(d) + 1/2 + sum_k SG_k(d)),  d = (X - campos)/|X - campos|.
//   blend     alpha = min(0.99, o * exp(power)); skip alpha < 1/255; stop before a
//             Gaussian that would take T below 1e-4; C += rgb alpha T; T *= (1 - alpha);
//             pixel = C + T * bg.
// The cull, the depth order and support membership are the FP32 decisions of the mirror
// (mirror32.cpp); every value that enters the image is FP64.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>

#include "oracle_internal.h"

namespace orc64 {

Cam64 cam64(const float* c) {
    Cam64 k;
    for (int j = 0; j < 12; ++j) k.V[j] = c[j];
    for (int j = 0; j < 3; ++j) k.campos[j] = c[12 + j];
    k.fx = c[15];
    k.fy = c[16];
    k.cx = c[17];
    k.cy = c[18];
    k.W = (int)c[19];
    k.H = (int)c[20];
    return k;
}

static double factorial(int n) {
    double f = 1.0;
    for (int j = 2; j <= n; ++j) f *= j;
    return f;
}

static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

// Coefficients (ascending powers of z) of (-1)^m d^m/dz^m P_l(z), where
// P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) z^(l-2k)  (Legendre polynomial).
static std::vector<double> legendre_q(int l, int m) {
    std::vector<double> p(l + 1, 0.0);
    for (int k = 0; 2 * k <= l; ++k)
        p[l - 2 * k] = std::pow(-1.0, k) * binom(l, k) * binom(2 * l - 2 * k, l) / std::pow(2.0, l);
    for (int d = 0; d < m; ++d) {
        std::vector<double> q(p.size() > 1 ? p.size() - 1 : 1, 0.0);
        for (size_t j = 1; j < p.size(); ++j) q[j - 1] = p[j] * (double)j;
        p = q;
    }
    if (m % 2) for (double& c : p) c = -c;
    return p;
}

static double poly(const std::vector<double>& c, double z) {
    double r = 0.0;
    for (size_t j = c.size(); j-- > 0;) r = r * z + c[j];
    return r;
}

static double poly_deriv(const std::vector<double>& c, double z) {
    double r = 0.0;
    for (size_t j = c.size(); j-- > 1;) r = r * z + c[j] * (double)j;
    return r;
}

static double sh_norm(int l, int m) {
    const int am = std::abs(m);
    const double k = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    return m == 0 ? k : std::sqrt(2.0) * k;
}

// Y_lm(d) = N_lm Q_l|m|(z) P_m(x, y), with P_m = Re (x+iy)^m for m > 0, Im (x+iy)^|m| for
// m < 0 and 1 for m = 0.  On the unit sphere (x+iy)^m = sin^m(theta) e^{i m phi}, so this
// is sqrt(2) N P_l^m(cos theta) cos(m phi) (resp. sin) as in the textbook definition.
double lobe_frame(const double f[3], double q[4], double R[3][3]) {
    const double n = std::sqrt(1.0 + f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    q[0] = 1.0 / n;
    for (int j = 0; j < 3; ++j) q[1 + j] = f[j] / n;
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    return n;
}

void lobe_axis(const orc_scene* s, int64_t i, int lobe, double mu[3]) {
    const int64_t S = s->stride;
    if (s->axis_mode == 0) {  // free: mu_k / |mu_k|
        for (int j = 0; j < 3; ++j) mu[j] = s->sg_axis[(lobe * 3 + j) * S + i];
        const double n = std::sqrt(mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]);
        for (int j = 0; j < 3; ++j) mu[j] /= n;
    } else if (s->axis_mode == 1) {  // world axes
        for (int j = 0; j < 3; ++j) mu[j] = (j == lobe) ? 1.0 : 0.0;
    } else {  // column `lobe` of the Gaussian's frame
        const double f[3] = {s->sg_axis[i], s->sg_axis[S + i], s->sg_axis[2 * S + i]};
        double q[4], R[3][3];
        lobe_frame(f, q, R);
        for (int j = 0; j < 3; ++j) mu[j] = R[j][lobe];
    }
}

double sh_basis(int l, int m, const double d[3]) {
    const int am = std::abs(m);
    const std::complex<double> w(d[0], d[1]);
    const std::complex<double> wp = std::pow(w, am);
    const double P = m > 0 ? wp.real() : (m < 0 ? wp.imag() : 1.0);
    return sh_norm(l, m) * poly(legendre_q(l, am), d[2]) * P;
}

void sh_basis_grad(int l, int m, const double d[3], double g[3]) {
    const int am = std::abs(m);
    const std::complex<double> w(d[0], d[1]);
    const std::vector<double> q = legendre_q(l, am);
    const double N = sh_norm(l, m), Q = poly(q, d[2]), dQ = poly_deriv(q, d[2]);
    double P, Px, Py;
    if (m == 0) {
        P = 1.0;
        Px = Py = 0.0;
    } else {
        const std::complex<double> wp = std::pow(w, am);
        const std::complex<double> wm = am >= 1 ? std::pow(w, am - 1) : std::complex<double>(0, 0);
        if (m > 0) {
            P = wp.real();
            Px = am * wm.real();
            Py = -am * wm.imag();
        } else {
            P = wp.imag();
            Px = am * wm.imag();
            Py = am * wm.real();
        }
    }
    g[0] = N * Q * Px;
    g[1] = N * Q * Py;
    g[2] = N * dQ * P;
}

Pre64 preprocess(const orc_scene* s, int64_t i, const float* cam) {
    Pre64 p;
    std::memset(&p, 0, sizeof(p));
    p.sup = orc32::support_of(s, i, cam);
    p.visible = p.sup.visible;
    p.depth_bits = p.sup.depth_bits;
    const Cam64 k = cam64(cam);
    const int64_t S = s->stride;
    for (int j = 0; j < 3; ++j) p.X[j] = s->mean[j * S + i];
    for (int r = 0; r < 3; ++r)
        p.t[r] = k.V[4 * r] * p.X[0] + k.V[4 * r + 1] * p.X[1] + k.V[4 * r + 2] * p.X[2] + k.V[4 * r + 3];
    p.opacity = s->opacity[i];
    // Eq. 3
    for (int j = 0; j < 4; ++j) p.qraw[j] = s->rot[j * S + i];
    p.qnorm = std::sqrt(p.qraw[0] * p.qraw[0] + p.qraw[1] * p.qraw[1] + p.qraw[2] * p.qraw[2] +
                        p.qraw[3] * p.qraw[3]);
    for (int j = 0; j < 4; ++j) p.q[j] = p.qraw[j] / p.qnorm;
    const double w = p.q[0], x = p.q[1], y = p.q[2], z = p.q[3];
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    std::memcpy(p.R, R, sizeof(R));
    for (int j = 0; j < 3; ++j) p.s[j] = s->scale[j * S + i];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) p.M[r][c] = R[r][c] * p.s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += p.M[r][l] * p.M[c][l];
            p.Sig[r][c] = acc;
        }
    // EWA: Jacobian of (fx x/z + cx, fy y/z + cy) at t, with x/z and y/z clamped
    const double tz = p.t[2];
    p.limx = 1.3 * (0.5 * k.W / k.fx);
    p.limy = 1.3 * (0.5 * k.H / k.fy);
    const double u0 = p.t[0] / tz, v0 = p.t[1] / tz;
    p.u = std::min(p.limx, std::max(-p.limx, u0));
    p.v = std::min(p.limy, std::max(-p.limy, v0));
    p.clampx = p.u != u0;
    p.clampy = p.v != v0;
    const double tx = p.u * tz, ty = p.v * tz;
    p.J00 = k.fx / tz;
    p.J02 = -k.fx * tx / (tz * tz);
    p.J11 = k.fy / tz;
    p.J12 = -k.fy * ty / (tz * tz);
    // T = J W, Sigma2D = T Sigma T^T + 0.3 I
    const double J[2][3] = {{p.J00, 0.0, p.J02}, {0.0, p.J11, p.J12}};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += J[r][l] * k.V[4 * l + c];
            p.Tm[r][c] = acc;
        }
    double S2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) acc += p.Tm[r][j] * p.Sig[j][l] * p.Tm[c][l];
            S2[r][c] = acc;
        }
    p.a = S2[0][0] + 0.3;
    p.b = S2[0][1];
    p.c = S2[1][1] + 0.3;
    p.det = p.a * p.c - p.b * p.b;
    p.A = p.c / p.det;
    p.B = -p.b / p.det;
    p.C = p.a / p.det;
    p.px = k.fx * p.t[0] / tz + k.cx;
    p.py = k.fy * p.t[1] / tz + k.cy;
    // colour: Eq. 4 (SH) + Eq. 5/7/9 (SG lobes), direction from the camera centre
    for (int j = 0; j < 3; ++j) p.dvec[j] = p.X[j] - k.campos[j];
    p.dlen = std::sqrt(p.dvec[0] * p.dvec[0] + p.dvec[1] * p.dvec[1] + p.dvec[2] * p.dvec[2]);
    for (int j = 0; j < 3; ++j) p.dir[j] = p.dvec[j] / p.dlen;
    // SH bands summed: all stored ones, or with adaptive degrees the ones the record's
    // projected size calls for (its FP32 pixel radius against the two thresholds)
    p.sh_top = s->sh_degree;
    if (s->sh_adaptive) {
        const float r = p.sup.radius;
        const int D = r < s->sh_radius[0] ? 0 : (r < s->sh_radius[1] ? 1 : 2);
        p.sh_top = D < s->sh_degree ? D : s->sh_degree;
    }
    double col[3] = {0.5, 0.5, 0.5};
    for (int l = 0; l <= p.sh_top; ++l)
        for (int m = -l; m <= l; ++m) {
            const int kk = l * l + l + m;
            const double Y = sh_basis(l, m, p.dir);
            for (int ch = 0; ch < 3; ++ch) col[ch] += s->sh[(kk * 3 + ch) * S + i] * Y;
        }
    for (int lobe = 0; lobe < s->num_lobes; ++lobe) {
        double mu[3];
        lobe_axis(s, i, lobe, mu);
        const double lam = s->sg_sharp[lobe * S + i];
        const double e = std::exp(lam * (mu[0] * p.dir[0] + mu[1] * p.dir[1] + mu[2] * p.dir[2] - 1.0));
        for (int ch = 0; ch < 3; ++ch) col[ch] += s->sg_amp[(lobe * 3 + ch) * S + i] * e;
    }
    for (int ch = 0; ch < 3; ++ch) {
        p.pre[ch] = col[ch];
        p.rgb[ch] = col[ch] < 0.0 ? 0.0 : col[ch];
    }
    return p;
}

double power64(const Pre64& p, int x, int y) {
    const double dx = p.px - (x + 0.5), dy = p.py - (y + 0.5);
    return -0.5 * (p.A * dx * dx + p.C * dy * dy) - p.B * dx * dy;
}

std::vector<Hit> support_list(const std::vector<Pre64>& pre, int x, int y) {
    std::vector<Hit> hits;
    for (int64_t i = 0; i < (int64_t)pre.size(); ++i)
        if (pre[i].visible && orc32::in_support(pre[i].sup, x, y))
            hits.push_back({pre[i].depth_bits, i});
    std::sort(hits.begin(), hits.end(), [](const Hit& a, const Hit& b) {
        return a.depth_bits != b.depth_bits ? a.depth_bits < b.depth_bits : a.i < b.i;
    });
    return hits;
}

void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& fn) {
    if (threads <= 1 || n < 2) {
        for (int64_t j = 0; j < n; ++j) fn(j);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&]() {
            for (int64_t j; (j = next.fetch_add(1)) < n;) fn(j);
        });
    for (auto& th : pool) th.join();
}

}  // namespace orc64

using namespace orc64;

namespace {
std::vector<Pre64> preprocess_view(const orc_scene* s, const float* cam, int threads) {
    std::vector<Pre64> pre(s->n);
    parallel_for((s->n + 1023) / 1024, threads, [&](int64_t blk) {
        for (int64_t i = blk * 1024; i < std::min<int64_t>(s->n, (blk + 1) * 1024); ++i)
            pre[i] = preprocess(s, i, cam);
    });
    return pre;
}
}  // namespace

extern "C" {

double orc_sh_basis(int32_t l, int32_t m, const double* d) { return sh_basis(l, m, d); }

void orc_preprocess64(const orc_scene* s, const float* cams, int32_t B, uint8_t* visible,
                      double* mean2d, double* conic, double* rgb, double* depth) {
    for (int v = 0; v < B; ++v) {
        const std::vector<Pre64> pre = preprocess_view(s, cams + 22 * v, 8);
        for (int64_t i = 0; i < s->n; ++i) {
            const int64_t r = (int64_t)v * s->n + i;
            const Pre64& p = pre[i];
            visible[r] = p.visible;
            mean2d[2 * r] = p.px;
            mean2d[2 * r + 1] = p.py;
            conic[3 * r] = p.A;
            conic[3 * r + 1] = p.B;
            conic[3 * r + 2] = p.C;
            for (int ch = 0; ch < 3; ++ch) rgb[3 * r + ch] = p.rgb[ch];
            depth[r] = p.t[2];
        }
    }
}

void orc_render_pixels(const orc_scene* s, const float* cams, int32_t B, const double* bg,
                       const int32_t* pix, int64_t P, double* out_rgb, double* out_T,
                       double* out_margin, int32_t* out_ncontrib, uint64_t* out_sig,
                       int32_t threads) {
    for (int v = 0; v < B; ++v) {
        std::vector<int64_t> mine;
        for (int64_t p = 0; p < P; ++p)
            if (pix[3 * p] == v) mine.push_back(p);
        if (mine.empty()) continue;
        const std::vector<Pre64> pre = preprocess_view(s, cams + 22 * v, threads);
        parallel_for((int64_t)mine.size(), threads, [&](int64_t jj) {
            const int64_t p = mine[jj];
            const int x = pix[3 * p + 1], y = pix[3 * p + 2];
            const std::vector<Hit> hits = support_list(pre, x, y);
            double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
            double m_img = INFINITY, m_grad = INFINITY;
            uint64_t sig = 1469598103934665603ull;
            int n = 0;
            for (const Hit& h : hits) {
                const Pre64& g = pre[h.i];
                const double oG = g.opacity * std::exp(power64(g, x, y));
                m_grad = std::min(m_grad, std::fabs(oG - 0.99) / 0.99);
                const double alpha = std::min(0.99, oG);
                m_img = std::min(m_img, std::fabs(alpha - 1.0 / 255.0) * 255.0);
                if (alpha < 1.0 / 255.0) continue;
                const double Tn = T * (1.0 - alpha);
                m_img = std::min(m_img, std::fabs(Tn - 1e-4) / 1e-4);
                if (Tn < 1e-4) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += g.rgb[ch] * alpha * T;
                T = Tn;
                ++n;
                sig = (sig ^ (uint64_t)(h.i * 2 + (oG > 0.99))) * 1099511628211ull;
                for (int ch = 0; ch < 3; ++ch)
                    sig = (sig ^ (uint64_t)(g.pre[ch] < 0.0)) * 1099511628211ull;
                sig = (sig ^ (uint64_t)(g.clampx * 2 + g.clampy)) * 1099511628211ull;
                sig = (sig ^ (uint64_t)g.sh_top) * 1099511628211ull;  // adaptive SH degree
            }
            for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = C[ch] + T * bg[ch];
            out_T[p] = T;
            out_margin[2 * p] = m_img;
            out_margin[2 * p + 1] = std::min(m_img, m_grad);
            out_ncontrib[p] = n;
            out_sig[p] = sig;
        });
    }
}

}  // extern "C"
