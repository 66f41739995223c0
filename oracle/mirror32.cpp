// FP32 binning mirror -- test infrastructure (see oracle.h).
//
// The integer outcomes of the rasterizer (which Gaussians survive the cull, their depth
// bits, screen means, radii, tile rectangles, the tile|depth keys, the stable sort and
// the per-tile ranges, and whether a pixel centre lies in a Gaussian's support) are
// decided by floating point.  This file takes those decisions in IEEE single precision
// with every operation written out in a fixed order and rounded on its own (compiled
// with -ffp-contract=off), so that the result is a function of the inputs alone.
//
//   Eq. 3   Sigma = R S S^T R^T from the normalised quaternion q and scale s.
//   EWA     2D covariance J W Sigma W^T J^T [Zwicker 2002; paper Sec. "Preliminaries"],
//           with the 3D-GS low-pass +0.3 on the diagonal and the 1.3x frustum clamp.
//   cull    view depth > near, det(Sigma2D) > 0, the ellipse reaches a tile of the image.
//   radius  ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det)).
//   tiles   the tiles the 3-sigma ellipse reaches (row spans, row_span32).
//   key     (global tile id << 32) | float bits of the view depth.
#include "oracle_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct Cam32 {
    float V[12];
    float campos[3];
    float fx, fy, cx, cy;
    int W, H;
    float near_plane;
};

Cam32 cam32(const float* c) {
    Cam32 k;
    std::memcpy(k.V, c, 12 * sizeof(float));
    std::memcpy(k.campos, c + 12, 3 * sizeof(float));
    k.fx = c[15];
    k.fy = c[16];
    k.cx = c[17];
    k.cy = c[18];
    k.W = (int)c[19];
    k.H = (int)c[20];
    k.near_plane = c[21];
    return k;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

struct Rec32 {
    bool projected;  // passed the near-plane and determinant culls, finite mean and radius
    bool visible;    // projected and the tile rectangle is not empty
    uint32_t depth_bits;
    float px, py;
    float A, B, C;  // conic
    float r;
    int x0, y0, x1, y1;  // candidate rectangle (inclusive tile coordinates)
    int tiles;           // tiles the ellipse reaches (row spans)
};

// Tiles the Gaussian's 3-sigma ellipse reaches, row by row.  E = {d : Q(d) <= k} with
// Q(d) = A dx^2 + 2 B dx dy + C dy^2 (the conic), k = 9.01 (the support is Q <= 9; the
// 0.1 % slack and a 1/64-pixel pad cover rounding, so no tile holding a supported pixel
// centre is lost).  For a row of tiles, the band of pixel-centre rows [ly, hy] cuts E in a
// convex set whose x-extent is
//   max: the ellipse's rightmost point (dx = sqrt(kC/det), dy = -B sqrt(k/(det C))) if
//        its dy lies in the band, else the larger of dx_hi(dy) at the band ends, where
//        dx_hi/lo(dy) = (-B dy +/- sqrt(A k - det dy^2)) / A, det = AC - B^2;
//   min: symmetrically (leftmost point at -dy).
// The row keeps the tiles whose pixel-centre columns meet that x-extent.
struct RowSpans {
    int ty0, ty1;       // rows to visit (inclusive)
    float ex, ey, dyr, det, invA, Ak;
    bool ok;
};

const float kSpanQ = 9.01f;
const float kSpanPad = 0.015625f;

RowSpans row_setup32(float px, float py, float A, float B, float C, int th, int TH) {
    RowSpans r;
    r.ok = false;
    r.det = A * C - B * B;
    if (!(r.det > 0.0f)) return r;
    r.ex = std::sqrt((kSpanQ * C) / r.det);
    r.ey = std::sqrt((kSpanQ * A) / r.det);
    r.dyr = -(B * std::sqrt(kSpanQ / (r.det * C)));
    r.invA = 1.0f / A;
    r.Ak = A * kSpanQ;
    float t0 = py - r.ey;
    t0 = t0 - kSpanPad;
    t0 = t0 - 0.5f;
    float t1 = py + r.ey;
    t1 = t1 + kSpanPad;
    t1 = t1 - 0.5f;
    // first and last pixel rows whose centre y + 1/2 lies in [py - ey - pad, py + ey + pad]
    const float y0 = std::ceil(t0), y1 = std::floor(t1);
    if (!(y0 <= y1)) return r;
    const float f0 = std::fmax(std::floor(y0 / (float)th), 0.0f);
    const float f1 = std::fmin(std::floor(y1 / (float)th), (float)(TH - 1));
    if (!(f0 <= f1)) return r;
    r.ty0 = (int)f0;
    r.ty1 = (int)f1;
    r.ok = true;
    return r;
}

// Columns [tx0, tx1] of row ty; false if the row holds none.
bool row_span32(const RowSpans& r, float px, float py, float B, int ty, int tw, int th, int TW,
                int* tx0, int* tx1) {
    const float ly = (float)(ty * th) + 0.5f, hy = (float)(ty * th + th) - 0.5f;
    const float eyp = r.ey + kSpanPad;
    const float u0 = std::fmax(ly - py, -eyp);
    const float u1 = std::fmin(hy - py, eyp);
    if (!(u0 <= u1)) return false;
    const float s0 = std::sqrt(std::fmax(0.0f, r.Ak - (r.det * u0) * u0));
    const float s1 = std::sqrt(std::fmax(0.0f, r.Ak - (r.det * u1) * u1));
    const float b0 = B * u0, b1 = B * u1;
    const float hi0 = (s0 - b0) * r.invA, hi1 = (s1 - b1) * r.invA;
    const float lo0 = (-(b0 + s0)) * r.invA, lo1 = (-(b1 + s1)) * r.invA;
    const float xmax = (u0 <= r.dyr && r.dyr <= u1) ? r.ex : std::fmax(hi0, hi1);
    const float xmin = (u0 <= -r.dyr && -r.dyr <= u1) ? -r.ex : std::fmin(lo0, lo1);
    const float xs0 = (px + xmin) - kSpanPad;
    const float xs1 = (px + xmax) + kSpanPad;
    // first and last pixel columns whose centre x + 1/2 lies in [xs0, xs1]
    const float x0 = std::ceil(xs0 - 0.5f), x1 = std::floor(xs1 - 0.5f);
    if (!(x0 <= x1)) return false;
    const float f0 = std::fmax(std::floor(x0 / (float)tw), 0.0f);
    const float f1 = std::fmin(std::floor(x1 / (float)tw), (float)(TW - 1));
    if (!(f0 <= f1)) return false;
    *tx0 = (int)f0;
    *tx1 = (int)f1;
    return true;
}

// One Gaussian seen from one camera, every operation rounded to float on its own.
Rec32 project32(const orc_scene* s, int64_t i, const Cam32& k, int tile_w, int tile_h) {
    Rec32 o;
    std::memset(&o, 0, sizeof(o));
    const int64_t S = s->stride;
    const float X0 = s->mean[i], X1 = s->mean[S + i], X2 = s->mean[2 * S + i];
    const float* V = k.V;
    // camera-space position, left-to-right sums
    float t[3];
    for (int r = 0; r < 3; ++r) {
        float acc = V[4 * r + 0] * X0;
        acc = acc + V[4 * r + 1] * X1;
        acc = acc + V[4 * r + 2] * X2;
        t[r] = acc + V[4 * r + 3];
    }
    const float tz = t[2];
    uint32_t zb;
    std::memcpy(&zb, &tz, 4);
    o.depth_bits = zb;
    if (!(tz > k.near_plane)) return o;

    // Eq. 3: rotation from the normalised quaternion (w, x, y, z)
    const float qw0 = s->rot[i], qx0 = s->rot[S + i], qy0 = s->rot[2 * S + i],
                qz0 = s->rot[3 * S + i];
    float nq = qw0 * qw0;
    nq = nq + qx0 * qx0;
    nq = nq + qy0 * qy0;
    nq = nq + qz0 * qz0;
    const float rq = 1.0f / std::sqrt(nq);
    const float w = qw0 * rq, x = qx0 * rq, y = qy0 * rq, z = qz0 * rq;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    const float sc[3] = {s->scale[i], s->scale[S + i], s->scale[2 * S + i]};
    float M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * sc[c];
    float Sig[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
            float acc = M[r][0] * M[c][0];
            acc = acc + M[r][1] * M[c][1];
            acc = acc + M[r][2] * M[c][2];
            Sig[r][c] = acc;
            Sig[c][r] = acc;
        }

    // EWA Jacobian with the 1.3x frustum clamp of x/z and y/z
    const float limx = 1.3f * ((0.5f * (float)k.W) / k.fx);
    const float limy = 1.3f * ((0.5f * (float)k.H) / k.fy);
    float u = t[0] / tz;
    u = std::fmin(limx, std::fmax(-limx, u));
    float v = t[1] / tz;
    v = std::fmin(limy, std::fmax(-limy, v));
    const float tx = u * tz, ty = v * tz;
    const float z2 = tz * tz;
    const float J00 = k.fx / tz;
    const float J02 = -((k.fx * tx) / z2);
    const float J11 = k.fy / tz;
    const float J12 = -((k.fy * ty) / z2);
    // T = J W (2x3); J has zeros at (0,1) and (1,0)
    float T[2][3];
    for (int c = 0; c < 3; ++c) {
        T[0][c] = J00 * V[c] + J02 * V[8 + c];
        T[1][c] = J11 * V[4 + c] + J12 * V[8 + c];
    }
    // U = T Sigma, Sigma2D = U T^T
    float U[2][3];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            float acc = T[r][0] * Sig[0][c];
            acc = acc + T[r][1] * Sig[1][c];
            acc = acc + T[r][2] * Sig[2][c];
            U[r][c] = acc;
        }
    float s00 = U[0][0] * T[0][0];
    s00 = s00 + U[0][1] * T[0][1];
    s00 = s00 + U[0][2] * T[0][2];
    float s01 = U[0][0] * T[1][0];
    s01 = s01 + U[0][1] * T[1][1];
    s01 = s01 + U[0][2] * T[1][2];
    float s11 = U[1][0] * T[1][0];
    s11 = s11 + U[1][1] * T[1][1];
    s11 = s11 + U[1][2] * T[1][2];
    const float a = s00 + 0.3f, b = s01, c = s11 + 0.3f;
    const float det = a * c - b * b;
    if (!(det > 0.0f)) return o;
    o.A = c / det;
    o.B = -(b / det);
    o.C = a / det;
    const float mid = 0.5f * (a + c);
    const float disc = mid * mid - det;
    const float l1 = mid + std::sqrt(std::fmax(0.1f, disc));
    const float rad = std::ceil(3.0f * std::sqrt(l1));
    const float px = k.fx * (t[0] / tz) + k.cx;
    const float py = k.fy * (t[1] / tz) + k.cy;
    if (rad != rad || px != px || py != py) return o;
    const int TW = ceil_div(k.W, tile_w), TH = ceil_div(k.H, tile_h);
    const float fx0 = std::floor((px - rad) / (float)tile_w);
    const float fx1 = std::floor((px + rad) / (float)tile_w);
    const float fy0 = std::floor((py - rad) / (float)tile_h);
    const float fy1 = std::floor((py + rad) / (float)tile_h);
    const float x0 = std::fmax(fx0, 0.0f), x1 = std::fmin(fx1, (float)(TW - 1));
    const float y0 = std::fmax(fy0, 0.0f), y1 = std::fmin(fy1, (float)(TH - 1));
    o.px = px;
    o.py = py;
    o.r = rad;
    o.projected = true;
    if (!(x0 <= x1 && y0 <= y1)) return o;
    o.x0 = (int)x0;
    o.x1 = (int)x1;
    o.y0 = (int)y0;
    o.y1 = (int)y1;
    const RowSpans rs = row_setup32(px, py, o.A, o.B, o.C, tile_h, TH);
    int hits = 0;
    if (rs.ok)
        for (int ty = rs.ty0; ty <= rs.ty1; ++ty) {
            int a0, a1;
            if (row_span32(rs, px, py, o.B, ty, tile_w, tile_h, TW, &a0, &a1)) hits += a1 - a0 + 1;
        }
    o.tiles = hits;
    o.visible = hits > 0;
    return o;
}

}  // namespace

// Used by forward64.cpp / adjoint64.cpp inside the oracle.
namespace orc32 {

Support support_of(const orc_scene* s, int64_t i, const float* cam) {
    const Cam32 k = cam32(cam);
    // the tile size only matters for the rectangle, which the support test does not use
    const Rec32 r = project32(s, i, k, 16, 16);
    Support o;
    o.visible = r.projected;
    o.depth_bits = r.depth_bits;
    o.px = r.px;
    o.py = r.py;
    o.qa = -0.5f * r.A;
    o.qb = -r.B;
    o.qc = -0.5f * r.C;
    o.radius = r.r;
    return o;
}

// Support membership of pixel (x, y): the Gaussian's exponent
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy,  dx = px - (x + 1/2), dy = py - (y + 1/2),
// evaluated as fma(dx, fma(qa, dx, qb*dy), (qc*dy)*dy) with qa=-A/2, qb=-B, qc=-C/2,
// and the pixel is in the support iff power >= -4.5 (Mahalanobis distance <= 3).
bool in_support(const Support& g, int x, int y) {
    const float dx = g.px - ((float)x + 0.5f);
    const float dy = g.py - ((float)y + 0.5f);
    const float u = std::fma(g.qa, dx, g.qb * dy);
    const float w = (g.qc * dy) * dy;
    const float power = std::fma(dx, u, w);
    return power >= -4.5f;
}

}  // namespace orc32

extern "C" {

void orc_mirror_preprocess(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                           int32_t tile_h, uint8_t* visible, uint32_t* depth_bits,
                           float* mean2d, float* conic, float* radius, int32_t* rect,
                           uint32_t* tiles_touched) {
    for (int v = 0; v < B; ++v) {
        const Cam32 k = cam32(cams + 22 * v);
        for (int64_t i = 0; i < s->n; ++i) {
            const int64_t r = (int64_t)v * s->n + i;
            const Rec32 o = project32(s, i, k, tile_w, tile_h);
            visible[r] = o.visible;
            depth_bits[r] = o.depth_bits;
            mean2d[2 * r] = o.px;
            mean2d[2 * r + 1] = o.py;
            conic[3 * r] = o.A;
            conic[3 * r + 1] = o.B;
            conic[3 * r + 2] = o.C;
            radius[r] = o.r;
            rect[4 * r] = o.x0;
            rect[4 * r + 1] = o.y0;
            rect[4 * r + 2] = o.x1;
            rect[4 * r + 3] = o.y1;
            tiles_touched[r] = o.visible ? (uint32_t)o.tiles : 0u;
        }
    }
}

int64_t orc_num_tiles(const float* cams, int32_t B, int32_t tile_w, int32_t tile_h) {
    int64_t total = 0;
    for (int v = 0; v < B; ++v) {
        const Cam32 k = cam32(cams + 22 * v);
        total += (int64_t)ceil_div(k.W, tile_w) * ceil_div(k.H, tile_h);
    }
    return total;
}

int64_t orc_mirror_count(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                         int32_t tile_h) {
    int64_t m = 0;
    for (int v = 0; v < B; ++v) {
        const Cam32 k = cam32(cams + 22 * v);
        for (int64_t i = 0; i < s->n; ++i) {
            const Rec32 o = project32(s, i, k, tile_w, tile_h);
            if (o.visible) m += o.tiles;
        }
    }
    return m;
}

void orc_stable_sort_pairs(int64_t m, uint64_t* keys, uint32_t* vals) {
    std::vector<int64_t> idx(m);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int64_t a, int64_t b) { return keys[a] < keys[b]; });
    std::vector<uint64_t> k2(m);
    std::vector<uint32_t> v2(m);
    for (int64_t j = 0; j < m; ++j) {
        k2[j] = keys[idx[j]];
        v2[j] = vals[idx[j]];
    }
    std::copy(k2.begin(), k2.end(), keys);
    std::copy(v2.begin(), v2.end(), vals);
}

void orc_mirror_bin(const orc_scene* s, const float* cams, int32_t B, int32_t tile_w,
                    int32_t tile_h, uint64_t* keys_in, uint32_t* vals_in, uint64_t* keys_out,
                    uint32_t* vals_out, uint32_t* ranges) {
    // Instances in record order (record r = v*n + i), the tiles the ellipse reaches in
// row-major order.
    int64_t m = 0;
    uint64_t tile_base = 0;
    for (int v = 0; v < B; ++v) {
        const Cam32 k = cam32(cams + 22 * v);
        const int TW = ceil_div(k.W, tile_w);
        for (int64_t i = 0; i < s->n; ++i) {
            const Rec32 o = project32(s, i, k, tile_w, tile_h);
            if (!o.visible) continue;
            const RowSpans rs = row_setup32(o.px, o.py, o.A, o.B, o.C, tile_h, ceil_div(k.H, tile_h));
            for (int ty = rs.ty0; ty <= rs.ty1; ++ty) {
                int a0, a1;
                if (!row_span32(rs, o.px, o.py, o.B, ty, tile_w, tile_h, TW, &a0, &a1)) continue;
                for (int tx = a0; tx <= a1; ++tx) {
                    const uint64_t tile = tile_base + (uint64_t)ty * TW + tx;
                    keys_in[m] = (tile << 32) | o.depth_bits;
                    vals_in[m] = (uint32_t)((int64_t)v * s->n + i);
                    ++m;
                }
            }
        }
        tile_base += (uint64_t)TW * ceil_div(k.H, tile_h);
    }
    std::copy(keys_in, keys_in + m, keys_out);
    std::copy(vals_in, vals_in + m, vals_out);
    orc_stable_sort_pairs(m, keys_out, vals_out);
    // per-tile [start, end); tiles without instances keep (0, 0)
    std::fill(ranges, ranges + 2 * tile_base, 0u);
    for (int64_t j = 0; j < m; ++j) {
        const uint64_t t = keys_out[j] >> 32;
        if (j == 0 || (keys_out[j - 1] >> 32) != t) ranges[2 * t] = (uint32_t)j;
        if (j == m - 1 || (keys_out[j + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
}

}  // extern "C"
