// Stage (a) of the rasterizer and its backward: per (view, Gaussian) projection and colour.
//
// Forward, per Gaussian i (one thread), parameters read once, then for every view v:
//   t = W X + t_v; cull if t.z <= near
//   Sigma = R S S^T R^T from q/|q| and s (Eq. 3)
//   Sigma2D = J W Sigma W^T J^T + 0.3 I, J the EWA Jacobian at t with x/z, y/z clamped
//             to 1.3x the half field of view (the projection of Sec. "Preliminaries")
//   conic = Sigma2D^-1, radius = ceil(3 sqrt(lambda_max)), screen mean, tile rectangle,
//   and how many tiles the 3-sigma ellipse reaches (row spans)
//   colour = max(0, SH(d) + 0.5 + sum_k SG_k(d)), d = (X - campos)/|X - campos| (Eq. 4-9)
//   and the record depth sort's pair (depth bits, or all ones for a culled record; the
//   record id with its tile count)
// Everything up to the tile rectangle and the conic uses correctly rounded operations in
// one fixed order (mul_rn/add_rn/...), so the cull, depth bits, radius and rectangle are
// a function of the inputs alone and identical on every run and launch shape.
#include <cuda_runtime.h>

#include "colour.cuh"
#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

struct Geometry {
    float Sig[3][3];  // 3D covariance (exactly rounded, fixed order)
    float R[3][3];
    float q[4];       // normalised quaternion
    float qnorm;
    float s[3];
};

__device__ __forceinline__ void geometry_exact(const sgs_gaussians& g, int64_t i, Geometry& G) {
    const int64_t S = g.stride;
    const float qw0 = __ldg(g.rot + i), qx0 = __ldg(g.rot + S + i), qy0 = __ldg(g.rot + 2 * S + i),
                qz0 = __ldg(g.rot + 3 * S + i);
    float nq = mul_rn(qw0, qw0);
    nq = add_rn(nq, mul_rn(qx0, qx0));
    nq = add_rn(nq, mul_rn(qy0, qy0));
    nq = add_rn(nq, mul_rn(qz0, qz0));
    const float sq = sqrt_rn(nq);
    const float rq = div_rn(1.0f, sq);
    const float w = mul_rn(qw0, rq), x = mul_rn(qx0, rq), y = mul_rn(qy0, rq), z = mul_rn(qz0, rq);
    G.q[0] = w; G.q[1] = x; G.q[2] = y; G.q[3] = z;
    G.qnorm = sq;
    const float xx = mul_rn(x, x), yy = mul_rn(y, y), zz = mul_rn(z, z);
    const float xy = mul_rn(x, y), xz = mul_rn(x, z), yz = mul_rn(y, z);
    const float wx = mul_rn(w, x), wy = mul_rn(w, y), wz = mul_rn(w, z);
    G.R[0][0] = sub_rn(1.0f, mul_rn(2.0f, add_rn(yy, zz)));
    G.R[0][1] = mul_rn(2.0f, sub_rn(xy, wz));
    G.R[0][2] = mul_rn(2.0f, add_rn(xz, wy));
    G.R[1][0] = mul_rn(2.0f, add_rn(xy, wz));
    G.R[1][1] = sub_rn(1.0f, mul_rn(2.0f, add_rn(xx, zz)));
    G.R[1][2] = mul_rn(2.0f, sub_rn(yz, wx));
    G.R[2][0] = mul_rn(2.0f, sub_rn(xz, wy));
    G.R[2][1] = mul_rn(2.0f, add_rn(yz, wx));
    G.R[2][2] = sub_rn(1.0f, mul_rn(2.0f, add_rn(xx, yy)));
    G.s[0] = __ldg(g.scale + i);
    G.s[1] = __ldg(g.scale + S + i);
    G.s[2] = __ldg(g.scale + 2 * S + i);
    float M[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = mul_rn(G.R[r][c], G.s[c]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            float acc = mul_rn(M[r][0], M[c][0]);
            acc = add_rn(acc, mul_rn(M[r][1], M[c][1]));
            acc = add_rn(acc, mul_rn(M[r][2], M[c][2]));
            G.Sig[r][c] = acc;
            G.Sig[c][r] = acc;
        }
}

struct Projected {
    bool visible;
    float t[3];
    float px, py;
    float A, B, C;
    float radius;
    int x0, y0, x1, y1;
    // EWA intermediates for the backward pass
    float u, v;  // clamped x/z, y/z
    bool clampx, clampy;
    float J00, J02, J11, J12;
    float T[2][3];
    float TS[2][3];  // T Sigma (project_fast only)
    float a, b, c;
};

// Exact-order projection of one Gaussian into one view.
__device__ __forceinline__ void project_exact(const View& cam, const float X[3], const Geometry& G,
                                              float inv_tw, float inv_th, Projected& P) {
    P.visible = false;
    const float* V = cam.V;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float acc = mul_rn(V[4 * r + 0], X[0]);
        acc = add_rn(acc, mul_rn(V[4 * r + 1], X[1]));
        acc = add_rn(acc, mul_rn(V[4 * r + 2], X[2]));
        P.t[r] = add_rn(acc, V[4 * r + 3]);
    }
    const float tz = P.t[2];
    if (!(tz > cam.near_plane)) return;
    const float limx = cam.limx, limy = cam.limy;
    const float u0 = div_rn(P.t[0], tz), v0 = div_rn(P.t[1], tz);
    P.u = fminf(limx, fmaxf(-limx, u0));
    P.v = fminf(limy, fmaxf(-limy, v0));
    P.clampx = P.u != u0;
    P.clampy = P.v != v0;
    const float tx = mul_rn(P.u, tz), ty = mul_rn(P.v, tz);
    const float z2 = mul_rn(tz, tz);
    P.J00 = div_rn(cam.fx, tz);
    P.J02 = -div_rn(mul_rn(cam.fx, tx), z2);
    P.J11 = div_rn(cam.fy, tz);
    P.J12 = -div_rn(mul_rn(cam.fy, ty), z2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        P.T[0][c] = add_rn(mul_rn(P.J00, V[c]), mul_rn(P.J02, V[8 + c]));
        P.T[1][c] = add_rn(mul_rn(P.J11, V[4 + c]), mul_rn(P.J12, V[8 + c]));
    }
    float U[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = mul_rn(P.T[r][0], G.Sig[0][c]);
            acc = add_rn(acc, mul_rn(P.T[r][1], G.Sig[1][c]));
            acc = add_rn(acc, mul_rn(P.T[r][2], G.Sig[2][c]));
            U[r][c] = acc;
        }
    float s00 = mul_rn(U[0][0], P.T[0][0]);
    s00 = add_rn(s00, mul_rn(U[0][1], P.T[0][1]));
    s00 = add_rn(s00, mul_rn(U[0][2], P.T[0][2]));
    float s01 = mul_rn(U[0][0], P.T[1][0]);
    s01 = add_rn(s01, mul_rn(U[0][1], P.T[1][1]));
    s01 = add_rn(s01, mul_rn(U[0][2], P.T[1][2]));
    float s11 = mul_rn(U[1][0], P.T[1][0]);
    s11 = add_rn(s11, mul_rn(U[1][1], P.T[1][1]));
    s11 = add_rn(s11, mul_rn(U[1][2], P.T[1][2]));
    P.a = add_rn(s00, 0.3f);
    P.b = s01;
    P.c = add_rn(s11, 0.3f);
    const float det = sub_rn(mul_rn(P.a, P.c), mul_rn(P.b, P.b));
    if (!(det > 0.0f)) return;
    P.A = div_rn(P.c, det);
    P.B = -div_rn(P.b, det);
    P.C = div_rn(P.a, det);
    const float mid = mul_rn(0.5f, add_rn(P.a, P.c));
    const float disc = sub_rn(mul_rn(mid, mid), det);
    const float l1 = add_rn(mid, sqrt_rn(fmaxf(0.1f, disc)));
    const float rad = ceilf(mul_rn(3.0f, sqrt_rn(l1)));
    const float px = add_rn(mul_rn(cam.fx, u0), cam.cx);  // u0, v0: the unclamped x/z, y/z
    const float py = add_rn(mul_rn(cam.fy, v0), cam.cy);
    if (rad != rad || px != px || py != py) return;
    const float fx0 = floorf(mul_rn(sub_rn(px, rad), inv_tw));  // == division by the tile side
    const float fx1 = floorf(mul_rn(add_rn(px, rad), inv_tw));
    const float fy0 = floorf(mul_rn(sub_rn(py, rad), inv_th));
    const float fy1 = floorf(mul_rn(add_rn(py, rad), inv_th));
    const float x0 = fmaxf(fx0, 0.0f), x1 = fminf(fx1, (float)(cam.tiles_x - 1));
    const float y0 = fmaxf(fy0, 0.0f), y1 = fminf(fy1, (float)(cam.tiles_y - 1));
    P.px = px;
    P.py = py;
    P.radius = rad;
    if (!(x0 <= x1 && y0 <= y1)) return;
    P.x0 = (int)x0;
    P.x1 = (int)x1;
    P.y0 = (int)y0;
    P.y1 = (int)y1;
    P.visible = true;
}

// Tiles the ellipse reaches (0: the Gaussian is culled), and the packed row table the
// duplicate kernel reads (16 words): word 0 = first row | rows << 16; words 1..15 = first
// column | (tiles in the earlier rows) << 16 per row; words past the last row are unused
// (the second 32-byte half is stored only for tables of more than kSpanRowsShort rows).
// More than kSpanRows rows or more than 65535 tiles mark a table the kernel recomputes
// instead.  The table is written to table[k * stride] (a thread's column of a shared-memory
// array).  Done for the 32 records of a warp at once (warp-collective; lanes whose record
// is not visible pass visible = false and get 0).  Each lane computes its own record's
// first row; the later (record, row) pairs of the warp are dealt out 32 at a time, so a
// lane with many rows does not hold up the warp: each pair's lane finds its record by a
// 5-step search of the inclusive scan of the later-row counts, takes the record's ellipse
// from that lane by shuffles and runs row_span on it (the same bits as the record's own
// lane would get).  Rows are written into the owner's table as first column |
// tiles in the row << 16 and turned into first column | tiles in the earlier rows << 16
// by the owner afterwards.  s_hits: one counter per thread of the block (shared memory).
__device__ __forceinline__ uint32_t count_tiles_warp(const Projected& P, bool visible, const View& cam,
                                                     const ViewTable& vt, uint32_t* table, int stride,
                                                     uint32_t* s_hits) {
    const int lane = threadIdx.x & 31;
    RowSpans rs;
    rs.ok = false;
    rs.ty0 = 0;
    rs.ty1 = -1;
    if (visible) rs = row_setup(P.px, P.py, P.A, P.B, P.C, vt.inv_tile_h, cam.tiles_y);
    const int rows = rs.ok ? rs.ty1 - rs.ty0 + 1 : 0;
    s_hits[threadIdx.x] = 0u;
    // each record's first row by its own lane (no shuffles)
    uint32_t hits_first = 0;
    if (rows > 0) {
        int a0 = 0, a1 = -1;
        row_span(rs, P.px, P.py, P.B, rs.ty0, vt.inv_tile_w, vt.tile_h, cam.tiles_x, a0, a1);
        hits_first = a1 >= a0 ? (uint32_t)(a1 - a0 + 1) : 0u;
        table[stride] = (uint32_t)(hits_first ? a0 : 0) | (hits_first << 16);
    }
    // the later rows, dealt out across the warp
    const int rest = rows > 1 ? rows - 1 : 0;
    int incl = rest;  // inclusive scan of the later rows over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFullMask, incl, 31);
    __syncwarp();
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + lane;
        int q = 0;  // records whose later rows end at or before pair e
#pragma unroll
        for (int b = 16; b > 0; b >>= 1) {
            const int v = __shfl_sync(kFullMask, incl, q + b - 1);
            if (v <= e) q += b;
        }
        q = min(q, 31);
        const int first = __shfl_sync(kFullMask, incl - rest, q);
        RowSpans rq;
        rq.ok = true;
        rq.ty0 = __shfl_sync(kFullMask, rs.ty0, q);
        rq.ty1 = __shfl_sync(kFullMask, rs.ty1, q);
        rq.ex = __shfl_sync(kFullMask, rs.ex, q);
        rq.ey = __shfl_sync(kFullMask, rs.ey, q);
        rq.dyr = __shfl_sync(kFullMask, rs.dyr, q);
        rq.det = __shfl_sync(kFullMask, rs.det, q);
        rq.invA = __shfl_sync(kFullMask, rs.invA, q);
        rq.Ak = __shfl_sync(kFullMask, rs.Ak, q);
        const float px = __shfl_sync(kFullMask, P.px, q), py = __shfl_sync(kFullMask, P.py, q);
        const float B = __shfl_sync(kFullMask, P.B, q);
        if (e < total) {
            const int k = e - first + 1;  // row index within the record (row 0 is its own lane's)
            int a0 = 0, a1 = -1;
            row_span(rq, px, py, B, rq.ty0 + k, vt.inv_tile_w, vt.tile_h, cam.tiles_x, a0, a1);
            const uint32_t len = a1 >= a0 ? (uint32_t)(a1 - a0 + 1) : 0u;
            const int owner = (int)(threadIdx.x & ~31u) + q;
            if (k < kSpanRows) table[(int)(q - lane) + (1 + k) * stride] = (uint32_t)(len ? a0 : 0) | (len << 16);
            if (len) atomicAdd(&s_hits[owner], len);
        }
    }
    __syncwarp();
    uint32_t hits = 0;
    for (int k = 0; k < min(rows, kSpanRows); ++k) {
        const uint32_t w = table[(1 + k) * stride];
        table[(1 + k) * stride] = (w & 0xffffu) | (min(hits, 0xffffu) << 16);
        hits += w >> 16;
    }
    hits = s_hits[threadIdx.x] + hits_first;
    const bool fits = rows <= kSpanRows && hits <= 0xffffu;
    table[0] = (uint32_t)rs.ty0 | ((fits ? (uint32_t)rows : kSpanRowsOverflow) << 16);
    return rs.ok ? hits : 0u;
}

// The view direction of Eq. 5, d = (X - campos)/|X - campos|, and 1/|X - campos| (one
// hardware reciprocal square root: the colour is not a binning decision).
__device__ __forceinline__ void view_direction(const View& cam, const float X[3], float d[3],
                                               float& inv_len) {
    const float dx = X[0] - cam.campos[0], dy = X[1] - cam.campos[1], dz = X[2] - cam.campos[2];
    inv_len = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    d[0] = dx * inv_len;
    d[1] = dy * inv_len;
    d[2] = dz * inv_len;
}

constexpr int kPreThreads = 128;

// A Gaussian's colour parameters held in a column of shared memory (stride kPreThreads):
// the view loops of the forward and the backward pass read them per view instead of keeping
// ~40 registers live.  Layout: sh, amplitudes, unit axes, sharpness, then |mu_k| (free
// axes) or the frame quaternion and |(1, f)| (frame).
template <int L, int K, int AX>
struct ColourShared {
    static constexpr int NSH = (L + 1) * (L + 1);
    static constexpr int NAX = (K > 0 && AX != kAxWorld) ? 3 * K : 0;
    static constexpr int NEXTRA = (K > 0 && AX == kAxFree) ? K : ((K > 0 && AX == kAxFrame) ? 5 : 0);
    static constexpr int COUNT = 3 * NSH + 3 * K + NAX + K + NEXTRA;
    float* p;

    __device__ __forceinline__ float& at(int j) const { return p[j * kPreThreads]; }

    __device__ __forceinline__ void load(const sgs_gaussians& g, int64_t i) const {
        const int64_t S = g.stride;
#pragma unroll
        for (int k = 0; k < 3 * NSH; ++k) at(k) = __ldg(g.sh + k * S + i);
        if constexpr (AX == kAxFrame && K > 0) {
            const float f[3] = {__ldg(g.sg_axis + i), __ldg(g.sg_axis + S + i), __ldg(g.sg_axis + 2 * S + i)};
            float q[4], R[3][3];
            const float n = frame_axes(f, q, R);
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) at(3 * NSH + 3 * K + 3 * k + c) = R[c][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) at(3 * NSH + 3 * K + NAX + K + j) = q[j];
            at(3 * NSH + 3 * K + NAX + K + 4) = n;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) at(3 * NSH + 3 * k + c) = __ldg(g.sg_amp + (k * 3 + c) * S + i);
            at(3 * NSH + 3 * K + NAX + k) = __ldg(g.sg_sharp + k * S + i);
            if constexpr (AX == kAxFree) {
                float m[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) m[c] = __ldg(g.sg_axis + (k * 3 + c) * S + i);
                const float n = axis_length(m);
                at(3 * NSH + 3 * K + NAX + K + k) = n;
                const float inv = 1.0f / n;
#pragma unroll
                for (int c = 0; c < 3; ++c) at(3 * NSH + 3 * K + 3 * k + c) = m[c] * inv;
            }
        }
    }

    __device__ __forceinline__ float csh(int k, int c) const { return at(3 * k + c); }
    __device__ __forceinline__ float camp(int k, int c) const { return at(3 * NSH + 3 * k + c); }
    __device__ __forceinline__ float caxis(int k, int c) const { return at(3 * NSH + 3 * K + 3 * k + c); }
    __device__ __forceinline__ float csharp(int k) const { return at(3 * NSH + 3 * K + NAX + k); }
    __device__ __forceinline__ float caxis_norm(int k) const { return at(3 * NSH + 3 * K + NAX + K + k); }
    __device__ __forceinline__ float cframe_q(int j) const { return at(3 * NSH + 3 * K + NAX + K + j); }
    __device__ __forceinline__ float cframe_norm() const { return at(3 * NSH + 3 * K + NAX + K + 4); }
};

template <int L, int K, int AX>
__global__ void __launch_bounds__(kPreThreads, 8) preprocess_kernel(const sgs_gaussians g, const ViewTable vt,
                                                                 float4* __restrict__ rec0,
                                                                 float4* __restrict__ rec1,
                                                                 float4* __restrict__ rec2,
                                                                 uint2* __restrict__ rect,
                                                                 uint32_t* __restrict__ tiles,
                                                                 uint4* __restrict__ spans,
                                                                 uint32_t* __restrict__ sort_keys,
                                                                 uint32_t* __restrict__ sort_vals,
                                                                 uint32_t* __restrict__ flags,
                                                                 const RecordValue rv) {
    using CS = ColourShared<L, K, AX>;
    __shared__ float s_colour[CS::COUNT * kPreThreads];
    __shared__ uint32_t s_table[16 * kPreThreads];
    __shared__ uint32_t s_hits[kPreThreads];
    // the lanes past n stay (the row counting is warp-collective) on a copy of the last
    // Gaussian and write nothing
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < g.n;
    if (__all_sync(kFullMask, !live)) return;  // whole warps past n leave
    const int64_t i = live ? i0 : g.n - 1;
    const int64_t S = g.stride;
    const float X[3] = {__ldg(g.mean + i), __ldg(g.mean + S + i), __ldg(g.mean + 2 * S + i)};
    const float opacity = __ldg(g.opacity + i);
    Geometry G;
    geometry_exact(g, i, G);
    const CS cp{s_colour + threadIdx.x};
    cp.load(g, i);
    uint32_t* table = s_table + threadIdx.x;
    for (int v = 0; v < vt.B; ++v) {
        const View& cam = vt.v[v];
        const int64_t r = (int64_t)v * g.n + i;
        Projected P;
        project_exact(cam, X, G, vt.inv_tile_w, vt.inv_tile_h, P);
        const uint32_t hits = count_tiles_warp(P, live && P.visible, cam, vt, table, kPreThreads, s_hits);
        if (!live) continue;
        // the record sort's pair: depth bits (depth > near > 0 orders like the floats)
        sort_keys[r] = hits ? __float_as_uint(P.t[2]) : 0xffffffffu;
        sort_vals[r] = rv.pack((uint32_t)r, hits);
        if (hits == 0u) {
            rect[r] = make_uint2(0u, 0u);
            tiles[r] = 0u;
            flags[r] = 0u;
            continue;
        }
        float d[3], inv_len;
        view_direction(cam, X, d, inv_len);
        float pre[3];
        const int D = record_sh_degree<L>(g, P.radius);
        colour_eval<L, K, AX>(cp, d, pre, (D + 1) * (D + 1));
        uint32_t mask = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (pre[c] < 0.0f) {
                pre[c] = 0.0f;
                mask |= 1u << c;
            }
        rec0[r] = make_float4(P.px, P.py, -0.5f * P.A, -P.B);
        rec1[r] = make_float4(-0.5f * P.C, opacity, P.t[2], P.radius);
        rec2[r] = make_float4(pre[0], pre[1], pre[2], __uint_as_float(mask));
        flags[r] = kFlagVisible | mask | (P.clampx ? kFlagClampX : 0u) | (P.clampy ? kFlagClampY : 0u) |
                   ((uint32_t)D << kFlagShift);
        rect[r] = make_uint2((uint32_t)P.x0 | ((uint32_t)P.y0 << 16),
                             (uint32_t)P.x1 | ((uint32_t)P.y1 << 16));
        tiles[r] = hits;
        // words 0-7 (one 32-byte sector) hold the tables of up to 7 rows; the second sector
        // is written only for longer ones, and the duplicate reads it only then
        const int chunks = (table[0] >> 16) > kSpanRowsShort ? 4 : 2;
        for (int k = 0; k < chunks; ++k)
            spans[4 * r + k] = make_uint4(table[(4 * k) * kPreThreads], table[(4 * k + 1) * kPreThreads],
                                          table[(4 * k + 2) * kPreThreads], table[(4 * k + 3) * kPreThreads]);
    }
}

// ------------------------------------------------------------------------------ backward
// The intermediates of the projection that the chain rule needs (t, the clamped x/z and
// y/z, J, T = J W, T Sigma and the conic), recomputed in plain single precision with fused
// multiply-adds and two approximate reciprocals.  The frustum-clamp decisions are the forward's, read
// from the record's flags (kFlagClampX/Y), so every branch is the one the forward took; the
// values differ from the forward's correctly rounded ones by a few units in the last place,
// far inside the gradients' tolerance.
__device__ __forceinline__ void project_fast(const View& cam, const float X[3], const Geometry& G, uint32_t f,
                                             Projected& P) {
    const float* V = cam.V;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        P.t[r] = fmaf(V[4 * r], X[0], fmaf(V[4 * r + 1], X[1], fmaf(V[4 * r + 2], X[2], V[4 * r + 3])));
    const float tz = P.t[2], iz = __fdividef(1.0f, tz);
    const float u0 = P.t[0] * iz, v0 = P.t[1] * iz;
    P.clampx = (f & kFlagClampX) != 0u;
    P.clampy = (f & kFlagClampY) != 0u;
    P.u = P.clampx ? copysignf(cam.limx, u0) : u0;
    P.v = P.clampy ? copysignf(cam.limy, v0) : v0;
    P.J00 = cam.fx * iz;
    P.J02 = -cam.fx * P.u * iz;
    P.J11 = cam.fy * iz;
    P.J12 = -cam.fy * P.v * iz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        P.T[0][c] = fmaf(P.J00, V[c], P.J02 * V[8 + c]);
        P.T[1][c] = fmaf(P.J11, V[4 + c], P.J12 * V[8 + c]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            P.TS[r][c] = fmaf(P.T[r][0], G.Sig[0][c], fmaf(P.T[r][1], G.Sig[1][c], P.T[r][2] * G.Sig[2][c]));
    P.a = fmaf(P.TS[0][0], P.T[0][0], fmaf(P.TS[0][1], P.T[0][1], fmaf(P.TS[0][2], P.T[0][2], 0.3f)));
    P.b = fmaf(P.TS[0][0], P.T[1][0], fmaf(P.TS[0][1], P.T[1][1], P.TS[0][2] * P.T[1][2]));
    P.c = fmaf(P.TS[1][0], P.T[1][0], fmaf(P.TS[1][1], P.T[1][1], fmaf(P.TS[1][2], P.T[1][2], 0.3f)));
    const float idet = __fdividef(1.0f, fmaf(P.a, P.c, -P.b * P.b));
    P.A = P.c * idet;
    P.B = -P.b * idet;
    P.C = P.a * idet;
}

template <int L, int K, int AX>
__global__ void __launch_bounds__(kPreThreads) preprocess_backward_kernel(
    const sgs_gaussians g, const ViewTable vt, const float4* __restrict__ rec0,
    const float4* __restrict__ rec1, const uint32_t* __restrict__ flags,
    float4* __restrict__ grad2d, int64_t R, sgs_grads out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int64_t S = g.stride;
    const float X[3] = {__ldg(g.mean + i), __ldg(g.mean + S + i), __ldg(g.mean + 2 * S + i)};
    Geometry G;
    geometry_exact(g, i, G);
    using CS = ColourShared<L, K, AX>;
    __shared__ float s_colour[CS::COUNT * kPreThreads];
    const CS cp{s_colour + threadIdx.x};
    cp.load(g, i);
    ColourGrads<L, K, AX> cg;
    cg.zero();
    float gX[3] = {0.0f, 0.0f, 0.0f};
    float gSig[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) gSig[r][c] = 0.0f;
    float gop = 0.0f;
    const float opacity = __ldg(g.opacity + i);
    // the next view's record flags and 2D gradients travel to shared memory while this
    // view's chain rule runs (double-buffered, one slot per thread)
    __shared__ __align__(16) float4 s_g[2][3][kPreThreads];
    __shared__ uint32_t s_t[2][kPreThreads];
    const int tx = threadIdx.x;
    auto prefetch = [&](int v, int b) {
        const int64_t r = (int64_t)v * g.n + i;
        async_copy4(&s_t[b][tx], flags + r);
#pragma unroll
        for (int c = 0; c < 2; ++c) async_copy16(&s_g[b][c][tx], grad2d + c * R + r);
        async_copy4(&s_g[b][2][tx].x, reinterpret_cast<const float*>(grad2d + 2 * R) + r);
        async_commit();
    };
    if (vt.B > 0) prefetch(0, 0);
    for (int v = 0; v < vt.B; ++v) {
        const int b = v & 1;
        if (v + 1 < vt.B) {
            prefetch(v + 1, b ^ 1);
            async_wait<1>();
        } else {
            async_wait<0>();
        }
        const uint32_t f = s_t[b][tx];
        if (!(f & kFlagVisible)) continue;
        const float4 g0 = s_g[b][0][tx], g1 = s_g[b][1][tx], g2 = s_g[b][2][tx];
        {
            // the reverse blend adds into the 2D gradients of visible records only: clearing
            // them here, once read, leaves the whole region zero for the next backward
            const int64_t r = (int64_t)v * g.n + i;
            grad2d[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            grad2d[R + r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            reinterpret_cast<float*>(grad2d + 2 * R)[r] = 0.0f;
        }
        const View& cam = vt.v[v];
        Projected P;
        project_fast(cam, X, G, f, P);
        gop += g1.y;
        // colour: the SH degree and the colour-clamp decisions are the forward's (flags)
        {
            float d[3], inv;
            view_direction(cam, X, d, inv);
            const int D = (int)((f >> kFlagShift) & 3u);
            const int nsh = (D + 1) * (D + 1);
            const float grgb[3] = {g1.z, g1.w, g2.x};
            float gpre[3], gd[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) gpre[c] = (f >> c) & 1u ? 0.0f : grgb[c];
            cg.accumulate(cp, d, gpre, gd, nsh);
            const float dot = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) gX[c] += (gd[c] - d[c] * dot) * inv;
        }
        // The reverse blend's sums over the pixels that blend the record below the alpha
        // clamp: S = gG (dx, dy, dx^2, dx dy, dy^2) with gG = dL/dalpha G, d = centre - pixel
        // centre.  power = -(A dx^2 + 2 B dx dy + C dy^2) / 2 and alpha = o G give
        // dL/d centre = -o (A S_x + B S_y, B S_x + C S_y), dL/d(A, B, C) = -o (S_xx / 2,
        // S_xy, S_yy / 2).
        const float A = P.A, B = P.B, C = P.C;
        const float gpx = -opacity * fmaf(A, g0.x, B * g0.y), gpy = -opacity * fmaf(B, g0.x, C * g0.y);
        const float gA = -0.5f * opacity * g0.z, gB = -opacity * g0.w, gC = -0.5f * opacity * g1.x;
        // conic -> Sigma2D:  dS = -Con G Con,  G = [[gA, gB/2], [gB/2, gC]]
        const float P00 = A * gA + 0.5f * B * gB, P01 = 0.5f * A * gB + B * gC;
        const float P10 = B * gA + 0.5f * C * gB, P11 = 0.5f * B * gB + C * gC;
        const float G2[2][2] = {{-(P00 * A + P01 * B), -(P00 * B + P01 * C)},
                                {-(P00 * B + P01 * C), -(P10 * B + P11 * C)}};
        // Sigma2D = T Sigma T^T:  dSigma += T^T G2 T,  dT = 2 G2 T Sigma
        const float(&TS)[2][3] = P.TS;
        float gT[2][3];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c) gT[rr][c] = 2.0f * (G2[rr][0] * TS[0][c] + G2[rr][1] * TS[1][c]);
        float GT[2][3];  // G2 T
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c) GT[rr][c] = G2[rr][0] * P.T[0][c] + G2[rr][1] * P.T[1][c];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) gSig[j][k] += P.T[0][j] * GT[0][k] + P.T[1][j] * GT[1][k];
        // T = J W
        const float* V = cam.V;
        const float gJ00 = gT[0][0] * V[0] + gT[0][1] * V[1] + gT[0][2] * V[2];
        const float gJ02 = gT[0][0] * V[8] + gT[0][1] * V[9] + gT[0][2] * V[10];
        const float gJ11 = gT[1][0] * V[4] + gT[1][1] * V[5] + gT[1][2] * V[6];
        const float gJ12 = gT[1][0] * V[8] + gT[1][1] * V[9] + gT[1][2] * V[10];
        const float tz = P.t[2], iz = __fdividef(1.0f, tz), iz2 = iz * iz, iz3 = iz2 * iz;
        const float tx = P.u * tz, ty = P.v * tz;
        float gt[3] = {0.0f, 0.0f, 0.0f};
        gt[2] += -cam.fx * iz2 * gJ00 - cam.fy * iz2 * gJ11 + 2.0f * cam.fx * tx * iz3 * gJ02 +
                 2.0f * cam.fy * ty * iz3 * gJ12;
        const float gtx = -cam.fx * iz2 * gJ02, gty = -cam.fy * iz2 * gJ12;
        if (P.clampx) gt[2] += gtx * P.u; else gt[0] += gtx;
        if (P.clampy) gt[2] += gty * P.v; else gt[1] += gty;
        // screen mean
        gt[0] += cam.fx * iz * gpx;
        gt[2] += -cam.fx * P.t[0] * iz2 * gpx;
        gt[1] += cam.fy * iz * gpy;
        gt[2] += -cam.fy * P.t[1] * iz2 * gpy;
        // t = W X + t_v
#pragma unroll
        for (int c = 0; c < 3; ++c) gX[c] += V[c] * gt[0] + V[4 + c] * gt[1] + V[8 + c] * gt[2];
    }
    // Sigma = M M^T, M = R diag(s):  dM = 2 dSigma_sym M
    float gR[3][3], gs[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 3; ++l) acc += (gSig[r][l] + gSig[l][r]) * (G.R[l][c] * G.s[c]);
            gR[r][c] = acc * G.s[c];
            gs[c] += acc * G.R[r][c];
        }
    const float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
    float gq[4];
    gq[0] = 2.0f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    gq[1] = 2.0f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.0f * x * gR[1][1] - w * gR[1][2] +
                    z * gR[2][0] + w * gR[2][1] - 2.0f * x * gR[2][2]);
    gq[2] = 2.0f * (-2.0f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                    w * gR[2][0] + z * gR[2][1] - 2.0f * y * gR[2][2]);
    gq[3] = 2.0f * (-2.0f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.0f * z * gR[1][1] +
                    y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    const float dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    const float iq = 1.0f / G.qnorm;
#pragma unroll
    for (int c = 0; c < 4; ++c) out.rot[c * S + i] = (gq[c] - G.q[c] * dot) * iq;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        out.mean[c * S + i] = gX[c];
        out.scale[c * S + i] = gs[c];
    }
    out.opacity[i] = gop;
    cg.store(cp, out, S, i);
}

template <int L, int K, int AX>
cudaError_t launch_pre(const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                       cudaStream_t s) {
    const int threads = 128;
    const int blocks = (int)((g.n + threads - 1) / threads);
    if (blocks > 0)
        preprocess_kernel<L, K, AX><<<blocks, threads, 0, s>>>(g, vt, p.rec0, p.rec1, p.rec2, p.rect,
                                                                 p.tiles, p.spans, p.sort_keys, p.sort_vals,
                                                                 p.flags, p.rv);
    return cudaGetLastError();
}

template <int L, int K, int AX>
cudaError_t launch_pre_bwd(const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                           float4* grad2d, int64_t R, const sgs_grads& out, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (int)((g.n + threads - 1) / threads);
    if (blocks > 0)
        preprocess_backward_kernel<L, K, AX>
            <<<blocks, threads, 0, s>>>(g, vt, p.rec0, p.rec1, p.flags, grad2d, R, out);
    return cudaGetLastError();
}

template <int L, int K>
cudaError_t dispatch_axis(bool fwd, const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                          float4* grad2d, int64_t R, const sgs_grads* out, cudaStream_t s) {
    if (g.axis_mode == SGS_AXIS_ORTHO_FIXED || g.axis_mode == SGS_AXIS_ORTHO_FRAME) {
        if constexpr (K <= 3) {
            if (g.axis_mode == SGS_AXIS_ORTHO_FIXED)
                return fwd ? launch_pre<L, K, kAxWorld>(g, vt, p, s)
                           : launch_pre_bwd<L, K, kAxWorld>(g, vt, p, grad2d, R, *out, s);
            return fwd ? launch_pre<L, K, kAxFrame>(g, vt, p, s)
                       : launch_pre_bwd<L, K, kAxFrame>(g, vt, p, grad2d, R, *out, s);
        }
        return cudaErrorInvalidValue;
    }
    return fwd ? launch_pre<L, K, kAxFree>(g, vt, p, s)
               : launch_pre_bwd<L, K, kAxFree>(g, vt, p, grad2d, R, *out, s);
}

template <int L>
cudaError_t dispatch_k(bool fwd, const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                       float4* grad2d, int64_t R, const sgs_grads* out, cudaStream_t s) {
    switch (g.num_lobes) {
        case 0: return dispatch_axis<L, 0>(fwd, g, vt, p, grad2d, R, out, s);
        case 1: return dispatch_axis<L, 1>(fwd, g, vt, p, grad2d, R, out, s);
        case 2: return dispatch_axis<L, 2>(fwd, g, vt, p, grad2d, R, out, s);
        case 3: return dispatch_axis<L, 3>(fwd, g, vt, p, grad2d, R, out, s);
        case 4: return dispatch_axis<L, 4>(fwd, g, vt, p, grad2d, R, out, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch(bool fwd, const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                     float4* grad2d, int64_t R, const sgs_grads* out, cudaStream_t s) {
    switch (g.sh_degree) {
        case 0: return dispatch_k<0>(fwd, g, vt, p, grad2d, R, out, s);
        case 1: return dispatch_k<1>(fwd, g, vt, p, grad2d, R, out, s);
        case 2: return dispatch_k<2>(fwd, g, vt, p, grad2d, R, out, s);
        case 3: return dispatch_k<3>(fwd, g, vt, p, grad2d, R, out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_preprocess(const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                              cudaStream_t s) {
    return dispatch(true, g, vt, p, nullptr, 0, nullptr, s);
}

cudaError_t launch_preprocess_backward(const sgs_gaussians& g, const ViewTable& vt,
                                       const RecordPtrs& p, float4* grad2d, int64_t R,
                                       const sgs_grads& out, cudaStream_t s) {
    return dispatch(false, g, vt, p, grad2d, R, &out, s);
}

}  // namespace sgs
