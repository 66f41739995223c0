// Stage (e): front-to-back alpha blending per pixel, and its reverse-mode pass.
//
// One CTA per (view, tile), the tiles taken most expensive first (vt.order).  Each warp
// owns an 8-pixel-wide block of the tile; a thread has one, two (packed f32x2 pairs in the
// blend_pair kernels) or four pixels of it.  The tile's depth-sorted instance list
// [start, end) is staged batch_depth Gaussians at a time in shared memory, gathered
// through the sorted record ids, with a mask of the warp blocks each Gaussian's support
// may reach; a warp visits only the Gaussians of its bit words.  Per pixel centre p:
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy;  skip if power < -4.5 (outside 3 sigma)
//   alpha = min(0.99, opacity exp(power));      skip if alpha < 1/255
//   T' = T (1 - alpha);                          stop before this Gaussian if T' < 1e-4
//   C += rgb alpha T;  T = T'
// and the pixel is C + T bg.  A warp stops visiting once all its pixels are finished, and
// the CTA stops fetching batches once __syncthreads_count reports every pixel finished.
//
// The backward pass walks each tile's list from the last contributor to the front,
// rebuilding T_k = T_{k+1} / (1 - alpha_k) from the stored final transmittance and
// carrying the normalised colour behind (acc += alpha (rgb - acc), starting at bg; the
// two-pixel kernel carries its dot product with the pixel's upstream gradient).  It
// recomputes power and alpha with the same operations as the forward pass, so every skip
// decision is identical; per Gaussian the warp's 9 gradient sums are reduced with shuffles
// and added by one scalar reduction instruction from nine lanes (the two-pixel kernel) or
// two 16-byte vector reductions and a scalar one (the others).  The sums are those of
// gG = dL/dalpha G (where the 0.99 clamp is not active) and its moments gG dx, gG dy,
// gG dx^2, gG dx dy, gG dy^2 (d = centre - pixel centre), and of alpha T dL/dC per channel:
// the power is a quadratic form in d, so its derivatives in the centre and the conic are
// linear in these sums, and the preprocess backward applies the opacity and the conic once
// per record instead of once per pixel.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

struct TileCoord {
    int v, tx, ty;
};

__device__ __forceinline__ TileCoord tile_of(const ViewTable& vt, uint32_t g) {
    int v = 0;
    while (v + 1 < vt.B && vt.v[v + 1].tile_base <= g) ++v;
    const uint32_t local = g - vt.v[v].tile_base;
    TileCoord c;
    c.v = v;
    c.tx = (int)(local % (uint32_t)vt.v[v].tiles_x);
    c.ty = (int)(local / (uint32_t)vt.v[v].tiles_x);
    return c;
}

// Thread-to-pixel map of a tile: each warp owns an 8-pixel-wide block of 4 * PPT rows
// (blocks row-major over the tile), lane l takes column l % 8 and rows l / 8 + 4 q,
// q < PPT.  Compact warp footprints let a whole warp skip a Gaussian whose ellipse misses
// its block.  Needs tile_w % 8 == 0 and tile_h % (4 PPT) == 0.
struct WarpBlock {
    int x0, y0;  // block origin inside the tile
};

template <int PPT>
__device__ __forceinline__ WarpBlock warp_block(const ViewTable& vt) {
    const int w = threadIdx.x >> 5, per_row = vt.tile_w >> 3;
    WarpBlock b;
    b.x0 = (w % per_row) * 8;
    b.y0 = (w / per_row) * 4 * PPT;
    return b;
}

// The warp blocks of the CTA's tile in which some pixel may blend the Gaussian: bit w for
// warp w.  A pixel blends it only inside its support, Q(d) <= 9 (Mahalanobis distance 3),
// and where its alpha o exp(-Q/2) reaches 1/255, that is Q <= 2 ln(255 o): for opacities
// below about 0.35 the second bound is the tighter one.  With Q(d) = A dx^2 + 2B dx dy +
// C dy^2 (the conic; records store (qa, qb, qc) = (-A/2, -B, -C/2)) and Qs the smaller
// bound widened by 0.11 % (and 0.002 for the alpha bound), the ellipse Q <= Qs is cut into
// the tile's bands of block rows.  Over a band's pixel-centre rows (padded by 1/64 pixel)
// its x-extent is exact: the rightmost x is the ellipse's rightmost point ex when that
// point's row -B ex / C falls in the band, else the larger chord end
// (-B y + sqrt(Qs A - det y^2)) / A at the band's two edge rows (the chord end is concave
// in y), and the leftmost mirrors it.  Each block column whose padded pixel-centre columns
// meet the extent gets its bit.  A blending pixel centre has Q within single-precision
// rounding of the bounds (the exponential's and logarithm's errors are below 1e-5 there),
// which the slack and the pad cover (the chord's own rounding is far below that slack), so
// a warp without its bit has no pixel that blends the Gaussian.  A degenerate conic or a
// non-finite centre sets every bit; an opacity at which no alpha reaches 1/255 none.  The
// divisions and square roots are the hardware's approximate ones (relative error a few
// 1e-7): the test needs no correctly rounded operation, the slack covers them many times.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Asks L2 for the records of the batch entries [first, first + cnt) (ids clamped like the
// staging's), one thread per entry: while the backward walks one staged batch, the gathers
// of the next one travel from DRAM (a hint; nothing waits for it).  The forward does not
// use it: it may stop a tile before its next batch, and the instructions cost more in its
// issue-bound loop than the latency they hide (measured 3.32 -> 3.50 ms).
__device__ __forceinline__ void prefetch_batch(const uint32_t* __restrict__ first, int cnt, uint32_t R,
                                               const float4* rec0, const float4* rec1, const float4* rec2) {
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const uint32_t id = min(first[j], R - 1);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rec0 + id));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rec1 + id));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rec2 + id));
    }
}

template <int PPT>
__device__ __forceinline__ uint32_t block_mask(const ViewTable& vt, const TileCoord& tc, float px, float py,
                                               float qa, float qb, float qc, float o) {
    constexpr int BH = 4 * PPT;  // pixel rows per block
    const float A = -2.0f * qa, B = -qb, C = -2.0f * qc;
    const float det = A * C - B * B;
    // Centre relative to the tile's first pixel centre.
    const float gx = px - ((float)(tc.tx * vt.tile_w) + 0.5f);
    const float gy = py - ((float)(tc.ty * vt.tile_h) + 0.5f);
    if (!(det > 0.0f && A > 0.0f && C > 0.0f && fabsf(gx) < 1e30f && fabsf(gy) < 1e30f)) return ~0u;
    // fminf keeps the support bound when the logarithm is NaN
    const float Qs = fminf(kSpanQ, (2.0f * __logf(o * 255.0f) + 0.002f) * (kSpanQ / 9.0f));
    if (!(Qs > 0.0f)) return 0u;
    const int nbx = vt.tile_w >> 3, nby = vt.tile_h / BH;
    const float k = __fdividef(Qs, det);
    const float ex = sqrt_approx(k * C), ey = sqrt_approx(k * A);
    const float dyr = __fdividef(-B * ex, C);  // row offset of the rightmost point
    const float iA = __fdividef(1.0f, A), Ak = A * Qs;
    const float b0 = fmaxf(ceilf((gy - ey - kSpanPad - (float)(BH - 1)) * (1.0f / BH)), 0.0f);
    const float b1 = fminf(floorf((gy + ey + kSpanPad) * (1.0f / BH)), (float)(nby - 1));
    uint32_t mask = 0;
    for (int b = (int)b0; b <= (int)b1; ++b) {
        const float u0 = fmaxf((float)(b * BH) - kSpanPad - gy, -ey);
        const float u1 = fminf((float)(b * BH + BH - 1) + kSpanPad - gy, ey);
        if (!(u0 <= u1)) continue;
        const float s0 = sqrt_approx(fmaxf(0.0f, Ak - det * u0 * u0));
        const float s1 = sqrt_approx(fmaxf(0.0f, Ak - det * u1 * u1));
        const float xmax = (u0 <= dyr && dyr <= u1) ? ex : fmaxf(s0 - B * u0, s1 - B * u1) * iA;
        const float xmin = (u0 <= -dyr && -dyr <= u1) ? -ex : fminf(-B * u0 - s0, -B * u1 - s1) * iA;
        // Block column c holds pixel-centre columns [8c, 8c + 7].
        const float c0 = fmaxf(ceilf((gx + xmin - kSpanPad - 7.0f) * 0.125f), 0.0f);
        const float c1 = fminf(floorf((gx + xmax + kSpanPad) * 0.125f), (float)(nbx - 1));
        if (c0 <= c1) {
            const int n = (int)c1 - (int)c0 + 1;
            mask |= ((1u << n) - 1u) << (b * nbx + (int)c0);
        }
    }
    return mask;
}

// Staged layouts of a batch entry in shared memory (field f of entry j at sb[j * fields + f],
// so that a visit finds all fields of its entry at one address plus constant offsets):
// kPlain: the three records as read, (px, py, qa, qb), (qc, o, depth, radius),
//         (r, g, b, clamp mask);
// kPairs: each scalar the two-pixel kernels combine with a pair of pixels duplicated into
//         a packed pair, (qa qa, qb qb), (qc qc, o o), (px px, py py), then the colour
//         record as read;
// kPairsColour: as kPairs, with the colour as pairs too and the record id beside blue:
//         (r r, g g), (b b, id 0) (id as the bits of a float).
enum StageLayout { kPlain = 0, kPairs = 1, kPairsColour = 2 };
constexpr int stage_fields(int layout) { return layout == kPlain ? 3 : layout == kPairs ? 4 : 5; }

// Stages one group of 32 batch entries (this warp's group g: entries 32 g + lane < cnt,
// from the tile's sorted list at `first`) in shared memory, and writes for every warp w of
// the CTA the 32-bit word of the group's entries that some pixel of w's block may blend
// (bits[w * words + g]; bit b = entry 32 g + b): a transpose of the entries' block masks by
// one ballot per warp.  The block masks are computed, or read from mask_in[j] (those a
// forward with the same warp blocks stored), and optionally stored to mask_out[j].  Without
// alpha_bound the masks take the support alone (the counting forwards, whose evaluation
// counts are those of the support test).
// Returns the record id of the lane's entry.  Warp-collective.
template <int PPT, int LAYOUT>
__device__ __forceinline__ uint32_t stage_group(const ViewTable& vt, const TileCoord& tc, int g, int cnt,
                                                const uint32_t* __restrict__ first, uint32_t R,
                                                const float4* __restrict__ rec0, const float4* __restrict__ rec1,
                                                const float4* __restrict__ rec2, float4* sb,
                                                uint32_t* bits, int words, uint16_t* __restrict__ mask_out,
                                                const uint16_t* __restrict__ mask_in, bool alpha_bound = true) {
    const int lane = threadIdx.x & 31, j = g * 32 + lane;
    uint32_t mask = 0, id = 0;
    if (j < cnt) {
        if (mask_in) mask = mask_in[j];
        id = min(first[j], R - 1);  // ids are < R by construction
        const float4 r0 = rec0[id], r1 = rec1[id], r2 = rec2[id];
        float4* e = sb + j * stage_fields(LAYOUT);
        if (LAYOUT == kPlain) {
            e[0] = r0;
            e[1] = r1;
            e[2] = r2;
        } else {
            e[0] = make_float4(r0.z, r0.z, r0.w, r0.w);
            e[1] = make_float4(r1.x, r1.x, r1.y, r1.y);
            e[2] = make_float4(r0.x, r0.x, r0.y, r0.y);
            if (LAYOUT == kPairs) {
                e[3] = r2;
            } else {
                e[3] = make_float4(r2.x, r2.x, r2.y, r2.y);
                e[4] = make_float4(r2.z, r2.z, __uint_as_float(id), 0.0f);
            }
        }
        if (!mask_in) mask = block_mask<PPT>(vt, tc, r0.x, r0.y, r0.z, r0.w, r1.x, alpha_bound ? r1.y : 1.0f);
        if (mask_out) mask_out[j] = (uint16_t)mask;
    }
    const int nw = (int)(blockDim.x >> 5);
    uint32_t mine = 0;
    for (int w = 0; w < nw; ++w) {
        const uint32_t b = __ballot_sync(kFullMask, (mask >> w) & 1u);
        if (lane == w) mine = b;
    }
    if (lane < nw) bits[lane * words + g] = mine;
    return id;
}

// Packed pairs of single-precision values for the f32x2 instructions of sm_100 and later:
// one instruction applies the operation to both halves, each half rounded exactly as the
// scalar operation (round to nearest even, subnormals kept).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk(f32x2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// A staged float4 field as its two packed pairs (x, y) and (z, w).
__device__ __forceinline__ ulonglong2 pairs(const float4* f) { return *reinterpret_cast<const ulonglong2*>(f); }

// Tile range clipped to the instances actually written (all of them unless overflowed).
__device__ __forceinline__ uint2 clamp_range(uint2 r, uint32_t m) {
    r.y = min(r.y, m);
    r.x = min(r.x, r.y);
    return r;
}

// The backward's tile-order cost of this CTA's tile: the largest position of a last
// contributor over the tile's pixels (the reverse walk starts there).  Block-collective,
// at the end of a forward kernel (every thread reaches it).
__device__ __forceinline__ void write_backward_key(const ViewTable& vt, uint32_t tile, uint32_t my_last) {
    __shared__ uint32_t s_top;
    const uint32_t wmax = __reduce_max_sync(kFullMask, my_last);
    if (threadIdx.x == 0) s_top = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && wmax) atomicMax(&s_top, wmax);
    __syncthreads();
    if (threadIdx.x == 0 && vt.tile_top) vt.tile_top[tile] = s_top;
}

// Per-pixel state of the forward walk.
struct FwdPixel {
    float pxc, pyc;  // pixel centre
    float T, C0, C1, C2;
    uint32_t last, evaluated, contributed;
    bool inside, done;
};

// PPT pixels per thread: pixel q of thread t is (t % tile_w, t / tile_w + q * tile_h / PPT)
// inside the tile, so one shared-memory read of a Gaussian serves PPT pixels.
template <int PPT, bool COUNT>
__global__ void __launch_bounds__(512) blend_kernel(const ViewTable vt, const uint2* __restrict__ ranges,
                                                     const uint32_t* __restrict__ vals, uint32_t R,
                                                     const float4* __restrict__ rec0,
                                                     const float4* __restrict__ rec1,
                                                     const float4* __restrict__ rec2, int batch,
                                                     float bg0, float bg1, float bg2,
                                                     float* __restrict__ out_rgb,
                                                     float* __restrict__ out_T,
                                                     float* __restrict__ pix_T,
                                                     uint32_t* __restrict__ pix_last,
                                                     uint2* __restrict__ pix_count,
                                                     const DeviceStatus* __restrict__ st) {
    extern __shared__ float4 sbuf[];
    const int words = (batch + 31) >> 5;
    uint32_t* bits = reinterpret_cast<uint32_t*>(sbuf + 3 * batch);
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    const uint32_t tile = vt.order ? vt.order[blockIdx.x] : blockIdx.x;
    const TileCoord tc = tile_of(vt, tile);
    const View& cam = vt.v[tc.v];
    const WarpBlock wb = warp_block<PPT>(vt);
    const int lx = wb.x0 + (threadIdx.x & 7), ly = wb.y0 + ((threadIdx.x >> 3) & 3);
    FwdPixel P[PPT];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int x = tc.tx * vt.tile_w + lx, y = tc.ty * vt.tile_h + ly + 4 * q;
        P[q].inside = x < cam.W && y < cam.H;
        P[q].pxc = (float)x + 0.5f;
        P[q].pyc = (float)y + 0.5f;
        P[q].T = 1.0f;
        P[q].C0 = P[q].C1 = P[q].C2 = 0.0f;
        P[q].last = P[q].evaluated = P[q].contributed = 0;
        P[q].done = !P[q].inside;
        all_done &= P[q].done;
    }
    const uint2 range = clamp_range(ranges[tile], st->m_clamped);
    const int n = (int)(range.y - range.x);
    for (int base = 0; base < n; base += batch) {
        if (__syncthreads_count(!all_done) == 0) break;
        const int cnt = min(batch, n - base), groups = (cnt + 31) >> 5;
        for (int g = (int)(threadIdx.x >> 5); g < groups; g += (int)(blockDim.x >> 5))
            stage_group<PPT, kPlain>(vt, tc, g, cnt, vals + range.x + base, R, rec0, rec1, rec2, sbuf, bits,
                                     words, nullptr, nullptr, !COUNT);
        __syncthreads();
        // this warp's entries in increasing order: the set bits of its words
        for (int g = 0; g < groups && !all_done; ++g) {
            for (uint32_t word = my_bits[g]; word != 0 && !all_done; word &= word - 1) {
                const int k = g * 32 + __ffs(word) - 1;
                const float4 a = sbuf[3 * k];
                const float4 b = sbuf[3 * k + 1];
                all_done = true;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    FwdPixel& p = P[q];
                    if (!p.done) {
                        const float power = support_power(a.z, a.w, b.x, a.x - p.pxc, a.y - p.pyc);
                        if (power >= kSupportPower) {  // also skips a NaN exponent
                            if (COUNT) ++p.evaluated;
                            const float alpha = fminf(kAlphaMax, b.y * __expf(power));
                            if (alpha >= kAlphaMin) {
                                const float Tn = p.T * (1.0f - alpha);
                                if (Tn < kTransmittanceMin) {
                                    p.done = true;
                                } else {
                                    const float4 c = sbuf[3 * k + 2];
                                    const float w = alpha * p.T;
                                    p.C0 += c.x * w;
                                    p.C1 += c.y * w;
                                    p.C2 += c.z * w;
                                    p.T = Tn;
                                    p.last = (uint32_t)(base + k + 1);
                                    if (COUNT) ++p.contributed;
                                }
                            }
                        }
                    }
                    all_done &= p.done;
                }
            }
        }
    }
    const int64_t hw = (int64_t)cam.W * cam.H;
    float* img = out_rgb + 3 * cam.pixel_base;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const FwdPixel& p = P[q];
        if (!p.inside) continue;
        const int64_t pi = (int64_t)(p.pyc - 0.5f) * cam.W + (int64_t)(p.pxc - 0.5f);
        img[pi] = p.C0 + p.T * bg0;
        img[hw + pi] = p.C1 + p.T * bg1;
        img[2 * hw + pi] = p.C2 + p.T * bg2;
        if (out_T) out_T[cam.pixel_base + pi] = p.T;
        pix_T[cam.pixel_base + pi] = p.T;
        pix_last[cam.pixel_base + pi] = p.last;
        if (COUNT) pix_count[cam.pixel_base + pi] = make_uint2(p.evaluated, p.contributed);
    }
    uint32_t my_last = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) my_last = max(my_last, P[q].last);
    write_backward_key(vt, tile, my_last);
}

// The forward with two pixels per thread in packed pairs: a lane's pixels share their
// column (rows r and r + 4 of its warp's 8x8 block), so the Gaussian's exponent, opacity
// product and transmittance update of both run as f32x2 instructions on the staged pairs,
// each half rounded exactly as the scalar pass rounds it; the decisions and the colour
// sums stay per pixel.
template <bool COUNT>
__device__ __forceinline__ void blend_pair_tile(const ViewTable& vt, const uint32_t tile,
                                                const uint2* __restrict__ ranges,
                                                const uint32_t* __restrict__ vals, uint32_t R,
                                                const float4* __restrict__ rec0,
                                                const float4* __restrict__ rec1,
                                                const float4* __restrict__ rec2, int batch,
                                                float bg0, float bg1, float bg2,
                                                float* __restrict__ out_rgb,
                                                float* __restrict__ out_T,
                                                float* __restrict__ pix_T,
                                                uint32_t* __restrict__ pix_last,
                                                uint2* __restrict__ pix_count,
                                                const DeviceStatus* __restrict__ st) {
    extern __shared__ float4 sbuf[];  // entries (qa qa, qb qb), (qc qc, o o), (px px, py py), rgb
    const int words = (batch + 31) >> 5;
    uint32_t* bits = reinterpret_cast<uint32_t*>(sbuf + stage_fields(kPairs) * batch);
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    const TileCoord tc = tile_of(vt, tile);
    const View& cam = vt.v[tc.v];
    const WarpBlock wb = warp_block<2>(vt);
    const int x = tc.tx * vt.tile_w + wb.x0 + (threadIdx.x & 7);
    const int y0 = tc.ty * vt.tile_h + wb.y0 + ((threadIdx.x >> 3) & 3), y1 = y0 + 4;
    const bool in0 = x < cam.W && y0 < cam.H, in1 = x < cam.W && y1 < cam.H;
    const f32x2 pcx = pk((float)x + 0.5f, (float)x + 0.5f), pcy = pk((float)y0 + 0.5f, (float)y1 + 0.5f);
    const f32x2 one = pk(1.0f, 1.0f);
    float T0 = 1.0f, T1 = 1.0f;
    float c00 = 0.0f, c01 = 0.0f, c02 = 0.0f, c10 = 0.0f, c11 = 0.0f, c12 = 0.0f;
    uint32_t last0 = 0, last1 = 0, ev0 = 0, ev1 = 0, ct0 = 0, ct1 = 0;
    bool done0 = !in0, done1 = !in1;
    bool all_done = done0 && done1;
    const uint2 range = clamp_range(ranges[tile], st->m_clamped);
    const int n = (int)(range.y - range.x);
    for (int base = 0; base < n; base += batch) {
        if (__syncthreads_count(!all_done) == 0) break;
        const int cnt = min(batch, n - base), groups = (cnt + 31) >> 5;
        for (int g = (int)(threadIdx.x >> 5); g < groups; g += (int)(blockDim.x >> 5))
            stage_group<2, kPairs>(vt, tc, g, cnt, vals + range.x + base, R, rec0, rec1, rec2, sbuf, bits,
                                   words, vt.masks ? vt.masks + range.x + base : nullptr, nullptr, !COUNT);
        __syncthreads();
        for (int g = 0; g < groups && !all_done; ++g) {
            for (uint32_t word = my_bits[g]; word != 0 && !all_done; word &= word - 1) {
                const int k = g * 32 + __ffs(word) - 1;
                const float4* e = sbuf + 4 * k;
                const ulonglong2 q = pairs(e), c = pairs(e + 1), pp = pairs(e + 2);
                // the exponent of support_power for both pixels
                const f32x2 dx = sub2(pp.x, pcx), dy = sub2(pp.y, pcy);
                const float2 pw = upk(fma2(dx, fma2(q.x, dx, mul2(q.y, dy)), mul2(mul2(c.x, dy), dy)));
                const float2 oG = upk(mul2(c.y, pk(__expf(pw.x), __expf(pw.y))));
                const float a0 = fminf(kAlphaMax, oG.x), a1 = fminf(kAlphaMax, oG.y);
                const bool s0 = !done0 && pw.x >= kSupportPower, s1 = !done1 && pw.y >= kSupportPower;
                const bool ok0 = s0 && a0 >= kAlphaMin, ok1 = s1 && a1 >= kAlphaMin;
                const f32x2 alpha = pk(a0, a1), T = pk(T0, T1);
                const float2 Tn = upk(mul2(T, sub2(one, alpha)));
                const float2 w = upk(mul2(alpha, T));
                const bool end0 = ok0 && Tn.x < kTransmittanceMin, end1 = ok1 && Tn.y < kTransmittanceMin;
                const bool add0 = ok0 && !end0, add1 = ok1 && !end1;
                if (COUNT) {
                    ev0 += s0;
                    ev1 += s1;
                    ct0 += add0;
                    ct1 += add1;
                }
                done0 |= end0;
                done1 |= end1;
                const float4 rgb = e[3];
                if (add0) {
                    c00 = fmaf(rgb.x, w.x, c00);
                    c01 = fmaf(rgb.y, w.x, c01);
                    c02 = fmaf(rgb.z, w.x, c02);
                    T0 = Tn.x;
                    last0 = (uint32_t)(base + k + 1);
                }
                if (add1) {
                    c10 = fmaf(rgb.x, w.y, c10);
                    c11 = fmaf(rgb.y, w.y, c11);
                    c12 = fmaf(rgb.z, w.y, c12);
                    T1 = Tn.y;
                    last1 = (uint32_t)(base + k + 1);
                }
                all_done = done0 && done1;
            }
        }
    }
    const int64_t hw = (int64_t)cam.W * cam.H;
    float* img = out_rgb + 3 * cam.pixel_base;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q ? in1 : in0)) continue;
        const int64_t pi = (int64_t)(q ? y1 : y0) * cam.W + x;
        const float T = q ? T1 : T0;
        img[pi] = (q ? c10 : c00) + T * bg0;
        img[hw + pi] = (q ? c11 : c01) + T * bg1;
        img[2 * hw + pi] = (q ? c12 : c02) + T * bg2;
        if (out_T) out_T[cam.pixel_base + pi] = T;
        pix_T[cam.pixel_base + pi] = T;
        pix_last[cam.pixel_base + pi] = q ? last1 : last0;
        if (COUNT) pix_count[cam.pixel_base + pi] = q ? make_uint2(ev1, ct1) : make_uint2(ev0, ct0);
    }
    write_backward_key(vt, tile, max(last0, last1));
}

// Tiles of a pass: the CTA's own (one CTA per tile, vt.order[blockIdx.x]) or, PERSIST,
// every tile whose slot in vt.order the CTA claims from *work (one atomic per tile, the
// slots in increasing order, i.e. the most expensive tiles first), until none is left.
// The grid of a persistent launch is the number of CTAs resident at once.
template <bool PERSIST, typename F>
__device__ __forceinline__ void for_each_tile(const ViewTable& vt, uint32_t* work, F&& body) {
    if (!PERSIST) {
        body(vt.order ? vt.order[blockIdx.x] : blockIdx.x);
        return;
    }
    __shared__ uint32_t s_slot;
    for (;;) {
        if (threadIdx.x == 0) s_slot = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t slot = s_slot;
        if ((int64_t)slot >= vt.num_tiles) break;  // uniform over the CTA
        body(vt.order ? vt.order[slot] : slot);
        __syncthreads();  // the claim word and the staging buffers are rewritten next
    }
}

template <bool COUNT, bool PERSIST>
__global__ void __launch_bounds__(512, 2) blend_pair_kernel(const ViewTable vt, const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ vals, uint32_t R,
                                                          const float4* __restrict__ rec0,
                                                          const float4* __restrict__ rec1,
                                                          const float4* __restrict__ rec2, int batch,
                                                          float bg0, float bg1, float bg2,
                                                          float* __restrict__ out_rgb,
                                                          float* __restrict__ out_T,
                                                          float* __restrict__ pix_T,
                                                          uint32_t* __restrict__ pix_last,
                                                          uint2* __restrict__ pix_count,
                                                          const DeviceStatus* __restrict__ st, uint32_t* work) {
    for_each_tile<PERSIST>(vt, work, [&](uint32_t tile) {
        blend_pair_tile<COUNT>(vt, tile, ranges, vals, R, rec0, rec1, rec2, batch, bg0, bg1, bg2, out_rgb, out_T,
                               pix_T, pix_last, pix_count, st);
    });
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// Sums 8 values over the warp with 9 shuffles (reduce-scatter): after halving steps at
// lane offsets 16, 8, 4 each lane holds one of the 8 values summed over 8 lanes, and two
// butterfly steps finish the sum.  Returns the total of value ((lane >> 2) & 7), complete
// in the lanes whose two low bits are 0.
__device__ __forceinline__ float warp_sum8(const float v[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = b4 ? v[4 + i] : v[i], send = b4 ? v[i] : v[4 + i];
        w[i] = keep + __shfl_xor_sync(kFullMask, send, 16);
    }
    float u[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b3 ? w[2 + i] : w[i], send = b3 ? w[i] : w[2 + i];
        u[i] = keep + __shfl_xor_sync(kFullMask, send, 8);
    }
    float x = (b2 ? u[1] : u[0]) + __shfl_xor_sync(kFullMask, b2 ? u[0] : u[1], 4);
    x += __shfl_xor_sync(kFullMask, x, 2);
    x += __shfl_xor_sync(kFullMask, x, 1);
    return x;
}

// Sums 9 values over the warp with 13 shuffles: the first 8 by the reduce-scatter of
// warp_sum8 and value 8 by butterflies over lane offsets 16, 8, 4; the two steps over
// offsets 2 and 1 carry both (the lanes with bit 1 clear value ((lane >> 2) & 7), the
// others value 8).  Returns in lanes with (lane & 3) == 0 the total of value
// ((lane >> 2) & 7), in lanes with (lane & 3) == 2 the total of value 8.
__device__ __forceinline__ float warp_sum9(const float v[9], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = b4 ? v[4 + i] : v[i], send = b4 ? v[i] : v[4 + i];
        w[i] = keep + __shfl_xor_sync(kFullMask, send, 16);
    }
    float u[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b3 ? w[2 + i] : w[i], send = b3 ? w[i] : w[2 + i];
        u[i] = keep + __shfl_xor_sync(kFullMask, send, 8);
    }
    const float x = (b2 ? u[1] : u[0]) + __shfl_xor_sync(kFullMask, b2 ? u[0] : u[1], 4);
    float e = v[8];
    e += __shfl_xor_sync(kFullMask, e, 16);
    e += __shfl_xor_sync(kFullMask, e, 8);
    e += __shfl_xor_sync(kFullMask, e, 4);
    float y = (b1 ? e : x) + __shfl_xor_sync(kFullMask, b1 ? x : e, 2);
    y += __shfl_xor_sync(kFullMask, y, 1);
    return y;
}

// *p += v in L2 (no return value).
__device__ __forceinline__ void red_add1(float* p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// grad += (a, b, c, d) as one 16-byte vector reduction in L2 (no return value).
__device__ __forceinline__ void red_add4(float4* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Per-pixel state of the reverse walk.
struct BwdPixel {
    float pxc, pyc;
    float T, g0, g1, g2, acc0, acc1, acc2;
    uint32_t last;
};

template <int PPT>
__global__ void __launch_bounds__(512) blend_backward_kernel(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, uint32_t R32,
    const float4* __restrict__ rec0, const float4* __restrict__ rec1, const float4* __restrict__ rec2,
    int batch, float bg0, float bg1, float bg2, const float* __restrict__ pix_T,
    const uint32_t* __restrict__ pix_last, const float* __restrict__ dL_drgb,
    float4* __restrict__ grad2d, int64_t R, const DeviceStatus* __restrict__ st) {
    extern __shared__ float4 sbuf[];
    const int words = (batch + 31) >> 5;
    uint32_t* sid = reinterpret_cast<uint32_t*>(sbuf + 3 * batch);
    uint32_t* bits = sid + batch;
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    __shared__ uint32_t s_max_last;
    const uint32_t tile = vt.order ? vt.order[blockIdx.x] : blockIdx.x;
    const TileCoord tc = tile_of(vt, tile);
    const View& cam = vt.v[tc.v];
    const WarpBlock wb = warp_block<PPT>(vt);
    const int lx = wb.x0 + (threadIdx.x & 7), ly = wb.y0 + ((threadIdx.x >> 3) & 3);
    const uint2 range = clamp_range(ranges[tile], st->m_clamped);
    if (threadIdx.x == 0) s_max_last = 0;
    __syncthreads();
    const int64_t hw = (int64_t)cam.W * cam.H;
    const float* gi = dL_drgb + 3 * cam.pixel_base;
    BwdPixel P[PPT];
    uint32_t my_last = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int x = tc.tx * vt.tile_w + lx, y = tc.ty * vt.tile_h + ly + 4 * q;
        BwdPixel& p = P[q];
        p.pxc = (float)x + 0.5f;
        p.pyc = (float)y + 0.5f;
        p.acc0 = bg0;
        p.acc1 = bg1;
        p.acc2 = bg2;
        p.T = 1.0f;
        p.g0 = p.g1 = p.g2 = 0.0f;
        p.last = 0;
        if (x < cam.W && y < cam.H) {
            const int64_t pi = (int64_t)y * cam.W + x;
            p.g0 = gi[pi];
            p.g1 = gi[hw + pi];
            p.g2 = gi[2 * hw + pi];
            p.T = pix_T[cam.pixel_base + pi];
            p.last = min(pix_last[cam.pixel_base + pi], range.y - range.x);
        }
        my_last = max(my_last, p.last);
    }
    const uint32_t wmax = __reduce_max_sync(kFullMask, my_last);
    if ((threadIdx.x & 31) == 0 && wmax) atomicMax(&s_max_last, wmax);
    __syncthreads();
    const int top = (int)s_max_last;
    const int lane = threadIdx.x & 31;
    const int warp_last = (int)wmax;  // no pixel of this warp blends an entry at or past it
    for (int hi = top; hi > 0; hi -= batch) {
        const int lo = max(0, hi - batch);
        __syncthreads();
        const int cnt = hi - lo, groups = (cnt + 31) >> 5;
        for (int g = (int)(threadIdx.x >> 5); g < groups; g += (int)(blockDim.x >> 5)) {
            const uint32_t id = stage_group<PPT, kPlain>(vt, tc, g, cnt, vals + range.x + lo, R32, rec0, rec1, rec2,
                                                         sbuf, bits, words, nullptr, nullptr);
            if (g * 32 + lane < cnt) sid[g * 32 + lane] = id;
        }
        __syncthreads();
        // this warp's entries below its last contributor, back to front
        const int lim = min(cnt, warp_last - lo);
        for (int g = ((lim + 31) >> 5) - 1; g >= 0; --g) {
            const int rem = lim - g * 32;
            for (uint32_t word = my_bits[g] & (rem >= 32 ? ~0u : (1u << rem) - 1u); word != 0;) {
                const int bit = 31 - __clz(word);
                word ^= 1u << bit;
                const int j = g * 32 + bit;
                const int k = lo + j;
                const float4 a = sbuf[3 * j];
                const float4 b = sbuf[3 * j + 1];
                const float4 c = sbuf[3 * j + 2];
                float d[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) d[i] = 0.0f;
                bool any = false;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    BwdPixel& p = P[q];
                    if ((uint32_t)k >= p.last) continue;
                    const float dx = a.x - p.pxc, dy = a.y - p.pyc;
                    const SupportTerms st = support_terms(a.z, a.w, b.x, dx, dy);
                    if (!(st.power >= kSupportPower)) continue;  // also skips a NaN exponent
                    const float G = __expf(st.power);
                    const float oG = b.y * G;
                    const float alpha = fminf(kAlphaMax, oG);
                    if (!(alpha >= kAlphaMin)) continue;
                    any = true;
                    p.T = __fdividef(p.T, 1.0f - alpha);
                    const float w = alpha * p.T;
                    d[6] = fmaf(p.g0, w, d[6]);
                    d[7] = fmaf(p.g1, w, d[7]);
                    d[8] = fmaf(p.g2, w, d[8]);
                    // colour behind minus this Gaussian's colour; acc += alpha (c - acc)
                    const float e0 = c.x - p.acc0, e1 = c.y - p.acc1, e2 = c.z - p.acc2;
                    const float dalpha = p.T * fmaf(p.g0, e0, fmaf(p.g1, e1, p.g2 * e2));
                    p.acc0 = fmaf(alpha, e0, p.acc0);
                    p.acc1 = fmaf(alpha, e1, p.acc1);
                    p.acc2 = fmaf(alpha, e2, p.acc2);
                    if (oG <= kAlphaMax) {
                        // wG = dL/dalpha G and its moments (the 2D gradient record's sums)
                        const float gG = dalpha * G;
                        const float gx = gG * dx, gy = gG * dy;
                        d[0] += gx;
                        d[1] += gy;
                        d[2] = fmaf(gx, dx, d[2]);
                        d[3] = fmaf(gx, dy, d[3]);
                        d[4] = fmaf(gy, dy, d[4]);
                        d[5] += gG;
                    }
                }
                if (__any_sync(kFullMask, any)) {
                    // lanes 0, 4, ..., 28 hold the sums of values 0..7; lanes 0 and 16 gather
                    // values 0-3 and 4-7 and add them with one 16-byte vector reduction each
                    const float s8 = warp_sum8(d, lane);
                    const float s9 = warp_sum(d[8]);
                    const float u1 = __shfl_down_sync(kFullMask, s8, 4);
                    const float u2 = __shfl_down_sync(kFullMask, s8, 8);
                    const float u3 = __shfl_down_sync(kFullMask, s8, 12);
                    const uint32_t id = sid[j];
                    if ((lane & 15) == 0) red_add4(grad2d + (lane >> 4) * R + id, s8, u1, u2, u3);
                    if (lane == 0) atomicAdd(reinterpret_cast<float*>(grad2d + 2 * R) + id, s9);
                }
            }
        }
    }
}

// The reverse walk with two pixels per thread in packed pairs (the pixel map of
// blend_pair_kernel).  The exponent, opacity product and gradient terms of both pixels run
// as f32x2 instructions, each half rounded exactly as the scalar pass rounds it, so every
// skip decision matches the forward.  The two pixels' transmittance and the dot products
// of their upstream gradients with the colour behind stay packed; a pixel that does not
// blend the Gaussian takes alpha 0, which leaves both unchanged and weights its terms
// zero.
__device__ __forceinline__ void blend_pair_backward_tile(
    const ViewTable& vt, const uint32_t tile, const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
    uint32_t R32, const float4* __restrict__ rec0, const float4* __restrict__ rec1, const float4* __restrict__ rec2,
    int batch, float bg0, float bg1, float bg2, const float* __restrict__ pix_T,
    const uint32_t* __restrict__ pix_last, const float* __restrict__ dL_drgb,
    float4* __restrict__ grad2d, int64_t R, const DeviceStatus* __restrict__ st) {
    // entries (qa qa, qb qb), (qc qc, o o), (px px, py py), (r r, g g), (b b, id 0)
    extern __shared__ float4 sbuf[];
    const int words = (batch + 31) >> 5;
    uint32_t* bits = reinterpret_cast<uint32_t*>(sbuf + stage_fields(kPairsColour) * batch);
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    __shared__ uint32_t s_max_last;
    const TileCoord tc = tile_of(vt, tile);
    const View& cam = vt.v[tc.v];
    const WarpBlock wb = warp_block<2>(vt);
    const int x = tc.tx * vt.tile_w + wb.x0 + (threadIdx.x & 7);
    const int y0 = tc.ty * vt.tile_h + wb.y0 + ((threadIdx.x >> 3) & 3), y1 = y0 + 4;
    const uint2 range = clamp_range(ranges[tile], st->m_clamped);
    if (threadIdx.x == 0) s_max_last = 0;
    __syncthreads();
    const int64_t hw = (int64_t)cam.W * cam.H;
    const float* gi = dL_drgb + 3 * cam.pixel_base;
    float g[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    float T[2] = {1.0f, 1.0f};  // the pixels' final transmittance, then packed into Tp
    uint32_t last[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int y = q ? y1 : y0;
        if (x < cam.W && y < cam.H) {
            const int64_t pi = (int64_t)y * cam.W + x;
            g[q][0] = gi[pi];
            g[q][1] = gi[hw + pi];
            g[q][2] = gi[2 * hw + pi];
            T[q] = pix_T[cam.pixel_base + pi];
            last[q] = min(pix_last[cam.pixel_base + pi], range.y - range.x);
        }
    }
    const f32x2 pcx = pk((float)x + 0.5f, (float)x + 0.5f), pcy = pk((float)y0 + 0.5f, (float)y1 + 0.5f);
    const f32x2 gr = pk(g[0][0], g[1][0]), gg = pk(g[0][1], g[1][1]), gb = pk(g[0][2], g[1][2]);
    const f32x2 one = pk(1.0f, 1.0f);
    f32x2 Tp = pk(T[0], T[1]);
    // the pixel's upstream gradient dotted with the colour behind (acc += alpha (rgb - acc),
    // from bg): one value per pixel carries what the three channels' accumulators would
    f32x2 gacc = fma2(gr, pk(bg0, bg0), fma2(gg, pk(bg1, bg1), mul2(gb, pk(bg2, bg2))));
    const uint32_t wmax = __reduce_max_sync(kFullMask, max(last[0], last[1]));
    if ((threadIdx.x & 31) == 0 && wmax) atomicMax(&s_max_last, wmax);
    __syncthreads();
    const int top = (int)s_max_last;
    const int lane = threadIdx.x & 31;
    // where this lane's total of warp_sum9 goes: value i < 8 (lane 4 i) to float 4 id + i of
    // the first 2D-gradient array (i < 4) or of the second, value 8 (lane 2) to the third
    const bool red_lane = (lane & 3) == 0 || lane == 2;
    float* const red_base = reinterpret_cast<float*>(grad2d) +
                            (lane == 2 ? 8 * R : (int64_t)((lane >> 4) & 1) * 4 * R + ((lane >> 2) & 3));
    const int red_step = lane == 2 ? 1 : 4;
    const int warp_last = (int)wmax;  // no pixel of this warp blends an entry at or past it
    for (int hi = top; hi > 0; hi -= batch) {
        const int lo = max(0, hi - batch);
        __syncthreads();
        const int cnt = hi - lo, groups = (cnt + 31) >> 5;
        for (int gr_ = (int)(threadIdx.x >> 5); gr_ < groups; gr_ += (int)(blockDim.x >> 5)) {
            stage_group<2, kPairsColour>(vt, tc, gr_, cnt, vals + range.x + lo, R32, rec0, rec1, rec2, sbuf,
                                         bits, words, nullptr, vt.masks ? vt.masks + range.x + lo : nullptr);
        }
        __syncthreads();
        if (lo > 0) prefetch_batch(vals + range.x + max(0, lo - batch), lo - max(0, lo - batch), R32, rec0, rec1, rec2);
        // this warp's entries below its last contributor, back to front
        const int lim = min(cnt, warp_last - lo);
        for (int grp = ((lim + 31) >> 5) - 1; grp >= 0; --grp) {
            const int rem = lim - grp * 32;
            for (uint32_t word = my_bits[grp] & (rem >= 32 ? ~0u : (1u << rem) - 1u); word != 0;) {
                const int bit = 31 - __clz(word);
                word ^= 1u << bit;
                const int j = grp * 32 + bit;
                const uint32_t k = (uint32_t)(lo + j);
                const float4* e = sbuf + 5 * j;
                const ulonglong2 q = pairs(e), c = pairs(e + 1), pp = pairs(e + 2);
                // support_terms for both pixels
                const f32x2 dx = sub2(pp.x, pcx), dy = sub2(pp.y, pcy);
                const f32x2 u = fma2(q.x, dx, mul2(q.y, dy)), t = mul2(c.x, dy);
                const float2 pw = upk(fma2(dx, u, mul2(t, dy)));
                const f32x2 G = pk(__expf(pw.x), __expf(pw.y));
                const float2 oG = upk(mul2(c.y, G));
                const float a0 = fminf(kAlphaMax, oG.x), a1 = fminf(kAlphaMax, oG.y);
                const bool use0 = k < last[0] && pw.x >= kSupportPower && a0 >= kAlphaMin;
                const bool use1 = k < last[1] && pw.y >= kSupportPower && a1 >= kAlphaMin;
                if (!__any_sync(kFullMask, use0 || use1)) continue;
                const f32x2 alpha = pk(use0 ? a0 : 0.0f, use1 ? a1 : 0.0f);
                // T before this Gaussian, T / (1 - alpha) as T times the hardware reciprocal
                // (the approximate division's own form); a pixel that does not blend it has
                // alpha 0, whose reciprocal of exactly 1 is exactly 1: its T stays as it is
                const float2 om = upk(sub2(one, alpha));
                Tp = mul2(Tp, pk(rcp_approx(om.x), rcp_approx(om.y)));
                const f32x2 w = mul2(alpha, Tp);
                // dL/dalpha = T g.(rgb - acc): the gradient's dot with this Gaussian's colour
                // minus its dot with the colour behind
                const ulonglong2 rg = pairs(e + 3), bb = pairs(e + 4);
                const f32x2 ge = sub2(fma2(gr, rg.x, fma2(gg, rg.y, mul2(gb, bb.x))), gacc);
                const f32x2 dalpha = mul2(Tp, ge);
                gacc = fma2(alpha, ge, gacc);  // alpha is 0 for a pixel that does not blend it
                // through alpha = o G only where the 0.99 clamp is not active: gG = dL/dalpha G
                // and its moments gG (dx, dy, dx^2, dx dy, dy^2), summed over the pixels; the
                // preprocess backward applies o and the conic once per record
                const float2 gGv = upk(mul2(dalpha, G));
                const f32x2 gG = pk(use0 && oG.x <= kAlphaMax ? gGv.x : 0.0f, use1 && oG.y <= kAlphaMax ? gGv.y : 0.0f);
                const f32x2 gx = mul2(gG, dx), gy = mul2(gG, dy);
                const float2 t0 = upk(gx), t1 = upk(gy);
                const float2 t2 = upk(mul2(gx, dx)), t3 = upk(mul2(gx, dy)), t4 = upk(mul2(gy, dy));
                const float2 t5 = upk(gG);
                const float2 t6 = upk(mul2(gr, w)), t7 = upk(mul2(gg, w)), t8 = upk(mul2(gb, w));
                float d[9];
                d[0] = t0.x + t0.y;
                d[1] = t1.x + t1.y;
                d[2] = t2.x + t2.y;
                d[3] = t3.x + t3.y;
                d[4] = t4.x + t4.y;
                d[5] = t5.x + t5.y;
                d[6] = t6.x + t6.y;
                d[7] = t7.x + t7.y;
                d[8] = t8.x + t8.y;
                // one reduction instruction: lanes 0, 4, ..., 28 add values 0..7, lane 2 value 8
                const float s = warp_sum9(d, lane);
                if (red_lane) red_add1(red_base + (size_t)(uint32_t)bb.y * red_step, s);
            }
        }
    }
}

template <bool PERSIST>
__global__ void __launch_bounds__(512, 2) blend_pair_backward_kernel(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, uint32_t R32,
    const float4* __restrict__ rec0, const float4* __restrict__ rec1, const float4* __restrict__ rec2,
    int batch, float bg0, float bg1, float bg2, const float* __restrict__ pix_T,
    const uint32_t* __restrict__ pix_last, const float* __restrict__ dL_drgb,
    float4* __restrict__ grad2d, int64_t R, const DeviceStatus* __restrict__ st, uint32_t* work) {
    for_each_tile<PERSIST>(vt, work, [&](uint32_t tile) {
        blend_pair_backward_tile(vt, tile, ranges, vals, R32, rec0, rec1, rec2, batch, bg0, bg1, bg2, pix_T,
                                 pix_last, dL_drgb, grad2d, R, st);
    });
}

__global__ void l1_zero_kernel(float* loss) { *loss = 0.0f; }

__global__ void __launch_bounds__(256) l1_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  int64_t count, float inv, float* loss, float* __restrict__ grad) {
    float acc = 0.0f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float e = img[j] - tgt[j];
        acc += fabsf(e);
        grad[j] = e > 0.0f ? inv : (e < 0.0f ? -inv : 0.0f);
    }
    acc = warp_sum(acc);
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        atomicAdd(loss, t * inv);
    }
}

}  // namespace

// Grid of a pass over the tiles: one CTA per tile, or (persistent) the CTAs that fit on
// the device at once, with the tile-claim counter cleared on the stream first.
template <typename K>
static cudaError_t tile_grid(K kernel, const ViewTable& vt, int threads, size_t smem, bool persistent,
                             unsigned* grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    *grid = (unsigned)vt.num_tiles;
    if (!persistent) return cudaSuccess;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
    const int64_t resident = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
    *grid = (unsigned)(resident < vt.num_tiles ? resident : vt.num_tiles);
    return cudaMemsetAsync(vt.work, 0, sizeof(uint32_t), s);
}

template <bool COUNT, bool PERSIST>
static cudaError_t blend_pair(const ViewTable& vt, const uint2* ranges, const uint32_t* vals, int64_t R,
                              const RecordPtrs& p, int batch, float bg0, float bg1, float bg2, float* out_rgb,
                              float* out_T, float* pix_T, uint32_t* pix_last, uint2* pix_count,
                              const DeviceStatus* st, cudaStream_t s) {
    const int threads = vt.tile_w * vt.tile_h / 2;
    const size_t smem =
        (size_t)batch * stage_fields(kPairs) * sizeof(float4) + (size_t)(threads / 32) * ((batch + 31) / 32) * 4;
    unsigned grid = 0;
    cudaError_t e = tile_grid(blend_pair_kernel<COUNT, PERSIST>, vt, threads, smem, PERSIST, &grid, s);
    if (e != cudaSuccess) return e;
    blend_pair_kernel<COUNT, PERSIST><<<grid, threads, smem, s>>>(vt, ranges, vals, (uint32_t)R, p.rec0, p.rec1,
                                                                  p.rec2, batch, bg0, bg1, bg2, out_rgb, out_T,
                                                                  pix_T, pix_last, pix_count, st, vt.work);
    return cudaGetLastError();
}

template <int PPT, bool COUNT>
static cudaError_t blend_ppt(const ViewTable& vt, const uint2* ranges, const uint32_t* vals, int64_t R,
                             const RecordPtrs& p, int batch, float bg0, float bg1, float bg2, float* out_rgb,
                             float* out_T, float* pix_T, uint32_t* pix_last, uint2* pix_count,
                             const DeviceStatus* st, cudaStream_t s) {
    const int threads = vt.tile_w * vt.tile_h / PPT;
    const size_t smem = (size_t)batch * 3 * sizeof(float4) + (size_t)(threads / 32) * ((batch + 31) / 32) * 4;
    cudaError_t e =
        cudaFuncSetAttribute(blend_kernel<PPT, COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // with no records every range is empty and no id is read; the kernel still writes bg
    blend_kernel<PPT, COUNT><<<(unsigned)vt.num_tiles, threads, smem, s>>>(vt, ranges, vals, (uint32_t)R, p.rec0, p.rec1,
                                                                    p.rec2, batch, bg0, bg1, bg2, out_rgb, out_T,
                                                                    pix_T, pix_last, pix_count, st);
    return cudaGetLastError();
}

template <int PPT>
static cudaError_t blend_backward_ppt(const ViewTable& vt, const uint2* ranges, const uint32_t* vals,
                                      const RecordPtrs& p, int batch, float bg0, float bg1, float bg2,
                                      const float* pix_T, const uint32_t* pix_last, const float* dL_drgb,
                                      float4* grad2d, int64_t R, const DeviceStatus* st, cudaStream_t s) {
    const int threads = vt.tile_w * vt.tile_h / PPT;
    const size_t smem =
        (size_t)batch * (3 * sizeof(float4) + sizeof(uint32_t)) + (size_t)(threads / 32) * ((batch + 31) / 32) * 4;
    cudaError_t e = cudaFuncSetAttribute(blend_backward_kernel<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    blend_backward_kernel<PPT><<<(unsigned)vt.num_tiles, threads, smem, s>>>(
        vt, ranges, vals, (uint32_t)R, p.rec0, p.rec1, p.rec2, batch, bg0, bg1, bg2, pix_T, pix_last, dL_drgb,
        grad2d, R, st);
    return cudaGetLastError();
}

cudaError_t launch_blend(const ViewTable& vt, const uint2* ranges, const uint32_t* vals,
                         int64_t R, const RecordPtrs& p, int batch, float bg0, float bg1, float bg2,
                         float* out_rgb, float* out_T, float* pix_T, uint32_t* pix_last,
                         uint2* pix_count, const DeviceStatus* st, cudaStream_t s) {
    if (vt.num_tiles == 0) return cudaSuccess;
#define SGS_BLEND(PPT, COUNT)                                                                                 \
    return blend_ppt<PPT, COUNT>(vt, ranges, vals, R, p, batch, bg0, bg1, bg2, out_rgb, out_T, pix_T, pix_last, \
                                 pix_count, st, s)
    if (vt.fwd_ppt == 2) {
#define SGS_PAIR(COUNT, PERSIST)                                                                                 \
    return blend_pair<COUNT, PERSIST>(vt, ranges, vals, R, p, batch, bg0, bg1, bg2, out_rgb, out_T, pix_T, pix_last, \
                                      pix_count, st, s)
        if (vt.count_pairs) {
            if (vt.persistent) SGS_PAIR(true, true);
            SGS_PAIR(true, false);
        }
        if (vt.persistent) SGS_PAIR(false, true);
        SGS_PAIR(false, false);
#undef SGS_PAIR
    }
    if (vt.count_pairs) SGS_BLEND(1, true);
    SGS_BLEND(1, false);
#undef SGS_BLEND
}

cudaError_t launch_blend_backward(const ViewTable& vt, const uint2* ranges, const uint32_t* vals,
                                  const RecordPtrs& p, int batch, float bg0, float bg1, float bg2,
                                  const float* pix_T, const uint32_t* pix_last,
                                  const float* dL_drgb, float4* grad2d, int64_t R,
                                  const DeviceStatus* st, cudaStream_t s) {
    if (vt.num_tiles == 0 || R == 0) return cudaSuccess;
    if (vt.bwd_ppt == 4)
        return blend_backward_ppt<4>(vt, ranges, vals, p, batch, bg0, bg1, bg2, pix_T, pix_last, dL_drgb, grad2d,
                                     R, st, s);
    if (vt.bwd_ppt == 2) {
        const int threads = vt.tile_w * vt.tile_h / 2;
        const size_t smem = (size_t)batch * stage_fields(kPairsColour) * sizeof(float4) +
                            (size_t)(threads / 32) * ((batch + 31) / 32) * 4;
        unsigned grid = 0;
        cudaError_t e = vt.persistent
                            ? tile_grid(blend_pair_backward_kernel<true>, vt, threads, smem, true, &grid, s)
                            : tile_grid(blend_pair_backward_kernel<false>, vt, threads, smem, false, &grid, s);
        if (e != cudaSuccess) return e;
        if (vt.persistent)
            blend_pair_backward_kernel<true><<<grid, threads, smem, s>>>(vt, ranges, vals, (uint32_t)R, p.rec0, p.rec1,
                                                                         p.rec2, batch, bg0, bg1, bg2, pix_T, pix_last,
                                                                         dL_drgb, grad2d, R, st, vt.work);
        else
            blend_pair_backward_kernel<false><<<grid, threads, smem, s>>>(vt, ranges, vals, (uint32_t)R, p.rec0,
                                                                          p.rec1, p.rec2, batch, bg0, bg1, bg2, pix_T,
                                                                          pix_last, dL_drgb, grad2d, R, st, vt.work);
        return cudaGetLastError();
    }
    return blend_backward_ppt<1>(vt, ranges, vals, p, batch, bg0, bg1, bg2, pix_T, pix_last, dL_drgb, grad2d, R,
                                 st, s);
}

cudaError_t launch_zero_grad2d(float4* grad2d, int64_t R, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    return cudaMemsetAsync(grad2d, 0, (size_t)R * (2 * sizeof(float4) + sizeof(float)), s);
}

cudaError_t launch_l1_loss(const float* img, const float* target, int64_t count, float scale, float* loss,
                           float* dL_dimg, cudaStream_t s) {
    l1_zero_kernel<<<1, 1, 0, s>>>(loss);
    if (count > 0) {
        const int64_t want = (count + 255) / 256;
        l1_kernel<<<(int)stride_grid(want, 8), 256, 0, s>>>(img, target, count, scale, loss, dL_dimg);
    }
    return cudaGetLastError();
}

}  // namespace sgs
