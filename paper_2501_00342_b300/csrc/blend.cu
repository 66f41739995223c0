// Stage (e): front-to-back alpha blending per pixel, and its reverse-mode pass.
//
// One CTA per (view, tile); the forward uses one pixel per thread, the backward two.  The
// tile's depth-sorted instance list
// [start, end) is staged batch_depth Gaussians at a time in shared memory (three float4
// records per Gaussian, gathered through the sorted record ids).  Per pixel centre p:
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy;  skip if power < -4.5 (outside 3 sigma)
//   alpha = min(0.99, opacity exp(power));      skip if alpha < 1/255
//   T' = T (1 - alpha);                          stop before this Gaussian if T' < 1e-4
//   C += rgb alpha T;  T = T'
// and the pixel is C + T bg.  A thread whose pixel is finished leaves the inner loop (its
// warp leaves when all 32 lanes have), and the CTA stops fetching batches once
// __syncthreads_count reports every pixel finished.
//
// The backward pass walks each tile's list from the last contributor to the front,
// rebuilding T_k = T_{k+1} / (1 - alpha_k) from the stored final transmittance and
// carrying the normalised colour behind (acc = acc (1 - alpha) + rgb alpha, starting at
// bg).  It recomputes power and alpha with the same operations as the forward pass, so
// every skip decision is identical; per Gaussian the warp's 9 gradient terms are summed
// with shuffles and added with one vector atomic per float4.
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

// The warp blocks of the CTA's tile that the Gaussian's support may reach: bit w for warp w.
// With Q(d) = A dx^2 + 2B dx dy + C dy^2 (the conic; records store (qa, qb, qc) =
// (-A/2, -B, -C/2)), the ellipse Q <= 9.01 is cut into the tile's bands of block rows.  Over
// a band's pixel-centre rows (padded by 1/64 pixel) its x-extent is exact: the rightmost
// x is the ellipse's rightmost point ex when that point's row -B ex / C falls in the band,
// else the larger chord end (-B y + sqrt(9.01 A - det y^2)) / A at the band's two edge rows
// (the chord end is concave in y), and the leftmost mirrors it.  Each block column whose
// padded pixel-centre columns meet the extent gets its bit.  A supported pixel centre has
// Q <= 9 up to single-precision rounding, which the 0.1 % slack and the pad cover (inside
// the Q <= 9 rows the chord's own rounding is far below that slack), so a warp without its
// bit has no supported pixel.  A degenerate conic or a non-finite centre sets every bit.
template <int PPT>
__device__ __forceinline__ uint32_t block_mask(const ViewTable& vt, const TileCoord& tc, float px, float py,
                                               float qa, float qb, float qc) {
    constexpr int BH = 4 * PPT;  // pixel rows per block
    const float A = -2.0f * qa, B = -qb, C = -2.0f * qc;
    const float det = A * C - B * B;
    // Centre relative to the tile's first pixel centre.
    const float gx = px - ((float)(tc.tx * vt.tile_w) + 0.5f);
    const float gy = py - ((float)(tc.ty * vt.tile_h) + 0.5f);
    if (!(det > 0.0f && A > 0.0f && C > 0.0f && fabsf(gx) < 1e30f && fabsf(gy) < 1e30f)) return ~0u;
    const int nbx = vt.tile_w >> 3, nby = vt.tile_h / BH;
    const float k = kSpanQ / det;
    const float ex = sqrtf(k * C), ey = sqrtf(k * A);
    const float dyr = -B * ex / C;  // row offset of the rightmost point
    const float iA = 1.0f / A, Ak = A * kSpanQ;
    const float b0 = fmaxf(ceilf((gy - ey - kSpanPad - (float)(BH - 1)) * (1.0f / BH)), 0.0f);
    const float b1 = fminf(floorf((gy + ey + kSpanPad) * (1.0f / BH)), (float)(nby - 1));
    uint32_t mask = 0;
    for (int b = (int)b0; b <= (int)b1; ++b) {
        const float u0 = fmaxf((float)(b * BH) - kSpanPad - gy, -ey);
        const float u1 = fminf((float)(b * BH + BH - 1) + kSpanPad - gy, ey);
        if (!(u0 <= u1)) continue;
        const float s0 = sqrtf(fmaxf(0.0f, Ak - det * u0 * u0));
        const float s1 = sqrtf(fmaxf(0.0f, Ak - det * u1 * u1));
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

// Stages one group of 32 batch entries (this warp's group g: entries 32 g + lane < cnt,
// from the tile's sorted list at `first`) in shared memory, and writes for every warp w of
// the CTA the 32-bit word of the group's entries whose support may reach w's block
// (bits[w * words + g]; bit b = entry 32 g + b): a transpose of the entries' block masks by
// one ballot per warp.  Returns the record id of the lane's entry.  Warp-collective.
template <int PPT>
__device__ __forceinline__ uint32_t stage_group(const ViewTable& vt, const TileCoord& tc, int g, int cnt,
                                                const uint32_t* __restrict__ first, uint32_t R,
                                                const float4* __restrict__ rec0, const float4* __restrict__ rec1,
                                                const float4* __restrict__ rec2, float4* s0, float4* s1,
                                                float4* s2, uint32_t* bits, int words) {
    const int lane = threadIdx.x & 31, j = g * 32 + lane;
    uint32_t mask = 0, id = 0;
    if (j < cnt) {
        id = min(first[j], R - 1);  // ids are < R by construction
        const float4 r0 = rec0[id], r1 = rec1[id];
        s0[j] = r0;
        s1[j] = r1;
        s2[j] = rec2[id];
        mask = block_mask<PPT>(vt, tc, r0.x, r0.y, r0.z, r0.w, r1.x);
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

// Tile range clipped to the instances actually written (all of them unless overflowed).
__device__ __forceinline__ uint2 clamp_range(uint2 r, uint32_t m) {
    r.y = min(r.y, m);
    r.x = min(r.x, r.y);
    return r;
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
    float4* s0 = sbuf;
    float4* s1 = sbuf + batch;
    float4* s2 = sbuf + 2 * batch;
    const int words = (batch + 31) >> 5;
    uint32_t* bits = reinterpret_cast<uint32_t*>(sbuf + 3 * batch);
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    const TileCoord tc = tile_of(vt, blockIdx.x);
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
    const uint2 range = clamp_range(ranges[blockIdx.x], st->m_clamped);
    const int n = (int)(range.y - range.x);
    for (int base = 0; base < n; base += batch) {
        if (__syncthreads_count(!all_done) == 0) break;
        const int cnt = min(batch, n - base), groups = (cnt + 31) >> 5;
        for (int g = (int)(threadIdx.x >> 5); g < groups; g += (int)(blockDim.x >> 5))
            stage_group<PPT>(vt, tc, g, cnt, vals + range.x + base, R, rec0, rec1, rec2, s0, s1, s2, bits, words);
        __syncthreads();
        // this warp's entries in increasing order: the set bits of its words
        for (int g = 0; g < groups && !all_done; ++g) {
            for (uint32_t word = my_bits[g]; word != 0 && !all_done; word &= word - 1) {
                const int k = g * 32 + __ffs(word) - 1;
                const float4 a = s0[k];
                const float4 b = s1[k];
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
                                    const float4 c = s2[k];
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
    float4* s0 = sbuf;
    float4* s1 = sbuf + batch;
    float4* s2 = sbuf + 2 * batch;
    const int words = (batch + 31) >> 5;
    uint32_t* sid = reinterpret_cast<uint32_t*>(sbuf + 3 * batch);
    uint32_t* bits = sid + batch;
    const uint32_t* my_bits = bits + (threadIdx.x >> 5) * words;
    __shared__ uint32_t s_max_last;
    const TileCoord tc = tile_of(vt, blockIdx.x);
    const View& cam = vt.v[tc.v];
    const WarpBlock wb = warp_block<PPT>(vt);
    const int lx = wb.x0 + (threadIdx.x & 7), ly = wb.y0 + ((threadIdx.x >> 3) & 3);
    const uint2 range = clamp_range(ranges[blockIdx.x], st->m_clamped);
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
            const uint32_t id =
                stage_group<PPT>(vt, tc, g, cnt, vals + range.x + lo, R32, rec0, rec1, rec2, s0, s1, s2, bits, words);
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
                const float4 a = s0[j];
                const float4 b = s1[j];
                const float4 c = s2[j];
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
                        // power = qa dx^2 + qb dx dy + qc dy^2, (qa, qb, qc) = (-A/2, -B, -C/2):
                        // d/d px = u + qa dx, d/d py = qb dx + 2 qc dy, d/d(qa, qb, qc) = (dx^2, dx dy, dy^2)
                        const float gG = dalpha * G;
                        const float gpow = gG * b.y;
                        d[0] = fmaf(gpow, fmaf(a.z, dx, st.u), d[0]);
                        d[1] = fmaf(gpow, fmaf(a.w, dx, st.t + st.t), d[1]);
                        const float h = -0.5f * gpow;
                        d[2] = fmaf(h * dx, dx, d[2]);
                        d[3] = fmaf(-gpow * dx, dy, d[3]);
                        d[4] = fmaf(h * dy, dy, d[4]);
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
                    if (lane == 0) atomicAdd(reinterpret_cast<float*>(grad2d + 2 * R + id), s9);
                }
            }
        }
    }
}

__global__ void l1_zero_kernel(float* loss) { *loss = 0.0f; }

__global__ void __launch_bounds__(256) l1_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  int64_t count, float* loss, float* __restrict__ grad) {
    const float inv = 1.0f / (float)count;
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
        if (vt.count_pairs) SGS_BLEND(2, true);
        SGS_BLEND(2, false);
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
    if (vt.bwd_ppt == 2)
        return blend_backward_ppt<2>(vt, ranges, vals, p, batch, bg0, bg1, bg2, pix_T, pix_last, dL_drgb, grad2d,
                                     R, st, s);
    return blend_backward_ppt<1>(vt, ranges, vals, p, batch, bg0, bg1, bg2, pix_T, pix_last, dL_drgb, grad2d, R,
                                 st, s);
}

cudaError_t launch_zero_grad2d(float4* grad2d, const uint32_t* tiles, int64_t R, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    // one plain clear of all three planes streams at full write bandwidth; skipping the
    // culled records saves little and costs a dependent load per record
    (void)tiles;
    return cudaMemsetAsync(grad2d, 0, (size_t)R * 3 * sizeof(float4), s);
}

cudaError_t launch_l1_loss(const float* img, const float* target, int64_t count, float* loss,
                           float* dL_dimg, cudaStream_t s) {
    l1_zero_kernel<<<1, 1, 0, s>>>(loss);
    if (count > 0) {
        const int64_t want = (count + 255) / 256;
        l1_kernel<<<(int)(want < 148 * 8 ? want : 148 * 8), 256, 0, s>>>(img, target, count, loss, dL_dimg);
    }
    return cudaGetLastError();
}

}  // namespace sgs
