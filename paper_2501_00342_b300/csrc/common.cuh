// Device-side definitions shared by the SG-Splatting kernels (sm_103a).
#pragma once
#include <cstdint>

#include "sgs.h"

namespace sgs {

constexpr uint32_t kFullMask = 0xffffffffu;
// Upper bound on the polls of any device-side spin (decoupled look-back).  A wait that
// reaches it sets SGS_ERR_TIMEOUT in the status word and gives up instead of hanging.
constexpr uint32_t kSpinLimit = 1u << 22;

// Per-view constants, passed by value as a kernel parameter (constant bank).
struct View {
    float V[12];
    float campos[3];
    float fx, fy, cx, cy;
    int32_t W, H;
    float near_plane;
    int32_t tiles_x, tiles_y;
    uint32_t tile_base;
    // 1.3 x the half field of view on x/z and y/z: 1.3 * ((0.5 * W) / fx), correctly
    // rounded single precision in that order (computed on the host)
    float limx, limy;
    int64_t pixel_base;
};

struct ViewTable {
    int32_t B;
    int32_t tile_w, tile_h;    // powers of two
    float inv_tile_w, inv_tile_h;  // exact reciprocals: x * inv == x / tile, bit for bit
    int32_t fwd_ppt, bwd_ppt;      // pixels per thread of the blend kernels
    int32_t count_pairs;           // the forward blend writes per-pixel pair counts
    int64_t num_tiles;
    const uint32_t* order;         // the blend's tile order (CTA b renders tile order[b]), or null
    uint32_t* tile_top;            // the forward's per-tile last-contributor position (or null)
    uint16_t* masks;               // per instance, the warp blocks its support may reach: the
                                   // two-pixel forward stores them, the two-pixel backward reads
                                   // them (null: computed)
    int32_t persistent;            // the two-pixel blend passes run as persistent kernels
    uint32_t* work;                // their tile-claim counter (cleared before each launch)
    View v[SGS_MAX_VIEWS];
};

// Device status word layout (first 256 bytes of the workspace).
struct DeviceStatus {
    int32_t status;        // OR of sgs_status bits
    uint32_t m_clamped;    // min(M, capacity): instances actually written
    unsigned long long m;  // exact instance count M
    uint32_t tile_counter[16];  // dynamic tile ids: [0] scan, [1..] sort passes
    uint32_t num_records;       // R, the length of the record sort
    uint32_t num_visible;       // records with instances: the record sort keeps only these
    uint32_t work[2];           // tile slots claimed by the persistent forward / backward blend
};

// Correctly rounded single-precision operations that the compiler may not fuse or
// reorder: the integer-deciding part of the preprocess is written with these only.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }

__device__ __forceinline__ void set_status(DeviceStatus* st, int32_t bits) {
    atomicOr(&st->status, bits);
}

// ---- decoupled look-back slots: 64-bit words, a tag in the high bits and a count below ----
// Asks L2 to fetch [p, p + bytes) from DRAM (a hint: nothing waits for it).  p and bytes
// must be multiples of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void slot_store(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long slot_load(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of a chained scan by decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016).  Walks the slots
// slot[j * stride], j = first, first - 1, ..., 0: a slot tagged `agg` (the tile's own
// count) is added and the walk goes on, a slot tagged `inc` (the tile's inclusive prefix)
// is added and ends it, any other tag means the tile has not published yet and the slot is
// polled again.  The slots are read kLookbackWindow at a time (independent loads, one
// round trip per window).  After `limit` polls that met an unpublished slot, SGS_ERR_TIMEOUT
// is set in the status word and the partial sum is returned: the wait never hangs, the
// result is then invalid.
constexpr int kLookbackWindow = 4;
__device__ __forceinline__ unsigned long long lookback_sum(const unsigned long long* slot, int64_t first,
                                                           size_t stride, unsigned long long value_mask,
                                                           unsigned long long tag_agg,
                                                           unsigned long long tag_inc, DeviceStatus* st,
                                                           uint32_t limit = kSpinLimit) {
    unsigned long long acc = 0;
    uint32_t spins = 0;
    int64_t j = first;
    while (j >= 0) {
        unsigned long long e[kLookbackWindow];
#pragma unroll
        for (int w = 0; w < kLookbackWindow; ++w)  // before slot 0: an inclusive prefix of 0
            e[w] = j - w >= 0 ? slot_load(slot + (size_t)(j - w) * stride) : tag_inc;
        int w = 0;
        bool done = false;
#pragma unroll
        for (; w < kLookbackWindow; ++w) {
            const unsigned long long tag = e[w] & ~value_mask;
            if (tag != tag_inc && tag != tag_agg) break;  // not published yet: poll it again
            acc += e[w] & value_mask;
            if (tag == tag_inc) {
                done = true;
                break;
            }
        }
        if (done) break;
        j -= w;
        if (w < kLookbackWindow && ++spins > limit) {
            set_status(st, SGS_ERR_TIMEOUT);
            break;
        }
    }
    return acc;
}

// Support exponent of a Gaussian at a pixel centre, in the fixed order
//   power = fma(dx, fma(qa, dx, qb*dy), (qc*dy)*dy),  dx = px - cx_pix, dy = py - cy_pix,
// with (qa, qb, qc) = (-A/2, -B, -C/2) the scaled conic.  Forward and backward kernels
// use this one function, so they take identical skip decisions.
__device__ __forceinline__ float support_power(float qa, float qb, float qc, float dx, float dy) {
    const float u = __fmaf_rn(qa, dx, __fmul_rn(qb, dy));
    const float w = __fmul_rn(__fmul_rn(qc, dy), dy);
    return __fmaf_rn(dx, u, w);
}

// The same exponent with its intermediates u = qa dx + qb dy and t = qc dy kept for the
// backward pass (d power/d dx = u + qa dx, d power/d dy = qb dx + 2 t).
struct SupportTerms {
    float power, u, t;
};
__device__ __forceinline__ SupportTerms support_terms(float qa, float qb, float qc, float dx, float dy) {
    SupportTerms s;
    s.u = __fmaf_rn(qa, dx, __fmul_rn(qb, dy));
    s.t = __fmul_rn(qc, dy);
    s.power = __fmaf_rn(dx, s.u, __fmul_rn(s.t, dy));
    return s;
}

// Tiles the Gaussian's 3-sigma ellipse reaches, row by row.  E = {d : Q(d) <= k} with
// Q(d) = A dx^2 + 2 B dx dy + C dy^2 (the conic), k = 9.01: the support is Q <= 9, and the
// 0.1 % slack plus a 1/64-pixel pad cover rounding, so no tile holding a supported pixel
// centre is dropped.  In a tile row, the band of pixel-centre rows [ly, hy] cuts E in a
// convex set whose x-extent is bounded by the ellipse's rightmost point
// (dx = sqrt(kC/det), dy = -B sqrt(k/(det C)), det = AC - B^2) when that lies in the band,
// else by dx_hi(dy) = (-B dy + sqrt(A k - det dy^2)) / A at the band ends (and
// symmetrically for the left end).  The row keeps the tiles holding a pixel-centre column
// inside that extent.  One fixed order of correctly rounded operations: the count in
// preprocess and the keys in duplicate agree exactly.
constexpr int kSpanRows = 15;                // rows kept in a record's packed table
constexpr uint32_t kSpanRowsShort = 7;       // rows whose table fits its first 32 bytes
static_assert(1 + kSpanRows == 16, "a row table is a header word and kSpanRows rows in 64 bytes");
static_assert(1 + kSpanRowsShort == 8, "a short table is a header word and its rows in 32 bytes");
constexpr uint32_t kSpanRowsOverflow = 0xffffu;
constexpr float kSpanQ = 9.01f;
constexpr float kSpanPad = 0.015625f;

struct RowSpans {
    int ty0, ty1;  // rows to visit
    float ex, ey, dyr, det, invA, Ak;
    bool ok;
};

__device__ __forceinline__ RowSpans row_setup(float px, float py, float A, float B, float C, float inv_th,
                                              int TH) {
    RowSpans r;
    r.ok = false;
    r.ty0 = 0;
    r.ty1 = -1;
    r.det = sub_rn(mul_rn(A, C), mul_rn(B, B));
    if (!(r.det > 0.0f)) return r;
    r.ex = sqrt_rn(div_rn(mul_rn(kSpanQ, C), r.det));
    r.ey = sqrt_rn(div_rn(mul_rn(kSpanQ, A), r.det));
    r.dyr = -mul_rn(B, sqrt_rn(div_rn(kSpanQ, mul_rn(r.det, C))));
    r.invA = div_rn(1.0f, A);
    r.Ak = mul_rn(A, kSpanQ);
    const float t0 = sub_rn(sub_rn(sub_rn(py, r.ey), kSpanPad), 0.5f);
    const float t1 = sub_rn(add_rn(add_rn(py, r.ey), kSpanPad), 0.5f);
    const float y0 = ceilf(t0), y1 = floorf(t1);  // pixel rows with centres in the extent
    if (!(y0 <= y1)) return r;
    const float f0 = fmaxf(floorf(mul_rn(y0, inv_th)), 0.0f);
    const float f1 = fminf(floorf(mul_rn(y1, inv_th)), (float)(TH - 1));
    if (!(f0 <= f1)) return r;
    r.ty0 = (int)f0;
    r.ty1 = (int)f1;
    r.ok = true;
    return r;
}

// Tile columns [tx0, tx1] of row ty (false: none).
__device__ __forceinline__ bool row_span(const RowSpans& r, float px, float py, float B, int ty, float inv_tw,
                                         int th, int TW, int& tx0, int& tx1) {
    const float ly = add_rn((float)(ty * th), 0.5f), hy = sub_rn((float)(ty * th + th), 0.5f);
    const float eyp = add_rn(r.ey, kSpanPad);
    const float u0 = fmaxf(sub_rn(ly, py), -eyp);
    const float u1 = fminf(sub_rn(hy, py), eyp);
    if (!(u0 <= u1)) return false;
    const float s0 = sqrt_rn(fmaxf(0.0f, sub_rn(r.Ak, mul_rn(mul_rn(r.det, u0), u0))));
    const float s1 = sqrt_rn(fmaxf(0.0f, sub_rn(r.Ak, mul_rn(mul_rn(r.det, u1), u1))));
    const float b0 = mul_rn(B, u0), b1 = mul_rn(B, u1);
    const float hi0 = mul_rn(sub_rn(s0, b0), r.invA), hi1 = mul_rn(sub_rn(s1, b1), r.invA);
    const float lo0 = mul_rn(-add_rn(b0, s0), r.invA), lo1 = mul_rn(-add_rn(b1, s1), r.invA);
    const float xmax = (u0 <= r.dyr && r.dyr <= u1) ? r.ex : fmaxf(hi0, hi1);
    const float xmin = (u0 <= -r.dyr && -r.dyr <= u1) ? -r.ex : fminf(lo0, lo1);
    const float xs0 = sub_rn(add_rn(px, xmin), kSpanPad);
    const float xs1 = add_rn(add_rn(px, xmax), kSpanPad);
    const float x0 = ceilf(sub_rn(xs0, 0.5f)), x1 = floorf(sub_rn(xs1, 0.5f));
    if (!(x0 <= x1)) return false;
    const float f0 = fmaxf(floorf(mul_rn(x0, inv_tw)), 0.0f);
    const float f1 = fminf(floorf(mul_rn(x1, inv_tw)), (float)(TW - 1));
    if (!(f0 <= f1)) return false;
    tx0 = (int)f0;
    tx1 = (int)f1;
    return true;
}

// Asynchronous global -> shared copies of 4 or 16 bytes (16: both addresses 16-byte
// aligned), committed as one group per async_commit; async_wait<N> waits until at most N
// of the thread's groups are still in flight.
__device__ __forceinline__ void async_copy4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void async_copy16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Per-record flags the preprocess leaves for its backward pass: the record's discrete
// decisions, so that the backward takes each branch the forward took without recomputing
// (bit for bit) the values that decided it.  Bits 0-2: colour channel c clamped at 0;
// bit 3 / 4: x/z / y/z clamped to the frustum limit; bits 5-6: the SH degree D the colour
// summed; bit 7: the record has instances.  0 for a culled record.
constexpr uint32_t kFlagClampX = 1u << 3;
constexpr uint32_t kFlagClampY = 1u << 4;
constexpr int kFlagShift = 5;
constexpr uint32_t kFlagVisible = 1u << 7;

constexpr float kSupportPower = -4.5f;     // Mahalanobis distance 3
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTransmittanceMin = 1e-4f;

}  // namespace sgs
