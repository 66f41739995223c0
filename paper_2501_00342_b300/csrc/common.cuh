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
    int64_t pixel_base;
};

struct ViewTable {
    int32_t B;
    int32_t tile_w, tile_h;
    int32_t pad;
    int64_t num_tiles;
    View v[SGS_MAX_VIEWS];
};

// Device status word layout (first 256 bytes of the workspace).
struct DeviceStatus {
    int32_t status;        // OR of sgs_status bits
    uint32_t m_clamped;    // min(M, capacity): instances actually written
    unsigned long long m;  // exact instance count M
    uint32_t tile_counter[16];  // dynamic tile ids: [0] scan, [1..] sort passes
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

// Support exponent of a Gaussian at a pixel centre, in the fixed order
//   power = fma(dx, fma(qa, dx, qb*dy), (qc*dy)*dy),  dx = px - cx_pix, dy = py - cy_pix,
// with (qa, qb, qc) = (-A/2, -B, -C/2) the scaled conic.  Forward and backward kernels
// use this one function, so they take identical skip decisions.
__device__ __forceinline__ float support_power(float qa, float qb, float qc, float dx, float dy) {
    const float u = __fmaf_rn(qa, dx, __fmul_rn(qb, dy));
    const float w = __fmul_rn(__fmul_rn(qc, dy), dy);
    return __fmaf_rn(dx, u, w);
}

constexpr float kSupportPower = -4.5f;     // Mahalanobis distance 3
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTransmittanceMin = 1e-4f;

}  // namespace sgs
