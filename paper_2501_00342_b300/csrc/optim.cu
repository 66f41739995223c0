// Training: fused Adam step over every parameter plane in one launch.
//
// The planes are cut into rows (mean x/y/z, the scale rows, ..., every SH coefficient's
// channel rows, the lobe rows); a row has n entries at stride `stride`.  Threads take four
// consecutive entries of one row (16-byte loads: strides are multiples of 4 and the planes
// 16-byte aligned), so the kernel streams raw, grad, m and v in and raw, act, m and v out:
// 32 bytes per entry, HBM-bound.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

constexpr int kMaxRows = 160;  // 3+3+4+1 + 48 (SH-3) + 4 x (3+3+1) lobe rows = 87

enum Act : int32_t { kIdentity = 0, kExp = 1, kSigmoid = 2 };

struct Row {
    float* raw;
    float* act;
    const float* grad;
    float* m;
    float* v;
    int32_t group;
    int32_t act_kind;
};

struct RowTable {
    int32_t rows;
    int64_t n;
    float lr[SGS_GROUP_COUNT];
    float c1[SGS_GROUP_COUNT];  // 1 / (1 - b1^t)
    float c2[SGS_GROUP_COUNT];  // 1 / (1 - b2^t)
    float beta1, beta2, eps;
    Row row[kMaxRows];
};

__device__ __forceinline__ float activate(float x, int kind) {
    if (kind == kExp) return expf(x);
    if (kind == kSigmoid) return 1.0f / (1.0f + expf(-x));
    return x;
}

// d act / d raw, from the activated value a
__device__ __forceinline__ float act_slope(float a, int kind) {
    if (kind == kExp) return a;
    if (kind == kSigmoid) return a * (1.0f - a);
    return 1.0f;
}

// Grid: blockIdx.y is the row (a block's row constants are uniform), blockIdx.x and the
// threads stride over the row's quads of four entries.
__global__ void __launch_bounds__(256) adam_kernel(const RowTable t) {
    const int64_t quads = (t.n + 3) / 4;
    const Row& w = t.row[blockIdx.y];
    const float lr = t.lr[w.group];
    if (lr == 0.0f) return;  // frozen group: nothing changes
    const float c1 = t.c1[w.group], c2 = t.c2[w.group];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = q * 4;
        // the stride is a multiple of 4: entries i0..i0+3 are inside the padded row
        float4 x = *reinterpret_cast<const float4*>(w.raw + i0);
        const float4 g4 = *reinterpret_cast<const float4*>(w.grad + i0);
        float4 m4 = *reinterpret_cast<const float4*>(w.m + i0);
        float4 v4 = *reinterpret_cast<const float4*>(w.v + i0);
        float* xs = &x.x;
        const float* gs = &g4.x;
        float* ms = &m4.x;
        float* vs = &v4.x;
        float a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k >= t.n) {  // padding of the last quad: left as it is
                a[k] = activate(xs[k], w.act_kind);
                continue;
            }
            const float g = gs[k] * act_slope(activate(xs[k], w.act_kind), w.act_kind);
            ms[k] = t.beta1 * ms[k] + (1.0f - t.beta1) * g;
            vs[k] = t.beta2 * vs[k] + (1.0f - t.beta2) * g * g;
            xs[k] -= lr * (ms[k] * c1) / (sqrtf(vs[k] * c2) + t.eps);
            a[k] = activate(xs[k], w.act_kind);
        }
        *reinterpret_cast<float4*>(w.raw + i0) = x;
        *reinterpret_cast<float4*>(w.m + i0) = m4;
        *reinterpret_cast<float4*>(w.v + i0) = v4;
        if (w.act != w.raw) *reinterpret_cast<float4*>(w.act + i0) = make_float4(a[0], a[1], a[2], a[3]);
    }
}

}  // namespace

cudaError_t launch_adam(const sgs_gaussians& layout, const sgs_grads& raw, const sgs_grads& act,
                        const sgs_grads& grad, const sgs_grads& m, const sgs_grads& v, const sgs_adam_config& cfg,
                        cudaStream_t s) {
    RowTable t;
    t.rows = 0;
    t.n = layout.n;
    t.beta1 = cfg.beta1;
    t.beta2 = cfg.beta2;
    t.eps = cfg.eps;
    for (int gi = 0; gi < SGS_GROUP_COUNT; ++gi) {
        t.lr[gi] = cfg.lr[gi];
        const double tt = cfg.step[gi] > 0 ? cfg.step[gi] : 1;
        t.c1[gi] = (float)(1.0 / (1.0 - std::pow((double)cfg.beta1, tt)));
        t.c2[gi] = (float)(1.0 / (1.0 - std::pow((double)cfg.beta2, tt)));
    }
    const int64_t S = layout.stride;
    auto add = [&](float* r, float* a, const float* g, float* mm, float* vv, int count, int group, int kind) {
        for (int k = 0; k < count; ++k) {
            Row& w = t.row[t.rows++];
            w.raw = r + k * S;
            w.act = a + k * S;
            w.grad = g + k * S;
            w.m = mm + k * S;
            w.v = vv + k * S;
            w.group = group;
            w.act_kind = kind;
        }
    };
    const int nsh = (layout.sh_degree + 1) * (layout.sh_degree + 1);
    const int K = layout.num_lobes;
    add(raw.mean, act.mean, grad.mean, m.mean, v.mean, 3, SGS_GROUP_MEAN, kIdentity);
    add(raw.scale, act.scale, grad.scale, m.scale, v.scale, 3, SGS_GROUP_SCALE, kExp);
    add(raw.rot, act.rot, grad.rot, m.rot, v.rot, 4, SGS_GROUP_ROT, kIdentity);
    add(raw.opacity, act.opacity, grad.opacity, m.opacity, v.opacity, 1, SGS_GROUP_OPACITY, kSigmoid);
    add(raw.sh, act.sh, grad.sh, m.sh, v.sh, 3, SGS_GROUP_SH_DC, kIdentity);
    if (nsh > 1)
        add(raw.sh + 3 * S, act.sh + 3 * S, grad.sh + 3 * S, m.sh + 3 * S, v.sh + 3 * S, 3 * (nsh - 1),
            SGS_GROUP_SH_REST, kIdentity);
    if (K > 0) {
        add(raw.sg_amp, act.sg_amp, grad.sg_amp, m.sg_amp, v.sg_amp, 3 * K, SGS_GROUP_SG, kIdentity);
        add(raw.sg_sharp, act.sg_sharp, grad.sg_sharp, m.sg_sharp, v.sg_sharp, K, SGS_GROUP_SG, kIdentity);
        const int axis_rows = layout.axis_mode == SGS_AXIS_FREE ? 3 * K : (layout.axis_mode == SGS_AXIS_ORTHO_FRAME ? 3 : 0);
        if (axis_rows)
            add(raw.sg_axis, act.sg_axis, grad.sg_axis, m.sg_axis, v.sg_axis, axis_rows, SGS_GROUP_SG, kIdentity);
    }
    if (layout.n == 0 || t.rows == 0) return cudaSuccess;
    // about 16 CTAs of 256 threads per SM over all rows together
    const int64_t quads = (layout.n + 3) / 4;
    const int64_t per_row = (quads + 255) / 256;
    const int64_t cap = (16 * (int64_t)sm_count() + t.rows - 1) / t.rows;
    const dim3 grid((unsigned)(per_row < cap ? per_row : (cap > 0 ? cap : 1)), (unsigned)t.rows);
    adam_kernel<<<grid, 256, 0, s>>>(t);
    return cudaGetLastError();
}

}  // namespace sgs
