// Measurement helper: the FP32 arithmetic throughput of the device, the denominator of
// the blend kernels' roofline (they are bound by the FP32 pipes and issue slots, not by
// memory).  Each thread runs kChains independent multiply-add chains x <- x * a + b for
// `iters` steps, either as scalar fma.rn.f32 or as packed fma.rn.f32x2 (two lanes of
// work per instruction); the caller times the launch with CUDA events.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;

__device__ __forceinline__ unsigned long long fma2_packed(unsigned long long x, unsigned long long a,
                                                         unsigned long long b) {
    unsigned long long r;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float fma1(float x, float a, float b) {
    float r;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(x), "f"(a), "f"(b));
    return r;
}

// a < 1 and b small keep every chain finite and away from subnormals
template <bool PAIRS>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(int iters, float a, float b, float* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    if constexpr (PAIRS) {
        const unsigned long long A = pack2(a, a), Bv = pack2(b, b);
        unsigned long long x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = pack2(1e-3f * (float)(t & 1023) + c, 0.5f + c);
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma2_packed(x[c], A, Bv);
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
            acc += lo + hi;
        }
    } else {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(t & 1023) + c;
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma1(x[c], a, b);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    }
    out[t] = acc;
}

}  // namespace
}  // namespace sgs

extern "C" sgs_status sgs_alu_probe_size(int64_t* threads) {
    if (!threads) return SGS_ERR_INVALID;
    *threads = (int64_t)sgs::sm_count() * sgs::kProbeBlocksPerSM * sgs::kProbeThreads;
    return SGS_OK;
}

extern "C" sgs_status sgs_alu_probe(int32_t packed, int32_t iters, float* out, double* fp32_ops,
                                    cudaStream_t stream) {
    if (iters < 1 || !out || !fp32_ops || (packed != 0 && packed != 1)) return SGS_ERR_INVALID;
    const int blocks = sgs::sm_count() * sgs::kProbeBlocksPerSM;
    const double threads = (double)blocks * sgs::kProbeThreads;
    *fp32_ops = threads * (double)iters * sgs::kChains * (packed ? 2.0 : 1.0);
    if (packed)
        sgs::alu_probe_kernel<true><<<blocks, sgs::kProbeThreads, 0, stream>>>(iters, 0.999999f, 1e-6f, out);
    else
        sgs::alu_probe_kernel<false><<<blocks, sgs::kProbeThreads, 0, stream>>>(iters, 0.999999f, 1e-6f, out);
    return cudaGetLastError() == cudaSuccess ? SGS_OK : SGS_ERR_CUDA;
}
