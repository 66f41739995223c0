// Stages (b) and (d): exclusive scan of tiles touched, tile|depth key duplication, and
// per-tile range identification over the sorted keys.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

// ---- decoupled look-back helpers (64-bit words: 2-bit flag | 62-bit value) ----
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ void store_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long load_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void fill_u32_kernel(uint32_t* p, uint32_t value, size_t count) {
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (size_t)gridDim.x * blockDim.x)
        p[j] = value;
}

// Single-pass exclusive scan (chained scan with decoupled look-back).  Each CTA takes
// the next tile id from a counter, so every predecessor tile is already running.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out, int64_t R,
                                                             unsigned long long* lookback,
                                                             DeviceStatus* st, int64_t capacity) {
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->tile_counter[0], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    if (base + kScanItems <= R) {
        const uint4* p4 = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 w = __ldg(p4 + q);
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) v[q] = (base + q < R) ? in[base + q] : 0u;
    }
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) sum += v[q];
    // warp inclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            const unsigned long long c = s_warp[w];
            s_warp[w] = acc;
            acc += c;
        }
        // acc = tile aggregate; look back for the exclusive prefix of this tile
        unsigned long long prefix = 0;
        if (tile == 0) {
            store_relaxed(lookback, kFlagInc | acc);
        } else {
            store_relaxed(lookback + tile, kFlagAgg | acc);
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const unsigned long long e = load_relaxed(lookback + j);
                const unsigned long long f = e & ~kValueMask;
                if (f == kFlagInc) {
                    prefix += e & kValueMask;
                    break;
                } else if (f == kFlagAgg) {
                    prefix += e & kValueMask;
                    --j;
                } else if (++spins > kSpinLimit) {
                    set_status(st, SGS_ERR_TIMEOUT);
                    break;
                }
            }
            store_relaxed(lookback + tile, kFlagInc | (prefix + acc));
        }
        s_prefix = prefix;
        const int64_t num_tiles = (R + kScanTile - 1) / kScanTile;
        if ((int64_t)tile == num_tiles - 1) {
            const unsigned long long m = prefix + acc;
            st->m = m;
            // on overflow nothing downstream runs: no instance is written, sorted or blended
            st->m_clamped = (uint32_t)(m <= (unsigned long long)capacity ? m : 0ull);
            if (m > (unsigned long long)capacity) set_status(st, SGS_ERR_CAPACITY);
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + s_warp[warp] + inc - sum;
    uint32_t o[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        o[q] = (uint32_t)run;
        run += v[q];
    }
    if (base + kScanItems <= R) {
        uint4* p4 = reinterpret_cast<uint4*>(out + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q)
            p4[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (base + q < R) out[base + q] = o[q];
    }
}

// One thread per record: writes its tiles_touched instances, rectangle row-major, at
// offsets[r].  The pre-sort order is therefore (record, tile row-major).
__global__ void __launch_bounds__(256) duplicate_kernel(const ViewTable vt, const uint2* __restrict__ rect,
                                                         const uint32_t* __restrict__ tiles,
                                                         const float4* __restrict__ rec1,
                                                         const uint32_t* __restrict__ offsets,
                                                         int64_t n, int64_t R, const DeviceStatus* st,
                                                         int64_t capacity,
                                                         unsigned long long* __restrict__ keys,
                                                         uint32_t* __restrict__ vals) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const uint32_t cnt = tiles[r];
    if (cnt == 0) return;
    if (st->m > (unsigned long long)capacity) return;  // overflow: reported by the scan
    uint32_t o = offsets[r];
    const uint2 rc = rect[r];
    const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
    const int v = (int)((uint64_t)r / (uint64_t)n);
    const uint32_t tile_base = vt.v[v].tile_base;
    const int TW = vt.v[v].tiles_x;
    const unsigned long long zbits = (unsigned long long)__float_as_uint(rec1[r].z);
    for (int ty = y0; ty <= y1; ++ty)
        for (int tx = x0; tx <= x1; ++tx) {
            if ((int64_t)o >= capacity) return;  // only after a failed scan (status is set)
            const unsigned long long t = tile_base + (uint32_t)(ty * TW + tx);
            keys[o] = (t << 32) | zbits;
            vals[o] = (uint32_t)r;
            ++o;
        }
}

__global__ void __launch_bounds__(256) ranges_kernel(const unsigned long long* __restrict__ keys,
                                                      const DeviceStatus* st, uint32_t num_tiles,
                                                      uint2* __restrict__ ranges) {
    const uint32_t m = st->m_clamped;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[j] >> 32);
        if (t >= num_tiles) continue;  // only after a failed sort (status is set)
        if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[t].x = j;
        if (j == m - 1 || (uint32_t)(keys[j + 1] >> 32) != t) ranges[t].y = j + 1;
    }
}

}  // namespace

cudaError_t launch_fill_u32(uint32_t* p, uint32_t value, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int threads = 256;
    const size_t want = (count + threads - 1) / threads;
    const int blocks = (int)(want < 148 * 32 ? want : 148 * 32);
    fill_u32_kernel<<<blocks, threads, 0, s>>>(p, value, count);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* tiles, uint32_t* offsets, int64_t R,
                        unsigned long long* scan_lookback, DeviceStatus* st, int64_t capacity,
                        cudaStream_t s) {
    const int64_t num_tiles = (R + kScanTile - 1) / kScanTile;
    if (num_tiles == 0) return cudaSuccess;
    scan_kernel<<<(unsigned)num_tiles, kScanThreads, 0, s>>>(tiles, offsets, R, scan_lookback, st,
                                                             capacity);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const ViewTable& vt, const RecordPtrs& p, const uint32_t* offsets,
                             int64_t n, int64_t R, DeviceStatus* st, int64_t capacity,
                             unsigned long long* keys, uint32_t* vals, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    const int threads = 256;
    duplicate_kernel<<<(unsigned)((R + threads - 1) / threads), threads, 0, s>>>(
        vt, p.rect, p.tiles, p.rec1, offsets, n, R, st, capacity, keys, vals);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const unsigned long long* keys, const DeviceStatus* st, int64_t capacity,
                          int64_t num_tiles, uint2* ranges, cudaStream_t s) {
    if (capacity == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (capacity + threads - 1) / threads;
    const int blocks = (int)(want < 148 * 64 ? want : 148 * 64);
    ranges_kernel<<<blocks, threads, 0, s>>>(keys, st, (uint32_t)num_tiles, ranges);
    return cudaGetLastError();
}

}  // namespace sgs
