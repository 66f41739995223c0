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

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Digit counts of the passes whose digit reaches into the tile bits, for the key of tile t
// (row of tiles [row_t0, row_end)).  Along a row the tile ids are consecutive, so such a
// digit is constant on segments of 2^s tiles (s = the pass's first bit minus 32, or 0 if
// the digit also holds depth bits): the key that opens a segment adds the segment length.
template <int RB>
__device__ __forceinline__ void count_tile_digits(uint32_t* h, int passes, unsigned long long key, uint32_t t,
                                                  uint32_t row_t0, uint32_t row_end) {
    constexpr int RADIX = 1 << RB;
    constexpr int MAXP = (64 + RB - 1) / RB;
    // pass 32 / RB is the first whose digit reaches past bit 31
#pragma unroll
    for (int p = 32 / RB; p < MAXP; ++p) {
        if (p >= passes) break;
        const int lo = p * RB;
        const int sh = lo > 32 ? lo - 32 : 0;
        const uint32_t mask = (1u << sh) - 1u;
        if (sh > 0 && t != row_t0 && (t & mask) != 0u) continue;  // not the first key of its segment
        const uint32_t seg_end = sh > 0 ? min(row_end, ((t >> sh) + 1u) << sh) : t + 1u;
        const uint32_t d = (uint32_t)(key >> lo) & (RADIX - 1);
        atomicAdd(&h[p * RADIX + d], seg_end - t);
    }
}

// One warp per group of 32 consecutive records.  Their instances occupy one contiguous
// output range (the scan's offsets are consecutive), so the warp fills it 32 slots at a
// time: for slot e a 5-step shuffle search finds the record (inclusive scan of the counts);
// the record's packed row table (written by preprocess: first column and tiles-before per
// row) gives the row by a branch-free count, and consecutive lanes write consecutive slots.
// A record whose table overflowed is filled afterwards by the whole warp, recomputing its
// rows with row_span.  The pre-sort order is (record, tile row-major).
// The radix sort's digit histograms are counted here too: digits wholly inside the depth
// bits are the same for all of a record's keys and are counted once per record (weighted by
// its count); the others per segment of consecutive tiles (count_tile_digits).
template <int RB>
__global__ void __launch_bounds__(256) duplicate_kernel(const ViewTable vt, const uint4* __restrict__ spans,
                                                         const uint32_t* __restrict__ tiles,
                                                         const float4* __restrict__ rec0,
                                                         const float4* __restrict__ rec1,
                                                         const uint32_t* __restrict__ offsets,
                                                         int64_t n, int64_t R, const DeviceStatus* st,
                                                         int64_t capacity,
                                                         unsigned long long* __restrict__ keys,
                                                         uint32_t* __restrict__ vals, int passes,
                                                         uint32_t* __restrict__ hist) {
    constexpr int RADIX = 1 << RB;
    __shared__ uint32_t h[kMaxSortPasses * RADIX];
    __shared__ uint4 tab_all[8][32][4];  // the row tables of each warp's 32 records
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint4 (*tab)[4] = tab_all[threadIdx.x >> 5];
    const bool overflow = st->m > (unsigned long long)capacity;  // reported by the scan
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t n32 = (uint32_t)n;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < R;
         base += warps * 32) {
        const int64_t r = base + lane;
        const uint32_t cnt = (r < R && !overflow) ? tiles[r] : 0u;
        if (!__ballot_sync(kFullMask, cnt != 0u)) continue;
        uint32_t zbits = 0, tbase = 0, hdr = 0;
        int TW = 0;
        if (cnt) {
            zbits = __float_as_uint(rec1[r].z);
            const int v = (int)((uint32_t)r / n32);
            tbase = vt.v[v].tile_base;
            TW = vt.v[v].tiles_x;
#pragma unroll
            for (int k = 0; k < 4; ++k) tab[lane][k] = spans[4 * r + k];
            hdr = tab[lane][0].x;
        }
        __syncwarp();
        const bool slow = cnt && (hdr >> 16) == kSpanRowsOverflow;
        // digits inside the depth bits: once per record, weighted by its instance count
        for (int p = 0; p < passes && (p + 1) * RB <= 32; ++p) {
            const uint32_t d = cnt ? (zbits >> (p * RB)) & (RADIX - 1) : RADIX;
            const uint32_t peers = __match_any_sync(kFullMask, d);
            const uint32_t group = __reduce_add_sync(peers, cnt);
            if (cnt && lane == 31 - __clz(peers)) atomicAdd(&h[p * RADIX + d], group);
        }
        uint32_t incl = cnt;  // inclusive warp scan of the counts
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, incl, k);
            if (lane >= k) incl += y;
        }
        const uint32_t total = __shfl_sync(kFullMask, incl, 31);
        const uint32_t obase = __shfl_sync(kFullMask, lane == 0 ? offsets[base] : 0u, 0);
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + lane;
            int q = 0;  // records whose range ends at or before slot e
#pragma unroll
            for (int bstep = 16; bstep > 0; bstep >>= 1) {
                const uint32_t v = __shfl_sync(kFullMask, incl, q + bstep - 1);
                if (v <= e) q += bstep;
            }
            q = min(q, 31);
            const uint32_t first = __shfl_sync(kFullMask, incl - cnt, q);
            const uint32_t cq = __shfl_sync(kFullMask, cnt, q);
            const uint32_t zb = __shfl_sync(kFullMask, zbits, q);
            const uint32_t tb = __shfl_sync(kFullMask, tbase, q);
            const int TWq = __shfl_sync(kFullMask, TW, q);
            const bool slow_q = __shfl_sync(kFullMask, (uint32_t)slow, q) != 0u;
            if (e < total && !slow_q) {
                const uint32_t* tq = reinterpret_cast<const uint32_t*>(tab[q]);
                const uint32_t local = e - first;
                const int rows = (int)(tq[0] >> 16);
                // the row holding slot `local`: the last row whose tiles-before <= local
                int k = 0;
                while (k + 1 < rows && (tq[2 + k] >> 16) <= local) ++k;
                const uint32_t rw = tq[1 + k];
                const uint32_t before = rw >> 16;
                const uint32_t after = k + 1 < rows ? (tq[2 + k] >> 16) : cq;
                const int ty = (int)(tq[0] & 0xffffu) + k;
                const uint32_t row_t0 = tb + (uint32_t)(ty * TWq) + (rw & 0xffffu);
                const uint32_t t = row_t0 + (local - before);
                const unsigned long long key = ((unsigned long long)t << 32) | zb;
                const uint32_t pos = obase + e;
                if ((int64_t)pos < capacity) {  // only false after a failed scan
                    keys[pos] = key;
                    vals[pos] = (uint32_t)(base + q);
                }
                count_tile_digits<RB>(h, passes, key, t, row_t0, row_t0 + (after - before));
            }
        }
        // records whose row table overflowed: the whole warp recomputes their rows
        uint32_t todo = __ballot_sync(kFullMask, slow);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const float4 aj = rec0[base + j];
            const float qc = rec1[base + j].x;
            const float px = aj.x, py = aj.y, A = -2.0f * aj.z, B = -aj.w, C = -2.0f * qc;
            const uint32_t zb = __shfl_sync(kFullMask, zbits, j);
            const uint32_t tb = __shfl_sync(kFullMask, tbase, j);
            const int TWj = __shfl_sync(kFullMask, TW, j);
            const int v = (int)((uint32_t)(base + j) / n32);
            uint32_t oj = obase + __shfl_sync(kFullMask, incl - cnt, j);
            const RowSpans rs = row_setup(px, py, A, B, C, vt.tile_h, vt.v[v].tiles_y);
            for (int row0 = rs.ty0; row0 <= rs.ty1; row0 += 32) {
                const int ty = row0 + lane;
                int c0 = 0, c1 = -1;
                if (ty <= rs.ty1 && !row_span(rs, px, py, B, ty, vt.tile_w, vt.tile_h, TWj, c0, c1)) c1 = -1;
                const uint32_t len = (uint32_t)(c1 - c0 + 1);
                uint32_t rincl = len;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFullMask, rincl, k);
                    if (lane >= k) rincl += y;
                }
                const uint32_t rtotal = __shfl_sync(kFullMask, rincl, 31);
                for (uint32_t e0 = 0; e0 < rtotal; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    int q = 0;
#pragma unroll
                    for (int bstep = 16; bstep > 0; bstep >>= 1) {
                        const uint32_t vv = __shfl_sync(kFullMask, rincl, q + bstep - 1);
                        if (vv <= e) q += bstep;
                    }
                    q = min(q, 31);
                    const uint32_t rfirst = __shfl_sync(kFullMask, rincl - len, q);
                    const uint32_t lq = __shfl_sync(kFullMask, len, q);
                    const int cq = __shfl_sync(kFullMask, c0, q);
                    if (e < rtotal) {
                        const uint32_t row_t0 = tb + (uint32_t)((row0 + q) * TWj + cq);
                        const uint32_t t = row_t0 + (e - rfirst);
                        const unsigned long long key = ((unsigned long long)t << 32) | zb;
                        const uint32_t pos = oj + e;
                        if ((int64_t)pos < capacity) {
                            keys[pos] = key;
                            vals[pos] = (uint32_t)(base + j);
                        }
                        count_tile_digits<RB>(h, passes, key, t, row_t0, row_t0 + lq);
                    }
                }
                oj += rtotal;
            }
        }
        __syncwarp();  // the tables are rewritten by the next group
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x)
        if (h[j]) atomicAdd(&hist[j], h[j]);
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
                             unsigned long long* keys, uint32_t* vals, int digit_bits, int passes,
                             uint32_t* hist, cudaStream_t s) {
    cudaError_t e = launch_fill_u32(hist, 0u, (size_t)kMaxSortPasses * 256, s);
    if (e != cudaSuccess || R == 0) return e;
    const int threads = 256;
    const int64_t want = (R + threads - 1) / threads;
    const unsigned blocks = (unsigned)(want < 148 * 8 ? want : 148 * 8);
    switch (digit_bits) {
#define SGS_DUP(RB) case RB: duplicate_kernel<RB><<<blocks, threads, 0, s>>>(vt, p.spans, p.tiles, p.rec0, \
        p.rec1, offsets, n, R, st, capacity, keys, vals, passes, hist); break;
        SGS_DUP(4) SGS_DUP(5) SGS_DUP(6) SGS_DUP(7) SGS_DUP(8)
#undef SGS_DUP
        default: return cudaErrorInvalidValue;
    }
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
