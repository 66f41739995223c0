// Stage (c): stable LSD radix sort of (uint64 or uint32 key, uint32 value) pairs, onesweep
// style.
//
//   1. digit histograms of every pass at once (one read of the keys), unless the caller
//      counted them already;
//   2. an exclusive scan per pass turns them into global bucket offsets;
//   3. per pass, one kernel: each CTA takes the next tile of keys (dynamic tile id, so every
//      earlier tile is already running), ranks its keys by digit within each warp (stable:
//      input order within the tile), publishes its per-digit counts, scans them into
//      CTA-local digit starts, stages the tile in shared memory in digit order, resolves
//      its global per-digit offsets by decoupled look-back over the earlier tiles, and
//      writes each digit's run as consecutive stores.  Optionally the first pass drops the
//      pairs whose key is all ones (the records without instances of the record sort).
// Digits are 4..10 bits; a sort of n bits uses the fewest passes of at most the requested
// width and the narrowest uniform width for that many passes (17 bits: 2 passes of 9).
// Look-back words are 64 bits: an 8-bit tag (2p+1 aggregate, 2p+2 inclusive for pass p)
// and a 56-bit count, so one table serves all passes of a sort after a single clear.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

// The lanes of the warp whose value d equals this lane's, from one ballot per bit of d
// (d < 2^BITS).  Same result as a match-any, without its long-latency shared-pipe
// instruction: a ballot per bit and one logic op per bit.
template <int BITS>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    uint32_t peers = kFullMask;
#pragma unroll
    for (int i = 0; i < BITS; ++i) {
        const uint32_t bit = (d >> i) & 1u;
        const uint32_t b = __ballot_sync(kFullMask, bit);
        peers &= bit ? b : ~b;
    }
    return peers;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr unsigned long long kCountMask = (1ull << 56) - 1;

// Digit of pass p: bits [first_bit + p*RB, first_bit + p*RB + width_p) of the key, where
// the last pass may be narrower so that no bit at or above key_bits is used.
__host__ __device__ __forceinline__ int pass_width(int p, int RB, int first_bit, int key_bits) {
    const int lo = first_bit + p * RB;
    return key_bits - lo < RB ? key_bits - lo : RB;
}

template <typename KeyT, int RB>
__global__ void __launch_bounds__(256) histogram_kernel(const KeyT* __restrict__ keys,
                                                        const uint32_t* m_ptr, int passes, int first_bit,
                                                        int key_bits, uint32_t* __restrict__ hist) {
    constexpr int RADIX = 1 << RB;
    extern __shared__ uint32_t h[];  // [passes][RADIX]
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const uint64_t m = *m_ptr;  // 64-bit loop index: base + stride cannot wrap
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const uint64_t idx = base + threadIdx.x;
        const bool valid = idx < m;
        const unsigned long long k = valid ? (unsigned long long)keys[idx] : 0ull;
        const uint32_t active = __ballot_sync(kFullMask, valid);
        for (int p = 0; p < passes; ++p) {
            const uint32_t mask = (1u << pass_width(p, RB, first_bit, key_bits)) - 1u;
            const uint32_t d = valid ? (uint32_t)(k >> (first_bit + p * RB)) & mask : RADIX;
            const uint32_t peers = digit_peers<RB + 1>(d) & active;
            if (valid && (threadIdx.x & 31) == 31 - __clz(peers))
                atomicAdd(&h[p * RADIX + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x)
        if (h[j]) atomicAdd(&hist[j], h[j]);
}

// One CTA per pass: exclusive scan over the RADIX buckets.
template <int RB>
__global__ void histogram_scan_kernel(const uint32_t* __restrict__ hist, uint32_t* __restrict__ goff) {
    constexpr int RADIX = 1 << RB;
    __shared__ uint32_t s[RADIX];
    const int p = blockIdx.x;
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) s[d] = hist[p * RADIX + d];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int j = 0; j < RADIX; ++j) {
            const uint32_t c = s[j];
            s[j] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) goff[p * RADIX + d] = s[d];
}

// Items per thread: 15 for 64-bit keys (3 CTAs per SM), 16 for 32-bit keys (4 CTAs per SM:
// 64 registers, about 52 KB of shared memory with 9-bit digits).
template <typename KeyT>
struct SortShape {
    static constexpr int ITEMS = sizeof(KeyT) == 8 ? 15 : 16;
    static constexpr int TILE = kSortThreads * ITEMS;
};

// The look-back tables are sized for tiles of kSortTile keys (sort_lookback_entries): no
// key width may use a smaller tile, or a sort would have more tiles than table rows.
static_assert(SortShape<uint32_t>::TILE >= kSortTile && SortShape<unsigned long long>::TILE >= kSortTile,
              "a sort tile is smaller than the tile the look-back tables are sized for");

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename KeyT, int RB>
struct OnesweepSmem {
    static constexpr int RADIX = 1 << RB;
    static constexpr int WARPS = kSortThreads / 32;
    static constexpr int TILE = SortShape<KeyT>::TILE;
    union {
        uint32_t warp_hist[WARPS][RADIX + 1];  // ranking; +1: sentinel bucket of the ragged tail
        struct {
            KeyT keys[TILE];  // staging, after the positions are in registers
            uint32_t vals[TILE];
        } stage;
    } u;
    uint32_t vbuf[TILE];  // the tile's values, copied in while the keys are ranked
    uint32_t digit_start[RADIX];
    uint32_t gbase[RADIX];
    uint32_t wsum[WARPS];
    uint32_t nvalid;  // items of the tile that are kept
    uint32_t tile;
};

template <typename KeyT, int RB, bool DROP>
__global__ void __launch_bounds__(kSortThreads, sizeof(KeyT) == 8 ? 3 : 4) onesweep_kernel(
    const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin, KeyT* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* m_ptr, const uint32_t* __restrict__ goff,
    unsigned long long* lookback, uint32_t* counter, int shift, int width, int pass, DeviceStatus* st,
    uint32_t ahead) {
    constexpr int RADIX = 1 << RB;
    constexpr int WARPS = kSortThreads / 32;
    constexpr int DPT = (RADIX + kSortThreads - 1) / kSortThreads;  // digits per thread
    constexpr int kSortItems = SortShape<KeyT>::ITEMS;
    constexpr int kSortTile = SortShape<KeyT>::TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<KeyT, RB>& sm = *reinterpret_cast<OnesweepSmem<KeyT, RB>*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t dmask = (1u << width) - 1u;
    if (threadIdx.x == 0) sm.tile = atomicAdd(counter, 1u);
    const uint32_t m = *m_ptr;  // in flight together with the tile claim
    for (int j = threadIdx.x; j < WARPS * (RADIX + 1); j += kSortThreads) (&sm.u.warp_hist[0][0])[j] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile;
    const uint64_t tile_start = (uint64_t)tile * kSortTile;
    if (tile_start >= m) return;  // whole CTA: nothing in this tile
    if (threadIdx.x == 0) {
        // the keys and values of the tile a CTA will claim about one CTA lifetime from now
        // (`ahead` = the CTAs resident at once) travel to L2 while this tile is sorted; the
        // ranges start 16-byte aligned (tile starts) and are cut down to 16-byte multiples,
        // so they end inside the m items
        const uint64_t ps = ((uint64_t)tile + ahead) * kSortTile;
        if (ps < m) {
            const uint32_t n = (uint32_t)(m - ps < (uint64_t)kSortTile ? m - ps : kSortTile);
            const uint32_t kb = (uint32_t)(n * sizeof(KeyT)) & ~15u, vb = (n * 4u) & ~15u;
            if (kb) prefetch_l2(kin + ps, kb);
            if (vb) prefetch_l2(vin + ps, vb);
        }
    }
    const uint32_t count = (uint32_t)(m - tile_start < (uint64_t)kSortTile ? m - tile_start : kSortTile);

    // load keys warp-striped: item k of lane l of warp w is element w*32*ITEMS + k*32 + l
    KeyT key[kSortItems];
    uint32_t rank[kSortItems];
    const uint32_t wbase = warp * 32 * kSortItems;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t e = wbase + k * 32 + lane;
        key[k] = e < count ? kin[tile_start + e] : (KeyT)0;
    }
    // the values travel to shared memory meanwhile (each thread copies what it stages)
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t e = wbase + k * 32 + lane;
        if (e < count) cp_async4(&sm.vbuf[e], vin + tile_start + e);
    }
    // stable warp-level ranking (items past the end go to the sentinel bucket RADIX)
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t e = wbase + k * 32 + lane;
        // items past the end, and (drop) all-ones keys, go to the sentinel bucket: not kept
        const bool keep = e < count && !(DROP && key[k] == (KeyT)~(KeyT)0);
        const uint32_t d = keep ? (uint32_t)(key[k] >> shift) & dmask : RADIX;
        // alternate the two ways of finding the lanes with the same digit so that the
        // ballots (ALU pipe) and match-any (shared pipe) run side by side
        const uint32_t peers = (k & 1) ? digit_peers<RB + 1>(d) : __match_any_sync(kFullMask, d);
        const int leader = 31 - __clz(peers);
        uint32_t prior = 0;
        if (lane == leader) {
            prior = sm.u.warp_hist[warp][d];
            sm.u.warp_hist[warp][d] = prior + __popc(peers);
        }
        prior = __shfl_sync(kFullMask, prior, leader);
        rank[k] = prior + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps (in place) and the tile total
    uint32_t total[DPT];
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = threadIdx.x * DPT + i;
        uint32_t acc = 0;
        if (d < RADIX) {
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = sm.u.warp_hist[w][d];
                sm.u.warp_hist[w][d] = acc;
                acc += c;
            }
        }
        total[i] = acc;
        tsum += acc;
    }
    // publish this tile's per-digit counts before anything else of the tile (successors
    // wait for them)
    const unsigned long long tag_agg = (unsigned long long)(2 * pass + 1) << 56;
    const unsigned long long tag_inc = (unsigned long long)(2 * pass + 2) << 56;
    unsigned long long* row = lookback + (size_t)tile * RADIX;
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = threadIdx.x * DPT + i;
        if (d < RADIX) slot_store(row + d, tile == 0 ? (tag_inc | (goff[d] + total[i])) : (tag_agg | total[i]));
    }
    // exclusive scan of the digit totals over the CTA -> CTA-local digit starts
    {
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < WARPS ? sm.wsum[lane] : 0u;
            uint32_t inc = w;
#pragma unroll
            for (int o = 1; o < WARPS; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullMask, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane < WARPS) sm.wsum[lane] = inc - w;
            if (lane == WARPS - 1) sm.nvalid = inc;
        }
        __syncthreads();
        uint32_t run = x - tsum + sm.wsum[warp];
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            const int d = threadIdx.x * DPT + i;
            if (d < RADIX) sm.digit_start[d] = run;
            run += total[i];
        }
    }
    __syncthreads();
    // CTA-local sorted position of every item (the warp histograms are read for the last
    // time here; the staging buffer that aliases them is written after the barrier)
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t e = wbase + k * 32 + lane;
        const uint32_t d = (uint32_t)(key[k] >> shift) & dmask;
        const bool keep = e < count && !(DROP && key[k] == (KeyT)~(KeyT)0);
        rank[k] = keep ? sm.digit_start[d] + sm.u.warp_hist[warp][d] + rank[k] : 0xffffffffu;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        if (rank[k] != 0xffffffffu) {
            sm.u.stage.keys[rank[k]] = key[k];
            sm.u.stage.vals[rank[k]] = sm.vbuf[wbase + k * 32 + lane];
        }
    }
    // look back for the global prefixes (late: the predecessors have had the staging time
    // to publish)
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = threadIdx.x * DPT + i;
        if (d >= RADIX) continue;
        unsigned long long prefix = goff[d];
        if (tile != 0) {
            // the inclusive prefix of a tile includes goff[d]
            prefix = lookback_sum(lookback + d, (int64_t)tile - 1, RADIX, kCountMask, tag_agg, tag_inc, st);
            slot_store(row + d, tag_inc | (prefix + total[i]));
        }
        sm.gbase[d] = (uint32_t)prefix - sm.digit_start[d];  // global minus CTA-local start
    }
    __syncthreads();
    const uint32_t nvalid = sm.nvalid;
    for (uint32_t j = threadIdx.x; j < nvalid; j += kSortThreads) {
        const KeyT kk = sm.u.stage.keys[j];
        const uint32_t d = (uint32_t)(kk >> shift) & dmask;
        const uint32_t dest = sm.gbase[d] + j;
        if (dest < m) {
            kout[dest] = kk;
            vout[dest] = sm.u.stage.vals[j];
        }
    }
}

template <typename KeyT>
__global__ void copy_pairs_kernel(const KeyT* __restrict__ ks, const uint32_t* __restrict__ vs,
                                  KeyT* __restrict__ kd, uint32_t* __restrict__ vd, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        kd[j] = ks[j];
        vd[j] = vs[j];
    }
}

__global__ void sort_init_kernel(DeviceStatus* st, uint32_t m) {
    st->status = 0;
    st->m_clamped = m;
    st->m = m;
    for (int j = 0; j < 16; ++j) st->tile_counter[j] = 0;
}

template <typename KeyT, int RB>
cudaError_t sort_impl(KeyT* k0, uint32_t* v0, KeyT* k1, uint32_t* v1,
                      const uint32_t* m_ptr, int64_t capacity, int first_bit, int key_bits, uint32_t* hist,
                      uint32_t* goff, uint32_t* counters, unsigned long long* lookback,
                      DeviceStatus* st, cudaStream_t s, cudaEvent_t hist_end, bool histogram_ready,
                      const uint32_t* m_rest, bool drop_first) {
    constexpr int RADIX = 1 << RB;
    const int passes = (key_bits - first_bit + RB - 1) / RB;
    cudaError_t e;
    if (!histogram_ready && (e = launch_fill_u32(hist, 0u, (size_t)passes * RADIX, s)) != cudaSuccess)
        return e;
    if ((e = launch_fill_u32(counters, 0u, kMaxSortPasses, s)) != cudaSuccess) return e;
    constexpr int kSortTile = SortShape<KeyT>::TILE;
    const size_t tiles = (size_t)((capacity + kSortTile - 1) / kSortTile);
    if ((e = launch_fill_u32(reinterpret_cast<uint32_t*>(lookback), 0u, tiles * RADIX * 2, s)) != cudaSuccess)
        return e;
    if (capacity == 0 || tiles == 0 || passes <= 0) {
        if (hist_end) return record_probe(hist_end, s);
        return cudaSuccess;
    }
    if (!histogram_ready) {
        const int64_t want = (capacity + 255) / 256;
        const int blocks = (int)stride_grid(want, 8);
        const size_t hs = (size_t)passes * RADIX * sizeof(uint32_t);
        if ((e = cudaFuncSetAttribute(histogram_kernel<KeyT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)hs)) != cudaSuccess)
            return e;
        histogram_kernel<KeyT, RB><<<blocks, 256, hs, s>>>(k0, m_ptr, passes, first_bit, key_bits, hist);
    }
    histogram_scan_kernel<RB><<<passes, RADIX < 32 ? 32 : (RADIX > 1024 ? 1024 : RADIX), 0, s>>>(hist, goff);
    if (hist_end && (e = record_probe(hist_end, s)) != cudaSuccess) return e;
    const size_t smem = sizeof(OnesweepSmem<KeyT, RB>);
    if ((e = cudaFuncSetAttribute(onesweep_kernel<KeyT, RB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    if (drop_first && (e = cudaFuncSetAttribute(onesweep_kernel<KeyT, RB, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel<KeyT, RB, false>, kSortThreads,
                                                           smem)) != cudaSuccess)
        return e;
    const uint32_t ahead = (uint32_t)(sm_count() * (per_sm > 0 ? per_sm : 1));
    for (int p = 0; p < passes; ++p) {
        const KeyT* kin = (p & 1) ? k1 : k0;
        const uint32_t* vin = (p & 1) ? v1 : v0;
        KeyT* kout = (p & 1) ? k0 : k1;
        uint32_t* vout = (p & 1) ? v0 : v1;
        const uint32_t* mp = p > 0 && m_rest ? m_rest : m_ptr;
        const uint32_t width = pass_width(p, RB, first_bit, key_bits);
        if (p == 0 && drop_first)
            onesweep_kernel<KeyT, RB, true><<<(unsigned)tiles, kSortThreads, smem, s>>>(
                kin, vin, kout, vout, mp, goff + p * RADIX, lookback, counters + p, first_bit + p * RB, width, p, st,
                ahead);
        else
            onesweep_kernel<KeyT, RB, false><<<(unsigned)tiles, kSortThreads, smem, s>>>(
                kin, vin, kout, vout, mp, goff + p * RADIX, lookback, counters + p, first_bit + p * RB, width, p, st,
                ahead);
    }
    return cudaGetLastError();
}

}  // namespace

void sort_digit_plan(int first_bit, int key_bits, int max_digit_bits, int* passes, int* digit_bits) {
    const int nbits = key_bits - first_bit;
    const int p = nbits <= 0 ? 0 : (nbits + max_digit_bits - 1) / max_digit_bits;
    int rb = p == 0 ? kMinDigitBits : (nbits + p - 1) / p;
    if (rb < kMinDigitBits) rb = kMinDigitBits;
    *passes = p;
    *digit_bits = rb;
}

int sort_passes(int key_bits, int digit_bits) { return sort_passes(0, key_bits, digit_bits); }

int sort_passes(int first_bit, int key_bits, int digit_bits) {
    int p, rb;
    sort_digit_plan(first_bit, key_bits, digit_bits, &p, &rb);
    return p;
}

size_t sort_lookback_entries(int64_t capacity, int digit_bits) {
    // the 64-bit key tile is the smaller one, so this bounds both key widths
    return (size_t)((capacity + kSortTile - 1) / kSortTile) * ((size_t)1 << digit_bits);
}

namespace {
template <typename KeyT>
cudaError_t launch_sort_t(KeyT* k0, uint32_t* v0, KeyT* k1, uint32_t* v1, const uint32_t* m_ptr, int64_t capacity,
                          int first_bit, int key_bits, int digit_bits, uint32_t* hist, uint32_t* goff,
                          uint32_t* counters, unsigned long long* lookback, DeviceStatus* st, cudaStream_t s,
                          cudaEvent_t hist_end, bool histogram_ready, const uint32_t* m_rest = nullptr,
                          bool drop_first = false) {
    int passes, rb;
    sort_digit_plan(first_bit, key_bits, digit_bits, &passes, &rb);
    switch (rb) {
#define SGS_SORT(RB)                                                                                          \
    case RB:                                                                                                  \
        return sort_impl<KeyT, RB>(k0, v0, k1, v1, m_ptr, capacity, first_bit, key_bits, hist, goff, counters, \
                                   lookback, st, s, hist_end, histogram_ready, m_rest, drop_first);
        SGS_SORT(4) SGS_SORT(5) SGS_SORT(6) SGS_SORT(7) SGS_SORT(8) SGS_SORT(9) SGS_SORT(10)
#undef SGS_SORT
        default: return cudaErrorInvalidValue;
    }
}

template <typename KeyT>
cudaError_t copy_pairs_t(const KeyT* ks, const uint32_t* vs, KeyT* kd, uint32_t* vd, int64_t m, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    const int64_t want = (m + 255) / 256;
    copy_pairs_kernel<KeyT><<<(int)stride_grid(want, 16), 256, 0, s>>>(ks, vs, kd, vd, m);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_sort(unsigned long long* k0, uint32_t* v0, unsigned long long* k1, uint32_t* v1,
                        const uint32_t* m_ptr, int64_t capacity, int first_bit, int key_bits, int digit_bits,
                        uint32_t* hist, uint32_t* goff, uint32_t* counters,
                        unsigned long long* lookback, DeviceStatus* st, cudaStream_t s,
                        cudaEvent_t hist_end, bool histogram_ready) {
    return launch_sort_t(k0, v0, k1, v1, m_ptr, capacity, first_bit, key_bits, digit_bits, hist, goff, counters,
                         lookback, st, s, hist_end, histogram_ready);
}

cudaError_t launch_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* m_ptr,
                        int64_t capacity, int first_bit, int key_bits, int digit_bits, uint32_t* hist,
                        uint32_t* goff, uint32_t* counters, unsigned long long* lookback, DeviceStatus* st,
                        cudaStream_t s, cudaEvent_t hist_end, bool histogram_ready, const uint32_t* m_rest,
                        bool drop_first) {
    if (key_bits > 32) return cudaErrorInvalidValue;
    return launch_sort_t(k0, v0, k1, v1, m_ptr, capacity, first_bit, key_bits, digit_bits, hist, goff, counters,
                         lookback, st, s, hist_end, histogram_ready, m_rest, drop_first);
}

cudaError_t launch_copy_pairs(const unsigned long long* ks, const uint32_t* vs, unsigned long long* kd,
                              uint32_t* vd, int64_t m, cudaStream_t s) {
    return copy_pairs_t(ks, vs, kd, vd, m, s);
}

cudaError_t launch_copy_pairs(const uint32_t* ks, const uint32_t* vs, uint32_t* kd, uint32_t* vd, int64_t m,
                              cudaStream_t s) {
    return copy_pairs_t(ks, vs, kd, vd, m, s);
}

cudaError_t launch_sort_init(DeviceStatus* st, uint32_t m, cudaStream_t s) {
    sort_init_kernel<<<1, 1, 0, s>>>(st, m);
    return cudaGetLastError();
}

}  // namespace sgs
