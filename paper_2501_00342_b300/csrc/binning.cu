// Stages (b) and (d) and their helpers: the digit histograms of the record depth sort, the
// exclusive scan of tiles touched in depth order, the duplication of the records into
// (tile id, record) instances in that order, the per-tile ranges over the sorted tile ids,
// and the blend's tile orders (most expensive tiles first).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

// ---- decoupled look-back words of the scan: 2-bit flag | 62-bit value ----
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

// One thread runs the scan's look-back over caller-provided slots (failure-detection test of
// the bounded wait): the status word lives in shared memory and is copied out.
__global__ void lookback_selftest_kernel(const unsigned long long* slots, int64_t n,
                                         unsigned long long* sum, int32_t* status) {
    __shared__ DeviceStatus s;
    if (threadIdx.x == 0) {
        s.status = 0;
        sum[0] = lookback_sum(slots, n - 1, 1, kValueMask, kFlagAgg, kFlagInc, &s);
        status[0] = s.status;
    }
}

__global__ void fill_u32_kernel(uint32_t* p, uint32_t value, size_t count) {
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (size_t)gridDim.x * blockDim.x)
        p[j] = value;
}

// Single-pass exclusive scan (chained scan with decoupled look-back).  Each CTA takes
// the next tile id from a counter, so every predecessor tile is already running.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const uint32_t* __restrict__ in,
                                                             const uint32_t* __restrict__ perm,
                                                             const RecordValue rv, const uint32_t* n_valid,
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
    if (perm) {  // counts carried by the depth-sorted record values; none past the kept ones
        const int64_t nv = n_valid ? (int64_t)*n_valid : R;
        if (base + kScanItems <= nv) {  // 16-byte loads: the thread's 16 values are consecutive
            const uint4* p4 = reinterpret_cast<const uint4*>(perm + base);
#pragma unroll
            for (int q = 0; q < kScanItems / 4; ++q) {
                const uint4 w = __ldg(p4 + q);
                v[4 * q] = rv.count(w.x, in);
                v[4 * q + 1] = rv.count(w.y, in);
                v[4 * q + 2] = rv.count(w.z, in);
                v[4 * q + 3] = rv.count(w.w, in);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kScanItems; ++q) v[q] = (base + q < nv) ? rv.count(perm[base + q], in) : 0u;
        }
    } else if (base + kScanItems <= R) {
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
            slot_store(lookback, kFlagInc | acc);
        } else {
            slot_store(lookback + tile, kFlagAgg | acc);
            prefix = lookback_sum(lookback, (int64_t)tile - 1, 1, kValueMask, kFlagAgg, kFlagInc, st);
            slot_store(lookback + tile, kFlagInc | (prefix + acc));
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

// Keys of the record sort: the float bits of the view depth of a record with instances
// (depth > near > 0, so the bits order like the values), 0xffffffff for the others.
// Digit histograms of every pass of the record sort over the keys of the records with
// instances (view depth bits; 0xffffffff marks the others, which the sort drops), per-warp
// shared copies.  The low digits of depth bits are spread: one shared atomic each; the
// high ones (exponent and top mantissa bits) repeat within a warp: the warp finds the lanes
// of each distinct digit with one match-any and adds it once.  Also stores R in
// st->num_records and adds the kept records to st->num_visible (cleared before the launch).
template <int RB>
__global__ void __launch_bounds__(256) record_hist_kernel(const uint32_t* __restrict__ keys, int64_t R,
                                                          DeviceStatus* st, uint32_t* __restrict__ hist) {
    constexpr int RADIX = 1 << RB;
    constexpr int passes = (32 + RB - 1) / RB;  // a 32-bit key in digits of RB bits (the last narrower)
    extern __shared__ uint32_t h[];  // [8 warps][passes][RADIX]
    for (int j = threadIdx.x; j < 8 * passes * RADIX; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* hw = h + warp * passes * RADIX;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->num_records = (uint32_t)R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t kept_count = 0;  // warp total (same in every lane)
    // warp-uniform trip count: every lane of a warp runs the same iterations; the keys of
    // kUnroll strides are loaded before any is counted (loads in flight together)
    constexpr int kUnroll = 4;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < R;
         base += kUnroll * stride) {
        uint32_t key[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t r = base + u * stride + lane;
            key[u] = r < R ? keys[r] : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const bool kept = key[u] != 0xffffffffu;
            const uint32_t live = __ballot_sync(kFullMask, kept);
            kept_count += __popc(live);
#pragma unroll
            for (int p = 0; p < passes; ++p) {
                const uint32_t d = (key[u] >> (p * RB)) & (RADIX - 1);
                if (2 * p < passes) {
                    if (kept) atomicAdd(&hw[p * RADIX + d], 1u);
                } else {
                    const uint32_t peers = __match_any_sync(kFullMask, kept ? d : 0xffffffffu) & live;
                    if (kept && lane == 31 - __clz(peers)) hw[p * RADIX + d] += __popc(peers);
                    __syncwarp();
                }
            }
        }
    }
    if (lane == 0 && kept_count) atomicAdd(&st->num_visible, kept_count);
    __syncthreads();
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) acc += h[w * passes * RADIX + j];
        if (acc) atomicAdd(&hist[j], acc);
    }
}

// Digit counts of the tile sort (its digits cover the tile id, bits 32 and up of a key) for
// the key of tile t in a row of tiles [row_t0, row_end).  Along a row the tile ids are
// consecutive, so the digit of pass p (bits p*RB.. of the tile id) is constant on segments
// of 2^(p*RB) tiles: the key that opens a segment adds the segment's length.
template <int RB>
__device__ __forceinline__ void count_tile_digits(uint32_t* h, int passes, uint32_t t, uint32_t row_t0,
                                                  uint32_t row_end) {
    constexpr int RADIX = 1 << RB;
    constexpr int MAXP = (32 + RB - 1) / RB;
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
        if (p >= passes) break;
        const int sh = p * RB;
        if (sh > 0 && t != row_t0 && (t & ((1u << sh) - 1u)) != 0u) continue;  // inside a segment
        const uint32_t seg_end = sh > 0 ? min(row_end, ((t >> sh) + 1u) << sh) : t + 1u;
        atomicAdd(&h[p * RADIX + ((t >> sh) & (RADIX - 1))], seg_end - t);
    }
}

// Writes the (tile id, record) instances in the order of the depth-sorted records
// (perm, RecordValue ids): sorted position j emits its record's offsets[j + 1] - offsets[j]
// tiles at offsets[j] (the scan taken in that order), tiles row-major.  One warp per 32
// consecutive sorted positions, whose instances fill one contiguous output range 32 slots
// at a time: slot e belongs to the record whose first slot is the last at or before e
// (the offsets relative to the warp's first are the inclusive scan of the counts; the
// records' first slots are found from one OR-reduction and one ballot), its packed row
// table (written by preprocess, staged in shared memory) gives the row, and consecutive lanes write
// consecutive slots.  A record whose table overflowed is filled afterwards by the whole
// warp, recomputing its rows with row_span.  Since every instance of a record has the same
// depth, this order is (depth bits, record) -- what the depth half of a stable LSD radix
// sort of (tile | depth) keys would produce -- so only the tile id is left to sort, and the
// depth never has to travel with the instances.  The digit histograms of that tile sort are
// counted here (count_tile_digits).
template <int RB>
__global__ void __launch_bounds__(256, 5) duplicate_kernel(const ViewTable vt, const uint4* __restrict__ spans,
                                                         const RecordValue rv,
                                                         const float4* __restrict__ rec0,
                                                         const float4* __restrict__ rec1,
                                                         const uint32_t* __restrict__ perm,
                                                         const uint32_t* __restrict__ offsets,
                                                         int64_t n, int64_t R, const DeviceStatus* st,
                                                         int64_t capacity,
                                                         uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ vals, int passes,
                                                         uint32_t* __restrict__ hist) {
    constexpr int RADIX = 1 << RB;
    constexpr int MAXP = (32 + RB - 1) / RB;  // passes of a tile-id sort
    __shared__ uint32_t h[MAXP * RADIX];
    __shared__ uint4 tab_all[8][32][4];  // the row tables of each warp's 32 records
    // (tile_base, tiles_x) of every view: read per record with a per-lane view index, which
    // the constant bank would serialise over the views of a warp
    __shared__ uint2 s_view[SGS_MAX_VIEWS];
    for (int j = threadIdx.x; j < passes * RADIX; j += blockDim.x) h[j] = 0;
    for (int j = threadIdx.x; j < vt.B; j += blockDim.x)
        s_view[j] = make_uint2(vt.v[j].tile_base, (uint32_t)vt.v[j].tiles_x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint4 (*tab)[4] = tab_all[threadIdx.x >> 5];
    const bool overflow = st->m > (unsigned long long)capacity;  // reported by the scan
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t n32 = (uint32_t)n;
    // only the first num_visible sorted positions hold records with instances (the record
    // sort dropped the others); the positions past them have no tiles
    const int64_t kept = min(R, (int64_t)st->num_visible);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < kept;
         base += warps * 32) {
        const int64_t j = base + lane;
        // the record's count from the scan: the difference of consecutive offsets
        const uint32_t m_end = st->m_clamped;
        const uint32_t o = j < R ? offsets[j] : m_end;
        // loaded together with the offsets (past the kept records it is stale and unused)
        const uint32_t pv = j < R ? perm[j] : 0u;
        uint32_t o_next = __shfl_down_sync(kFullMask, o, 1);
        if (lane == 31) o_next = base + 32 < R ? offsets[base + 32] : m_end;
        const uint32_t cnt = overflow ? 0u : o_next - o;
        if (!__ballot_sync(kFullMask, cnt != 0u)) continue;
        const uint32_t r = cnt ? rv.id(pv) : 0u;
        uint32_t tbase = 0, hdr = 0;
        int TW = 0;
        if (cnt) {
            const uint2 vw = s_view[r / n32];
            tbase = vw.x;
            TW = (int)vw.y;
            // the table's first sector; the second only for more than kSpanRowsShort rows
            // (words past a table's last row are never read)
            tab[lane][0] = spans[4 * (size_t)r];
            tab[lane][1] = spans[4 * (size_t)r + 1];
            hdr = tab[lane][0].x;
            if ((hdr >> 16) > kSpanRowsShort && (hdr >> 16) != kSpanRowsOverflow) {
                tab[lane][2] = spans[4 * (size_t)r + 2];
                tab[lane][3] = spans[4 * (size_t)r + 3];
            }
        }
        __syncwarp();
        const bool slow = cnt && (hdr >> 16) == kSpanRowsOverflow;
        // For a record of at most 32 instances whose rows all have tiles: bit s set where a
        // row starts (slot s of the record, bit 0 for row 0), so that a slot's row is the
        // count of row starts at or before it.  0: the slots search the table instead.
        uint32_t rowmask = 0u;
        if (cnt && cnt <= 32u && !slow) {
            const uint32_t* tl = reinterpret_cast<const uint32_t*>(tab[lane]);
            const int rws = (int)(hdr >> 16);
            uint32_t mask = 1u, prev = 0u;
            bool ok = true;
            for (int rr = 1; rr < rws; ++rr) {
                const uint32_t b = tl[1 + rr] >> 16;  // tiles before row rr
                ok &= b != prev;                      // else row rr - 1 is empty
                prev = b;
                mask |= b < 32u ? 1u << b : 0u;
            }
            ok &= prev < cnt;  // else the last row is empty
            rowmask = ok ? mask : 0u;
        }
        const uint32_t obase = __shfl_sync(kFullMask, o, 0);
        const uint32_t incl = overflow ? 0u : o_next - obase;  // inclusive warp scan of the counts
        const uint32_t total = __shfl_sync(kFullMask, incl, 31);
        // Every kept record has at least one instance, so the records' first slots are
        // distinct and increasing: slot e belongs to record (records starting at or before
        // e) - 1.  A record without instances (past the kept ones) starts nowhere.
        const uint32_t start = cnt ? incl - cnt : 0xffffffffu;
        const uint32_t le_mask = lane == 31 ? kFullMask : (2u << lane) - 1u;
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + lane;
            const uint32_t rel = start - e0;  // wraps past 32 for records starting before e0
            const uint32_t starts = __reduce_or_sync(kFullMask, cnt && rel < 32u ? 1u << rel : 0u);
            const int earlier = __popc(__ballot_sync(kFullMask, cnt && start < e0));
            const int q = min(max(earlier + __popc(starts & le_mask) - 1, 0), 31);
            const uint32_t first = __shfl_sync(kFullMask, start, q);
            const uint32_t cq = __shfl_sync(kFullMask, cnt, q);
            const uint32_t tb = __shfl_sync(kFullMask, tbase, q);
            const uint32_t rq = __shfl_sync(kFullMask, r, q);
            const int TWq = __shfl_sync(kFullMask, TW, q);
            const bool slow_q = __shfl_sync(kFullMask, (uint32_t)slow, q) != 0u;
            const uint32_t rm = __shfl_sync(kFullMask, rowmask, q);
            if (e < total && !slow_q) {
                const uint32_t* tq = reinterpret_cast<const uint32_t*>(tab[q]);
                const uint32_t local = e - first;
                const int rows = (int)(tq[0] >> 16);
                // the row holding slot `local`: the last row whose tiles-before <= local
                int k = 0;
                if (rm) {
                    k = __popc(rm & (local >= 31u ? kFullMask : (2u << local) - 1u)) - 1;
                } else {
                    while (k + 1 < rows && (tq[2 + k] >> 16) <= local) ++k;
                }
                const uint32_t rw = tq[1 + k];
                const uint32_t before = rw >> 16;
                const uint32_t after = k + 1 < rows ? (tq[2 + k] >> 16) : cq;
                const int ty = (int)(tq[0] & 0xffffu) + k;
                const uint32_t row_t0 = tb + (uint32_t)(ty * TWq) + (rw & 0xffffu);
                const uint32_t t = row_t0 + (local - before);
                const uint32_t pos = obase + e;
                if ((int64_t)pos < capacity) {  // only false after a failed scan
                    keys[pos] = t;
                    vals[pos] = rq;
                }
                count_tile_digits<RB>(h, passes, t, row_t0, row_t0 + (after - before));
            }
        }
        // records whose row table overflowed: the whole warp recomputes their rows
        uint32_t todo = __ballot_sync(kFullMask, slow);
        while (todo) {
            const int jj = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t rj = __shfl_sync(kFullMask, r, jj);
            const float4 aj = rec0[rj];
            const float qc = rec1[rj].x;
            const float px = aj.x, py = aj.y, A = -2.0f * aj.z, B = -aj.w, C = -2.0f * qc;
            const uint32_t tb = __shfl_sync(kFullMask, tbase, jj);
            const int TWj = __shfl_sync(kFullMask, TW, jj);
            const int v = (int)(rj / n32);
            uint32_t oj = obase + __shfl_sync(kFullMask, incl - cnt, jj);
            const RowSpans rs = row_setup(px, py, A, B, C, vt.inv_tile_h, vt.v[v].tiles_y);
            for (int row0 = rs.ty0; row0 <= rs.ty1; row0 += 32) {
                const int ty = row0 + lane;
                int c0 = 0, c1 = -1;
                if (ty <= rs.ty1 && !row_span(rs, px, py, B, ty, vt.inv_tile_w, vt.tile_h, TWj, c0, c1)) c1 = -1;
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
                        const uint32_t pos = oj + e;
                        if ((int64_t)pos < capacity) {
                            keys[pos] = t;
                            vals[pos] = rj;
                        }
                        count_tile_digits<RB>(h, passes, t, row_t0, row_t0 + lq);
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

// Per-tile [start, end) of the sorted instances: four tile ids per thread (one 16-byte
// load) plus the two neighbours, which the adjacent threads load too (cache hits).
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ tile_ids,
                                                      const DeviceStatus* st, uint32_t num_tiles,
                                                      uint2* __restrict__ ranges) {
    const uint64_t m = st->m_clamped;  // 64-bit loop index: q + stride cannot wrap
    const uint64_t nq = (m + 3) / 4;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j0 = 4 * q;
        uint32_t t[6];  // t[0]: id at j0 - 1, t[1..4]: ids at j0..j0+3, t[5]: id at j0 + 4
        if (j0 + 4 <= m) {
            const uint4 v = reinterpret_cast<const uint4*>(tile_ids)[q];
            t[1] = v.x, t[2] = v.y, t[3] = v.z, t[4] = v.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) t[1 + k] = j0 + k < m ? tile_ids[j0 + k] : 0xffffffffu;
        }
        t[0] = j0 > 0 ? tile_ids[j0 - 1] : 0xffffffffu;
        t[5] = j0 + 4 < m ? tile_ids[j0 + 4] : 0xffffffffu;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t j = j0 + k;
            const uint32_t c = t[1 + k];
            if (j >= m || c >= num_tiles) continue;  // c >= num_tiles only after a failed sort
            if (t[k] != c) ranges[c].x = (uint32_t)j;
            if (t[k + 2] != c) ranges[c].y = (uint32_t)(j + 1);
        }
    }
}

// The blend's tile order: tile ids by decreasing cost, so that the CTAs of the most
// expensive tiles start first and a launch does not end on a few long tiles.  The cost of
// tile t is the position of its last contributor top[t] (how far a walk of the tile's
// list goes), or, where top is null or top[t] is 0, the length of its instance list
// (ranges).  The backward passes the tops of the forward it differentiates; the forward
// passes those of the previous forward of the same plan (zero after a new workspace), a
// schedule hint only: any order gives the same images.  One CTA: a counting sort into 64
// buckets of the cost's magnitude (two per power of two), most expensive bucket first;
// within a bucket the order is whatever the shared-memory atomics give (the tiles of a
// launch are independent, so the images do not depend on it).
__device__ __forceinline__ int cost_bucket(uint32_t c) {
    if (c < 2u) return (int)c;
    const int l = 31 - __clz(c);  // 1..31
    return min(63, 2 * l + (int)((c >> (l - 1)) & 1u));
}

__global__ void __launch_bounds__(1024) tile_order_kernel(const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ top, uint32_t num_tiles,
                                                          uint32_t* __restrict__ order) {
    __shared__ uint32_t hist[64];
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    auto cost = [&](uint32_t t) {
        const uint32_t c = top ? top[t] : 0u;
        if (c || !ranges) return c;
        const uint2 r = ranges[t];
        return r.y > r.x ? r.y - r.x : 0u;
    };
    for (uint32_t t = threadIdx.x; t < num_tiles; t += blockDim.x) atomicAdd(&hist[cost_bucket(cost(t))], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {  // bucket starts, the most expensive bucket first
        uint32_t acc = 0;
        for (int b = 63; b >= 0; --b) {
            const uint32_t c = hist[b];
            hist[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < num_tiles; t += blockDim.x)
        order[atomicAdd(&hist[cost_bucket(cost(t))], 1u)] = t;
}

}  // namespace

cudaError_t launch_lookback_selftest(const unsigned long long* slots, int64_t n, unsigned long long* sum,
                                    int32_t* status, cudaStream_t s) {
    lookback_selftest_kernel<<<1, 32, 0, s>>>(slots, n, sum, status);
    return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, uint32_t value, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int threads = 256;
    const size_t want = (count + threads - 1) / threads;
    const int blocks = (int)stride_grid((int64_t)want, 32);
    fill_u32_kernel<<<blocks, threads, 0, s>>>(p, value, count);
    return cudaGetLastError();
}

RecordValue record_value(int64_t R) {
    RecordValue rv;
    rv.id_bits = 1;
    while (rv.id_bits < 32 && ((int64_t)1 << rv.id_bits) < R) ++rv.id_bits;
    return rv;
}

cudaError_t launch_scan(const uint32_t* tiles, const uint32_t* perm, uint32_t* offsets, int64_t R,
                        unsigned long long* scan_lookback, DeviceStatus* st, int64_t capacity,
                        cudaStream_t s) {
    const int64_t num_tiles = (R + kScanTile - 1) / kScanTile;
    if (num_tiles == 0) return cudaSuccess;
    scan_kernel<<<(unsigned)num_tiles, kScanThreads, 0, s>>>(tiles, perm, record_value(R),
                                                             perm ? &st->num_visible : nullptr, offsets, R,
                                                             scan_lookback, st, capacity);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const ViewTable& vt, const RecordPtrs& p, const uint32_t* perm,
                             const uint32_t* offsets, int64_t n, int64_t R, DeviceStatus* st,
                             int64_t capacity, uint32_t* keys, uint32_t* vals, int digit_bits,
                             int passes, uint32_t* hist, cudaStream_t s) {
    cudaError_t e = launch_fill_u32(hist, 0u, (size_t)kHistEntries, s);
    if (e != cudaSuccess || R == 0) return e;
    if (passes > (32 + digit_bits - 1) / digit_bits) return cudaErrorInvalidValue;
    const int threads = 256;
    const int64_t want = (R + threads - 1) / threads;
    // 48 registers: 5 CTAs per SM, two waves of them over the grid-stride loop (the kernel
    // waits on the depth-ordered gathers of the row tables; more warps keep more in flight)
    const unsigned blocks = (unsigned)stride_grid(want, 10);
    switch (digit_bits) {
#define SGS_DUP(RB) case RB: duplicate_kernel<RB><<<blocks, threads, 0, s>>>(vt, p.spans, record_value(R), p.rec0, \
        p.rec1, perm, offsets, n, R, st, capacity, keys, vals, passes, hist); break;
        SGS_DUP(4) SGS_DUP(5) SGS_DUP(6) SGS_DUP(7) SGS_DUP(8) SGS_DUP(9) SGS_DUP(10)
#undef SGS_DUP
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const uint2* ranges, const uint32_t* top, int64_t num_tiles, uint32_t* order,
                              cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    tile_order_kernel<<<1, 1024, 0, s>>>(ranges, top, (uint32_t)num_tiles, order);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* keys, const DeviceStatus* st, int64_t capacity,
                          int64_t num_tiles, uint2* ranges, cudaStream_t s) {
    if (capacity == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (capacity / 4 + threads) / threads;
    const int blocks = (int)stride_grid(want, 32);
    ranges_kernel<<<blocks, threads, 0, s>>>(keys, st, (uint32_t)num_tiles, ranges);
    return cudaGetLastError();
}

}  // namespace sgs

namespace sgs {
cudaError_t launch_record_hist(const uint32_t* keys, int64_t R, DeviceStatus* st, int digit_bits, uint32_t* hist,
                               cudaStream_t s) {
    int passes, rb;
    sort_digit_plan(0, 32, digit_bits, &passes, &rb);
    if (passes != (32 + rb - 1) / rb) return cudaErrorInvalidValue;  // the kernel's pass count
    cudaError_t e = launch_fill_u32(hist, 0u, (size_t)passes << rb, s);
    if (e == cudaSuccess) e = launch_fill_u32(&st->num_visible, 0u, 1, s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int64_t want = (R + threads - 1) / threads;
    const unsigned blocks = (unsigned)stride_grid(want, 8);
    const size_t smem = (size_t)8 * passes * ((size_t)1 << rb) * sizeof(uint32_t);
    switch (rb) {
#define SGS_RH(RB)                                                                                              \
    case RB:                                                                                                     \
        if ((e = cudaFuncSetAttribute(record_hist_kernel<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                      (int)smem)) != cudaSuccess)                                                \
            return e;                                                                                            \
        record_hist_kernel<RB><<<blocks, threads, smem, s>>>(keys, R, st, hist);                                 \
        break;
        SGS_RH(4) SGS_RH(5) SGS_RH(6) SGS_RH(7) SGS_RH(8)
#undef SGS_RH
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace sgs
