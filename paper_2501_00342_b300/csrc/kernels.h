// Host-side launch interface between the C ABI (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "common.cuh"

namespace sgs {

// Streaming multiprocessors of the current device, read from the device once per device.
// The grid-stride kernels size their grids as a multiple of it.
inline int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

// Grid of a grid-stride loop: enough CTAs for `want`, at most per_sm per multiprocessor.
inline int64_t stride_grid(int64_t want, int per_sm) {
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return want < 1 ? 1 : (want < cap ? want : cap);
}

// Records a timing probe on s.  While s is being captured into a CUDA graph the record
// becomes an event-record node of the graph (a plain record would only mark a fork point).
inline cudaError_t record_probe(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(
        ev, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Values of the record sort: the record id in the low id_bits bits (id_bits = bits of
// R - 1, at least 1) and, in the 32 - id_bits bits above, the record's tile count, or the
// all-ones count (also when no bit is left) for "read tiles[id]".  The scan then takes the
// counts in depth order without gathering them.
struct RecordValue {
    int id_bits;
    __host__ __device__ uint32_t id_mask() const { return (uint32_t)((1ull << id_bits) - 1ull); }
    __host__ __device__ uint32_t count_max() const { return (uint32_t)((1ull << (32 - id_bits)) - 1ull); }
    __host__ __device__ uint32_t pack(uint32_t id, uint32_t count) const {
        return id_bits == 32 ? id : id | (min(count, count_max()) << id_bits);
    }
    __host__ __device__ uint32_t id(uint32_t v) const { return v & id_mask(); }
    // the count of value v (tiles: the per-record counts it falls back to)
    __device__ uint32_t count(uint32_t v, const uint32_t* tiles) const {
        const uint32_t c = (uint32_t)((unsigned long long)v >> id_bits);
        return c == count_max() ? tiles[v & id_mask()] : c;
    }
};
RecordValue record_value(int64_t R);

struct RecordPtrs {
    float4* rec0;  // px, py, -A/2, -B
    float4* rec1;  // -C/2, opacity, depth, radius
    float4* rec2;  // r, g, b, clamp mask
    uint2* rect;
    uint32_t* tiles;
    uint4* spans;  // [4][R] packed tile-row table per record (see count_tiles)
    uint32_t* flags;  // per record: visible, clamp decisions, SH degree (kFlag* bits)
    // the record sort's input, written by the preprocess: keys (view depth bits of a record
    // with instances, 0xffffffff for the others) and values (RecordValue)
    uint32_t* sort_keys;
    uint32_t* sort_vals;
    RecordValue rv;
};

// (a) preprocess and its backward
cudaError_t launch_preprocess(const sgs_gaussians& g, const ViewTable& vt, const RecordPtrs& p,
                              cudaStream_t s);
// Reads the 2D gradients of the visible records and clears them (the region is zero after
// the call: the next reverse blend adds into zeros).
cudaError_t launch_preprocess_backward(const sgs_gaussians& g, const ViewTable& vt,
                                       const RecordPtrs& p, float4* grad2d, int64_t R,
                                       const sgs_grads& out, cudaStream_t s);

// (b), (d): scan + duplicate, ranges
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
cudaError_t launch_fill_u32(uint32_t* p, uint32_t value, size_t count, cudaStream_t s);
// The scan's bounded look-back over slots[0, n) from slot n-1 (sum and status word out).
cudaError_t launch_lookback_selftest(const unsigned long long* slots, int64_t n, unsigned long long* sum,
                                     int32_t* status, cudaStream_t s);

// Digit histograms of the record sort over its keys (written by the preprocess); also stores
// R in st->num_records.
cudaError_t launch_record_hist(const uint32_t* keys, int64_t R, DeviceStatus* st, int digit_bits, uint32_t* hist,
                               cudaStream_t s);
// Exclusive scan of the counts of the depth-sorted record values perm (RecordValue; the
// positions at and past st->num_visible, which the record sort left unwritten, count 0),
// or of tiles[j] when perm is null.
cudaError_t launch_scan(const uint32_t* tiles, const uint32_t* perm, uint32_t* offsets, int64_t R,
                        unsigned long long* scan_lookback, DeviceStatus* st, int64_t capacity,
                        cudaStream_t s);
// Also counts the tile sort's digit histograms for digits of digit_bits bits over `passes`
// passes (hist: kHistEntries u32, cleared here).
cudaError_t launch_duplicate(const ViewTable& vt, const RecordPtrs& p, const uint32_t* perm,
                             const uint32_t* offsets, int64_t n, int64_t R, DeviceStatus* st,
                             int64_t capacity, uint32_t* keys, uint32_t* vals, int digit_bits,
                             int passes, uint32_t* hist, cudaStream_t s);
// The blend's tile order: tile ids by decreasing cost into order[num_tiles], the cost being
// top[t] (a tile's last-contributor position) where top is given and non-zero, else the
// instance-list length from ranges.
cudaError_t launch_tile_order(const uint2* ranges, const uint32_t* top, int64_t num_tiles, uint32_t* order,
                              cudaStream_t s);
cudaError_t launch_ranges(const uint32_t* tile_ids, const DeviceStatus* st, int64_t capacity,
                          int64_t num_tiles, uint2* ranges, cudaStream_t s);

// (c) onesweep radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 15;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxSortPasses = 16;
constexpr int kMinDigitBits = 4;
constexpr int kMaxDigitBits = 10;
constexpr int kHistEntries = kMaxSortPasses * (1 << kMaxDigitBits);  // hist / goff length
// Passes and uniform digit width of a sort of key bits [first_bit, key_bits) with digits of
// at most max_digit_bits: the fewest passes, then the narrowest width for them.
void sort_digit_plan(int first_bit, int key_bits, int max_digit_bits, int* passes, int* digit_bits);
size_t sort_lookback_entries(int64_t capacity, int digit_bits);
// Sorts m = *m_ptr pairs (m <= capacity) stably on key bits [first_bit, key_bits); result in
// (k0,v0) if the pass count is even, else in (k1,v1).  digit_bits is the widest digit
// allowed (see sort_digit_plan).  With histogram_ready the digit histograms in hist were
// already counted (by the duplicate kernel).  hist/goff: kHistEntries u32 each; counters:
// kMaxSortPasses u32 (zeroed here); lookback: sort_lookback_entries u64 for the planned
// digit width.
cudaError_t launch_sort(unsigned long long* k0, uint32_t* v0, unsigned long long* k1, uint32_t* v1,
                        const uint32_t* m_ptr, int64_t capacity, int first_bit, int key_bits, int digit_bits,
                        uint32_t* hist, uint32_t* goff, uint32_t* counters,
                        unsigned long long* lookback, DeviceStatus* st, cudaStream_t s,
                        cudaEvent_t hist_end, bool histogram_ready = false);
// The same sort for 32-bit keys (key_bits <= 32; 16 bytes moved per pair and pass).  With
// drop_first the first pass removes the pairs whose key is 0xffffffff (stable for the
// rest); the hist must then count only the kept keys and m_rest holds their number, the
// length of every later pass.
cudaError_t launch_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* m_ptr,
                        int64_t capacity, int first_bit, int key_bits, int digit_bits, uint32_t* hist,
                        uint32_t* goff, uint32_t* counters, unsigned long long* lookback, DeviceStatus* st,
                        cudaStream_t s, cudaEvent_t hist_end, bool histogram_ready = false,
                        const uint32_t* m_rest = nullptr, bool drop_first = false);
int sort_passes(int key_bits, int digit_bits);
int sort_passes(int first_bit, int key_bits, int digit_bits);

// (e) blend and its backward
cudaError_t launch_blend(const ViewTable& vt, const uint2* ranges, const uint32_t* vals,
                         int64_t R, const RecordPtrs& p, int batch, float bg0, float bg1, float bg2,
                         float* out_rgb, float* out_T, float* pix_T, uint32_t* pix_last,
                         uint2* pix_count, const DeviceStatus* st, cudaStream_t s);
cudaError_t launch_blend_backward(const ViewTable& vt, const uint2* ranges, const uint32_t* vals,
                                  const RecordPtrs& p, int batch, float bg0, float bg1, float bg2,
                                  const float* pix_T, const uint32_t* pix_last,
                                  const float* dL_drgb, float4* grad2d, int64_t R,
                                  const DeviceStatus* st, cudaStream_t s);
// grad2d: per record the reverse blend's pixel sums (S_x, S_y, S_xx, S_xy) and
// (S_yy, S_1, dL/dr, dL/dg) as float4[2][R], then dL/db as float[R] (from grad2d + 2 R);
// S_m sums gG m, gG = dL/dalpha exp(power), m the moments 1, dx, dy, dx^2, dx dy, dy^2 of
// d = centre - pixel centre, and the preprocess backward turns them into the centre,
// conic and opacity gradients.  Cleared once when a workspace is bound; the preprocess
// backward clears what the reverse blend wrote.
cudaError_t launch_zero_grad2d(float4* grad2d, int64_t R, cudaStream_t s);

// training: fused Adam step over all parameter planes
cudaError_t launch_adam(const sgs_gaussians& layout, const sgs_grads& raw, const sgs_grads& act,
                        const sgs_grads& grad, const sgs_grads& m, const sgs_grads& v, const sgs_adam_config& cfg,
                        cudaStream_t s);
// loss[0] = scale * sum |img - target|, dL_dimg = scale * sign(img - target)
cudaError_t launch_l1_loss(const float* img, const float* target, int64_t count, float scale, float* loss,
                           float* dL_dimg, cudaStream_t s);
cudaError_t launch_copy_pairs(const unsigned long long* ks, const uint32_t* vs, unsigned long long* kd,
                              uint32_t* vd, int64_t m, cudaStream_t s);
cudaError_t launch_copy_pairs(const uint32_t* ks, const uint32_t* vs, uint32_t* kd, uint32_t* vd, int64_t m,
                              cudaStream_t s);
cudaError_t launch_sort_init(DeviceStatus* st, uint32_t m, cudaStream_t s);

}  // namespace sgs
