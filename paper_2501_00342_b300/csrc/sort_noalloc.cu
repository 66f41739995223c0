// sgs_sort_pairs_noalloc: the radix sort of sgs_sort_pairs with its scratch memory in a
// fixed, file-scope device array instead of a caller-provided buffer, for callers that
// cannot allocate device memory.
//
// The array below is part of the library image: every GPU that loads the library holds
// it (SGS_SORT_NOALLOC_SCRATCH_BYTES, about 3.3 MB) until the process exits.  In host
// code its name only stands for the device symbol; the device address is looked up once
// per device with cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "sgs.h"

namespace {

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kMaxPairs = (size_t)SGS_SORT_NOALLOC_MAX_PAIRS;
constexpr size_t kMaxLookbackEntries = (kMaxPairs + sgs::kSortTile - 1) / sgs::kSortTile * 256;
// layout: status | alternate keys | alternate values | histograms | offsets | counters | look-back
constexpr size_t kOffKeys = 256;
constexpr size_t kOffVals = kOffKeys + round256(8 * kMaxPairs);
constexpr size_t kOffHist = kOffVals + round256(4 * kMaxPairs);
constexpr size_t kOffGoff = kOffHist + round256(4 * sgs::kMaxSortPasses * 256);
constexpr size_t kOffCounters = kOffGoff + round256(4 * sgs::kMaxSortPasses * 256);
constexpr size_t kOffLookback = kOffCounters + round256(4 * sgs::kMaxSortPasses);
constexpr size_t kScratchBytes = kOffLookback + round256(8 * kMaxLookbackEntries);
static_assert(kScratchBytes == SGS_SORT_NOALLOC_SCRATCH_BYTES, "header and layout disagree");

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    void* ptr = nullptr;
};
DeviceScratch g_device_scratch[kMaxDevices];

// Device address of g_sort_scratch on the current device (looked up on first use).
cudaError_t scratch_on_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    DeviceScratch& d = g_device_scratch[dev];
    std::call_once(d.once, [&d] { d.err = cudaGetSymbolAddress(&d.ptr, g_sort_scratch); });
    if (d.err != cudaSuccess) return d.err;
    *out = static_cast<unsigned char*>(d.ptr);
    return cudaSuccess;
}

}  // namespace

extern "C" sgs_status sgs_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t m,
                                             int32_t key_bits, int32_t digit_bits,
                                             cudaStream_t stream) {
    if (m < 0 || m > (int64_t)kMaxPairs || key_bits < 1 || key_bits > 64 || digit_bits < 4 ||
        digit_bits > 8 || sgs::sort_passes(key_bits, digit_bits) > sgs::kMaxSortPasses)
        return SGS_ERR_INVALID;
    if (m == 0) return SGS_OK;
    if (!keys || !vals) return SGS_ERR_INVALID;
    unsigned char* base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) return SGS_ERR_CUDA;
    sgs::DeviceStatus* st = reinterpret_cast<sgs::DeviceStatus*>(base);
    unsigned long long* k1 = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(base + kOffVals);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    uint32_t* goff = reinterpret_cast<uint32_t*>(base + kOffGoff);
    uint32_t* counters = reinterpret_cast<uint32_t*>(base + kOffCounters);
    unsigned long long* lb = reinterpret_cast<unsigned long long*>(base + kOffLookback);
    unsigned long long* k0 = reinterpret_cast<unsigned long long*>(keys);
    // the status word, histograms, counters and look-back entries the sort reads are
    // written or cleared by launch_sort_init / launch_sort on every call
    if (sgs::launch_sort_init(st, (uint32_t)m, stream) != cudaSuccess) return SGS_ERR_CUDA;
    if (sgs::launch_sort(k0, vals, k1, v1, &st->m_clamped, m, 0, key_bits, digit_bits, hist, goff, counters, lb,
                         st, stream, nullptr) != cudaSuccess)
        return SGS_ERR_CUDA;
    if (sgs::sort_passes(key_bits, digit_bits) & 1)
        if (sgs::launch_copy_pairs(k1, v1, k0, vals, m, stream) != cudaSuccess) return SGS_ERR_CUDA;
    return SGS_OK;
}
