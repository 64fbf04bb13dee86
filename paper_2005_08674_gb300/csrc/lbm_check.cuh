// lbm_check.cuh -- the bounds-checked build of the library (compiled with
// -DLBM_CHECK into liblbm_check.so), a stand-in for a device memory checker.
//
// In that build every global access of the step kernels (the storage
// accessors, the cp.async.bulk tile copies and the L2 prefetches) first asks
// in_bounds() whether the whole access lies inside one population buffer
// registered by the host, and every shared-memory slot access asks
// in_slot() whether it lies inside its slot.  An access that fails is not
// made: a load yields zero, a store or copy is dropped.  The failure is
// counted and the first failing address kept in device memory, and
// lbm_check_read() reports them, so the test of this build can assert that
// a run made none -- without any access ever leaving its buffer, and without
// a trap.  In the ordinary build both checks are the constant true and
// compile away.
//
// There is no relocatable device code, so every translation unit has its own
// copy of the device-side table; each .cu file registers the buffers its own
// kernels touch (check_add / check_remove), on the current device.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace lbmk {

#ifdef LBM_CHECK

struct CheckRange {
  unsigned long long lo, hi;  // [lo, hi) in bytes
};
constexpr int kCheckRanges = 64;

static __device__ CheckRange g_check_ranges[kCheckRanges];
static __device__ int g_check_n;
static __device__ unsigned long long g_check_count;
static __device__ unsigned long long g_check_first;

__device__ __forceinline__ void check_fail(unsigned long long what) {
  if (atomicAdd(&g_check_count, 1ull) == 0ull) g_check_first = what;
}

// True if [p, p + bytes) lies inside one registered buffer.
__device__ __forceinline__ bool in_bounds(const void* p, unsigned long long bytes) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  const int n = g_check_n;
  for (int r = 0; r < n; ++r)
    if (a >= g_check_ranges[r].lo && a + bytes <= g_check_ranges[r].hi) return true;
  check_fail(a);
  return false;
}

// True if bytes [off, off + bytes) lie inside a shared-memory slot of `size`
// bytes (a failure is recorded with the top bit set and the offset).
__device__ __forceinline__ bool in_slot(long long off, long long bytes, long long size) {
  if (off >= 0 && off + bytes <= size) return true;
  check_fail(0x8000000000000000ull | (unsigned long long)(off & 0x7fffffffffffffffll));
  return false;
}

// Host side: this translation unit's registry, mirrored into its device table.
struct CheckRegistry {
  std::mutex mu;
  std::vector<CheckRange> ranges;
  void upload() {
    cudaDeviceSynchronize();  // no kernel of this unit reads the table meanwhile
    const int n = (int)ranges.size();
    if (n) cudaMemcpyToSymbol(g_check_ranges, ranges.data(), n * sizeof(CheckRange));
    cudaMemcpyToSymbol(g_check_n, &n, sizeof n);
  }
};

static CheckRegistry& check_registry() {
  static CheckRegistry r;
  return r;
}

// LBM_CHECK_SHRINK=<bytes> registers every buffer that many bytes short, so
// that the test of this build can see the checker reject accesses (to memory
// that is still valid: the rejected access is simply not made).
static void check_add(const void* p, size_t bytes) {
  if (!p) return;
  const char* s = std::getenv("LBM_CHECK_SHRINK");
  const size_t shrink = s ? (size_t)std::strtoull(s, nullptr, 10) : 0;
  CheckRegistry& r = check_registry();
  std::lock_guard<std::mutex> lk(r.mu);
  if ((int)r.ranges.size() >= kCheckRanges) return;  // table full: later buffers are reported as violations
  const unsigned long long lo = reinterpret_cast<unsigned long long>(p);
  r.ranges.push_back({lo, lo + (bytes > shrink ? bytes - shrink : 0)});
  r.upload();
}

static void check_remove(const void* p) {
  if (!p) return;
  CheckRegistry& r = check_registry();
  std::lock_guard<std::mutex> lk(r.mu);
  const unsigned long long lo = reinterpret_cast<unsigned long long>(p);
  for (size_t k = 0; k < r.ranges.size(); ++k)
    if (r.ranges[k].lo == lo) {
      r.ranges.erase(r.ranges.begin() + (long)k);
      r.upload();
      return;
    }
}

// Count and first failing address of this unit's checks since the last reset.
static void check_read(unsigned long long* count, unsigned long long* first, bool reset) {
  cudaDeviceSynchronize();
  cudaMemcpyFromSymbol(count, g_check_count, sizeof *count);
  cudaMemcpyFromSymbol(first, g_check_first, sizeof *first);
  if (reset) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_check_count, &z, sizeof z);
    cudaMemcpyToSymbol(g_check_first, &z, sizeof z);
  }
}

constexpr bool kChecked = true;

#else

__device__ __forceinline__ constexpr bool in_bounds(const void*, unsigned long long) { return true; }
__device__ __forceinline__ constexpr bool in_slot(long long, long long, long long) { return true; }
static inline void check_add(const void*, size_t) {}
static inline void check_remove(const void*) {}
static inline void check_read(unsigned long long* count, unsigned long long* first, bool) {
  *count = 0;
  *first = 0;
}
constexpr bool kChecked = false;

#endif

}  // namespace lbmk
