// rbm_permutation_noalloc: the random division of one step computed without
// allocating any memory.
//
// The regular entry points allocate their scratch with cudaMalloc in
// rbm_init.  Some callers cannot do that: a host application whose memory
// manager owns every byte of device memory (a framework's caching allocator,
// a fixed budget that an extra cudaMalloc would break), or a real-time loop
// that must never block on, or fail in, an allocation.  This entry point
// serves them: its scratch (bucket counters, bucket slots, the spill list,
// the finished-block ticket) is a file-scope device array of fixed size that
// every GPU loading the library holds until the process exits, and the
// caller passes only the output buffer.
//
// Limits and sharing:
//   - at most kNoAllocMaxN = 65536 particles; larger n is rejected with
//     RBM_ERR_INVALID and rbm_last_error() says why;
//   - every call on a device uses the same array and the array keeps the last
//     call's contents; each call clears the counters it needs at its start,
//     on its stream, so back-to-back calls are fine, but calls whose work
//     overlaps on the GPU (two streams, or two host threads) race on the
//     array and give wrong permutations;
//   - a call looks up the array's device address with cudaGetSymbolAddress
//     (with that device current) whenever its stream is not capturing, so
//     the address stays right after a cudaDeviceReset reloads the module; a
//     call made while the stream is being captured reuses the address of the
//     last call on that device, so make one call on the device before any
//     stream capture.
#include <cstdio>
#include <mutex>

#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr uint32_t kNoAllocMaxN = 1u << 16;
constexpr int kNoAllocBucketBits = 7;                  // 128 buckets: at most 512 members on average
constexpr uint32_t kNoAllocBuckets = 1u << kNoAllocBucketBits;
constexpr uint32_t kNoAllocSlotCap = 768;              // mean 512 + 8 sqrt(512) + 64, rounded up
constexpr uint32_t kNoAllocSortCap = 2048;

// Word offsets of the pieces inside the array.
constexpr size_t kOffCnt = 0;
constexpr size_t kOffStart = kOffCnt + kNoAllocBuckets;
constexpr size_t kOffOvfCnt = kOffStart + kNoAllocBuckets;
constexpr size_t kOffDone = kOffOvfCnt + 1;
constexpr size_t kOffOvf = 64 * ((kOffDone + 1 + 63) / 64);                // 256-byte aligned
constexpr size_t kOffSlots = kOffOvf + kNoAllocMaxN;
constexpr size_t kScratchWords = kOffSlots + static_cast<size_t>(kNoAllocBuckets) * kNoAllocSlotCap;

// About 650 KB per device.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device: looked up again on
// every call outside stream capture (a device reset reloads the module and
// may move it), taken from the last lookup on that device during capture.
cudaError_t scratch_on_current_device(cudaStream_t st, uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<uint32_t*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rbm

using namespace rbm;

extern "C" rbm_status rbm_permutation_noalloc(int64_t n, uint64_t seed, uint32_t replica, int64_t m,
                                              uint32_t* perm_dev, void* cuda_stream) {
  if (n > static_cast<int64_t>(kNoAllocMaxN)) {
    char msg[160];
    snprintf(msg, sizeof(msg), "rbm_permutation_noalloc: n = %lld exceeds the maximum of %u particles",
             static_cast<long long>(n), kNoAllocMaxN);
    set_last_error_text(msg);
    return RBM_ERR_INVALID;
  }
  if (n < 2) {
    set_last_error_text("rbm_permutation_noalloc: n must be at least 2");
    return RBM_ERR_INVALID;
  }
  if (m < 0) {
    set_last_error_text("rbm_permutation_noalloc: the step index m must not be negative");
    return RBM_ERR_INVALID;
  }
  if (!perm_dev) {
    set_last_error_text("rbm_permutation_noalloc: perm_dev is a null pointer");
    return RBM_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t* base = nullptr;
  cudaError_t e = scratch_on_current_device(st, &base);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    set_last_error_text(msg);
    return RBM_ERR_CUDA;
  }

  PermScratch ps;
  ps.cnt = base + kOffCnt;
  ps.start = base + kOffStart;
  ps.ovf_cnt = base + kOffOvfCnt;
  ps.done = base + kOffDone;
  ps.ovf = base + kOffOvf;
  ps.slots = base + kOffSlots;
  ps.perm = perm_dev;
  int bits = 0;
  while (bits < kNoAllocBucketBits && (static_cast<uint64_t>(n) >> bits) > 512) ++bits;
  ps.bucket_bits = bits;
  ps.nbuckets = 1u << bits;
  ps.slot_cap = kNoAllocSlotCap < static_cast<uint32_t>(n) ? kNoAllocSlotCap : static_cast<uint32_t>(n);
  ps.sort_cap = kNoAllocSortCap;
  ps.separate_scan = false;

  // The counters, the spill count and the ticket must start at zero.
  e = cudaMemsetAsync(base, 0, sizeof(uint32_t) * kOffOvf, st);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "cudaMemsetAsync: %s", cudaGetErrorString(e));
    set_last_error_text(msg);
    return RBM_ERR_CUDA;
  }
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  LaunchCfg cfg;
  launch_bucket_scatter(ps, static_cast<uint32_t>(n), key, replica, nullptr, m, cfg, st);
  StepParams<float> a{};
  a.n = static_cast<uint32_t>(n);
  a.p = 2;
  a.seed = key;
  a.replica = replica;
  a.m_ptr = nullptr;
  a.m_off = m;
  launch_rbm_tail<float>(ps, 1, /*mode: permutation only*/ 0, &a, false, cfg, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "kernel launch: %s", cudaGetErrorString(e));
    set_last_error_text(msg);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}
