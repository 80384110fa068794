// Grid-wide barrier of a cooperative launch (all blocks co-resident), with a
// bounded wait.
#pragma once

#include <cstdint>

#include "rbm_device.cuh"

namespace rbm {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// Barrier on a monotonic arrival counter: the G arrivals of one barrier
// occupy counter values [t - G, t), t a multiple of G, so each block's thread
// 0 arrives with an acquire-release add and polls (acquire) until the counter
// reaches the next multiple of G.  Returns false (every thread of the block)
// when the wait ran out, RBM_ERR_TIMEOUT latched, or when `leave` asks this
// block to leave without arriving.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long wait_ns, int32_t* status,
                                             bool leave) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (leave) {
      ok = 0;
    } else {
      const unsigned long long g = gridDim.x;
      const unsigned long long old = atom_add_acq_rel_gpu(bar, 1ull);
      const unsigned long long target = (old / g + 1ull) * g;
      if (old + 1ull != target) {
        const unsigned long long t0 = global_ns();
        // The iteration bound holds even if the timer were not advancing.
        const unsigned long long max_iter = wait_ns / 8 + 4096;
        unsigned long long iter = 0;
        while (ld_acquire_gpu(bar) < target) {
          ++iter;
          if (iter > 2048) __nanosleep(32);
          if (iter >= max_iter || ((iter & 63u) == 0 && global_ns() - t0 > wait_ns)) {
            ok = 0;
            latch_status(status, RBM_ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace rbm
