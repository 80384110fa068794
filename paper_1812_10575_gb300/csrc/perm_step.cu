// RBM-1 step on the GPU: random division by a bucketed sort of 64-bit Philox
// keys with an id tie-break, and the in-batch interaction + -grad V +
// Brownian increment + Euler-Maruyama update fused into the sort kernel.
//
// Algorithm "randomdiv" (Sec. 2.1 of arXiv:1812.10575) per step m:
//   1. key_i = Philox(i, m, r, 0); the random division is the id list sorted
//      by (key, id); batch q = sorted positions [q p, min(q p + p, N)).
//   2. every batch C_q moves by eq. "firstalgorithm":
//      X^i += dt (1/(|C_q|-1) sum_{j in C_q, j != i} K(X^i - X^j) - grad V(X^i))
//             + sigma sqrt(dt) z_i.
// The sort runs in two passes over buckets of the top `bucket_bits` key bits:
//   k_bucket_scatter  - one Philox per particle, an atomic slot in its bucket
//                       (overflowing members go to a spill list);
//   k_bucket_sort_step - one block per bucket: regenerate the keys, counting
//                       sort by the next kSubBits key bits in shared memory,
//                       insertion sort of the few members sharing a sub-bucket
//                       by (key, id), write the bucket's stretch of the
//                       permutation, and step every batch that lies wholly
//                       inside the bucket (p <= 32: one group of p lanes per
//                       batch, positions exchanged by warp shuffles).
// Batches that straddle a bucket boundary are stepped afterwards by the last
// block to finish (few buckets) or by k_straddle_fixup (many buckets).  They
// read only positions no other batch writes, so every update uses the
// positions of step m as the explicit scheme requires.
// The random division of a step depends on the step index alone, not on the
// positions: with a double-buffered scratch (buffer m mod 2 for step m), the
// sort kernel of step m can also bucket the ids of step m + 1 (lookahead), so
// that a run of steps needs no k_bucket_scatter launch after its first.
#include <cstdio>

#include "rbm_batch.cuh"
#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {

namespace {

__device__ __forceinline__ uint32_t bucket_of(uint64_t key, int bits) {
  return bits ? static_cast<uint32_t>(key >> (64 - bits)) : 0u;
}

constexpr int kSortThreads = 256;
constexpr int kSortPer = 8;                              // members per thread
constexpr uint32_t kSortCapMax = kSortThreads * kSortPer;  // largest bucket sorted in shared memory
constexpr int kSubBits = 10;
constexpr uint32_t kSub = 1u << kSubBits;                // sub-buckets of a bucket

// The kSubBits key bits below the bucket bits (monotone in the key inside a bucket).
__device__ __forceinline__ uint32_t sub_of(uint64_t key, int bits) {
  return static_cast<uint32_t>((key << bits) >> (64 - kSubBits));
}

struct PermArgs {
  uint32_t* cnt;                // buffer 0; buffer 1 follows each array (double_buffer)
  uint32_t* start;
  uint32_t* slots;
  uint32_t* ovf_cnt;
  uint32_t* ovf;
  uint32_t* done;
  int double_buffer;
  int lookahead;                // the sort kernel also buckets the ids of step m + 1
  uint32_t* perm;
  uint32_t n;
  int bits;
  uint32_t nbuckets;
  uint32_t slot_cap;
  uint32_t sort_cap;
  uint32_t row_cap;             // member rows staged in shared memory by the sort kernel (0: none)
  int separate_scan;
  uint2 seed;
  uint32_t replica;
  const int64_t* m_ptr;
  int64_t m_off;
  const int* skip;
};

__device__ __forceinline__ bool perm_skipped(const PermArgs& a) { return a.skip != nullptr && *a.skip != 0; }

__device__ __forceinline__ uint32_t perm_step_index(const PermArgs& a) {
  const int64_t m = (a.m_ptr ? *a.m_ptr : 0) + a.m_off;
  return static_cast<uint32_t>(static_cast<uint64_t>(m));
}

// The scratch of step m: buffer m mod 2 of a double-buffered scratch.
__device__ __forceinline__ PermArgs for_step(PermArgs a, uint32_t m32) {
  if (a.double_buffer && (m32 & 1u)) {
    a.cnt += a.nbuckets;
    a.start += a.nbuckets;
    a.slots += static_cast<size_t>(a.nbuckets) * a.slot_cap;
    a.ovf_cnt += 1;
    a.ovf += a.n;
    a.done += 1;
  }
  return a;
}

// Id i of step m32 into its bucket's next slot, or the spill list.
__device__ __forceinline__ void scatter_one(const PermArgs& a, uint32_t i, uint32_t m32) {
  const uint64_t key = perm_key(i, m32, a.replica, a.seed);
  const uint32_t b = bucket_of(key, a.bits);
  const uint32_t pos = atomicAdd(&a.cnt[b], 1u);
  if (pos < a.slot_cap) {
    a.slots[static_cast<size_t>(b) * a.slot_cap + pos] = i;
  } else {
    const uint32_t o = atomicAdd(a.ovf_cnt, 1u);  // o < n: the list holds every particle
    a.ovf[o] = i;
  }
}

PermArgs make_perm_args(const PermScratch& ps, uint32_t n, uint2 seed, uint32_t replica, const int64_t* m_ptr,
                        int64_t m_off) {
  PermArgs a;
  a.cnt = ps.cnt; a.start = ps.start; a.slots = ps.slots; a.ovf_cnt = ps.ovf_cnt; a.ovf = ps.ovf;
  a.done = ps.done; a.perm = ps.perm; a.n = n; a.bits = ps.bucket_bits; a.nbuckets = ps.nbuckets;
  a.double_buffer = ps.double_buffer ? 1 : 0; a.lookahead = 0;
  a.slot_cap = ps.slot_cap; a.sort_cap = ps.sort_cap; a.row_cap = 0; a.separate_scan = ps.separate_scan ? 1 : 0;
  a.seed = seed; a.replica = replica; a.m_ptr = m_ptr; a.m_off = m_off; a.skip = ps.skip;
  return a;
}

// ---------------------------------------------------------------------------
// Pass 1: bucket every particle by the top bits of its key.
// ---------------------------------------------------------------------------
__global__ void k_bucket_scatter(PermArgs pa_in) {
  if (perm_skipped(pa_in)) return;
  const uint32_t m32 = perm_step_index(pa_in);
  const PermArgs a = for_step(pa_in, m32);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) scatter_one(a, i, m32);
}

// Exclusive scan of the bucket counts by one block (many-bucket case): each
// thread sums a run of consecutive counters, the block scans the run totals,
// then each thread writes its run's starts (two block barriers in all).
__global__ void __launch_bounds__(1024) k_bucket_scan(PermArgs pa_in) {
  if (perm_skipped(pa_in)) return;
  const PermArgs a = for_step(pa_in, perm_step_index(pa_in));
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t per = (a.nbuckets + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(a.nbuckets, threadIdx.x * per), hi = min(a.nbuckets, lo + per);
  uint32_t sum = 0;
  for (uint32_t b = lo; b < hi; ++b) sum += a.cnt[b];
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < nwarps) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nwarps) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t run = ((warp > 0) ? s_warp[warp - 1] : 0u) + incl - sum;
  for (uint32_t b = lo; b < hi; ++b) {
    const uint32_t v = a.cnt[b];
    a.start[b] = run;
    run += v;
  }
}

// Sum of v over the block, returned to every thread.
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w];
  return t;
}

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Exclusive scan of a[0, kSub) in shared memory by the whole block.
__device__ void sub_exclusive_scan(uint32_t* a, uint32_t* s_warp) {
  constexpr uint32_t per = kSub / kSortThreads;
  const uint32_t lo = threadIdx.x * per;
  uint32_t v[per];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    v[i] = a[lo + i];
    sum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t run = incl - sum;
  run += warps_before(s_warp, warp, lane);
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    a[lo + i] = run;
    run += v[i];
  }
  __syncthreads();
}

// Steps the batches that straddle bucket boundaries b in [b_begin, b_end)
// (each batch once: from the first boundary strictly inside it).
template <typename T, int D, int MODE>
__device__ void step_straddling(const StepParams<T>& a, uint32_t m32, const PermArgs& pa, uint32_t b_begin,
                                uint32_t b_end, uint32_t b_stride_groups, uint32_t group_offset) {
  const int p = a.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / p;
  const int nwarps = blockDim.x >> 5;
  const int g = lane / p, lg = lane - g * p;
  const uint32_t per_round = static_cast<uint32_t>(gpw * nwarps);
  for (uint32_t r0 = b_begin; r0 < b_end; r0 += per_round * b_stride_groups) {
    const uint32_t b = r0 + (group_offset + static_cast<uint32_t>(warp * gpw + g)) ;
    bool valid = (g < gpw) && (b < b_end) && (b > 0);
    uint32_t id = 0;
    int bs = p;
    if (valid) {
      const uint32_t s = pa.start[b];
      const uint32_t up = static_cast<uint32_t>(p);
      valid = (s % up != 0) && (s < a.n);
      if (valid) {
        const uint32_t q = s / up;
        valid = pa.start[b - 1] <= q * up;      // first boundary inside batch q
        if (valid) {
          const uint32_t lo = q * up, hi = min(lo + up, a.n);
          bs = static_cast<int>(hi - lo);
          valid = lg < bs;
          if (valid) id = pa.perm[lo + lg];
        }
      }
    }
    batch_group<T, D, MODE>(a, m32, id, valid, lg, bs);
  }
}

// Asynchronous copy of one position row (4, 8, 16 or 32 bytes) from global
// into shared memory (cp.async; 16-byte pieces bypass L1).
template <typename T, int D>
__device__ __forceinline__ void cp_async_row(unsigned char* dst, const T* src) {
  constexpr int kBytes = Ld<D>::value * static_cast<int>(sizeof(T));
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if constexpr (kBytes == 32) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + 16u), "l"(src + 2) : "memory");
  } else if constexpr (kBytes == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(src), "n"(kBytes) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// As step_batches, with each member's row taken from the block's staging
// area when it was staged there (slot index below nstage) and from the
// position array otherwise.
template <typename T, int D, int MODE>
__device__ __forceinline__ void step_batches_staged(const StepParams<T>& a, uint32_t m32, const uint32_t* ids,
                                                    const uint16_t* slot_of, const unsigned char* srow,
                                                    uint32_t nstage, uint32_t ids_base, uint32_t q0, uint32_t count) {
  const int p = a.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / p;
  const int nwarps = blockDim.x >> 5;
  const uint32_t per_round = static_cast<uint32_t>(gpw * nwarps);
  const int g = lane / p, lg = lane - g * p;
  const T* staged = reinterpret_cast<const T*>(srow);
  for (uint32_t r0 = 0; r0 < count; r0 += per_round) {
    const uint32_t kb = r0 + static_cast<uint32_t>(warp * gpw + g);
    bool valid = (g < gpw) && (kb < count);
    uint32_t id = 0;
    int bs = p;
    Row<T, D> r{};
    if (valid) {
      const uint32_t q = q0 + kb;
      const uint32_t lo = q * static_cast<uint32_t>(p);
      const uint32_t hi = min(lo + static_cast<uint32_t>(p), a.n);
      bs = static_cast<int>(hi - lo);
      valid = lg < bs;
      if (valid) {
        const uint32_t pos = lo + lg - ids_base;
        id = ids[pos];
        const uint32_t t = slot_of[pos];
        r = (t < nstage) ? load_row<T, D>(staged, t) : load_row<T, D>(a.x, id);
      }
    }
    batch_group_row<T, D, MODE>(a, m32, id, valid, lg, bs, r);
  }
}

// ---------------------------------------------------------------------------
// Pass 2: one block per bucket.
// ---------------------------------------------------------------------------
// Four blocks per SM (registers capped at 64; a few bytes spill): at N = 2^24
// 722 us per step against 795 us with three.
// The rows of a bucket's members are fetched into shared memory by cp.async
// as soon as their ids are read, before the keys are regenerated and sorted,
// so every block keeps its whole bucket of random row reads in flight while
// it sorts (the random gathers are the step's DRAM latency).
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(kSortThreads, 4) k_bucket_sort_step(PermArgs pa_in, StepParams<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr uint32_t kRowBytes = Ld<D>::value * sizeof(T);
  unsigned char* srow = smem_raw;                                  // [row_cap] staged rows, by slot index
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem_raw + static_cast<size_t>(pa_in.row_cap) * kRowBytes);
  uint32_t* sid = reinterpret_cast<uint32_t*>(skey + pa_in.sort_cap);  // [sort_cap] ids, sorted
  uint16_t* sslot = reinterpret_cast<uint16_t*>(sid + pa_in.sort_cap); // [sort_cap] slot index of each sorted id
  uint32_t* ssub = reinterpret_cast<uint32_t*>(sslot + pa_in.sort_cap);  // [kSub] sub-bucket counts, then starts
  __shared__ uint32_t s_red[32];
  __shared__ uint32_t s_fill;
  __shared__ int s_last;
  if (perm_skipped(pa_in)) return;

  const uint32_t b = blockIdx.x;
  const uint32_t m32 = perm_step_index(pa_in);
  const PermArgs pa = for_step(pa_in, m32);

  uint32_t start;
  if (pa.separate_scan) {
    start = pa.start[b];
  } else {
    uint32_t part = 0;
    for (uint32_t t = threadIdx.x; t < b; t += blockDim.x) part += pa.cnt[t];
    start = block_sum(part, s_red);
    if (threadIdx.x == 0) pa.start[b] = start;
  }
  const uint32_t nb = pa.cnt[b];
  const uint32_t nslot = min(nb, pa.slot_cap);
  const uint32_t nstage = (MODE != kModePerm) ? min(nslot, pa.row_cap) : 0u;
  const uint32_t* ids;
  const bool fits = nb <= pa.sort_cap;

  if (fits) {
    for (uint32_t u = threadIdx.x; u < kSub; u += blockDim.x) ssub[u] = 0;
    if (nb > nslot) {  // members that spilled to the overflow list, staged after the slot members
      if (threadIdx.x == 0) s_fill = nslot;
      __syncthreads();
      const uint32_t novf = *pa.ovf_cnt;
      for (uint32_t t = threadIdx.x; t < novf; t += blockDim.x) {
        const uint32_t id = pa.ovf[t];
        if (bucket_of(perm_key(id, m32, pa.replica, pa.seed), pa.bits) == b) sid[atomicAdd(&s_fill, 1u)] = id;
      }
    }
    __syncthreads();
  }
  uint64_t key[kSortPer];
  uint32_t idr[kSortPer], subr[kSortPer];
  if (fits) {
    // ids, then every staged member's row in flight, then the keys
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
      const uint32_t t = threadIdx.x + k * kSortThreads;
      if (t < nb) idr[k] = (t < nslot) ? pa.slots[static_cast<size_t>(b) * pa.slot_cap + t] : sid[t];
    }
    if (MODE != kModePerm) {
#pragma unroll
      for (int k = 0; k < kSortPer; ++k) {
        const uint32_t t = threadIdx.x + k * kSortThreads;
        if (t < nstage) cp_async_row<T, D>(srow + t * kRowBytes, a.x + static_cast<size_t>(idr[k]) * Ld<D>::value);
      }
      cp_async_commit();
    }
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
      const uint32_t t = threadIdx.x + k * kSortThreads;
      if (t < nb) {
        key[k] = perm_key(idr[k], m32, pa.replica, pa.seed);
        const uint32_t sub = sub_of(key[k], pa.bits);
        subr[k] = sub | (atomicAdd(&ssub[sub], 1u) << 16);
      }
    }
  }
  if (pa_in.lookahead) {
    // bucket this block's share of the ids for step m + 1 (the other buffer)
    // while this bucket's rows are in flight
    const PermArgs nx = for_step(pa_in, m32 + 1u);
    const uint32_t chunk = (pa.n + gridDim.x - 1) / gridDim.x;
    const uint32_t i0 = min(pa.n, b * chunk), i1 = min(pa.n, i0 + chunk);
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) scatter_one(nx, i, m32 + 1u);
  }

  if (fits) {
    __syncthreads();
    sub_exclusive_scan(ssub, s_red);
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
      const uint32_t t = threadIdx.x + k * kSortThreads;
      if (t < nb) {
        const uint32_t pos = ssub[subr[k] & 0xffffu] + (subr[k] >> 16);
        skey[pos] = key[k];
        sid[pos] = idr[k];
        sslot[pos] = static_cast<uint16_t>(t);
      }
    }
    __syncthreads();
    for (uint32_t u = threadIdx.x; u < kSub; u += blockDim.x) {  // insertion sort of each sub-bucket
      const uint32_t lo = ssub[u], hi = (u + 1 < kSub) ? ssub[u + 1] : nb;
      for (uint32_t x = lo + 1; x < hi; ++x) {
        const uint64_t kx = skey[x];
        const uint32_t ix = sid[x];
        const uint16_t tx = sslot[x];
        uint32_t y = x;
        while (y > lo && key_less(kx, ix, skey[y - 1], sid[y - 1])) {
          skey[y] = skey[y - 1];
          sid[y] = sid[y - 1];
          sslot[y] = sslot[y - 1];
          --y;
        }
        skey[y] = kx;
        sid[y] = ix;
        sslot[y] = tx;
      }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) pa.perm[start + t] = sid[t];
    ids = sid;
  } else {
    // Rare: a bucket larger than the shared-memory sort.  Rank every member by
    // counting the members before it in (key, id) order.
    const uint32_t novf = (nb > nslot) ? *pa.ovf_cnt : 0u;
    const uint32_t total = nslot + novf;
    for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
      const uint32_t ide = (e < nslot) ? pa.slots[static_cast<size_t>(b) * pa.slot_cap + e] : pa.ovf[e - nslot];
      const uint64_t ke = perm_key(ide, m32, pa.replica, pa.seed);
      if (e >= nslot && bucket_of(ke, pa.bits) != b) continue;
      uint32_t rank = 0;
      for (uint32_t f = 0; f < total; ++f) {
        const uint32_t idf = (f < nslot) ? pa.slots[static_cast<size_t>(b) * pa.slot_cap + f] : pa.ovf[f - nslot];
        const uint64_t kf = perm_key(idf, m32, pa.replica, pa.seed);
        if (f >= nslot && bucket_of(kf, pa.bits) != b) continue;
        rank += key_less(kf, idf, ke, ide) ? 1u : 0u;
      }
      pa.perm[start + rank] = ide;
    }
    __syncthreads();
    ids = pa.perm + start;
  }

  if (MODE != kModePerm) {
    if (fits) cp_async_wait_all();
    __syncthreads();
    const uint32_t up = static_cast<uint32_t>(a.p);
    const uint32_t end = start + nb;
    const uint32_t q0 = (start + up - 1) / up;
    const uint32_t q_end = (end == a.n) ? (a.n + up - 1) / up : end / up;
    const uint32_t count = (q_end > q0) ? q_end - q0 : 0u;
    if (fits) step_batches_staged<T, D, MODE>(a, m32, ids, sslot, srow, nstage, start, q0, count);
    else step_batches<T, D, MODE>(a, m32, ids, start, q0, count);
  }

  if (pa.separate_scan) {
    __syncthreads();
    if (threadIdx.x == 0) pa.cnt[b] = 0;  // ready for the next step
    return;
  }

  // Last block to finish: straddling batches and the counter reset.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(pa.done, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (MODE != kModePerm) step_straddling<T, D, MODE>(a, m32, pa, 0, pa.nbuckets, 1, 0);
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < pa.nbuckets; t += blockDim.x) pa.cnt[t] = 0;
  if (threadIdx.x == 0) {
    *pa.ovf_cnt = 0;
    *pa.done = 0;
  }
}

// Many-bucket case: straddling batches over a grid, then the spill counter reset.
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) k_straddle_fixup(PermArgs pa_in, StepParams<T> a) {
  if (perm_skipped(pa_in)) return;
  const uint32_t m32 = perm_step_index(pa_in);
  const PermArgs pa = for_step(pa_in, m32);
  const int gpw = 32 / a.p;
  const uint32_t per_block = static_cast<uint32_t>(gpw * (blockDim.x >> 5));
  if (MODE != kModePerm)
    step_straddling<T, D, MODE>(a, m32, pa, 0, pa.nbuckets, gridDim.x, blockIdx.x * per_block);
  if (blockIdx.x == 0 && threadIdx.x == 0) *pa.ovf_cnt = 0;
}

// Batches larger than a warp (p > 32): one block per batch, all members'
// new positions staged in xout before any is written back.
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) k_batch_generic(PermArgs pa, StepParams<T> a) {
  if (perm_skipped(pa)) return;
  const uint32_t m32 = step_index(a);
  const uint32_t up = static_cast<uint32_t>(a.p);
  const uint32_t lo = blockIdx.x * up;
  const uint32_t hi = min(lo + up, a.n);
  const uint32_t bs = hi - lo;
  const T inv = (bs > 1) ? T(1) / static_cast<T>(bs - 1) : T(0);
  for (uint32_t e = threadIdx.x; e < bs; e += blockDim.x) {
    const uint32_t id = pa.perm[lo + e];
    Row<T, D> r = load_row<T, D>(a.x, id);
    T fk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) fk[k] = T(0);
    for (uint32_t f = 0; f < bs; ++f) {
      if (f == e) continue;
      const Row<T, D> o = load_row<T, D>(a.x, pa.perm[lo + f]);
      add_pair_force_rt<T, D>(a.kf, a.kparam, a.radius_sq, r.x, o.x, fk);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) fk[k] = (bs > 1) ? fk[k] * inv : T(0);
    if (MODE == kModeForces) {
      Row<T, D> f;
#pragma unroll
      for (int k = 0; k < D; ++k) f.x[k] = fk[k];
      f.pad = T(0);
      store_row<T, D>(a.fout, id, f);
    } else {
      T y[D];
      scheme_update<T, D>(a, id, m32, r.x, fk, y);
#pragma unroll
      for (int k = 0; k < D; ++k) r.x[k] = y[k];
      store_row<T, D>(a.xout, lo + e, r);
    }
  }
  if (MODE != kModeStep) return;
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < bs; e += blockDim.x)
    store_row<T, D>(a.x, pa.perm[lo + e], load_row<T, D>(a.xout, lo + e));
}

__global__ void k_set_i64(int64_t* dst, int64_t v) { *dst = v; }
__global__ void k_add_i64(int64_t* dst, int64_t v) { *dst += v; }

// Dynamic shared memory of the sort kernel: row_cap staged rows of row_bytes,
// then keys, ids and slot indices of up to sort_cap members, then the
// sub-bucket counters.
size_t sort_smem_bytes(uint32_t sort_cap, uint32_t row_cap, uint32_t row_bytes) {
  return static_cast<size_t>(row_cap) * row_bytes +
         static_cast<size_t>(sort_cap) * (sizeof(uint64_t) + sizeof(uint32_t) + sizeof(uint16_t)) +
         kSub * sizeof(uint32_t);
}

// Rows staged per bucket: every slot member, at most one per sort position,
// rounded up to 16 rows.
uint32_t staged_rows(const PermScratch& ps) {
  const uint32_t cap = ((ps.slot_cap + 15u) / 16u) * 16u;
  return cap < kSortCapMax ? cap : kSortCapMax;
}

template <typename T, int D>
void launch_tail_d(const PermScratch& ps, int mode, const StepParams<T>& a, bool lookahead, const LaunchCfg& cfg,
                   cudaStream_t st) {
  PermArgs pa = make_perm_args(ps, a.n, a.seed, a.replica, a.m_ptr, a.m_off);
  pa.lookahead = (lookahead && ps.double_buffer) ? 1 : 0;
  const bool small_p = a.p <= 32;
  const int kmode = small_p ? mode : kModePerm;
  pa.row_cap = (kmode == kModePerm) ? 0u : staged_rows(ps);
  const size_t smem = sort_smem_bytes(ps.sort_cap, pa.row_cap, Ld<D>::value * sizeof(T));
  const int block = kSortThreads;
  if (ps.separate_scan) {
    k_bucket_scan<<<1, 1024, 0, st>>>(pa);
    mark_launch(cfg, st, "k_bucket_scan");
  }
  auto launch_sort = [&](auto kern) { kern<<<ps.nbuckets, kSortThreads, smem, st>>>(pa, a); };
  if (kmode == kModeStep) launch_sort(k_bucket_sort_step<T, D, kModeStep>);
  else if (kmode == kModeForces) launch_sort(k_bucket_sort_step<T, D, kModeForces>);
  else launch_sort(k_bucket_sort_step<T, D, kModePerm>);
  mark_launch(cfg, st, "k_bucket_sort_step");
  if (ps.separate_scan) {
    const int gpw = small_p ? 32 / a.p : 1;
    const uint32_t per_block = static_cast<uint32_t>(gpw * (block / 32));
    const uint32_t grid = max(1u, (ps.nbuckets + per_block - 1) / per_block);
    if (kmode == kModeStep) k_straddle_fixup<T, D, kModeStep><<<grid, block, 0, st>>>(pa, a);
    else if (kmode == kModeForces) k_straddle_fixup<T, D, kModeForces><<<grid, block, 0, st>>>(pa, a);
    else k_straddle_fixup<T, D, kModePerm><<<1, 32, 0, st>>>(pa, a);
    mark_launch(cfg, st, "k_straddle_fixup");
  }
  if (!small_p && mode != kModePerm) {
    const uint32_t nbatch = (a.n + a.p - 1) / a.p;
    if (mode == kModeStep) k_batch_generic<T, D, kModeStep><<<nbatch, block, 0, st>>>(pa, a);
    else k_batch_generic<T, D, kModeForces><<<nbatch, block, 0, st>>>(pa, a);
    mark_launch(cfg, st, "k_batch_generic");
  }
}

}  // namespace

void launch_bucket_scatter(const PermScratch& ps, uint32_t n, uint2 seed, uint32_t replica, const int64_t* m_ptr,
                           int64_t m_off, const LaunchCfg& cfg, cudaStream_t st) {
  const PermArgs pa = make_perm_args(ps, n, seed, replica, m_ptr, m_off);
  const int block = 256;
  const uint32_t want = (n + block - 1) / block;
  const uint32_t grid = max(1u, min(want, static_cast<uint32_t>(cfg.num_sms * 8)));
  k_bucket_scatter<<<grid, block, 0, st>>>(pa);
  mark_launch(cfg, st, "k_bucket_scatter");
}

template <typename T>
void launch_rbm_tail(const PermScratch& ps, int d, int mode, const void* params, bool lookahead, const LaunchCfg& cfg,
                     cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  if (d == 1) launch_tail_d<T, 1>(ps, mode, a, lookahead, cfg, st);
  else if (d == 2) launch_tail_d<T, 2>(ps, mode, a, lookahead, cfg, st);
  else launch_tail_d<T, 3>(ps, mode, a, lookahead, cfg, st);
}

template void launch_rbm_tail<float>(const PermScratch&, int, int, const void*, bool, const LaunchCfg&,
                                     cudaStream_t);
template void launch_rbm_tail<double>(const PermScratch&, int, int, const void*, bool, const LaunchCfg&,
                                      cudaStream_t);

uint32_t max_sort_cap() { return kSortCapMax; }

int rbm_tail_launches(const PermScratch& ps, int p) {
  int n = 1;                      // sort (+ fused step)
  if (ps.separate_scan) n += 2;   // scan, straddle fix-up
  if (p > 32) n += 1;             // generic batch kernel
  return n;
}

namespace {
template <typename T, int D>
cudaError_t allow_sort_smem_d(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_bucket_sort_step<T, D, kModePerm>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bucket_sort_step<T, D, kModeStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bucket_sort_step<T, D, kModeForces>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  return e;
}
}  // namespace

cudaError_t prepare_rbm_kernels() {
  // The largest shared-memory sort with the largest staged rows (32-byte
  // rows of d = 3 FP64) plus static shared data.
  const int bytes = static_cast<int>(sort_smem_bytes(kSortCapMax, kSortCapMax, 32)) + 1024;
  cudaError_t e = allow_sort_smem_d<float, 1>(bytes);
  if (e == cudaSuccess) e = allow_sort_smem_d<float, 2>(bytes);
  if (e == cudaSuccess) e = allow_sort_smem_d<float, 3>(bytes);
  if (e == cudaSuccess) e = allow_sort_smem_d<double, 1>(bytes);
  if (e == cudaSuccess) e = allow_sort_smem_d<double, 2>(bytes);
  if (e == cudaSuccess) e = allow_sort_smem_d<double, 3>(bytes);
  return e;
}

void launch_set_i64(int64_t* dst, int64_t value, cudaStream_t st) { k_set_i64<<<1, 1, 0, st>>>(dst, value); }
void launch_add_i64(int64_t* dst, int64_t value, cudaStream_t st) { k_add_i64<<<1, 1, 0, st>>>(dst, value); }

}  // namespace rbm
