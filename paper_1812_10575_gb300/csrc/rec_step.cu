// RBM-1 steps of large systems with the positions moving through the step
// as records, so that every pass over the state streams through DRAM in
// runs instead of gathering random rows.
//
// Algorithm "randomdiv" (Sec. 2.1 of arXiv:1812.10575) per step m: the ids
// sorted by (key, id), key = Philox(id, m, r, 0), batch q = sorted positions
// [q p, min(q p + p, N)), each batch moved by eq. "firstalgorithm".  The sort
// is a two-level bucketing by the top key bits followed by a sort of each
// small bucket in shared memory; here the buckets carry the particles' rows,
// not their ids:
//   record    = the row (x, y, z, id in the pad lane) and 32 key bits (the
//               bits below the top-level digit);
//   top level = 2^top_bits buckets by the top key bits, fixed-capacity
//               regions; each writer groups its records by bucket in shared
//               memory, reserves one run per bucket it feeds (one atomic per
//               block and bucket) and stores each run with consecutive
//               threads on consecutive rows, so records land in runs of tens
//               of rows;
//   sub level = 2^sub_bits sub-buckets per top bucket by the next key bits,
//               filled the same way by k_rec_split;
//   k_rec_scan   - the sorted start of every sub-bucket (the sub-buckets in
//                  (top, sub) order are the random division in key order);
//   k_rec_step   - one block per sub-bucket (about 2048 records, the rows
//                  of the sub-bucket a block one wave later takes prefetched
//                  into L2): sort by the remaining key bits (counting sort on
//                  11 bits, then each record ranked among the few sharing its
//                  digit, full keys recomputed only on ties of the carried
//                  bits), step every batch lying wholly inside it, park
//                  the members of batches crossing its ends, and send every
//                  moved record to its top-level bucket of step m + 1 (key
//                  of m + 1 computed here) - or, at the last step of a run,
//                  to its id-range bucket (about N / ntop consecutive ids);
//   k_rec_fixup  - the batches crossing sub-bucket ends, from the parked
//                  members, sent on the same way (written by id at the last
//                  step);
//   k_rec_place  - after the last step, the records of each id-range bucket
//                  to the caller's array by id, consecutive blocks on one
//                  bucket so that the rows being written stay in L2 until
//                  their sectors are complete.
// A run of K steps starts with k_rec_scatter, which reads the caller's array
// in id order and fills the top level of its first step; the caller's array
// holds the positions again after the run's last step.  Every update reads
// the positions of step m only (batches are disjoint), as the explicit scheme
// requires.  Capacities are the mean count plus twelve standard deviations
// of the binomial count (and a constant); a count beyond one (never seen for
// Philox keys) latches RBM_ERR_STATE and nothing is written past the region.
#include <algorithm>
#include <cmath>

#include "rbm_batch.cuh"
#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr uint32_t kSubTarget = 2048;   // mean records per sub-bucket
constexpr uint32_t kSubCapMax = 3072;   // largest sub-bucket sorted in shared memory
constexpr int kStepThreads = 512;
constexpr int kStepPer = kSubCapMax / kStepThreads;  // records per thread of k_rec_step
constexpr int kSplitThreads = 512;
constexpr int kSplitPer = 8;            // records per thread of k_rec_scatter
constexpr uint32_t kChunk = kSplitThreads * kSplitPer;
constexpr int kSubThreads = 384;        // k_rec_split: 384 threads of 6 records, four blocks per SM
constexpr int kSubPer = 6;
constexpr uint32_t kSubChunk = kSubThreads * kSubPer;
constexpr int kPlaceThreads = 256;      // k_rec_place: 256 threads of 8 records
constexpr int kPlacePer = 8;
constexpr uint32_t kPlaceChunk = kPlaceThreads * kPlacePer;
constexpr int kFineBits = 11;           // counting-sort digit inside a sub-bucket
constexpr uint32_t kFine = 1u << kFineBits;
constexpr int kMaxDigitBits = 11;       // top and sub digits: at most 2048 values
constexpr int kSide = 32;               // parked members per sub-bucket (p <= 32)
constexpr uint32_t kPrefetchAhead = 456; // k_rec_step blocks resident at once (152 SMs x 3)
constexpr size_t kStageBytes = kChunk * (sizeof(float4) + sizeof(uint32_t) + sizeof(uint8_t));  // scatter staging

// Dynamic shared memory of k_rec_split: the chunk's records in arrival order
// (rows, keys), the arrival index of each grouped position, and the
// sub-bucket counters and run starts.
size_t split_smem(uint32_t nsub) {
  return static_cast<size_t>(kSubChunk) * (sizeof(float4) + sizeof(uint32_t) + sizeof(uint16_t)) +
         2 * static_cast<size_t>(nsub) * sizeof(uint32_t);
}

struct RecArgs {
  float4* top_rows;     // [ntop * top_cap]
  uint32_t* top_keys;
  float4* sub_rows;     // [nbuckets * sub_cap]
  uint32_t* sub_keys;
  uint32_t* top_fill;   // [2][ntop] records per top bucket, by step parity
  uint32_t* sub_fill;   // [2][nbuckets]
  uint32_t* sub_start;  // [nbuckets + 1]
  float4* side;         // [nbuckets * kSide]
  uint32_t top_cap, sub_cap, ntop, nsub, nbuckets;
  uint32_t id_mul;      // last step: id-range bucket umulhi(id, id_mul)
  int top_bits, sub_bits;
};

__device__ __forceinline__ uint32_t rec_id(const float4& r) { return __float_as_uint(r.w); }

__device__ __forceinline__ uint32_t top_of(uint64_t key, int top_bits) {
  return top_bits ? static_cast<uint32_t>(key >> (64 - top_bits)) : 0u;
}
// The 32 key bits below the top-level digit.
__device__ __forceinline__ uint32_t key32_of(uint64_t key, int top_bits) {
  return static_cast<uint32_t>((key << top_bits) >> 32);
}
__device__ __forceinline__ uint32_t sub_of(uint32_t k32, int sub_bits) {
  return sub_bits ? (k32 >> (32 - sub_bits)) : 0u;
}

__device__ __forceinline__ Row<float, 3> to_row(const float4& v) {
  Row<float, 3> r;
  r.x[0] = v.x; r.x[1] = v.y; r.x[2] = v.z; r.pad = v.w;
  return r;
}
__device__ __forceinline__ float4 to_rec(const Row<float, 3>& r) { return make_float4(r.x[0], r.x[1], r.x[2], r.pad); }

// The new position of particle id in the caller's array (its pad lane left as
// the caller wrote it).
__device__ __forceinline__ void write_position(float* x, uint32_t id, const Row<float, 3>& r) {
  float* row = x + static_cast<size_t>(id) * 4;
  *reinterpret_cast<float2*>(row) = make_float2(r.x[0], r.x[1]);
  row[2] = r.x[2];
}

// Top-level bucket and carried key bits of particle id at step m1.
__device__ __forceinline__ void top_key(const StepParams<float>& a, const RecArgs& g, uint32_t id, uint32_t m1,
                                        uint32_t& t, uint32_t& k32) {
  const uint64_t key = perm_key(id, m1, a.replica, a.keys);
  t = top_of(key, g.top_bits);
  k32 = key32_of(key, g.top_bits);
}

__device__ __forceinline__ void put_top(const StepParams<float>& a, const RecArgs& g, uint32_t t, uint32_t pos,
                                        const float4& rec, uint32_t k32) {
  if (pos < g.top_cap) {
    const size_t at = static_cast<size_t>(t) * g.top_cap + pos;
    g.top_rows[at] = rec;
    g.top_keys[at] = k32;
  } else {
    latch_status(a.status, RBM_ERR_STATE);
  }
}

// Record pos of id-range bucket t (last step of a run).
__device__ __forceinline__ void put_id(const StepParams<float>& a, const RecArgs& g, uint32_t t, uint32_t pos,
                                       const float4& rec) {
  if (pos < g.top_cap) g.top_rows[static_cast<size_t>(t) * g.top_cap + pos] = rec;
  else latch_status(a.status, RBM_ERR_STATE);
}

// The buckets [0, len) counted in s_hist (len <= 2048, kThreads threads):
// reserves the run of every non-empty bucket u in the global counter fill[u]
// (one atomic per bucket; consecutive threads on consecutive counters, so
// that a warp's atomics fall in one line, and issued before the scan so that
// their latency overlaps it), turns s_hist into the local starts (exclusive
// prefix sum) and sets s_base[u] = run start - local start, so that local
// position j of bucket u lands at s_base[u] + j.  Ends with a barrier.
template <int kThreads>
__device__ __forceinline__ void reserve_runs(uint32_t* s_hist, uint32_t len, uint32_t* s_warp, uint32_t* s_base,
                                             uint32_t* fill) {
  constexpr uint32_t per = (2048u + kThreads - 1) / kThreads;  // len <= per * kThreads
  uint32_t r[per];
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t u = threadIdx.x + i * static_cast<uint32_t>(kThreads);
    const uint32_t c = (u < len) ? s_hist[u] : 0u;
    r[i] = c ? atomicAdd(&fill[u], c) : 0u;
  }
  const uint32_t lo = threadIdx.x * per;
  uint32_t v[per], sum = 0;
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    v[i] = (lo + i < len) ? s_hist[lo + i] : 0u;
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
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t u = threadIdx.x + i * static_cast<uint32_t>(kThreads);
    if (u < len) s_base[u] = r[i];
  }
  __syncthreads();
  uint32_t run = incl - sum;
  run += warps_before(s_warp, warp, lane);
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    if (lo + i < len) {
      s_hist[lo + i] = run;
      s_base[lo + i] -= run;
    }
    run += v[i];
  }
  __syncthreads();
}

// The run holding local position j: the largest u < len with start[u] <= j
// (never an empty run: its successor would start at the same place).
__device__ __forceinline__ uint32_t run_of(const uint32_t* start, uint32_t len, uint32_t j) {
  uint32_t lo = 0, hi = len;  // start[lo] <= j, and j < start[hi] for hi < len
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (start[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The block's records, grouped by bucket in shared memory, out to their runs
// in the buckets: consecutive threads store consecutive rows of one run, so
// the stores cover whole lines instead of one line per record.
//   s_rows/s_keys[j], j < nrec: records in bucket order; s_start[u]: local
//   start of bucket u; s_shift[u]: the start of the run reserved in bucket u
//   minus s_start[u] (so that local position j lands at s_shift[u] + j);
//   s_bkt[j]: the bucket of position j when there are at most 256 buckets
//   (else null: found by binary search over s_start).
constexpr uint32_t kByteBuckets = 256;
template <typename Put>
__device__ __forceinline__ void store_runs(uint32_t nrec, uint32_t nbkt, const uint32_t* s_start,
                                           const uint32_t* s_shift, const uint8_t* s_bkt, Put put) {
  for (uint32_t j = threadIdx.x; j < nrec; j += blockDim.x) {
    const uint32_t u = s_bkt ? s_bkt[j] : run_of(s_start, nbkt, j);
    put(u, s_shift[u] + j, j);
  }
}


// ---------------------------------------------------------------------------
// First step of a run: the caller's rows in id order into the top level
// (block b takes rows [(block0 + b) C, ...), C = kChunk).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSplitThreads, 2) k_rec_scatter(StepParams<float> a, RecArgs g, uint32_t block0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_rows = reinterpret_cast<float4*>(smem_raw);              // [kChunk] records by bucket
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_rows + kChunk);   // [kChunk]
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(s_keys + kChunk);       // [kChunk] bucket of each position
  __shared__ uint32_t s_hist[1u << kMaxDigitBits];  // counts, then local starts
  __shared__ uint32_t s_base[1u << kMaxDigitBits];
  __shared__ uint32_t s_warp[32];
  const uint32_t m32 = step_index(a);
  const uint32_t par = m32 & 1u;
  const uint32_t i0 = (block0 + blockIdx.x) * kChunk;
  const uint32_t nrec = min(kChunk, a.n - i0);
  if (threadIdx.x == 0) {  // the chunk's rows into L2 while the keys are drawn
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.x + static_cast<size_t>(i0) * 4),
                 "r"(nrec * 16u) : "memory");
  }
  for (uint32_t u = threadIdx.x; u < g.ntop; u += blockDim.x) s_hist[u] = 0;
  __syncthreads();
  uint32_t tr[kSplitPer], k32[kSplitPer];
#pragma unroll
  for (int k = 0; k < kSplitPer; ++k) {
    const uint32_t e = k * kSplitThreads + threadIdx.x;
    if (e < nrec) {
      uint32_t t;
      top_key(a, g, i0 + e, m32, t, k32[k]);
      tr[k] = t | (atomicAdd(&s_hist[t], 1u) << 16);
    }
  }
  float4 v[kSplitPer];  // every row in flight before the first store
#pragma unroll
  for (int k = 0; k < kSplitPer; ++k) {
    const uint32_t e = k * kSplitThreads + threadIdx.x;
    if (e < nrec) v[k] = reinterpret_cast<const float4*>(a.x)[i0 + e];
  }
  __syncthreads();
  reserve_runs<kSplitThreads>(s_hist, g.ntop, s_warp, s_base, g.top_fill + par * g.ntop);
#pragma unroll
  for (int k = 0; k < kSplitPer; ++k) {
    const uint32_t e = k * kSplitThreads + threadIdx.x;
    if (e < nrec) {
      const uint32_t at = s_hist[tr[k] & 0xffffu] + (tr[k] >> 16);
      v[k].w = __uint_as_float(i0 + e);
      s_rows[at] = v[k];
      s_keys[at] = k32[k];
      s_bkt[at] = static_cast<uint8_t>(tr[k]);
    }
  }
  __syncthreads();
  store_runs(nrec, g.ntop, s_hist, s_base, g.ntop <= kByteBuckets ? s_bkt : nullptr,
             [&](uint32_t t, uint32_t pos, uint32_t j) {
    put_top(a, g, t, pos, s_rows[j], s_keys[j]);
  });
}

// ---------------------------------------------------------------------------
// Top level -> sub level: block (t, j) takes records [j C, (j+1) C) of top
// bucket t (C = kSubChunk).  The rows go straight into shared memory in
// arrival order (cp.async) while the keys are counted; each grouped position
// then names the arrival index it holds, and the runs are stored by
// consecutive threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSubThreads, 4) k_rec_split(StepParams<float> a, RecArgs g, uint32_t chunks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_rows = reinterpret_cast<float4*>(smem_raw);                 // [kSubChunk] arrival order
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_rows + kSubChunk);   // [kSubChunk] arrival order
  uint16_t* s_inv = reinterpret_cast<uint16_t*>(s_keys + kSubChunk);    // [kSubChunk] arrival index by position
  uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_inv + kSubChunk);    // [nsub] counts, then local starts
  uint32_t* s_base = s_hist + g.nsub;                                    // [nsub] run starts (shifted)
  __shared__ uint32_t s_warp[32];
  const uint32_t m32 = step_index(a);
  const uint32_t par = m32 & 1u;
  const uint32_t t = blockIdx.x / chunks, j = blockIdx.x - t * chunks;
  const uint32_t filled = g.top_fill[par * g.ntop + t];
  if (j == 0 && threadIdx.x == 0 && filled > g.top_cap) latch_status(a.status, RBM_ERR_STATE);
  const uint32_t count = min(filled, g.top_cap);
  const uint32_t lo = j * kSubChunk;
  if (lo >= count) return;  // uniform over the block
  const uint32_t nrec = min(kSubChunk, count - lo);
  const size_t src0 = static_cast<size_t>(t) * g.top_cap + lo;
  for (uint32_t e = threadIdx.x; e < nrec; e += blockDim.x) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(s_rows + e));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(g.top_rows + src0 + e) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (uint32_t u = threadIdx.x; u < g.nsub; u += blockDim.x) s_hist[u] = 0;
  __syncthreads();
  uint32_t ur[kSubPer];
#pragma unroll
  for (int k = 0; k < kSubPer; ++k) {
    const uint32_t e = k * kSubThreads + threadIdx.x;
    if (e < nrec) {
      const uint32_t kk = g.top_keys[src0 + e];
      s_keys[e] = kk;
      const uint32_t u = sub_of(kk, g.sub_bits);
      ur[k] = u | (atomicAdd(&s_hist[u], 1u) << 16);
    }
  }
  __syncthreads();
  reserve_runs<kSubThreads>(s_hist, g.nsub, s_warp, s_base, g.sub_fill + par * g.nbuckets + t * g.nsub);
#pragma unroll
  for (int k = 0; k < kSubPer; ++k) {
    const uint32_t e = k * kSubThreads + threadIdx.x;
    if (e < nrec) s_inv[s_hist[ur[k] & 0xffffu] + (ur[k] >> 16)] = static_cast<uint16_t>(e);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // runs out, the sub-bucket of each position read off its key
  for (uint32_t jj = threadIdx.x; jj < nrec; jj += blockDim.x) {
    const uint32_t e = s_inv[jj];
    const uint32_t kk = s_keys[e];
    const uint32_t u = sub_of(kk, g.sub_bits);
    const uint32_t pos = s_base[u] + jj;
    if (pos < g.sub_cap) {
      const size_t at = static_cast<size_t>(t * g.nsub + u) * g.sub_cap + pos;
      g.sub_rows[at] = s_rows[e];
      g.sub_keys[at] = kk;
    } else {
      latch_status(a.status, RBM_ERR_STATE);
    }
  }
}

// ---------------------------------------------------------------------------
// Sorted start of every sub-bucket (one block); clears the counters the
// next step fills.  A total other than N latches RBM_ERR_STATE.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_rec_scan(StepParams<float> a, RecArgs g) {
  constexpr uint32_t kPer = 4, kSpan = 1024 * kPer;  // counts per thread and per pass
  __shared__ uint32_t s_cnt[kSpan];
  __shared__ uint32_t s_warp[32];
  const uint32_t m32 = step_index(a);
  const uint32_t par = m32 & 1u, np = par ^ 1u;
  const uint32_t* cnt = g.sub_fill + par * g.nbuckets;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t nb = g.nbuckets;
  uint32_t carry = 0;  // total of the passes before
  for (uint32_t base = 0; base < nb; base += kSpan) {
    // coalesced in, kPer consecutive counts per thread, coalesced out
    for (uint32_t i = threadIdx.x; i < kSpan; i += blockDim.x) s_cnt[i] = (base + i < nb) ? cnt[base + i] : 0u;
    __syncthreads();
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      v[k] = s_cnt[threadIdx.x * kPer + k];
      sum += v[k];
    }
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
      if (lane < nwarps) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t run = carry + ((warp > 0) ? s_warp[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      s_cnt[threadIdx.x * kPer + k] = run;
      run += v[k];
    }
    carry += s_warp[nwarps - 1];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kSpan && base + i < nb; i += blockDim.x) g.sub_start[base + i] = s_cnt[i];
    __syncthreads();  // s_cnt and s_warp free for the next pass
  }
  if (threadIdx.x == 0) {
    g.sub_start[nb] = carry;
    if (carry != a.n) latch_status(a.status, RBM_ERR_STATE);
  }
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) g.sub_fill[np * nb + b] = 0;
  for (uint32_t u = threadIdx.x; u < g.ntop; u += blockDim.x) g.top_fill[np * g.ntop + u] = 0;
}

// The sub-bucket holding sorted position pos (largest b with start[b] <=
// pos), for pos < start[hi0].
__device__ __forceinline__ uint32_t sub_bucket_at(const uint32_t* start, uint32_t hi0, uint32_t pos) {
  uint32_t lo = 0, hi = hi0;  // start[lo] <= pos < start[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (start[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Records of positions [lo, hi) other than pp whose carried bits equal fe
// and that come before record e in (key, id) order: the full keys are drawn
// again.  Two records of a sub-bucket share all their carried bits about once
// in eight sub-buckets, so the caller counts equal bits in its loop and calls
// this only then.
__device__ __forceinline__ uint32_t rec_rank_ties(const StepParams<float>& a, uint32_t m32, const float4* srow,
                                               const uint32_t* sfine, const uint16_t* sidx, uint32_t lo, uint32_t hi,
                                               uint32_t pp, uint32_t fe, uint32_t e) {
  const uint32_t ide = rec_id(srow[e]);
  const uint64_t ke = perm_key(ide, m32, a.replica, a.keys);
  uint32_t before = 0;
  for (uint32_t j = lo; j < hi; ++j) {
    if (j == pp || sfine[j] != fe) continue;
    const uint32_t idj = rec_id(srow[sidx[j]]);
    const uint64_t kj = perm_key(idj, m32, a.replica, a.keys);
    if (kj < ke || (kj == ke && idj < ide)) ++before;
  }
  return before;
}

// ---------------------------------------------------------------------------
// One block per sub-bucket: sort, step the contained batches, park the
// members of crossing batches, send the moved records on (or, at the last
// step of a run, write the positions by id).
// ---------------------------------------------------------------------------
template <bool kLast, int KF, bool kPlain>
__global__ void __launch_bounds__(kStepThreads, 3) k_rec_step(StepParams<float> a, RecArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* srow = reinterpret_cast<float4*>(smem_raw);                 // [sub_cap] records, slot order
  // sfine: the bits below the sub digit by provisional position, later the
  // next step's carried key bits by slot
  uint32_t* sfine = reinterpret_cast<uint32_t*>(srow + g.sub_cap);     // [sub_cap]
  uint16_t* sidx = reinterpret_cast<uint16_t*>(sfine + g.sub_cap);    // [sub_cap] slot of each sorted position
  uint8_t* spark = reinterpret_cast<uint8_t*>(sidx + g.sub_cap);      // [sub_cap] 1: member of a crossing batch
  uint32_t* s_base = reinterpret_cast<uint32_t*>(spark + g.sub_cap);   // [ntop] run starts in the top level
  __shared__ uint32_t s_hist[kFine];
  __shared__ uint32_t s_warp[32];
  const uint32_t b = blockIdx.x;
  const uint32_t m32 = step_index(a);
  const uint32_t par = m32 & 1u;
  // the sub-bucket a block starting about one wave later takes is
  // prefetched into L2; its count is loaded together with this block's
  const uint32_t bn = b + kPrefetchAhead;
  const bool pf = threadIdx.x == 0 && bn < g.nbuckets;
  const uint32_t filled_next = pf ? g.sub_fill[par * g.nbuckets + bn] : 0u;
  const uint32_t filled = g.sub_fill[par * g.nbuckets + b];
  if (threadIdx.x == 0 && filled > g.sub_cap) latch_status(a.status, RBM_ERR_STATE);
  const uint32_t cnt = min(filled, g.sub_cap);
  const uint32_t start = g.sub_start[b];
  const size_t src0 = static_cast<size_t>(b) * g.sub_cap;
  for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(srow + e));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(g.sub_rows + src0 + e) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (pf) {
    const uint32_t cn = min(filled_next, g.sub_cap);
    if (cn > 0) {
      const size_t at = static_cast<size_t>(bn) * g.sub_cap;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g.sub_rows + at), "r"(cn * 16u) : "memory");
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g.sub_keys + at),
                   "r"(((cn + 3u) & ~3u) * 4u) : "memory");
    }
  }
  // the carried key bits of this thread's records, in flight across the
  // clearing barrier (the slots past cnt, about a third of the kStepPer,
  // are predicated off)
  uint32_t fr[kStepPer];  // key bits, then digit | provisional rank << 16
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e < cnt) fr[k] = g.sub_keys[src0 + e];
  }
  for (uint32_t u = threadIdx.x; u < kFine; u += blockDim.x) s_hist[u] = 0;
  __syncthreads();
  // counting sort by the kFineBits bits below the sub digit
  // the fixed-size loops stop at the first slot past cnt (a sub-bucket holds
  // about 2048 of the at most 3072 slots)
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    const uint32_t d = (fr[k] << g.sub_bits) >> (32 - kFineBits);
    fr[k] = d | (atomicAdd(&s_hist[d], 1u) << 16);
  }
  __syncthreads();
  {  // exclusive scan of s_hist
    constexpr uint32_t per = kFine / kStepThreads;
    const uint32_t lo = threadIdx.x * per;
    uint32_t v[per], sum = 0;
#pragma unroll
    for (uint32_t i = 0; i < per; ++i) {
      v[i] = s_hist[lo + i];
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
      s_hist[lo + i] = run;
      run += v[i];
    }
  }
  __syncthreads();
  asm volatile("cp.async.wait_all;" ::: "memory");
  // provisional positions: digit order, arbitrary inside a digit; the slot
  // and the bits below the sub digit stored by provisional position
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    const uint32_t d = fr[k] & 0xffffu;
    const uint32_t pp = s_hist[d] + (fr[k] >> 16);
    sidx[pp] = static_cast<uint16_t>(e);
    sfine[pp] = g.sub_keys[src0 + e] << g.sub_bits;  // read again (cached) rather than held across the scan
    spark[e] = 0;
    fr[k] = pp | (d << 16);
  }
  __syncthreads();  // also publishes every thread's staged records
  // final position of each record: its digit's start plus the number of the
  // digit's records before it in (key, id) order (a digit holds about one);
  // the digit's bits are read in a run, the slots only on equal bits
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    const uint32_t d = fr[k] >> 16;
    const uint32_t lo = s_hist[d], hi = (d + 1 < kFine) ? s_hist[d + 1] : cnt;
    uint32_t rank = 0;
    if (hi - lo > 1) {
      const uint32_t pp = fr[k] & 0xffffu;
      const uint32_t fe = sfine[pp];
      uint32_t equal = 0;  // records with the same carried bits, itself included
      // the digit's first four members read together (predicated), the rest
      // (a digit of more than four: about one in fifty) one by one
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        if (lo + q < hi) {
          const uint32_t fj = sfine[lo + q];
          rank += (fj < fe) ? 1u : 0u;
          equal += (fj == fe) ? 1u : 0u;
        }
      }
      for (uint32_t j = lo + 4; j < hi; ++j) {
        const uint32_t fj = sfine[j];
        rank += (fj < fe) ? 1u : 0u;
        equal += (fj == fe) ? 1u : 0u;
      }
      if (equal > 1) rank += rec_rank_ties(a, m32, srow, sfine, sidx, lo, hi, pp, fe, e);
    }
    fr[k] = lo + rank;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    sidx[fr[k]] = static_cast<uint16_t>(e);
  }
  // the digit starts are no longer read: clear the counters of the next
  // step's top-level buckets (of the id-range buckets at the last step) here,
  // not behind a barrier of their own
  for (uint32_t u = threadIdx.x; u < g.ntop; u += blockDim.x) s_hist[u] = 0;
  __syncthreads();

  // batches lying wholly inside [start, end)
  const uint32_t up = static_cast<uint32_t>(a.p);
  const uint32_t end = start + cnt;
  const uint32_t q0 = (start + up - 1) / up;
  const uint32_t q_end = (end == a.n) ? (a.n + up - 1) / up : end / up;
  const uint32_t count = (q_end > q0) ? q_end - q0 : 0u;
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gpw = 32 / a.p;
    const uint32_t per_round = static_cast<uint32_t>(gpw * (kStepThreads / 32));
    const int gi = lane / a.p, lg = lane - gi * a.p;
    for (uint32_t r0 = 0; r0 < count; r0 += per_round) {
      const uint32_t kb = r0 + static_cast<uint32_t>(warp * gpw + gi);
      bool valid = (gi < gpw) && (kb < count);
      int bs = a.p;
      uint32_t slot = 0, id = 0;
      Row<float, 3> r{};
      if (valid) {
        const uint32_t lo = (q0 + kb) * up;
        bs = static_cast<int>(min(lo + up, a.n) - lo);
        valid = lg < bs;
        if (valid) {
          slot = sidx[lo + lg - start];
          r = to_row(srow[slot]);
          id = rec_id(srow[slot]);
        }
      }
      if (batch_group_update<float, 3, KF, kPlain>(a, m32, id, valid, lg, bs, r)) srow[slot] = to_rec(r);
    }
  }
  // members of batches crossing the ends (sorted positions before q0 p and
  // from q_end p on): parked under the sub-bucket that holds the batch's
  // first member
  const uint32_t head = (count > 0) ? q0 * up - start : cnt;   // all members when no batch fits inside
  const uint32_t tail = (count > 0) ? min(cnt, q_end * up - start) : cnt;
  const uint32_t ncross = head + (cnt - tail);
  {
    for (uint32_t c = threadIdx.x; c < ncross; c += blockDim.x) {
      const uint32_t e = (c < head) ? c : tail + (c - head);
      const uint32_t pos = start + e;
      const uint32_t q = pos / up;
      const uint32_t qp = q * up;
      const uint16_t slot = sidx[e];
      spark[slot] = 1;
      // an earlier sub-bucket (qp < start[b])
      const uint32_t bf = (qp >= start) ? b : sub_bucket_at(g.sub_start, b, qp);
      g.side[static_cast<size_t>(bf) * kSide + (pos - qp)] = srow[slot];
    }
  }
  __syncthreads();

  // the moved records to their top-level buckets of step m + 1 (at the last
  // step of a run, to their id-range buckets; s_hist was cleared before the
  // batches were stepped)
  const uint32_t np = par ^ 1u;
  constexpr uint32_t kParked = 0xffffffffu;
  uint32_t tr[kStepPer], k32[kStepPer];
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    tr[k] = kParked;
    if (!spark[e]) {
      uint32_t t;
      if (kLast) t = __umulhi(rec_id(srow[e]), g.id_mul);
      else top_key(a, g, rec_id(srow[e]), m32 + 1u, t, k32[k]);
      tr[k] = t | (atomicAdd(&s_hist[t], 1u) << 16);
    }
  }
  __syncthreads();
  reserve_runs<kStepThreads>(s_hist, g.ntop, s_warp, s_base, g.top_fill + np * g.ntop);  // local start of each bucket's run
  // the records in bucket order: sidx[j] the slot at position j, spark[j]
  // (read for the last time in the loop above) its bucket
#pragma unroll
  for (int k = 0; k < kStepPer; ++k) {
    const uint32_t e = threadIdx.x + k * kStepThreads;
    if (e >= cnt) break;
    if (tr[k] != kParked) {
      const uint32_t at = s_hist[tr[k] & 0xffffu] + (tr[k] >> 16);
      sidx[at] = static_cast<uint16_t>(e);
      spark[at] = static_cast<uint8_t>(tr[k]);
      if (!kLast) sfine[e] = k32[k];
    }
  }
  __syncthreads();
  store_runs(cnt - ncross, g.ntop, s_hist, s_base, g.ntop <= kByteBuckets ? spark : nullptr,
             [&](uint32_t t, uint32_t pos, uint32_t j) {
    const uint32_t e = sidx[j];
    if (kLast) put_id(a, g, t, pos, srow[e]);
    else put_top(a, g, t, pos, srow[e], sfine[e]);
  });
}

// ---------------------------------------------------------------------------
// The batch crossing the end of each sub-bucket (at most one starts in a
// sub-bucket and ends past it), from its parked members.
// ---------------------------------------------------------------------------
template <bool kLast, int KF, bool kPlain>
__global__ void __launch_bounds__(256) k_rec_fixup(StepParams<float> a, RecArgs g) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / a.p;
  const int gi = lane / a.p, lg = lane - gi * a.p;
  const uint32_t b = (blockIdx.x * (blockDim.x >> 5) + warp) * gpw + gi;
  const uint32_t m32 = step_index(a);
  const uint32_t up = static_cast<uint32_t>(a.p);
  bool valid = (gi < gpw) && b < g.nbuckets;
  int bs = a.p;
  uint32_t id = 0;
  Row<float, 3> r{};
  if (valid) {
    const uint32_t start = g.sub_start[b], end = g.sub_start[b + 1];
    valid = end > start;
    if (valid) {
      const uint32_t qp = ((end - 1) / up) * up;
      const uint32_t hi = min(qp + up, a.n);
      valid = qp >= start && hi > end;
      bs = static_cast<int>(hi - qp);
      valid = valid && lg < bs;
      if (valid) {
        const float4 v = g.side[static_cast<size_t>(b) * kSide + lg];
        r = to_row(v);
        id = rec_id(v);
      }
    }
  }
  if (!batch_group_update<float, 3, KF, kPlain>(a, m32, id, valid, lg, bs, r)) return;
  if (kLast) {
    write_position(a.x, id, r);
  } else {
    uint32_t t, k32;
    top_key(a, g, id, m32 + 1u, t, k32);
    const uint32_t np = (m32 & 1u) ^ 1u;
    put_top(a, g, t, atomicAdd(&g.top_fill[np * g.ntop + t], 1u), to_rec(r), k32);
  }
}

// ---------------------------------------------------------------------------
// After the last step of a run: the records of id-range bucket t (the ids i
// with umulhi(i, id_mul) = t, about N / ntop consecutive ids) to the caller's
// array by id, for the buckets t0, t0 + 1, ...  Block (t - t0, j) takes
// records [j C, (j+1) C) of bucket t
// (C = kPlaceChunk), every load in flight before the first store; consecutive
// blocks take consecutive chunks of one bucket, so the rows written at any
// time lie in a few windows of the array that L2 holds until their sectors
// are complete.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPlaceThreads) k_rec_place(StepParams<float> a, RecArgs g, uint32_t chunks,
                                                              uint32_t t0) {
  const uint32_t tb = blockIdx.x / chunks, j = blockIdx.x - tb * chunks;
  const uint32_t t = t0 + tb;
  const uint32_t np = (step_index(a) & 1u) ^ 1u;
  const uint32_t count = min(g.top_fill[np * g.ntop + t], g.top_cap);
  const uint32_t lo = j * kPlaceChunk;
  if (lo >= count) return;  // uniform over the block
  const float4* src = g.top_rows + static_cast<size_t>(t) * g.top_cap;
  float4 v[kPlacePer];
#pragma unroll
  for (int k = 0; k < kPlacePer; ++k) {
    const uint32_t e = lo + k * kPlaceThreads + threadIdx.x;
    if (e < count) v[k] = src[e];
  }
#pragma unroll
  for (int k = 0; k < kPlacePer; ++k) {
    const uint32_t e = lo + k * kPlaceThreads + threadIdx.x;
    if (e < count) write_position(a.x, rec_id(v[k]), to_row(v[k]));
  }
}

// Dynamic shared memory of k_rec_step: records, sort bits, sorted slots and
// crossing flags of sub_cap records (a multiple of 32, so the run starts
// that follow are aligned), then ntop run starts.
size_t step_smem(uint32_t sub_cap, uint32_t ntop) {
  return static_cast<size_t>(sub_cap) * (sizeof(float4) + sizeof(uint32_t) + sizeof(uint16_t) + sizeof(uint8_t)) +
         static_cast<size_t>(ntop) * sizeof(uint32_t);
}

RecArgs make_args(const RecScratch& rs) {
  RecArgs g;
  g.top_rows = rs.top_rows; g.top_keys = rs.top_keys; g.sub_rows = rs.sub_rows; g.sub_keys = rs.sub_keys;
  g.top_fill = rs.top_fill; g.sub_fill = rs.sub_fill; g.sub_start = rs.sub_start; g.side = rs.side;
  g.top_cap = rs.top_cap; g.sub_cap = rs.sub_cap; g.ntop = rs.ntop; g.nsub = rs.nsub; g.nbuckets = rs.ntop * rs.nsub;
  g.top_bits = rs.top_bits; g.sub_bits = rs.sub_bits;
  g.id_mul = rs.id_mul;
  return g;
}

uint32_t round_up(uint32_t v, uint32_t q) { return (v + q - 1) / q * q; }

}  // namespace

bool rec_eligible(int dtype, int d, int p, int scheme) {
  return dtype == RBM_F32 && d == 3 && p >= 2 && p <= kSide && scheme != RBM_SCHEME_VERLET;
}

// Bucket geometry for n records: 2^(top_bits + sub_bits) sub-buckets of at
// most kSubTarget records on average (or 2^tuned_bits sub-buckets when
// tuned_bits > 0), the bits split between the levels so that both
// distributions write runs of tens of records.
void rec_geometry(uint32_t n, int tuned_bits, RecScratch* rs) {
  int bits = 0;
  while (bits < 2 * kMaxDigitBits && (static_cast<uint64_t>(kSubTarget) << bits) < n) ++bits;
  if (tuned_bits > 0) bits = tuned_bits < 2 * kMaxDigitBits ? tuned_bits : 2 * kMaxDigitBits;
  rs->top_bits = bits / 2;
  rs->sub_bits = bits - rs->top_bits;
  rs->ntop = 1u << rs->top_bits;
  rs->nsub = 1u << rs->sub_bits;
  const double top_mean = static_cast<double>(n) / rs->ntop;
  const double sub_mean = top_mean / rs->nsub;
  rs->top_cap = round_up(static_cast<uint32_t>(top_mean + 12.0 * std::sqrt(top_mean) + 1024.0), 32);
  // the last step's id-range buckets umulhi(id, M), M = floor(2^32 ntop / n):
  // every id < n maps below ntop (id M / 2^32 < ntop) and a bucket holds at
  // most floor(2^32 / M) + 1 ids, within the capacity for every geometry used
  // (the capacity is raised if ever it is not)
  const uint64_t mul = (static_cast<uint64_t>(rs->ntop) << 32) / (n > 0 ? n : 1u);
  rs->id_mul = mul > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(mul);
  const uint64_t id_max = rs->id_mul ? (0x100000000ull / rs->id_mul) + 1 : n;
  if (id_max > rs->top_cap) rs->top_cap = round_up(static_cast<uint32_t>(id_max), 32);
  const uint32_t sc = round_up(static_cast<uint32_t>(sub_mean + 12.0 * std::sqrt(sub_mean) + 64.0), 32);
  rs->sub_cap = sc < kSubCapMax ? sc : kSubCapMax;
}

cudaError_t rec_alloc(uint32_t n, RecScratch* rs) {
  const size_t top = static_cast<size_t>(rs->ntop) * rs->top_cap;
  const size_t nb = static_cast<size_t>(rs->ntop) * rs->nsub;
  const size_t sub = nb * rs->sub_cap;
  cudaError_t e = cudaMalloc(&rs->top_rows, top * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&rs->top_keys, top * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&rs->sub_rows, sub * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&rs->sub_keys, sub * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&rs->top_fill, 2 * rs->ntop * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&rs->sub_fill, 2 * nb * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&rs->sub_start, (nb + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&rs->side, nb * kSide * sizeof(float4));
  (void)n;
  return e;
}

void rec_free(RecScratch* rs) {
  cudaFree(rs->top_rows); cudaFree(rs->top_keys); cudaFree(rs->sub_rows); cudaFree(rs->sub_keys);
  cudaFree(rs->top_fill); cudaFree(rs->sub_fill); cudaFree(rs->sub_start); cudaFree(rs->side);
  *rs = RecScratch{};
}

namespace {

// The sort-and-step kernel and the fix-up of one step, with the kernel
// family fixed at compile time on the plain configuration (Euler-Maruyama,
// additive noise, no projection, no noise refinement), or any configuration
// with the family chosen at run time (KF < 0).  The same arithmetic in every
// instance.
template <int KF, bool kPlain>
void launch_step_pair(bool last, const StepParams<float>& a, const RecArgs& g, size_t smem, uint32_t fix_grid,
                      const LaunchCfg& cfg, cudaStream_t st) {
  if (last) {
    k_rec_step<true, KF, kPlain><<<g.nbuckets, kStepThreads, smem, st>>>(a, g);
    mark_launch(cfg, st, "k_rec_step_last");
    k_rec_fixup<true, KF, kPlain><<<fix_grid, 256, 0, st>>>(a, g);
    mark_launch(cfg, st, "k_rec_fixup_last");
  } else {
    k_rec_step<false, KF, kPlain><<<g.nbuckets, kStepThreads, smem, st>>>(a, g);
    mark_launch(cfg, st, "k_rec_step");
    k_rec_fixup<false, KF, kPlain><<<fix_grid, 256, 0, st>>>(a, g);
    mark_launch(cfg, st, "k_rec_fixup");
  }
}

template <int KF, bool kPlain>
cudaError_t allow_step_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_rec_step<false, KF, kPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rec_step<true, KF, kPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

using StepPairLaunch = void (*)(bool, const StepParams<float>&, const RecArgs&, size_t, uint32_t, const LaunchCfg&,
                                cudaStream_t);

StepPairLaunch step_pair_for(const StepParams<float>& a) {
  const bool plain = a.scheme == RBM_SCHEME_EULER && !a.gbm && !a.renorm && a.noise_refine <= 1u;
  if (!plain) return launch_step_pair<-1, false>;
  switch (a.kf) {
    case RBM_K_COULOMB: return launch_step_pair<RBM_K_COULOMB, true>;
    case RBM_K_BOUNDED_CONF: return launch_step_pair<RBM_K_BOUNDED_CONF, true>;
    case RBM_K_GAUSS_AGG: return launch_step_pair<RBM_K_GAUSS_AGG, true>;
    case RBM_K_REG_ATTRACT: return launch_step_pair<RBM_K_REG_ATTRACT, true>;
    case RBM_K_SMOOTH_TEST: return launch_step_pair<RBM_K_SMOOTH_TEST, true>;
    case RBM_K_LINEAR: return launch_step_pair<RBM_K_LINEAR, true>;
    default: return launch_step_pair<-1, true>;
  }
}

}  // namespace

cudaError_t prepare_rec_kernels() {
  const int bytes = static_cast<int>(step_smem(kSubCapMax, 1u << kMaxDigitBits));
  cudaError_t e = allow_step_smem<-1, false>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<-1, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_COULOMB, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_BOUNDED_CONF, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_GAUSS_AGG, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_REG_ATTRACT, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_SMOOTH_TEST, true>(bytes);
  if (e == cudaSuccess) e = allow_step_smem<RBM_K_LINEAR, true>(bytes);
  // the scatter stages 4096 records (84 KB) besides 16 KB of counters (two blocks per SM), the split 2304
  // records (50 KB) besides its counters (four blocks per SM)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rec_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(split_smem(1u << kMaxDigitBits)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rec_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kStageBytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rec_split, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rec_scatter, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

int rec_launches_per_step(const RecScratch&) { return 4; }  // split, scan, step, fix-up

// `count` RBM-1 steps from step (m_ptr ? *m_ptr : 0) + a.m_off: clear the
// counters, fill the first step's top level from the caller's array, then
// per step split, scan, step and fix-up; after the last step (whose fix-up
// writes the crossing batches by id) k_rec_place writes the positions.
namespace {

// The first id of id-range bucket t (the smallest i with umulhi(i, mul) >= t),
// at most n.
uint32_t first_id_of(uint32_t t, uint32_t mul, uint32_t n) {
  const uint64_t v = ((static_cast<uint64_t>(t) << 32) + mul - 1) / mul;
  return v < n ? static_cast<uint32_t>(v) : n;
}

void launch_place(const RecScratch& rs, const RecArgs& g, const StepParams<float>& a, uint32_t t0, uint32_t t1,
                  const LaunchCfg& cfg, cudaStream_t st) {
  const uint32_t pchunks = (rs.top_cap + kPlaceChunk - 1) / kPlaceChunk;
  k_rec_place<<<(t1 - t0) * pchunks, kPlaceThreads, 0, st>>>(a, g, pchunks, t0);
  mark_launch(cfg, st, "k_rec_place");
}

// Steps m_off .. m_off + count - 1 of a run whose first top level is filled
// (the last one sends its records to the id-range buckets).
cudaError_t launch_rec_steps(const RecScratch& rs, const RecArgs& g, const StepParams<float>& a0, int64_t count,
                             const LaunchCfg& cfg, cudaStream_t st) {
  const uint32_t chunks = (rs.top_cap + kSubChunk - 1) / kSubChunk;
  const size_t smem = step_smem(rs.sub_cap, rs.ntop);
  const int gpw = 32 / a0.p;
  const uint32_t fix_groups = 8u * static_cast<uint32_t>(gpw);
  const uint32_t fix_grid = (g.nbuckets + fix_groups - 1) / fix_groups;
  const StepPairLaunch step_pair = step_pair_for(a0);
  for (int64_t k = 0; k < count; ++k) {
    StepParams<float> a = a0;
    a.m_off = a0.m_off + k;
    const bool last = (k + 1 == count);
    k_rec_split<<<rs.ntop * chunks, kSubThreads, split_smem(rs.nsub), st>>>(a, g, chunks);
    mark_launch(cfg, st, "k_rec_split");
    k_rec_scan<<<1, 1024, 0, st>>>(a, g);
    mark_launch(cfg, st, "k_rec_scan");
    step_pair(last, a, g, smem, fix_grid, cfg, st);
  }
  return cudaGetLastError();
}

cudaError_t clear_fill(const RecScratch& rs, const RecArgs& g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(rs.top_fill, 0, 2 * rs.ntop * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rs.sub_fill, 0, 2 * size_t(g.nbuckets) * sizeof(uint32_t), st);
  return e;
}

}  // namespace

cudaError_t launch_rec_run(const RecScratch& rs, const void* params, int64_t count, const LaunchCfg& cfg,
                           cudaStream_t st) {
  const StepParams<float> a0 = *static_cast<const StepParams<float>*>(params);
  const RecArgs g = make_args(rs);
  cudaError_t e = clear_fill(rs, g, st);
  if (e != cudaSuccess) return e;
  k_rec_scatter<<<(a0.n + kChunk - 1) / kChunk, kSplitThreads, kStageBytes, st>>>(a0, g, 0u);
  mark_launch(cfg, st, "k_rec_scatter");
  e = launch_rec_steps(rs, g, a0, count, cfg, st);
  if (e == cudaSuccess && count > 0) {  // the last step's records to the caller's array by id
    StepParams<float> a = a0;
    a.m_off = a0.m_off + count - 1;
    launch_place(rs, g, a, 0u, rs.ntop, cfg, st);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_rec_host_step(const RecScratch& rs, const void* params, void* x_host, const LaunchCfg& cfg,
                                 cudaStream_t st, cudaStream_t copy_st, cudaEvent_t* ev) {
  const StepParams<float> a = *static_cast<const StepParams<float>*>(params);
  const RecArgs g = make_args(rs);
  constexpr size_t kRow = 4 * sizeof(float);
  char* host = static_cast<char*>(x_host);
  char* dev = reinterpret_cast<char*>(a.x);
  cudaError_t e = cudaEventRecord(ev[0], st);  // the copies wait for the work before the call
  if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_st, ev[0], 0);
  if (e == cudaSuccess) e = clear_fill(rs, g, st);
  // in: chunk j of the rows copied on copy_st, then scattered on st
  const uint32_t nblk = (a.n + kChunk - 1) / kChunk;
  for (int j = 0; j < kHostChunks && e == cudaSuccess; ++j) {
    const uint32_t b0 = static_cast<uint32_t>(uint64_t(nblk) * j / kHostChunks);
    const uint32_t b1 = static_cast<uint32_t>(uint64_t(nblk) * (j + 1) / kHostChunks);
    if (b1 == b0) continue;
    const size_t r0 = size_t(b0) * kChunk, r1 = std::min(size_t(b1) * kChunk, size_t(a.n));
    e = cudaMemcpyAsync(dev + r0 * kRow, host + r0 * kRow, (r1 - r0) * kRow, cudaMemcpyHostToDevice, copy_st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + j], copy_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1 + j], 0);
    if (e == cudaSuccess) {
      k_rec_scatter<<<b1 - b0, kSplitThreads, kStageBytes, st>>>(a, g, b0);
      mark_launch(cfg, st, "k_rec_scatter");
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = launch_rec_steps(rs, g, a, 1, cfg, st);
  // out: the rows of id-range buckets [t0, t1) placed on st, then copied on copy_st
  for (int j = 0; j < kHostChunks && e == cudaSuccess; ++j) {
    const uint32_t t0 = static_cast<uint32_t>(uint64_t(rs.ntop) * j / kHostChunks);
    const uint32_t t1 = static_cast<uint32_t>(uint64_t(rs.ntop) * (j + 1) / kHostChunks);
    if (t1 == t0) continue;
    launch_place(rs, g, a, t0, t1, cfg, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + kHostChunks + j], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_st, ev[1 + kHostChunks + j], 0);
    const size_t i0 = first_id_of(t0, rs.id_mul, a.n);
    const size_t i1 = (t1 == rs.ntop) ? a.n : first_id_of(t1, rs.id_mul, a.n);
    if (e == cudaSuccess && i1 > i0)
      e = cudaMemcpyAsync(host + i0 * kRow, dev + i0 * kRow, (i1 - i0) * kRow, cudaMemcpyDeviceToHost, copy_st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * kHostChunks], copy_st);  // st waits for the copies out
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1 + 2 * kHostChunks], 0);
  return e;
}

}  // namespace rbm
