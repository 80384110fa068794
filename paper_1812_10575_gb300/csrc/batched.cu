// Batched replicas: many independent particle systems of uneven size N_r,
// all advanced by one RBM-1 step (Algorithm "randomdiv", Sec. 2.1 of
// arXiv:1812.10575) in one launch.  The paper notes that batches can be
// updated in parallel once the random division is known (Sec. 2.3 item 3);
// here the unit of parallel work is a whole replica.
//
// Replica r owns rows [off_r, off_r + N_r) of the concatenated position array
// and its own ids 0 .. N_r - 1; its random division sorts those ids by the
// Philox key of counter (id, m, r, 0) with an id tie-break, exactly as a
// single system with replica index r.  Every block takes a fixed list of
// replicas (largest first, dealt to the blocks in snake order so the sums of
// N_r per block stay close) and runs, for each replica, with block-level
// synchronisation only:
//   1. a shared-memory histogram of B_r = ceil(N_r / target) buckets
//      (monotone in the key; keys are regenerated from Philox wherever they
//      are needed, never stored; each particle's bucket is kept as 16 bits
//      in id order for the scatter);
//   2. scan, scatter of ids to bucket order;
//   3. per bucket: counting sort in shared memory by the next 10 key bits and
//      insertion sort of equal sub-buckets by (key, id); the sorted ids form
//      the replica's stretch of the permutation, and the batches lying wholly
//      inside the bucket are stepped at once from the sorted ids (groups of p
//      lanes, positions exchanged by warp shuffles);
//   4. the batches straddling bucket boundaries, from the permutation.
// A replica of at most one bucket skips 1-2 and sorts its ids directly.  If a
// bucket outgrows shared memory or holds fewer than p members, the replica
// takes the general mode: whole permutation first, then every batch.
// No block waits on another, so the launch cannot deadlock whatever the
// residency.
#include "rbm_batch.cuh"
#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr uint32_t kBSubBits = 10;    // sub-buckets of about one member for buckets of about 1024
                                       // (the clearing, scan and visit of every sub-bucket cost more than
                                       // the insertion sort saves with 2^11)
constexpr uint32_t kBSub = 1u << kBSubBits;
constexpr uint32_t kBCap = 2048;       // largest bucket sorted in shared memory
constexpr uint32_t kBMaxBuckets = 512;  // per replica
static_assert(kBMaxBuckets <= 65536, "bucket indices are kept as 16 bits");

struct BatchedArgs {
  const uint32_t* order;        // replica ids, block-major
  const uint32_t* block_begin;  // [G + 1] slice of `order` per block
  const uint64_t* offs;         // [R + 1] first row of each replica
  uint32_t* tmp;                // [rows] ids grouped by bucket
  uint32_t* perm;               // [rows] permutation (replica-local ids)
  uint16_t* bkt;                // [rows] bucket of each particle (histogram pass -> scatter pass)
  uint32_t bucket_target;       // mean members per bucket
  uint32_t rep_base;            // replica index in the counters = list index + rep_base
};

__device__ __forceinline__ bool bkey_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Exclusive scan of a[0, len) for any len by the whole block.
__device__ void block_scan_any(uint32_t* a, uint32_t len, uint32_t* s_warp) {
  const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(len, threadIdx.x * per), hi = min(len, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += a[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = (lane < nw) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = (warp > 0 ? s_warp[warp - 1] : 0u) + incl - sum;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  __syncthreads();
}

// Sorts the nb members of one bucket, given by ids[0, nb) in arbitrary order
// (or the identity 0 .. nb-1 when ids is null), into b_id[0, nb) by
// (key, id): counting sort by the kBSubBits key bits below the bucket bits,
// then insertion sort inside each sub-bucket.  Keys are regenerated.
__device__ void sort_bucket(const uint32_t* ids, uint32_t nb, uint32_t B, uint32_t m32, uint32_t r, const PhiloxKeys& ks,
                            uint64_t* a_key, uint64_t* b_key, uint32_t* a_id, uint32_t* b_id, uint32_t* a_sub,
                            uint32_t* s_sub, uint32_t* s_warp) {
  for (uint32_t u = threadIdx.x; u < kBSub; u += blockDim.x) s_sub[u] = 0;
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
    const uint32_t id = ids ? ids[j] : j;
    const uint64_t key = perm_key(id, m32, r, ks);
    const uint32_t sub = static_cast<uint32_t>(__umul64hi(key, static_cast<uint64_t>(B) << kBSubBits)) & (kBSub - 1u);
    a_key[j] = key;
    a_id[j] = id;
    a_sub[j] = sub | (atomicAdd(&s_sub[sub], 1u) << 16);
  }
  __syncthreads();
  block_scan_any(s_sub, kBSub, s_warp);
  for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
    const uint32_t pos = s_sub[a_sub[j] & 0xffffu] + (a_sub[j] >> 16);
    b_key[pos] = a_key[j];
    b_id[pos] = a_id[j];
  }
  __syncthreads();
  for (uint32_t u = threadIdx.x; u < kBSub; u += blockDim.x) {
    const uint32_t lo = s_sub[u], hi = (u + 1 < kBSub) ? s_sub[u + 1] : nb;
    for (uint32_t x = lo + 1; x < hi; ++x) {
      const uint64_t kx = b_key[x];
      const uint32_t ix = b_id[x];
      uint32_t y = x;
      while (y > lo && bkey_less(kx, ix, b_key[y - 1], b_id[y - 1])) {
        b_key[y] = b_key[y - 1];
        b_id[y] = b_id[y - 1];
        --y;
      }
      b_key[y] = kx;
      b_id[y] = ix;
    }
  }
  __syncthreads();
}

// FP32 rows of one or two coordinates: registers capped so that two blocks
// of 1024 threads fit on an SM (64 warps resident).
template <typename T, int D>
constexpr int batched_min_blocks() {
  return (sizeof(T) == 4 && D <= 2) ? 2 : 1;
}

// KF >= 0: the kernel family fixed at compile time for the plain
// configuration (kPlain: Euler-Maruyama, additive noise, no projection, no
// noise refinement); the same arithmetic as the run-time form.
template <typename T, int D, int MODE, int KF = -1, bool kPlain = false>
__global__ void __launch_bounds__(1024, batched_min_blocks<T, D>()) k_rbm_batched(BatchedArgs ba, StepParams<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* a_key = reinterpret_cast<uint64_t*>(smem_raw);  // [kBCap]
  uint64_t* b_key = a_key + kBCap;                          // [kBCap]
  uint32_t* a_id = reinterpret_cast<uint32_t*>(b_key + kBCap);
  uint32_t* b_id = a_id + kBCap;
  uint32_t* a_sub = b_id + kBCap;
  uint32_t* s_sub = a_sub + kBCap;                          // [kBSub]
  __shared__ uint32_t s_hist[kBMaxBuckets + 1];
  __shared__ uint32_t s_fill[kBMaxBuckets];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_general;

  if (skipped(a)) return;  // uniform: the flag does not change during the launch
  const uint32_t m32 = step_index(a);
  const uint32_t up = static_cast<uint32_t>(a.p);
  const uint32_t begin = ba.block_begin[blockIdx.x], end_list = ba.block_begin[blockIdx.x + 1];
  const uint32_t count_list = end_list - begin;
  for (uint32_t k = 0; k < count_list; ++k) {
    // odd blocks walk their list backwards: large and small replicas are in
    // flight together, so the replicas being worked on fit in L2
    const uint32_t li = (blockIdx.x & 1u) ? end_list - 1u - k : begin + k;
    const uint32_t ri = ba.order[li];
    const uint32_t r = ri + ba.rep_base;  // replica index of the Philox counters
    const uint64_t off = ba.offs[ri];
    const uint32_t n = static_cast<uint32_t>(ba.offs[ri + 1] - off);
    uint32_t B = (n + ba.bucket_target - 1) / ba.bucket_target;
    B = max(1u, min(B, kBMaxBuckets));
    uint32_t* tmp = ba.tmp + off;
    uint32_t* perm = ba.perm + off;
    StepParams<T> ar = a;
    ar.x = a.x + off * Ld<D>::value;
    ar.fout = a.fout ? a.fout + off * Ld<D>::value : nullptr;
    ar.n = n;
    ar.replica = r;

    if (B == 1 && n <= kBCap) {
      // the whole replica is one bucket: sort the ids directly, step every batch
      sort_bucket(nullptr, n, 1u, m32, r, a.keys, a_key, b_key, a_id, b_id, a_sub, s_sub, s_warp);
      for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) perm[j] = b_id[j];
      if (MODE != kModePerm) step_batches<T, D, MODE, KF, kPlain>(ar, m32, b_id, 0u, 0u, (n + up - 1) / up);
      __syncthreads();
      continue;
    }

    // 1. bucket histogram (keys regenerated, never stored; each particle's
    //    bucket kept in global scratch, in id order, for the scatter)
    uint16_t* bkt = ba.bkt + off;
    for (uint32_t b = threadIdx.x; b <= B; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t b = static_cast<uint32_t>(__umul64hi(perm_key(i, m32, r, a.keys), B));
      bkt[i] = static_cast<uint16_t>(b);
      atomicAdd(&s_hist[b], 1u);
    }
    __syncthreads();
    // 2. bucket starts (s_hist[B] becomes n), scatter of ids; a bucket too
    //    large for shared memory or smaller than a batch selects the general
    //    mode (whole permutation first, then every batch from it)
    block_scan_any(s_hist, B + 1, s_warp);
    if (threadIdx.x == 0) s_general = 0;
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
      s_fill[b] = s_hist[b];
      const uint32_t nb = s_hist[b + 1] - s_hist[b];
      if (nb > kBCap || nb < up) s_general = 1;
    }
    __syncthreads();
    const bool general = (MODE == kModePerm) || s_general != 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) tmp[atomicAdd(&s_fill[bkt[i]], 1u)] = i;
    __syncthreads();
    // 3. sort every bucket; outside the general mode step the batches lying
    //    wholly inside it straight from the sorted ids in shared memory
    for (uint32_t b = 0; b < B; ++b) {
      const uint32_t s = s_hist[b], nb = s_hist[b + 1] - s;
      if (nb <= kBCap) {
        sort_bucket(tmp + s, nb, B, m32, r, a.keys, a_key, b_key, a_id, b_id, a_sub, s_sub, s_warp);
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) perm[s + j] = b_id[j];
        if (!general) {
          const uint32_t end = s + nb;
          const uint32_t q0 = (s + up - 1) / up;
          const uint32_t q_end = (end == n) ? (n + up - 1) / up : end / up;
          step_batches<T, D, MODE, KF, kPlain>(ar, m32, b_id, s, q0, (q_end > q0) ? q_end - q0 : 0u);
        }
      } else {
        // a bucket beyond the shared-memory sort (general mode): rank by counting
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
          const uint32_t idj = tmp[s + j];
          const uint64_t kj = perm_key(idj, m32, r, a.keys);
          uint32_t rank = 0;
          for (uint32_t f = 0; f < nb; ++f) {
            const uint32_t idf = tmp[s + f];
            rank += bkey_less(perm_key(idf, m32, r, a.keys), idf, kj, idj) ? 1u : 0u;
          }
          perm[s + rank] = idj;
        }
      }
      __syncthreads();
    }
    // 4. the batches not stepped yet: those straddling a bucket boundary
    //    (each from the first boundary strictly inside it), or all of them in
    //    the general mode; members read from the permutation just written
    if (MODE != kModePerm) {
      if (general) {
        step_batches<T, D, MODE, KF, kPlain>(ar, m32, perm, 0u, 0u, (n + up - 1) / up);
      } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int gpw = 32 / a.p, nwarps = blockDim.x >> 5;
        const int g = lane / a.p, lg = lane - g * a.p;
        const uint32_t per_round = static_cast<uint32_t>(gpw * nwarps);
        for (uint32_t r0 = 1; r0 < B; r0 += per_round) {
          const uint32_t b = r0 + static_cast<uint32_t>(warp * gpw + g);
          bool valid = (g < gpw) && (b < B);
          uint32_t id = 0;
          int bs = a.p;
          if (valid) {
            const uint32_t sb = s_hist[b];
            valid = (sb % up) != 0;                 // buckets hold >= p members: one boundary per batch
            if (valid) {
              const uint32_t lo = (sb / up) * up, hi = min(lo + up, n);
              bs = static_cast<int>(hi - lo);
              valid = lg < bs;
              if (valid) id = perm[lo + lg];
            }
          }
          batch_group<T, D, MODE, KF, kPlain>(ar, m32, id, valid, lg, bs);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int D>
size_t batched_smem() {
  return static_cast<size_t>(kBCap) * (8 + 8 + 4 + 4 + 4) + kBSub * 4;
}

template <typename T, int D, int MODE>
cudaError_t launch_batched_k(const BatchedScratch& bs, const StepParams<T>& a, cudaStream_t st) {
  BatchedArgs ba;
  ba.order = bs.order;
  ba.block_begin = bs.block_begin;
  ba.offs = bs.offs;
  ba.tmp = bs.tmp;
  ba.perm = bs.perm;
  ba.bkt = bs.bkt;
  ba.bucket_target = static_cast<uint32_t>(bs.bucket_target);
  ba.rep_base = bs.rep_base;
  const size_t smem = batched_smem<T, D>();
  if constexpr (sizeof(T) == 4 && MODE == kModeStep) {
    // FP32 steps of the plain configuration take the kernel family's own instance
    if (a.scheme == RBM_SCHEME_EULER && !a.gbm && !a.renorm && a.noise_refine <= 1u) {
      switch (a.kf) {
#define RBM_BATCHED_KF(kf) \
  case kf:                 \
    k_rbm_batched<T, D, kModeStep, kf, true><<<bs.grid, bs.threads, smem, st>>>(ba, a); \
    return cudaGetLastError();
        RBM_BATCHED_KF(RBM_K_INV1D)
        RBM_BATCHED_KF(RBM_K_COULOMB)
        RBM_BATCHED_KF(RBM_K_BOUNDED_CONF)
        RBM_BATCHED_KF(RBM_K_GAUSS_AGG)
        RBM_BATCHED_KF(RBM_K_REG_ATTRACT)
        RBM_BATCHED_KF(RBM_K_SMOOTH_TEST)
        RBM_BATCHED_KF(RBM_K_LINEAR)
#undef RBM_BATCHED_KF
        default: break;
      }
    }
  }
  k_rbm_batched<T, D, MODE><<<bs.grid, bs.threads, smem, st>>>(ba, a);
  return cudaGetLastError();
}

// The dynamic shared-memory allowance of the FP32 step instances of the
// plain configuration.
template <typename T, int D, int KF>
cudaError_t allow_plain_kf(int smem) {
  return cudaFuncSetAttribute(k_rbm_batched<T, D, kModeStep, KF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem);
}

template <typename T, int D>
cudaError_t allow_plain_smem(int smem) {
  if constexpr (sizeof(T) != 4) {
    (void)smem;
    return cudaSuccess;
  } else {
    cudaError_t e = allow_plain_kf<T, D, RBM_K_INV1D>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_COULOMB>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_BOUNDED_CONF>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_GAUSS_AGG>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_REG_ATTRACT>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_SMOOTH_TEST>(smem);
    if (e == cudaSuccess) e = allow_plain_kf<T, D, RBM_K_LINEAR>(smem);
    return e;
  }
}

template <typename T, int D>
cudaError_t prepare_batched_d(int threads, int* blocks_per_sm) {
  const int smem = static_cast<int>(batched_smem<T, D>());
  cudaError_t e = cudaFuncSetAttribute(k_rbm_batched<T, D, kModePerm>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rbm_batched<T, D, kModeStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rbm_batched<T, D, kModeForces>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = allow_plain_smem<T, D>(smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_rbm_batched<T, D, kModeStep>, threads, smem);
  return e;
}

}  // namespace

int batched_max_buckets() { return static_cast<int>(kBMaxBuckets); }

cudaError_t prepare_batched_kernels(int dtype, int d, int threads, int* blocks_per_sm) {
  if (dtype == RBM_F32) {
    if (d == 1) return prepare_batched_d<float, 1>(threads, blocks_per_sm);
    if (d == 2) return prepare_batched_d<float, 2>(threads, blocks_per_sm);
    return prepare_batched_d<float, 3>(threads, blocks_per_sm);
  }
  if (d == 1) return prepare_batched_d<double, 1>(threads, blocks_per_sm);
  if (d == 2) return prepare_batched_d<double, 2>(threads, blocks_per_sm);
  return prepare_batched_d<double, 3>(threads, blocks_per_sm);
}

template <typename T>
cudaError_t launch_batched(const BatchedScratch& bs, int d, int mode, const void* params, const LaunchCfg& cfg,
                           cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  cudaError_t e;
  if (d == 1) {
    e = (mode == kModeStep) ? launch_batched_k<T, 1, kModeStep>(bs, a, st)
      : (mode == kModeForces) ? launch_batched_k<T, 1, kModeForces>(bs, a, st)
                              : launch_batched_k<T, 1, kModePerm>(bs, a, st);
  } else if (d == 2) {
    e = (mode == kModeStep) ? launch_batched_k<T, 2, kModeStep>(bs, a, st)
      : (mode == kModeForces) ? launch_batched_k<T, 2, kModeForces>(bs, a, st)
                              : launch_batched_k<T, 2, kModePerm>(bs, a, st);
  } else {
    e = (mode == kModeStep) ? launch_batched_k<T, 3, kModeStep>(bs, a, st)
      : (mode == kModeForces) ? launch_batched_k<T, 3, kModeForces>(bs, a, st)
                              : launch_batched_k<T, 3, kModePerm>(bs, a, st);
  }
  mark_launch(cfg, st, "k_rbm_batched");
  return e;
}

template cudaError_t launch_batched<float>(const BatchedScratch&, int, int, const void*, const LaunchCfg&,
                                           cudaStream_t);
template cudaError_t launch_batched<double>(const BatchedScratch&, int, int, const void*, const LaunchCfg&,
                                            cudaStream_t);

}  // namespace rbm
