// RBM-r, the Random Batch Method with replacement (Sec. 2.2 of
// arXiv:1812.10575, Algorithm "fullyrandom"): iteration k picks a random set
// C_k of p distinct particles and moves its members by one Euler-Maruyama step
// of size tau of the p-particle system (eq. "secondalgB"), every force taken
// from the positions before the iteration; iterations act strictly in order.
// floor(N/p) iterations (at least one) make one step: the pseudo-time of one
// RBM-1 step (Algorithm "randomreplacement").
//
// The iterations of a step are executed in rounds that reproduce the
// sequential order exactly.  Every particle keeps the ascending list of the
// iterations it belongs to and a pointer to the first one not yet run; an
// iteration is ready when it is the pointed-to entry of all its members.
// Ready iterations have pairwise disjoint sets, so a round runs them all at
// once, then advances its members' pointers.  Every particle is thus moved by
// its iterations in increasing k, each time from the position the previous
// one left: the sequential result, up to the rounding of each iteration.
//
// One cooperative launch per step, one block per SM:
//   A. draw the sets (Philox stream 7, rejection of repeated ids, slot =
//      draw order) and count each particle's occurrences;       | grid barrier
//   B. exclusive scan of the counts (per-block chunks, then block offsets);
//   C. fill each particle's occurrence list;                      | barriers
//   D. sort each list (they hold about p K / N = 1 entry), pointers to 0;
//   E. rounds: mark the ready iterations | barrier | run them (one thread per
//      iteration, noise of slot s from Philox stream 8), advance pointers,
//      count down the iterations left | barrier | until none is left.
// Data written by other blocks is read through L2 (ld.global.cg).  Every
// grid barrier wait is bounded; a wait that runs out latches RBM_ERR_TIMEOUT.
#include <algorithm>

#include "rbm_device.cuh"
#include "rbm_grid.cuh"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr int kRrThreads = 512;
constexpr uint32_t kStreamRrSet = 7;
constexpr uint32_t kStreamRrNoise = 8;
constexpr uint32_t kRrMaxRounds = 1u << 20;

struct RrArgs {
  uint32_t* set;        // [K p] members, iteration-major, slot order
  uint32_t* cnt;        // [N] occurrence counters (zero between steps)
  uint32_t* start;      // [N + 1] first list entry of each particle
  uint32_t* occ;        // [K p] iterations of each particle, ascending
  uint32_t* next;       // [N] first list entry not yet run
  uint8_t* flag;        // [K] 0 pending, 1 ready this round, 2 done
  uint32_t* btot;       // [G] per-block totals of the scan
  uint32_t* remaining;  // [1] iterations not yet run
  uint32_t* rounds;     // [1] rounds taken by the last step
  unsigned long long* bar;
  uint32_t K;
  unsigned long long wait_ns;
};

__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }

template <typename T, int D>
__device__ __forceinline__ Row<T, D> load_row_cg(const T* X, uint64_t i) {
  Row<T, D> r;
  r.pad = T(0);
  const T* q = X + i * Ld<D>::value;
#pragma unroll
  for (int k = 0; k < D; ++k) r.x[k] = __ldcg(q + k);
  if constexpr (D == 3) r.pad = __ldcg(q + 3);
  return r;
}

// The p distinct members of iteration k in draw order: the words w0..w3 of
// the Philox blocks (k mod 2^32, k div 2^32, r, 7*256 + c), c < 256, each
// mapped to floor(w N / 2^32); repeats skipped; any slot still empty after
// 1024 words takes the smallest id not yet in the set.
__device__ void draw_set(uint64_t k, uint32_t n, int p, uint32_t replica, uint2 seed, uint32_t* set) {
  int got = 0;
  for (uint32_t c = 0; c < 256u && got < p; ++c) {
    const uint4 w = philox4x32_10(
        make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(k >> 32), replica, kStreamRrSet * 256u + c), seed);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (got >= p) break;
      const uint32_t id = __umulhi(ws[q], n);
      bool taken = false;
      for (int s = 0; s < got; ++s) taken |= (set[s] == id);
      if (!taken) set[got++] = id;
    }
  }
  for (uint32_t id = 0; got < p; ++id) {
    bool taken = false;
    for (int s = 0; s < got; ++s) taken |= (set[s] == id);
    if (!taken) set[got++] = id;
  }
}

// Brownian increment of slot s of iteration k: Box-Muller pairs from the
// blocks (k mod 2^32, k div 2^32, r, 8*256 + 2 s + t), t < ceil(D/2).
template <typename T, int D>
__device__ __forceinline__ void slot_noise(uint64_t k, int s, uint32_t replica, uint2 seed, T (&z)[D]) {
#pragma unroll
  for (int t = 0; 2 * t < D; ++t) {
    const uint4 a = philox4x32_10(make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(k >> 32), replica,
                                             kStreamRrNoise * 256u + 2u * static_cast<uint32_t>(s) + t),
                                  seed);
    T z0, z1;
    normal_pair(a, z0, z1);
    z[2 * t] = z0;
    if (2 * t + 1 < D) z[2 * t + 1] = z1;
  }
}

// One iteration by one thread: forces of all members from their positions
// before the iteration (sum over the other slots in slot order), then each
// member's Euler-Maruyama update.  PMAX = 4 keeps the members in registers
// (loops unrolled); PMAX = 32 keeps them in local memory (loops rolled).
template <typename T, int D, int PMAX>
__device__ void run_iteration(const StepParams<T>& a, uint64_t k, const uint32_t* set) {
  constexpr bool kSmall = PMAX <= 4;
  const int p = a.p;
  uint32_t id[PMAX];
  Row<T, D> row[PMAX];
  if constexpr (kSmall) {
#pragma unroll
    for (int s = 0; s < PMAX; ++s) {
      if (s < p) {
        id[s] = ldcg(set + s);
        row[s] = load_row_cg<T, D>(a.x, id[s]);
      }
    }
  } else {
#pragma unroll 1
    for (int s = 0; s < p; ++s) {
      id[s] = ldcg(set + s);
      row[s] = load_row_cg<T, D>(a.x, id[s]);
    }
  }
  const T inv = T(1) / static_cast<T>(p - 1);
  auto member = [&](int s) {
    T acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = T(0);
    if constexpr (kSmall) {
#pragma unroll
      for (int t = 0; t < PMAX; ++t) {
        if (t < p && t != s) add_pair_force_rt<T, D>(a.kf, a.kparam, a.radius_sq, row[s].x, row[t].x, acc);
      }
    } else {
#pragma unroll 1
      for (int t = 0; t < p; ++t) {
        if (t != s) add_pair_force_rt<T, D>(a.kf, a.kparam, a.radius_sq, row[s].x, row[t].x, acc);
      }
    }
    T fk[D], z[D], y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) fk[c] = acc[c] * inv;
    if (a.sq != T(0)) {
      slot_noise<T, D>(k, s, a.replica, a.seed, z);
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) z[c] = T(0);
    }
    euler_apply<T, D>(a, row[s].x, fk, z, y);
    Row<T, D> out = row[s];
#pragma unroll
    for (int c = 0; c < D; ++c) out.x[c] = y[c];
    store_row<T, D>(a.x, id[s], out);
  };
  if constexpr (kSmall) {
#pragma unroll
    for (int s = 0; s < PMAX; ++s) {
      if (s < p) member(s);
    }
  } else {
#pragma unroll 1
    for (int s = 0; s < p; ++s) member(s);
  }
}

// Sum of v over the block (every thread gets it).
__device__ __forceinline__ uint32_t rr_block_sum(uint32_t v, uint32_t* s_red) {
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

template <typename T, int D, int PMAX>
__global__ void __launch_bounds__(kRrThreads, 1) k_rbmr_step(RrArgs ra, StepParams<T> a) {
  __shared__ uint32_t s_red[32];
  __shared__ uint32_t s_val;
  const uint32_t G = gridDim.x;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, gsize = G * blockDim.x;
  const int64_t m = (a.m_ptr ? *a.m_ptr : 0) + a.m_off;
  const uint64_t k0 = static_cast<uint64_t>(m) * ra.K;
  const uint32_t n = a.n;
  const uint32_t p = static_cast<uint32_t>(a.p);

  // A. sets, occurrence counts
  if (gtid == 0) *ra.remaining = ra.K;
  for (uint32_t j = gtid; j < ra.K; j += gsize) {
    uint32_t* sj = ra.set + static_cast<size_t>(j) * p;
    draw_set(k0 + j, n, a.p, a.replica, a.seed, sj);
    for (uint32_t s = 0; s < p; ++s) atomicAdd(&ra.cnt[sj[s]], 1u);
    ra.flag[j] = 0;
  }
  if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;

  // B. exclusive scan of the counts: block chunks, then block offsets
  const uint32_t per = (n + G - 1) / G;
  const uint32_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
  const uint32_t sub = (hi - lo + blockDim.x - 1) / blockDim.x;
  const uint32_t tlo = min(hi, lo + threadIdx.x * sub), thi = min(hi, tlo + sub);
  uint32_t tsum = 0;
  for (uint32_t i = tlo; i < thi; ++i) tsum += ldcg(ra.cnt + i);
  uint32_t incl = tsum;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_red[warp] = incl;
  __syncthreads();
  uint32_t texcl = incl - tsum, btotal = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
    if (w < warp) texcl += s_red[w];
    btotal += s_red[w];
  }
  if (threadIdx.x == 0) ra.btot[blockIdx.x] = btotal;
  if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;
  if (threadIdx.x == 0) {
    uint32_t pre = 0;
    for (uint32_t b = 0; b < blockIdx.x; ++b) pre += ldcg(ra.btot + b);
    s_val = pre;
  }
  __syncthreads();
  uint32_t run = s_val + texcl;
  for (uint32_t i = tlo; i < thi; ++i) {
    const uint32_t c = ldcg(ra.cnt + i);
    ra.start[i] = run;
    ra.cnt[i] = 0;  // becomes the fill counter of C
    run += c;
  }
  if (gtid == 0) ra.start[n] = ra.K * p;
  if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;

  // C. occurrence lists
  for (uint32_t j = gtid; j < ra.K; j += gsize) {
    for (uint32_t s = 0; s < p; ++s) {
      const uint32_t c = ldcg(ra.set + static_cast<size_t>(j) * p + s);
      const uint32_t pos = atomicAdd(&ra.cnt[c], 1u);
      ra.occ[ldcg(ra.start + c) + pos] = j;
    }
  }
  if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;

  // D. sort every list ascending; pointers to the first entry; counters to 0
  for (uint32_t i = gtid; i < n; i += gsize) {
    const uint32_t b0 = ldcg(ra.start + i), b1 = ldcg(ra.start + i + 1);
    for (uint32_t x = b0 + 1; x < b1; ++x) {
      const uint32_t v = ldcg(ra.occ + x);
      uint32_t y = x;
      while (y > b0 && ldcg(ra.occ + y - 1) > v) {
        ra.occ[y] = ldcg(ra.occ + y - 1);
        --y;
      }
      ra.occ[y] = v;
    }
    ra.next[i] = 0;
    ra.cnt[i] = 0;
  }
  if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;

  // E. rounds
  uint32_t round = 0;
  while (true) {
    for (uint32_t j = gtid; j < ra.K; j += gsize) {
      if (ra.flag[j] != 0) continue;
      bool ready = true;
      for (uint32_t s = 0; s < p && ready; ++s) {
        const uint32_t c = ldcg(ra.set + static_cast<size_t>(j) * p + s);
        ready = ldcg(ra.occ + ldcg(ra.start + c) + ldcg(ra.next + c)) == j;
      }
      if (ready) ra.flag[j] = 1;
    }
    if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;
    uint32_t ran = 0;
    for (uint32_t j = gtid; j < ra.K; j += gsize) {
      if (ra.flag[j] != 1) continue;
      const uint32_t* sj = ra.set + static_cast<size_t>(j) * p;
      run_iteration<T, D, PMAX>(a, k0 + j, sj);
      ra.flag[j] = 2;
      for (uint32_t s = 0; s < p; ++s) {
        const uint32_t c = ldcg(sj + s);
        ra.next[c] = ldcg(ra.next + c) + 1u;  // no other iteration of this round holds c
      }
      ++ran;
    }
    ran = rr_block_sum(ran, s_red);
    if (threadIdx.x == 0 && ran) atomicSub(ra.remaining, ran);
    ++round;
    if (!grid_barrier(ra.bar, ra.wait_ns, a.status, false)) return;
    if (threadIdx.x == 0) s_val = ldcg(ra.remaining);
    __syncthreads();
    if (s_val == 0) break;
    if (round >= kRrMaxRounds) {  // every block stops at the same round
      if (gtid == 0) latch_status(a.status, RBM_ERR_TIMEOUT);
      break;
    }
  }
  if (gtid == 0) *ra.rounds = round;
}

// The sets of one step only (diagnostic): set[j p + s] of iteration m K + j.
__global__ void k_rbmr_sets(uint32_t* set, uint32_t K, uint32_t n, int p, uint32_t replica, uint2 seed, int64_t m) {
  const uint64_t k0 = static_cast<uint64_t>(m) * K;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x)
    draw_set(k0 + j, n, p, replica, seed, set + static_cast<size_t>(j) * p);
}

template <typename T, int D, int PMAX>
cudaError_t launch_k(const RbmrScratch& rs, const StepParams<T>& a, uint64_t wait_ns, cudaStream_t st) {
  RrArgs ra;
  ra.set = rs.set;
  ra.cnt = rs.cnt;
  ra.start = rs.start;
  ra.occ = rs.occ;
  ra.next = rs.next;
  ra.flag = rs.flag;
  ra.btot = rs.btot;
  ra.remaining = rs.remaining;
  ra.rounds = rs.rounds;
  ra.bar = rs.bar;
  ra.K = rs.K;
  ra.wait_ns = wait_ns;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(rs.grid);
  cfg.blockDim = dim3(kRrThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rbmr_step<T, D, PMAX>, ra, a);
}

template <typename T, int D>
cudaError_t launch_d(const RbmrScratch& rs, const StepParams<T>& a, uint64_t wait_ns, cudaStream_t st) {
  return (a.p <= 4) ? launch_k<T, D, 4>(rs, a, wait_ns, st) : launch_k<T, D, 32>(rs, a, wait_ns, st);
}

template <typename T, int D>
cudaError_t occupancy_d(int* nb) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_rbmr_step<T, D, 4>, kRrThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rbmr_step<T, D, 32>, kRrThreads, 0);
  *nb = (e == cudaSuccess) ? std::min(a, b) : 0;
  return e;
}

}  // namespace

int rbmr_threads() { return kRrThreads; }

cudaError_t rbmr_blocks_per_sm(int dtype, int d, int* nb) {
  if (dtype == RBM_F32) return d == 1 ? occupancy_d<float, 1>(nb) : d == 2 ? occupancy_d<float, 2>(nb) : occupancy_d<float, 3>(nb);
  return d == 1 ? occupancy_d<double, 1>(nb) : d == 2 ? occupancy_d<double, 2>(nb) : occupancy_d<double, 3>(nb);
}

template <typename T>
cudaError_t launch_rbmr(const RbmrScratch& rs, int d, const void* params, uint64_t wait_ns, const LaunchCfg& cfg,
                        cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  const cudaError_t e = (d == 1) ? launch_d<T, 1>(rs, a, wait_ns, st)
                      : (d == 2) ? launch_d<T, 2>(rs, a, wait_ns, st)
                                 : launch_d<T, 3>(rs, a, wait_ns, st);
  mark_launch(cfg, st, "k_rbmr_step");
  return e;
}

template cudaError_t launch_rbmr<float>(const RbmrScratch&, int, const void*, uint64_t, const LaunchCfg&,
                                        cudaStream_t);
template cudaError_t launch_rbmr<double>(const RbmrScratch&, int, const void*, uint64_t, const LaunchCfg&,
                                         cudaStream_t);

cudaError_t launch_rbmr_sets(uint32_t* set, uint32_t K, uint32_t n, int p, uint32_t replica, uint64_t seed,
                             int64_t m, cudaStream_t st) {
  const uint32_t grid = std::max(1u, std::min((K + 255u) / 256u, 4096u));
  k_rbmr_sets<<<grid, 256, 0, st>>>(set, K, n, p, replica,
                                    make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)), m);
  return cudaGetLastError();
}

}  // namespace rbm
