// RBM-1 step as one cooperative persistent kernel (systems of up to about
// eight million particles): one block per SM, all blocks resident, no
// grid-wide barrier in the common case and no atomics outside shared memory
// except one per (block, bucket).
//
// The random division is the id list sorted by the 64-bit Philox key with an
// id tie-break (Algorithm "randomdiv", Sec. 2.1 of arXiv:1812.10575; any
// uniform shuffle serves and this one is reproducible).  Keys are spread over
// B = k * gridDim buckets by the monotone map bucket = floor(key * B / 2^64),
// so concatenating the buckets in order after sorting each one gives the
// global order.  The random division depends on the step index only, so the
// bucketing of step m + 1 runs at the end of step m's launch (lookahead) and
// the launch boundary orders it before its use; a run's first step is
// bucketed by a launch of its own (prologue).  Per step:
//   phase 1 (of step m + 1, or the prologue): every block histograms the
//            buckets of its contiguous id range (shared-memory counters),
//            reserves its stretch of each bucket with one global atomicAdd
//            per bucket (the order of blocks inside a bucket is arbitrary:
//            phase 3 sorts every bucket completely) and scatters its ids into
//            the buckets' slots (kCap per bucket by default);
//   phase 2: every block scans the bucket totals into bucket starts (the
//            global position of each bucket in the permutation);
//   phase 3: block c takes buckets c, c + G, ...: loads the members' ids and
//            positions into shared memory, sorts them (a counting sort by the
//            next 10 key bits, then insertion sort of the few ids sharing a
//            sub-bucket by (key, id)), writes that stretch of the permutation
//            and steps every batch lying wholly inside the bucket.  The batch
//            that straddles the bucket's right boundary is stepped by the
//            same block: its missing members are the smallest keys of the
//            next bucket, selected by block-wide argmin rounds.
// When some straddling batch reaches beyond the two buckets around its
// boundary (tiny buckets: small N or large p) or a bucket outgrows shared
// memory, every block sees it in the bucket starts, and instead a further
// barrier and a phase 4 step those batches, one warp each, from the
// permutation in global memory.  A bucket that outgrows its slots (with
// kCap slots, a deviation of many standard deviations from the mean of about
// 1024) makes every block regroup its ids compactly at the bucket starts
// behind two barriers before phase 3.  The bucket totals come in three
// buffers (step m uses buffer m mod 3): the launch of step m reads its own,
// fills step m + 1's and clears step m + 2's, which the launch of step m - 1
// read, so no barrier is spent on clearing.  Slots come in two buffers
// (m mod 2).  Every update reads the positions of step m only (explicit
// scheme); no particle is written by two blocks.  Barrier
// waits are bounded by wall time; a wait that runs out latches
// RBM_ERR_TIMEOUT and the kernel returns.
#include "rbm_batch.cuh"
#include "rbm_device.cuh"
#include "rbm_grid.cuh"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr int kCoopThreads = 1024;
constexpr uint32_t kSubBits = 10;
constexpr uint32_t kSub = 1u << kSubBits;  // sub-buckets inside a bucket (one per thread)
constexpr uint32_t kCap = 2048;            // largest bucket sorted in shared memory; slots per bucket
constexpr int kMaxAdjacentPick = 7;        // straddling batches handled in phase 3 need <= 7 picks

struct CoopArgs {
  uint32_t* hist;              // [3 B] bucket totals, buffer m mod 3 for step m
  uint32_t* slots;             // [2 B slot_cap] ids grouped by bucket, buffer m mod 2
  uint32_t slot_cap;           // slots per bucket (<= kCap)
  uint32_t* tmp;               // [N] ids grouped by bucket, compact (bucket overflow only)
  uint32_t* perm;              // [N] the permutation
  unsigned long long* bar;     // [1] barrier arrival counter (monotonic)
  uint32_t n;
  uint32_t nbuckets;           // B = k G
  uint2 seed;
  PhiloxKeys keys;             // round keys of seed
  uint32_t replica;
  unsigned long long wait_ns;  // bound of one barrier wait
  int skip_arrival;            // test hook: the step first waits at a grid barrier block 0 leaves
  int prologue;                // phase 1 of step m only
  int lookahead;               // after the step, phase 1 of step m + 1
  int64_t* m_bump;             // graph replay: the step counter, advanced once every block has read it
  unsigned long long* arrive;  // [1] blocks that have read the step counter (the last one resets it)
};

// Grid barrier of this kernel (rbm_grid.cuh), with the test hook that lets
// block 0 leave without arriving.
__device__ bool grid_barrier(const CoopArgs& ca, int32_t* status, bool leave) {
  return ::rbm::grid_barrier(ca.bar, ca.wait_ns, status, leave);
}

// Exclusive scan of a[0, len) in shared memory by the whole block.
__device__ void block_exclusive_scan(uint32_t* a, uint32_t len, uint32_t* s_warp) {
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

__device__ __forceinline__ uint64_t fine_index(uint64_t key, uint32_t nbuckets) {
  return __umul64hi(key, static_cast<uint64_t>(nbuckets) << kSubBits);  // in [0, B * kSub)
}

__device__ __forceinline__ bool key_less2(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Shared-memory layout of one block (row array sized for the run's type).
struct CoopSmem {
  uint64_t* a_key;    // [kCap] keys, load order
  uint64_t* b_key;    // [kCap] keys, sorted order
  unsigned char* rows;  // [kCap] position rows, load order
  uint32_t* a_id;     // [kCap] ids, load order
  uint32_t* b_id;     // [kCap] ids, sorted order
  uint32_t* a_sub;    // [kCap] sub-bucket | rank << 16
  uint32_t* b_j;      // [kCap] load index of each sorted member
  uint32_t* s_sub;    // [kSub] sub-bucket counts, then starts
  uint32_t* s_cnt;    // [B] histogram, then this block's offsets
  uint32_t* s_start;  // [B + 1] bucket starts
};

template <typename T, int D>
__device__ __forceinline__ CoopSmem carve(unsigned char* raw, uint32_t B) {
  CoopSmem m;
  m.a_key = reinterpret_cast<uint64_t*>(raw);
  m.b_key = m.a_key + kCap;
  m.rows = reinterpret_cast<unsigned char*>(m.b_key + kCap);
  m.a_id = reinterpret_cast<uint32_t*>(m.rows + static_cast<size_t>(kCap) * sizeof(Row<T, D>));
  m.b_id = m.a_id + kCap;
  m.a_sub = m.b_id + kCap;
  m.b_j = m.a_sub + kCap;
  m.s_sub = m.b_j + kCap;
  m.s_cnt = m.s_sub + kSub;
  m.s_start = m.s_cnt + B;
  return m;
}

template <typename T, int D>
size_t coop_smem_bytes_t(uint32_t nbuckets) {
  return static_cast<size_t>(kCap) * (8 + 8 + sizeof(Row<T, D>) + 4 * 4) + kSub * 4 + (2 * nbuckets + 1) * 4;
}

// Phase 1 of step mm for this block's ids [i_lo, i_hi): bucket histogram in
// shared memory, one reservation per (block, bucket) on the totals h, and the
// ids scattered into the buckets' slots sl (ids beyond a full bucket's slots
// are dropped here and regrouped by the step that reads them).
__device__ void bucket_ids(const CoopArgs& ca, uint32_t mm, uint32_t B, uint32_t i_lo, uint32_t i_hi, uint32_t* h,
                           uint32_t* sl, uint32_t* s_cnt) {
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) s_cnt[b] = 0;
  __syncthreads();
  for (uint32_t i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
    const uint64_t key = perm_key(i, mm, ca.replica, ca.keys);
    atomicAdd(&s_cnt[static_cast<uint32_t>(fine_index(key, B) >> kSubBits)], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
    const uint32_t cnt = s_cnt[b];
    s_cnt[b] = b * ca.slot_cap + (cnt ? atomicAdd(&h[b], cnt) : 0u);  // this block's first slot in bucket b
  }
  __syncthreads();
  for (uint32_t i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
    const uint64_t key = perm_key(i, mm, ca.replica, ca.keys);
    const uint32_t b = static_cast<uint32_t>(fine_index(key, B) >> kSubBits);
    const uint32_t slot = atomicAdd(&s_cnt[b], 1u);
    if (slot < (b + 1u) * ca.slot_cap) sl[slot] = i;
  }
}

// The e smallest (key, id) among the candidates each thread holds (up to
// two: (k0, i0), (k1, i1); absent ones have valid flag false), ascending,
// into sel[0, e).  One block-wide argmin per pick with a single barrier:
// every warp publishes its minimum (double-buffered by pick parity) and every
// thread then reduces the warp minima itself.  (key, id) pairs are distinct,
// so pick r is the minimum above pick r - 1.
__device__ void select_smallest(uint64_t k0, uint32_t i0, bool v0, uint64_t k1, uint32_t i1, bool v1, int e,
                                uint32_t* sel, uint64_t* s_wkey, uint32_t* s_wid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t lk = 0;
  uint32_t li = 0;
  bool have_last = false;
  for (int r = 0; r < e; ++r) {
    uint64_t* wk = s_wkey + (r & 1) * 32;
    uint32_t* wi = s_wid + (r & 1) * 32;
    uint64_t bk = ~0ull;
    uint32_t bi = ~0u;
    if (v0 && (!have_last || key_less2(lk, li, k0, i0))) {
      bk = k0;
      bi = i0;
    }
    if (v1 && (!have_last || key_less2(lk, li, k1, i1)) && key_less2(k1, i1, bk, bi)) {
      bk = k1;
      bi = i1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (key_less2(ok, oi, bk, bi)) {
        bk = ok;
        bi = oi;
      }
    }
    if (lane == 0) {
      wk[warp] = bk;
      wi[warp] = bi;
    }
    __syncthreads();
    bk = (lane < nw) ? wk[lane] : ~0ull;
    bi = (lane < nw) ? wi[lane] : ~0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (key_less2(ok, oi, bk, bi)) {
        bk = ok;
        bi = oi;
      }
    }
    if (threadIdx.x == 0) sel[r] = bi;
    lk = bk;
    li = bi;
    have_last = true;
  }
  __syncthreads();
}

// Phase 4: warp w of block c takes boundaries c + w G, c + (w + W) G, ...
template <typename T, int D, int MODE>
__device__ void straddles_from_permutation(const CoopArgs& ca, const StepParams<T>& a, const CoopSmem& sm,
                                           uint32_t B, uint32_t m32) {
  const uint32_t G = gridDim.x, c = blockIdx.x, up = static_cast<uint32_t>(a.p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nwarps = blockDim.x >> 5;
  for (uint32_t b = c + static_cast<uint32_t>(warp) * G; b < B; b += nwarps * G) {  // warp-uniform
    bool valid = b > 0;
    uint32_t id = 0;
    int bs = a.p;
    if (valid) {
      const uint32_t s = sm.s_start[b];
      valid = (s % up != 0) && (s < a.n);
      if (valid) {
        const uint32_t q = s / up;
        valid = sm.s_start[b - 1] <= q * up;
        if (valid) {
          const uint32_t lo = q * up, hi = min(lo + up, a.n);
          bs = static_cast<int>(hi - lo);
          valid = lane < bs;
          if (valid) id = ca.perm[lo + lane];
        }
      }
    }
    batch_group<T, D, MODE>(a, m32, id, valid, lane < a.p ? lane : 0, bs);
  }
}

template <typename T, int D, int MODE>
__global__ void __launch_bounds__(kCoopThreads, 1) k_rbm_coop(CoopArgs ca, StepParams<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t B = ca.nbuckets;
  const CoopSmem sm = carve<T, D>(smem_raw, B);
  Row<T, D>* rows = reinterpret_cast<Row<T, D>*>(sm.rows);
  __shared__ uint32_t s_warp[32];
  __shared__ uint64_t s_wkey[64];
  __shared__ uint32_t s_wid[64];
  __shared__ uint32_t s_sel[kMaxAdjacentPick];
  __shared__ int s_general, s_compact;

  if (skipped(a)) return;  // uniform: the flag does not change during the launch
  const uint32_t G = gridDim.x, c = blockIdx.x;
  const uint64_t m64 = static_cast<uint64_t>((a.m_ptr ? *a.m_ptr : 0) + a.m_off);
  const uint32_t m32 = static_cast<uint32_t>(m64);
  const size_t slot_words = static_cast<size_t>(B) * ca.slot_cap;
  uint32_t* h_cur = ca.hist + (m64 % 3u) * B;          // step m's totals
  uint32_t* h_next = ca.hist + ((m64 + 1u) % 3u) * B;  // step m + 1's (filled at the end)
  uint32_t* h_free = ca.hist + ((m64 + 2u) % 3u) * B;  // step m - 1's, cleared for step m + 2
  uint32_t* sl_cur = ca.slots + (m64 & 1u) * slot_words;
  uint32_t* sl_next = ca.slots + ((m64 + 1u) & 1u) * slot_words;
  const uint32_t per = (ca.n + G - 1) / G;
  const uint32_t i_lo = min(ca.n, c * per), i_hi = min(ca.n, i_lo + per);
  const uint32_t up = static_cast<uint32_t>(a.p);

  if (ca.prologue) {
    bucket_ids(ca, m32, B, i_lo, i_hi, h_cur, sl_cur, sm.s_cnt);
    return;
  }
  if (ca.m_bump) {
    // the last block to have read the step counter advances it (no waiting)
    __syncthreads();
    if (threadIdx.x == 0 && ::rbm::atom_add_acq_rel_gpu(ca.arrive, 1ull) == G - 1) {
      *ca.arrive = 0;
      *ca.m_bump += 1;
    }
  }
  if (ca.skip_arrival && !grid_barrier(ca, a.status, c == 0)) return;  // test hook: no block passes
  for (uint32_t b = c * blockDim.x + threadIdx.x; b < B; b += G * blockDim.x) h_free[b] = 0;

  // phase 2: bucket starts (and the sub-bucket counters of phase 3 cleared)
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) sm.s_start[b] = h_cur[b];
  for (uint32_t u = threadIdx.x; u < kSub; u += blockDim.x) sm.s_sub[u] = 0;
  if (threadIdx.x == 0) {
    sm.s_start[B] = 0;
    s_general = 0;
    s_compact = 0;
  }
  __syncthreads();
  block_exclusive_scan(sm.s_start, B + 1, s_warp);  // s_start[B] becomes N
  if (sm.s_start[B] != ca.n) {
    // totals not filled for this step (a launch whose barrier wait ran out):
    // every block sees the same sum and leaves without writing
    if (threadIdx.x == 0) latch_status(a.status, RBM_ERR_STATE);
    return;
  }
  // Can every straddling batch be completed from its two adjacent buckets?
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
    const uint32_t nb = sm.s_start[b + 1] - sm.s_start[b];
    if (nb > ca.slot_cap) s_compact = 1;
    if (MODE != kModePerm) {
      bool general = nb > kCap;
      const uint32_t s = sm.s_start[b];
      if (b > 0 && s % up != 0 && s < a.n) {
        const uint32_t lo = (s / up) * up, hi = min(lo + up, a.n);
        general = general || lo < sm.s_start[b - 1] || hi > sm.s_start[b + 1] ||
                  hi - s > static_cast<uint32_t>(kMaxAdjacentPick);
      }
      if (general) s_general = 1;
    }
  }
  __syncthreads();
  const bool general = s_general != 0;
  const bool compact = s_compact != 0;
  if (compact) {
    // some bucket outgrew its slots: every block regroups its ids compactly,
    // counting places on the cleared buffer (cleared again afterwards)
    if (!grid_barrier(ca, a.status, false)) return;
    for (uint32_t i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
      const uint64_t key = perm_key(i, m32, ca.replica, ca.keys);
      const uint32_t b = static_cast<uint32_t>(fine_index(key, B) >> kSubBits);
      ca.tmp[sm.s_start[b] + atomicAdd(&h_free[b], 1u)] = i;
    }
    if (!grid_barrier(ca, a.status, false)) return;
    for (uint32_t b = c * blockDim.x + threadIdx.x; b < B; b += G * blockDim.x) h_free[b] = 0;
  }

  // phase 3: sort each of this block's buckets, write the permutation, step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b = c; b < B; b += G) {
    const uint32_t s = sm.s_start[b], nb = sm.s_start[b + 1] - s;
    const uint32_t end = s + nb;
    if (nb <= kCap) {
      // The batch straddling the right boundary is completed here from the
      // smallest keys of the next bucket (non-general mode).
      const bool straddle = (MODE != kModePerm) && !general && end < a.n && end % up != 0;
      const uint32_t n1 = straddle ? sm.s_start[b + 2] - end : 0u;
      // issue every global load of this bucket first: ids, positions, the next bucket's ids
      // (s_sub was cleared before the last barrier)
      const uint32_t t0 = threadIdx.x, t1 = threadIdx.x + blockDim.x;  // nb, n1 <= kCap = 2 * blockDim
      const uint32_t* ids = compact ? ca.tmp + s : sl_cur + static_cast<size_t>(b) * ca.slot_cap;
      const uint32_t* next_ids = compact ? ca.tmp + end : sl_cur + static_cast<size_t>(b + 1) * ca.slot_cap;
      const uint32_t id0 = (t0 < nb) ? ids[t0] : 0u;
      const uint32_t id1 = (t1 < nb) ? ids[t1] : 0u;
      const uint32_t nid0 = (t0 < n1) ? next_ids[t0] : 0u;
      const uint32_t nid1 = (t1 < n1) ? next_ids[t1] : 0u;
      Row<T, D> x0{}, x1{}, selrow{};
      if (MODE != kModePerm) {
        if (t0 < nb) x0 = load_row<T, D>(a.x, id0);
        if (t1 < nb) x1 = load_row<T, D>(a.x, id1);
      }
      if (t0 < nb) {
        const uint64_t key = perm_key(id0, m32, ca.replica, ca.keys);
        const uint32_t sub = static_cast<uint32_t>(fine_index(key, B)) & (kSub - 1u);
        const uint32_t rank = atomicAdd(&sm.s_sub[sub], 1u);
        sm.a_key[t0] = key;
        sm.a_id[t0] = id0;
        sm.a_sub[t0] = sub | (rank << 16);
      }
      if (t1 < nb) {
        const uint64_t key = perm_key(id1, m32, ca.replica, ca.keys);
        const uint32_t sub = static_cast<uint32_t>(fine_index(key, B)) & (kSub - 1u);
        const uint32_t rank = atomicAdd(&sm.s_sub[sub], 1u);
        sm.a_key[t1] = key;
        sm.a_id[t1] = id1;
        sm.a_sub[t1] = sub | (rank << 16);
      }
      if (straddle) {
        const uint32_t lo = (end / up) * up, hi = min(lo + up, a.n);
        const int pick = static_cast<int>(hi - end);
        const uint64_t nk0 = (t0 < n1) ? perm_key(nid0, m32, ca.replica, ca.keys) : ~0ull;
        const uint64_t nk1 = (t1 < n1) ? perm_key(nid1, m32, ca.replica, ca.keys) : ~0ull;
        select_smallest(nk0, nid0, t0 < n1, nk1, nid1, t1 < n1, pick, s_sel, s_wkey, s_wid);
        // the lanes of the last warp that step the picked members load their
        // rows now; the registers are read only at the straddling step
        const int own = static_cast<int>(end - lo);
        if (warp == (static_cast<int>(blockDim.x) >> 5) - 1 && lane >= own && lane < own + pick)
          selrow = load_row<T, D>(a.x, s_sel[lane - own]);
      }
      if (MODE != kModePerm) {
        if (t0 < nb) rows[t0] = x0;
        if (t1 < nb) rows[t1] = x1;
      }
      __syncthreads();
      block_exclusive_scan(sm.s_sub, kSub, s_warp);
      for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        const uint32_t pos = sm.s_sub[sm.a_sub[j] & 0xffffu] + (sm.a_sub[j] >> 16);
        sm.b_key[pos] = sm.a_key[j];
        sm.b_id[pos] = sm.a_id[j];
        sm.b_j[pos] = j;
      }
      __syncthreads();
      for (uint32_t u = threadIdx.x; u < kSub; u += blockDim.x) {
        const uint32_t lo = sm.s_sub[u], hi = (u + 1 < kSub) ? sm.s_sub[u + 1] : nb;
        for (uint32_t x = lo + 1; x < hi; ++x) {  // insertion sort of one sub-bucket
          const uint64_t kx = sm.b_key[x];
          const uint32_t ix = sm.b_id[x], jx = sm.b_j[x];
          uint32_t y = x;
          while (y > lo && key_less2(kx, ix, sm.b_key[y - 1], sm.b_id[y - 1])) {
            sm.b_key[y] = sm.b_key[y - 1];
            sm.b_id[y] = sm.b_id[y - 1];
            sm.b_j[y] = sm.b_j[y - 1];
            --y;
          }
          sm.b_key[y] = kx;
          sm.b_id[y] = ix;
          sm.b_j[y] = jx;
        }
      }
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) ca.perm[s + j] = sm.b_id[j];
      if (MODE != kModePerm) {
        // batches wholly inside the bucket, positions from shared memory
        const uint32_t q0 = (s + up - 1) / up;
        const uint32_t q_end = (end == a.n) ? (a.n + up - 1) / up : end / up;
        const uint32_t count = (q_end > q0) ? q_end - q0 : 0u;
        const int gpw = 32 / a.p, nwarps = blockDim.x >> 5;
        const uint32_t per_round = static_cast<uint32_t>(gpw * nwarps);
        const int g = lane / a.p, lg = lane - g * a.p;
        for (uint32_t r0 = 0; r0 < count; r0 += per_round) {
          const uint32_t kb = r0 + static_cast<uint32_t>(warp * gpw + g);
          bool valid = (g < gpw) && (kb < count);
          uint32_t id = 0;
          int bs = a.p;
          Row<T, D> row{};
          if (valid) {
            const uint32_t lo = (q0 + kb) * up;
            const uint32_t hi = min(lo + up, a.n);
            bs = static_cast<int>(hi - lo);
            valid = lg < bs;
            if (valid) {
              const uint32_t t = lo + lg - s;
              id = sm.b_id[t];
              row = rows[sm.b_j[t]];
            }
          }
          batch_group_row<T, D, MODE>(a, m32, id, valid, lg, bs, row);
        }
        // the batch straddling the right boundary: own tail + picked members,
        // on the last warp (idle in the contained batches above when they
        // fill fewer than all warps)
        if (!general && end < a.n && end % up != 0 && warp == (static_cast<int>(blockDim.x) >> 5) - 1) {
          const uint32_t lo = (end / up) * up, hi = min(lo + up, a.n);
          const int own = static_cast<int>(end - lo), pick = static_cast<int>(hi - end);
          const bool v = lane < own + pick;
          uint32_t idv = 0;
          Row<T, D> row{};
          if (lane < own) {
            const uint32_t t = lo + lane - s;
            idv = sm.b_id[t];
            row = rows[sm.b_j[t]];
          } else if (v) {
            idv = s_sel[lane - own];
            row = selrow;
          }
          batch_group_row<T, D, MODE>(a, m32, idv, v, lane < a.p ? lane : 0, own + pick, row);
        }
      }
    } else {
      // A bucket beyond the shared-memory sort (general and compact mode):
      // rank each member by counting the members before it.
      for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        const uint32_t idj = ca.tmp[s + j];
        const uint64_t kj = perm_key(idj, m32, ca.replica, ca.keys);
        uint32_t rank = 0;
        for (uint32_t f = 0; f < nb; ++f) {
          const uint32_t idf = ca.tmp[s + f];
          rank += key_less2(perm_key(idf, m32, ca.replica, ca.keys), idf, kj, idj) ? 1u : 0u;
        }
        ca.perm[s + rank] = idj;
      }
      __syncthreads();
      if (MODE != kModePerm) {
        const uint32_t q0 = (s + up - 1) / up;
        const uint32_t q_end = (end == a.n) ? (a.n + up - 1) / up : end / up;
        step_batches<T, D, MODE>(a, m32, ca.perm + s, s, q0, (q_end > q0) ? q_end - q0 : 0u);
      }
    }
    // s_sub is read no more in this bucket: clear it for the next one
    for (uint32_t u = threadIdx.x; u < kSub; u += blockDim.x) sm.s_sub[u] = 0;
    if (b + G < B) __syncthreads();
  }
  if (MODE != kModePerm && general) {
    if (!grid_barrier(ca, a.status, false)) return;
    // phase 4 (general mode): batches straddling a bucket boundary; warp w
    // takes boundaries c + w G, c + (w + W) G, ... (W warps per block); the
    // first boundary inside a batch takes it
    straddles_from_permutation<T, D, MODE>(ca, a, sm, B, m32);
  }
  // phase 1 of step m + 1 (reads no position; the next launch reads its totals and slots)
  if (ca.lookahead) bucket_ids(ca, m32 + 1u, B, i_lo, i_hi, h_next, sl_next, sm.s_cnt);
}

// The latency floor of the step kernel's launch shape: the same cooperative
// launch (grid, block, dynamic shared memory) with no work (a step in the
// common case waits at no grid barrier).
__global__ void __launch_bounds__(kCoopThreads, 1) k_coop_floor(int32_t* status) { (void)status; }

template <typename T, int D, int MODE>
cudaError_t launch_coop_k(const CoopScratch& cs, const StepParams<T>& a, const CoopArgs& ca, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs.grid);
  cfg.blockDim = dim3(kCoopThreads);
  cfg.dynamicSmemBytes = coop_smem_bytes_t<T, D>(cs.nbuckets);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rbm_coop<T, D, MODE>, ca, a);
}

template <typename T, int D>
cudaError_t set_attr_d(int* min_blocks) {
  const int bytes = static_cast<int>(coop_smem_bytes_t<T, D>(coop_max_buckets()));
  cudaError_t e =
      cudaFuncSetAttribute(k_rbm_coop<T, D, kModePerm>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rbm_coop<T, D, kModeStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rbm_coop<T, D, kModeForces>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int nb = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbm_coop<T, D, kModeStep>, kCoopThreads, bytes);
  if (e == cudaSuccess && nb < *min_blocks) *min_blocks = nb;
  return e;
}

}  // namespace

uint32_t coop_max_buckets() { return 8192; }
uint32_t coop_slot_capacity() { return kCap; }

cudaError_t launch_coop_floor(const CoopScratch& cs, size_t smem_bytes, uint64_t wait_ns, int32_t* status,
                              cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_coop_floor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(coop_smem_bytes_t<double, 3>(coop_max_buckets())));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs.grid);
  cfg.blockDim = dim3(kCoopThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)wait_ns;
  return cudaLaunchKernelEx(&cfg, k_coop_floor, status);
}

size_t coop_smem_bytes(int dtype, int d, uint32_t nbuckets) {
  if (dtype == RBM_F32) return d == 1 ? coop_smem_bytes_t<float, 1>(nbuckets) : d == 2 ? coop_smem_bytes_t<float, 2>(nbuckets)
                                                                                        : coop_smem_bytes_t<float, 3>(nbuckets);
  return d == 1 ? coop_smem_bytes_t<double, 1>(nbuckets) : d == 2 ? coop_smem_bytes_t<double, 2>(nbuckets)
                                                                  : coop_smem_bytes_t<double, 3>(nbuckets);
}
uint32_t coop_bucket_target() { return 1024; }

cudaError_t prepare_coop_kernels(int* blocks_per_sm) {
  int nb = 1 << 20;
  cudaError_t e = set_attr_d<float, 1>(&nb);
  if (e == cudaSuccess) e = set_attr_d<float, 2>(&nb);
  if (e == cudaSuccess) e = set_attr_d<float, 3>(&nb);
  if (e == cudaSuccess) e = set_attr_d<double, 1>(&nb);
  if (e == cudaSuccess) e = set_attr_d<double, 2>(&nb);
  if (e == cudaSuccess) e = set_attr_d<double, 3>(&nb);
  *blocks_per_sm = (e == cudaSuccess) ? nb : 0;
  return e;
}

template <typename T>
cudaError_t launch_coop(const CoopScratch& cs, int d, int mode, const void* params, uint64_t wait_ns,
                        int skip_arrival, bool prologue, bool lookahead, bool bump_step, const LaunchCfg& cfg,
                        cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  CoopArgs ca;
  ca.hist = cs.hist;
  ca.slots = cs.slots;
  ca.slot_cap = cs.slot_cap;
  ca.tmp = cs.tmp;
  ca.perm = cs.perm;
  ca.bar = cs.bar;
  ca.n = a.n;
  ca.nbuckets = cs.nbuckets;
  ca.seed = a.seed;
  ca.keys = a.keys;
  ca.replica = a.replica;
  ca.wait_ns = wait_ns;
  ca.skip_arrival = prologue ? 0 : skip_arrival;
  ca.prologue = prologue ? 1 : 0;
  ca.lookahead = lookahead ? 1 : 0;
  ca.m_bump = (bump_step && !prologue) ? const_cast<int64_t*>(a.m_ptr) : nullptr;
  ca.arrive = cs.arrive;
  cudaError_t e;
  if (d == 1) {
    e = (mode == kModeStep) ? launch_coop_k<T, 1, kModeStep>(cs, a, ca, st)
      : (mode == kModeForces) ? launch_coop_k<T, 1, kModeForces>(cs, a, ca, st)
                              : launch_coop_k<T, 1, kModePerm>(cs, a, ca, st);
  } else if (d == 2) {
    e = (mode == kModeStep) ? launch_coop_k<T, 2, kModeStep>(cs, a, ca, st)
      : (mode == kModeForces) ? launch_coop_k<T, 2, kModeForces>(cs, a, ca, st)
                              : launch_coop_k<T, 2, kModePerm>(cs, a, ca, st);
  } else {
    e = (mode == kModeStep) ? launch_coop_k<T, 3, kModeStep>(cs, a, ca, st)
      : (mode == kModeForces) ? launch_coop_k<T, 3, kModeForces>(cs, a, ca, st)
                              : launch_coop_k<T, 3, kModePerm>(cs, a, ca, st);
  }
  mark_launch(cfg, st, prologue ? "k_rbm_coop_prologue" : "k_rbm_coop");
  return e;
}

template cudaError_t launch_coop<float>(const CoopScratch&, int, int, const void*, uint64_t, int, bool, bool, bool,
                                        const LaunchCfg&, cudaStream_t);
template cudaError_t launch_coop<double>(const CoopScratch&, int, int, const void*, uint64_t, int, bool, bool, bool,
                                         const LaunchCfg&, cudaStream_t);

}  // namespace rbm
