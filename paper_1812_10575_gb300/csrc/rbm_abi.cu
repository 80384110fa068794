// C ABI of the library (include/rbm.h): context life cycle, parameter
// checks, scratch sizing, step dispatch and CUDA-graph replay.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "rbm_device.cuh"
#include "rbm_internal.h"

using namespace rbm;

struct rbm_ctx {
  rbm_params prm{};
  int ld = 1;
  size_t elem = 4;
  size_t row_bytes = 4;
  void* x = nullptr;            // caller's positions
  cudaStream_t stream = nullptr;
  int64_t m = 0;                // host copy of the step counter
  int64_t m_dev_value = -1;     // value last written to m_dev by the host side
  int32_t* status = nullptr;    // device
  int32_t* status_host = nullptr;  // pinned mirror of the status word (allocated at init)
  int64_t* m_dev = nullptr;     // device step counter read by graph replays
  void* xtmp = nullptr;         // second position buffer (direct step, generic batches)
  void* xprev = nullptr;        // Verlet: V_0 before the first step, X_{n-1} afterwards
  int64_t verlet_m0 = -1;       // Verlet: step index of the Taylor start
  void* partial = nullptr;      // direct-sum partial forces, partial_rows rows
  size_t partial_rows = 0;
  PermScratch ps;
  CoopScratch cs;
  bool batched = false;
  BatchedScratch bs;
  std::vector<int64_t> rep_n;   // replica sizes (batched contexts)
  // surrogate
  bool sur_on = false;
  SurrogateScratch ss;
  int32_t sur_every = 100, sur_iters_first = 2000, sur_iters = 200, sur_max_rounds = 1;
  int64_t sur_adam_total = 0;    // Adam iterations run so far
  bool sur_trained = false;
  bool sur_norm_given = false;   // normalisation set by the caller: keep it
  int64_t sur_last = 0;          // step of the last checkpoint
  // drift-aware schedule: the network's error on each checkpoint's fresh
  // queries before retraining (the error over the interval it drove) sets
  // the next interval; at the shortest interval an error above the
  // tolerance hands the steps to the RBM-1 fallback
  int32_t sur_interval = 100;    // steps until the next checkpoint
  int32_t sur_min_interval = 1;
  float sur_drift = -1.0f;       // last drift error (-1: none measured yet)
  bool sur_forced_off = false;   // the last checkpoint handed the steps to the fallback
  int64_t sur_forced = 0;        // intervals handed to the fallback so far
  cudaGraphExec_t sur_graph = nullptr;
  int64_t sur_graph_len = 0;
  int batched_blocks_per_sm = 0;
  bool use_coop = false;
  int64_t prepared_m = -1;   // bucket-sort path: the step whose bucket buffer is filled (-1: none)
  bool use_small = false;       // N <= 2048: the whole step in one block (the replica kernel)
  bool use_rec = false;         // RBM steps by the record path (rec_step.cu)
  RecScratch rec;
  cudaStream_t copy_stream = nullptr;  // record path, host buffers: the chunked copies
  cudaEvent_t host_ev[2 * kHostChunks + 2] = {};
  int coop_blocks_per_sm = 0;
  LaunchCfg cfg;
  rbm_tuning tuning{};
  int32_t latched = RBM_OK;     // host copy of a device error
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // by method (surrogate: sur_graph)
  int64_t graph_len[4] = {0, 0, 0, 0};
  RbmrScratch rs;                // RBM-r scratch, allocated on first use
  int32_t noise_refine = 1;      // Brownian increments shared with runs of step dt / noise_refine
};

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char* what, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

#define RBM_CUDA(call)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) {                   \
      set_error(#call, e_);                    \
      return RBM_ERR_CUDA;                     \
    }                                          \
  } while (0)

bool valid_kernel(int32_t k) { return k >= RBM_K_INV1D && k <= RBM_K_LINEAR; }

// The device status word, its pinned host mirror (read back by rbm_sync
// within the stream) and the device step counter, all cleared.  Allocated
// at init so that rbm_sync never allocates.
bool alloc_status(rbm_ctx* c) {
  if (cudaMalloc(&c->status, sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&c->m_dev, sizeof(int64_t)) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&c->status_host), sizeof(int32_t), cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaFree(c->status);
    cudaFree(c->m_dev);
    c->status = nullptr;
    c->m_dev = nullptr;
    c->status_host = nullptr;
    return false;
  }
  *c->status_host = 0;
  cudaMemset(c->status, 0, sizeof(int32_t));
  cudaMemset(c->m_dev, 0, sizeof(int64_t));
  return true;
}

void free_status(rbm_ctx* c) {
  cudaFree(c->status);
  cudaFree(c->m_dev);
  if (c->status_host) cudaFreeHost(c->status_host);
  c->status = nullptr;
  c->m_dev = nullptr;
  c->status_host = nullptr;
}

rbm_status check_params(const rbm_params* p) {
  if (!p) return RBM_ERR_INVALID;
  if (p->n < 2 || p->n > (int64_t(1) << 31)) return RBM_ERR_INVALID;
  if (p->d < 1 || p->d > 3) return RBM_ERR_INVALID;
  if (p->p < 2 || p->p > p->n || p->p > 4096) return RBM_ERR_INVALID;
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return RBM_ERR_INVALID;
  if (!(p->sigma >= 0.0) || !std::isfinite(p->sigma)) return RBM_ERR_INVALID;
  if (p->dtype != RBM_F32 && p->dtype != RBM_F64) return RBM_ERR_INVALID;
  if (p->v != RBM_V_ZERO && p->v != RBM_V_QUADRATIC) return RBM_ERR_INVALID;
  if (!valid_kernel(p->k)) return RBM_ERR_INVALID;
  if (p->k == RBM_K_INV1D && p->d != 1) return RBM_ERR_INVALID;
  if (!std::isfinite(p->v_coef) || !std::isfinite(p->k_param)) return RBM_ERR_INVALID;
  if (p->flags & ~(RBM_FLAG_RENORM_SPHERE | RBM_FLAG_GBM_NOISE)) return RBM_ERR_INVALID;
  if (p->scheme != RBM_SCHEME_EULER && p->scheme != RBM_SCHEME_SPLIT && p->scheme != RBM_SCHEME_VERLET)
    return RBM_ERR_INVALID;
  // the second-order system carries no noise and no projection (Appendix A)
  if (p->scheme == RBM_SCHEME_VERLET && (p->sigma != 0.0 || (p->flags & RBM_FLAG_RENORM_SPHERE)))
    return RBM_ERR_INVALID;
  if (p->scheme == RBM_SCHEME_SPLIT &&
      (p->p != 2 || (p->k != RBM_K_INV1D && p->k != RBM_K_COULOMB && p->k != RBM_K_LINEAR)))
    return RBM_ERR_INVALID;
  return RBM_OK;
}

void free_scratch(rbm_ctx* c) {
  PermScratch& s = c->ps;
  cudaFree(s.cnt); cudaFree(s.start); cudaFree(s.slots); cudaFree(s.ovf_cnt); cudaFree(s.ovf);
  cudaFree(s.done); cudaFree(s.perm);
  s = PermScratch{};
  cudaFree(c->cs.hist); cudaFree(c->cs.slots); cudaFree(c->cs.tmp); cudaFree(c->cs.bar); cudaFree(c->cs.arrive);
  c->cs = CoopScratch{};
  cudaFree(c->bs.order); cudaFree(c->bs.block_begin); cudaFree(c->bs.offs);
  cudaFree(c->bs.tmp); cudaFree(c->bs.perm); cudaFree(c->bs.bkt);
  {
    const int threads = c->bs.threads, target = c->bs.bucket_target;
    c->bs = BatchedScratch{};
    c->bs.threads = threads;
    c->bs.bucket_target = target;
  }
  {
    RbmrScratch& rs = c->rs;
    cudaFree(rs.set); cudaFree(rs.cnt); cudaFree(rs.start); cudaFree(rs.occ); cudaFree(rs.next);
    cudaFree(rs.flag); cudaFree(rs.btot); cudaFree(rs.remaining); cudaFree(rs.rounds); cudaFree(rs.bar);
    rs = RbmrScratch{};
  }
  rec_free(&c->rec);
  c->use_rec = false;
  cudaFree(c->xtmp);
  c->xtmp = nullptr;
  cudaFree(c->partial);
  c->partial = nullptr;
  c->partial_rows = 0;
}

void drop_graphs(rbm_ctx* c) {
  for (int i = 0; i < 4; ++i) {
    if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    c->graph[i] = nullptr;
    c->graph_len[i] = 0;
  }
}

uint32_t next_pow2(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Bucket geometry: about 1024 members per bucket by default (measured at
// N = 2^24 with the lookahead scatter: 796 us per step against 907 us with
// 512 and 1161 us with 256; even at 2^22); slots hold the
// mean plus eight standard deviations plus 64, the shared-memory sort twice
// that (power of two, at most max_sort_cap()); members beyond either bound take the
// spill list and the counting fallback, so any bucket size stays correct.
rbm_status alloc_scratch(rbm_ctx* c) {
  const uint32_t n = static_cast<uint32_t>(c->prm.n);
  PermScratch& s = c->ps;
  int bits = c->tuning.bucket_bits;
  if (bits <= 0) {
    bits = 0;
    while (bits < 22 && (static_cast<uint64_t>(n) >> bits) > 1024) ++bits;
  }
  if (bits > 24) bits = 24;
  s.bucket_bits = bits;
  s.nbuckets = 1u << bits;
  const double mean = static_cast<double>(n) / s.nbuckets;
  uint32_t cap = c->tuning.slot_cap > 0 ? static_cast<uint32_t>(c->tuning.slot_cap)
                                        : static_cast<uint32_t>(mean + 8.0 * std::sqrt(mean) + 64.0);
  if (cap > n) cap = n;
  s.slot_cap = cap;
  uint32_t sc = c->tuning.sort_cap > 0 ? next_pow2(static_cast<uint32_t>(c->tuning.sort_cap))
                                       : next_pow2(2 * cap);
  if (sc > max_sort_cap()) sc = max_sort_cap();
  if (sc < 2) sc = 2;
  s.sort_cap = sc;
  s.separate_scan = s.nbuckets > 1024;
  // two buffers: step m uses buffer m mod 2, and a step's sort kernel may
  // bucket the next step's ids into the other one
  s.double_buffer = true;
  RBM_CUDA(cudaMalloc(&s.cnt, sizeof(uint32_t) * 2 * s.nbuckets));
  RBM_CUDA(cudaMalloc(&s.start, sizeof(uint32_t) * 2 * s.nbuckets));
  RBM_CUDA(cudaMalloc(&s.slots, sizeof(uint32_t) * 2 * static_cast<size_t>(s.nbuckets) * s.slot_cap));
  RBM_CUDA(cudaMalloc(&s.ovf_cnt, sizeof(uint32_t) * 2));
  RBM_CUDA(cudaMalloc(&s.ovf, sizeof(uint32_t) * 2 * static_cast<size_t>(n)));
  RBM_CUDA(cudaMalloc(&s.done, sizeof(uint32_t) * 2));
  RBM_CUDA(cudaMalloc(&s.perm, sizeof(uint32_t) * n));
  RBM_CUDA(cudaMalloc(&c->xtmp, c->row_bytes * n));
  // Partial sums of the split direct sum: up to 64 chunks of N rows, at most 2^24 rows.
  c->partial_rows = std::min<size_t>(static_cast<size_t>(n) * 64, size_t(1) << 24);
  RBM_CUDA(cudaMalloc(&c->partial, c->row_bytes * c->partial_rows));
  RBM_CUDA(cudaMemset(s.cnt, 0, sizeof(uint32_t) * 2 * s.nbuckets));
  RBM_CUDA(cudaMemset(s.ovf_cnt, 0, sizeof(uint32_t) * 2));
  RBM_CUDA(cudaMemset(s.done, 0, sizeof(uint32_t) * 2));
  c->prepared_m = -1;
  c->cfg.block = c->tuning.block > 0 ? c->tuning.block : 256;
  c->cfg.direct_block = c->tuning.direct_block > 0 ? c->tuning.direct_block : 256;

  // Cooperative single-kernel path: one block per SM, B = k * grid buckets of
  // about 1024 members on average, B <= coop_max_buckets() (N up to about
  // 8M); batches of at most a warp.  Chosen automatically up to 11 buckets
  // per block (N about 1.7M): beyond that the multi-kernel path is faster
  // (measured with both paths bucketing ahead, d = 3, p = 2: 2^20 79 vs
  // 130 us, 2^21 149 vs 141 us, 2^22 299 vs 205 us); path = 2 forces it.
  const uint32_t grid = static_cast<uint32_t>(c->cfg.num_sms);
  const uint32_t k = static_cast<uint32_t>((static_cast<uint64_t>(n) + static_cast<uint64_t>(grid) *
                                            coop_bucket_target() - 1) / (static_cast<uint64_t>(grid) *
                                                                         coop_bucket_target()));
  const bool coop_fits = c->coop_blocks_per_sm >= 1 && c->prm.p <= 32 && k >= 1 && k * grid <= coop_max_buckets();
  c->use_coop = (c->tuning.path == 2 || (c->tuning.path == 0 && k <= 11)) && coop_fits;
  // Small systems: one block sorts all N keys in shared memory and steps
  // every batch (no grid barrier); the replica kernel with one replica.
  // Chosen automatically up to N = 1536 in FP32 and N = 384 in FP64 (the
  // measured crossovers with the cooperative kernel: FP32 14.3 vs 17.7 us at
  // N = 1000, even near 2048; FP64 25 vs 31 us at N = 256 but 52 vs 25 us at
  // N = 1000, where the FP64 transcendental work of Box-Muller and the split
  // pair flow on one SM outweighs the grid barriers).
  const bool small_fits = !c->batched && n <= 2048 && c->prm.p <= 32;
  const bool small_auto = n <= (c->prm.dtype == RBM_F32 ? 1536u : 384u);
  c->use_small = (c->tuning.path == 3 || (c->tuning.path == 0 && small_auto)) && small_fits;
  // Record path: FP32 d = 3 systems beyond the cooperative kernel's range
  // (automatic), or any size when forced (path 4).
  const bool rec_fits = !c->batched && rec_eligible(c->prm.dtype, c->prm.d, c->prm.p, c->prm.scheme);
  c->use_rec = rec_fits && !c->use_small &&
               (c->tuning.path == 4 || (c->tuning.path == 0 && !c->use_coop));
  if (c->use_rec) {
    c->use_coop = false;
    rec_geometry(n, c->tuning.bucket_bits, &c->rec);
    RBM_CUDA(rec_alloc(n, &c->rec));
  }
  if (c->use_small) {
    c->use_coop = false;
    BatchedScratch& bs = c->bs;
    int bpsm = 0;
    cudaError_t e = prepare_batched_kernels(c->prm.dtype, c->prm.d, 1024, &bpsm);
    if (e != cudaSuccess || bpsm < 1) {
      set_error("prepare_batched_kernels", e == cudaSuccess ? cudaErrorInvalidConfiguration : e);
      return RBM_ERR_CUDA;
    }
    bs.threads = 1024;
    bs.bucket_target = 2048;
    bs.grid = 1;
    bs.rep_base = static_cast<uint32_t>(c->prm.replica);
    const uint32_t order0 = 0, begin01[2] = {0, 1};
    const uint64_t offs01[2] = {0, n};
    RBM_CUDA(cudaMalloc(&bs.order, sizeof(uint32_t)));
    RBM_CUDA(cudaMalloc(&bs.block_begin, 2 * sizeof(uint32_t)));
    RBM_CUDA(cudaMalloc(&bs.offs, 2 * sizeof(uint64_t)));
    RBM_CUDA(cudaMemcpy(bs.order, &order0, sizeof(uint32_t), cudaMemcpyHostToDevice));
    RBM_CUDA(cudaMemcpy(bs.block_begin, begin01, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice));
    RBM_CUDA(cudaMemcpy(bs.offs, offs01, 2 * sizeof(uint64_t), cudaMemcpyHostToDevice));
    RBM_CUDA(cudaMalloc(&bs.tmp, sizeof(uint32_t) * n));
    RBM_CUDA(cudaMalloc(&bs.perm, sizeof(uint32_t) * n));
    RBM_CUDA(cudaMalloc(&bs.bkt, sizeof(uint16_t) * n));
  }
  if (c->use_coop) {
    CoopScratch& cs = c->cs;
    cs.grid = grid;
    cs.nbuckets = k * grid;
    RBM_CUDA(cudaMalloc(&cs.hist, sizeof(uint32_t) * 3 * cs.nbuckets));
    RBM_CUDA(cudaMemset(cs.hist, 0, sizeof(uint32_t) * 3 * cs.nbuckets));
    cs.slot_cap = coop_slot_capacity();
    if (c->tuning.slot_cap > 0 && static_cast<uint32_t>(c->tuning.slot_cap) < cs.slot_cap)
      cs.slot_cap = static_cast<uint32_t>(c->tuning.slot_cap);
    RBM_CUDA(cudaMalloc(&cs.slots, sizeof(uint32_t) * 2 * static_cast<size_t>(cs.nbuckets) * cs.slot_cap));
    RBM_CUDA(cudaMalloc(&cs.tmp, sizeof(uint32_t) * n));
    RBM_CUDA(cudaMalloc(&cs.bar, sizeof(unsigned long long)));
    RBM_CUDA(cudaMemset(cs.bar, 0, sizeof(unsigned long long)));
    RBM_CUDA(cudaMalloc(&cs.arrive, sizeof(unsigned long long)));
    RBM_CUDA(cudaMemset(cs.arrive, 0, sizeof(unsigned long long)));
    cs.perm = s.perm;
  }
  return RBM_OK;
}

// Round keys of Philox4x32-10 for a seed: (k0, k1) + r (W0, W1) mod 2^32.
PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys ks;
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = k0;
    ks.k1[r] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return ks;
}

template <typename T>
StepParams<T> step_params(const rbm_ctx* c, const int64_t* m_ptr, int64_t m_off) {
  StepParams<T> a{};
  const rbm_params& p = c->prm;
  a.x = static_cast<T*>(c->x);
  a.xout = static_cast<T*>(c->xtmp);
  a.fout = nullptr;
  a.status = c->status;
  a.n = static_cast<uint32_t>(p.n);
  a.p = p.p;
  a.kf = p.k;
  a.vkind = p.v;
  a.renorm = (p.flags & RBM_FLAG_RENORM_SPHERE) ? 1 : 0;
  a.gbm = (p.flags & RBM_FLAG_GBM_NOISE) ? 1 : 0;
  a.scheme = p.scheme;
  a.dt = static_cast<T>(p.dt);
  a.sq = static_cast<T>(p.sigma * std::sqrt(p.dt));
  a.vcoef = static_cast<T>(p.v_coef);
  a.kparam = static_cast<T>(p.k_param);
  a.radius_sq = static_cast<T>(p.k_param * p.k_param);
  a.seed = make_uint2(static_cast<uint32_t>(p.seed), static_cast<uint32_t>(p.seed >> 32));
  a.replica = p.replica;
  a.m_ptr = m_ptr;
  a.m_off = m_off;
  a.xprev = static_cast<T*>(c->xprev);
  a.verlet_m0 = c->verlet_m0;
  a.noise_refine = static_cast<uint32_t>(c->noise_refine);
  // IEEE division in the run's precision, as the kernels would compute it
  a.inv_pm1 = T(1) / static_cast<T>(p.p - 1);
  a.keys = philox_keys(p.seed);
  return a;
}

uint2 seed_of(const rbm_ctx* c) {
  return make_uint2(static_cast<uint32_t>(c->prm.seed), static_cast<uint32_t>(c->prm.seed >> 32));
}

bool uses_bucket_path(const rbm_ctx* c) { return !c->batched && !c->use_small && !c->use_coop; }
bool uses_lookahead(const rbm_ctx* c) { return !c->batched && !c->use_small && !c->use_rec; }

// Lookahead paths: clear the bucketing filled ahead (if any), so that every
// buffer is clean.  Bucket-sort path: the filled buffer; cooperative path:
// all three bucket-total buffers (its slots need no clearing).
rbm_status forget_prepared(rbm_ctx* c, cudaStream_t st) {
  if (c->use_coop && !c->use_small && !c->batched) {
    RBM_CUDA(cudaMemsetAsync(c->cs.hist, 0, sizeof(uint32_t) * 3 * c->cs.nbuckets, st));
  } else if (c->prepared_m >= 0 && uses_bucket_path(c)) {
    const size_t par = static_cast<size_t>(c->prepared_m & 1);
    RBM_CUDA(cudaMemsetAsync(c->ps.cnt + par * c->ps.nbuckets, 0, sizeof(uint32_t) * c->ps.nbuckets, st));
    RBM_CUDA(cudaMemsetAsync(c->ps.ovf_cnt + par, 0, sizeof(uint32_t), st));
  }
  c->prepared_m = -1;
  return RBM_OK;
}

// Before a captured run of RBM steps from step m: bucket step m unless the
// previous call did.
rbm_status prepare_lookahead(rbm_ctx* c, int64_t m, cudaStream_t st) {
  if (!uses_lookahead(c) || c->prepared_m == m) return RBM_OK;
  rbm_status fs = forget_prepared(c, st);
  if (fs != RBM_OK) return fs;
  if (c->use_coop) {
    const uint64_t wait_ns = 1000ull * 1000000ull;
    cudaError_t e;
    if (c->prm.dtype == RBM_F32) {
      StepParams<float> a = step_params<float>(c, nullptr, m);
      e = launch_coop<float>(c->cs, c->prm.d, 1, &a, wait_ns, 0, true, false, false, c->cfg, st);
    } else {
      StepParams<double> a = step_params<double>(c, nullptr, m);
      e = launch_coop<double>(c->cs, c->prm.d, 1, &a, wait_ns, 0, true, false, false, c->cfg, st);
    }
    if (e != cudaSuccess) {
      set_error("cudaLaunchKernelEx (cooperative)", e);
      return RBM_ERR_CUDA;
    }
  } else {
    launch_bucket_scatter(c->ps, static_cast<uint32_t>(c->prm.n), seed_of(c), c->prm.replica, nullptr, m, c->cfg,
                          st);
    RBM_CUDA(cudaGetLastError());
  }
  c->prepared_m = m;
  return RBM_OK;
}

// Host memory the device can address directly (pinned and mapped into the
// device's address space: on this platform the SMs read and write it over the
// host link): its device address, else null (pageable memory).
void* mapped_device_pointer(void* host) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();  // clear the (not sticky) error an unknown pointer leaves
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

__global__ void k_copy16(uint4* __restrict__ dst, const uint4* __restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_copy4(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

// Copy of the positions by the SMs (16-byte words when both ends allow).
cudaError_t copy_by_kernel(void* dst, const void* src, size_t bytes, const LaunchCfg& cfg, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(dst) % 16 == 0) && (reinterpret_cast<uintptr_t>(src) % 16 == 0) &&
                   bytes % 16 == 0;
  const size_t n = vec ? bytes / 16 : bytes / 4;  // rows are whole 4-byte words
  if (n == 0) return cudaSuccess;
  const size_t want = (n + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(std::min<size_t>(want, static_cast<size_t>(cfg.num_sms) * 8));
  if (vec) {
    k_copy16<<<blocks, 256, 0, st>>>(static_cast<uint4*>(dst), static_cast<const uint4*>(src), n);
    mark_launch(cfg, st, "k_copy16");
  } else {
    k_copy4<<<blocks, 256, 0, st>>>(static_cast<uint32_t*>(dst), static_cast<const uint32_t*>(src), n);
    mark_launch(cfg, st, "k_copy4");
  }
  return cudaGetLastError();
}

// Enqueue `count` RBM steps of the record path from step (*m_ptr or 0) + m_off.
rbm_status enqueue_rec(rbm_ctx* c, const int64_t* m_ptr, int64_t m_off, int64_t count, cudaStream_t st) {
  StepParams<float> a = step_params<float>(c, m_ptr, m_off);
  cudaError_t e = launch_rec_run(c->rec, &a, count, c->cfg, st);
  if (e != cudaSuccess) {
    set_error("record-path launch", e);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}

// Enqueue one RBM step (mode 1), the permutation only (0) or the forces (2).
rbm_status enqueue_rbm(rbm_ctx* c, int mode, const int64_t* m_ptr, int64_t m_off, void* fout, cudaStream_t st,
                       const int* skip = nullptr) {
  if (c->batched || c->use_small) {
    cudaError_t e;
    if (c->prm.dtype == RBM_F32) {
      StepParams<float> a = step_params<float>(c, m_ptr, m_off);
      a.fout = static_cast<float*>(fout);
      a.skip = skip;
      e = launch_batched<float>(c->bs, c->prm.d, mode, &a, c->cfg, st);
    } else {
      StepParams<double> a = step_params<double>(c, m_ptr, m_off);
      a.fout = static_cast<double*>(fout);
      a.skip = skip;
      e = launch_batched<double>(c->bs, c->prm.d, mode, &a, c->cfg, st);
    }
    if (e != cudaSuccess) {
      set_error("k_rbm_batched launch", e);
      return RBM_ERR_CUDA;
    }
    return RBM_OK;
  }
  if (c->use_coop) {
    const uint64_t wait_ns = 1000ull * static_cast<uint64_t>(c->tuning.wait_limit_us > 0 ? c->tuning.wait_limit_us
                                                                                          : 1000000);
    const int skip_hook = c->tuning.test_skip_arrival;
    // The bucketing of a step (phase 1) runs at the end of the previous
    // step's launch (lookahead) or in a prologue launch of its own: eager
    // calls launch the prologue unless the previous call bucketed this step;
    // a captured run of steps relies on the host to bucket its first step
    // before each replay (prepare_lookahead); steps gated by the surrogate's
    // flag bucket their own ids.
    const bool lookahead = (mode == 1) && skip == nullptr;
    // Graph replay of RBM steps: the step launch advances the device step
    // counter itself once every block has read it, so each captured step
    // reads the counter with offset 0.
    const bool bump = (m_ptr != nullptr) && lookahead;
    if (bump) m_off = 0;
    bool prologue = false;
    if (m_ptr == nullptr) {
      if (skip != nullptr || c->prepared_m != m_off) {
        rbm_status fs = forget_prepared(c, st);
        if (fs != RBM_OK) return fs;
        prologue = true;
      }
    } else {
      prologue = !lookahead;
    }
    cudaError_t e = cudaSuccess;
    for (int launch = prologue ? 0 : 1; launch < 2 && e == cudaSuccess; ++launch) {
      if (c->prm.dtype == RBM_F32) {
        StepParams<float> a = step_params<float>(c, m_ptr, m_off);
        a.fout = static_cast<float*>(fout);
        a.skip = skip;
        e = launch_coop<float>(c->cs, c->prm.d, mode, &a, wait_ns, skip_hook, launch == 0, lookahead, bump, c->cfg,
                               st);
      } else {
        StepParams<double> a = step_params<double>(c, m_ptr, m_off);
        a.fout = static_cast<double*>(fout);
        a.skip = skip;
        e = launch_coop<double>(c->cs, c->prm.d, mode, &a, wait_ns, skip_hook, launch == 0, lookahead, bump, c->cfg,
                                st);
      }
    }
    if (e != cudaSuccess) {
      set_error("cudaLaunchKernelEx (cooperative)", e);
      return RBM_ERR_CUDA;
    }
    if (m_ptr == nullptr) c->prepared_m = lookahead ? m_off + 1 : -1;
    return RBM_OK;
  }
  // Record path: steps (not permutation or force queries, not steps gated
  // by the surrogate's flag) move the positions as records.
  if (c->use_rec && mode == 1 && skip == nullptr) return enqueue_rec(c, m_ptr, m_off, 1, st);
  // Bucket-sort path.  A step (not a permutation or force query, not a
  // step gated by the surrogate's flag) also buckets the ids of the next step
  // (lookahead).  Eager calls skip the scatter when the previous call filled
  // this step's buffer; a captured run of steps relies on the host to fill
  // its first step's buffer before each replay (prepare_bucket_path).
  const bool lookahead = (mode == 1) && skip == nullptr;
  c->ps.skip = skip;
  if (m_ptr == nullptr) {
    if (skip != nullptr || c->prepared_m != m_off) {
      rbm_status fs = forget_prepared(c, st);
      if (fs != RBM_OK) return fs;
      launch_bucket_scatter(c->ps, static_cast<uint32_t>(c->prm.n), seed_of(c), c->prm.replica, nullptr, m_off,
                            c->cfg, st);
    }
  } else if (!lookahead) {
    launch_bucket_scatter(c->ps, static_cast<uint32_t>(c->prm.n), seed_of(c), c->prm.replica, m_ptr, m_off, c->cfg,
                          st);
  }
  if (c->prm.dtype == RBM_F32) {
    StepParams<float> a = step_params<float>(c, m_ptr, m_off);
    a.fout = static_cast<float*>(fout);
    a.skip = skip;
    launch_rbm_tail<float>(c->ps, c->prm.d, mode, &a, lookahead, c->cfg, st);
  } else {
    StepParams<double> a = step_params<double>(c, m_ptr, m_off);
    a.fout = static_cast<double*>(fout);
    a.skip = skip;
    launch_rbm_tail<double>(c->ps, c->prm.d, mode, &a, lookahead, c->cfg, st);
  }
  c->ps.skip = nullptr;
  if (m_ptr == nullptr) c->prepared_m = lookahead ? m_off + 1 : -1;
  RBM_CUDA(cudaGetLastError());
  return RBM_OK;
}

// Enqueue one direct step (mode 0), forces (1) or forces at queries (2).
rbm_status enqueue_direct(rbm_ctx* c, int mode, const int64_t* m_ptr, int64_t m_off, const void* q, uint32_t nq,
                          void* fout, cudaStream_t st) {
  if (c->prm.dtype == RBM_F32) {
    StepParams<float> a = step_params<float>(c, m_ptr, m_off);
    a.fout = static_cast<float*>(fout);
    launch_direct<float>(c->prm.d, mode, &a, static_cast<const float*>(q), nq, c->partial, c->partial_rows, c->cfg,
                         st);
  } else {
    StepParams<double> a = step_params<double>(c, m_ptr, m_off);
    a.fout = static_cast<double*>(fout);
    launch_direct<double>(c->prm.d, mode, &a, static_cast<const double*>(q), nq, c->partial, c->partial_rows,
                          c->cfg, st);
  }
  RBM_CUDA(cudaGetLastError());
  if (mode == 0)
    RBM_CUDA(cudaMemcpyAsync(c->x, c->xtmp, c->row_bytes * static_cast<size_t>(c->prm.n),
                             cudaMemcpyDeviceToDevice, st));
  return RBM_OK;
}

rbm_status enqueue_surrogate_step(rbm_ctx* c, const int64_t* m_ptr, int64_t m_off, cudaStream_t st);
rbm_status enqueue_train_round(rbm_ctx* c, int32_t iters, int32_t round, cudaStream_t st);

// RBM-r scratch for this context (once; not during graph capture).
rbm_status ensure_rbmr(rbm_ctx* c) {
  if (c->rs.set) return RBM_OK;
  if (c->batched) return RBM_ERR_UNSUPPORTED;
  if (c->prm.p > 32 || c->prm.scheme != RBM_SCHEME_EULER || (c->prm.flags & RBM_FLAG_GBM_NOISE))
    return RBM_ERR_UNSUPPORTED;
  int nb = 0;
  cudaError_t e = rbmr_blocks_per_sm(c->prm.dtype, c->prm.d, &nb);
  if (e != cudaSuccess || nb < 1) {
    set_error("rbmr_blocks_per_sm", e == cudaSuccess ? cudaErrorInvalidConfiguration : e);
    return RBM_ERR_CUDA;
  }
  RbmrScratch& rs = c->rs;
  const uint64_t n = static_cast<uint64_t>(c->prm.n), p = static_cast<uint64_t>(c->prm.p);
  const uint64_t K = std::max<uint64_t>(1, n / p);
  rs.K = static_cast<uint32_t>(K);
  rs.grid = static_cast<uint32_t>(c->cfg.num_sms);
  RBM_CUDA(cudaMalloc(&rs.set, sizeof(uint32_t) * K * p));
  RBM_CUDA(cudaMalloc(&rs.cnt, sizeof(uint32_t) * n));
  RBM_CUDA(cudaMemset(rs.cnt, 0, sizeof(uint32_t) * n));
  RBM_CUDA(cudaMalloc(&rs.start, sizeof(uint32_t) * (n + 1)));
  RBM_CUDA(cudaMalloc(&rs.occ, sizeof(uint32_t) * K * p));
  RBM_CUDA(cudaMalloc(&rs.next, sizeof(uint32_t) * n));
  RBM_CUDA(cudaMalloc(&rs.flag, K));
  RBM_CUDA(cudaMalloc(&rs.btot, sizeof(uint32_t) * rs.grid));
  RBM_CUDA(cudaMalloc(&rs.remaining, sizeof(uint32_t)));
  RBM_CUDA(cudaMalloc(&rs.rounds, sizeof(uint32_t)));
  RBM_CUDA(cudaMemset(rs.rounds, 0, sizeof(uint32_t)));
  RBM_CUDA(cudaMalloc(&rs.bar, sizeof(unsigned long long)));
  RBM_CUDA(cudaMemset(rs.bar, 0, sizeof(unsigned long long)));
  return RBM_OK;
}

rbm_status enqueue_rbmr(rbm_ctx* c, const int64_t* m_ptr, int64_t m_off, cudaStream_t st) {
  if (c->noise_refine > 1) return RBM_ERR_UNSUPPORTED;  // RBM-r draws its own increments per iteration
  const uint64_t wait_ns = 1000ull * static_cast<uint64_t>(c->tuning.wait_limit_us > 0 ? c->tuning.wait_limit_us
                                                                                        : 1000000);
  cudaError_t e;
  if (c->prm.dtype == RBM_F32) {
    StepParams<float> a = step_params<float>(c, m_ptr, m_off);
    e = launch_rbmr<float>(c->rs, c->prm.d, &a, wait_ns, c->cfg, st);
  } else {
    StepParams<double> a = step_params<double>(c, m_ptr, m_off);
    e = launch_rbmr<double>(c->rs, c->prm.d, &a, wait_ns, c->cfg, st);
  }
  if (e != cudaSuccess) {
    set_error("cudaLaunchKernelEx (RBM-r)", e);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}

rbm_status enqueue_step(rbm_ctx* c, int32_t method, const int64_t* m_ptr, int64_t m_off, cudaStream_t st) {
  if (c->prm.scheme == RBM_SCHEME_VERLET && !c->xprev) return RBM_ERR_STATE;  // no velocities yet
  if (method == RBM_METHOD_RBM) return enqueue_rbm(c, 1, m_ptr, m_off, nullptr, st);
  if (method == RBM_METHOD_RBMR) return enqueue_rbmr(c, m_ptr, m_off, st);
  if (method == RBM_METHOD_SURROGATE) return enqueue_surrogate_step(c, m_ptr, m_off, st);
  return enqueue_direct(c, 0, m_ptr, m_off, nullptr, 0, nullptr, st);
}

rbm_status usable(const rbm_ctx* c) {
  if (!c) return RBM_ERR_INVALID;
  if (c->latched != RBM_OK) return RBM_ERR_STATE;
  return RBM_OK;
}

rbm_status capture_graph(rbm_ctx* c, int32_t method, int64_t len) {
  if (!c->cap_stream) RBM_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  RBM_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  rbm_status st = RBM_OK;
  if (method == RBM_METHOD_RBM && c->use_rec) {
    st = enqueue_rec(c, c->m_dev, 0, len, c->cap_stream);  // one run: positions in x_dev again at its end
  } else {
    for (int64_t s = 0; s < len && st == RBM_OK; ++s) st = enqueue_step(c, method, c->m_dev, s, c->cap_stream);
  }
  // The cooperative RBM step advances the device step counter itself.
  const bool self_bumping = (method == RBM_METHOD_RBM && c->use_coop);
  if (st == RBM_OK && !self_bumping) launch_add_i64(c->m_dev, len, c->cap_stream);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != RBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("cudaStreamEndCapture", e);
    return RBM_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error("cudaGraphInstantiate", e);
    return RBM_ERR_CUDA;
  }
  if (method == RBM_METHOD_SURROGATE) {
    c->sur_graph = ex;
    c->sur_graph_len = len;
  } else {
    c->graph[method] = ex;
    c->graph_len[method] = len;
  }
  return RBM_OK;
}

// Replicas sorted by size (largest first) and dealt to the blocks in snake
// order (0, 1, .., G-1, G-1, .., 0, ...), so each block's total stays close
// to the mean; every block then walks its own list.
rbm_status build_batched_schedule(rbm_ctx* c) {
  BatchedScratch& bs = c->bs;
  const int32_t nrep = static_cast<int32_t>(c->rep_n.size());
  int bpsm = 0;
  cudaError_t e = prepare_batched_kernels(c->prm.dtype, c->prm.d, bs.threads, &bpsm);
  if (e != cudaSuccess || bpsm < 1) {
    set_error("prepare_batched_kernels", e == cudaSuccess ? cudaErrorInvalidConfiguration : e);
    return RBM_ERR_CUDA;
  }
  c->batched_blocks_per_sm = bpsm;
  uint32_t grid = static_cast<uint32_t>(c->cfg.num_sms) * static_cast<uint32_t>(bpsm);
  if (grid > static_cast<uint32_t>(nrep)) grid = static_cast<uint32_t>(nrep);
  std::vector<int32_t> idx(nrep);
  for (int32_t r = 0; r < nrep; ++r) idx[r] = r;
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return c->rep_n[x] > c->rep_n[y]; });
  std::vector<std::vector<uint32_t>> lists(grid);
  for (int32_t k = 0; k < nrep; ++k) {
    const uint32_t round = static_cast<uint32_t>(k) / grid, pos = static_cast<uint32_t>(k) % grid;
    const uint32_t blk = (round % 2 == 0) ? pos : grid - 1 - pos;
    lists[blk].push_back(static_cast<uint32_t>(idx[k]));
  }
  std::vector<uint32_t> order, begin(grid + 1, 0);
  for (uint32_t g = 0; g < grid; ++g) {
    begin[g] = static_cast<uint32_t>(order.size());
    order.insert(order.end(), lists[g].begin(), lists[g].end());
  }
  begin[grid] = static_cast<uint32_t>(order.size());
  cudaFree(bs.order);
  cudaFree(bs.block_begin);
  bs.order = nullptr;
  bs.block_begin = nullptr;
  RBM_CUDA(cudaMalloc(&bs.order, sizeof(uint32_t) * order.size()));
  RBM_CUDA(cudaMalloc(&bs.block_begin, sizeof(uint32_t) * begin.size()));
  RBM_CUDA(cudaMemcpy(bs.order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(bs.block_begin, begin.data(), sizeof(uint32_t) * begin.size(), cudaMemcpyHostToDevice));
  bs.grid = grid;
  return RBM_OK;
}

rbm_status alloc_batched(rbm_ctx* c) {
  BatchedScratch& bs = c->bs;
  const int32_t nrep = static_cast<int32_t>(c->rep_n.size());
  std::vector<uint64_t> offs(nrep + 1, 0);
  for (int32_t r = 0; r < nrep; ++r) offs[r + 1] = offs[r] + static_cast<uint64_t>(c->rep_n[r]);
  const size_t rows = static_cast<size_t>(offs[nrep]);
  RBM_CUDA(cudaMalloc(&bs.offs, sizeof(uint64_t) * offs.size()));
  RBM_CUDA(cudaMemcpy(bs.offs, offs.data(), sizeof(uint64_t) * offs.size(), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMalloc(&bs.tmp, sizeof(uint32_t) * rows));
  RBM_CUDA(cudaMalloc(&bs.perm, sizeof(uint32_t) * rows));
  RBM_CUDA(cudaMalloc(&bs.bkt, sizeof(uint16_t) * rows));
  RBM_CUDA(cudaMalloc(&c->xtmp, c->row_bytes * rows));
  return build_batched_schedule(c);
}

// One step of the surrogate method: the network step (runs when the flag is
// set) and the RBM step gated on the same flag (runs when it is clear).
rbm_status enqueue_surrogate_step(rbm_ctx* c, const int64_t* m_ptr, int64_t m_off, cudaStream_t st) {
  StepParams<float> a = step_params<float>(c, m_ptr, m_off);
  cudaError_t e = sur_step(c->ss, &a, c->cfg, st);
  if (e != cudaSuccess) {
    set_error("surrogate step", e);
    return RBM_ERR_CUDA;
  }
  return enqueue_rbm(c, 1, m_ptr, m_off, nullptr, st, c->ss.flag);
}

void free_surrogate(rbm_ctx* c) {
  SurrogateScratch& s = c->ss;
  cudaFree(s.theta); cudaFree(s.mom1); cudaFree(s.mom2); cudaFree(s.wq); cudaFree(s.w2f); cudaFree(s.w2b);
  cudaFree(s.norm); cudaFree(s.adam_t); cudaFree(s.flag); cudaFree(s.err); cudaFree(s.counters);
  cudaFree(s.partial); cudaFree(s.qidx); cudaFree(s.q); cudaFree(s.fq); cudaFree(s.fpred);
  s = SurrogateScratch{};
  if (c->sur_graph) cudaGraphExecDestroy(c->sur_graph);
  c->sur_graph = nullptr;
  c->sur_on = false;
}

// A checkpoint at the current step: sample queries, direct forces at them,
// (first time) the normalisation, `iters` Adam iterations on 3/4 of them,
// then the held-out error and the selection flag.
rbm_status enqueue_checkpoint(rbm_ctx* c, int32_t iters, bool first, cudaStream_t st) {
  SurrogateScratch& s = c->ss;
  StepParams<float> a = step_params<float>(c, nullptr, c->m);
  cudaError_t e = sur_sample(s, &a, st);
  if (e != cudaSuccess) {
    set_error("surrogate sample", e);
    return RBM_ERR_CUDA;
  }
  rbm_status r = enqueue_direct(c, 2, nullptr, c->m, s.q, s.nq, s.fq, st);
  if (r != RBM_OK) return r;
  if (!first) {  // the network as it drove the last interval, on the fresh queries
    e = sur_forces(s, c->status, s.q, s.nq, s.fpred, c->cfg, st);
    if (e == cudaSuccess) e = sur_drift(s, c->status, st);
    if (e != cudaSuccess) {
      set_error("surrogate drift check", e);
      return RBM_ERR_CUDA;
    }
  }
  if (first && !c->sur_norm_given) e = sur_norm(s, c->status, st);
  if (e != cudaSuccess) {
    set_error("surrogate checkpoint", e);
    return RBM_ERR_CUDA;
  }
  return enqueue_train_round(c, iters, 0, st);
}

// Round `round` (0-based) of a checkpoint: `iters` Adam iterations on the
// current queries (minibatches continue cyclically through the training
// share) with the peak rate lr / 2^round, then the held-out error and flag.
rbm_status enqueue_train_round(rbm_ctx* c, int32_t iters, int32_t round, cudaStream_t st) {
  SurrogateScratch& s = c->ss;
  const uint32_t batch = std::min<uint32_t>(4096u, s.ntrain);
  cudaError_t e = cudaSuccess;
  if (iters > 0) {
    const uint32_t begin0 = static_cast<uint32_t>((static_cast<uint64_t>(c->sur_adam_total) * batch) % s.ntrain);
    e = sur_train(s, c->status, s.q, s.fq, s.ntrain, iters, batch, begin0, std::ldexp(1.0f, -std::min(round, 60)),
                  c->cfg, st);
    c->sur_adam_total += iters;
  }
  if (e == cudaSuccess) e = sur_forces(s, c->status, s.q, s.nq, s.fpred, c->cfg, st);
  if (e == cudaSuccess) e = sur_check(s, c->status, st);
  if (e != cudaSuccess) {
    set_error("surrogate training", e);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}

// A full checkpoint: the first round (iters_first at the first checkpoint,
// iters_per_checkpoint later), then further rounds of iters_per_checkpoint
// while the held-out error is above the tolerance, up to max_rounds rounds.
// Each round restarts the geometric rate decay from a peak halved at every
// restart (warm restarts as in SGDR, Loshchilov & Hutter 2017, with a
// geometric instead of a cosine decay), so a restart cannot undo the
// convergence of the round before it.
// Reading the error back after each round is the one host synchronisation of
// the surrogate method; the steps themselves never wait on the host.
//
// Drift: the network fitted at a checkpoint goes stale as the particles
// move, so at each later checkpoint its error on the fresh queries (before
// retraining) is the error it had over the interval it just drove.  Above
// the tolerance the next interval is halved (down to the shortest,
// train_every / 16); at the shortest interval the steps go to the RBM-1
// fallback until a checkpoint measures the drift within the tolerance again;
// at or below half the tolerance the interval doubles back towards
// train_every.
rbm_status run_checkpoint(rbm_ctx* c) {
  const bool first = !c->sur_trained;
  const int64_t drove = c->m - c->sur_last;  // length of the interval the network last drove
  rbm_status st = enqueue_checkpoint(c, first ? c->sur_iters_first : c->sur_iters, first, c->stream);
  if (st != RBM_OK) return st;
  c->sur_trained = true;
  c->sur_last = c->m;
  for (int32_t round = 1; round < c->sur_max_rounds && c->sur_iters > 0; ++round) {
    float err = 0.0f;
    RBM_CUDA(cudaMemcpyAsync(&err, c->ss.err, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    RBM_CUDA(cudaStreamSynchronize(c->stream));
    if (std::isfinite(err) && err <= c->ss.tol) break;
    st = enqueue_train_round(c, c->sur_iters, round, c->stream);
    if (st != RBM_OK) return st;
  }
  if (first) {
    c->sur_interval = c->sur_every;
    c->sur_forced_off = false;
    return RBM_OK;
  }
  float drift = 0.0f;
  RBM_CUDA(cudaMemcpyAsync(&drift, c->ss.err + 1, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  RBM_CUDA(cudaStreamSynchronize(c->stream));
  c->sur_drift = drift;
  const int32_t len = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(drove, c->sur_every)));
  if (!(std::isfinite(drift) && drift <= c->ss.tol)) {
    c->sur_forced_off = len <= c->sur_min_interval;
    c->sur_interval = std::max(c->sur_min_interval, len / 2);
  } else {
    c->sur_forced_off = false;
    c->sur_interval = (drift <= 0.5f * c->ss.tol) ? std::min(c->sur_every, 2 * len) : len;
  }
  if (c->sur_forced_off) {
    RBM_CUDA(cudaMemsetAsync(c->ss.flag, 0, sizeof(int), c->stream));
    c->sur_forced += 1;
  }
  return RBM_OK;
}

}  // namespace

void rbm::set_last_error_text(const char* text) { snprintf(g_last_error, sizeof(g_last_error), "%s", text); }

namespace {

// sum_i |a_i - b_i|^2 over n rows of ld values (the first d of each row)
// into *out (FP64, atomically).
template <typename T>
__global__ void k_sq_gap(const T* __restrict__ a, const T* __restrict__ b, uint32_t n, int ld, int d, double* out) {
  double s = 0.0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int k = 0; k < d; ++k) {
      const double e = static_cast<double>(a[static_cast<size_t>(i) * ld + k]) - b[static_cast<size_t>(i) * ld + k];
      s += e * e;
    }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// E(T) of eq. "errorformula": root mean square distance of two runs of n particles.
rbm_status rms_gap(const rbm_ctx* c, const void* a, const void* b, uint32_t n, double* e) {
  double* dsum = nullptr;
  RBM_CUDA(cudaMalloc(&dsum, sizeof(double)));
  RBM_CUDA(cudaMemset(dsum, 0, sizeof(double)));
  const unsigned blocks = std::min<unsigned>((n + 255) / 256, static_cast<unsigned>(c->cfg.num_sms) * 4);
  if (c->prm.dtype == RBM_F32)
    k_sq_gap<float><<<std::max(blocks, 1u), 256>>>(static_cast<const float*>(a), static_cast<const float*>(b), n,
                                                   c->ld, c->prm.d, dsum);
  else
    k_sq_gap<double><<<std::max(blocks, 1u), 256>>>(static_cast<const double*>(a), static_cast<const double*>(b), n,
                                                    c->ld, c->prm.d, dsum);
  double h = 0.0;
  const cudaError_t e1 = cudaMemcpy(&h, dsum, sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dsum);
  if (e1 != cudaSuccess) {
    set_error("rms_gap", e1);
    return RBM_ERR_CUDA;
  }
  *e = std::sqrt(h / static_cast<double>(n));
  return RBM_OK;
}

// A pilot run: n particles from x0 (device, copied), parameters prm with
// batch size p and step dt, noise refinement r, `steps` steps of `method`;
// the final positions into xout (device, n rows).
rbm_status pilot_run(const rbm_params& base, int32_t p, double dt, int32_t r, int64_t steps, int32_t method,
                     const void* x0, void* xout, size_t bytes) {
  RBM_CUDA(cudaMemcpy(xout, x0, bytes, cudaMemcpyDeviceToDevice));
  rbm_params prm = base;
  prm.p = p;
  prm.dt = dt;
  rbm_ctx* pc = nullptr;
  rbm_status st = rbm_init(&prm, xout, nullptr, &pc);
  if (st != RBM_OK) return st;
  st = rbm_set_noise_refinement(pc, r);
  if (st == RBM_OK) st = rbm_run(pc, steps, method);
  const rbm_status ss = rbm_sync(pc);
  if (st == RBM_OK) st = ss;
  rbm_free(pc);
  return st;
}

}  // namespace

extern "C" {

const char* rbm_last_error(void) { return g_last_error; }

const char* rbm_status_string(int32_t status) {
  switch (status) {
    case RBM_OK: return "ok";
    case RBM_ERR_INVALID: return "invalid argument";
    case RBM_ERR_CUDA: return "CUDA runtime error";
    case RBM_ERR_NOMEM: return "out of memory";
    case RBM_ERR_TIMEOUT: return "device wait timed out";
    case RBM_ERR_NONFINITE: return "non-finite position";
    case RBM_ERR_STATE: return "context unusable after an earlier error";
    case RBM_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

rbm_status rbm_init(const rbm_params* prm, void* x_dev, void* cuda_stream, rbm_ctx** out) {
  if (!out) return RBM_ERR_INVALID;
  *out = nullptr;
  rbm_status st = check_params(prm);
  if (st != RBM_OK) return st;
  if (!x_dev || (reinterpret_cast<uintptr_t>(x_dev) & 15u)) return RBM_ERR_INVALID;
  rbm_ctx* c = new (std::nothrow) rbm_ctx();
  if (!c) return RBM_ERR_NOMEM;
  c->prm = *prm;
  c->ld = (prm->d == 3) ? 4 : prm->d;
  c->elem = (prm->dtype == RBM_F32) ? 4 : 8;
  c->row_bytes = c->elem * c->ld;
  c->x = x_dev;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    c->cfg.num_sms = sms;
  {
    cudaError_t e = prepare_rbm_kernels();
    if (e == cudaSuccess) e = prepare_rec_kernels();
    if (e == cudaSuccess) e = prepare_coop_kernels(&c->coop_blocks_per_sm);
    if (e != cudaSuccess) {
      set_error("prepare_rbm_kernels", e);
      delete c;
      return RBM_ERR_CUDA;
    }
  }
  if (!alloc_status(c)) {
    delete c;
    return RBM_ERR_NOMEM;
  }
  c->tuning.graph_steps = 100;
  st = alloc_scratch(c);
  if (st != RBM_OK) {
    free_scratch(c);
    free_status(c);
    delete c;
    return st == RBM_ERR_CUDA ? RBM_ERR_NOMEM : st;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_scratch(c);
    free_status(c);
    delete c;
    return RBM_ERR_CUDA;
  }
  *out = c;
  return RBM_OK;
}

rbm_status rbm_step(rbm_ctx* ctx) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  st = enqueue_step(ctx, RBM_METHOD_RBM, nullptr, ctx->m, ctx->stream);
  if (st == RBM_OK) ctx->m += 1;
  return st;
}

rbm_status rbm_direct_step(rbm_ctx* ctx) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (ctx->batched) return RBM_ERR_UNSUPPORTED;
  st = enqueue_step(ctx, RBM_METHOD_DIRECT, nullptr, ctx->m, ctx->stream);
  if (st == RBM_OK) ctx->m += 1;
  return st;
}

rbm_status rbm_run(rbm_ctx* ctx, int64_t steps, int32_t method) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (steps < 0 || (method != RBM_METHOD_RBM && method != RBM_METHOD_DIRECT && method != RBM_METHOD_SURROGATE &&
                     method != RBM_METHOD_RBMR))
    return RBM_ERR_INVALID;
  if (ctx->batched && method != RBM_METHOD_RBM) return RBM_ERR_UNSUPPORTED;
  if (method == RBM_METHOD_RBMR) {
    st = ensure_rbmr(ctx);
    if (st != RBM_OK) return st;
  }
  if (method == RBM_METHOD_SURROGATE) {
    if (!ctx->sur_on) return RBM_ERR_STATE;
    while (steps > 0) {
      if (!ctx->sur_trained || ctx->m - ctx->sur_last >= ctx->sur_interval) {
        st = run_checkpoint(ctx);
        if (st != RBM_OK) return st;
      }
      const int64_t cycle = std::min<int64_t>(steps, ctx->sur_interval - (ctx->m - ctx->sur_last));
      if (cycle == ctx->sur_interval) {  // a whole cycle: replay its graph (one per interval length)
        if (!ctx->sur_graph || ctx->sur_graph_len != cycle) {
          if (ctx->sur_graph) cudaGraphExecDestroy(ctx->sur_graph);
          ctx->sur_graph = nullptr;
          st = capture_graph(ctx, RBM_METHOD_SURROGATE, cycle);
          if (st != RBM_OK) return st;
        }
        if (ctx->m_dev_value != ctx->m) launch_set_i64(ctx->m_dev, ctx->m, ctx->stream);
        st = forget_prepared(ctx, ctx->stream);  // its RBM steps scatter their own ids
        if (st != RBM_OK) return st;
        RBM_CUDA(cudaGraphLaunch(ctx->sur_graph, ctx->stream));
        ctx->m += cycle;
        ctx->m_dev_value = ctx->m;
      } else {
        for (int64_t s2 = 0; s2 < cycle; ++s2) {
          st = enqueue_step(ctx, RBM_METHOD_SURROGATE, nullptr, ctx->m, ctx->stream);
          if (st != RBM_OK) return st;
          ctx->m += 1;
        }
      }
      steps -= cycle;
    }
    return RBM_OK;
  }
  const int64_t len = ctx->tuning.graph_steps > 0 ? ctx->tuning.graph_steps : 100;
  while (steps >= len) {
    if (!ctx->graph[method] || ctx->graph_len[method] != len) {
      if (ctx->graph[method]) cudaGraphExecDestroy(ctx->graph[method]);
      ctx->graph[method] = nullptr;
      st = capture_graph(ctx, method, len);
      if (st != RBM_OK) return st;
    }
    if (ctx->m_dev_value != ctx->m) launch_set_i64(ctx->m_dev, ctx->m, ctx->stream);
    if (method == RBM_METHOD_RBM) {
      st = prepare_lookahead(ctx, ctx->m, ctx->stream);
      if (st != RBM_OK) return st;
    }
    RBM_CUDA(cudaGraphLaunch(ctx->graph[method], ctx->stream));
    ctx->m += len;
    ctx->m_dev_value = ctx->m;
    if (method == RBM_METHOD_RBM && uses_lookahead(ctx)) ctx->prepared_m = ctx->m;  // the last step's lookahead
    steps -= len;
  }
  if (steps > 0 && method == RBM_METHOD_RBM && ctx->use_rec) {
    st = enqueue_rec(ctx, nullptr, ctx->m, steps, ctx->stream);  // the remaining steps as one run
    if (st != RBM_OK) return st;
    ctx->m += steps;
    return RBM_OK;
  }
  for (; steps > 0; --steps) {
    st = enqueue_step(ctx, method, nullptr, ctx->m, ctx->stream);
    if (st != RBM_OK) return st;
    ctx->m += 1;
  }
  return RBM_OK;
}

rbm_status rbm_sync(rbm_ctx* ctx) {
  if (!ctx) return RBM_ERR_INVALID;
  // the status word rides the stream into pinned memory (allocated at init):
  // one wait, not two; the stream is drained even when the copy cannot be
  // enqueued, so the call always returns after the stream's work
  const cudaError_t ec = cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                         ctx->stream);
  const cudaError_t ew = cudaStreamSynchronize(ctx->stream);
  if (ec != cudaSuccess) {
    set_error("cudaMemcpyAsync(status)", ec);
    return RBM_ERR_CUDA;
  }
  if (ew != cudaSuccess) {
    set_error("cudaStreamSynchronize", ew);
    return RBM_ERR_CUDA;
  }
  const int32_t s = *static_cast<volatile int32_t*>(ctx->status_host);
  if (s != 0 && ctx->latched == RBM_OK) ctx->latched = s;
  return static_cast<rbm_status>(ctx->latched);
}

rbm_status rbm_step_host(rbm_ctx* ctx, void* x_host, int32_t method) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!x_host || (method != RBM_METHOD_RBM && method != RBM_METHOD_DIRECT && method != RBM_METHOD_SURROGATE &&
                  method != RBM_METHOD_RBMR))
    return RBM_ERR_INVALID;
  if (method == RBM_METHOD_SURROGATE && !ctx->sur_on) return RBM_ERR_STATE;
  if (method == RBM_METHOD_RBMR) {
    st = ensure_rbmr(ctx);
    if (st != RBM_OK) return st;
  }
  const size_t bytes = ctx->row_bytes * static_cast<size_t>(ctx->prm.n);
  // Pinned host memory mapped into the device's address space is read and
  // written by a copy kernel when the positions are small (up to 16 MB: the
  // copy engine's setup dominates there; measured e2e at N = 1e5, 1.6 MB:
  // 1.57e9 against 1.50e9 particle-steps/s); larger or pageable buffers take
  // cudaMemcpyAsync (at 400 MB the copy engine was 2 % faster).
  void* mapped = (bytes <= (size_t(16) << 20)) ? mapped_device_pointer(x_host) : nullptr;
  if (!mapped && method == RBM_METHOD_RBM && ctx->use_rec) {
    // the record path copies in and scatters, and places and copies out, in
    // chunks on two streams (the kernels of one chunk under the next one's copy)
    if (!ctx->copy_stream) RBM_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : ctx->host_ev)
      if (!ev) RBM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    StepParams<float> a = step_params<float>(ctx, nullptr, ctx->m);
    const cudaError_t e = launch_rec_host_step(ctx->rec, &a, x_host, ctx->cfg, ctx->stream, ctx->copy_stream,
                                               ctx->host_ev);
    if (e != cudaSuccess) {
      set_error("record-path host step", e);
      return RBM_ERR_CUDA;
    }
    ctx->m += 1;
    return rbm_sync(ctx);
  }
  if (mapped) RBM_CUDA(copy_by_kernel(ctx->x, mapped, bytes, ctx->cfg, ctx->stream));
  else RBM_CUDA(cudaMemcpyAsync(ctx->x, x_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  st = enqueue_step(ctx, method, nullptr, ctx->m, ctx->stream);
  if (st != RBM_OK) return st;
  ctx->m += 1;
  if (mapped) RBM_CUDA(copy_by_kernel(mapped, ctx->x, bytes, ctx->cfg, ctx->stream));
  else RBM_CUDA(cudaMemcpyAsync(x_host, ctx->x, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return rbm_sync(ctx);
}

rbm_status rbm_get_step(const rbm_ctx* ctx, int64_t* m) {
  if (!ctx || !m) return RBM_ERR_INVALID;
  *m = ctx->m;
  return RBM_OK;
}

rbm_status rbm_set_step(rbm_ctx* ctx, int64_t m) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (m < 0) return RBM_ERR_INVALID;
  ctx->m = m;
  return RBM_OK;
}

rbm_status rbm_set_noise_refinement(rbm_ctx* ctx, int32_t r) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (r < 1 || r > 65536) return RBM_ERR_INVALID;
  if (r == ctx->noise_refine) return RBM_OK;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);  // the captured launches carry the old value
  if (ctx->sur_graph) cudaGraphExecDestroy(ctx->sur_graph);
  ctx->sur_graph = nullptr;
  ctx->sur_graph_len = 0;
  ctx->noise_refine = r;
  return RBM_OK;
}

rbm_status rbm_get_noise_refinement(const rbm_ctx* ctx, int32_t* r) {
  if (!ctx || !r) return RBM_ERR_INVALID;
  *r = ctx->noise_refine;
  return RBM_OK;
}

rbm_status rbm_set_tuning(rbm_ctx* ctx, const rbm_tuning* tuning) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!tuning) return RBM_ERR_INVALID;
  if (tuning->bucket_bits < 0 || tuning->bucket_bits > 24 || tuning->slot_cap < 0 || tuning->sort_cap < 0 ||
      tuning->sort_cap > 4096 || tuning->graph_steps < 0 || tuning->path < 0 || tuning->path > 4 ||
      tuning->wait_limit_us < 0 || tuning->test_skip_arrival < 0 || tuning->test_skip_arrival > 1)
    return RBM_ERR_INVALID;
  if ((tuning->block != 0 && tuning->block != 256) ||
      (tuning->direct_block != 0 && (tuning->direct_block < 32 || tuning->direct_block > 1024 ||
                                     tuning->direct_block % 32 != 0)))
    return RBM_ERR_INVALID;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  if (ctx->batched) {  // batched contexts take only the graph length here
    ctx->tuning.graph_steps = tuning->graph_steps > 0 ? tuning->graph_steps : 100;
    return RBM_OK;
  }
  free_scratch(ctx);
  ctx->tuning = *tuning;
  if (ctx->tuning.graph_steps == 0) ctx->tuning.graph_steps = 100;
  st = alloc_scratch(ctx);
  if (st != RBM_OK) {
    ctx->latched = st;
    return st;
  }
  RBM_CUDA(cudaDeviceSynchronize());
  return RBM_OK;
}

rbm_status rbm_get_tuning(const rbm_ctx* ctx, rbm_tuning* tuning) {
  if (!ctx || !tuning) return RBM_ERR_INVALID;
  *tuning = ctx->tuning;
  tuning->bucket_bits = ctx->ps.bucket_bits;
  tuning->slot_cap = static_cast<int32_t>(ctx->use_coop ? ctx->cs.slot_cap : ctx->ps.slot_cap);
  tuning->sort_cap = static_cast<int32_t>(ctx->ps.sort_cap);
  tuning->block = ctx->cfg.block;
  tuning->direct_block = ctx->cfg.direct_block;
  tuning->path = ctx->use_small ? 3 : ctx->use_coop ? 2 : ctx->use_rec ? 4 : 1;
  return RBM_OK;
}

rbm_status rbm_free(rbm_ctx* ctx) {
  if (!ctx) return RBM_ERR_INVALID;
  cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx);
  free_surrogate(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (cudaEvent_t ev : ctx->host_ev)
    if (ev) cudaEventDestroy(ev);
  free_scratch(ctx);
  cudaFree(ctx->xprev);
  free_status(ctx);
  delete ctx;
  return RBM_OK;
}

rbm_status rbm_permutation(rbm_ctx* ctx, uint32_t* perm_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!perm_dev) return RBM_ERR_INVALID;
  st = enqueue_rbm(ctx, 0, nullptr, ctx->m, nullptr, ctx->stream);
  if (st != RBM_OK) return st;
  RBM_CUDA(cudaMemcpyAsync(perm_dev, (ctx->batched || ctx->use_small) ? ctx->bs.perm : ctx->ps.perm,
                           sizeof(uint32_t) * static_cast<size_t>(ctx->prm.n),
                           cudaMemcpyDeviceToDevice, ctx->stream));
  return RBM_OK;
}

rbm_status rbm_forces(rbm_ctx* ctx, int32_t method, void* f_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!f_dev || (reinterpret_cast<uintptr_t>(f_dev) & 15u)) return RBM_ERR_INVALID;
  if (method == RBM_METHOD_RBM) return enqueue_rbm(ctx, 2, nullptr, ctx->m, f_dev, ctx->stream);
  if (method == RBM_METHOD_DIRECT) {
    if (ctx->batched) return RBM_ERR_UNSUPPORTED;
    return enqueue_direct(ctx, 1, nullptr, ctx->m, nullptr, 0, f_dev, ctx->stream);
  }
  return RBM_ERR_INVALID;
}

rbm_status rbm_direct_forces_at(rbm_ctx* ctx, const void* q_dev, int64_t nq, void* f_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (nq < 0 || nq > (int64_t(1) << 31)) return RBM_ERR_INVALID;
  if (ctx->batched) return RBM_ERR_UNSUPPORTED;
  if (nq == 0) return RBM_OK;
  if (!q_dev || !f_dev || (reinterpret_cast<uintptr_t>(q_dev) & 15u) || (reinterpret_cast<uintptr_t>(f_dev) & 15u))
    return RBM_ERR_INVALID;
  return enqueue_direct(ctx, 2, nullptr, ctx->m, q_dev, static_cast<uint32_t>(nq), f_dev, ctx->stream);
}

rbm_status rbm_step_profiled(rbm_ctx* ctx, int32_t method, float* kernel_ms, int32_t capacity, int32_t* nkernels,
                             char* names, int32_t names_len) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!kernel_ms || !nkernels || capacity < 1 ||
      (method != RBM_METHOD_RBM && method != RBM_METHOD_DIRECT && method != RBM_METHOD_SURROGATE &&
       method != RBM_METHOD_RBMR))
    return RBM_ERR_INVALID;
  if (method == RBM_METHOD_SURROGATE && !ctx->sur_on) return RBM_ERR_STATE;
  if (method == RBM_METHOD_RBMR) {
    st = ensure_rbmr(ctx);
    if (st != RBM_OK) return st;
  }
  constexpr int kMax = 16;
  cudaEvent_t ev[kMax + 1];
  const char* nm[kMax + 1] = {};
  for (int i = 0; i <= kMax; ++i) RBM_CUDA(cudaEventCreate(&ev[i]));
  int nev = 0;
  LaunchCfg saved = ctx->cfg;
  ctx->cfg.events = ev;
  ctx->cfg.nevents = &nev;
  ctx->cfg.max_events = kMax + 1;
  ctx->cfg.names = nm;
  mark_launch(ctx->cfg, ctx->stream, "start");
  // The record path profiles a run of two steps: its first step's kernels
  // are those of every step of a run but the last.
  const int64_t nsteps = (method == RBM_METHOD_RBM && ctx->use_rec) ? 2 : 1;
  if (nsteps == 2) st = enqueue_rec(ctx, nullptr, ctx->m, 2, ctx->stream);
  else st = enqueue_step(ctx, method, nullptr, ctx->m, ctx->stream);
  ctx->cfg = saved;
  if (st == RBM_OK) {
    ctx->m += nsteps;
    cudaError_t e = cudaEventSynchronize(ev[nev - 1]);
    const int nk = nev - 1;
    *nkernels = nk;
    std::string joined;
    for (int i = 0; i < nk && i < capacity && e == cudaSuccess; ++i) {
      e = cudaEventElapsedTime(&kernel_ms[i], ev[i], ev[i + 1]);
      if (i) joined += ";";
      joined += nm[i + 1] ? nm[i + 1] : "?";
    }
    if (names && names_len > 0) {
      std::strncpy(names, joined.c_str(), static_cast<size_t>(names_len) - 1);
      names[names_len - 1] = 0;
    }
    if (e != cudaSuccess) {
      set_error("cudaEventElapsedTime", e);
      st = RBM_ERR_CUDA;
    }
  }
  for (int i = 0; i <= kMax; ++i) cudaEventDestroy(ev[i]);
  if (st == RBM_OK) st = rbm_sync(ctx);
  return st;
}

rbm_status rbm_batched_init(const rbm_params* base, int32_t nrep, const int64_t* n_host, void* x_dev,
                            void* cuda_stream, rbm_ctx** out) {
  if (!out) return RBM_ERR_INVALID;
  *out = nullptr;
  if (!base || !n_host || nrep < 1) return RBM_ERR_INVALID;
  int64_t total = 0;
  for (int32_t r = 0; r < nrep; ++r) {
    if (n_host[r] < 2 || n_host[r] > (int64_t(1) << 20)) return RBM_ERR_INVALID;
    total += n_host[r];
  }
  if (total != base->n) return RBM_ERR_INVALID;
  rbm_params prm = *base;
  prm.p = std::max<int32_t>(2, prm.p);
  // validate the shared parameters as for one system of size max(N_r, p)
  rbm_params chk = prm;
  chk.n = std::max<int64_t>(total, prm.p);
  rbm_status st = check_params(&chk);
  if (st != RBM_OK) return st;
  if (prm.p > 32 || prm.scheme != RBM_SCHEME_EULER) return RBM_ERR_INVALID;
  if (!x_dev || (reinterpret_cast<uintptr_t>(x_dev) & 15u)) return RBM_ERR_INVALID;
  rbm_ctx* c = new (std::nothrow) rbm_ctx();
  if (!c) return RBM_ERR_NOMEM;
  c->prm = prm;
  c->batched = true;
  c->rep_n.assign(n_host, n_host + nrep);
  c->ld = (prm.d == 3) ? 4 : prm.d;
  c->elem = (prm.dtype == RBM_F32) ? 4 : 8;
  c->row_bytes = c->elem * c->ld;
  c->x = x_dev;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    c->cfg.num_sms = sms;
  c->tuning.graph_steps = 100;
  if (!alloc_status(c)) {
    delete c;
    return RBM_ERR_NOMEM;
  }
  st = alloc_batched(c);
  if (st != RBM_OK || cudaDeviceSynchronize() != cudaSuccess) {
    free_scratch(c);
    free_status(c);
    delete c;
    return st != RBM_OK ? st : RBM_ERR_CUDA;
  }
  *out = c;
  return RBM_OK;
}

rbm_status rbm_batched_set_launch(rbm_ctx* ctx, int32_t threads, int32_t bucket_target) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->batched) return RBM_ERR_INVALID;
  if ((threads != 256 && threads != 512 && threads != 1024) || bucket_target < 64 || bucket_target > 2048)
    return RBM_ERR_INVALID;
  int bpsm = 0;
  if (prepare_batched_kernels(ctx->prm.dtype, ctx->prm.d, threads, &bpsm) != cudaSuccess || bpsm < 1)
    return RBM_ERR_UNSUPPORTED;  // this block size does not fit the kernel's registers; shape unchanged
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  ctx->bs.threads = threads;
  ctx->bs.bucket_target = bucket_target;
  return build_batched_schedule(ctx);
}

rbm_status rbm_autotune(rbm_ctx* ctx, int32_t trial_steps, const char* table_path, char* report, int32_t report_len) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (trial_steps < 1) return RBM_ERR_INVALID;
  // workload signature: kind, dtype, d, p, kernel, rows, replicas, size sum of squares
  std::ostringstream sig;
  uint64_t sq = 0;
  for (int64_t n : ctx->rep_n) sq += static_cast<uint64_t>(n) * static_cast<uint64_t>(n);
  sig << (ctx->batched ? "batched" : "single") << ":" << ctx->prm.dtype << ":" << ctx->prm.d << ":" << ctx->prm.p
      << ":" << ctx->prm.k << ":" << ctx->prm.n << ":" << ctx->rep_n.size() << ":" << sq;
  const std::string key = sig.str();
  std::string found;
  if (table_path) {
    std::ifstream in(table_path);
    std::string line;
    while (std::getline(in, line))
      if (line.compare(0, key.size() + 1, key + " ") == 0) found = line.substr(key.size() + 1);
  }
  std::string result;
  if (!found.empty()) {
    std::istringstream is(found);
    int a = 0, b = 0;
    is >> a >> b;
    if (ctx->batched) st = rbm_batched_set_launch(ctx, a, b);
    else {
      rbm_tuning t = ctx->tuning;
      t.path = a;
      t.direct_block = 0;
      st = rbm_set_tuning(ctx, &t);
    }
    result = "table " + key + " " + found;
  } else {
    // time candidates on a scratch copy of the state (the step index is left as it is)
    RBM_CUDA(cudaStreamSynchronize(ctx->stream));
    const size_t bytes = ctx->row_bytes * static_cast<size_t>(ctx->prm.n);
    void* scratch = nullptr;
    RBM_CUDA(cudaMalloc(&scratch, bytes));
    void* real_x = ctx->x;
    std::vector<std::pair<int, int>> cands;
    if (ctx->batched) {
      // mean bucket sizes well below the 2048-member shared-memory sort, so
      // the counting fallback for an oversized bucket stays out of the trial
      for (int th : {256, 512, 1024})
        for (int bt : {256, 512, 1024}) cands.push_back({th, bt});
    } else {
      cands.push_back({1, 0});
      cands.push_back({2, 0});
      cands.push_back({3, 0});
      cands.push_back({4, 0});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> best_c = cands[0];
    std::ostringstream rep;
    for (const auto& cd : cands) {
      if (ctx->batched) {
        st = rbm_batched_set_launch(ctx, cd.first, cd.second);
        if (st == RBM_ERR_UNSUPPORTED) {  // block size not available for this kernel
          st = RBM_OK;
          continue;
        }
      } else {
        rbm_tuning t = ctx->tuning;
        t.path = cd.first;
        st = rbm_set_tuning(ctx, &t);
        if (st == RBM_OK && ((ctx->use_small ? 3 : ctx->use_coop ? 2 : ctx->use_rec ? 4 : 1) != cd.first))
          continue;  // not available
      }
      if (st != RBM_OK) break;
      cudaMemcpyAsync(scratch, real_x, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
      ctx->x = scratch;
      const int64_t m0 = ctx->m;
      enqueue_step(ctx, RBM_METHOD_RBM, nullptr, m0, ctx->stream);  // warm-up
      cudaEventRecord(e0, ctx->stream);
      if (ctx->use_rec) {  // the record path runs its steps as one run, as rbm_run does
        enqueue_rec(ctx, nullptr, m0, trial_steps, ctx->stream);
      } else {
        for (int32_t s = 0; s < trial_steps; ++s) enqueue_step(ctx, RBM_METHOD_RBM, nullptr, m0, ctx->stream);
      }
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      ctx->x = real_x;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= static_cast<float>(trial_steps);
      rep << cd.first << "," << cd.second << "=" << ms << "ms ";
      if (ms < best) {
        best = ms;
        best_c = cd;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    ctx->x = real_x;
    if (st == RBM_OK) {
      if (ctx->batched) st = rbm_batched_set_launch(ctx, best_c.first, best_c.second);
      else {
        rbm_tuning t = ctx->tuning;
        t.path = best_c.first;
        st = rbm_set_tuning(ctx, &t);
      }
    }
    if (st == RBM_OK && table_path) {
      std::ofstream outf(table_path, std::ios::app);
      outf << key << " " << best_c.first << " " << best_c.second << "\n";
    }
    std::ostringstream r2;
    r2 << "searched " << key << " best " << best_c.first << " " << best_c.second << " (" << best << " ms/step): "
       << rep.str();
    result = r2.str();
  }
  if (report && report_len > 0) {
    std::strncpy(report, result.c_str(), static_cast<size_t>(report_len) - 1);
    report[report_len - 1] = 0;
  }
  return st;
}

rbm_status rbm_set_batch_size(rbm_ctx* ctx, int32_t p) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  rbm_params chk = ctx->prm;
  chk.p = p;
  if (ctx->batched) {
    chk.n = std::max<int64_t>(chk.n, p);
    if (p > 32) return RBM_ERR_INVALID;
  }
  st = check_params(&chk);
  if (st != RBM_OK) return st;
  if (p == ctx->prm.p) return RBM_OK;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  if (ctx->sur_graph) cudaGraphExecDestroy(ctx->sur_graph);
  ctx->sur_graph = nullptr;
  ctx->sur_graph_len = 0;
  ctx->prm.p = p;
  free_scratch(ctx);
  st = ctx->batched ? alloc_batched(ctx) : alloc_scratch(ctx);
  if (st != RBM_OK) {
    ctx->latched = st;
    return st;
  }
  RBM_CUDA(cudaDeviceSynchronize());
  return RBM_OK;
}

rbm_status rbm_autotune_accuracy(rbm_ctx* ctx, const int32_t* ps, int32_t nps, double eps, double horizon,
                                 int32_t max_halvings, int64_t pilot_n, int32_t trial_steps, const char* table_path,
                                 int32_t* p_out, double* dt_out, int32_t* met_out, char* report, int32_t report_len) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ps || nps < 1 || nps > 16 || !(eps > 0) || !(horizon > 0) || max_halvings < 0 || max_halvings > 8 ||
      pilot_n < 2 || trial_steps < 1)
    return RBM_ERR_INVALID;
  if (ctx->prm.scheme == RBM_SCHEME_VERLET) return RBM_ERR_UNSUPPORTED;  // needs velocities: not a pilot
  for (int32_t i = 0; i < nps; ++i) {
    rbm_params chk = ctx->prm;
    chk.p = ps[i];
    chk.n = std::max<int64_t>(chk.n, ps[i]);
    if (check_params(&chk) != RBM_OK || (ctx->batched && ps[i] > 32)) return RBM_ERR_INVALID;
  }
  const double dt = ctx->prm.dt;
  std::ostringstream sig;
  sig << "accuracy:" << (ctx->batched ? "batched" : "single") << ":" << ctx->prm.dtype << ":" << ctx->prm.d << ":"
      << ctx->prm.k << ":" << ctx->prm.n << ":" << ctx->rep_n.size() << ":" << dt << ":" << eps << ":" << horizon
      << ":" << max_halvings;
  for (int32_t i = 0; i < nps; ++i) sig << ":" << ps[i];
  const std::string key = sig.str();
  std::string found;
  if (table_path) {
    std::ifstream in(table_path);
    std::string line;
    while (std::getline(in, line))
      if (line.compare(0, key.size() + 1, key + " ") == 0) found = line.substr(key.size() + 1);
  }
  int32_t best_p = ctx->prm.p, best_k = 0, met = 0;
  std::ostringstream rep;
  if (!found.empty()) {
    std::istringstream is(found);
    is >> best_p >> best_k >> met;
    rep << "table " << key << " " << found;
  } else {
    RBM_CUDA(cudaStreamSynchronize(ctx->stream));
    // pilot: the first pilot_n particles of a single system, or the replica
    // whose size is closest to pilot_n (with its own replica index)
    rbm_params base = ctx->prm;
    size_t row0 = 0;
    uint32_t npil = static_cast<uint32_t>(std::min<int64_t>(pilot_n, ctx->prm.n));
    if (ctx->batched) {
      size_t off = 0, best_off = 0;
      int64_t best_gap = -1;
      for (size_t r = 0; r < ctx->rep_n.size(); ++r) {
        const int64_t gap = std::llabs(ctx->rep_n[r] - pilot_n);
        if (best_gap < 0 || gap < best_gap) {
          best_gap = gap;
          best_off = off;
          npil = static_cast<uint32_t>(ctx->rep_n[r]);
          base.replica = static_cast<uint32_t>(r);
        }
        off += static_cast<size_t>(ctx->rep_n[r]);
      }
      row0 = best_off;
    }
    base.n = npil;
    const size_t bytes = ctx->row_bytes * npil;
    void *x0 = nullptr, *xref = nullptr, *xrun = nullptr;
    RBM_CUDA(cudaMalloc(&x0, bytes));
    RBM_CUDA(cudaMalloc(&xref, bytes));
    RBM_CUDA(cudaMalloc(&xrun, bytes));
    RBM_CUDA(cudaMemcpy(x0, static_cast<const char*>(ctx->x) + row0 * ctx->row_bytes, bytes,
                        cudaMemcpyDeviceToDevice));
    // the direct reference at dt / 2^(H+1) on the Brownian path every run shares
    const int32_t rref = 1 << (max_halvings + 1);
    const int64_t steps_ref = std::llround(horizon / (dt / rref));
    st = pilot_run(base, std::min<int32_t>(2, static_cast<int32_t>(npil)), dt / rref, 1, steps_ref,
                   RBM_METHOD_DIRECT, x0, xref, bytes);
    std::vector<std::vector<double>> err(nps, std::vector<double>(max_halvings + 1, -1.0));
    for (int32_t i = 0; i < nps && st == RBM_OK; ++i) {
      if (ps[i] > static_cast<int32_t>(npil)) continue;
      for (int32_t k = 0; k <= max_halvings && st == RBM_OK; ++k) {
        const int32_t r = 1 << (max_halvings + 1 - k);
        st = pilot_run(base, ps[i], dt / (1 << k), r, std::llround(horizon / (dt / (1 << k))), RBM_METHOD_RBM, x0,
                       xrun, bytes);
        if (st == RBM_OK) st = rms_gap(ctx, xrun, xref, npil, &err[i][k]);
      }
    }
    cudaFree(x0);
    cudaFree(xref);
    cudaFree(xrun);
    if (st != RBM_OK) return st;
    // full-size step time of each p on a scratch copy of the state
    std::vector<double> ms(nps, -1.0);
    {
      const size_t full = ctx->row_bytes * static_cast<size_t>(ctx->prm.n);
      void* scratch = nullptr;
      RBM_CUDA(cudaMalloc(&scratch, full));
      void* real_x = ctx->x;
      const int64_t m0 = ctx->m;
      const int32_t p0 = ctx->prm.p;
      const int32_t len0 = ctx->tuning.graph_steps;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int32_t i = 0; i < nps && st == RBM_OK; ++i) {
        st = rbm_set_batch_size(ctx, ps[i]);
        if (st != RBM_OK) break;
        ctx->tuning.graph_steps = trial_steps + 1;  // eager steps: no capture inside the timing
        RBM_CUDA(cudaMemcpyAsync(scratch, real_x, full, cudaMemcpyDeviceToDevice, ctx->stream));
        ctx->x = scratch;
        st = rbm_run(ctx, 1, RBM_METHOD_RBM);  // warm-up
        cudaEventRecord(e0, ctx->stream);
        if (st == RBM_OK) st = rbm_run(ctx, trial_steps, RBM_METHOD_RBM);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[i] = t / trial_steps;
        ctx->x = real_x;
        ctx->m = m0;
        ctx->tuning.graph_steps = len0;
        drop_graphs(ctx);
        if (st == RBM_OK) st = forget_prepared(ctx, ctx->stream);  // the trial's lookahead bucketing
        RBM_CUDA(cudaStreamSynchronize(ctx->stream));
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaFree(scratch);
      ctx->x = real_x;
      ctx->m = m0;
      if (st != RBM_OK) return st;
      st = rbm_set_batch_size(ctx, p0);
      if (st != RBM_OK) return st;
    }
    // least time to T with E(T) <= eps; otherwise the smallest error
    double best_time = -1.0, best_err = -1.0;
    for (int32_t i = 0; i < nps; ++i) {
      rep << "p=" << ps[i] << " (" << ms[i] << " ms/step) E:";
      for (int32_t k = 0; k <= max_halvings; ++k) rep << " " << err[i][k];
      rep << "; ";
      for (int32_t k = 0; k <= max_halvings; ++k) {
        if (err[i][k] < 0) continue;
        const double time = std::llround(horizon / (dt / (1 << k))) * ms[i];
        if (err[i][k] <= eps) {
          if (!met || time < best_time) {
            met = 1;
            best_time = time;
            best_p = ps[i];
            best_k = k;
          }
          break;  // finer steps only cost more for this p
        }
        if (!met && (best_err < 0 || err[i][k] < best_err)) {
          best_err = err[i][k];
          best_p = ps[i];
          best_k = k;
        }
      }
    }
    rep << "chosen p=" << best_p << " dt=" << dt / (1 << best_k) << (met ? "" : " (eps not met)")
        << " pilot n=" << npil << " reference dt=" << dt / rref;
    if (table_path) {
      std::ofstream outf(table_path, std::ios::app);
      outf << key << " " << best_p << " " << best_k << " " << met << "\n";
    }
  }
  st = rbm_set_batch_size(ctx, best_p);
  if (st != RBM_OK) return st;
  if (p_out) *p_out = best_p;
  if (dt_out) *dt_out = dt / (1 << best_k);
  if (met_out) *met_out = met;
  if (report && report_len > 0) {
    std::strncpy(report, rep.str().c_str(), static_cast<size_t>(report_len) - 1);
    report[report_len - 1] = 0;
  }
  return RBM_OK;
}

rbm_status rbm_surrogate_config(rbm_ctx* ctx, int32_t train_every, double fallback_tol, int64_t n_queries,
                                int32_t iters_first, int32_t iters_per_checkpoint, int32_t max_rounds, double lr) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (ctx->batched || ctx->prm.d < 2 || ctx->prm.dtype != RBM_F32 || ctx->prm.scheme != RBM_SCHEME_EULER ||
      (ctx->prm.flags & RBM_FLAG_GBM_NOISE))
    return RBM_ERR_UNSUPPORTED;
  if (train_every < 1 || !(fallback_tol > 0) || n_queries < 8 || n_queries > (int64_t(1) << 24) || iters_first < 0 ||
      iters_per_checkpoint < 0 || max_rounds < 1 || !(lr > 0))
    return RBM_ERR_INVALID;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  free_surrogate(ctx);
  {
    cudaError_t e = prepare_surrogate_kernels();
    if (e != cudaSuccess) {
      set_error("prepare_surrogate_kernels", e);
      return RBM_ERR_CUDA;
    }
  }
  SurrogateScratch& s = ctx->ss;
  s.d = ctx->prm.d;
  const int np = surrogate_param_count(s.d);
  s.nq = static_cast<uint32_t>(n_queries);
  s.ntrain = std::max<uint32_t>(1u, s.nq - s.nq / 4);
  s.lr = static_cast<float>(lr);
  s.tol = static_cast<float>(fallback_tol);
  s.partial_blocks = std::max<uint32_t>(32u, 512u);
  RBM_CUDA(cudaMalloc(&s.theta, sizeof(float) * np));
  RBM_CUDA(cudaMalloc(&s.mom1, sizeof(float) * np));
  RBM_CUDA(cudaMalloc(&s.mom2, sizeof(float) * np));
  RBM_CUDA(cudaMalloc(&s.wq, sizeof(float) * np));
  RBM_CUDA(cudaMalloc(&s.w2f, 64 * 64 * 2));
  RBM_CUDA(cudaMalloc(&s.w2b, 64 * 64 * 2));
  RBM_CUDA(cudaMalloc(&s.norm, sizeof(float) * 5));  // mu (d), s, sF
  RBM_CUDA(cudaMalloc(&s.adam_t, sizeof(int)));
  RBM_CUDA(cudaMalloc(&s.flag, sizeof(int)));
  RBM_CUDA(cudaMalloc(&s.err, 2 * sizeof(float)));  // held-out error after training, drift error
  RBM_CUDA(cudaMalloc(&s.counters, 2 * sizeof(unsigned long long)));
  RBM_CUDA(cudaMalloc(&s.partial, sizeof(float) * (np + 1) * s.partial_blocks));
  RBM_CUDA(cudaMalloc(&s.qidx, sizeof(uint32_t) * s.nq));
  RBM_CUDA(cudaMalloc(&s.q, sizeof(float) * ctx->ld * s.nq));
  RBM_CUDA(cudaMalloc(&s.fq, sizeof(float) * ctx->ld * s.nq));
  RBM_CUDA(cudaMalloc(&s.fpred, sizeof(float) * ctx->ld * s.nq));
  const float norm0[5] = {0.0f, 0.0f, s.d == 3 ? 0.0f : 1.0f, 1.0f, 1.0f};
  RBM_CUDA(cudaMemcpy(s.norm, norm0, sizeof(norm0), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemset(s.adam_t, 0, sizeof(int)));
  RBM_CUDA(cudaMemset(s.flag, 0, sizeof(int)));
  RBM_CUDA(cudaMemset(s.err, 0, 2 * sizeof(float)));
  RBM_CUDA(cudaMemset(s.counters, 0, 2 * sizeof(unsigned long long)));
  {
    cudaError_t e = sur_init(s, ctx->status, ctx->prm.seed ^ 0x5EED5EEDull, ctx->stream);
    if (e != cudaSuccess) {
      set_error("surrogate init", e);
      return RBM_ERR_CUDA;
    }
  }
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->sur_on = true;
  ctx->sur_every = train_every;
  ctx->sur_interval = train_every;
  ctx->sur_min_interval = std::max(1, train_every / 16);
  ctx->sur_drift = -1.0f;
  ctx->sur_forced_off = false;
  ctx->sur_forced = 0;
  ctx->sur_iters_first = iters_first;
  ctx->sur_iters = iters_per_checkpoint;
  ctx->sur_max_rounds = max_rounds;
  ctx->sur_adam_total = 0;
  ctx->sur_trained = false;
  ctx->sur_norm_given = false;
  return RBM_OK;
}

rbm_status rbm_surrogate_train(rbm_ctx* ctx, int32_t iters) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (iters < 0) return RBM_ERR_INVALID;
  st = enqueue_checkpoint(ctx, iters, !ctx->sur_trained, ctx->stream);
  if (st == RBM_OK) {
    ctx->sur_trained = true;
    ctx->sur_last = ctx->m;
  }
  return st;
}

rbm_status rbm_surrogate_stats(rbm_ctx* ctx, double* last_rel_err, int64_t* n_surrogate_steps,
                               int64_t* n_fallback_steps, int32_t* active, int64_t* n_adam_steps) {
  if (!ctx) return RBM_ERR_INVALID;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  float err = 0.0f;
  unsigned long long cnt[2] = {0, 0};
  int flag = 0;
  RBM_CUDA(cudaMemcpy(&err, ctx->ss.err, sizeof(float), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(cnt, ctx->ss.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(&flag, ctx->ss.flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (last_rel_err) *last_rel_err = err;
  if (n_surrogate_steps) *n_surrogate_steps = static_cast<int64_t>(cnt[0]);
  if (n_fallback_steps) *n_fallback_steps = static_cast<int64_t>(cnt[1]);
  if (active) *active = flag;
  if (n_adam_steps) *n_adam_steps = ctx->sur_adam_total;
  return RBM_OK;
}

rbm_status rbm_surrogate_drift(const rbm_ctx* ctx, double* drift_err, int32_t* interval, int32_t* forced_off,
                               int64_t* n_forced_intervals) {
  if (!ctx) return RBM_ERR_INVALID;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (drift_err) *drift_err = ctx->sur_drift;
  if (interval) *interval = ctx->sur_interval;
  if (forced_off) *forced_off = ctx->sur_forced_off ? 1 : 0;
  if (n_forced_intervals) *n_forced_intervals = ctx->sur_forced;
  return RBM_OK;
}

rbm_status rbm_surrogate_params(rbm_ctx* ctx, float* theta_host, float* norm_host) {
  if (!ctx) return RBM_ERR_INVALID;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (theta_host)
    RBM_CUDA(cudaMemcpy(theta_host, ctx->ss.theta, sizeof(float) * surrogate_param_count(ctx->ss.d),
                        cudaMemcpyDeviceToHost));
  if (norm_host)
    RBM_CUDA(cudaMemcpy(norm_host, ctx->ss.norm, sizeof(float) * (ctx->ss.d + 2), cudaMemcpyDeviceToHost));
  return RBM_OK;
}

rbm_status rbm_surrogate_set_params(rbm_ctx* ctx, const float* theta_host, const float* norm_host) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  const int np = surrogate_param_count(ctx->ss.d);
  if (theta_host) {
    RBM_CUDA(cudaMemcpy(ctx->ss.theta, theta_host, sizeof(float) * np, cudaMemcpyHostToDevice));
    RBM_CUDA(cudaMemset(ctx->ss.mom1, 0, sizeof(float) * np));
    RBM_CUDA(cudaMemset(ctx->ss.mom2, 0, sizeof(float) * np));
    RBM_CUDA(cudaMemset(ctx->ss.adam_t, 0, sizeof(int)));
  }
  if (norm_host) {
    RBM_CUDA(cudaMemcpy(ctx->ss.norm, norm_host, sizeof(float) * (ctx->ss.d + 2), cudaMemcpyHostToDevice));
    ctx->sur_norm_given = true;
  }
  cudaError_t e = sur_publish(ctx->ss, ctx->status, ctx->stream);
  if (e != cudaSuccess) {
    set_error("surrogate publish", e);
    return RBM_ERR_CUDA;
  }
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  return RBM_OK;
}

rbm_status rbm_surrogate_forces(rbm_ctx* ctx, const void* q_dev, int64_t nq, void* f_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (nq < 0 || nq > (int64_t(1) << 31) || (nq > 0 && (!q_dev || !f_dev))) return RBM_ERR_INVALID;
  if (nq == 0) return RBM_OK;
  cudaError_t e = sur_forces(ctx->ss, ctx->status, static_cast<const float*>(q_dev), static_cast<uint32_t>(nq),
                             static_cast<float*>(f_dev), ctx->cfg, ctx->stream);
  if (e != cudaSuccess) {
    set_error("surrogate forces", e);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}

rbm_status rbm_surrogate_gradient(rbm_ctx* ctx, const void* x_dev, const void* f_target_dev, int64_t nb,
                                  float* grad_host, double* loss_host) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (nb < 1 || nb > static_cast<int64_t>(ctx->ss.partial_blocks) * 128 || !x_dev || !f_target_dev || !grad_host)
    return RBM_ERR_INVALID;
  cudaError_t e = sur_gradient(ctx->ss, ctx->status, static_cast<const float*>(x_dev),
                               static_cast<const float*>(f_target_dev), static_cast<uint32_t>(nb), ctx->stream);
  if (e != cudaSuccess) {
    set_error("surrogate gradient", e);
    return RBM_ERR_CUDA;
  }
  const int np = surrogate_param_count(ctx->ss.d);
  const uint32_t nblocks = static_cast<uint32_t>((nb + 127) / 128);
  std::vector<float> part(static_cast<size_t>(nblocks) * (np + 1));
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  RBM_CUDA(cudaMemcpy(part.data(), ctx->ss.partial, sizeof(float) * part.size(), cudaMemcpyDeviceToHost));
  double loss = 0.0;
  for (int i = 0; i <= np; ++i) {
    double g = 0.0;
    for (uint32_t b = 0; b < nblocks; ++b) g += part[static_cast<size_t>(b) * (np + 1) + i];
    if (i < np) grad_host[i] = static_cast<float>(g);
    else loss = g;
  }
  if (loss_host) *loss_host = loss;
  return rbm_sync(ctx);
}

rbm_status rbm_verlet_set_velocity(rbm_ctx* ctx, const void* v_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!v_dev) return RBM_ERR_INVALID;
  if (ctx->prm.scheme != RBM_SCHEME_VERLET) return RBM_ERR_STATE;
  const size_t bytes = ctx->row_bytes * static_cast<size_t>(ctx->prm.n);
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (!ctx->xprev) RBM_CUDA(cudaMalloc(&ctx->xprev, bytes));
  RBM_CUDA(cudaMemcpyAsync(ctx->xprev, v_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->verlet_m0 = ctx->m;
  drop_graphs(ctx);  // captured steps hold the index of the Taylor start
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  return RBM_OK;
}

rbm_status rbm_verlet_get_previous(rbm_ctx* ctx, void* prev_dev, int32_t* taylor_pending) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!prev_dev || !taylor_pending) return RBM_ERR_INVALID;
  if (ctx->prm.scheme != RBM_SCHEME_VERLET || !ctx->xprev) return RBM_ERR_STATE;
  const size_t bytes = ctx->row_bytes * static_cast<size_t>(ctx->prm.n);
  RBM_CUDA(cudaMemcpyAsync(prev_dev, ctx->xprev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  *taylor_pending = (ctx->verlet_m0 == ctx->m) ? 1 : 0;
  return RBM_OK;
}

rbm_status rbm_verlet_set_previous(rbm_ctx* ctx, const void* prev_dev, int32_t taylor_pending) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!prev_dev || (taylor_pending != 0 && taylor_pending != 1)) return RBM_ERR_INVALID;
  if (ctx->prm.scheme != RBM_SCHEME_VERLET) return RBM_ERR_STATE;
  st = rbm_verlet_set_velocity(ctx, prev_dev);            // copies the buffer, drops graphs
  if (st != RBM_OK) return st;
  if (!taylor_pending) ctx->verlet_m0 = ctx->m - 1;       // the Taylor start lies behind
  return RBM_OK;
}

// Surrogate state: every value a later checkpoint or step reads, so that a
// run saved after step m and loaded into a context configured the same way
// continues bit for bit.
namespace {
constexpr uint32_t kSurStateMagic = 0x52425347u;  // "RBSG"
struct SurStateHeader {
  uint32_t magic, version, np, pad;
  int32_t adam_t, flag, trained, norm_given;
  float err, drift_err;
  uint64_t counters[2];
  int64_t last, adam_total;
  float norm[6];
  int32_t interval, forced_off;
  int64_t forced;
};
size_t sur_state_bytes(int d) {
  return sizeof(SurStateHeader) + 3 * sizeof(float) * static_cast<size_t>(surrogate_param_count(d));
}
}  // namespace

rbm_status rbm_surrogate_state_size(const rbm_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return RBM_ERR_INVALID;
  *bytes = static_cast<int64_t>(sur_state_bytes(ctx->sur_on ? ctx->ss.d : ctx->prm.d));
  return RBM_OK;
}

rbm_status rbm_surrogate_save(rbm_ctx* ctx, void* host_buf, int64_t bytes) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (!host_buf || bytes < static_cast<int64_t>(sur_state_bytes(ctx->ss.d))) return RBM_ERR_INVALID;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  const size_t np = static_cast<size_t>(surrogate_param_count(ctx->ss.d));
  SurStateHeader h{};
  h.magic = kSurStateMagic;
  h.version = 3;
  h.np = static_cast<uint32_t>(np);
  RBM_CUDA(cudaMemcpy(&h.adam_t, ctx->ss.adam_t, sizeof(int), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(&h.flag, ctx->ss.flag, sizeof(int), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(&h.err, ctx->ss.err, sizeof(float), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(&h.drift_err, ctx->ss.err + 1, sizeof(float), cudaMemcpyDeviceToHost));
  h.interval = ctx->sur_interval;
  h.forced_off = ctx->sur_forced_off ? 1 : 0;
  h.forced = ctx->sur_forced;
  RBM_CUDA(cudaMemcpy(h.counters, ctx->ss.counters, sizeof(h.counters), cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(h.norm, ctx->ss.norm, sizeof(float) * 5, cudaMemcpyDeviceToHost));
  h.trained = ctx->sur_trained ? 1 : 0;
  h.norm_given = ctx->sur_norm_given ? 1 : 0;
  h.last = ctx->sur_last;
  h.adam_total = ctx->sur_adam_total;
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  std::memcpy(out, &h, sizeof(h));
  float* f = reinterpret_cast<float*>(out + sizeof(h));
  RBM_CUDA(cudaMemcpy(f, ctx->ss.theta, sizeof(float) * np, cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(f + np, ctx->ss.mom1, sizeof(float) * np, cudaMemcpyDeviceToHost));
  RBM_CUDA(cudaMemcpy(f + 2 * np, ctx->ss.mom2, sizeof(float) * np, cudaMemcpyDeviceToHost));
  return RBM_OK;
}

rbm_status rbm_surrogate_load(rbm_ctx* ctx, const void* host_buf, int64_t bytes) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!ctx->sur_on) return RBM_ERR_STATE;
  if (!host_buf || bytes < static_cast<int64_t>(sur_state_bytes(ctx->ss.d))) return RBM_ERR_INVALID;
  SurStateHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  const size_t np = static_cast<size_t>(surrogate_param_count(ctx->ss.d));
  if (h.magic != kSurStateMagic || h.version != 3 || h.np != np || h.interval < 1) return RBM_ERR_INVALID;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  const float* f = reinterpret_cast<const float*>(static_cast<const unsigned char*>(host_buf) + sizeof(h));
  RBM_CUDA(cudaMemcpy(ctx->ss.theta, f, sizeof(float) * np, cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.mom1, f + np, sizeof(float) * np, cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.mom2, f + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.adam_t, &h.adam_t, sizeof(int), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.flag, &h.flag, sizeof(int), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.err, &h.err, sizeof(float), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.err + 1, &h.drift_err, sizeof(float), cudaMemcpyHostToDevice));
  ctx->sur_interval = h.interval;
  ctx->sur_forced_off = h.forced_off != 0;
  ctx->sur_forced = h.forced;
  RBM_CUDA(cudaMemcpy(ctx->ss.counters, h.counters, sizeof(h.counters), cudaMemcpyHostToDevice));
  RBM_CUDA(cudaMemcpy(ctx->ss.norm, h.norm, sizeof(float) * 5, cudaMemcpyHostToDevice));
  ctx->sur_trained = h.trained != 0;
  ctx->sur_norm_given = h.norm_given != 0;
  ctx->sur_last = h.last;
  ctx->sur_adam_total = h.adam_total;
  cudaError_t e = sur_publish(ctx->ss, ctx->status, ctx->stream);  // the bf16 views of theta
  if (e != cudaSuccess) {
    set_error("surrogate publish", e);
    return RBM_ERR_CUDA;
  }
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  return RBM_OK;
}

rbm_status rbm_rbmr_sets(rbm_ctx* ctx, int64_t m, uint32_t* sets_dev) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!sets_dev || m < 0) return RBM_ERR_INVALID;
  st = ensure_rbmr(ctx);
  if (st != RBM_OK) return st;
  cudaError_t e = launch_rbmr_sets(sets_dev, ctx->rs.K, static_cast<uint32_t>(ctx->prm.n), ctx->prm.p,
                                   static_cast<uint32_t>(ctx->prm.replica), ctx->prm.seed, m, ctx->stream);
  if (e != cudaSuccess) {
    set_error("k_rbmr_sets", e);
    return RBM_ERR_CUDA;
  }
  return RBM_OK;
}

rbm_status rbm_rbmr_info(rbm_ctx* ctx, int64_t* iterations_per_step, int32_t* rounds_last) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  st = ensure_rbmr(ctx);
  if (st != RBM_OK) return st;
  RBM_CUDA(cudaStreamSynchronize(ctx->stream));
  uint32_t rounds = 0;
  RBM_CUDA(cudaMemcpy(&rounds, ctx->rs.rounds, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (iterations_per_step) *iterations_per_step = ctx->rs.K;
  if (rounds_last) *rounds_last = static_cast<int32_t>(rounds);
  return RBM_OK;
}

rbm_status rbm_latency_floor(rbm_ctx* ctx, float* us) {
  rbm_status st = usable(ctx);
  if (st != RBM_OK) return st;
  if (!us) return RBM_ERR_INVALID;
  if (!ctx->use_coop) return RBM_ERR_STATE;
  const size_t smem = coop_smem_bytes(ctx->prm.dtype, ctx->prm.d, ctx->cs.nbuckets);
  const uint64_t wait_ns = 1000ull * 1000000ull;
  cudaEvent_t e0, e1;
  RBM_CUDA(cudaEventCreate(&e0));
  RBM_CUDA(cudaEventCreate(&e1));
  cudaError_t e = launch_coop_floor(ctx->cs, smem, wait_ns, ctx->status, ctx->stream);  // warm-up
  constexpr int kReps = 20;
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
  for (int r = 0; r < kReps && e == cudaSuccess; ++r) e = launch_coop_floor(ctx->cs, smem, wait_ns, ctx->status, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_error("latency floor", e);
    return RBM_ERR_CUDA;
  }
  *us = 1000.0f * ms / kReps;
  return rbm_sync(ctx);
}

rbm_status rbm_launches_per_step(const rbm_ctx* ctx, int32_t method, int32_t* launches) {
  if (!ctx || !launches) return RBM_ERR_INVALID;
  // RBM-1 inside a run: the previous step bucketed this one's ids (lookahead)
  if (method == RBM_METHOD_RBM && ctx->use_rec)
    *launches = rec_launches_per_step(ctx->rec);  // split, scan, step, fix-up (a run adds its first step's scatter)
  else if (method == RBM_METHOD_RBM)
    *launches = (ctx->use_coop || ctx->batched || ctx->use_small) ? 1 : rbm_tail_launches(ctx->ps, ctx->prm.p);
  else if (method == RBM_METHOD_DIRECT) *launches = 2;  // upper bound: sum (+ chunk reduction)
  else if (method == RBM_METHOD_SURROGATE)  // network step + the flag-gated RBM step that buckets its own ids
    *launches = 1 + (ctx->use_small ? 1 : ctx->use_coop ? 2 : 1 + rbm_tail_launches(ctx->ps, ctx->prm.p));
  else if (method == RBM_METHOD_RBMR) *launches = 1;
  else return RBM_ERR_INVALID;
  return RBM_OK;
}

}  // extern "C"
