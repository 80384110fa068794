// Internal declarations shared by the library's translation units: scratch
// layout of a context and the host-side launchers of each kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rbm.h"

namespace rbm {

// Permutation scratch (one particle system or one replica set).
struct PermScratch {
  // Each of cnt .. done holds two buffers when double_buffer is set (step m
  // uses buffer m mod 2; buffer 1 follows buffer 0 in each array).
  uint32_t* cnt = nullptr;      // [nbuckets] members per bucket (zero between steps)
  uint32_t* start = nullptr;    // [nbuckets] first sorted position of each bucket
  uint32_t* slots = nullptr;    // [nbuckets * slot_cap] member ids, bucket-major
  uint32_t* ovf_cnt = nullptr;  // [1] members that did not fit their bucket's slots
  uint32_t* ovf = nullptr;      // [n] those members' ids
  uint32_t* done = nullptr;     // [1] finished-block ticket (last block runs the fix-up)
  bool double_buffer = false;
  uint32_t* perm = nullptr;     // [n] the random permutation of this step
  int bucket_bits = 0;
  uint32_t nbuckets = 1;
  uint32_t slot_cap = 0;
  uint32_t sort_cap = 0;
  bool separate_scan = false;   // large bucket counts: scan and fix-up kernels of their own
  const int* skip = nullptr;    // when set and non-zero the kernels do nothing (surrogate mode)
};

// Cooperative single-kernel step scratch.
struct CoopScratch {
  uint32_t* hist = nullptr;     // [3 nbuckets] bucket totals, buffer m mod 3 for step m (zero initially)
  uint32_t* slots = nullptr;    // [2 nbuckets slot_cap] ids grouped by bucket, buffer m mod 2
  uint32_t slot_cap = 0;        // slots per bucket, at most coop_slot_capacity()
  uint32_t* tmp = nullptr;      // [n] ids grouped by bucket, compact (bucket overflow only)
  uint32_t* perm = nullptr;     // [n] (shared with PermScratch::perm)
  unsigned long long* bar = nullptr;  // [1] grid barrier arrival counter
  unsigned long long* arrive = nullptr;  // [1] blocks that have read the step counter (zero between launches)
  uint32_t grid = 0;            // blocks (one per SM)
  uint32_t nbuckets = 0;        // k * grid
};

// Record-path scratch (rec_step.cu): the positions of a large system moving
// through each step as records (row with the id in its pad lane, 32 key bits)
// in two levels of buckets.
struct RecScratch {
  int top_bits = 0, sub_bits = 0;
  uint32_t ntop = 1, nsub = 1;      // buckets per level
  uint32_t top_cap = 0, sub_cap = 0;  // records per top bucket / per sub-bucket
  uint32_t id_mul = 0;              // last step's id-range bucket: umulhi(id, id_mul) < ntop
  float4* top_rows = nullptr;       // [ntop * top_cap]
  uint32_t* top_keys = nullptr;
  float4* sub_rows = nullptr;       // [ntop * nsub * sub_cap]
  uint32_t* sub_keys = nullptr;
  uint32_t* top_fill = nullptr;     // [2 ntop] fill counters by step parity
  uint32_t* sub_fill = nullptr;     // [2 ntop nsub]
  uint32_t* sub_start = nullptr;    // [ntop nsub + 1] sorted start of each sub-bucket
  float4* side = nullptr;           // [ntop nsub * 32] members of batches crossing sub-bucket ends
};

// Batched-replica scratch.
struct BatchedScratch {
  uint32_t* order = nullptr;        // replica ids, block-major
  uint32_t* block_begin = nullptr;  // [grid + 1]
  uint64_t* offs = nullptr;         // [nrep + 1] first row of each replica
  uint32_t* tmp = nullptr;          // [rows]
  uint32_t* perm = nullptr;         // [rows]
  uint16_t* bkt = nullptr;          // [rows] bucket of each particle, from the histogram pass
  uint32_t grid = 0;
  int threads = 512;
  int bucket_target = 1024;
  uint32_t rep_base = 0;            // added to the replica index in the Philox counters
};

// RBM-r scratch (rbmr.cu); all device pointers.
struct RbmrScratch {
  uint32_t* set = nullptr;        // [K p]
  uint32_t* cnt = nullptr;        // [N] zero between steps
  uint32_t* start = nullptr;      // [N + 1]
  uint32_t* occ = nullptr;        // [K p]
  uint32_t* next = nullptr;       // [N]
  uint8_t* flag = nullptr;        // [K]
  uint32_t* btot = nullptr;       // [grid]
  uint32_t* remaining = nullptr;  // [1]
  uint32_t* rounds = nullptr;     // [1]
  unsigned long long* bar = nullptr;  // [1] grid barrier counter
  uint32_t K = 0;                 // iterations per step
  uint32_t grid = 0;              // blocks (one per SM)
};

// Surrogate-network state (surrogate.cu); all device pointers.
struct SurrogateScratch {
  float* theta = nullptr;
  float* mom1 = nullptr;
  float* mom2 = nullptr;
  float* wq = nullptr;
  uint16_t* w2f = nullptr;
  uint16_t* w2b = nullptr;
  float* norm = nullptr;
  int* adam_t = nullptr;
  int* flag = nullptr;
  float* err = nullptr;              // [0] held-out error after training, [1] drift error
  unsigned long long* counters = nullptr;
  float* partial = nullptr;
  uint32_t partial_blocks = 0;
  uint32_t* qidx = nullptr;
  float* q = nullptr;
  float* fq = nullptr;
  float* fpred = nullptr;
  uint32_t nq = 0, ntrain = 0;
  float lr = 1e-3f, tol = 1e-2f;
  int d = 2;                        // network dimension (2 or 3); query rows of Ld<d> floats
};

struct LaunchCfg {
  int block = 256;
  int direct_block = 256;
  int num_sms = 152;
  // Profiling: when `events` is set, every launcher records events[(*nevents)++]
  // on its stream after each kernel and appends the kernel's name to `names`.
  cudaEvent_t* events = nullptr;
  int* nevents = nullptr;
  int max_events = 0;
  const char** names = nullptr;
};

// Record a profiling event after a launch (no-op unless profiling).
inline void mark_launch(const LaunchCfg& cfg, cudaStream_t st, const char* name) {
  if (!cfg.events || !cfg.nevents || *cfg.nevents >= cfg.max_events) return;
  if (cfg.names) cfg.names[*cfg.nevents] = name;
  cudaEventRecord(cfg.events[*cfg.nevents], st);
  ++*cfg.nevents;
}

// RBM step pieces (perm_step.cu).  `mode`: 0 = write the permutation only,
// 1 = step, 2 = interaction forces only.
void launch_bucket_scatter(const PermScratch& ps, uint32_t n, uint2 seed, uint32_t replica, const int64_t* m_ptr,
                           int64_t m_off, const LaunchCfg& cfg, cudaStream_t st);
template <typename T>
void launch_rbm_tail(const PermScratch& ps, int d, int mode, const void* params, bool lookahead, const LaunchCfg& cfg,
                     cudaStream_t st);
void set_last_error_text(const char* text);  // text returned by rbm_last_error()
cudaError_t prepare_rbm_kernels();  // per-device kernel attributes, called by rbm_init
void launch_set_i64(int64_t* dst, int64_t value, cudaStream_t st);
void launch_add_i64(int64_t* dst, int64_t value, cudaStream_t st);
int rbm_tail_launches(const PermScratch& ps, int p);
// Largest bucket the shared-memory sort of the multi-kernel path takes.
uint32_t max_sort_cap();

// Record path (rec_step.cu): FP32, d = 3, p <= 32, any scheme but Verlet.
bool rec_eligible(int dtype, int d, int p, int scheme);
void rec_geometry(uint32_t n, int tuned_bits, RecScratch* rs);
cudaError_t rec_alloc(uint32_t n, RecScratch* rs);
void rec_free(RecScratch* rs);
cudaError_t prepare_rec_kernels();
// `count` RBM-1 steps from the step of `params` (StepParams<float>).
cudaError_t launch_rec_run(const RecScratch& rs, const void* params, int64_t count, const LaunchCfg& cfg,
                           cudaStream_t st);
// Kernel launches of one step of a run (after its first step's scatter).
int rec_launches_per_step(const RecScratch& rs);
// One record-path step of positions held in host memory (x_host, N rows of
// 16 bytes; a.x the device copy): the rows are copied in and scattered, and
// placed and copied out, in kHostChunks chunks, the copies on copy_st and
// the kernels on st, each chunk's kernels overlapping the next chunk's copy.
// ev: 2 kHostChunks + 2 events.  On return st is ordered after the copies out.
constexpr int kHostChunks = 8;
cudaError_t launch_rec_host_step(const RecScratch& rs, const void* params, void* x_host, const LaunchCfg& cfg,
                                 cudaStream_t st, cudaStream_t copy_st, cudaEvent_t* ev);

// Cooperative step (coop_step.cu): mode as for launch_rbm_tail.
cudaError_t prepare_coop_kernels(int* blocks_per_sm);
uint32_t coop_max_buckets();
uint32_t coop_slot_capacity();
size_t coop_smem_bytes(int dtype, int d, uint32_t nbuckets);
cudaError_t launch_coop_floor(const CoopScratch& cs, size_t smem_bytes, uint64_t wait_ns, int32_t* status,
                              cudaStream_t st);
uint32_t coop_bucket_target();
template <typename T>
// prologue: only bucket the ids of the step; lookahead: after the step,
// bucket the ids of the next one.
// bump_step: the step launch advances the device step counter a.m_ptr once
// every block has read it (graph replay).
cudaError_t launch_coop(const CoopScratch& cs, int d, int mode, const void* params, uint64_t wait_ns, int skip_arrival,
                        bool prologue, bool lookahead, bool bump_step, const LaunchCfg& cfg, cudaStream_t st);

// Batched replicas (batched.cu): mode as for launch_rbm_tail.
int batched_max_buckets();
cudaError_t prepare_batched_kernels(int dtype, int d, int threads, int* blocks_per_sm);
template <typename T>
cudaError_t launch_batched(const BatchedScratch& bs, int d, int mode, const void* params, const LaunchCfg& cfg,
                           cudaStream_t st);

// Surrogate network (surrogate.cu).
int surrogate_param_count(int d);
cudaError_t prepare_surrogate_kernels();
cudaError_t sur_init(const SurrogateScratch& ss, int32_t* status, uint64_t seed, cudaStream_t st);
cudaError_t sur_publish(const SurrogateScratch& ss, int32_t* status, cudaStream_t st);
cudaError_t sur_sample(const SurrogateScratch& ss, const void* params, cudaStream_t st);
cudaError_t sur_norm(const SurrogateScratch& ss, int32_t* status, cudaStream_t st);
cudaError_t sur_train(const SurrogateScratch& ss, int32_t* status, const float* xs, const float* ts, uint32_t ntrain,
                      int iters, uint32_t batch, uint32_t begin0, float lr_scale, const LaunchCfg& cfg,
                      cudaStream_t st);
cudaError_t sur_gradient(const SurrogateScratch& ss, int32_t* status, const float* xs, const float* ts, uint32_t nb,
                         cudaStream_t st);
cudaError_t sur_forces(const SurrogateScratch& ss, int32_t* status, const float* q, uint32_t nq, float* fout,
                       const LaunchCfg& cfg, cudaStream_t st);
cudaError_t sur_check(const SurrogateScratch& ss, int32_t* status, cudaStream_t st);
cudaError_t sur_drift(const SurrogateScratch& ss, int32_t* status, cudaStream_t st);
cudaError_t sur_step(const SurrogateScratch& ss, const void* params, const LaunchCfg& cfg, cudaStream_t st);

// Direct O(N^2) pieces (direct.cu).  `mode`: 0 = step (into xout), 1 =
// forces at the particles (into fout), 2 = forces at query points.
template <typename T>
void launch_direct(int d, int mode, const void* params, const T* q, uint32_t nq, void* partial, size_t partial_rows,
                   const LaunchCfg& cfg, cudaStream_t st);

// RBM-r (rbmr.cu).
int rbmr_threads();
cudaError_t rbmr_blocks_per_sm(int dtype, int d, int* nb);
template <typename T>
cudaError_t launch_rbmr(const RbmrScratch& rs, int d, const void* params, uint64_t wait_ns, const LaunchCfg& cfg,
                        cudaStream_t st);
cudaError_t launch_rbmr_sets(uint32_t* set, uint32_t K, uint32_t n, int p, uint32_t replica, uint64_t seed,
                             int64_t m, cudaStream_t st);

}  // namespace rbm
