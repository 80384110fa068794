// Direct O(N^2) forward-Euler step (the reference method of Sec. 4.1 of
// arXiv:1812.10575, eq. "interactingps"):
//   F^K_i = 1/(N-1) sum_{j != i} K(X^i - X^j),
//   X^i  <- X^i + dt (F^K_i - grad V(X^i)) + sigma sqrt(dt) z_i,
// with z_i the same Brownian increment the RBM step of step m draws.
//
// Layout of the work: each thread owns R targets (register blocking), a block
// of 256 threads owns 256 R consecutive targets, and the source range is
// split into S equal chunks across blockIdx.y so that small systems still
// fill every SM.  Sources stream through shared memory in tiles of 256 rows;
// every warp reads the same source row at once (a broadcast) and applies it
// to its R targets, so the inner loop is bound by the FP32 (or FP64) pipe:
// per pair D subtractions, D multiply-adds for |x|^2, the kernel's scale
// s(|x|^2) and D multiply-adds into the accumulator.  In FP32 the targets are
// taken two at a time on packed two-lane instructions (the scale per lane),
// which halves the issue slots of everything but the scale.  With S > 1 every chunk
// writes its partial sums and k_direct_finish adds them in chunk order (the
// result does not depend on scheduling).
//
// K(0) := 0.  The source tiles that overlap the block's own targets (where
// j = i occurs) run the pair loop with the test; all other tiles run it
// unchecked.  A target whose sum still comes out non-finite (a distinct
// source at exactly its position, where K = 1/x or x/|x|^3 is infinite) is
// summed again over its source chunk with the test, reading the sources from
// global memory.
#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {

namespace {

constexpr int kDirectStep = 0;
constexpr int kDirectForces = 1;
constexpr int kDirectQuery = 2;
constexpr int kDirectThreads = 256;

template <typename T, int D>
struct SrcRow;  // one source row in shared memory
template <> struct SrcRow<float, 1> { float x; };
template <> struct SrcRow<float, 2> { float2 x; };
template <> struct SrcRow<float, 3> { float4 x; };
template <> struct SrcRow<double, 1> { double x; };
template <> struct SrcRow<double, 2> { double2 x; };
template <> struct SrcRow<double, 3> { double x[4]; };

template <typename T, int D>
__device__ __forceinline__ void src_store(SrcRow<T, D>& s, const Row<T, D>& r) {
  if constexpr (D == 1) {
    s.x = r.x[0];
  } else if constexpr (D == 2 && sizeof(T) == 4) {
    s.x = make_float2(r.x[0], r.x[1]);
  } else if constexpr (D == 2) {
    s.x = make_double2(r.x[0], r.x[1]);
  } else if constexpr (sizeof(T) == 4) {
    s.x = make_float4(r.x[0], r.x[1], r.x[2], 0.0f);
  } else {
    s.x[0] = r.x[0]; s.x[1] = r.x[1]; s.x[2] = r.x[2]; s.x[3] = 0.0;
  }
}

template <typename T, int D>
__device__ __forceinline__ void src_load(const SrcRow<T, D>& s, T (&x)[D]) {
  if constexpr (D == 1) {
    x[0] = s.x;
  } else if constexpr (D == 2) {
    x[0] = s.x.x; x[1] = s.x.y;
  } else if constexpr (sizeof(T) == 4) {
    const float4 v = s.x;
    x[0] = v.x; x[1] = v.y; x[2] = v.z;
  } else {
    x[0] = s.x[0]; x[1] = s.x[1]; x[2] = s.x[2];
  }
}

// acc += K(xi - xj); CHECKED applies K(0) := 0 explicitly.
template <typename T, int D, int KF, bool CHECKED>
__device__ __forceinline__ void add_pair(const T (&xi)[D], const T (&xj)[D], T kparam, T radius_sq, T (&acc)[D]) {
  T x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = fsub_rn(xi[k], xj[k]);
  const T r2 = sqnorm_rn<T, D>(x);
  T s = kernel_scale<KF>(r2, kparam, radius_sq);
  if (CHECKED) s = (r2 == T(0)) ? T(0) : s;
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = fma(s, x[k], acc[k]);
}

// Packed two-lane FP32 arithmetic (sm_100 family): one instruction applies
// the same round-to-nearest operation to two independent lanes, so a pair of
// targets against one source costs half the FP32 issue slots of the scalar
// loop and gives the same bits.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// acc_a += K(xa - xj), acc_b += K(xb - xj) (no coincidence test) with the
// arithmetic of add_pair<float, D, KF, false> on two packed lanes: the same
// differences, squared norm (x0 x0, then fused x1 x1 and x2 x2) and fused
// accumulation, the kernel's scale per lane.
template <int D, int KF>
__device__ __forceinline__ void add_pair2(const unsigned long long (&xab)[D], const float (&xj)[D], float kparam,
                                          float radius_sq, unsigned long long (&acc)[D]) {
  unsigned long long x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = f2_sub(xab[k], f2_pack(xj[k], xj[k]));
  unsigned long long r2 = f2_mul(x[0], x[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) r2 = f2_fma(x[k], x[k], r2);
  float r2a, r2b;
  f2_unpack(r2, r2a, r2b);
  const unsigned long long sc =
      f2_pack(kernel_scale<KF>(r2a, kparam, radius_sq), kernel_scale<KF>(r2b, kparam, radius_sq));
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = f2_fma(sc, x[k], acc[k]);
}

struct DirectArgs {
  const void* q;   // query points (mode kDirectQuery)
  uint32_t nq;     // targets
  void* partial;   // [S][ntargets] rows of partial sums (S > 1)
  uint32_t split;  // S
  uint32_t chunk;  // sources per chunk (multiple of the tile)
};

// Finish one target: fk = acc / (N - 1), then update / write.
template <typename T, int D, int MODE>
__device__ __forceinline__ void finish_target(const StepParams<T>& a, uint32_t i, const Row<T, D>& ri,
                                              const T (&acc)[D]) {
  const T inv = T(1) / static_cast<T>(a.n - 1);
  T fk[D];
#pragma unroll
  for (int k = 0; k < D; ++k) fk[k] = acc[k] * inv;
  if (MODE != kDirectStep) {
    Row<T, D> f;
#pragma unroll
    for (int k = 0; k < D; ++k) f.x[k] = fk[k];
    f.pad = T(0);
    store_row<T, D>(a.fout, i, f);
    return;
  }
  const uint32_t m32 = step_index(a);
  T y[D];
  scheme_update<T, D>(a, i, m32, ri.x, fk, y);
  Row<T, D> out = ri;
#pragma unroll
  for (int k = 0; k < D; ++k) out.x[k] = y[k];
  store_row<T, D>(a.xout, i, out);
}

template <typename T, int D, int KF, int MODE, int R>
__global__ void __launch_bounds__(kDirectThreads) k_direct(StepParams<T> a, DirectArgs da) {
  __shared__ SrcRow<T, D> tile[kDirectThreads];
  const T* targets = (MODE == kDirectQuery) ? static_cast<const T*>(da.q) : a.x;
  const uint32_t ntarget = (MODE == kDirectQuery) ? da.nq : a.n;
  const uint32_t base = blockIdx.x * kDirectThreads * R + threadIdx.x;
  Row<T, D> ri[R];
  T acc[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = base + r * kDirectThreads;
    if (i < ntarget) {
      ri[r] = load_row<T, D>(targets, i);
    } else {
      // far-away dummy target: every pair term stays finite
#pragma unroll
      for (int k = 0; k < D; ++k) ri[r].x[k] = T(1e18);
      ri[r].pad = T(0);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) acc[r][k] = T(0);
  }
  const uint32_t j_begin = blockIdx.y * da.chunk;
  const uint32_t j_end = min(a.n, j_begin + da.chunk);
  // sources [j0, j0 + cnt) overlap this block's targets [t_lo, t_hi) only on R tiles
  const uint32_t t_lo = blockIdx.x * kDirectThreads * R, t_hi = t_lo + kDirectThreads * R;

  for (uint32_t j0 = j_begin; j0 < j_end; j0 += kDirectThreads) {
    const uint32_t cnt = min(static_cast<uint32_t>(kDirectThreads), j_end - j0);
    __syncthreads();
    if (threadIdx.x < cnt) src_store<T, D>(tile[threadIdx.x], load_row<T, D>(a.x, j0 + threadIdx.x));
    __syncthreads();
    const bool diagonal = (MODE != kDirectQuery) && j0 < t_hi && j0 + cnt > t_lo;  // block-uniform
    if (diagonal) {
      for (uint32_t jj = 0; jj < cnt; ++jj) {
        T xj[D];
        src_load<T, D>(tile[jj], xj);
#pragma unroll
        for (int r = 0; r < R; ++r) add_pair<T, D, KF, true>(ri[r].x, xj, a.kparam, a.radius_sq, acc[r]);
      }
    } else if constexpr (sizeof(T) == 4 && R % 2 == 0) {
      // targets (0, 1), (2, 3), ... on packed lanes
      unsigned long long xab[R / 2][D], acc2[R / 2][D];
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          xab[h][k] = f2_pack(ri[2 * h].x[k], ri[2 * h + 1].x[k]);
          acc2[h][k] = f2_pack(acc[2 * h][k], acc[2 * h + 1][k]);
        }
      }
#pragma unroll 4
      for (uint32_t jj = 0; jj < cnt; ++jj) {
        T xj[D];
        src_load<T, D>(tile[jj], xj);
#pragma unroll
        for (int h = 0; h < R / 2; ++h) add_pair2<D, KF>(xab[h], xj, a.kparam, a.radius_sq, acc2[h]);
      }
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
#pragma unroll
        for (int k = 0; k < D; ++k) f2_unpack(acc2[h][k], acc[2 * h][k], acc[2 * h + 1][k]);
      }
    } else {
#pragma unroll 4
      for (uint32_t jj = 0; jj < cnt; ++jj) {
        T xj[D];
        src_load<T, D>(tile[jj], xj);
#pragma unroll
        for (int r = 0; r < R; ++r) add_pair<T, D, KF, false>(ri[r].x, xj, a.kparam, a.radius_sq, acc[r]);
      }
    }
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = base + r * kDirectThreads;
    if (i >= ntarget) continue;
    bool finite = true;
#pragma unroll
    for (int k = 0; k < D; ++k) finite = finite && isfinite(acc[r][k]);
    if (!finite) {  // a source at exactly this target's position: sum again with K(0) := 0
#pragma unroll
      for (int k = 0; k < D; ++k) acc[r][k] = T(0);
      for (uint32_t j = j_begin; j < j_end; ++j) {
        const Row<T, D> rj = load_row<T, D>(a.x, j);
        add_pair<T, D, KF, true>(ri[r].x, rj.x, a.kparam, a.radius_sq, acc[r]);
      }
    }
    if (da.split > 1) {
      Row<T, D> p;
#pragma unroll
      for (int k = 0; k < D; ++k) p.x[k] = acc[r][k];
      p.pad = T(0);
      store_row<T, D>(static_cast<T*>(da.partial) + static_cast<size_t>(blockIdx.y) * ntarget * Ld<D>::value, i, p);
    } else {
      finish_target<T, D, MODE>(a, i, ri[r], acc[r]);
    }
  }
}

// Adds the S partial sums of every target in chunk order and finishes it.
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) k_direct_finish(StepParams<T> a, DirectArgs da) {
  const T* targets = (MODE == kDirectQuery) ? static_cast<const T*>(da.q) : a.x;
  const uint32_t ntarget = (MODE == kDirectQuery) ? da.nq : a.n;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntarget) return;
  T acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = T(0);
  for (uint32_t s = 0; s < da.split; ++s) {
    const Row<T, D> p =
        load_row<T, D>(static_cast<const T*>(da.partial) + static_cast<size_t>(s) * ntarget * Ld<D>::value, i);
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] += p.x[k];
  }
  finish_target<T, D, MODE>(a, i, load_row<T, D>(targets, i), acc);
}

template <typename T> constexpr int targets_per_thread() { return sizeof(T) == 4 ? 4 : 2; }

template <typename T, int D, int KF>
void launch_direct_k(int mode, const StepParams<T>& a, const T* q, uint32_t nq, void* partial, size_t partial_rows,
                     const LaunchCfg& cfg, cudaStream_t st) {
  constexpr int R = targets_per_thread<T>();
  const uint32_t nt = (mode == kDirectQuery) ? nq : a.n;
  const uint32_t per_block = kDirectThreads * R;
  const uint32_t tiles = (nt + per_block - 1) / per_block;
  // Split the sources so the grid fills whole waves of resident blocks:
  // the smallest split (<= 64) whose last wave is at least 90 % full, among
  // splits that give every SM work and keep chunks of >= 16 sources; when no
  // split gives every SM work (small systems), the largest one allowed.
  static int resident = 0;  // blocks of this instantiation per SM
  if (resident == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_direct<T, D, KF, kDirectStep, R>, kDirectThreads, 0) !=
            cudaSuccess || nb < 1)
      nb = 1;
    resident = nb;
  }
  const uint64_t wave = static_cast<uint64_t>(cfg.num_sms) * resident;
  uint32_t split = 1, largest = 1;
  double best = -1.0;
  for (uint32_t sp = 1; sp <= 64; ++sp) {
    if (static_cast<uint64_t>(sp) * nt > partial_rows && sp > 1) break;
    if (sp > 1 && a.n / sp < 16u) break;
    largest = sp;
    const uint64_t blocks = static_cast<uint64_t>(tiles) * sp;
    const double waves = static_cast<double>(blocks) / static_cast<double>(wave);
    const double eff = waves / static_cast<double>((blocks + wave - 1) / wave);
    if (blocks < static_cast<uint64_t>(cfg.num_sms) && sp < 64) continue;
    if (eff > best + 1e-9) {
      best = eff;
      split = sp;
    }
    if (eff >= 0.9) break;
  }
  if (best < 0.0) split = largest;  // no split reaches every SM: as many chunks as allowed
  DirectArgs da;
  da.q = q;
  da.nq = nq;
  da.partial = partial;
  da.split = split;
  // chunks of whole 16-row multiples (a tile multiple when the chunks are large)
  const uint32_t chunk_rows = (a.n + split - 1) / split;
  da.chunk = (chunk_rows >= kDirectThreads) ? (chunk_rows + kDirectThreads - 1) / kDirectThreads * kDirectThreads
                                           : (chunk_rows + 15u) / 16u * 16u;
  const dim3 grid(tiles, split);
  if (mode == kDirectStep) k_direct<T, D, KF, kDirectStep, R><<<grid, kDirectThreads, 0, st>>>(a, da);
  else if (mode == kDirectForces) k_direct<T, D, KF, kDirectForces, R><<<grid, kDirectThreads, 0, st>>>(a, da);
  else k_direct<T, D, KF, kDirectQuery, R><<<grid, kDirectThreads, 0, st>>>(a, da);
  mark_launch(cfg, st, "k_direct");
  if (split > 1) {
    const uint32_t g2 = (nt + 255) / 256;
    if (mode == kDirectStep) k_direct_finish<T, D, kDirectStep><<<g2, 256, 0, st>>>(a, da);
    else if (mode == kDirectForces) k_direct_finish<T, D, kDirectForces><<<g2, 256, 0, st>>>(a, da);
    else k_direct_finish<T, D, kDirectQuery><<<g2, 256, 0, st>>>(a, da);
    mark_launch(cfg, st, "k_direct_finish");
  }
}

template <typename T, int D>
void launch_direct_d(int mode, const StepParams<T>& a, const T* q, uint32_t nq, void* partial, size_t partial_rows,
                     const LaunchCfg& cfg, cudaStream_t st) {
  switch (a.kf) {
    case RBM_K_INV1D:
      if constexpr (D == 1) launch_direct_k<T, D, RBM_K_INV1D>(mode, a, q, nq, partial, partial_rows, cfg, st);
      break;
    case RBM_K_COULOMB: launch_direct_k<T, D, RBM_K_COULOMB>(mode, a, q, nq, partial, partial_rows, cfg, st); break;
    case RBM_K_BOUNDED_CONF:
      launch_direct_k<T, D, RBM_K_BOUNDED_CONF>(mode, a, q, nq, partial, partial_rows, cfg, st);
      break;
    case RBM_K_GAUSS_AGG:
      launch_direct_k<T, D, RBM_K_GAUSS_AGG>(mode, a, q, nq, partial, partial_rows, cfg, st);
      break;
    case RBM_K_REG_ATTRACT:
      launch_direct_k<T, D, RBM_K_REG_ATTRACT>(mode, a, q, nq, partial, partial_rows, cfg, st);
      break;
    case RBM_K_SMOOTH_TEST:
      launch_direct_k<T, D, RBM_K_SMOOTH_TEST>(mode, a, q, nq, partial, partial_rows, cfg, st);
      break;
    default: launch_direct_k<T, D, RBM_K_LINEAR>(mode, a, q, nq, partial, partial_rows, cfg, st); break;
  }
}

}  // namespace

template <typename T>
void launch_direct(int d, int mode, const void* params, const T* q, uint32_t nq, void* partial, size_t partial_rows,
                   const LaunchCfg& cfg, cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  if (d == 1) launch_direct_d<T, 1>(mode, a, q, nq, partial, partial_rows, cfg, st);
  else if (d == 2) launch_direct_d<T, 2>(mode, a, q, nq, partial, partial_rows, cfg, st);
  else launch_direct_d<T, 3>(mode, a, q, nq, partial, partial_rows, cfg, st);
}

#ifdef RBM_DIRECT_F32
template void launch_direct<float>(int, int, const void*, const float*, uint32_t, void*, size_t, const LaunchCfg&,
                                   cudaStream_t);
#endif
#ifdef RBM_DIRECT_F64
template void launch_direct<double>(int, int, const void*, const double*, uint32_t, void*, size_t, const LaunchCfg&,
                                    cudaStream_t);
#endif

}  // namespace rbm
