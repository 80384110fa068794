// Direct O(N^2) forward-Euler step (the reference method of Sec. 4.1 of
// arXiv:1812.10575, eq. "interactingps"):
//   F^K_i = 1/(N-1) sum_{j != i} K(X^i - X^j),
//   X^i  <- X^i + dt (F^K_i - grad V(X^i)) + sigma sqrt(dt) z_i,
// with z_i the same Brownian increment the RBM step of step m draws.
//
// One thread per target particle i; source particles stream through shared
// memory in tiles of blockDim rows, every warp reading the same source row at
// once (a broadcast), so the inner loop is FP32/FP64-pipe bound: per pair D
// subtractions, D multiply-adds for |x|^2, the kernel's scale s(|x|^2) and D
// multiply-adds into the accumulator.  K(0) := 0 removes the i = j term
// without a branch on the index.  The kernel family is a template parameter
// so the pair loop carries no dispatch.
#include "rbm_device.cuh"
#include "rbm_internal.h"

namespace rbm {

namespace {

constexpr int kDirectStep = 0;
constexpr int kDirectForces = 1;
constexpr int kDirectQuery = 2;

template <typename T, int D, int KF, int MODE>
__global__ void k_direct(StepParams<T> a, const T* __restrict__ q, uint32_t nq) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);          // blockDim rows of D values
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t ntarget = (MODE == kDirectQuery) ? nq : a.n;
  const bool valid = i < ntarget;
  Row<T, D> ri;
  if (valid) {
    ri = load_row<T, D>((MODE == kDirectQuery) ? q : a.x, i);
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) ri.x[k] = T(0);
    ri.pad = T(0);
  }
  T acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = T(0);

  for (uint32_t j0 = 0; j0 < a.n; j0 += blockDim.x) {
    const uint32_t cnt = min(static_cast<uint32_t>(blockDim.x), a.n - j0);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const Row<T, D> rj = load_row<T, D>(a.x, j0 + threadIdx.x);
#pragma unroll
      for (int k = 0; k < D; ++k) tile[threadIdx.x * D + k] = rj.x[k];
    }
    __syncthreads();
#pragma unroll 8
    for (uint32_t jj = 0; jj < cnt; ++jj) {
      T x[D];
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = fsub_rn(ri.x[k], tile[jj * D + k]);
      const T r2 = sqnorm_rn<T, D>(x);
      const T s = (r2 == T(0)) ? T(0) : kernel_scale<KF>(r2, a.kparam, a.radius_sq);
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] += s * x[k];
    }
  }
  if (!valid) return;
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
  euler_update<T, D>(a, i, m32, ri.x, fk, y);
#pragma unroll
  for (int k = 0; k < D; ++k) ri.x[k] = y[k];
  store_row<T, D>(a.xout, i, ri);
}

template <typename T, int D, int KF>
void launch_direct_k(int mode, const StepParams<T>& a, const T* q, uint32_t nq, const LaunchCfg& cfg,
                     cudaStream_t st) {
  const int block = cfg.direct_block;
  const uint32_t nt = (mode == kDirectQuery) ? nq : a.n;
  const uint32_t grid = max(1u, (nt + block - 1) / block);
  const size_t smem = static_cast<size_t>(block) * D * sizeof(T);
  if (mode == kDirectStep) k_direct<T, D, KF, kDirectStep><<<grid, block, smem, st>>>(a, q, nq);
  else if (mode == kDirectForces) k_direct<T, D, KF, kDirectForces><<<grid, block, smem, st>>>(a, q, nq);
  else k_direct<T, D, KF, kDirectQuery><<<grid, block, smem, st>>>(a, q, nq);
  mark_launch(cfg, st, "k_direct");
}

template <typename T, int D>
void launch_direct_d(int mode, const StepParams<T>& a, const T* q, uint32_t nq, const LaunchCfg& cfg,
                     cudaStream_t st) {
  switch (a.kf) {
    case RBM_K_INV1D:
      if constexpr (D == 1) launch_direct_k<T, D, RBM_K_INV1D>(mode, a, q, nq, cfg, st);
      break;
    case RBM_K_COULOMB: launch_direct_k<T, D, RBM_K_COULOMB>(mode, a, q, nq, cfg, st); break;
    case RBM_K_BOUNDED_CONF: launch_direct_k<T, D, RBM_K_BOUNDED_CONF>(mode, a, q, nq, cfg, st); break;
    case RBM_K_GAUSS_AGG: launch_direct_k<T, D, RBM_K_GAUSS_AGG>(mode, a, q, nq, cfg, st); break;
    case RBM_K_REG_ATTRACT: launch_direct_k<T, D, RBM_K_REG_ATTRACT>(mode, a, q, nq, cfg, st); break;
    case RBM_K_SMOOTH_TEST: launch_direct_k<T, D, RBM_K_SMOOTH_TEST>(mode, a, q, nq, cfg, st); break;
    default: launch_direct_k<T, D, RBM_K_LINEAR>(mode, a, q, nq, cfg, st); break;
  }
}

}  // namespace

template <typename T>
void launch_direct(int d, int mode, const void* params, const T* q, uint32_t nq, const LaunchCfg& cfg,
                   cudaStream_t st) {
  const StepParams<T>& a = *static_cast<const StepParams<T>*>(params);
  if (d == 1) launch_direct_d<T, 1>(mode, a, q, nq, cfg, st);
  else if (d == 2) launch_direct_d<T, 2>(mode, a, q, nq, cfg, st);
  else launch_direct_d<T, 3>(mode, a, q, nq, cfg, st);
}

#ifdef RBM_DIRECT_F32
template void launch_direct<float>(int, int, const void*, const float*, uint32_t, const LaunchCfg&, cudaStream_t);
#endif
#ifdef RBM_DIRECT_F64
template void launch_direct<double>(int, int, const void*, const double*, uint32_t, const LaunchCfg&, cudaStream_t);
#endif

}  // namespace rbm
