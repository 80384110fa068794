// Batch updates shared by the RBM step kernels: one batch of the random
// division per group of p consecutive lanes of a warp (p <= 32), positions
// exchanged by warp shuffles, then -grad V, the Brownian increment and the
// Euler-Maruyama update of eq. "firstalgorithm" (arXiv:1812.10575, Sec. 2.1),
// or the exact pair flow of the splitting scheme (Sec. 2.3 item 5).
#pragma once

#include "rbm_device.cuh"

namespace rbm {

constexpr int kModePerm = 0;    // write the permutation only
constexpr int kModeStep = 1;    // step the batches
constexpr int kModeForces = 2;  // write the interaction forces only

// fk = 1/(|C|-1) sum_{j in C, j != i} K(X^i - X^j) for this lane's member i of
// the batch held by the p lanes from `base` (other members' rows by
// shuffles); zero for a singleton.  All 32 lanes call it together.
template <typename T, int D, int KF = -1>
__device__ __forceinline__ void batch_force(const StepParams<T>& a, bool valid, int lg, int bs, int base,
                                            const Row<T, D>& r, T (&fk)[D]) {
  const int p = a.p;
#pragma unroll
  for (int k = 0; k < D; ++k) fk[k] = T(0);
  for (int j = 1; j < p; ++j) {
    int sg = lg + j;
    if (sg >= p) sg -= p;
    T xj[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xj[k] = __shfl_sync(0xffffffffu, r.x[k], base + sg);
    if (valid && sg < bs) add_pair_force_rt<T, D, KF>(a.kf, a.kparam, a.radius_sq, r.x, xj, fk);
  }
  if (!valid) return;
  const T inv = (bs == p) ? a.inv_pm1 : (bs > 1) ? T(1) / static_cast<T>(bs - 1) : T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) fk[k] = (bs > 1) ? fk[k] * inv : T(0);
}

// ---------------------------------------------------------------------------
// One batch per group of p consecutive lanes (p <= 32).  All 32 lanes of the
// warp call these together (the shuffles use the full mask); lanes outside a
// valid batch member pass valid = false.
//   bs    - members of this batch (p, or N mod p for the last batch)
//   lg    - this lane's index inside its group
//   r     - this lane's position row (any value when !valid)
// ---------------------------------------------------------------------------

// The step of this lane's member: r becomes its new row (the pad lane kept);
// returns valid.  The in-batch force, -grad V, the Brownian increment of
// (id, m) and the Euler-Maruyama update (or the exact pair flow of the
// splitting scheme, or the Verlet recurrence).  KF >= 0 fixes the kernel
// family at compile time; kPlain (the caller has checked: Euler-Maruyama,
// additive noise, no projection, no noise refinement) drops the other
// schemes' branches.  The arithmetic is the same in every form.
template <typename T, int D, int KF = -1, bool kPlain = false>
__device__ __forceinline__ bool batch_group_update(const StepParams<T>& a, uint32_t m32, uint32_t id, bool valid,
                                                   int lg, int bs, Row<T, D>& r) {
  const int lane = threadIdx.x & 31;
  const int base = lane - lg;
  if (!valid) {
#pragma unroll
    for (int k = 0; k < D; ++k) r.x[k] = T(0);
  }
  if constexpr (kPlain) {
    T fk[D];
    batch_force<T, D, KF>(a, valid, lg, bs, base, r, fk);
    if (!valid) return false;
    T y[D];
    euler_update_plain<T, D>(a, id, m32, r.x, fk, y);
#pragma unroll
    for (int k = 0; k < D; ++k) r.x[k] = y[k];
    return true;
  }
  if (a.scheme == RBM_SCHEME_SPLIT) {
    // Exact pair flow of K (p = 2), then the Euler-Maruyama step of V and noise.
    const int src = base + (lg ^ 1);
    T xj[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xj[k] = __shfl_sync(0xffffffffu, r.x[k], src);
    if (!valid) return false;
    T y0[D];
#pragma unroll
    for (int k = 0; k < D; ++k) y0[k] = r.x[k];
    if (bs == 2) {
      T delta[D], mid[D];
      T len2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        delta[k] = r.x[k] - xj[k];
        mid[k] = T(0.5) * (r.x[k] + xj[k]);
        len2 += delta[k] * delta[k];
      }
      T dd[D];
#pragma unroll
      for (int k = 0; k < D; ++k) dd[k] = fsub_rn(r.x[k], xj[k]);
      if (sqnorm_rn<T, D>(dd) != T(0)) {
        const T len = sqrt(len2);
        const T newlen = (a.kf == RBM_K_INV1D)    ? sqrt(len2 + T(4) * a.dt)
                         : (a.kf == RBM_K_LINEAR) ? len * exp_rt(T(-2) * a.kparam * a.dt)
                                                  : cbrt(len2 * len + T(6) * a.dt);
#pragma unroll
        for (int k = 0; k < D; ++k) y0[k] = mid[k] + T(0.5) * newlen * (delta[k] / len);
      }
    }
    T fk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) fk[k] = T(0);
    T y[D];
    euler_update<T, D>(a, id, m32, y0, fk, y, true);
#pragma unroll
    for (int k = 0; k < D; ++k) r.x[k] = y[k];
    return true;
  }
  T fk[D];
  batch_force<T, D, KF>(a, valid, lg, bs, base, r, fk);
  if (!valid) return false;
  T y[D];
  scheme_update<T, D>(a, id, m32, r.x, fk, y);
#pragma unroll
  for (int k = 0; k < D; ++k) r.x[k] = y[k];
  return true;
}

template <typename T, int D, int MODE, int KF = -1, bool kPlain = false>
__device__ __forceinline__ void batch_group_row(const StepParams<T>& a, uint32_t m32, uint32_t id, bool valid, int lg,
                                                int bs, Row<T, D> r) {
  if (!valid) {
#pragma unroll
    for (int k = 0; k < D; ++k) r.x[k] = T(0);
    r.pad = T(0);
  }
  if (MODE == kModeStep) {
    if (batch_group_update<T, D, KF, kPlain>(a, m32, id, valid, lg, bs, r)) store_row<T, D>(a.x, id, r);
    return;
  }
  const int lane = threadIdx.x & 31;
  T fk[D];
  batch_force<T, D, KF>(a, valid, lg, bs, lane - lg, r, fk);
  if (!valid) return;
  Row<T, D> f;
#pragma unroll
  for (int k = 0; k < D; ++k) f.x[k] = fk[k];
  f.pad = T(0);
  store_row<T, D>(a.fout, id, f);
}

// As batch_group_row, with the row loaded from the position array.
template <typename T, int D, int MODE, int KF = -1, bool kPlain = false>
__device__ __forceinline__ void batch_group(const StepParams<T>& a, uint32_t m32, uint32_t id, bool valid, int lg,
                                            int bs) {
  Row<T, D> r{};
  if (valid) r = load_row<T, D>(a.x, id);
  batch_group_row<T, D, MODE, KF, kPlain>(a, m32, id, valid, lg, bs, r);
}

// Steps the batches whose first sorted position is q0 + k (k < count), ids
// read from `ids` at offset (batch start - ids_base).  Warp-uniform loop.
template <typename T, int D, int MODE, int KF = -1, bool kPlain = false>
__device__ __forceinline__ void step_batches(const StepParams<T>& a, uint32_t m32, const uint32_t* ids, uint32_t ids_base,
                             uint32_t q0, uint32_t count) {
  const int p = a.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / p;                       // batch groups per warp
  const int nwarps = blockDim.x >> 5;
  const uint32_t per_round = static_cast<uint32_t>(gpw * nwarps);
  const int g = lane / p, lg = lane - g * p;
  for (uint32_t r0 = 0; r0 < count; r0 += per_round) {
    const uint32_t kb = r0 + static_cast<uint32_t>(warp * gpw + g);
    bool valid = (g < gpw) && (kb < count);
    uint32_t id = 0;
    int bs = p;
    if (valid) {
      const uint32_t q = q0 + kb;
      const uint32_t lo = q * static_cast<uint32_t>(p);
      const uint32_t hi = min(lo + static_cast<uint32_t>(p), a.n);
      bs = static_cast<int>(hi - lo);
      valid = lg < bs;
      if (valid) id = ids[lo + lg - ids_base];
    }
    batch_group<T, D, MODE, KF, kPlain>(a, m32, id, valid, lg, bs);
  }
}

}  // namespace rbm
