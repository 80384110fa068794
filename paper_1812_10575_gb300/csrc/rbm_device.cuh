// Device-side building blocks of the RBM-1 hot path: the counter-based RNG,
// Box-Muller Brownian increments, the interaction kernels K, -grad V, the
// Euler-Maruyama update and row loads/stores of the N x ld position array.
//
// Everything here is written from the paper (arXiv:1812.10575) and from
// Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11) for
// Philox; no code is shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rbm.h"

namespace rbm {

// ---------------------------------------------------------------------------
// Philox4x32-10.  A round maps counter (c0,c1,c2,c3), key (k0,k1) to
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
// advances by the Weyl increments (W0, W1) between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += kPhiloxW0;
      k.y += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The round keys of Philox4x32-10 for one seed (the Weyl sequence k + r W,
// r = 0..9), computed once on the host and read by the kernels from their
// launch parameters instead of being advanced in every call.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& ks) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ ks.k0[round], lo1, hi0 ^ c.w ^ ks.k1[round], lo0);
  }
  return c;
}

constexpr uint32_t kStreamPerm = 0;
constexpr uint32_t kStreamNoise = 1;

// Permutation key of particle `id` at step m (counter word 1 = m mod 2^32).
__device__ __forceinline__ uint64_t perm_key(uint32_t id, uint32_t m32, uint32_t replica, uint2 seed) {
  const uint4 w = philox4x32_10(make_uint4(id, m32, replica, kStreamPerm * 256u), seed);
  return (static_cast<uint64_t>(w.y) << 32) | w.x;
}
__device__ __forceinline__ uint64_t perm_key(uint32_t id, uint32_t m32, uint32_t replica, const PhiloxKeys& ks) {
  const uint4 w = philox4x32_10(make_uint4(id, m32, replica, kStreamPerm * 256u), ks);
  return (static_cast<uint64_t>(w.y) << 32) | w.x;
}

// ---------------------------------------------------------------------------
// Box-Muller pairs of particle `id` at step m.  FP64 runs: pair t from the
// 64-bit words w1 = a1:a0 and w2 = a3:a2 of draw (id, m, r, 256 + t),
// u = ((w >> 11) + 1) 2^-53.  FP32 runs: u = ((w >> 8) + 1) 2^-24 of one
// 32-bit word, and one draw (id, m, r, 256 + q) gives two pairs: pair 2q
// from words a1, a3 (the top 24 bits of w1, w2, as FP64 runs read them),
// pair 2q + 1 from words a0, a2.  z0 = sqrt(-2 ln u1) cos(2 pi u2),
// z1 = sqrt(-2 ln u1) sin(2 pi u2).
// ---------------------------------------------------------------------------
// FP32 radius r^2 = -2 ln u for u = k 2^-24, k = 1 .. 2^24.  With
// t = 1 - u = (2^24 - k) 2^-24 exact: for t < 2^-7 the series
// -ln(1 - t) = t + t^2/2 + t^3/3 + t^4/4 + ... to the t^4 term (relative
// error below t^4/5 < 2^-30), which keeps r^2 accurate where u is close to 1;
// otherwise the hardware base-2 logarithm, -2 ln 2 log2(u) (absolute error
// at most 2^-22 in log2 u on [1/2, 1), where here |log2 u| > 2^-7 log2 e,
// and 2 ulp below 1/2), so that r = sqrt(r^2) is off by less than 2e-6.
__device__ __forceinline__ float box_muller_r2(uint32_t k) {
  const uint32_t v = (1u << 24) - k;
  if (v < (1u << 17)) {
    const float t = static_cast<float>(v) * 0x1p-24f;
    return 2.0f * t * fmaf(t, fmaf(t, fmaf(t, 0.25f, 0.333333333f), 0.5f), 1.0f);
  }
  return -1.38629436112f * __log2f(static_cast<float>(k) * 0x1p-24f);
}

// FP32: r from r^2 above by the hardware reciprocal square root (r = 0 at
// u = 1); the angle is taken as 2 pi u2 - pi in (-pi, pi], where the hardware
// sine and cosine are accurate to about 4e-7 absolute, and the signs turned
// back (cos(a - pi) = -cos a, sin(a - pi) = -sin a).
__device__ __forceinline__ void normal_pair_words(uint32_t w1, uint32_t w2, float& z0, float& z1) {
  const float u2 = static_cast<float>((w2 >> 8) + 1u) * 0x1p-24f;
  const float r2 = box_muller_r2((w1 >> 8) + 1u);
  const float rad = (r2 > 0.0f) ? r2 * rsqrtf(r2) : 0.0f;
  float s, c;
  __sincosf(fmaf(6.28318530718f, u2, -3.14159265359f), &s, &c);
  z0 = -rad * c;
  z1 = -rad * s;
}

__device__ __forceinline__ void normal_pair(uint4 a, float& z0, float& z1) { normal_pair_words(a.y, a.w, z0, z1); }

__device__ __forceinline__ void normal_pair(uint4 a, double& z0, double& z1) {
  const uint64_t w1 = (static_cast<uint64_t>(a.y) << 32) | a.x;
  const uint64_t w2 = (static_cast<uint64_t>(a.w) << 32) | a.z;
  const double u1 = static_cast<double>((w1 >> 11) + 1u) * 0x1p-53;
  const double u2 = static_cast<double>((w2 >> 11) + 1u) * 0x1p-53;
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

template <typename T, int D>
__device__ __forceinline__ void brownian(uint32_t id, uint32_t m32, uint32_t replica, const PhiloxKeys& ks,
                                         T (&z)[D]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; 4 * q < D; ++q) {  // two pairs per draw
      const uint4 a = philox4x32_10(make_uint4(id, m32, replica, kStreamNoise * 256u + q), ks);
      float z0, z1;
      normal_pair_words(a.y, a.w, z0, z1);
      z[4 * q] = z0;
      if (4 * q + 1 < D) z[4 * q + 1] = z1;
      if (4 * q + 2 < D) {
        normal_pair_words(a.x, a.z, z0, z1);
        z[4 * q + 2] = z0;
        if (4 * q + 3 < D) z[4 * q + 3] = z1;
      }
    }
  } else {
#pragma unroll
    for (int t = 0; 2 * t < D; ++t) {
      const uint4 a = philox4x32_10(make_uint4(id, m32, replica, kStreamNoise * 256u + t), ks);
      T z0, z1;
      normal_pair(a, z0, z1);
      z[2 * t] = z0;
      if (2 * t + 1 < D) z[2 * t + 1] = z1;
    }
  }
}

// The increment of step m when one Brownian path is shared across step
// sizes (the synchronous coupling of Sec. 3, eq. "coupling", extended to
// runs with different dt): a run with step dt and refinement r takes
// z = r^(-1/2) sum_{k<r} z(id, m r + k), the normalised sum of the r standard
// normal draws a run with step dt/r makes over the same interval, so
// sqrt(dt) z equals the sum of its sqrt(dt/r) z_k.  Fine step indices are
// taken mod 2^32, as m is.
template <typename T, int D>
__device__ __forceinline__ void brownian_refined(uint32_t id, uint32_t m32, uint32_t refine, uint32_t replica,
                                                 const PhiloxKeys& ks, T (&z)[D]) {
  T sum[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = T(0);
  for (uint32_t f = 0; f < refine; ++f) {
    T zf[D];
    brownian<T, D>(id, m32 * refine + f, replica, ks, zf);
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] += zf[k];
  }
  const T root = sqrt(static_cast<T>(refine));
#pragma unroll
  for (int k = 0; k < D; ++k) z[k] = sum[k] / root;
}

// Hint: bring the line holding *p into L2 (no value is returned, nothing waits).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// Positions: row i of the N x ld array, ld = D (D = 1, 2) or 4 (D = 3).
// ---------------------------------------------------------------------------
template <int D> struct Ld { static constexpr int value = (D == 3) ? 4 : D; };

template <typename T, int D>
struct Row {
  T x[D];
  T pad;  // lane 4 of a d = 3 row, preserved bit for bit
};

template <typename T, int D>
__device__ __forceinline__ Row<T, D> load_row(const T* __restrict__ X, uint64_t i) {
  Row<T, D> r;
  r.pad = T(0);
  if constexpr (D == 3 && sizeof(T) == 4) {
    const float4 v = reinterpret_cast<const float4*>(X)[i];
    r.x[0] = v.x; r.x[1] = v.y; r.x[2] = v.z; r.pad = v.w;
  } else if constexpr (D == 3) {
    const double2 a = reinterpret_cast<const double2*>(X)[2 * i];
    const double2 b = reinterpret_cast<const double2*>(X)[2 * i + 1];
    r.x[0] = a.x; r.x[1] = a.y; r.x[2] = b.x; r.pad = b.y;
  } else if constexpr (D == 2 && sizeof(T) == 4) {
    const float2 v = reinterpret_cast<const float2*>(X)[i];
    r.x[0] = v.x; r.x[1] = v.y;
  } else if constexpr (D == 2) {
    const double2 v = reinterpret_cast<const double2*>(X)[i];
    r.x[0] = v.x; r.x[1] = v.y;
  } else {
    r.x[0] = X[i];
  }
  return r;
}

template <typename T, int D>
__device__ __forceinline__ void store_row(T* __restrict__ X, uint64_t i, const Row<T, D>& r) {
  if constexpr (D == 3 && sizeof(T) == 4) {
    reinterpret_cast<float4*>(X)[i] = make_float4(r.x[0], r.x[1], r.x[2], r.pad);
  } else if constexpr (D == 3) {
    reinterpret_cast<double2*>(X)[2 * i] = make_double2(r.x[0], r.x[1]);
    reinterpret_cast<double2*>(X)[2 * i + 1] = make_double2(r.x[2], r.pad);
  } else if constexpr (D == 2 && sizeof(T) == 4) {
    reinterpret_cast<float2*>(X)[i] = make_float2(r.x[0], r.x[1]);
  } else if constexpr (D == 2) {
    reinterpret_cast<double2*>(X)[i] = make_double2(r.x[0], r.x[1]);
  } else {
    X[i] = r.x[0];
  }
}

// ---------------------------------------------------------------------------
// Interaction kernels.  Every family is K(x) = s(|x|^2) x; the squared norm
// that decides coincidence (K(0) := 0) and the bounded-confidence cut-off is
// computed as fma(x2,x2, fma(x1,x1, x0*x0)) with round-to-nearest intrinsics
// so the decision is reproducible in the run's precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float ffma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fsub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double fsub_rn(double a, double b) { return __dsub_rn(a, b); }

template <typename T, int D>
__device__ __forceinline__ T sqnorm_rn(const T (&x)[D]) {
  T r2 = fmul_rn(x[0], x[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) r2 = ffma_rn(x[k], x[k], r2);
  return r2;
}

// Single special-function-unit operations (hand-written PTX): approximate
// reciprocal and reciprocal square root, with subnormal inputs and results
// flushed to zero.  Relative error is a few ulp; a zero input gives +inf.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// s(|x|^2) with K(x) = s x, for a non-zero squared norm r2.  FP32 uses the
// approximate special-function operations above (squared norms below the
// smallest normal float count as zero there).
template <int KF>
__device__ __forceinline__ float kernel_scale(float r2, float kparam, float radius_sq) {
  if constexpr (KF == RBM_K_INV1D) {
    return rcp_approx(r2);                       // 1/x = x / x^2
  } else if constexpr (KF == RBM_K_COULOMB) {
    const float ri = rsqrt_approx(r2);
    return ri * ri * ri;                         // x/|x|^3
  } else if constexpr (KF == RBM_K_BOUNDED_CONF) {
    return (r2 < radius_sq) ? -1.0f : 0.0f;      // -x 1{|x| < R}
  } else if constexpr (KF == RBM_K_GAUSS_AGG) {
    return -__expf(-0.5f * r2);                  // -x exp(-|x|^2/2)
  } else if constexpr (KF == RBM_K_REG_ATTRACT) {
    return -rcp_approx(r2 + kparam);             // -x/(|x|^2 + eps)
  } else if constexpr (KF == RBM_K_SMOOTH_TEST) {
    return rcp_approx(1.0f + r2);                // x/(1+|x|^2)
  } else {
    return -kparam;                              // -c x
  }
}

template <int KF>
__device__ __forceinline__ double kernel_scale(double r2, double kparam, double radius_sq) {
  if constexpr (KF == RBM_K_INV1D) {
    return 1.0 / r2;
  } else if constexpr (KF == RBM_K_COULOMB) {
    return 1.0 / (r2 * sqrt(r2));
  } else if constexpr (KF == RBM_K_BOUNDED_CONF) {
    return (r2 < radius_sq) ? -1.0 : 0.0;
  } else if constexpr (KF == RBM_K_GAUSS_AGG) {
    return -exp(-0.5 * r2);
  } else if constexpr (KF == RBM_K_REG_ATTRACT) {
    return -1.0 / (r2 + kparam);
  } else if constexpr (KF == RBM_K_SMOOTH_TEST) {
    return 1.0 / (1.0 + r2);
  } else {
    return -kparam;
  }
}

// Runtime-dispatched form for the RBM paths (a few evaluations per particle).
template <typename T>
__device__ __forceinline__ T kernel_scale_rt(int kf, T r2, T kparam, T radius_sq) {
  switch (kf) {
    case RBM_K_INV1D: return kernel_scale<RBM_K_INV1D>(r2, kparam, radius_sq);
    case RBM_K_COULOMB: return kernel_scale<RBM_K_COULOMB>(r2, kparam, radius_sq);
    case RBM_K_BOUNDED_CONF: return kernel_scale<RBM_K_BOUNDED_CONF>(r2, kparam, radius_sq);
    case RBM_K_GAUSS_AGG: return kernel_scale<RBM_K_GAUSS_AGG>(r2, kparam, radius_sq);
    case RBM_K_REG_ATTRACT: return kernel_scale<RBM_K_REG_ATTRACT>(r2, kparam, radius_sq);
    case RBM_K_SMOOTH_TEST: return kernel_scale<RBM_K_SMOOTH_TEST>(r2, kparam, radius_sq);
    default: return kernel_scale<RBM_K_LINEAR>(r2, kparam, radius_sq);
  }
}

// acc += K(xi - xj): the kernel family KF fixed at compile time, or (KF < 0)
// chosen at run time from kf; the same arithmetic either way.
template <typename T, int D, int KF = -1>
__device__ __forceinline__ void add_pair_force_rt(int kf, T kparam, T radius_sq, const T (&xi)[D], const T (&xj)[D],
                                                  T (&acc)[D]) {
  T x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = fsub_rn(xi[k], xj[k]);
  const T r2 = sqnorm_rn<T, D>(x);
  T s;
  if constexpr (KF < 0) s = (r2 == T(0)) ? T(0) : kernel_scale_rt<T>(kf, r2, kparam, radius_sq);
  else s = (r2 == T(0)) ? T(0) : kernel_scale<KF>(r2, kparam, radius_sq);
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] += s * x[k];
}

// ---------------------------------------------------------------------------
// Parameters of one step as the kernels see them.
// ---------------------------------------------------------------------------
template <typename T>
struct StepParams {
  T* x;               // positions, N x ld (in place for RBM)
  T* xout;            // direct step output / generic-batch staging, N x ld
  T* fout;            // diagnostic force output, N x ld (or null)
  int32_t* status;    // latched device status
  uint32_t n;
  int32_t p;
  int32_t kf;         // rbm_kernel
  int32_t vkind;      // rbm_potential
  int32_t renorm;
  int32_t gbm;        // 1: multiplicative noise sigma X dB
  int32_t scheme;     // rbm_scheme
  T dt, sq;           // tau, sigma sqrt(tau)
  T vcoef, kparam, radius_sq;
  uint2 seed;
  uint32_t replica;
  const int64_t* m_ptr;  // step counter in device memory (graph replay) or null
  int64_t m_off;         // added to *m_ptr (or the step itself when m_ptr is null)
  const int* skip;       // when set and non-zero, the RBM step kernels do nothing (surrogate mode)
  T* xprev;              // Verlet: V_0 before the first step, X_{n-1} afterwards (N x ld)
  int64_t verlet_m0;     // Verlet: the step index of the Taylor start
  uint32_t noise_refine; // r > 1: the increment of step m sums the r increments of fine steps m r + k
  T inv_pm1;             // 1/(p - 1) in the run's precision (IEEE division, on the host)
  PhiloxKeys keys;       // round keys of `seed`
};

template <typename T>
__device__ __forceinline__ bool skipped(const StepParams<T>& a) {
  return a.skip != nullptr && *a.skip != 0;
}

template <typename T>
__device__ __forceinline__ uint32_t step_index(const StepParams<T>& a) {
  const int64_t m = (a.m_ptr ? *a.m_ptr : 0) + a.m_off;
  return static_cast<uint32_t>(static_cast<uint64_t>(m));
}

// Sum of s_warp[0 .. warp): the totals of the warps before the calling one
// in a block scan, added by the warp's lanes at once.
__device__ __forceinline__ uint32_t warps_before(const uint32_t* s_warp, int warp, int lane) {
  uint32_t v = (lane < warp) ? s_warp[lane] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void latch_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

template <typename T> __device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

__device__ __forceinline__ float exp_rt(float v) { return expf(v); }
__device__ __forceinline__ double exp_rt(double v) { return exp(v); }

// y = x + dt (fk - grad V(x)) + sigma sqrt(dt) z for given increments z, then
// the optional projection onto the unit sphere; latches RBM_ERR_NONFINITE on a
// non-finite result.  Multiplicative noise (gbm): the noise term is
// sigma sqrt(dt) x z, or, after the exact pair flow of the splitting scheme
// (split_flow), the exact geometric flow y = x exp(-s^2/2 + s z) + dt (fk -
// grad V(x)), s = sigma sqrt(dt) (Ito).
template <typename T, int D>
__device__ __forceinline__ void euler_apply(const StepParams<T>& a, const T (&x)[D], const T (&fk)[D],
                                            const T (&z)[D], T (&y)[D], bool split_flow = false) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T fv = (a.vkind == RBM_V_QUADRATIC) ? -a.vcoef * x[k] : T(0);
    if (!a.gbm) y[k] = x[k] + a.dt * (fk[k] + fv) + a.sq * z[k];
    else if (split_flow) y[k] = x[k] * exp_rt(T(-0.5) * a.sq * a.sq + a.sq * z[k]) + a.dt * (fk[k] + fv);
    else y[k] = x[k] + a.dt * (fk[k] + fv) + a.sq * x[k] * z[k];
  }
  if (a.renorm) {
    T nrm = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) nrm += y[k] * y[k];
    nrm = sqrt(nrm);
#pragma unroll
    for (int k = 0; k < D; ++k) y[k] = y[k] / nrm;
  }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) ok = ok && finite_val(y[k]);
  if (!ok) latch_status(a.status, RBM_ERR_NONFINITE);
}

// Verlet scheme of the second-order system (Appendix A, Sec. 4.1): with
// F = fk - grad V(x), y = x + dt v + dt^2 F / 2 at the first step (xprev
// holds v = V_0) and y = 2 x - x_prev + dt^2 F afterwards; x becomes the new
// x_prev.  m32 is the step index the kernel read when it started (a graph
// replay advances the device counter during the step); the Taylor start is
// the step whose index agrees with verlet_m0 mod 2^32.  Latches
// RBM_ERR_NONFINITE on a non-finite result.
template <typename T, int D>
__device__ __forceinline__ void verlet_update(const StepParams<T>& a, uint32_t id, uint32_t m32, const T (&x)[D],
                                              const T (&fk)[D], T (&y)[D]) {
  const bool first = (m32 == static_cast<uint32_t>(static_cast<uint64_t>(a.verlet_m0)));
  const T* q = a.xprev + static_cast<uint64_t>(id) * Ld<D>::value;
  T* w = a.xprev + static_cast<uint64_t>(id) * Ld<D>::value;
  const T tt = a.dt * a.dt;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T fv = (a.vkind == RBM_V_QUADRATIC) ? -a.vcoef * x[k] : T(0);
    const T f = fk[k] + fv;
    const T pk = q[k];
    y[k] = first ? x[k] + a.dt * pk + T(0.5) * tt * f : T(2) * x[k] - pk + tt * f;
    w[k] = x[k];
    ok = ok && finite_val(y[k]);
  }
  if (!ok) latch_status(a.status, RBM_ERR_NONFINITE);
}

// The Euler-Maruyama update of particle `id` at step m with its Brownian
// increment (id, m) (synchronous coupling of RBM-1 and the direct step).
template <typename T, int D>
__device__ __forceinline__ void euler_update(const StepParams<T>& a, uint32_t id, uint32_t m32, const T (&x)[D],
                                             const T (&fk)[D], T (&y)[D], bool split_flow = false) {
  T z[D];
  if (a.sq != T(0)) {
    if (a.noise_refine > 1u) brownian_refined<T, D>(id, m32, a.noise_refine, a.replica, a.keys, z);
    else brownian<T, D>(id, m32, a.replica, a.keys, z);
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) z[k] = T(0);
  }
  euler_apply<T, D>(a, x, fk, z, y, split_flow);
}

// euler_update for the plain configuration (Euler-Maruyama, additive noise,
// no projection, no noise refinement), with its arithmetic.
template <typename T, int D>
__device__ __forceinline__ void euler_update_plain(const StepParams<T>& a, uint32_t id, uint32_t m32, const T (&x)[D],
                                                   const T (&fk)[D], T (&y)[D]) {
  T z[D];
  if (a.sq != T(0)) {
    brownian<T, D>(id, m32, a.replica, a.keys, z);
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) z[k] = T(0);
  }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T fv = (a.vkind == RBM_V_QUADRATIC) ? -a.vcoef * x[k] : T(0);
    y[k] = x[k] + a.dt * (fk[k] + fv) + a.sq * z[k];
    ok = ok && finite_val(y[k]);
  }
  if (!ok) latch_status(a.status, RBM_ERR_NONFINITE);
}

// The update of the configured scheme after the interaction force fk.
template <typename T, int D>
__device__ __forceinline__ void scheme_update(const StepParams<T>& a, uint32_t id, uint32_t m32, const T (&x)[D],
                                              const T (&fk)[D], T (&y)[D]) {
  if (a.scheme == RBM_SCHEME_VERLET) verlet_update<T, D>(a, id, m32, x, fk, y);
  else euler_update<T, D>(a, id, m32, x, fk, y);
}

}  // namespace rbm
