// Learned mean-field surrogate: a d -> 64 -> 64 -> d tanh MLP (d = 2, 3) approximating
// the interaction force F(x) = 1/(N-1) sum_j K(x - X^j), i.e. the mean-field
// force K * mu of eq. "nonlinearfp" (arXiv:1812.10575) on the empirical
// measure, trained on direct-sum forces at sampled particles and used in
// place of the random-batch force while its held-out relative error stays
// below a tolerance.  The paper has no surrogate; the definitions (network,
// normalisation, loss, Adam, bfloat16 operands) are those of the oracle
// module oracle/mlp.py.
//
//   xh = (x - mu)/s,  h1 = tanh(W1 xh + b1),  h2 = tanh(W2 h1 + b2),
//   (positions, queries and forces in rows of ld = d (d = 2) or 4 (d = 3) floats)
//   y = W3 h2 + b3,   F(x) = sF y,           loss = 1/B sum |y - F_target/sF|^2
//
// The 64 x 64 contractions run on the tensor cores (tcgen05.mma, BF16
// operands in shared memory, FP32 accumulators in tensor memory): the forward
// product h1 W2^T, and in training dh1 = dz2 W2 and the weight gradient
// dW2 = dz2^T h1 over each 128-sample tile.  The 2-wide layers, the biases,
// tanh (its derivative as 1 - tanh^2), the loss and Adam run on the FP32 pipe
// and the special-function unit.  Weights are read rounded to
// bfloat16 everywhere; FP32 masters, Adam moments and the bias terms stay in
// FP32.  Every mbarrier wait is bounded; a wait that runs out latches
// RBM_ERR_TIMEOUT and the block frees its tensor memory and returns.
#include "rbm_device.cuh"
#include "rbm_internal.h"
#include "tc.cuh"

#include <algorithm>

namespace rbm {
namespace {

constexpr int kH = 64;
constexpr uint32_t kWaitIter = 1u << 24;

// Parameter layout of the d -> 64 -> 64 -> d network (float offsets):
// W1[64][d], b1[64], W2[64][64], b2[64], W3[d][64], b3[d].
template <int D>
struct Lay {
  static constexpr int OW1 = 0, OB1 = kH * D, OW2 = OB1 + kH, OB2 = OW2 + kH * kH, OW3 = OB2 + kH,
                       OB3 = OW3 + kH * D, NP = OB3 + D;
};

// A network input or output row: d floats of a row of Ld<d> floats.
template <int D>
__device__ __forceinline__ void load_vec(const float* base, uint32_t i, float (&v)[D]) {
  if constexpr (D == 2) {
    const float2 t = reinterpret_cast<const float2*>(base)[i];
    v[0] = t.x; v[1] = t.y;
  } else {
    const float4 t = reinterpret_cast<const float4*>(base)[i];
    v[0] = t.x; v[1] = t.y; v[2] = t.z;
  }
}
template <int D>
__device__ __forceinline__ void store_vec(float* base, uint32_t i, const float (&v)[D], float pad = 0.0f) {
  if constexpr (D == 2) reinterpret_cast<float2*>(base)[i] = make_float2(v[0], v[1]);
  else reinterpret_cast<float4*>(base)[i] = make_float4(v[0], v[1], v[2], pad);
}

struct SurArgs {
  float* theta;      // [NP] FP32 masters
  float* mom1;       // [NP] Adam first moments
  float* mom2;       // [NP] Adam second moments
  float* wq;         // [NP] weights rounded to bf16 (biases exact)
  uint16_t* w2f;     // W2 as the B operand of h1 W2^T   (N = out, K = in), core layout
  uint16_t* w2b;     // W2 as the B operand of dz2 W2    (N = in, K = out), core layout
  float* norm;       // mu (d), s, sF
  int* adam_t;       // Adam steps taken before the current checkpoint
  int* flag;         // 1: the surrogate drives the steps, 0: the RBM fallback does
  float* err;        // [0] last held-out relative error, [1] last drift error
  unsigned long long* counters;  // steps taken by the surrogate, by the fallback
  float* partial;    // [blocks][NP + 1] per-block gradient and loss
  uint32_t* qidx;    // [nq] sampled particle ids
  float* q;          // [nq][ld] query positions
  float* fq;         // [nq][ld] direct forces at the queries
  float* fpred;      // [nq][ld] surrogate forces at the queries
  uint32_t nq, ntrain;
  float lr, tol;
  int32_t* status;
};

template <int D>
__device__ __forceinline__ bool is_weight(int i) {
  using L = Lay<D>;
  return (i >= L::OW1 && i < L::OB1) || (i >= L::OW2 && i < L::OB2) || (i >= L::OW3 && i < L::OB3);
}

// Publish parameter i to the bf16 views (wq and the two W2 operand layouts).
template <int D>
__device__ __forceinline__ void publish(const SurArgs& s, int i, float th) {
  using L = Lay<D>;
  s.wq[i] = is_weight<D>(i) ? tc::bf16_round(th) : th;
  if (i >= L::OW2 && i < L::OB2) {
    const uint32_t o = static_cast<uint32_t>(i - L::OW2) / kH, in = static_cast<uint32_t>(i - L::OW2) % kH;
    const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(th));
    s.w2f[tc::core_off(o, in, kH) >> 1] = b;
    s.w2b[tc::core_off(in, o, kH) >> 1] = b;
  }
}

// Initial parameters: every weight and bias of a layer uniform in
// [-c/sqrt(fan_in), c/sqrt(fan_in)) (Philox, counter (i, 0, 0, stream 3)),
// c = 1 except c = 3 for the input layer, whose units then switch on the
// scale of one cluster of particles rather than of the whole cloud.
template <int D>
__global__ void k_sur_init(SurArgs s, uint2 seed) {
  using L = Lay<D>;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L::NP; i += gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, 0u, 3u * 256u), seed);
    const float u = static_cast<float>(w.x >> 8) * 0x1p-23f - 1.0f;  // uniform in [-1, 1)
    // 3/sqrt(d) for the input layer, 1/sqrt(64) for the others
    const float bound = (i < L::OW2) ? (D == 2 ? 3.0f * 0.70710678f : 3.0f * 0.57735027f) : 0.125f;
    const float th = u * bound;
    s.theta[i] = th;
    s.mom1[i] = 0.0f;
    s.mom2[i] = 0.0f;
    publish<D>(s, i, th);
  }
}

// Re-derive the bf16 views after the host replaced the parameters.
template <int D>
__global__ void k_sur_publish(SurArgs s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Lay<D>::NP; i += gridDim.x * blockDim.x)
    publish<D>(s, i, s.theta[i]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tanh z = sign(z) (1 - 2/(e^{2|z|} + 1)), straight from the definition, with
// the hardware base-2 exponential (e^{2|z|} = 2^{2 log2(e) |z|}) and
// reciprocal.  Absolute error about 1e-7 (2e-6 at worst, from rounding the
// exponent's argument); e^{2|z|} = inf gives exactly 1.
__device__ __forceinline__ float act_tanh(float z) {
  const float e = ex2_approx(2.8853900817779268f * fabsf(z));
  return copysignf(1.0f - 2.0f * rcp_approx(e + 1.0f), z);
}

// Pre-activation of hidden unit k of layer 1: b1 + sum_c W1[k][c] xh[c],
// accumulated from the last input coordinate to the first.
template <int D>
__device__ __forceinline__ float layer1_z(const float* sW1, const float* sB1, int k, const float (&xh)[D]) {
  float z = sB1[k];
#pragma unroll
  for (int c = D - 1; c >= 0; --c) z = fmaf(sW1[D * k + c], xh[c], z);
  return z;
}

// Layer 1 of one sample into its row of the A operand (and, for training, its
// column of the transposed copy).
template <int D>
__device__ __forceinline__ void layer1_to_smem(const float* sW1, const float* sB1, const float (&xh)[D],
                                               unsigned char* a_smem, uint32_t row, unsigned char* at_smem) {
#pragma unroll
  for (int kb = 0; kb < 8; ++kb) {
    float h[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = act_tanh(layer1_z<D>(sW1, sB1, kb * 8 + c, xh));
    *reinterpret_cast<uint4*>(a_smem + tc::core_off(row, kb * 8, kH)) = tc::pack_bf16x8(h);
    if (at_smem) {  // transposed copy: B operand of the weight gradient (N = feature, K = sample)
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<__nv_bfloat16*>(at_smem + tc::core_off(kb * 8 + c, row, 128)) = __float2bfloat16_rn(h[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Inference: MODE 0 steps the particles (FP32) in place when the flag
// selects the surrogate; MODE 1 writes the surrogate force at query points.
// ---------------------------------------------------------------------------
template <int MODE, int D>
__global__ void __launch_bounds__(128) k_sur_infer(SurArgs s, StepParams<float> a, const float* qpts, uint32_t nq,
                                                   float* fout) {
  using L = Lay<D>;
  __shared__ __align__(1024) unsigned char sA[128 * kH * 2];
  __shared__ __align__(1024) unsigned char sW[kH * kH * 2];
  __shared__ float sW1[D * kH], sB1[kH], sB2[kH], sW3[D * kH], sB3[D], sNorm[D + 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_go;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (MODE == 0) {
    if (tid == 0) {
      const int go = *s.flag;
      s_go = go;
      if (blockIdx.x == 0) atomicAdd(go ? &s.counters[0] : &s.counters[1], 1ull);
    }
    __syncthreads();
    if (!s_go) return;
  }
  for (int i = tid; i < kH * kH * 2 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sW)[i] = reinterpret_cast<const uint4*>(s.w2f)[i];
  for (int i = tid; i < D * kH; i += blockDim.x) {
    sW1[i] = s.wq[L::OW1 + i];
    sW3[i] = s.wq[L::OW3 + i];
  }
  if (tid < kH) {
    sB1[tid] = s.wq[L::OB1 + tid];
    sB2[tid] = s.wq[L::OB2 + tid];
  }
  if (tid < D) sB3[tid] = s.wq[L::OB3 + tid];
  if (tid < D + 2) sNorm[tid] = s.norm[tid];
  if (warp == 0) tc::tmem_alloc(&tslot, 64);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t n = (MODE == 0) ? a.n : nq;
  const uint32_t ntiles = (n + 127) / 128;
  const uint32_t m32 = step_index(a);
  const float* xin = (MODE == 0) ? a.x : qpts;
  uint32_t phase = 0;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t i = t * 128 + tid;
    const bool valid = i < n;
    float x[D], xh[D];
    float pad = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = 0.0f;
    if (valid) {
      load_vec<D>(xin, i, x);
      if constexpr (D == 3) pad = xin[static_cast<size_t>(i) * 4 + 3];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) xh[c] = (x[c] - sNorm[c]) / sNorm[D];
    layer1_to_smem<D>(sW1, sB1, xh, sA, tid, nullptr);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      tc::gemm_128xN(tmem, sA, sW, kH, kH, false);
      tc::commit(&mbar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kWaitIter));
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) {
      if (tid == 0) latch_status(s.status, RBM_ERR_TIMEOUT);
      break;
    }
    float z[kH];
    tc::tmem_ld64(tmem + ((static_cast<uint32_t>(warp) * 32u) << 16), z);
    float yo[D];
#pragma unroll
    for (int c = 0; c < D; ++c) yo[c] = sB3[c];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      const float h2 = act_tanh(z[o] + sB2[o]);
#pragma unroll
      for (int c = 0; c < D; ++c) yo[c] = fmaf(sW3[c * kH + o], h2, yo[c]);
    }
    float fk[D];
#pragma unroll
    for (int c = 0; c < D; ++c) fk[c] = sNorm[D + 1] * yo[c];
    if (valid) {
      if (MODE == 0) {
        float y[D];
        euler_update<float, D>(a, i, m32, x, fk, y);
        store_vec<D>(a.x, i, y, pad);
      } else {
        store_vec<D>(fout, i, fk);
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // tensor memory and sA free for the next tile
    tc::fence_after_sync();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// Sum of v over the 128 threads of the block, returned to every thread.
__device__ __forceinline__ float block128_sum(float v, float* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  const float t = s_red[0] + s_red[1] + s_red[2] + s_red[3];
  __syncthreads();
  return t;
}

constexpr int kStage = kH + 1;  // padded row of the column-reduction stage

// Dynamic shared memory of k_sur_grad (bytes).
constexpr size_t kGradSmem = 128 * kH * 2       // sA: h1 (A of the forward product), then dz2 (A of dh1)
                             + kH * 128 * 2     // sH1T: h1^T, B of dW2 (N = feature, K = sample)
                             + 128 * 128 * 2    // sDT: dz2^T, rows >= 64 zero, A of dW2
                             + 2 * kH * kH * 2  // W2 in the two B layouts
                             + 128 * kStage * 4;  // column-reduction stage

// ---------------------------------------------------------------------------
// Gradient of the loss over one 128-sample tile per block: samples
// (begin + blockIdx.x * 128 + tid) mod ntrain of (xs, ts), weight 1/batch,
// samples past `batch` weighted zero.  Writes the block's gradient and loss
// to partial[blockIdx.x].
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128) k_sur_grad(SurArgs s, const float* xs, const float* ts, uint32_t ntrain,
                                                  uint32_t begin, uint32_t batch) {
  using L = Lay<D>;
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char* sA = gsm;
  unsigned char* sH1T = sA + 128 * kH * 2;
  unsigned char* sDT = sH1T + kH * 128 * 2;
  unsigned char* sWf = sDT + 128 * 128 * 2;
  unsigned char* sWb = sWf + kH * kH * 2;
  float* stage = reinterpret_cast<float*>(sWb + kH * kH * 2);
  __shared__ float sW1[D * kH], sB1[kH], sB2[kH], sW3[D * kH], sB3[D], sNorm[D + 2], s_red[4];
  __shared__ float s_dy[128][D], s_xh[128][D];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kH * kH * 2 / 16; i += blockDim.x) {
    reinterpret_cast<uint4*>(sWf)[i] = reinterpret_cast<const uint4*>(s.w2f)[i];
    reinterpret_cast<uint4*>(sWb)[i] = reinterpret_cast<const uint4*>(s.w2b)[i];
  }
  for (int i = tid; i < 128 * 128 * 2 / 16; i += blockDim.x) reinterpret_cast<uint4*>(sDT)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < D * kH; i += blockDim.x) {
    sW1[i] = s.wq[L::OW1 + i];
    sW3[i] = s.wq[L::OW3 + i];
  }
  if (tid < kH) {
    sB1[tid] = s.wq[L::OB1 + tid];
    sB2[tid] = s.wq[L::OB2 + tid];
  }
  if (tid < D) sB3[tid] = s.wq[L::OB3 + tid];
  if (tid < D + 2) sNorm[tid] = s.norm[tid];
  if (warp == 0) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t t_z2 = tmem, t_dh1 = tmem + 64, t_dw2 = tmem + 128;
  const uint32_t lane_base = (static_cast<uint32_t>(warp) * 32u) << 16;
  float* part = s.partial + static_cast<size_t>(blockIdx.x) * (L::NP + 1);

  // forward
  const uint32_t smp = (begin + blockIdx.x * 128u + static_cast<uint32_t>(tid)) % ntrain;
  const bool inb = blockIdx.x * 128u + static_cast<uint32_t>(tid) < batch;
  float x[D], tf[D], xh[D];
  load_vec<D>(xs, smp, x);
  load_vec<D>(ts, smp, tf);
#pragma unroll
  for (int c = 0; c < D; ++c) xh[c] = (x[c] - sNorm[c]) / sNorm[D];
  layer1_to_smem<D>(sW1, sB1, xh, sA, tid, sH1T);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    tc::gemm_128xN(t_z2, sA, sWf, kH, kH, false);
    tc::commit(&mbar);
  }
  bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, kWaitIter));
  tc::fence_after_sync();
  float buf[kH];
  float yo[D];
#pragma unroll
  for (int c = 0; c < D; ++c) yo[c] = sB3[c];
  if (ok) {
    tc::tmem_ld64(t_z2 + lane_base, buf);
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      buf[o] = act_tanh(buf[o] + sB2[o]);  // h2
#pragma unroll
      for (int c = 0; c < D; ++c) yo[c] = fmaf(sW3[c * kH + o], buf[o], yo[c]);
    }
  }
  // loss and output gradient
  const float inv_b = 1.0f / static_cast<float>(batch);
  float rr[D], dy[D];
  float lsq = 0.0f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    rr[c] = inb ? yo[c] - tf[c] / sNorm[D + 1] : 0.0f;
    dy[c] = 2.0f * rr[c] * inv_b;
    s_dy[tid][c] = dy[c];
    s_xh[tid][c] = xh[c];
    lsq += rr[c] * rr[c];
  }
  // dW3 = dy^T h2 by columns of the stage
#pragma unroll
  for (int o = 0; o < kH; ++o) stage[tid * kStage + o] = buf[o];
  __syncthreads();
  if (tid < kH) {
    float g[D];
#pragma unroll
    for (int c = 0; c < D; ++c) g[c] = 0.0f;
    for (int r = 0; r < 128; ++r) {
      const float h2 = stage[r * kStage + tid];
#pragma unroll
      for (int c = 0; c < D; ++c) g[c] = fmaf(s_dy[r][c], h2, g[c]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) part[L::OW3 + c * kH + tid] = g[c];
  }
  __syncthreads();
  // dz2 = (W3^T dy) (1 - h2^2); db2 by columns; dz2 into the two A operands
  float dz2[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float w = sW3[(D - 1) * kH + o] * dy[D - 1];
#pragma unroll
    for (int c = D - 2; c >= 0; --c) w = fmaf(sW3[c * kH + o], dy[c], w);
    dz2[o] = w * fmaf(-buf[o], buf[o], 1.0f);
    stage[tid * kStage + o] = dz2[o];
  }
#pragma unroll
  for (int kb = 0; kb < 8; ++kb) {
    *reinterpret_cast<uint4*>(sA + tc::core_off(tid, kb * 8, kH)) = tc::pack_bf16x8(&dz2[kb * 8]);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      *reinterpret_cast<__nv_bfloat16*>(sDT + tc::core_off(kb * 8 + c, tid, 128)) =
          __float2bfloat16_rn(dz2[kb * 8 + c]);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0 && ok) {
    tc::gemm_128xN(t_dh1, sA, sWb, kH, kH, false);      // dh1[s][in]  = sum_o dz2[s][o] W2[o][in]
    tc::gemm_128xN(t_dw2, sDT, sH1T, kH, 128, false);   // dW2[o][in] = sum_s dz2[s][o] h1[s][in]
    tc::commit(&mbar);
  }
  if (tid < kH) {
    float g = 0.0f;
    for (int r = 0; r < 128; ++r) g += stage[r * kStage + tid];
    part[L::OB2 + tid] = g;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float gb = block128_sum(dy[c], s_red);
    if (tid == 0) part[L::OB3 + c] = gb;
  }
  {
    const float ls = block128_sum(lsq, s_red);
    if (tid == 0) part[L::NP] = ls * inv_b;
  }
  ok = ok && __syncthreads_and(tc::mbar_wait(&mbar, 1, kWaitIter));
  tc::fence_after_sync();
  if (ok) {
    tc::tmem_ld64(t_dh1 + lane_base, buf);
#pragma unroll
    for (int k = 0; k < kH; ++k) {  // dz1 = dh1 (1 - h1^2), h1 recomputed as in the forward pass
      const float h1 = act_tanh(layer1_z<D>(sW1, sB1, k, xh));
      stage[tid * kStage + k] = buf[k] * fmaf(-h1, h1, 1.0f);
    }
    if (warp < 2) {  // lanes 0..63 hold the 64 rows of dW2
      tc::tmem_ld64(t_dw2 + lane_base, buf);
      const int o = warp * 32 + lane;
#pragma unroll
      for (int in = 0; in < kH; ++in) part[L::OW2 + o * kH + in] = buf[in];
    }
  }
  __syncthreads();
  if (ok && tid < kH) {
    float g[D], gb = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) g[c] = 0.0f;
    for (int r = 0; r < 128; ++r) {
      const float dd = stage[r * kStage + tid];
#pragma unroll
      for (int c = 0; c < D; ++c) g[c] = fmaf(dd, s_xh[r][c], g[c]);
      gb += dd;
    }
#pragma unroll
    for (int c = 0; c < D; ++c) part[L::OW1 + D * tid + c] = g[c];
    part[L::OB1 + tid] = gb;
  }
  if (!ok && tid == 0) latch_status(s.status, RBM_ERR_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Adam on the summed block gradients (fixed block order), then the bf16 views.
// Iteration `it` of `iters` in one training call uses the rate
// lr * 0.01^(it / (iters - 1)): a geometric decay to lr/100 over the call.
template <int D>
__global__ void k_sur_adam(SurArgs s, uint32_t nblocks, int it, int iters) {
  constexpr int kNP = Lay<D>::NP;
  const int t = *s.adam_t + it + 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(t)), c2 = 1.0f - powf(b2, static_cast<float>(t));
  const float lr = s.lr * powf(0.01f, static_cast<float>(it) / static_cast<float>(iters > 1 ? iters - 1 : 1));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
    // the block partials summed in block order; up to a minibatch of 4096
    // samples (32 blocks) every load is issued before the first add
    constexpr uint32_t kUnroll = 32;
    float pb[kUnroll];
#pragma unroll
    for (uint32_t b = 0; b < kUnroll; ++b)
      pb[b] = (b < nblocks) ? s.partial[static_cast<size_t>(b) * (kNP + 1) + i] : 0.0f;
    float g = 0.0f;
#pragma unroll
    for (uint32_t b = 0; b < kUnroll; ++b)
      if (b < nblocks) g += pb[b];
    for (uint32_t b = kUnroll; b < nblocks; ++b) g += s.partial[static_cast<size_t>(b) * (kNP + 1) + i];
    const float m = b1 * s.mom1[i] + (1.0f - b1) * g;
    const float v = b2 * s.mom2[i] + (1.0f - b2) * g * g;
    s.mom1[i] = m;
    s.mom2[i] = v;
    const float th = s.theta[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    s.theta[i] = th;
    publish<D>(s, i, th);
  }
}

__global__ void k_sur_adam_bump(SurArgs s, int iters) { *s.adam_t += iters; }

// Sampled query particles: id = floor(u N) from Philox (id = q, step m, stream 2).
template <int D>
__global__ void k_sur_sample(SurArgs s, StepParams<float> a) {
  const uint32_t m32 = step_index(a);
  for (uint32_t qi = blockIdx.x * blockDim.x + threadIdx.x; qi < s.nq; qi += gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(qi, m32, a.replica, 2u * 256u), a.seed);
    const uint32_t id = __umulhi(w.x, a.n);
    s.qidx[qi] = id;
    if constexpr (D == 2) reinterpret_cast<float2*>(s.q)[qi] = reinterpret_cast<const float2*>(a.x)[id];
    else reinterpret_cast<float4*>(s.q)[qi] = reinterpret_cast<const float4*>(a.x)[id];
  }
}

// Input and output scales from the first checkpoint's queries (one block).
// mu = mean position, s^2 = mean squared distance to mu per coordinate,
// sF^2 = mean squared force per coordinate.
template <int D>
__global__ void k_sur_norm(SurArgs s) {
  constexpr int kA = D + 2;
  __shared__ double red[kA][32];
  double acc[kA];
#pragma unroll
  for (int k = 0; k < kA; ++k) acc[k] = 0.0;
  for (uint32_t i = threadIdx.x; i < s.nq; i += blockDim.x) {
    float x[D], f[D];
    load_vec<D>(s.q, i, x);
    load_vec<D>(s.fq, i, f);
    double xx = 0.0, ff = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      acc[c] += x[c];
      xx += static_cast<double>(x[c]) * x[c];
      ff += static_cast<double>(f[c]) * f[c];
    }
    acc[D] += xx;
    acc[D + 1] += ff;
  }
  for (int k = 0; k < kA; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[kA];
    for (int k = 0; k < kA; ++k) {
      t[k] = 0.0;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t[k] += red[k][w];
    }
    const double n = s.nq;
    double var = t[D] / n;
    for (int c = 0; c < D; ++c) {
      const double mc = t[c] / n;
      var -= mc * mc;
      s.norm[c] = static_cast<float>(mc);
    }
    var = fmax(var, 0.0) / D;
    const double fs = sqrt(t[D + 1] / (static_cast<double>(D) * n));
    s.norm[D] = static_cast<float>(var > 0 ? sqrt(var) : 1.0);
    s.norm[D + 1] = static_cast<float>(fs > 0 ? fs : 1.0);
  }
}

// Relative error ||F_net - F||_2 / ||F||_2 over queries [lo, nq) (one
// block): the held-out quarter after training (drift = 0: also sets the
// selection flag), or every query of a fresh sample before training (drift =
// 1: the error of the network as it drove the interval just ended, into
// err[1]).
template <int D>
__global__ void k_sur_check(SurArgs s, int drift) {
  __shared__ double red[2][32];
  double e = 0, f = 0;
  const uint32_t lo = drift ? 0u : s.ntrain;
  for (uint32_t i = lo + threadIdx.x; i < s.nq; i += blockDim.x) {
    float pv[D], tv[D];
    load_vec<D>(s.fpred, i, pv);
    load_vec<D>(s.fq, i, tv);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double dv = static_cast<double>(pv[c]) - tv[c];
      e += dv * dv;
      f += static_cast<double>(tv[c]) * tv[c];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    f += __shfl_xor_sync(0xffffffffu, f, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e;
    red[1][threadIdx.x >> 5] = f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0, tf = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      te += red[0][w];
      tf += red[1][w];
    }
    const float rel = static_cast<float>(tf > 0 ? sqrt(te / tf) : 0.0);
    if (drift) {
      s.err[1] = rel;
    } else {
      s.err[0] = rel;
      *s.flag = (isfinite(rel) && rel <= s.tol) ? 1 : 0;
    }
  }
}

SurArgs make_args(const SurrogateScratch& ss, int32_t* status) {
  SurArgs s;
  s.theta = ss.theta;
  s.mom1 = ss.mom1;
  s.mom2 = ss.mom2;
  s.wq = ss.wq;
  s.w2f = ss.w2f;
  s.w2b = ss.w2b;
  s.norm = ss.norm;
  s.adam_t = ss.adam_t;
  s.flag = ss.flag;
  s.err = ss.err;
  s.counters = ss.counters;
  s.partial = ss.partial;
  s.qidx = ss.qidx;
  s.q = ss.q;
  s.fq = ss.fq;
  s.fpred = ss.fpred;
  s.nq = ss.nq;
  s.ntrain = ss.ntrain;
  s.lr = ss.lr;
  s.tol = ss.tol;
  s.status = status;
  return s;
}

}  // namespace

int surrogate_param_count(int d) { return d == 3 ? Lay<3>::NP : Lay<2>::NP; }

// A grid of five 128-thread blocks per SM (all that 96 registers a thread
// allow) looping over the 128-row tiles: measured 3 % faster than four and
// than six; eight blocks with the accumulators read in 16-column pieces to fit
// 64 registers ran the step 2x slower.
uint32_t infer_grid(uint32_t tiles, int num_sms) {
  return std::max(1u, std::min(tiles, static_cast<uint32_t>(num_sms) * 5u));
}

cudaError_t prepare_surrogate_kernels() {
  cudaError_t e =
      cudaFuncSetAttribute(k_sur_grad<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kGradSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sur_grad<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kGradSmem));
  return e;
}

// Each wrapper runs the kernel of the network's dimension (ss.d = 2 or 3).
#define SUR_BY_D(launch) \
  do {                   \
    if (ss.d == 3) {     \
      constexpr int D = 3; \
      launch;            \
    } else {             \
      constexpr int D = 2; \
      launch;            \
    }                    \
  } while (0)

cudaError_t sur_init(const SurrogateScratch& ss, int32_t* status, uint64_t seed, cudaStream_t st) {
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  SUR_BY_D((k_sur_init<D><<<18, 256, 0, st>>>(make_args(ss, status), key)));
  return cudaGetLastError();
}

cudaError_t sur_publish(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  SUR_BY_D((k_sur_publish<D><<<18, 256, 0, st>>>(make_args(ss, status))));
  return cudaGetLastError();
}

cudaError_t sur_sample(const SurrogateScratch& ss, const void* params, cudaStream_t st) {
  const StepParams<float>& a = *static_cast<const StepParams<float>*>(params);
  SUR_BY_D((k_sur_sample<D><<<(ss.nq + 255) / 256, 256, 0, st>>>(make_args(ss, a.status), a)));
  return cudaGetLastError();
}

cudaError_t sur_norm(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  SUR_BY_D((k_sur_norm<D><<<1, 1024, 0, st>>>(make_args(ss, status))));
  return cudaGetLastError();
}

cudaError_t sur_train(const SurrogateScratch& ss, int32_t* status, const float* xs, const float* ts, uint32_t ntrain,
                      int iters, uint32_t batch, uint32_t begin0, float lr_scale, const LaunchCfg& cfg,
                      cudaStream_t st) {
  SurArgs s = make_args(ss, status);
  s.lr *= lr_scale;
  const uint32_t nblocks = (batch + 127) / 128;
  for (int it = 0; it < iters; ++it) {
    const uint32_t begin = static_cast<uint32_t>((static_cast<uint64_t>(begin0) + static_cast<uint64_t>(it) * batch) %
                                                 ntrain);
    SUR_BY_D((k_sur_grad<D><<<nblocks, 128, kGradSmem, st>>>(s, xs, ts, ntrain, begin, batch)));
    mark_launch(cfg, st, "k_sur_grad");
    SUR_BY_D((k_sur_adam<D><<<18, 256, 0, st>>>(s, nblocks, it, iters)));
    mark_launch(cfg, st, "k_sur_adam");
  }
  k_sur_adam_bump<<<1, 1, 0, st>>>(s, iters);
  return cudaGetLastError();
}

cudaError_t sur_gradient(const SurrogateScratch& ss, int32_t* status, const float* xs, const float* ts, uint32_t nb,
                         cudaStream_t st) {
  const uint32_t nblocks = (nb + 127) / 128;
  SUR_BY_D((k_sur_grad<D><<<nblocks, 128, kGradSmem, st>>>(make_args(ss, status), xs, ts, nb, 0u, nb)));
  return cudaGetLastError();
}

cudaError_t sur_forces(const SurrogateScratch& ss, int32_t* status, const float* q, uint32_t nq, float* fout,
                       const LaunchCfg& cfg, cudaStream_t st) {
  StepParams<float> a{};
  a.status = status;
  const uint32_t tiles = (nq + 127) / 128;
  SUR_BY_D((k_sur_infer<1, D><<<infer_grid(tiles, cfg.num_sms), 128, 0, st>>>(make_args(ss, status), a, q, nq,
                                                                                     fout)));
  mark_launch(cfg, st, "k_sur_forces");
  return cudaGetLastError();
}

cudaError_t sur_check(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  SUR_BY_D((k_sur_check<D><<<1, 1024, 0, st>>>(make_args(ss, status), 0)));
  return cudaGetLastError();
}

cudaError_t sur_drift(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  SUR_BY_D((k_sur_check<D><<<1, 1024, 0, st>>>(make_args(ss, status), 1)));
  return cudaGetLastError();
}

cudaError_t sur_step(const SurrogateScratch& ss, const void* params, const LaunchCfg& cfg, cudaStream_t st) {
  const StepParams<float>& a = *static_cast<const StepParams<float>*>(params);
  const uint32_t tiles = (a.n + 127) / 128;
  SUR_BY_D((k_sur_infer<0, D><<<infer_grid(tiles, cfg.num_sms), 128, 0, st>>>(make_args(ss, a.status), a,
                                                                                     nullptr, 0u, nullptr)));
  mark_launch(cfg, st, "k_sur_step");
  return cudaGetLastError();
}

#undef SUR_BY_D

}  // namespace rbm
