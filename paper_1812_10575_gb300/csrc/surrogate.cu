// Learned mean-field surrogate: a 2 -> 64 -> 64 -> 2 tanh MLP approximating
// the interaction force F(x) = 1/(N-1) sum_j K(x - X^j), i.e. the mean-field
// force K * mu of eq. "nonlinearfp" (arXiv:1812.10575) on the empirical
// measure, trained on direct-sum forces at sampled particles and used in
// place of the random-batch force while its held-out relative error stays
// below a tolerance.  The paper has no surrogate; the definitions (network,
// normalisation, loss, Adam, bfloat16 operands) are those of the oracle
// module oracle/mlp.py.
//
//   xh = (x - mu)/s,  h1 = tanh(W1 xh + b1),  h2 = tanh(W2 h1 + b2),
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
constexpr int kOW1 = 0, kOB1 = 128, kOW2 = 192, kOB2 = 4288, kOW3 = 4352, kOB3 = 4480, kNP = 4482;
constexpr uint32_t kWaitIter = 1u << 24;

struct SurArgs {
  float* theta;      // [kNP] FP32 masters
  float* mom1;       // [kNP] Adam first moments
  float* mom2;       // [kNP] Adam second moments
  float* wq;         // [kNP] weights rounded to bf16 (biases exact)
  uint16_t* w2f;     // W2 as the B operand of h1 W2^T   (N = out, K = in), core layout
  uint16_t* w2b;     // W2 as the B operand of dz2 W2    (N = in, K = out), core layout
  float* norm;       // mu_x, mu_y, s, sF
  int* adam_t;       // Adam steps taken before the current checkpoint
  int* flag;         // 1: the surrogate drives the steps, 0: the RBM fallback does
  float* err;        // [0] last held-out relative error, [1] last drift error
  unsigned long long* counters;  // steps taken by the surrogate, by the fallback
  float* partial;    // [blocks][kNP + 1] per-block gradient and loss
  uint32_t* qidx;    // [nq] sampled particle ids
  float* q;          // [nq][2] query positions
  float* fq;         // [nq][2] direct forces at the queries
  float* fpred;      // [nq][2] surrogate forces at the queries
  uint32_t nq, ntrain;
  float lr, tol;
  int32_t* status;
};

__device__ __forceinline__ bool is_weight(int i) {
  return (i >= kOW1 && i < kOB1) || (i >= kOW2 && i < kOB2) || (i >= kOW3 && i < kOB3);
}

// Publish parameter i to the bf16 views (wq and the two W2 operand layouts).
__device__ __forceinline__ void publish(const SurArgs& s, int i, float th) {
  s.wq[i] = is_weight(i) ? tc::bf16_round(th) : th;
  if (i >= kOW2 && i < kOB2) {
    const uint32_t o = static_cast<uint32_t>(i - kOW2) / kH, in = static_cast<uint32_t>(i - kOW2) % kH;
    const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(th));
    s.w2f[tc::core_off(o, in, kH) >> 1] = b;
    s.w2b[tc::core_off(in, o, kH) >> 1] = b;
  }
}

// Initial parameters: every weight and bias of a layer uniform in
// [-c/sqrt(fan_in), c/sqrt(fan_in)) (Philox, counter (i, 0, 0, stream 3)),
// c = 1 except c = 3 for the input layer, whose units then switch on the
// scale of one cluster of particles rather than of the whole cloud.
__global__ void k_sur_init(SurArgs s, uint2 seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, 0u, 3u * 256u), seed);
    const float u = static_cast<float>(w.x >> 8) * 0x1p-23f - 1.0f;  // uniform in [-1, 1)
    const float bound = (i < kOW2) ? 3.0f * 0.70710678f : 0.125f;    // 3/sqrt(2), 1/sqrt(64)
    const float th = u * bound;
    s.theta[i] = th;
    s.mom1[i] = 0.0f;
    s.mom2[i] = 0.0f;
    publish(s, i, th);
  }
}

// Re-derive the bf16 views after the host replaced the parameters.
__global__ void k_sur_publish(SurArgs s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) publish(s, i, s.theta[i]);
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

// Pre-activation of hidden unit k of layer 1.
__device__ __forceinline__ float layer1_z(const float* sW1, const float* sB1, int k, float xh0, float xh1) {
  return fmaf(sW1[2 * k], xh0, fmaf(sW1[2 * k + 1], xh1, sB1[k]));
}

// Layer 1 of one sample into its row of the A operand (and, for training, its
// column of the transposed copy).
__device__ __forceinline__ void layer1_to_smem(const float* sW1, const float* sB1, float xh0, float xh1,
                                               unsigned char* a_smem, uint32_t row, unsigned char* at_smem) {
#pragma unroll
  for (int kb = 0; kb < 8; ++kb) {
    float h[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = act_tanh(layer1_z(sW1, sB1, kb * 8 + c, xh0, xh1));
    *reinterpret_cast<uint4*>(a_smem + tc::core_off(row, kb * 8, kH)) = tc::pack_bf16x8(h);
    if (at_smem) {  // transposed copy: B operand of the weight gradient (N = feature, K = sample)
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<__nv_bfloat16*>(at_smem + tc::core_off(kb * 8 + c, row, 128)) = __float2bfloat16_rn(h[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Inference: MODE 0 steps the particles (d = 2, FP32) in place when the flag
// selects the surrogate; MODE 1 writes the surrogate force at query points.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(128) k_sur_infer(SurArgs s, StepParams<float> a, const float* qpts, uint32_t nq,
                                                   float* fout) {
  __shared__ __align__(1024) unsigned char sA[128 * kH * 2];
  __shared__ __align__(1024) unsigned char sW[kH * kH * 2];
  __shared__ float sW1[2 * kH], sB1[kH], sB2[kH], sW3[2 * kH], sB3[2], sNorm[4];
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
  sW1[tid] = s.wq[kOW1 + tid];
  sW3[tid] = s.wq[kOW3 + tid];
  if (tid < kH) {
    sB1[tid] = s.wq[kOB1 + tid];
    sB2[tid] = s.wq[kOB2 + tid];
  }
  if (tid < 2) sB3[tid] = s.wq[kOB3 + tid];
  if (tid < 4) sNorm[tid] = s.norm[tid];
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
    const float2 x = valid ? reinterpret_cast<const float2*>(xin)[i] : make_float2(0.0f, 0.0f);
    const float xh0 = (x.x - sNorm[0]) / sNorm[2], xh1 = (x.y - sNorm[1]) / sNorm[2];
    layer1_to_smem(sW1, sB1, xh0, xh1, sA, tid, nullptr);
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
    float y0 = sB3[0], y1 = sB3[1];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      const float h2 = act_tanh(z[o] + sB2[o]);
      y0 = fmaf(sW3[o], h2, y0);
      y1 = fmaf(sW3[kH + o], h2, y1);
    }
    const float f0 = sNorm[3] * y0, f1 = sNorm[3] * y1;
    if (valid) {
      if (MODE == 0) {
        const float xv[2] = {x.x, x.y}, fk[2] = {f0, f1};
        float y[2];
        euler_update<float, 2>(a, i, m32, xv, fk, y);
        reinterpret_cast<float2*>(a.x)[i] = make_float2(y[0], y[1]);
      } else {
        reinterpret_cast<float2*>(fout)[i] = make_float2(f0, f1);
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
__global__ void __launch_bounds__(128) k_sur_grad(SurArgs s, const float* xs, const float* ts, uint32_t ntrain,
                                                  uint32_t begin, uint32_t batch) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char* sA = gsm;
  unsigned char* sH1T = sA + 128 * kH * 2;
  unsigned char* sDT = sH1T + kH * 128 * 2;
  unsigned char* sWf = sDT + 128 * 128 * 2;
  unsigned char* sWb = sWf + kH * kH * 2;
  float* stage = reinterpret_cast<float*>(sWb + kH * kH * 2);
  __shared__ float sW1[2 * kH], sB1[kH], sB2[kH], sW3[2 * kH], sB3[2], sNorm[4], s_red[4];
  __shared__ float s_dy[128][2], s_xh[128][2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kH * kH * 2 / 16; i += blockDim.x) {
    reinterpret_cast<uint4*>(sWf)[i] = reinterpret_cast<const uint4*>(s.w2f)[i];
    reinterpret_cast<uint4*>(sWb)[i] = reinterpret_cast<const uint4*>(s.w2b)[i];
  }
  for (int i = tid; i < 128 * 128 * 2 / 16; i += blockDim.x) reinterpret_cast<uint4*>(sDT)[i] = make_uint4(0, 0, 0, 0);
  sW1[tid] = s.wq[kOW1 + tid];
  sW3[tid] = s.wq[kOW3 + tid];
  if (tid < kH) {
    sB1[tid] = s.wq[kOB1 + tid];
    sB2[tid] = s.wq[kOB2 + tid];
  }
  if (tid < 2) sB3[tid] = s.wq[kOB3 + tid];
  if (tid < 4) sNorm[tid] = s.norm[tid];
  if (warp == 0) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t t_z2 = tmem, t_dh1 = tmem + 64, t_dw2 = tmem + 128;
  const uint32_t lane_base = (static_cast<uint32_t>(warp) * 32u) << 16;
  float* part = s.partial + static_cast<size_t>(blockIdx.x) * (kNP + 1);

  // forward
  const uint32_t smp = (begin + blockIdx.x * 128u + static_cast<uint32_t>(tid)) % ntrain;
  const bool inb = blockIdx.x * 128u + static_cast<uint32_t>(tid) < batch;
  const float2 x = reinterpret_cast<const float2*>(xs)[smp];
  const float2 tf = reinterpret_cast<const float2*>(ts)[smp];
  const float xh0 = (x.x - sNorm[0]) / sNorm[2], xh1 = (x.y - sNorm[1]) / sNorm[2];
  layer1_to_smem(sW1, sB1, xh0, xh1, sA, tid, sH1T);
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
  float y0 = sB3[0], y1 = sB3[1];
  if (ok) {
    tc::tmem_ld64(t_z2 + lane_base, buf);
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      buf[o] = act_tanh(buf[o] + sB2[o]);  // h2
      y0 = fmaf(sW3[o], buf[o], y0);
      y1 = fmaf(sW3[kH + o], buf[o], y1);
    }
  }
  // loss and output gradient
  const float inv_b = 1.0f / static_cast<float>(batch);
  const float r0 = inb ? y0 - tf.x / sNorm[3] : 0.0f, r1 = inb ? y1 - tf.y / sNorm[3] : 0.0f;
  const float dy0 = 2.0f * r0 * inv_b, dy1 = 2.0f * r1 * inv_b;
  s_dy[tid][0] = dy0;
  s_dy[tid][1] = dy1;
  s_xh[tid][0] = xh0;
  s_xh[tid][1] = xh1;
  // dW3 = dy^T h2 by columns of the stage
#pragma unroll
  for (int o = 0; o < kH; ++o) stage[tid * kStage + o] = buf[o];
  __syncthreads();
  if (tid < kH) {
    float g0 = 0.0f, g1 = 0.0f;
    for (int r = 0; r < 128; ++r) {
      const float h2 = stage[r * kStage + tid];
      g0 = fmaf(s_dy[r][0], h2, g0);
      g1 = fmaf(s_dy[r][1], h2, g1);
    }
    part[kOW3 + tid] = g0;
    part[kOW3 + kH + tid] = g1;
  }
  __syncthreads();
  // dz2 = (W3^T dy) (1 - h2^2); db2 by columns; dz2 into the two A operands
  float dz2[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    dz2[o] = fmaf(sW3[o], dy0, sW3[kH + o] * dy1) * fmaf(-buf[o], buf[o], 1.0f);
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
    part[kOB2 + tid] = g;
  }
  {
    const float gb0 = block128_sum(dy0, s_red), gb1 = block128_sum(dy1, s_red);
    const float ls = block128_sum(r0 * r0 + r1 * r1, s_red);
    if (tid == 0) {
      part[kOB3] = gb0;
      part[kOB3 + 1] = gb1;
      part[kNP] = ls * inv_b;
    }
  }
  ok = ok && __syncthreads_and(tc::mbar_wait(&mbar, 1, kWaitIter));
  tc::fence_after_sync();
  if (ok) {
    tc::tmem_ld64(t_dh1 + lane_base, buf);
#pragma unroll
    for (int k = 0; k < kH; ++k) {  // dz1 = dh1 (1 - h1^2), h1 recomputed as in the forward pass
      const float h1 = act_tanh(layer1_z(sW1, sB1, k, xh0, xh1));
      stage[tid * kStage + k] = buf[k] * fmaf(-h1, h1, 1.0f);
    }
    if (warp < 2) {  // lanes 0..63 hold the 64 rows of dW2
      tc::tmem_ld64(t_dw2 + lane_base, buf);
      const int o = warp * 32 + lane;
#pragma unroll
      for (int in = 0; in < kH; ++in) part[kOW2 + o * kH + in] = buf[in];
    }
  }
  __syncthreads();
  if (ok && tid < kH) {
    float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
    for (int r = 0; r < 128; ++r) {
      const float d = stage[r * kStage + tid];
      g0 = fmaf(d, s_xh[r][0], g0);
      g1 = fmaf(d, s_xh[r][1], g1);
      gb += d;
    }
    part[kOW1 + 2 * tid] = g0;
    part[kOW1 + 2 * tid + 1] = g1;
    part[kOB1 + tid] = gb;
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
__global__ void k_sur_adam(SurArgs s, uint32_t nblocks, int it, int iters) {
  const int t = *s.adam_t + it + 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(t)), c2 = 1.0f - powf(b2, static_cast<float>(t));
  const float lr = s.lr * powf(0.01f, static_cast<float>(it) / static_cast<float>(iters > 1 ? iters - 1 : 1));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
    float g = 0.0f;
    for (uint32_t b = 0; b < nblocks; ++b) g += s.partial[static_cast<size_t>(b) * (kNP + 1) + i];
    const float m = b1 * s.mom1[i] + (1.0f - b1) * g;
    const float v = b2 * s.mom2[i] + (1.0f - b2) * g * g;
    s.mom1[i] = m;
    s.mom2[i] = v;
    const float th = s.theta[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    s.theta[i] = th;
    publish(s, i, th);
  }
}

__global__ void k_sur_adam_bump(SurArgs s, int iters) { *s.adam_t += iters; }

// Sampled query particles: id = floor(u N) from Philox (id = q, step m, stream 2).
__global__ void k_sur_sample(SurArgs s, StepParams<float> a) {
  const uint32_t m32 = step_index(a);
  for (uint32_t qi = blockIdx.x * blockDim.x + threadIdx.x; qi < s.nq; qi += gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(qi, m32, a.replica, 2u * 256u), a.seed);
    const uint32_t id = __umulhi(w.x, a.n);
    s.qidx[qi] = id;
    reinterpret_cast<float2*>(s.q)[qi] = reinterpret_cast<const float2*>(a.x)[id];
  }
}

// Input and output scales from the first checkpoint's queries (one block).
__global__ void k_sur_norm(SurArgs s) {
  __shared__ double red[4][32];
  double acc[4] = {0, 0, 0, 0};
  for (uint32_t i = threadIdx.x; i < s.nq; i += blockDim.x) {
    const float2 x = reinterpret_cast<const float2*>(s.q)[i];
    const float2 f = reinterpret_cast<const float2*>(s.fq)[i];
    acc[0] += x.x;
    acc[1] += x.y;
    acc[2] += static_cast<double>(x.x) * x.x + static_cast<double>(x.y) * x.y;
    acc[3] += static_cast<double>(f.x) * f.x + static_cast<double>(f.y) * f.y;
  }
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t[k] += red[k][w];
    const double n = s.nq;
    const double mx = t[0] / n, my = t[1] / n;
    const double var = fmax(t[2] / n - mx * mx - my * my, 0.0) / 2.0;
    const double fs = sqrt(t[3] / (2.0 * n));
    s.norm[0] = static_cast<float>(mx);
    s.norm[1] = static_cast<float>(my);
    s.norm[2] = static_cast<float>(var > 0 ? sqrt(var) : 1.0);
    s.norm[3] = static_cast<float>(fs > 0 ? fs : 1.0);
  }
}

// Relative error ||F_net - F||_2 / ||F||_2 over queries [lo, nq) (one
// block): the held-out quarter after training (drift = 0: also sets the
// selection flag), or every query of a fresh sample before training (drift =
// 1: the error of the network as it drove the interval just ended, into
// err[1]).
__global__ void k_sur_check(SurArgs s, int drift) {
  __shared__ double red[2][32];
  double e = 0, f = 0;
  const uint32_t lo = drift ? 0u : s.ntrain;
  for (uint32_t i = lo + threadIdx.x; i < s.nq; i += blockDim.x) {
    const float2 p = reinterpret_cast<const float2*>(s.fpred)[i];
    const float2 t = reinterpret_cast<const float2*>(s.fq)[i];
    const double dx = static_cast<double>(p.x) - t.x, dyv = static_cast<double>(p.y) - t.y;
    e += dx * dx + dyv * dyv;
    f += static_cast<double>(t.x) * t.x + static_cast<double>(t.y) * t.y;
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

int surrogate_param_count() { return kNP; }

cudaError_t prepare_surrogate_kernels() {
  return cudaFuncSetAttribute(k_sur_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kGradSmem));
}

cudaError_t sur_init(const SurrogateScratch& ss, int32_t* status, uint64_t seed, cudaStream_t st) {
  k_sur_init<<<18, 256, 0, st>>>(make_args(ss, status),
                                 make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
  return cudaGetLastError();
}

cudaError_t sur_publish(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  k_sur_publish<<<18, 256, 0, st>>>(make_args(ss, status));
  return cudaGetLastError();
}

cudaError_t sur_sample(const SurrogateScratch& ss, const void* params, cudaStream_t st) {
  const StepParams<float>& a = *static_cast<const StepParams<float>*>(params);
  k_sur_sample<<<(ss.nq + 255) / 256, 256, 0, st>>>(make_args(ss, a.status), a);
  return cudaGetLastError();
}

cudaError_t sur_norm(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  k_sur_norm<<<1, 1024, 0, st>>>(make_args(ss, status));
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
    k_sur_grad<<<nblocks, 128, kGradSmem, st>>>(s, xs, ts, ntrain, begin, batch);
    mark_launch(cfg, st, "k_sur_grad");
    k_sur_adam<<<18, 256, 0, st>>>(s, nblocks, it, iters);
    mark_launch(cfg, st, "k_sur_adam");
  }
  k_sur_adam_bump<<<1, 1, 0, st>>>(s, iters);
  return cudaGetLastError();
}

cudaError_t sur_gradient(const SurrogateScratch& ss, int32_t* status, const float* xs, const float* ts, uint32_t nb,
                         cudaStream_t st) {
  const uint32_t nblocks = (nb + 127) / 128;
  k_sur_grad<<<nblocks, 128, kGradSmem, st>>>(make_args(ss, status), xs, ts, nb, 0u, nb);
  return cudaGetLastError();
}

cudaError_t sur_forces(const SurrogateScratch& ss, int32_t* status, const float* q, uint32_t nq, float* fout,
                       const LaunchCfg& cfg, cudaStream_t st) {
  StepParams<float> a{};
  a.status = status;
  const uint32_t tiles = (nq + 127) / 128;
  const uint32_t grid = std::min<uint32_t>(tiles, static_cast<uint32_t>(cfg.num_sms) * 4u);
  k_sur_infer<1><<<std::max(grid, 1u), 128, 0, st>>>(make_args(ss, status), a, q, nq, fout);
  mark_launch(cfg, st, "k_sur_forces");
  return cudaGetLastError();
}

cudaError_t sur_check(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  k_sur_check<<<1, 1024, 0, st>>>(make_args(ss, status), 0);
  return cudaGetLastError();
}

cudaError_t sur_drift(const SurrogateScratch& ss, int32_t* status, cudaStream_t st) {
  k_sur_check<<<1, 1024, 0, st>>>(make_args(ss, status), 1);
  return cudaGetLastError();
}

cudaError_t sur_step(const SurrogateScratch& ss, const void* params, const LaunchCfg& cfg, cudaStream_t st) {
  const StepParams<float>& a = *static_cast<const StepParams<float>*>(params);
  const uint32_t tiles = (a.n + 127) / 128;
  const uint32_t grid = std::min<uint32_t>(tiles, static_cast<uint32_t>(cfg.num_sms) * 4u);
  k_sur_infer<0><<<std::max(grid, 1u), 128, 0, st>>>(make_args(ss, a.status), a, nullptr, 0u, nullptr);
  mark_launch(cfg, st, "k_sur_step");
  return cudaGetLastError();
}

}  // namespace rbm
