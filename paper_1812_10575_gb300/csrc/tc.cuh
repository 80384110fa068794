// Blackwell (sm_103a) tensor-core building blocks, hand-written PTX:
// tensor-memory allocation, shared-memory matrix descriptors for BF16
// operands in the canonical no-swizzle K-major layout, tcgen05.mma with FP32
// accumulation in tensor memory, completion through an mbarrier, and loads of
// the accumulator back to registers.
//
// Operand layout (no swizzle, K-major): the matrix is tiled into core
// matrices of 8 rows x 16 bytes (8 bf16 along K), each stored as 128
// contiguous bytes, row r at byte 16 r.  Core matrix (i, j) (i along M/N, j
// along K) of an R x K operand sits at ((i * (K/8)) + j) * 128, so the
// leading-dimension byte offset (next core matrix along K) is 128 and the
// stride-dimension byte offset (next core matrix along M/N) is K/8 * 128.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace rbm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of an R x K K-major bf16 operand.
__device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t k, uint32_t K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// Shared-memory matrix descriptor: start address, LBO, SBO (bytes), the
// descriptor version of this architecture, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one K = 16 slice; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
  const uint32_t acc = accumulate ? 1u : 0u;
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc));
}

// D = A (R x K) * B^T where A is 128 x K, B is N x K, both K-major in shared
// memory at a_smem / b_smem (layouts as core_off with the given K).
__device__ __forceinline__ void gemm_128xN(uint32_t d_tmem, const void* a_smem, const void* b_smem, uint32_t N,
                                           uint32_t K, bool accumulate_first) {
  const uint32_t idesc = idesc_bf16_f32(128, N);
  const uint32_t sbo = (K >> 3) << 7;
  const uint32_t a0 = smem_u32(a_smem), b0 = smem_u32(b_smem);
  for (uint32_t kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = smem_desc(a0 + kk * 256, 128, sbo);
    const uint64_t bd = smem_desc(b0 + kk * 256, 128, sbo);
    mma_bf16(d_tmem, ad, bd, idesc, accumulate_first || kk > 0);
  }
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

// Bounded wait for the given phase parity of an mbarrier; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_iter) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < max_iter && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
  }
  return done != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor-memory allocation by one full warp; the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 64 consecutive FP32 columns of this thread's lane (warp w reads lanes
// 32w .. 32w+31; taddr must carry that lane base in bits 16..).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,"
      "%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 64; ++c) v[c] = __uint_as_float(r[c]);
}

// Eight bf16 values (one 16-byte core-matrix row segment) from floats.
__device__ __forceinline__ uint4 pack_bf16x8(const float* f) {
  uint4 u;
  u.x = (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(f[1]))) << 16) |
        __bfloat16_as_ushort(__float2bfloat16_rn(f[0]));
  u.y = (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(f[3]))) << 16) |
        __bfloat16_as_ushort(__float2bfloat16_rn(f[2]));
  u.z = (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(f[5]))) << 16) |
        __bfloat16_as_ushort(__float2bfloat16_rn(f[4]));
  u.w = (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(f[7]))) << 16) |
        __bfloat16_as_ushort(__float2bfloat16_rn(f[6]));
  return u;
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

}  // namespace tc
}  // namespace rbm
