// tc.cuh -- fifth-generation tensor-core primitives (tcgen05, sm_100a
// family) as inline PTX: tensor-memory allocation, single-thread MMA issue
// with shared-memory matrix descriptors, completion through an mbarrier,
// and tensor-memory loads for the epilogue.
//
// Operands use the canonical K-major layout without swizzling: a matrix of
// R rows (M or N) and K columns is a grid of core matrices of 8 rows x 16
// bytes (8 x 4 FP32/TF32 values) stored row after row (16 bytes per row,
// 128 bytes per core matrix); the core matrix at (row group r/8, column
// group q/4) starts at (r/8) * SBO + (q/4) * LBO, so LBO is the byte step
// between core matrices along K and SBO the step between 8-row groups.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ibm {

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units, the fixed descriptor version bit (46), no swizzle, base offset 0.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands
// K-major, dense: D format F32 (bits 4-5 = 1), A and B format TF32 (bits
// 7-9 and 10-12 = 2), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory allocation by one full warp; the base address is written to
// shared memory.  ncols: a power of two in [32, 512].
__device__ __forceinline__ void tc_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem))),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tensor-core operations around thread synchronisation.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tensor memory) = A * B^T (+ D if accumulate), issued by one thread.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far by this thread
// has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(bar)))
               : "memory");
}

// Warp-wide loads of 4 / 8 consecutive 32-bit columns of the calling
// thread's tensor-memory lane (shape 32x32b: thread t of the warp reads lane
// base + t).  taddr: lane in bits 31-16, column in bits 15-0; a warp may
// only address the 32-lane quarter (warp id % 4) of tensor memory.
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float *v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// Wait until this thread's tensor-memory loads have landed in registers.
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x ~ hi + lo with hi = x rounded to TF32 (nearest, ties away; |x - hi| <=
// 2^-11 |x|) and lo = (x - hi) rounded to TF32 as well, so the tensor core
// takes both exactly instead of truncating the low bits of lo (an unbiased
// error <= 2^-22 |x|).  The products hi*hi' + hi*lo' + lo*hi' of two split
// operands then carry about 22 bits (the dropped lo*lo' term is <= 2^-22).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}

}  // namespace ibm
