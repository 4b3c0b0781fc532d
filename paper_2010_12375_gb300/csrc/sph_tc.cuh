// Fifth-generation tensor-core building blocks (tcgen05) for the dense layers of the learned
// stand-in: one warpgroup (128 threads) per CTA multiplies a 128-row tile A [128 x K] by a
// weight matrix B [N x K]^T, both bf16 in shared memory, into FP32 accumulators in tensor
// memory (TMEM): TMEM lane r holds row r, column c output c.
//
// Operand layout in shared memory (no swizzle, K-major): the canonical core-matrix layout,
// 8 rows x 16 bytes per core matrix, core matrices stacked R/8 deep along the rows and then
// K/8 along K. Element (row, k) of an R-row operand sits at byte
//   ((k / 8) * (R / 8) + row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2.
// One MMA instruction covers K = 16 (two core matrices along K, leading-dimension offset
// (R / 8) * 128 bytes between them; stride-dimension offset 128 bytes between 8-row groups).
//
// Synchronisation: threads write operands with ordinary stores, then fence.proxy.async and
// a CTA barrier hand them to the tensor core; one thread issues the MMAs and commits them to
// an mbarrier; every thread waits on that mbarrier with a bounded spin (a wait that runs out
// sets the caller's error flag and the CTA skips the tile's results) before reading TMEM.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace sph {
namespace tc {

constexpr unsigned kWaitLimit = 1u << 24;   // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of an R-row operand in the core-matrix layout
__device__ __forceinline__ int core_offset(int R, int row, int k) {
  return ((k >> 3) * (R >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, leading- and stride-dimension byte
// offsets (each stored >> 4 in 14 bits), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 for M = 128, N outputs: FP32 accumulators, bf16 A and
// B, both K-major, dense.
template <int N>
__host__ __device__ constexpr uint32_t instr_desc() {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "M = 128 needs N a multiple of 16 in [16, 256]");
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// TMEM columns for N accumulators: a power of two, at least 32
__host__ __device__ constexpr int tmem_cols(int N) { return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256; }

// Allocation by warp 0 (all its lanes); the base address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t base, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(cols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// ordinary shared-memory stores made visible to the tensor core
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// D[tmem_d] (+)= A[128 x K] B[N x K]^T, issued by one thread; A and B in the core-matrix
// layout at shared addresses a and b; then the MMAs are committed to bar.
template <int N>
__device__ __forceinline__ void mma_tile(uint32_t tmem_d, uint32_t a, uint32_t b, int K, bool accumulate,
                                         uint64_t* bar) {
  constexpr uint32_t idesc = instr_desc<N>();
  for (int j = 0; j < K / 16; ++j) {
    const uint64_t da = smem_desc(a + j * 2 * 16 * 128, 16 * 128, 128);
    const uint64_t db = smem_desc(b + j * 2 * (N / 8) * 128, (N / 8) * 128, 128);
    const uint32_t acc = (accumulate || j > 0) ? 1u : 0u;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// Bounded wait for the current phase of bar; true when it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (unsigned spin = 0; spin < kWaitLimit && !done; ++spin)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
  return done != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w of the warpgroup reads lanes
// 32 w .. 32 w + 31; thread = lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// TMEM address of column c of warp w's lanes
__device__ __forceinline__ uint32_t tmem_addr(uint32_t base, int warp, int c) {
  return base + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
}

}  // namespace tc
}  // namespace sph
