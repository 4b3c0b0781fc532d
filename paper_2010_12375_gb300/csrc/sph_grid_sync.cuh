// Grid-wide barrier for cooperative launches (all blocks co-resident, which the runtime
// guarantees or refuses the launch). Thread 0 of each block publishes the block's writes
// (fence), arrives on the counter and waits, with a bounded spin, for the last block to
// advance the generation; the fence after the wait makes the other blocks' writes visible to
// this block's later (plain, coherent) loads. A wait that gives up sets ERR_TIMEOUT and
// returns false: the caller returns, and the other blocks then time out at their next
// barrier, so a launch always ends.
#pragma once
#include "sph_kernels.h"

namespace sph {

constexpr unsigned kBarrierSpinLimit = 1u << 24;   // polls of 64 ns sleeps: about a second

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, Global* g) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* genp = &bar->gen;
    const unsigned my = *genp;               // this barrier cannot complete before we arrive
    __threadfence();                         // release this block's writes
    if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned spins = 0;
      while (*genp == my) {
        if (++spins > kBarrierSpinLimit) {
          atomicOr(&g->err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();                         // acquire the other blocks' writes
  }
  __syncthreads();
  return ok != 0;
}


}  // namespace sph
