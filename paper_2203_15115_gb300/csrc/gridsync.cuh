// Grid-wide barrier for cooperatively launched kernels (every CTA of the
// grid co-resident).  Its waits are bounded: a wait that runs out sets an
// error flag that every CTA sees, and the kernel returns.
#pragma once

#include <cuda_runtime.h>

namespace afd {

// Grid barrier state: arrivals and the generation, zeroed before the launch.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;       // 1: a wait ran out
  int pad;
};

constexpr unsigned int GRID_WAIT_LIMIT = 1u << 24;   // polls of ~0.1 us: well over a second

// Barrier over all CTAs of a cooperative launch.  Returns false on every CTA
// once any CTA's wait has run out (the kernel then returns).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// *t_arrive (thread 0, when given): when this CTA reached the barrier.
__device__ __forceinline__ bool grid_barrier(GridBarrier* b, unsigned int& gen,
                                             unsigned long long* t_arrive = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (t_arrive) *t_arrive = global_ns();
    int ok = 1;
    const unsigned int target = gen + 1u;
    const unsigned int nblocks = gridDim.x;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == nblocks - 1u) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicExch(&b->gen, target);
    } else {
      volatile unsigned int* vg = &b->gen;
      volatile int* ve = &b->err;
      unsigned int polls = 0;
      while (*vg != target) {
        if (*ve || ++polls > GRID_WAIT_LIMIT) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    if (*(volatile int*)&b->err) ok = 0;
    gen = target;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace afd
