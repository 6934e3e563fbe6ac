// tsf_grid.cuh -- whole-GPU kernels: a grid barrier for cooperative
// launches and the launcher they go through.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tsf_internal.cuh"

namespace tsf {

// Grid barrier over the co-resident blocks of a cooperative launch.
// bar[0] counts arrivals, bar[1] is the generation (both start at 0).  A
// block that waits more than `limit` polls (~2^24 by default) sets kErrSpin
// and gets false; the
// caller then returns, so every block leaves at its next barrier and the
// kernel ends with the error bit set instead of hanging.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, uint32_t* status,
                                             unsigned limit = 1u << 24) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned it = 0;
      while (*vgen == gen) {
        if (++it > limit) {
          atomicOr(status, kErrSpin);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Launches a cooperative kernel on st and waits for it.  One such kernel
// runs at a time in the process (fields solved concurrently on other
// streams would otherwise hold parts of two grids resident, each waiting
// at its barrier for the other's blocks).  Returns the launch status.
cudaError_t cooperative_launch(const void* fn, dim3 grid, dim3 block, void** args, cudaStream_t st);

// Blocks for a whole-GPU kernel of `threads` threads per block: one per SM,
// on at most 128 SMs.
int cooperative_blocks(const void* fn, int threads);

}  // namespace tsf
