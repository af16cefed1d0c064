// Grid-wide barrier for persistent kernels launched cooperatively (every
// CTA resident). It spins on a generation counter with an iteration limit:
// on timeout it raises a sticky error flag, every CTA leaves at its next
// barrier, and the host reports the failure instead of hanging.
#pragma once

#include "internal.cuh"

namespace stokes {
namespace gsync {

constexpr long long kSpinLimit = 1ll << 22;  // x ~256 ns sleep: about one second

struct Barrier {
  unsigned* count;
  unsigned* gen;
  int* err;
};

// Returns false if the barrier timed out (here or in another CTA).
__device__ __forceinline__ bool grid_sync(const Barrier& b) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = b.gen;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(b.count, 1u) + 1u;
    if (arrived == gridDim.x) {
      *b.count = 0u;
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g0) {
        if (++spins > kSpinLimit || *(volatile int*)b.err) {
          atomicExch(b.err, 1);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)b.err == 0;
}

}  // namespace gsync
}  // namespace stokes
