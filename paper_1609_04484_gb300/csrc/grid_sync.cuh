// Grid-wide barrier for persistent kernels launched cooperatively (every
// CTA resident). It spins with an iteration limit: on timeout it raises a
// sticky error flag, every CTA leaves at its next barrier, and the host
// reports the failure instead of hanging.
#pragma once

#include "internal.cuh"

namespace stokes {
namespace gsync {

constexpr long long kSpinLimit = 1ll << 24;  // polls of ~0.1-1 us: about 2-16 seconds

// count: arrivals since the launch began (zeroed before each launch);
// err: sticky timeout flag.
struct Barrier {
  unsigned* count;
  unsigned* gen;  // unused by this barrier; kept for the buffer layout
  int* err;
};

// Barrier number `epoch` (counted per CTA, 1, 2, ...) is complete once
// gridDim.x * epoch CTAs have arrived: arrivals only add to the counter, so
// no CTA waits on another's read-modify-write, and waiters poll it with
// short sleeps. Returns false if the barrier timed out (here or elsewhere).
__device__ __forceinline__ bool grid_sync(const Barrier& b, unsigned& epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    __threadfence();
    atomicAdd(b.count, 1u);
    const unsigned target = epoch * gridDim.x;
    volatile unsigned* vc = b.count;
    long long spins = 0;
    while (*vc < target) {
      if (++spins > kSpinLimit || *(volatile int*)b.err) {
        atomicExch(b.err, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)b.err == 0;
}

}  // namespace gsync
}  // namespace stokes
