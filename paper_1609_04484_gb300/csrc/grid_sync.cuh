// Grid-wide barrier for persistent kernels launched cooperatively (every
// CTA resident). It spins with an iteration limit: on timeout it raises a
// sticky error flag, every CTA leaves at its next barrier, and the host
// reports the failure instead of hanging.
#pragma once

#include <cstdlib>

#include "internal.cuh"

namespace stokes {
namespace gsync {

constexpr long long kSpinLimit = 1ll << 24;  // polls of ~0.1-1 us: about 2-16 seconds

// The poll limit of every barrier launched from now on: kSpinLimit, or the
// value of the environment variable STOKES_WAIT_POLLS (read at each launch;
// a small value makes the waits give up at once, which the failure tests
// use to exercise the error path).
inline long long spin_limit() {
  const char* e = std::getenv("STOKES_WAIT_POLLS");
  if (!e || !*e) return kSpinLimit;
  const long long v = std::atoll(e);
  return v >= 0 ? v : kSpinLimit;
}

// count: arrivals since the launch began (zeroed before each launch);
// err: sticky timeout flag; limit: polls before a waiter gives up.
struct Barrier {
  unsigned* count;
  unsigned* gen;  // unused by this barrier; kept for the buffer layout
  int* err;
  long long limit;
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
      if (++spins > b.limit || *(volatile int*)b.err) {
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
