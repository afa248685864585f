// Grid-wide barrier for cooperatively launched kernels (all blocks co-resident), with a bounded
// wait: a block that waits longer than the launch's limit (status[ST_SPIN] when the host set one,
// else kSpinLimit, ~2 s) sets status[ST_TIMEOUT] and an abort
// flag, and every block then leaves the kernel at its next barrier.  No wait is unbounded.
#pragma once
#include "common.cuh"

namespace gev {

struct GridBar {
  unsigned* count;  // arrivals in the current generation
  unsigned* gen;    // generation counter
  int* status;      // status words; ST_TIMEOUT receives the site code on timeout
  int* abort_flag;  // non-zero once any block gave up
};

// Returns false when the kernel must stop (a wait timed out somewhere).
__device__ __forceinline__ bool grid_sync(const GridBar& g, int site) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = g.gen;
    volatile int* vab = g.abort_flag;
    const unsigned my_gen = *vgen;
    __threadfence();
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned arrived = atomicAdd(g.count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(g.count, 0u);
      __threadfence();
      atomicAdd(g.gen, 1u);
    } else {
      const long long lim = spin_limit(g.status);
      long long it = 0;
      while (*vgen == my_gen) {
        if (*vab) { ok = 0; break; }
        if (++it > lim) {
          atomicCAS(&g.status[ST_TIMEOUT], 0, site);
          atomicExch(g.abort_flag, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*vab) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace gev
