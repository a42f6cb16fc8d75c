// Grid-wide barrier with a bounded wait, for kernels launched with
// cudaLaunchCooperativeKernel (every CTA resident at once).
//
// The arrival counter only grows during a launch: barrier k completes when it
// reaches (k + 1) * gridDim.x.  The host zeroes it, stream-ordered, before each
// launch.  Arrival is a release add at GPU scope after a CTA barrier and a
// fence; the wait is an acquire load at GPU scope followed by a fence and a
// CTA barrier, so every write of every CTA before the barrier is visible to
// every thread after it.
//
// The wait ends after kBarrierTimeoutNs of global time or kBarrierMaxSpins
// polls, whichever comes first.  The CTA that gives up stores RIX_ETIMEOUT in
// the job's status word and the barrier returns false; a CTA that sees a
// non-zero status while waiting gives up at once.  Callers return on false.
#pragma once

#include <cuda_runtime.h>

#include "../../include/rix.h"

namespace rix {

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s
constexpr unsigned int kBarrierMaxSpins = 1u << 26;

struct GridBarrier {
  unsigned int* count;   // zeroed before the launch
  int* status;           // the job's device status word (0 = fine)
  unsigned int target;   // per-CTA copy: arrivals the next barrier waits for
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_barrier(GridBarrier& b) {
  __shared__ int ok;
  __syncthreads();
  b.target += gridDim.x;
  if (threadIdx.x == 0) {
    int good = 1;
    __threadfence();
    red_release_gpu_add(b.count, 1u);
    const unsigned long long t0 = global_ns();
    unsigned int spins = 0;
    while (ld_acquire_gpu(b.count) < b.target) {
      if ((++spins & 63u) == 0) {
        if (*reinterpret_cast<volatile int*>(b.status) != 0) { good = 0; break; }
        if (spins >= kBarrierMaxSpins || global_ns() - t0 > kBarrierTimeoutNs) {
          atomicCAS(b.status, 0, RIX_ETIMEOUT);
          good = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace rix
