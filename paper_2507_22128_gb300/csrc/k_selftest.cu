// Self-test of the failure-detection path: a cooperative kernel whose first
// CTA never arrives at the bounded grid barrier, so the other CTAs' wait runs
// out and reports RIX_ETIMEOUT through a status word instead of hanging.
#include <cuda_runtime.h>

#include "grid_sync.cuh"
#include "rix_internal.cuh"

namespace rix {
namespace {

__global__ void k_missing_arrival(unsigned int* count, int* status, int* gave_up) {
  GridBarrier bar{count, status, 0u};
  if (blockIdx.x == 0) return;     // never arrives
  if (!grid_barrier(bar) && threadIdx.x == 0) atomicAdd(gave_up, 1);
}

}  // namespace

int selftest_barrier(Ctx* ctx, int* status_out, int* gave_up_out) {
  cudaStream_t st = ctx->mem_stream;
  int* words = nullptr;            // [0] arrival counter, [1] status, [2] CTAs that gave up
  RIX_CUDA(::rix::malloc_async((void**)&words, 4 * sizeof(int), st));
  int rc = RIX_OK;
  if (cudaMemsetAsync(words, 0, 4 * sizeof(int), st) != cudaSuccess) rc = set_error(RIX_ECUDA, "memset");
  if (rc == RIX_OK) {
    unsigned int* count = reinterpret_cast<unsigned int*>(words);
    int* status = words + 1;
    int* gave_up = words + 2;
    void* args[] = {&count, &status, &gave_up};
    note_launch();
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_missing_arrival, dim3(ctx->num_sms), dim3(32),
                                                      args, 0, st);
    if (e != cudaSuccess) rc = set_error(RIX_ECUDA, "self-test launch: %s", cudaGetErrorString(e));
  }
  int host[4] = {0, 0, 0, 0};
  if (rc == RIX_OK && cudaMemcpyAsync(host, words, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = set_error(RIX_ECUDA, "read-back");
  cudaFreeAsync(words, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == RIX_OK) rc = set_error(RIX_ECUDA, "self-test sync");
  if (rc == RIX_OK) {
    *status_out = host[1];
    *gave_up_out = host[2];
  }
  return rc;
}

}  // namespace rix
