// rix_grid_noalloc: rix_grid without any device allocation at call time.
//
// Some callers cannot allocate device memory when they grid: a host loop
// with a latency budget that must not stall on the allocator (cudaMalloc and
// cudaFree can synchronise the whole device), a process in which another
// allocator (for example a framework's caching allocator) has already
// reserved nearly all of the GPU's memory so a new cudaMalloc would fail,
// or a host program that does not let a library own device allocations.
// This entry point grids into a scratch area that is part of the library
// image itself: a file-scope __device__ array of fixed size, which every GPU
// that loads the library holds from load until process exit.
#include <cuda_runtime.h>

#include <mutex>

#include "rix_internal.cuh"

namespace rix {
namespace {

constexpr size_t kNoAllocBytes = RIX_GRID_NOALLOC_MAX_BYTES;
constexpr size_t kNoAllocElems = kNoAllocBytes / sizeof(float2);

// The shared scratch.  In host code the name is only a host-side stand-in for
// the device symbol; its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) float2 g_grid_scratch[kNoAllocElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_addr[kMaxDevices] = {};

// Device address of the scratch on `device` (which must be current), looked
// up once per device and kept for the life of the process.  The cache
// assumes the device's primary context lives as long as the process: after a
// cudaDeviceReset the cached address is stale, so a process that resets a
// device must not call rix_grid_noalloc on it again.
int scratch_address(int device, float2** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(RIX_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
    if (e != cudaSuccess)
      return set_error(RIX_ECUDA, "cudaGetSymbolAddress(grid scratch): %s", cudaGetErrorString(e));
    g_addr[device] = static_cast<float2*>(p);
  }
  *out = g_addr[device];
  return RIX_OK;
}

}  // namespace
}  // namespace rix

extern "C" int rix_grid_noalloc(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream);

// rix_job_s is defined in rix_api.cu; this file reaches the job through the
// accessor below, also defined there.
namespace rix {
Job* job_of(rix_job_t job);
}

namespace {
int grid_noalloc_impl(rix::Job* J, int part, const void* vis, void* image_out, cudaStream_t st) {
  using namespace rix;
  if (!J->partitioned) return set_error(RIX_ESTATE, "rix_set_uv_partition has not been called");
  if (part < 0 || part >= J->n_part) return set_error(RIX_EINVAL, "partition %d out of range", part);
  if (J->fp64) return set_error(RIX_EINVAL, "rix_grid_noalloc supports FP32 jobs only");
  if (!vis || !image_out) return set_error(RIX_EINVAL, "NULL vis or image_out");
  float2* scratch = nullptr;
  RIX_TRY(scratch_address(J->ctx->device, &scratch));
  RIX_TRY(op_grid_into_scratch(J, part, static_cast<const float2*>(vis), static_cast<float*>(image_out), scratch,
                               kNoAllocElems, st));
  // rix_job_destroy waits for the streams the job's calls ran on
  return note_stream(J, st);
}
}  // namespace

extern "C" int rix_grid_noalloc(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream) {
  using namespace rix;
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job* J = job_of(job);
  // run on the job's device and give the caller back the device it had current
  int prev = -1;
  RIX_CUDA(cudaGetDevice(&prev));
  if (prev != J->ctx->device) RIX_CUDA(cudaSetDevice(J->ctx->device));
  const int rc = grid_noalloc_impl(J, part, vis, image_out, (cudaStream_t)stream);
  if (prev != J->ctx->device) {
    const cudaError_t e = cudaSetDevice(prev);
    if (rc == RIX_OK && e != cudaSuccess) return set_error(RIX_ECUDA, "restoring device %d: %s", prev, cudaGetErrorString(e));
  }
  return rc;
}
