// The C ABI of include/rix.h: argument checks, job state, call ordering and
// dispatch to the FP32 / FP64 device paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "rix_internal.cuh"

struct rix_ctx_s {
  rix::Ctx c;
};
struct rix_job_s {
  rix::Job j;
};
struct rix_batch_s {
  rix::Batch b;
};

namespace rix {

static thread_local char g_err[1024] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

const char* last_error() { return g_err; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

// Device memory comes from one stream-ordered pool per device that the
// library owns: it keeps up to kPoolKeep bytes of freed memory reserved
// across synchronisations, so that the temporaries of the next calls (the
// PSF's regrouping, the partition's sort) reuse them instead of mapping new
// memory; the device's default pool (release threshold 0) would return them
// to the system at every synchronisation.  The pools live until the process
// exits.
constexpr uint64_t kPoolKeep = 8ull << 30;
constexpr int kMaxDevices = 64;
static cudaMemPool_t g_pool[kMaxDevices] = {};
static std::mutex g_pool_mu;

static cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kPoolKeep;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

static std::atomic<unsigned long long> g_allocs{0};
cudaError_t malloc_async(void** p, size_t bytes, cudaStream_t st) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  cudaMemPool_t pool = device_pool();
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

// ---- opt-in kernel timing ----
static std::atomic<bool> g_timing{false};
static std::mutex g_tmu;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_tev[kTimeClasses];
static cudaEvent_t g_topen[kTimeClasses] = {};
bool timing_on() { return g_timing.load(std::memory_order_relaxed); }

void timing_mark(int cls, cudaStream_t st, bool begin) {
  if (!timing_on()) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, st);
  if (begin) {
    g_topen[cls] = e;
  } else if (g_topen[cls]) {
    g_tev[cls].push_back({g_topen[cls], e});
    g_topen[cls] = nullptr;
  } else {
    cudaEventDestroy(e);
  }
}

// Buffers come from the stream-ordered pool on the context's private stream:
// allocation waits for that stream only, and release (cudaFreeAsync) never
// synchronises the device, so tearing down one job does not stall others.
int DevBuf::alloc(Ctx* ctx, size_t nbytes) {
  if (nbytes == 0) nbytes = 16;
  if (p && bytes >= nbytes) return RIX_OK;   // reuse: re-partitioning a job keeps its buffers
  release();
  void* q = nullptr;
  cudaError_t e = ::rix::malloc_async(&q, nbytes, ctx->mem_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->mem_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(RIX_ENOMEM, "device allocation of %zu bytes: %s", nbytes, cudaGetErrorString(e));
  }
  p = q;
  bytes = nbytes;
  owner = ctx;
  return RIX_OK;
}

void DevBuf::release() {
  if (p) cudaFreeAsync(p, owner->mem_stream);
  p = nullptr;
  bytes = 0;
}

int check_status(Job* job) {
  int st = 0;
  RIX_CUDA(cudaMemcpyAsync(&st, job->status.p, sizeof(int), cudaMemcpyDeviceToHost, job->ctx->mem_stream));
  RIX_CUDA(cudaStreamSynchronize(job->ctx->mem_stream));
  if (st == RIX_ETIMEOUT) return set_error(RIX_ETIMEOUT, "a grid barrier of a cooperative kernel timed out");
  if (st != 0) return set_error(st, "device-side error %d", st);
  return RIX_OK;
}

int note_stream(Job* job, cudaStream_t st) {
  for (auto& pr : job->touched)
    if (pr.first == st) {
      RIX_CUDA(cudaEventRecord(pr.second, st));
      return RIX_OK;
    }
  cudaEvent_t ev;
  RIX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  job->touched.push_back({st, ev});
  RIX_CUDA(cudaEventRecord(ev, st));
  return RIX_OK;
}

// upper bound of resident device bytes of a job (admission control)
static size_t workspace_bytes(const rix_job_desc& d, int64_t nrow) {
  const size_t real = d.precision == RIX_FP64 ? 8 : 4;
  const size_t cplx = 2 * real;
  const size_t n = (size_t)d.n, ng = 2 * n;
  const size_t np = d.n_wplanes > 0 ? (size_t)d.n_wplanes : 1;
  const size_t P = (size_t)d.n_part;
  const size_t ns = (size_t)nrow * (size_t)d.nchan;
  size_t b = 0;
  b += (size_t)nrow * 24 + ns * 4;                 // uvw, weights
  b += ns * std::min<size_t>(P, 2) * 8;            // sorted keys and samples (overlap counted twice)
  b += ns * std::min<size_t>(P, 2) * 4 * real;     // per-entry kernel geometry
  b += ns / 512 * 4 + 64;                          // work items
  b += n * n * (real + 8) + 4 * n * n * (real + 8); // corrections + n-1 tables (image and PSF)
  if (d.n_wplanes > 0) b += np * n * n * cplx;     // corr x phase screens of the image grid's planes
  b += P * 4 * n * n * real;                       // Gamma filters
  b += 3 * 4 * n * n * cplx + 2 * n * n * real;    // fill scratch
  // per partition: planes (windows are at most the full grid), transpose buffer,
  // images, PSF and its spectrum, minor-cycle state
  const size_t per = 2 * np * ng * ng * cplx + np * ng * n * cplx + (6 + P) * n * n * real +
                     4 * n * n * real + 4 * n * n * cplx + 10 * n * n * real;
  b += P * per;
  return b;
}

static int check_desc(const rix_job_desc* d) {
  if (!d) return set_error(RIX_EINVAL, "desc is NULL");
  if (d->n < 32 || d->n > 4096 || (d->n & (d->n - 1))) return set_error(RIX_EINVAL, "n must be a power of two in [32, 4096]");
  if (!(d->cell_rad > 0.0) || d->cell_rad * d->n >= 1.0) return set_error(RIX_EINVAL, "cell_rad out of range");
  if (d->n_wplanes != 0 && (d->n_wplanes < kW + 1 || d->n_wplanes > 64))
    return set_error(RIX_EINVAL, "n_wplanes must be 0 or in [%d, 64]", kW + 1);
  if (d->nchan < 1 || d->nchan > 65536 || !d->freq_hz) return set_error(RIX_EINVAL, "bad channels");
  for (int c = 0; c < d->nchan; ++c)
    if (!(d->freq_hz[c] > 0.0)) return set_error(RIX_EINVAL, "frequencies must be positive");
  if (d->precision != RIX_FP32 && d->precision != RIX_FP64) return set_error(RIX_EINVAL, "bad precision");
  if (d->n_part < 1 || d->n_part > kMaxPart) return set_error(RIX_EINVAL, "n_part must be in [1, %d]", kMaxPart);
  if (d->tile != 0 && d->tile != 16 && d->tile != 32) return set_error(RIX_EINVAL, "tile must be 16 or 32");
  if (d->tile == 32 && d->n_wplanes > 0) return set_error(RIX_EINVAL, "tile 32 needs a coplanar job (shared memory)");
  if (d->precision == RIX_FP64 && d->n > 2048) return set_error(RIX_EINVAL, "FP64 jobs support n <= 2048");
  if (d->weighting != RIX_WEIGHT_NATURAL && d->weighting != RIX_WEIGHT_UNIFORM)
    return set_error(RIX_EINVAL, "weighting must be RIX_WEIGHT_NATURAL or RIX_WEIGHT_UNIFORM");
  if (d->exchange != RIX_EXCHANGE_IMAGE && d->exchange != RIX_EXCHANGE_SPECTRAL)
    return set_error(RIX_EINVAL, "exchange must be RIX_EXCHANGE_IMAGE or RIX_EXCHANGE_SPECTRAL");
  return RIX_OK;
}

static int check_part(Job* job, int part) {
  if (!job->partitioned) return set_error(RIX_ESTATE, "rix_set_uv_partition has not been called");
  if (part < 0 || part >= job->n_part) return set_error(RIX_EINVAL, "partition %d out of range", part);
  return RIX_OK;
}

static int ensure_images(Job* job, Part& pt, cudaStream_t st) {
  const size_t img = (size_t)job->desc.n * job->desc.n * (job->fp64 ? 8 : 4);
  RIX_TRY(pt.model.alloc(job->ctx, img));
  RIX_CUDA(cudaMemsetAsync(pt.model.p, 0, img, st));
  RIX_TRY(pt.resid.alloc(job->ctx, img));
  RIX_TRY(pt.delta.alloc(job->ctx, img));
  return RIX_OK;
}

// a new partitioning restarts every partition at cycle 0 (buffers are kept)
static void reset_partitions(Job* job) {
  for (int p = 0; p < kMaxPart; ++p) {
    Part& pt = job->part[p];
    pt.cycle = 0;
    pt.minor_done = 0;
    pt.psf_ready = false;
    pt.lambda_set = false;
    pt.ms_ncomp_cap = 0;
    pt.ms_p_cycle = 0;
  }
}

Job* job_of(rix_job_t job) { return &job->j; }

}  // namespace rix

using namespace rix;

// ------------------------------------------------------------------------
extern "C" {

const char* rix_last_error(void) { return rix::last_error(); }

uint64_t rix_kernel_launches(void) { return rix::g_launches.load(); }

uint64_t rix_device_allocations(void) { return rix::g_allocs.load(); }

int rix_timing_enable(int on) {
  rix::g_timing.store(on != 0);
  return RIX_OK;
}

int rix_timing_read(int kernel_class, double* total_ms, double* busy_ms, int64_t* launches) {
  if (kernel_class < 0 || kernel_class >= rix::kTimeClasses || !total_ms || !busy_ms || !launches)
    return set_error(RIX_EINVAL, "bad timing query");
  std::lock_guard<std::mutex> lk(rix::g_tmu);
  auto& ev = rix::g_tev[kernel_class];
  double tot = 0.0;
  std::vector<std::pair<double, double>> iv;   // intervals relative to the first start
  for (auto& pr : ev) {
    float ms = 0.f, a = 0.f, b = 0.f;
    if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess &&
        cudaEventElapsedTime(&a, ev[0].first, pr.first) == cudaSuccess &&
        cudaEventElapsedTime(&b, ev[0].first, pr.second) == cudaSuccess) {
      tot += ms;
      iv.push_back({a, b});
    }
  }
  // union of the intervals: device time during which any launch of the class ran
  std::sort(iv.begin(), iv.end());
  double busy = 0.0, cs = 0.0, ce = -1e300;
  for (auto& x : iv) {
    if (x.first > ce) {
      if (ce > cs) busy += ce - cs;
      cs = x.first;
      ce = x.second;
    } else {
      ce = std::max(ce, x.second);
    }
  }
  if (ce > cs) busy += ce - cs;
  for (auto& pr : ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  *launches = (int64_t)iv.size();
  ev.clear();
  *total_ms = tot;
  *busy_ms = busy;
  return RIX_OK;
}

int rix_create(rix_ctx_t* ctx, int device, size_t mem_budget_bytes) {
  if (!ctx) return set_error(RIX_EINVAL, "ctx is NULL");
  *ctx = nullptr;
  int ndev = 0;
  RIX_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(RIX_EINVAL, "device %d out of range (%d devices)", device, ndev);
  RIX_CUDA(cudaSetDevice(device));
  rix_ctx_s* c = new (std::nothrow) rix_ctx_s();
  if (!c) return set_error(RIX_ENOMEM, "host allocation");
  c->c.device = device;
  c->c.budget = mem_budget_bytes;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete c;
    return set_error(RIX_ECUDA, "cudaGetDeviceProperties");
  }
  c->c.num_sms = prop.multiProcessorCount;
  if (cudaStreamCreateWithFlags(&c->c.mem_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return set_error(RIX_ECUDA, "stream creation");
  }
  int rc = fft_init_twiddles(&c->c);
  if (rc != RIX_OK) {
    delete c;
    return rc;
  }
  *ctx = c;
  return RIX_OK;
}

int rix_destroy(rix_ctx_t ctx) {
  if (!ctx) return RIX_OK;
  if (ctx->c.jobs > 0) return set_error(RIX_EBUSY, "context still owns %d jobs", ctx->c.jobs);
  cudaSetDevice(ctx->c.device);
  ctx->c.tw32.release();
  ctx->c.tw64.release();
  cudaStreamSynchronize(ctx->c.mem_stream);
  cudaStreamDestroy(ctx->c.mem_stream);
  delete ctx;
  return RIX_OK;
}

size_t rix_job_workspace_bytes(const rix_job_desc* desc, int64_t nrow) {
  if (check_desc(desc) != RIX_OK || nrow < 0) return 0;
  return workspace_bytes(*desc, nrow);
}

int rix_job_create(rix_ctx_t ctx, const rix_job_desc* desc, int64_t max_rows, rix_job_t* job) {
  if (!ctx || !job) return set_error(RIX_EINVAL, "NULL argument");
  *job = nullptr;
  RIX_TRY(check_desc(desc));
  if (max_rows < 0 || max_rows * (int64_t)desc->nchan > (int64_t)0x7fffffff)
    return set_error(RIX_EINVAL, "max_rows out of range");
  const size_t need = workspace_bytes(*desc, max_rows);
  if (ctx->c.budget && ctx->c.reserved + need > ctx->c.budget)
    return set_error(RIX_ENOMEM, "memory budget: %zu reserved + %zu needed > %zu", ctx->c.reserved, need, ctx->c.budget);
  RIX_CUDA(cudaSetDevice(ctx->c.device));
  rix_job_s* js = new (std::nothrow) rix_job_s();
  if (!js) return set_error(RIX_ENOMEM, "host allocation");
  Job& J = js->j;
  J.ctx = &ctx->c;
  J.desc = *desc;
  J.freq.assign(desc->freq_hz, desc->freq_hz + desc->nchan);
  J.desc.freq_hz = J.freq.data();
  J.inv_lambda_h.resize(desc->nchan);
  for (int c = 0; c < desc->nchan; ++c) J.inv_lambda_h[c] = J.freq[c] / kC;
  J.max_rows = max_rows;
  J.ng = 2 * desc->n;
  J.tile = desc->tile ? desc->tile : 16;
  J.nw = desc->n_wplanes;
  J.ww = desc->n_wplanes > 0 ? kW : 1;
  J.fp64 = desc->precision == RIX_FP64;
  J.n_part = desc->n_part;
  int rc = J.inv_lambda.alloc(J.ctx, desc->nchan * sizeof(double));
  if (rc == RIX_OK) rc = J.status.alloc(J.ctx, sizeof(int));
  if (rc == RIX_OK && cudaMemset(J.status.p, 0, sizeof(int)) != cudaSuccess) rc = set_error(RIX_ECUDA, "status word");
  if (rc == RIX_OK && cudaMemcpy(J.inv_lambda.p, J.inv_lambda_h.data(), desc->nchan * sizeof(double),
                                 cudaMemcpyHostToDevice) != cudaSuccess)
    rc = set_error(RIX_ECUDA, "frequency upload");
  for (int p = 0; rc == RIX_OK && p < kMaxPart; ++p)
    if (cudaEventCreateWithFlags(&J.part[p].ev_minor[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&J.part[p].ev_minor[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&J.part[p].ev_psf, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&J.part[p].ev_major, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&J.part[p].ev_prep, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&J.part[p].ev_done, cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(RIX_ECUDA, "event creation");
  if (rc == RIX_OK && cudaEventCreateWithFlags(&J.ev_batch, cudaEventDisableTiming) != cudaSuccess)
    rc = set_error(RIX_ECUDA, "event creation");
  if (rc != RIX_OK) {
    delete js;
    return rc;
  }
  J.reserved = need;
  ctx->c.reserved += need;
  ctx->c.jobs += 1;
  *job = js;
  return RIX_OK;
}

int rix_job_destroy(rix_job_t job) {
  if (!job) return RIX_OK;
  Job& J = job->j;
  cudaSetDevice(J.ctx->device);
  // wait for this job's own work only (other jobs keep running); an error of
  // the wait (an event last recorded in a stream capture) is not left behind
  // for the next call's launch checks
  for (auto& pr : J.touched) {
    if (cudaEventSynchronize(pr.second) != cudaSuccess) cudaGetLastError();
    cudaEventDestroy(pr.second);
  }
  J.touched.clear();
  for (int p = 0; p < kMaxPart; ++p) {
    for (int k = 0; k < 2; ++k)
      if (J.part[p].ev_minor[k]) cudaEventDestroy(J.part[p].ev_minor[k]);
    if (J.part[p].ev_psf) cudaEventDestroy(J.part[p].ev_psf);
    if (J.part[p].ev_major) cudaEventDestroy(J.part[p].ev_major);
    if (J.part[p].ev_prep) cudaEventDestroy(J.part[p].ev_prep);
    if (J.part[p].ev_done) cudaEventDestroy(J.part[p].ev_done);
    if (J.part[p].own_stream) {
      cudaStreamSynchronize(J.part[p].own_stream);
      cudaStreamDestroy(J.part[p].own_stream);
    }
  }
  if (J.ev_batch) cudaEventDestroy(J.ev_batch);
  J.ctx->reserved -= J.reserved;
  J.ctx->jobs -= 1;
  delete job;
  return RIX_OK;
}

int rix_job_sync(rix_job_t job) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  RIX_CUDA(cudaSetDevice(job->j.ctx->device));
  for (auto& pr : job->j.touched) RIX_CUDA(cudaEventSynchronize(pr.second));
  RIX_CUDA(cudaGetLastError());
  return check_status(&job->j);
}

int rix_selftest_barrier_timeout(rix_ctx_t ctx, int* status_out, int* gave_up_out) {
  if (!ctx || !status_out || !gave_up_out) return set_error(RIX_EINVAL, "NULL argument");
  RIX_CUDA(cudaSetDevice(ctx->c.device));
  return selftest_barrier(&ctx->c, status_out, gave_up_out);
}

int rix_job_get_stats(rix_job_t job, rix_job_stats* out) {
  if (!job || !out) return set_error(RIX_EINVAL, "NULL argument");
  *out = job->j.stats;
  for (int p = 0; p < kMaxPart; ++p) out->cycle[p] = job->j.part[p].cycle;
  return RIX_OK;
}

static int rix_set_uv_partition_impl(rix_job_t job, const double* uvw_m, int64_t nrow, const float* weight,
                         const double* ell_px, double delta_px, uint8_t* mask_out, rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  cudaStream_t st = (cudaStream_t)stream;
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  J.partitioned = false;
  reset_partitions(&J);
  timing_mark(kTimePartition, st, true);
  RIX_TRY(partition_job(&J, uvw_m, nrow, weight, ell_px, delta_px, mask_out, st));
  if (J.fp64) RIX_TRY(grid_build_corrections<double>(&J, st));
  else RIX_TRY(grid_build_corrections<float>(&J, st));
  if (J.fp64) RIX_TRY(grid_entry_geometry<double>(&J, st));
  else RIX_TRY(grid_entry_geometry<float>(&J, st));
  if (J.fp64) RIX_TRY(grid_work_order<double>(&J, st));
  else RIX_TRY(grid_work_order<float>(&J, st));
  if (J.fp64) RIX_TRY(fill_init<double>(&J, st));
  else RIX_TRY(fill_init<float>(&J, st));
  for (int p = 0; p < J.n_part; ++p) RIX_TRY(ensure_images(&J, J.part[p], st));
  timing_mark(kTimePartition, st, false);
  J.partitioned = true;
  return RIX_OK;
}

static int rix_get_sorted_entries_impl(rix_job_t job, uint32_t* keys_out, uint32_t* samples_out, rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  if (!J.partitioned) return set_error(RIX_ESTATE, "not partitioned");
  cudaStream_t st = (cudaStream_t)stream;
  if (J.n_entries == 0) return RIX_OK;
  if (keys_out) RIX_CUDA(cudaMemcpyAsync(keys_out, J.keys.p, J.n_entries * 4, cudaMemcpyDeviceToDevice, st));
  if (samples_out) RIX_CUDA(cudaMemcpyAsync(samples_out, J.samples.p, J.n_entries * 4, cudaMemcpyDeviceToDevice, st));
  return RIX_OK;
}

__global__ void k_fill_ones(float* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0f;
}

static int rix_get_weights_impl(rix_job_t job, float* weight_out, rix_stream_t stream) {
  if (!job || !weight_out) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  if (!J.partitioned) return set_error(RIX_ESTATE, "not partitioned");
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ns = J.stats.n_samples;
  if (ns == 0) return RIX_OK;
  if (J.weight.p) {
    RIX_CUDA(cudaMemcpyAsync(weight_out, J.weight.p, ns * sizeof(float), cudaMemcpyDeviceToDevice, st));
  } else {
    note_launch();
    k_fill_ones<<<(unsigned)std::min<int64_t>(ceil_div(ns, 256), (int64_t)J.ctx->num_sms * 8), 256, 0, st>>>(weight_out, ns);
    RIX_CUDA(cudaGetLastError());
  }
  return RIX_OK;
}

static int rix_degrid_impl(rix_job_t job, int part, const void* image, void* vis_out, rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  if (!image || !vis_out) return set_error(RIX_EINVAL, "NULL image or vis_out");
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (J.fp64) return op_degrid<double>(&J, part, (const double*)image, (double2*)vis_out, st);
  return op_degrid<float>(&J, part, (const float*)image, (float2*)vis_out, st);
}

static int rix_grid_impl(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  if (!vis || !image_out) return set_error(RIX_EINVAL, "NULL vis or image_out");
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (J.fp64) return op_grid<double>(&J, part, (const double2*)vis, (double*)image_out, st);
  return op_grid<float>(&J, part, (const float2*)vis, (float*)image_out, st);
}

// Computes the partition's PSF once (on `st`) and makes `st` wait for it,
// whichever stream computed it.
static int ensure_psf(Job& J, int part, cudaStream_t st) {
  Part& pt = J.part[part];
  if (!pt.psf_ready) {
    if (J.fp64) RIX_TRY(op_psf<double>(&J, part, st));
    else RIX_TRY(op_psf<float>(&J, part, st));
    RIX_CUDA(cudaEventRecord(pt.ev_psf, st));
  }
  RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_psf, 0));
  return RIX_OK;
}

static int rix_psf_impl(rix_job_t job, int part, void* psf_out, double* weight_sum_out, rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RIX_TRY(ensure_psf(J, part, st));
  if (psf_out) {
    const size_t b = (size_t)4 * J.desc.n * J.desc.n * (J.fp64 ? 8 : 4);
    RIX_CUDA(cudaMemcpyAsync(psf_out, J.part[part].psf.p, b, cudaMemcpyDeviceToDevice, st));
  }
  if (weight_sum_out) *weight_sum_out = J.part[part].wsum;
  return RIX_OK;
}

static int rix_major_cycle_impl(rix_job_t job, int part, const void* vis_obs, const void* model, void* residual_out,
                    rix_stream_t stream) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  if (!vis_obs) return set_error(RIX_EINVAL, "vis_obs is NULL");
  Part& pt = J.part[part];
  if (pt.minor_done < pt.cycle) return set_error(RIX_ESTATE, "partition %d: minor cycle %d not done", part, pt.cycle);
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t img = (size_t)J.desc.n * J.desc.n * (J.fp64 ? 8 : 4);
  // order after this partition's previous minor cycle, whatever stream it used
  if (pt.minor_done > 0) RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_minor[pt.minor_done & 1], 0));
  if (model) RIX_CUDA(cudaMemcpyAsync(pt.model.p, model, img, cudaMemcpyDeviceToDevice, st));
  if (J.fp64) RIX_TRY(op_major<double>(&J, part, (const double2*)vis_obs, pt.resid.as<double>(), st));
  else RIX_TRY(op_major<float>(&J, part, (const float2*)vis_obs, pt.resid.as<float>(), st));
  RIX_CUDA(cudaEventRecord(pt.ev_major, st));
  if (residual_out) RIX_CUDA(cudaMemcpyAsync(residual_out, pt.resid.p, img, cudaMemcpyDeviceToDevice, st));
  pt.cycle += 1;
  return RIX_OK;
}

static int minor_precheck(Job& J, int part, cudaStream_t st) {
  RIX_TRY(check_part(&J, part));
  Part& pt = J.part[part];
  if (pt.cycle == 0 || pt.minor_done >= pt.cycle)
    return set_error(RIX_ESTATE, "partition %d: run the major cycle before the minor cycle", part);
  const int n = pt.cycle;
  // this partition's major cycle of this cycle, whatever stream it ran on
  RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_major, 0));
  for (int q = 0; q < J.n_part; ++q) {
    if (q == part) continue;
    if (J.part[q].minor_done < n - 1)
      return set_error(RIX_ESTATE, "partition %d cycle %d needs partition %d's minor cycle %d", part, n, q, n - 1);
    // the other partitions' previous-cycle publish (Phi_q^{n-1}); waiting on
    // that cycle's event, not the latest, lets same-cycle minor cycles overlap
    if (n >= 2) RIX_CUDA(cudaStreamWaitEvent(st, J.part[q].ev_minor[(n - 1) & 1], 0));
  }
  for (int q = 0; q < J.n_part; ++q) RIX_TRY(ensure_psf(J, q, st));
  return RIX_OK;
}

static int rix_minor_cycle_msclean_impl(rix_job_t job, int part, const rix_msclean_params* prm, void* delta_out,
                            rix_stream_t stream) {
  if (!job || !prm) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (prm->n_scales < 1 || prm->n_scales > kMaxScales || !prm->scales || prm->scales[0] != 0.0f)
    return set_error(RIX_EINVAL, "scales: 1..%d radii with scales[0] = 0", kMaxScales);
  for (int i = 1; i < prm->n_scales; ++i)
    if (!(prm->scales[i] > 0.0f) || prm->scales[i] >= (float)J.desc.n / 2) return set_error(RIX_EINVAL, "bad scale %d", i);
  if (!(prm->gain > 0.0 && prm->gain <= 1.0) || prm->niter < 0 || !(prm->threshold >= 0.0))
    return set_error(RIX_EINVAL, "bad gain / niter / threshold");
  RIX_TRY(minor_precheck(J, part, st));
  if (J.fp64) RIX_TRY(op_msclean<double>(&J, part, prm, (double*)delta_out, st));
  else RIX_TRY(op_msclean<float>(&J, part, prm, (float*)delta_out, st));
  J.part[part].minor_done += 1;
  RIX_CUDA(cudaEventRecord(J.part[part].ev_minor[J.part[part].minor_done & 1], st));
  return RIX_OK;
}

static int check_fista_params(const Job& J, const rix_fista_params* prm) {
  const int maxlev = ilog2(J.desc.n) - 3;
  if (prm->iters < 0 || prm->levels < 1 || prm->levels > maxlev)
    return set_error(RIX_EINVAL, "iters >= 0 and levels in [1, %d]", maxlev);
  if (!(prm->lambda > 0.0) && !(prm->lambda_rel > 0.0) && !(prm->sched_a > 0.0))
    return set_error(RIX_EINVAL, "lambda, lambda_rel or sched_a must be > 0");
  if (prm->dictionary != RIX_DICT_DB4 && prm->dictionary != RIX_DICT_DB1_8)
    return set_error(RIX_EINVAL, "dictionary must be RIX_DICT_DB4 or RIX_DICT_DB1_8");
  if (prm->sched_a < 0.0 || (prm->sched_a > 0.0 && !(prm->sched_b > 0.0)))
    return set_error(RIX_EINVAL, "schedule: sched_a >= 0 and sched_b > 0");
  return RIX_OK;
}

static int rix_minor_cycle_fista_batch_impl(rix_job_t job, int n_parts, const int32_t* parts,
                                            const rix_fista_params* prm, rix_stream_t stream) {
  if (!job || !prm || !parts) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  if (n_parts < 1 || n_parts > J.n_part) return set_error(RIX_EINVAL, "n_parts must be in [1, %d]", J.n_part);
  for (int i = 0; i < n_parts; ++i) {
    RIX_TRY(check_part(&J, parts[i]));
    for (int k = 0; k < i; ++k)
      if (parts[k] == parts[i]) return set_error(RIX_EINVAL, "partition %d listed twice", parts[i]);
  }
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RIX_TRY(check_fista_params(J, prm));
  for (int i = 0; i < n_parts; ++i)
    if (J.part[parts[i]].cycle != J.part[parts[0]].cycle)
      return set_error(RIX_ESTATE, "the batch's partitions are at different cycles");
  // Each partition prepares and finishes on a stream of its own (the job's),
  // which starts after the caller's work on `stream` and waits, as one call
  // per partition would, for this partition's major cycle and the other
  // partitions' previous minor cycles only; `stream` runs the loop and, at
  // return, waits for everything.
  RIX_CUDA(cudaEventRecord(J.ev_batch, st));
  int pl[kMaxPart];
  cudaStream_t ps[kMaxPart];
  for (int i = 0; i < n_parts; ++i) {
    Part& pt = J.part[parts[i]];
    if (!pt.own_stream) RIX_CUDA(cudaStreamCreateWithFlags(&pt.own_stream, cudaStreamNonBlocking));
    RIX_CUDA(cudaStreamWaitEvent(pt.own_stream, J.ev_batch, 0));
    RIX_TRY(minor_precheck(J, parts[i], pt.own_stream));
    pl[i] = parts[i];
    ps[i] = pt.own_stream;
  }
  if (J.fp64) RIX_TRY(op_fista_batch<double>(&J, n_parts, pl, prm, st, ps));
  else RIX_TRY(op_fista_batch<float>(&J, n_parts, pl, prm, st, ps));
  for (int i = 0; i < n_parts; ++i) {
    Part& pt = J.part[parts[i]];
    pt.minor_done += 1;
    RIX_CUDA(cudaEventRecord(pt.ev_minor[pt.minor_done & 1], st));
  }
  return RIX_OK;
}

static int rix_minor_cycle_fista_impl(rix_job_t job, int part, const rix_fista_params* prm, void* delta_out,
                          rix_stream_t stream) {
  if (!job || !prm) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RIX_TRY(check_fista_params(J, prm));
  RIX_TRY(minor_precheck(J, part, st));
  if (J.fp64) RIX_TRY(op_fista<double>(&J, part, prm, (double*)delta_out, st));
  else RIX_TRY(op_fista<float>(&J, part, prm, (float*)delta_out, st));
  J.part[part].minor_done += 1;
  RIX_CUDA(cudaEventRecord(J.part[part].ev_minor[J.part[part].minor_done & 1], st));
  return RIX_OK;
}

int rix_get_components(rix_job_t job, int part, int32_t* count, int32_t capacity, int32_t* scale_out,
                       int32_t* pixel_out, double* amp_out, rix_stream_t stream) {
  if (!job || !count) return set_error(RIX_EINVAL, "NULL argument");
  RIX_CUDA(cudaSetDevice(job->j.ctx->device));
  return get_components(&job->j, part, count, capacity, scale_out, pixel_out, amp_out, (cudaStream_t)stream);
}

static int rix_get_model_impl(rix_job_t job, int part, void* image_out, rix_stream_t stream) {
  if (!job || !image_out) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (J.part[part].minor_done > 0)
    RIX_CUDA(cudaStreamWaitEvent(st, J.part[part].ev_minor[J.part[part].minor_done & 1], 0));
  const size_t img = (size_t)J.desc.n * J.desc.n * (J.fp64 ? 8 : 4);
  RIX_CUDA(cudaMemcpyAsync(image_out, J.part[part].model.p, img, cudaMemcpyDeviceToDevice, st));
  return RIX_OK;
}

static int rix_combine_impl(rix_job_t job, void* image_out, rix_stream_t stream) {
  if (!job || !image_out) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  if (!J.partitioned) return set_error(RIX_ESTATE, "not partitioned");
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  for (int q = 0; q < J.n_part; ++q)
    if (J.part[q].minor_done > 0) RIX_CUDA(cudaStreamWaitEvent(st, J.part[q].ev_minor[J.part[q].minor_done & 1], 0));
  if (J.fp64) return op_combine<double>(&J, (double*)image_out, st);
  return op_combine<float>(&J, (float*)image_out, st);
}

int rix_job_set_psf_method(rix_job_t job, int32_t method) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  if (method != RIX_PSF_AUTO && method != RIX_PSF_DOUBLE_GRID && method != RIX_PSF_TILES)
    return set_error(RIX_EINVAL, "PSF method must be RIX_PSF_AUTO, RIX_PSF_DOUBLE_GRID or RIX_PSF_TILES");
  Job& J = job->j;
  J.psf_method = method;
  for (int p = 0; p < kMaxPart; ++p) {
    J.part[p].psf_ready = false;
    J.part[p].ms_p_cycle = 0;
  }
  return RIX_OK;
}

// ---- gridder tuning and batched major cycles ------------------------------
int rix_job_tune(rix_job_t job, int32_t chunk_limit, int32_t ctas_per_sm) {
  if (!job) return set_error(RIX_EINVAL, "job is NULL");
  if (chunk_limit < 1 || chunk_limit > 256 || ctas_per_sm < 0 || ctas_per_sm > 8)
    return set_error(RIX_EINVAL, "chunk_limit in [1, 256] and ctas_per_sm in [0, 8]");
  Job& J = job->j;
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  J.fp_ctas_per_sm = ctas_per_sm;
  if (chunk_limit != J.chunk_limit) {
    J.chunk_limit = chunk_limit;
    if (J.partitioned) {
      // the jobs' own work finishes before the chunk lists are rebuilt
      for (auto& pr : J.touched) RIX_CUDA(cudaEventSynchronize(pr.second));
      cudaStream_t st = J.ctx->mem_stream;
      if (J.fp64) RIX_TRY(grid_work_order<double>(&J, st));
      else RIX_TRY(grid_work_order<float>(&J, st));
      RIX_CUDA(cudaStreamSynchronize(st));
    }
  }
  return RIX_OK;
}

int rix_batch_create(rix_ctx_t ctx, int32_t n, const rix_job_t* jobs, const int32_t* parts, rix_batch_t* batch) {
  if (!ctx || !jobs || !parts || !batch) return set_error(RIX_EINVAL, "NULL argument");
  *batch = nullptr;
  if (n < 1 || n > 4096) return set_error(RIX_EINVAL, "a batch holds 1 .. 4096 pairs");
  RIX_CUDA(cudaSetDevice(ctx->c.device));
  rix_batch_s* bs = new (std::nothrow) rix_batch_s();
  if (!bs) return set_error(RIX_ENOMEM, "host allocation");
  Batch& B = bs->b;
  B.ctx = &ctx->c;
  B.n = n;
  int rc = RIX_OK;
  for (int i = 0; i < n && rc == RIX_OK; ++i) {
    if (!jobs[i]) { rc = set_error(RIX_EINVAL, "job %d is NULL", i); break; }
    Job* J = &jobs[i]->j;
    if (J->ctx != &ctx->c) rc = set_error(RIX_EINVAL, "job %d belongs to another context", i);
    else if ((rc = check_part(J, parts[i])) != RIX_OK) break;
    else if (J->fp64 || J->nw < kW || J->tile != 16)
      rc = set_error(RIX_EINVAL, "job %d: batches hold FP32 w-stacked jobs with tile 16", i);
    for (int k = 0; k < i && rc == RIX_OK; ++k)
      if (B.jobs[k] == J && B.parts[k] == parts[i]) rc = set_error(RIX_EINVAL, "pair %d listed twice", i);
    if (rc == RIX_OK) {
      B.jobs.push_back(J);
      B.parts.push_back(parts[i]);
      rc = ensure_planes_f32(J, parts[i]);
    }
  }
  if (rc == RIX_OK) B.ctas_per_sm = B.jobs[0]->fp_ctas_per_sm;
  if (rc == RIX_OK) rc = batch_build(&B);
  for (int k = 0; k < Batch::kStreams && rc == RIX_OK; ++k)
    if (cudaStreamCreateWithFlags(&B.streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B.ev_join[k], cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(RIX_ECUDA, "batch streams");
  if (rc == RIX_OK && cudaEventCreateWithFlags(&B.ev_fork, cudaEventDisableTiming) != cudaSuccess)
    rc = set_error(RIX_ECUDA, "batch events");
  if (rc != RIX_OK) {
    rix_batch_destroy(bs);
    return rc;
  }
  *batch = bs;
  return RIX_OK;
}

int rix_batch_destroy(rix_batch_t batch) {
  if (!batch) return RIX_OK;
  Batch& B = batch->b;
  cudaSetDevice(B.ctx->device);
  for (int k = 0; k < Batch::kStreams; ++k) {
    if (B.streams[k]) {
      if (cudaStreamSynchronize(B.streams[k]) != cudaSuccess) cudaGetLastError();
      cudaStreamDestroy(B.streams[k]);
    }
    if (B.ev_join[k]) cudaEventDestroy(B.ev_join[k]);
  }
  if (B.ev_fork) cudaEventDestroy(B.ev_fork);
  delete batch;
  return RIX_OK;
}

int rix_batch_major_cycle(rix_batch_t batch, const void* const* vis_obs, void* const* residual_out,
                          rix_stream_t stream) {
  if (!batch || !vis_obs) return set_error(RIX_EINVAL, "NULL argument");
  Batch& B = batch->b;
  RIX_CUDA(cudaSetDevice(B.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<const float2*> vis(B.n);
  for (int i = 0; i < B.n; ++i) {
    Job* J = B.jobs[i];
    Part& pt = J->part[B.parts[i]];
    if (!J->partitioned) return set_error(RIX_ESTATE, "pair %d: the job is not partitioned", i);
    if (!vis_obs[i]) return set_error(RIX_EINVAL, "pair %d: vis_obs is NULL", i);
    if (pt.minor_done < pt.cycle) return set_error(RIX_ESTATE, "pair %d: minor cycle %d not done", i, pt.cycle);
    vis[i] = static_cast<const float2*>(vis_obs[i]);
  }
  // order after each pair's previous minor cycle; under stream capture the
  // graph is replayed after work the caller has ordered itself (an event
  // recorded before the capture cannot be waited on inside it)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RIX_CUDA(cudaStreamIsCapturing(st, &cap));
  for (int i = 0; i < B.n && cap == cudaStreamCaptureStatusNone; ++i) {
    Part& pt = B.jobs[i]->part[B.parts[i]];
    if (pt.minor_done > 0) RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_minor[pt.minor_done & 1], 0));
  }
  RIX_TRY(op_major_batch(&B, vis.data(), st));
  for (int i = 0; i < B.n; ++i) {
    Job* J = B.jobs[i];
    Part& pt = J->part[B.parts[i]];
    if (residual_out && residual_out[i])
      RIX_CUDA(cudaMemcpyAsync(residual_out[i], pt.resid.p, (size_t)J->desc.n * J->desc.n * sizeof(float),
                               cudaMemcpyDeviceToDevice, st));
    // a captured cycle is not an executed one: the jobs' events and cycle
    // counters stay as they were (an event recorded in a capture could not
    // be waited on by later calls)
    if (cap != cudaStreamCaptureStatusNone) continue;
    RIX_CUDA(cudaEventRecord(pt.ev_major, st));
    pt.cycle += 1;
    RIX_TRY(note_stream(J, st));
  }
  return RIX_OK;
}

int rix_gridder_probe(rix_job_t job, int part, const void* vis_obs, int32_t reps, double* ms_out) {
  if (!job || !vis_obs || !ms_out || reps < 1) return set_error(RIX_EINVAL, "bad argument");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  if (J.fp64 || J.nw < kW || J.tile != 16) return set_error(RIX_EINVAL, "the probe times the FP32 w-stacked gridder");
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  for (auto& pr : J.touched) RIX_CUDA(cudaEventSynchronize(pr.second));
  RIX_TRY(ensure_planes_f32(&J, part));
  Part& pt = J.part[part];
  cudaStream_t st = J.ctx->mem_stream;
  cudaEvent_t e0, e1;
  RIX_CUDA(cudaEventCreate(&e0));
  RIX_CUDA(cudaEventCreate(&e1));
  int rc = gather_y(&J, pt.ent_begin, pt.ent_count, vis_obs, st);
  if (rc == RIX_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = set_error(RIX_ECUDA, "event");
  for (int r = 0; r < reps && rc == RIX_OK; ++r)
    rc = launch_tiles_fp(&J, kResid, pt.item_begin, pt.item_count, pt.ent_begin, pt.ent_count, pt.win_lo, pt.win_n,
                         pt.model_planes.p, pt.resid_planes.p, vis_obs, st);
  float ms = 0.f;
  if (rc == RIX_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = set_error(RIX_ECUDA, "probe timing");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == RIX_OK) *ms_out = ms / reps;
  return rc;
}

int rix_major_cycle_probe(rix_job_t job, int part, const void* vis_obs, int32_t reps, double* ms_out) {
  if (!job || !vis_obs || !ms_out || reps < 1) return set_error(RIX_EINVAL, "bad argument");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  for (auto& pr : J.touched) RIX_CUDA(cudaEventSynchronize(pr.second));
  cudaStream_t st = J.ctx->mem_stream;
  const size_t img = (size_t)J.desc.n * J.desc.n * (J.fp64 ? 8 : 4);
  void* tmp = nullptr;
  if (malloc_async(&tmp, img, st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(RIX_ENOMEM, "probe image");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RIX_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = set_error(RIX_ECUDA, "events");
  // one untimed pass (first-use buffers), then the timed ones
  for (int r = 0; r <= reps && rc == RIX_OK; ++r) {
    if (r == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = set_error(RIX_ECUDA, "event");
    if (rc != RIX_OK) break;
    rc = J.fp64 ? op_major<double>(&J, part, static_cast<const double2*>(vis_obs), static_cast<double*>(tmp), st)
                : op_major<float>(&J, part, static_cast<const float2*>(vis_obs), static_cast<float*>(tmp), st);
  }
  float ms = 0.f;
  if (rc == RIX_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = set_error(RIX_ECUDA, "probe timing");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(tmp, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == RIX_OK) rc = set_error(RIX_ECUDA, "probe");
  if (rc == RIX_OK) *ms_out = ms / reps;
  return rc;
}

// ---- band-limited exchange ------------------------------------------------
int rix_phi_support(rix_job_t job, int part, int64_t* count_out) {
  if (!job || !count_out) return set_error(RIX_EINVAL, "NULL argument");
  RIX_TRY(check_part(&job->j, part));
  *count_out = job->j.part[part].ring_count;
  return RIX_OK;
}

static int rix_phi_pack_impl(rix_job_t job, int part, void* packed_out, rix_stream_t stream) {
  if (!job || !packed_out) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  Part& pt = J.part[part];
  if (pt.minor_done < 1) return set_error(RIX_ESTATE, "partition %d has no completed minor cycle", part);
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_minor[pt.minor_done & 1], 0));
  if (J.fp64) return op_phi_pack<double>(&J, part, static_cast<double2*>(packed_out), st);
  return op_phi_pack<float>(&J, part, static_cast<float2*>(packed_out), st);
}

static int rix_phi_unpack_impl(rix_job_t job, int part, const void* packed, void* phi_out, rix_stream_t stream) {
  if (!job || !packed || !phi_out) return set_error(RIX_EINVAL, "NULL argument");
  Job& J = job->j;
  RIX_TRY(check_part(&J, part));
  RIX_CUDA(cudaSetDevice(J.ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (J.fp64) return op_phi_unpack<double>(&J, part, static_cast<const double2*>(packed), static_cast<double*>(phi_out), st);
  return op_phi_unpack<float>(&J, part, static_cast<const float2*>(packed), static_cast<float*>(phi_out), st);
}

// ---- baseline-dependent averaging (context-level preprocessing) ----------
namespace {
// windows, counts and output offsets on the device; the row total on the host
struct BdaPlan {
  int32_t* window = nullptr;
  uint32_t* count = nullptr;
  uint32_t* offset = nullptr;
  uint32_t* total = nullptr;
  cudaStream_t st = nullptr;
  ~BdaPlan() {
    if (window) cudaFreeAsync(window, st);
    if (count) cudaFreeAsync(count, st);
    if (offset) cudaFreeAsync(offset, st);
    if (total) cudaFreeAsync(total, st);
  }
};

int bda_plan(Ctx* ctx, const double* uvw, int64_t nt, int64_t nbl, const double* freq, int nchan, int n,
             double cell, double max_shift, cudaStream_t st, BdaPlan& pl, int64_t* nrow) {
  pl.st = st;
  if (malloc_async(&pl.window, nbl * sizeof(int32_t), st) != cudaSuccess ||
      malloc_async(&pl.count, nbl * sizeof(uint32_t), st) != cudaSuccess ||
      malloc_async(&pl.offset, nbl * sizeof(uint32_t), st) != cudaSuccess ||
      malloc_async(&pl.total, sizeof(uint32_t), st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(RIX_ENOMEM, "averaging plan");
  }
  RIX_TRY(bda_windows(ctx, uvw, nt, nbl, freq, nchan, n, cell, max_shift, pl.window, pl.count, st));
  RIX_TRY(scan_exclusive_u32(pl.count, pl.offset, nbl, pl.total, st));
  uint32_t tot = 0;
  RIX_CUDA(cudaMemcpyAsync(&tot, pl.total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RIX_CUDA(cudaStreamSynchronize(st));
  *nrow = tot;
  return RIX_OK;
}
}  // namespace

int rix_bda_rows(rix_ctx_t ctx, const double* uvw_m, int64_t n_times, int64_t n_baselines, const double* freq_hz,
                 int32_t nchan, int32_t n, double cell_rad, double max_shift_px, int32_t* window_out,
                 int64_t* nrow_out, rix_stream_t stream) {
  if (!ctx || !uvw_m || !nrow_out) return set_error(RIX_EINVAL, "NULL argument");
  RIX_CUDA(cudaSetDevice(ctx->c.device));
  cudaStream_t st = (cudaStream_t)stream;
  BdaPlan pl;
  RIX_TRY(bda_plan(&ctx->c, uvw_m, n_times, n_baselines, freq_hz, nchan, n, cell_rad, max_shift_px, st, pl,
                   nrow_out));
  if (window_out) {
    RIX_CUDA(cudaMemcpyAsync(window_out, pl.window, n_baselines * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RIX_CUDA(cudaStreamSynchronize(st));
  }
  return RIX_OK;
}

int rix_bda_average(rix_ctx_t ctx, const double* uvw_m, const void* vis, const float* weight, int64_t n_times,
                    int64_t n_baselines, const double* freq_hz, int32_t nchan, int32_t precision, int32_t n,
                    double cell_rad, double max_shift_px, double* uvw_out, void* vis_out, float* weight_out,
                    int64_t nrow_capacity, int64_t* nrow_out, rix_stream_t stream) {
  if (!ctx || !uvw_m || !vis || !uvw_out || !vis_out || !weight_out) return set_error(RIX_EINVAL, "NULL argument");
  if (precision != RIX_FP32 && precision != RIX_FP64) return set_error(RIX_EINVAL, "bad precision");
  RIX_CUDA(cudaSetDevice(ctx->c.device));
  cudaStream_t st = (cudaStream_t)stream;
  BdaPlan pl;
  int64_t nrow = 0;
  RIX_TRY(bda_plan(&ctx->c, uvw_m, n_times, n_baselines, freq_hz, nchan, n, cell_rad, max_shift_px, st, pl, &nrow));
  if (nrow > nrow_capacity)
    return set_error(RIX_EINVAL, "averaging gives %lld rows, the output holds %lld", (long long)nrow,
                     (long long)nrow_capacity);
  if (nrow_out) *nrow_out = nrow;
  if (precision == RIX_FP64)
    return bda_average<double2>(&ctx->c, uvw_m, static_cast<const double2*>(vis), weight, n_times, n_baselines,
                                nchan, pl.window, pl.offset, uvw_out, static_cast<double2*>(vis_out), weight_out, st);
  return bda_average<float2>(&ctx->c, uvw_m, static_cast<const float2*>(vis), weight, n_times, n_baselines, nchan,
                             pl.window, pl.offset, uvw_out, static_cast<float2*>(vis_out), weight_out, st);
}

// ---- public wrappers: run the call, then note the stream the job used ----
#define RIX_NOTE(job, stream, call)                                           \
  do {                                                                        \
    const int rc_ = (call);                                                   \
    if (job && rc_ == RIX_OK) return ::rix::note_stream(&job->j, (cudaStream_t)stream); \
    return rc_;                                                               \
  } while (0)

int rix_set_uv_partition(rix_job_t job, const double* uvw_m, int64_t nrow, const float* weight,
                         const double* ell_px, double delta_px, uint8_t* mask_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_set_uv_partition_impl(job, uvw_m, nrow, weight, ell_px, delta_px, mask_out, stream));
}
int rix_get_sorted_entries(rix_job_t job, uint32_t* keys_out, uint32_t* samples_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_get_sorted_entries_impl(job, keys_out, samples_out, stream));
}
int rix_get_weights(rix_job_t job, float* weight_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_get_weights_impl(job, weight_out, stream));
}
int rix_degrid(rix_job_t job, int part, const void* image, void* vis_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_degrid_impl(job, part, image, vis_out, stream));
}
int rix_grid(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_grid_impl(job, part, vis, image_out, stream));
}
int rix_psf(rix_job_t job, int part, void* psf_out, double* weight_sum_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_psf_impl(job, part, psf_out, weight_sum_out, stream));
}
int rix_major_cycle(rix_job_t job, int part, const void* vis_obs, const void* model, void* residual_out,
                    rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_major_cycle_impl(job, part, vis_obs, model, residual_out, stream));
}
int rix_minor_cycle_msclean(rix_job_t job, int part, const rix_msclean_params* prm, void* delta_out,
                            rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_minor_cycle_msclean_impl(job, part, prm, delta_out, stream));
}
int rix_minor_cycle_fista_batch(rix_job_t job, int n_parts, const int32_t* parts, const rix_fista_params* prm,
                                rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_minor_cycle_fista_batch_impl(job, n_parts, parts, prm, stream));
}
int rix_minor_cycle_fista(rix_job_t job, int part, const rix_fista_params* prm, void* delta_out,
                          rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_minor_cycle_fista_impl(job, part, prm, delta_out, stream));
}
int rix_get_model(rix_job_t job, int part, void* image_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_get_model_impl(job, part, image_out, stream));
}
int rix_combine(rix_job_t job, void* image_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_combine_impl(job, image_out, stream));
}
int rix_phi_pack(rix_job_t job, int part, void* packed_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_phi_pack_impl(job, part, packed_out, stream));
}
int rix_phi_unpack(rix_job_t job, int part, const void* packed, void* phi_out, rix_stream_t stream) {
  RIX_NOTE(job, stream, rix_phi_unpack_impl(job, part, packed, phi_out, stream));
}


}  // extern "C"

