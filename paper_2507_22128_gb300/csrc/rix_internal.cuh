// Internal declarations shared by the translation units of librix.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rix.h"

namespace rix {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
const char* last_error();
// counts the kernels the library runs (all host threads), including the
// kernel nodes of replayed CUDA graphs
void note_launch(long long n = 1);
unsigned long long launch_count();
// Every device allocation of the library (pooled, stream-ordered) goes
// through malloc_async, which counts it (rix_device_allocations).
cudaError_t malloc_async(void** p, size_t bytes, cudaStream_t st);
template <typename T>
cudaError_t malloc_async(T** p, size_t bytes, cudaStream_t st) {
  return malloc_async(reinterpret_cast<void**>(p), bytes, st);
}

// Opt-in device timing of kernel classes (CUDA events recorded on the launch
// stream around each launch; streams under capture are skipped).
enum TimedClass : int { kTimeTiles = 0, kTimeFft = 1, kTimePartition = 2, kTimeMinorLoop = 3, kTimeClasses = 4 };
bool timing_on();
void timing_mark(int cls, cudaStream_t st, bool begin);

#define RIX_CUDA(...)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                                     \
    if (e_ != cudaSuccess)                                                              \
      return ::rix::set_error(RIX_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__,            \
                              #__VA_ARGS__, cudaGetErrorString(e_));                    \
  } while (0)

#define RIX_TRY(...)               \
  do {                             \
    int r_ = (__VA_ARGS__);        \
    if (r_ != RIX_OK) return r_;   \
  } while (0)

#define RIX_LAUNCH_CHECK() RIX_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// numeric types
// ---------------------------------------------------------------------------
template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <typename R> using cplx = typename Cplx<R>::T;

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im);
template <> __host__ __device__ __forceinline__ float2 cmake<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 cmake<double2>(double re, double im) {
  return make_double2(re, im);
}
// On the device a complex sum or difference is one packed FP32x2 instruction
// (each lane rounded as the scalar one)
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  unsigned long long x, y, d;
  float2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
  return r;
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  unsigned long long x, y, d;
  float2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
  return r;
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}

constexpr double kC = 299792458.0;
constexpr int kW = 8;            // ES kernel support (cells)
constexpr double kBeta = 18.4;   // 2.30 * kW

// ---------------------------------------------------------------------------
// gridder building blocks shared by k_grid.cu and k_tiles_fp.cu
// ---------------------------------------------------------------------------
enum GridMode : int { kDegrid = 0, kGrid = 1, kResid = 2, kPsf = 3 };

// Exponential-of-semicircle kernel weight of tap i for a sample whose first
// tap sits d in [0, 1) cells after its kernel's left edge:
// phi(z) = exp(beta (sqrt(1 - z^2) - 1)), z = (d + i) 2/W - 1.
template <typename R> __device__ __forceinline__ R es_weight(R d, int i);
template <> __device__ __forceinline__ float es_weight<float>(float d, int i) {
  const float z = (d + (float)i) * (2.0f / kW) - 1.0f;
  const float t = fmaxf(1.0f - z * z, 0.0f);
  return expf((float)kBeta * (sqrtf(t) - 1.0f));
}
template <> __device__ __forceinline__ double es_weight<double>(double d, int i) {
  const double z = (d + (double)i) * (2.0 / kW) - 1.0;
  const double t = fmax(1.0 - z * z, 0.0);
  return exp(kBeta * (sqrt(t) - 1.0));
}

// Per sorted entry, fixed for the job: the kernel offsets du = ceil(xs) - xs,
// dv, dw (rounded once from FP64 to the job's precision) and the first tap
// relative to the entry's tile origin (ou | ov << 8).  Computed once at
// partition time with the FP64 arithmetic the kernels used to repeat every
// major cycle (GB300 runs FP64 at 1/64 of the FP32 rate).
template <typename R>
struct alignas(4 * sizeof(R)) EntryGeom {
  R du, dv, dw;
  uint32_t ouv;
};

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct Ctx;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Ctx* owner = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(Ctx* ctx, size_t nbytes);      // frees any previous allocation first
  void release();
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct Ctx {
  int device = 0;
  size_t budget = 0;          // 0 = unlimited
  size_t reserved = 0;        // sum of admitted job workspaces
  int jobs = 0;
  int num_sms = 0;
  cudaStream_t mem_stream = nullptr;   // stream-ordered allocation and release
  DevBuf tw32, tw64;          // FFT twiddle tables, length kTwMax
};

constexpr int kTwLog = 14;
constexpr int kTwMax = 1 << kTwLog;   // largest 1D FFT length (4N for N = 4096)

// ---------------------------------------------------------------------------
// FFT plans (see k_fft.cu)
// ---------------------------------------------------------------------------
enum FactorMode : int {
  kFacNone = 0,     // value * (-1)^(a+b)
  kFacReal = 1,     // value * corr[b][a] * (-1)^(a+b)
  kFacPhase = 2,    // value * corr[b][a] * exp(-+2 pi i w_p (n - 1)) * (-1)^(a+b)
};

// Describes the pixel-side factor of a transform between an M x M real image
// (centred on an L x L grid) and the window [lo, lo + S)^2 of its spectrum.
struct XformGeom {
  int M, L, logL, lo, S;
  int nplanes;
  int mode;                    // FactorMode
  const void* corr;            // Real [M][M] or null
  const double* nm1;           // double [M][M]: n - 1 per pixel (kFacPhase)
  double w0, dw;               // plane p sits at w0 + p * dw (kFacPhase)
  int herm = 0;                // inverse rows: complete columns [S, L) by conjugate symmetry
  // kFacPhase, optional: cplx [nplanes][M][M] of corr * exp(-2 pi i w_p (n-1)),
  // the factors tabulated once per job (build_screen_table); corr and nm1
  // are then not read by the row passes
  const void* screen = nullptr;
  // inverse rows: planes per CTA row of the grid (0: all), set by inv_rows
  int pg = 0;
};
// screen[p][b][a] = corr[b][a] * exp(-2 pi i (w0 + p dw) nm1[b][a]) for the
// geometry g (kFacPhase), the same values the row passes would form
template <typename R>
int build_screen_table(const Ctx* ctx, const XformGeom& g, cplx<R>* screen, cudaStream_t st);

// the longest transform the row and column passes support (a power of two)
template <typename R>
int fft_max_len();
template <typename R>
int fwd_rows(const Ctx* ctx, const XformGeom& g, const R* img, cplx<R>* T, cudaStream_t st);
template <typename R>
int fwd_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* T, cplx<R>* spec, cudaStream_t st);
// spectral operator applied between the forward and inverse column transforms
enum SpecOp : int { kOpNone = 0, kOpMulReal = 1, kOpMulCplx = 2, kOpAxpyReal = 3 };
template <typename R>
int inv_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* spec, int op, const void* tab,
             const void* tab2, cplx<R>* T, cudaStream_t st);
template <typename R>
int conv_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* Tin, int op, const void* tab,
              const void* tab2, cplx<R>* Tout, cudaStream_t st);
// Inverse row pass: img = (accumulate ? img : 0) + scale * the planes' sum.
// With several planes it may split them into G groups (inv_rows_groups, at
// most max_groups; -1 = the pass's own limit), each summed into an image of
// group_buf (G * M * M reals) or, when group_buf is null, of a temporary
// stream-ordered allocation.
template <typename R>
int inv_rows(const Ctx* ctx, const XformGeom& g, const cplx<R>* T, R* img, double scale,
             int accumulate, cudaStream_t st, R* group_buf = nullptr, int max_groups = -1);
// the number of plane groups inv_rows uses for g with at most max_groups
template <typename R>
int inv_rows_groups(const Ctx* ctx, const XformGeom& g, int max_groups);

int fft_init_twiddles(Ctx* ctx);

// ---------------------------------------------------------------------------
// partition / sort (see k_partition.cu)
// ---------------------------------------------------------------------------
struct SampleGeomParams {
  const double* uvw;          // [nrow][3]
  const double* inv_lambda;   // [nchan] f / c
  int64_t nrow;
  int nchan;
  int ng;                     // grid side 2N
  double scale;               // cell * ng
  double half;                // ng / 2
  double ndl;                 // N * cell
  int nw, ww;                 // w-planes (0 = coplanar), w support
  double w_min, dw;
};

int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                       cudaStream_t st);
int radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                   int64_t n, int bits, cudaStream_t st, bool* result_in_tmp);

// ---------------------------------------------------------------------------
// job
// ---------------------------------------------------------------------------
constexpr int kMaxPart = RIX_MAX_PART;
constexpr int kMaxScales = 8;

struct Part {
  int64_t ent_begin = 0, ent_count = 0;     // range in the sorted entries
  int64_t item_begin = 0, item_count = 0;   // range in the work items
  double wsum = 0.0;
  int win_lo = 0, win_n = 0;                // uv window on the 2N grid
  int pwin_lo = 0, pwin_n = 0;              // uv window on the 4N PSF grid
  int cycle = 0;                            // major cycles issued
  int minor_done = 0;                       // minor cycles issued
  bool psf_ready = false;
  bool lambda_set = false;
  DevBuf model_planes, resid_planes, tbuf;  // [nw][S][S], [nw][S][S], [nw][S][N]
  DevBuf groups;                            // plane-group images of the inverse row pass, [G][N][N]
  DevBuf model, resid, delta;               // N x N Real
  DevBuf outbox[2];                         // Phi_p^n by cycle parity (image, or ring-support coefficients)
  DevBuf ring_idx;                          // ring support of Gamma_p, half plane ju <= N (flat u-major indices)
  int64_t ring_count = 0;
  DevBuf rho[kMaxPart];                     // rho_{q->p}, N x N
  DevBuf psf;                               // 2N x 2N Real
  DevBuf hspec;                             // centred spectrum of the PSF, (2N)^2 complex
  DevBuf lambda_dev;                        // double: FISTA lambda
  // fill scratch: two (2N)^2 spectra, two [2N][N] transpose buffers, an image
  DevBuf fs_a, fs_b, ft_a, ft_b, fimg;
  DevBuf fspec;                             // P spectra: slot p = own residual, slot q = rho_{q->p}
  DevBuf fi_state;                          // FISTA: [max Mx, max |residual| of cycle 1, ||residual||^2, -]
  // minor-cycle state
  DevBuf ms_R, ms_P, ms_B, ms_comp, ms_state;   // ms-CLEAN
  DevBuf fi_alpha, fi_alpha_prev, fi_y, fi_mx, fi_c, fi_x, fi_d;   // FISTA
  int ms_ncomp_cap = 0;
  // the cycle whose composite PSF ms_P holds (0: none) and its scales: from
  // cycle 2 on the composite PSF of Eq. 7 no longer changes, so later cycles
  // with the same scales reuse ms_P and the scale spectra in ms_B
  int ms_p_cycle = 0;
  std::vector<float> ms_p_scales;
  // recorded after the minor cycle of each cycle parity (cycle n -> [n % 2])
  cudaEvent_t ev_minor[2] = {nullptr, nullptr};
  cudaEvent_t ev_psf = nullptr;             // recorded after the PSF is computed
  cudaEvent_t ev_major = nullptr;           // recorded after each major cycle
  // batched minor cycles: the partition's own stream and two join events
  cudaStream_t own_stream = nullptr;
  cudaEvent_t ev_prep = nullptr, ev_done = nullptr;
  DevBuf sync;                              // grid-barrier arrival counters of the cooperative kernels
};

struct Job {
  Ctx* ctx = nullptr;
  rix_job_desc desc{};
  std::vector<double> freq;
  std::vector<double> inv_lambda_h;
  int64_t max_rows = 0;
  size_t reserved = 0;
  int ng = 0, tile = 16, nw = 0, ww = 1;
  bool fp64 = false;
  bool partitioned = false;
  rix_job_stats stats{};
  // resident inputs
  DevBuf uvw, weight, inv_lambda;
  // sort
  DevBuf keys, samples, items;              // entries and work-item begin offsets (+1 sentinel)
  // Gridder order: within every work item the entries are reordered by their
  // first tap (the cell their kernel footprint starts at), so runs of
  // entries with one footprint are contiguous; a chunk is a run of at most 32
  // such entries.  egeom and gsamples are in this order; `samples` keeps the
  // sorted order rix_get_sorted_entries reports.
  DevBuf egeom;                             // per entry: kernel offsets and tap origin (EntryGeom<R>)
  DevBuf gsamples;                          // per entry: sample index
  DevBuf ysamp;                             // FP32 w-stacked: per entry {w re v, w im v, w, 0} of the last gridding call
  DevBuf chunks;                            // entry offset of each chunk (+1 sentinel: n_entries)
  DevBuf item_chunk;                        // first chunk of each work item (+1 sentinel: the chunk count)
  int64_t n_entries = 0, n_items = 0;
  int bt = 0, bw = 0, bp = 0;
  // corrections
  DevBuf corr_img, corr_psf;                // Real [N][N], [2N][2N]
  DevBuf nm1_img, nm1_psf;                  // double n - 1 per pixel (w-stacked)
  DevBuf screen_img;                        // w-stacked: corr x phase screen per plane, image grid
  DevBuf gam;                               // Real [P][2N][2N] filters (u-major spectra)
  Part part[kMaxPart];
  double ells[kMaxPart];
  int n_part = 1;
  cudaEvent_t ev_batch = nullptr;           // batched minor cycles: call entry, then loop end
  DevBuf status;                            // int: 0, or the RIX_E* code a device-side wait raised
  // streams the job's calls ran on, each with an event recorded after the call
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> touched;
  // tuning of the FP32 w-stacked gridder (rix_job_tune): entries per chunk
  // (at most 32) and resident CTAs per SM (0: as many as fit)
  int chunk_limit = 64;
  int fp_ctas_per_sm = 0;
  bool gorder = false;   // egeom (and gsamples) in the gridder order
  int psf_method = 0;    // RIX_PSF_* (rix_job_set_psf_method)
};

// The major cycles of several (job, partition) pairs with one gridder launch
// (rix_batch_*): per pair the gridder's arguments and tensor maps, uploaded
// once by batch_build.
struct Batch {
  Ctx* ctx = nullptr;
  int n = 0;
  std::vector<Job*> jobs;
  std::vector<int> parts;
  DevBuf descs, maps, item_start;
  int64_t total_items = 0;
  int ctas_per_sm = 0;
  // the pairs' transforms run on these streams, forked from and joined to
  // the caller's stream by events
  static constexpr int kStreams = 4;
  cudaStream_t streams[kStreams] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kStreams] = {};
};
// k_tiles_fp.cu: the descriptors (the pairs' plane buffers must exist), the
// weighted visibilities of one partition, and the batch's gridder launch
int batch_build(Batch* b);
int gather_y(const Job* job, int64_t ent_begin, int64_t ent_count, const void* vis, cudaStream_t st);
int batch_gridder(const Batch* b, cudaStream_t st);
// k_grid.cu: the pairs' major cycles (image -> planes, one gridder launch,
// planes -> residual images into each partition's resident residual)
int op_major_batch(Batch* b, const float2* const* vis, cudaStream_t st);
int ensure_planes_f32(Job* job, int p);

// records that `st` carries work of `job` (for rix_job_destroy)
int note_stream(Job* job, cudaStream_t st);
// reads the job's device status word (the caller has synchronised the job's
// streams); RIX_ETIMEOUT if a bounded device-side wait gave up
int check_status(Job* job);
// wavelet_filters.cu: Daubechies low-pass filter with p vanishing moments
// (2p taps written to h); returns 2p or a negative RIX_E* code
int daubechies_lowpass(int p, double* h);
// k_selftest.cu: bounded-barrier timeout self-test (rix_selftest_barrier_timeout)
int selftest_barrier(Ctx* ctx, int* status_out, int* gave_up_out);

// gridder entry points (k_grid.cu)
template <typename R>
int grid_build_corrections(Job* job, cudaStream_t st);
template <typename R>
int grid_entry_geometry(Job* job, cudaStream_t st);
// gridder order and chunks of the job's entries (k_tiles_fp.cu), after
// grid_entry_geometry
template <typename R>
int grid_work_order(Job* job, cudaStream_t st);
// The FP32 w-stacked gridder with register-resident kernel footprints
// (k_tiles_fp.cu): mode kGrid spreads w * vis into out_planes, kResid
// degrids model_planes and spreads w * (vis - model visibility); planes
// [n_wplanes][S][S] complex on the partition's uv window [win_lo, win_lo + S)
// (out_planes zeroed by the caller).  Tile side 16.
int launch_tiles_fp(const Job* job, int mode, int64_t item_begin, int64_t item_count, int64_t ent_begin,
                    int64_t ent_count, int win_lo, int S, const void* model_planes, void* out_planes, const void* vis,
                    cudaStream_t st);
// The PSF gridding of partition p on the same gridder (FP32 w-stacked jobs
// with tile 16): unit visibilities times the weights spread on the PSF grid
// (coordinate x = u_lambda * scale + half) into planes [n_wplanes][S][S]
// complex on the partition's PSF window (S = its side; zeroed by the caller).
int launch_psf_fp(const Job* job, int p, double scale, double half, void* planes, cudaStream_t st);
template <typename R>
int op_degrid(Job* job, int p, const R* image, cplx<R>* vis_out, cudaStream_t st);
template <typename R>
int op_grid(Job* job, int p, const cplx<R>* vis, R* image_out, cudaStream_t st);
template <typename R>
int op_major(Job* job, int p, const cplx<R>* vis, R* residual, cudaStream_t st);
template <typename R>
int op_psf(Job* job, int p, cudaStream_t st);

int op_grid_into_scratch(Job* job, int p, const float2* vis, float* image_out, float2* scratch,
                         size_t scratch_elems, cudaStream_t st);

// baseline-dependent averaging (k_bda.cu): per baseline the window k_b and
// its number of windows, then the averaged rows at the exclusive scan of the
// counts
int bda_windows(Ctx* ctx, const double* uvw, int64_t nt, int64_t nbl, const double* freq, int nchan, int n,
                double cell, double max_shift, int32_t* window, uint32_t* count, cudaStream_t st);
template <typename C>
int bda_average(Ctx* ctx, const double* uvw, const C* vis, const float* weight, int64_t nt, int64_t nbl, int nchan,
                const int32_t* window, const uint32_t* offset, double* uvw_out, C* vis_out, float* w_out,
                cudaStream_t st);

// partition entry point (k_partition.cu)
int partition_job(Job* job, const double* uvw, int64_t nrow, const float* weight,
                  const double* ell_px, double delta, uint8_t* mask_out, cudaStream_t st);

// minor cycles (k_minor.cu)
template <typename R>
int fill_init(Job* job, cudaStream_t st);
template <typename R>
int op_msclean(Job* job, int p, const rix_msclean_params* prm, R* delta_out, cudaStream_t st);
template <typename R>
int op_fista(Job* job, int p, const rix_fista_params* prm, R* delta_out, cudaStream_t st);
// The FISTA minor cycles of partitions parts[0 .. nb) with one loop launch on
// `st`; the preparation and finish of parts[i] run on ps[i], ordered after
// the caller's work by the caller.
template <typename R>
int op_fista_batch(Job* job, int nb, const int* parts, const rix_fista_params* prm, cudaStream_t st,
                   const cudaStream_t* ps);
template <typename R>
int op_combine(Job* job, R* out, cudaStream_t st);
// band-limited exchange (k_minor.cu): the ring-support coefficients of
// Gamma_p F pad i_bar_p, and Phi_p rebuilt from such coefficients
template <typename R>
int op_phi_pack(Job* job, int p, cplx<R>* out, cudaStream_t st);
template <typename R>
int op_phi_unpack(Job* job, int p, const cplx<R>* coef, R* out, cudaStream_t st);

// persistent FISTA iteration loop (k_fista*.cu): all `iters` iterations of
// the minor cycles of one or more partitions in one cooperative launch.
// Images are N x N, the transposes (N+1) x N complex, mx / c the u-major
// (2N)^2 fill tables.
template <typename R>
struct FistaLoop {
  R* alpha;
  R* y;
  R* x;
  R* g;
  R* tmp;
  cplx<R>* ta;
  cplx<R>* tb;
  const R* mx;
  const cplx<R>* c;
  R* d;                    // N x N: 2 crop F^-1 c, formed by the loop
  const R* state;          // [max Mx, max |residual| of cycle 1]
  const cplx<R>* tw;       // twiddle table, length kTwMax
  unsigned int* barrier;   // arrival counter (zeroed by the call, stream-ordered)
  int* status;             // the job's status word
  double lambda, lambda_rel;
  int n, levels, iters;
  int dict;                // RIX_DICT_DB4 or RIX_DICT_DB1_8
  double sched_a, sched_bn;   // sched_a > 0: lambda = sched_a * sqrt(state[2]) * sched_bn
  // RIX_DICT_DB1_8 only: member m's coefficients at alpha / y + m N^2, its
  // level buffers at xs / bs + m N^2 (N x N each), W alpha written to delta
  // after the last iteration
  R* xs;
  R* bs;
  R* delta;
};
// The loops f[0 .. nb) (nb <= kMaxPart) share n, levels, iters and the
// dictionary; they run as one launch with f[0].barrier as its barrier.  One
// instance per precision and dictionary (k_fista_*.cu).
template <typename R, int DICT>
int fista_loop_dict(const Ctx* ctx, const FistaLoop<R>* f, int nb, cudaStream_t st);
int get_components(Job* job, int part, int32_t* count, int32_t capacity, int32_t* scale_out,
                   int32_t* pixel_out, double* amp_out, cudaStream_t st);

inline int ilog2(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace rix
