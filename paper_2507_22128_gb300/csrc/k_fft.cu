// Hand-written FFT stages (the F, F^dagger of Eq. 2 and the padded
// convolutions of the minor cycles).
//
// Every transform maps between a real M x M image, centred on an L x L grid
// (pixel offset a' = a - M/2 sits at grid index a' mod L, multiplied by
// (-1)^(a'+b') so that spectrum index j holds frequency j - L/2), and the
// window [lo, lo + S)^2 of its spectrum, stored u-major: spec[ju][jv].
// A 2D transform is two passes over HBM:
//   rows    one CTA transforms a batch of image rows in shared memory,
//           skipping the zero padding and writing only the window columns,
//           transposed (T[ju][b]) so that the column pass reads contiguously;
//   columns one CTA transforms a batch of window columns, again skipping
//           zeros, and writes the window rows contiguously.
// The 1D transforms are radix-16/8/4/2 Stockham (autosort) passes on data
// held in shared memory (one pad slot every 16 entries against bank
// conflicts), twiddles read from a table computed on the host in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rix_internal.cuh"
#include "fft_device.cuh"

namespace rix {
namespace {

template <typename R, int VPT>
__global__ void __launch_bounds__(kFftThreads, (VPT == 0 && sizeof(R) == 4) ? 4 : 1) k_fwd_rows(KArgs a, const R* __restrict__ img,
                                                          cplx<R>* __restrict__ T,
                                                          const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  RIX_FFT_SMEM
  fwd_rows_block<R, VPT>(a, img, T, tw, s, s2, blockIdx.x, blockIdx.y);
}

// three CTAs per SM: the shared memory of two 2048-point rows allows no more,
// and the register accumulators of the plane sum need the room
template <typename R, int VPT>
__global__ void __launch_bounds__(kFftThreads, (VPT == 0 && sizeof(R) == 4) ? 3 : 1) k_inv_rows(KArgs a, const cplx<R>* __restrict__ T,
                                                          R* __restrict__ img, double scale, int accumulate,
                                                          const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  RIX_FFT_SMEM
  inv_rows_block<R, VPT>(a, T, img, scale, accumulate, tw, s, s2, blockIdx.x, blockIdx.y);
}

template <typename R, int VPT>
__global__ void __launch_bounds__(kFftThreads, (VPT == 0 && sizeof(R) == 4) ? 4 : 1) k_fwd_cols(KArgs a, const cplx<R>* __restrict__ T,
                                                          cplx<R>* __restrict__ spec,
                                                          const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  RIX_FFT_SMEM
  fwd_cols_block<R, VPT>(a, T, spec, tw, s, s2, blockIdx.x, blockIdx.y);
}

template <typename R, int VPT>
__global__ void __launch_bounds__(kFftThreads, (VPT == 0 && sizeof(R) == 4) ? 4 : 1) k_inv_cols(KArgs a, const cplx<R>* __restrict__ spec, int op,
                                                          const void* tab, const void* tab2,
                                                          cplx<R>* __restrict__ T,
                                                          const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  RIX_FFT_SMEM
  inv_cols_block<R, VPT>(a, spec, op, tab, tab2, T, tw, s, s2, blockIdx.x, blockIdx.y);
}

template <typename R, int VPT>
__global__ void __launch_bounds__(kFftThreads, (VPT == 0 && sizeof(R) == 4) ? 4 : 1) k_conv_cols(KArgs a, const cplx<R>* __restrict__ Tin, int op,
                                                           const void* tab, const void* tab2,
                                                           cplx<R>* __restrict__ Tout,
                                                           const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  RIX_FFT_SMEM
  conv_cols_block<R, VPT>(a, Tin, op, tab, tab2, Tout, tw, s, s2, blockIdx.x, blockIdx.y);
}

// screen[p][pix] = corr[pix] * exp(-2 pi i (w0 + p dw) nm1[pix]), formed as
// the row passes form it (wscreen)
template <typename R>
__global__ void k_screen_table(int64_t npix, int nplanes, double w0, double dw, const R* __restrict__ corr,
                               const double* __restrict__ nm1, cplx<R>* __restrict__ screen) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix * nplanes;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / npix);
    const int64_t pix = i - (int64_t)p * npix;
    const cplx<R> e = wscreen<R, -1>(w0 + p * dw, nm1[pix]);
    const R c = corr[pix];
    screen[i] = cmake<cplx<R>>(e.x * c, e.y * c);
  }
}

// img = (accumulate ? img : 0) + sum over g < G of part[g]
template <typename R>
__global__ void k_sum_groups(R* __restrict__ img, const R* __restrict__ part, int G, int64_t n, int accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R v = accumulate ? img[i] : R(0);
    for (int g = 0; g < G; ++g) v += part[(int64_t)g * n + i];
    img[i] = v;
  }
}

// ------------------------------------------------------------------- host ----
// rows per CTA for a given values-per-thread setting
template <typename R>
int batch_for(const Ctx* ctx, int vpt, int L, int nunits, int nz) {
  int B = std::max(1, kFftThreads * vpt / L);
  // keep ~2 CTAs per SM busy when the problem is small, but give every thread
  // at least one radix-4 item per pass
  const int bmin = std::max(1, (kFftThreads * 4) / L);
  while (B > bmin && (int64_t)ceil_div(nunits, B) * nz < 2LL * ctx->num_sms) B >>= 1;
  return B;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
  RIX_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return RIX_OK;
}

template <typename R>
int check_geom(const XformGeom& g) {
  if (g.L < 32 || g.L > kTwMax || (g.L & (g.L - 1)) || (1 << g.logL) != g.L || g.M < 4 || g.M > g.L ||
      (g.M & 3) || g.lo < 0 || g.S <= 0 || g.nplanes <= 0)
    return set_error(RIX_EINVAL, "bad transform geometry (M=%d L=%d lo=%d S=%d)", g.M, g.L, g.lo, g.S);
  if (kFftThreads * Vpt<R>::kLarge < g.L) return set_error(RIX_EINVAL, "transform length %d too large", g.L);
  return RIX_OK;
}

// Launches kernel K<R, VPT> with the batch chosen for VPT.  `units` is the
// number of rows (or columns) to transform, `nz` the grid's y extent.
#define RIX_FFT_LAUNCH(KERNEL, units, nz, ...)                                                   \
  do {                                                                                           \
    timing_mark(kTimeFft, st, true);                                                             \
    if (use_inplace<R>(g.L)) {                                                                   \
      constexpr int V = Vpt<R>::kLarge;                                                          \
      const int B = batch_for<R>(ctx, V, g.L, (units), (nz));                                    \
      KArgs a = make_args<R>(g, B);                                                              \
      const size_t sm = (size_t)B * a.stride * sizeof(cplx<R>);                                  \
      RIX_TRY(set_smem(KERNEL<R, V>, sm));                                                       \
      KERNEL<R, V><<<dim3((unsigned)ceil_div((units), B), (nz)), kFftThreads, sm, st>>>(a, __VA_ARGS__); \
    } else {                                                                                     \
      const int B = batch_for<R>(ctx, kPingPongVals<R>, g.L, (units), (nz));                    \
      KArgs a = make_args<R>(g, B);                                                              \
      const size_t sm = 2 * (size_t)B * a.stride * sizeof(cplx<R>);                              \
      RIX_TRY(set_smem(KERNEL<R, 0>, sm));                                                       \
      KERNEL<R, 0><<<dim3((unsigned)ceil_div((units), B), (nz)), kFftThreads, sm, st>>>(a, __VA_ARGS__); \
    }                                                                                            \
    ::rix::note_launch();                                                                        \
    timing_mark(kTimeFft, st, false);                                                            \
    RIX_LAUNCH_CHECK();                                                                          \
  } while (0)

}  // namespace

template <typename R>
int fft_max_len() {
  int L = 1;
  while (2 * L <= kTwMax && kFftThreads * Vpt<R>::kLarge >= 2 * L) L *= 2;
  return L;
}
template int fft_max_len<float>();
template int fft_max_len<double>();

int fft_init_twiddles(Ctx* ctx) {
  std::vector<double2> t64(kTwMax);
  std::vector<float2> t32(kTwMax);
  for (int k = 0; k < kTwMax; ++k) {
    const double ang = 2.0 * M_PI * (double)k / (double)kTwMax;
    t64[k] = make_double2(std::cos(ang), -std::sin(ang));
    t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
  }
  RIX_TRY(ctx->tw64.alloc(ctx, kTwMax * sizeof(double2)));
  RIX_TRY(ctx->tw32.alloc(ctx, kTwMax * sizeof(float2)));
  RIX_CUDA(cudaMemcpy(ctx->tw64.p, t64.data(), kTwMax * sizeof(double2), cudaMemcpyHostToDevice));
  RIX_CUDA(cudaMemcpy(ctx->tw32.p, t32.data(), kTwMax * sizeof(float2), cudaMemcpyHostToDevice));
  return RIX_OK;
}

template <typename R>
int build_screen_table(const Ctx* ctx, const XformGeom& g, cplx<R>* screen, cudaStream_t st) {
  if (g.mode != kFacPhase || !g.corr || !g.nm1 || g.M <= 0 || g.nplanes <= 0)
    return set_error(RIX_EINVAL, "screen table needs a w-stacked geometry");
  const int64_t npix = (int64_t)g.M * g.M;
  const int blocks = (int)std::min<int64_t>(ceil_div(npix * g.nplanes, 256), (int64_t)ctx->num_sms * 16);
  ::rix::note_launch();
  k_screen_table<R><<<blocks, 256, 0, st>>>(npix, g.nplanes, g.w0, g.dw, static_cast<const R*>(g.corr), g.nm1,
                                            screen);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}
template <typename R>
int fwd_rows(const Ctx* ctx, const XformGeom& g, const R* img, cplx<R>* T, cudaStream_t st) {
  RIX_TRY(check_geom<R>(g));
  RIX_FFT_LAUNCH(k_fwd_rows, g.M, g.nplanes, img, T, twiddles<R>(ctx));
  return RIX_OK;
}

template <typename R>
int fwd_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* T, cplx<R>* spec, cudaStream_t st) {
  RIX_TRY(check_geom<R>(g));
  RIX_FFT_LAUNCH(k_fwd_cols, g.S, g.nplanes, T, spec, twiddles<R>(ctx));
  return RIX_OK;
}

template <typename R>
int inv_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* spec, int op, const void* tab,
             const void* tab2, cplx<R>* T, cudaStream_t st) {
  RIX_TRY(check_geom<R>(g));
  RIX_FFT_LAUNCH(k_inv_cols, g.S, g.nplanes, spec, op, tab, tab2, T, twiddles<R>(ctx));
  return RIX_OK;
}

template <typename R>
int conv_cols(const Ctx* ctx, const XformGeom& g, const cplx<R>* Tin, int op, const void* tab,
              const void* tab2, cplx<R>* Tout, cudaStream_t st) {
  RIX_TRY(check_geom<R>(g));
  if (g.lo != 0 || g.S > g.L || g.nplanes != 1) return set_error(RIX_EINVAL, "conv_cols needs a window starting at 0");
  RIX_FFT_LAUNCH(k_conv_cols, g.S, 1, Tin, op, tab, tab2, Tout, twiddles<R>(ctx));
  return RIX_OK;
}

// The planes of one row batch are summed by one CTA.  With many planes and
// few row batches the grid ends in a nearly empty wave; split the planes into
// G groups (grid rows) when that takes fewer plane-transforms per SM slot,
// each group summing into its own image, and add the G images after.  At most
// max_groups groups (a divisor of the plane count).
template <typename R>
int inv_rows_groups(const Ctx* ctx, const XformGeom& g, int max_groups) {
  const int P = g.nplanes;
  int G = 1;
  if (P > 1 && max_groups > 1) {
    const int V = use_inplace<R>(g.L) ? Vpt<R>::kLarge : kPingPongVals<R>;
    const int B = batch_for<R>(ctx, V, g.L, g.M, 1);
    const size_t sm = (use_inplace<R>(g.L) ? 1 : 2) * (size_t)B * padded_len(g.L) * sizeof(cplx<R>);
    int per_sm = 0;
    if (use_inplace<R>(g.L)) {
      RIX_TRY(set_smem(k_inv_rows<R, Vpt<R>::kLarge>, sm));
      RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inv_rows<R, Vpt<R>::kLarge>, kFftThreads, sm));
    } else {
      RIX_TRY(set_smem(k_inv_rows<R, 0>, sm));
      RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inv_rows<R, 0>, kFftThreads, sm));
    }
    const int64_t slots = (int64_t)ctx->num_sms * std::max(per_sm, 1);
    const int64_t rowb = ceil_div(g.M, B);
    double best = 1e300;
    for (int c = 1; c <= P && c <= 16 && c <= max_groups; c *= 2) {
      if (P % c) continue;
      const double cost = (double)ceil_div(rowb * c, slots) * (P / c) + 0.1 * c;   // + the group sum
      if (cost < best) { best = cost; G = c; }
    }
  }
  return G;
}

template <typename R>
int inv_rows(const Ctx* ctx, const XformGeom& g0, const cplx<R>* T, R* img, double scale, int accumulate,
             cudaStream_t st, R* group_buf, int max_groups) {
  RIX_TRY(check_geom<R>(g0));
  XformGeom g = g0;
  const int P = g.nplanes;
  const int G = inv_rows_groups<R>(ctx, g, max_groups < 0 ? 16 : max_groups);
  if (G < 0) return G;
  if (G == 1) {
    RIX_FFT_LAUNCH(k_inv_rows, g.M, 1, T, img, scale, accumulate, twiddles<R>(ctx));
    return RIX_OK;
  }
  const int64_t n = (int64_t)g.M * g.M;
  // the group images: the caller's buffer, else a stream-ordered temporary
  // released on every way out
  struct StreamFree {
    void* p = nullptr;
    cudaStream_t s;
    ~StreamFree() {
      if (p) cudaFreeAsync(p, s);
    }
  } part{nullptr, st};
  R* parts = group_buf;
  if (!parts) {
    if (malloc_async(&part.p, (size_t)G * n * sizeof(R), st) != cudaSuccess) {
      part.p = nullptr;
      cudaGetLastError();
      return set_error(RIX_ENOMEM, "plane-group images (%zu bytes)", (size_t)G * n * sizeof(R));
    }
    parts = static_cast<R*>(part.p);
  }
  g.pg = P / G;
  RIX_FFT_LAUNCH(k_inv_rows, g.M, G, T, parts, scale, 0, twiddles<R>(ctx));
  ::rix::note_launch();
  k_sum_groups<R><<<(int)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 8), 256, 0, st>>>(
      img, parts, G, n, accumulate);
  if (cudaGetLastError() != cudaSuccess) return set_error(RIX_ECUDA, "group sum launch");
  return RIX_OK;
}

#define RIX_FFT_INST(R)                                                                                  \
  template int fwd_rows<R>(const Ctx*, const XformGeom&, const R*, cplx<R>*, cudaStream_t);              \
  template int fwd_cols<R>(const Ctx*, const XformGeom&, const cplx<R>*, cplx<R>*, cudaStream_t);        \
  template int inv_cols<R>(const Ctx*, const XformGeom&, const cplx<R>*, int, const void*, const void*,   \
                           cplx<R>*, cudaStream_t);                                                      \
  template int conv_cols<R>(const Ctx*, const XformGeom&, const cplx<R>*, int, const void*, const void*,  \
                            cplx<R>*, cudaStream_t);                                                     \
  template int inv_rows<R>(const Ctx*, const XformGeom&, const cplx<R>*, R*, double, int, cudaStream_t, R*, int); \
  template int inv_rows_groups<R>(const Ctx*, const XformGeom&, int);                                     \
  template int build_screen_table<R>(const Ctx*, const XformGeom&, cplx<R>*, cudaStream_t);
RIX_FFT_INST(float)
RIX_FFT_INST(double)

}  // namespace rix
