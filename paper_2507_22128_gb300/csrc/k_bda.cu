// Baseline-dependent averaging: the remedy the paper names for unbalanced
// uv partitions (Sec. 6.2: the dense uv centre of Sgr B2 left the outer node
// idle; Sec. 7 item d), after Wijnholds et al. (2018).
//
// Rows are time-major (row = t * n_baselines + b).  Per baseline, the
// largest per-step (u, v) change at the highest channel frequency, in cells
// of the N x N image's Fourier grid, is
//     s_b = max_t sqrt(du^2 + dv^2) (N dl),
// and the baseline's times are averaged in consecutive windows of
//     k_b = min(n_times, max(1, floor(max_shift / s_b)))   (n_times if s_b = 0)
// samples, the last one shorter, so the track moves at most max_shift cells
// within a window.  An averaged row holds the mean uvw of its window and per
// channel the weight sum and the weighted mean visibility.  Output rows are
// baseline-major.  The window arithmetic is FP64 with every product, sum and
// quotient rounded separately (it decides an integer); the sums are FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rix_internal.cuh"

namespace rix {
namespace {

// one warp per baseline: k_b and the number of windows
__global__ void k_bda_windows(const double* __restrict__ uvw, int64_t nt, int64_t nbl, double inv_lambda, double ncell,
                              double max_shift, int32_t* __restrict__ window, uint32_t* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = warp; b < nbl; b += nwarps) {
    double best = 0.0;
    for (int64_t t = lane; t + 1 < nt; t += 32) {
      const double* p0 = uvw + (t * nbl + b) * 3;
      const double* p1 = uvw + ((t + 1) * nbl + b) * 3;
      const double du = __dmul_rn(__dadd_rn(p1[0], -p0[0]), inv_lambda);
      const double dv = __dmul_rn(__dadd_rn(p1[1], -p0[1]), inv_lambda);
      const double step = __dmul_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(du, du), __dmul_rn(dv, dv))), ncell);
      best = fmax(best, step);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) {
      int64_t k = nt;
      if (best > 0.0) {
        const double q = floor(__ddiv_rn(max_shift, best));
        k = q < 1.0 ? 1 : (q >= (double)nt ? nt : (int64_t)q);
      }
      window[b] = (int32_t)k;
      count[b] = (uint32_t)((nt + k - 1) / k);
    }
  }
}

template <typename C>
__device__ __forceinline__ C to_cplx(double re, double im);
template <> __device__ __forceinline__ float2 to_cplx<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ double2 to_cplx<double2>(double re, double im) {
  return make_double2(re, im);
}

// one warp per baseline: its windows in time order; lanes over channels
// (and lanes 0-2 over the uvw coordinates)
template <typename C>
__global__ void k_bda_average(const double* __restrict__ uvw, const C* __restrict__ vis,
                              const float* __restrict__ weight, int64_t nt, int64_t nbl, int nchan,
                              const int32_t* __restrict__ window, const uint32_t* __restrict__ offset,
                              double* __restrict__ uvw_out, C* __restrict__ vis_out, float* __restrict__ w_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = warp; b < nbl; b += nwarps) {
    const int64_t k = window[b];
    const int64_t rows = (nt + k - 1) / k;
    for (int64_t g = 0; g < rows; ++g) {
      const int64_t t0 = g * k, t1 = min(nt, t0 + k);
      const int64_t out = (int64_t)offset[b] + g;
      if (lane < 3) {
        double s = 0.0;
        for (int64_t t = t0; t < t1; ++t) s += uvw[(t * nbl + b) * 3 + lane];
        uvw_out[out * 3 + lane] = s / (double)(t1 - t0);
      }
      for (int c = lane; c < nchan; c += 32) {
        double sw = 0.0, sr = 0.0, si = 0.0;
        for (int64_t t = t0; t < t1; ++t) {
          const int64_t i = (t * nbl + b) * nchan + c;
          const double w = weight ? (double)weight[i] : 1.0;
          const C v = vis[i];
          sw += w;
          sr += w * (double)v.x;
          si += w * (double)v.y;
        }
        const int64_t o = out * nchan + c;
        w_out[o] = (float)sw;
        vis_out[o] = sw > 0.0 ? to_cplx<C>(sr / sw, si / sw) : to_cplx<C>(0.0, 0.0);
      }
    }
  }
}

int check_args(int64_t nt, int64_t nbl, const double* freq, int nchan, int n, double cell, double max_shift) {
  if (nt < 1 || nbl < 1 || nt * nbl > (int64_t)0x7fffffff / 4 || !freq || nchan < 1 || n < 1 || !(cell > 0.0) ||
      !(max_shift >= 0.0))
    return set_error(RIX_EINVAL, "bad averaging arguments");
  for (int c = 0; c < nchan; ++c)
    if (!(freq[c] > 0.0)) return set_error(RIX_EINVAL, "frequencies must be positive");
  return RIX_OK;
}

}  // namespace

int bda_windows(Ctx* ctx, const double* uvw, int64_t nt, int64_t nbl, const double* freq, int nchan, int n,
                double cell, double max_shift, int32_t* window, uint32_t* count, cudaStream_t st) {
  RIX_TRY(check_args(nt, nbl, freq, nchan, n, cell, max_shift));
  const double f_max = *std::max_element(freq, freq + nchan);
  const double inv_lambda = f_max / kC;
  const double ncell = (double)n * cell;
  const int blocks = (int)std::min<int64_t>(ceil_div(nbl * 32, 256), (int64_t)ctx->num_sms * 16);
  ::rix::note_launch();
  k_bda_windows<<<blocks, 256, 0, st>>>(uvw, nt, nbl, inv_lambda, ncell, max_shift, window, count);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

template <typename C>
int bda_average(Ctx* ctx, const double* uvw, const C* vis, const float* weight, int64_t nt, int64_t nbl, int nchan,
                const int32_t* window, const uint32_t* offset, double* uvw_out, C* vis_out, float* w_out,
                cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(ceil_div(nbl * 32, 256), (int64_t)ctx->num_sms * 16);
  ::rix::note_launch();
  k_bda_average<C><<<blocks, 256, 0, st>>>(uvw, vis, weight, nt, nbl, nchan, window, offset, uvw_out, vis_out, w_out);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

template int bda_average<float2>(Ctx*, const double*, const float2*, const float*, int64_t, int64_t, int,
                                 const int32_t*, const uint32_t*, double*, float2*, float*, cudaStream_t);
template int bda_average<double2>(Ctx*, const double*, const double2*, const float*, int64_t, int64_t, int,
                                  const int32_t*, const uint32_t*, double*, double2*, float*, cudaStream_t);

}  // namespace rix
