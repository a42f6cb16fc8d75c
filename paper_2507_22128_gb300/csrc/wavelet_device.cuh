// Device code of the Db4 wavelet transform (the dictionary of the FISTA
// minor cycle, Eq. 4-5): one tile of one analysis level (with the FISTA step
// fused into the final coefficients) and one tile of one synthesis level.
// Shared by the per-level kernels and the persistent minor-cycle loop.
#pragma once

#include <cuda_runtime.h>

#include "rix_internal.cuh"

namespace rix {
namespace {

// --------------------------------------------------------------- Db4 DWT ----
// Daubechies 4-vanishing-moment low-pass filter (8 taps, minimum phase,
// normalised to sum sqrt(2)); g[i] = (-1)^i h[7 - i].
// Compile-time constants: every use below has a compile-time tap index, so the
// taps fold into immediates (no constant-bank loads or FP64 conversions).
__device__ constexpr double kDb4[8] = {0.23037781330885523,  0.7148465705525415,   0.6308807679295904,
                                       -0.02798376941698385, -0.18703481171888114, 0.030841381835986965,
                                       0.032883011666982945, -0.010597401784997278};

template <typename R> __device__ __forceinline__ constexpr R db_h(int i) { return (R)kDb4[i]; }
template <typename R> __device__ __forceinline__ constexpr R db_g(int i) {
  return (i & 1) ? -(R)kDb4[7 - i] : (R)kDb4[7 - i];
}

// ------------------------------------------------- fused Db4 DWT levels ----
// Analysis of one level: a CTA owns a kTB x kTB block of each of the four
// subbands of an n x n block (n a power of two), stages the periodic
// (2 kTB + 6)^2 input tile, filters its rows (low and high) and then its
// columns.  Subband layout of a level: [Y][X] with Y < n/2 column-low,
// X < n/2 row-low.  Every global load of a tile is issued before the first
// one is used.
constexpr int kTB = 16;
constexpr int kTin = 2 * kTB + 6;

// FISTA step fused into the analysis of the gradient (Beck & Teboulle 2009):
// at each final coefficient g:  a' = S_{lam/L}(y - g/L),  y = a' + mom (a' - a),  a = a'
template <typename R>
struct StepArgs {
  R* alpha;
  R* y;
  R inv_l, thr;         // 1 / L and lambda / L (both 0 when L = 0: the step is a no-op)
  bool active;
  R mom;
};

template <typename R>
struct DwtSmem {
  R tin[kTin][kTin + 1];
  R trow[kTin][2 * kTB + 1];     // [input row][lo x | hi x]
};

// one kTB x kTB output block (bx, by) of each subband; 256 threads
template <typename R, bool kStep>
__device__ __forceinline__ void dwt_tile(const R* __restrict__ src, int lds, int n, R* __restrict__ coef,
                                         R* __restrict__ ll, int ld, int last, const StepArgs<R>& st, int bx, int by,
                                         DwtSmem<R>& sm) {
  constexpr int TIN = kTin;
  constexpr int NLD = (TIN * TIN + 255) / 256;
  auto& tin = sm.tin;
  auto& trow = sm.trow;
  const int h = n / 2;
  const int y0 = by * kTB, x0 = bx * kTB;
  const int ty = threadIdx.x / kTB, tx = threadIdx.x - ty * kTB;   // 256 threads = kTB x kTB
  const int y = y0 + ty, x = x0 + tx;
  const bool own = y < h && x < h;
  // the coefficients this thread updates: quadrants 1-3, and 0 at the last level
  R yq[4], aq[4];
  if (kStep && own) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q == 0 && !last) continue;
      const int64_t i = (int64_t)((q >> 1) * h + y) * ld + (q & 1) * h + x;
      yq[q] = st.y[i];
      aq[q] = st.alpha[i];
    }
  }
  R v[NLD];
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int t = threadIdx.x + 256 * k;
    if (t < TIN * TIN) {
      const int r = t / TIN, c = t - r * TIN;
      v[k] = src[(int64_t)((2 * y0 + r) & (n - 1)) * lds + ((2 * x0 + c) & (n - 1))];
    }
  }
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int t = threadIdx.x + 256 * k;
    if (t < TIN * TIN) {
      const int r = t / TIN, c = t - r * TIN;
      tin[r][c] = v[k];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TIN * kTB; t += blockDim.x) {
    const int r = t / kTB, xx = t - r * kTB;
    R a = R(0), d = R(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const R w = tin[r][2 * xx + i];
      a += db_h<R>(i) * w;
      d += db_g<R>(i) * w;
    }
    trow[r][xx] = a;
    trow[r][kTB + xx] = d;
  }
  __syncthreads();
  if (own) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cy = q >> 1, cx = q & 1;
      R g = R(0);
#pragma unroll
      for (int i = 0; i < 8; ++i) g += (cy ? db_g<R>(i) : db_h<R>(i)) * trow[2 * ty + i][cx * kTB + tx];
      const int64_t idx = (int64_t)(cy * h + y) * ld + cx * h + x;
      if (q == 0 && !last) {
        ll[(int64_t)y * ld + x] = g;
      } else if (kStep) {
        const R z = yq[q] - g * st.inv_l;
        const R az = fabs(z) - st.thr;
        const R an = (st.active && az > R(0)) ? copysign(az, z) : R(0);
        st.y[idx] = an + st.mom * (an - aq[q]);
        st.alpha[idx] = an;
      } else {
        coef[idx] = g;
      }
    }
  }
  __syncthreads();
}

// Synthesis of one level: out (n x n, ld) from the LL block `llin` (ld) and
// the detail subbands of `coef` (ld); a CTA owns a kTS x kTS output block.
constexpr int kTS = 32;
constexpr int kRK = kTS / 2 + 4;
template <typename R>
struct IdwtSmem {
  R cq[4][kRK][kRK + 1];         // quadrant tiles: LL, row-high, col-high, HH
  R tr[2][kRK][kTS + 1];         // after row synthesis: [column half][coef row][c]
};

template <typename R>
__device__ __forceinline__ void idwt_tile(const R* __restrict__ llin, const R* __restrict__ coef, int n,
                                          R* __restrict__ out, int ld, int bx, int by, IdwtSmem<R>& sm) {
  constexpr int RK = kRK;
  auto& cq = sm.cq;
  auto& tr = sm.tr;
  const int h = n / 2;
  const int m0 = by * kTS, c0 = bx * kTS;
  const int kb_m = (m0 >> 1) - 4, kb_c = (c0 >> 1) - 4;
  constexpr int NLD = (4 * RK * RK + 255) / 256;
  R v[NLD];
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int t = threadIdx.x + 256 * k;
    if (t < 4 * RK * RK) {
      const int q = t / (RK * RK), rem = t - q * RK * RK;
      const int rk = rem / RK, ck = rem - rk * RK;
      const int km = (kb_m + rk) & (h - 1), kc = (kb_c + ck) & (h - 1);   // periodic; h a power of two
      const int cy = q >> 1, cx = q & 1;
      v[k] = (q == 0) ? llin[(int64_t)km * ld + kc] : coef[(int64_t)(cy * h + km) * ld + (cx * h + kc)];
    }
  }
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int t = threadIdx.x + 256 * k;
    if (t < 4 * RK * RK) {
      const int q = t / (RK * RK), rem = t - q * RK * RK;
      const int rk = rem / RK, ck = rem - rk * RK;
      cq[q][rk][ck] = v[k];
    }
  }
  __syncthreads();
  // rows: tr[cy][rk][c] = sum over the 4 taps of the parity of c
  for (int t = threadIdx.x; t < 2 * RK * kTS; t += blockDim.x) {
    const int cy = t / (RK * kTS), rem = t - cy * RK * kTS;
    const int rk = rem / kTS, cl = rem - rk * kTS;
    const int c = c0 + cl;
    const bool odd = c & 1;
    const int kc = (c >> 1) - kb_c;             // tap i = 2 j + (c & 1) reads coefficient (c - i) / 2
    R v = R(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const R hh = odd ? db_h<R>(2 * j + 1) : db_h<R>(2 * j);
      const R gg = odd ? db_g<R>(2 * j + 1) : db_g<R>(2 * j);
      v += hh * cq[2 * cy][rk][kc - j] + gg * cq[2 * cy + 1][rk][kc - j];
    }
    tr[cy][rk][cl] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kTS * kTS; t += blockDim.x) {
    const int ml = t / kTS, cl = t - ml * kTS;
    const int m = m0 + ml, c = c0 + cl;
    if (m >= n || c >= n) continue;
    const bool odd = m & 1;
    const int km = (m >> 1) - kb_m;
    R v = R(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const R hh = odd ? db_h<R>(2 * j + 1) : db_h<R>(2 * j);
      const R gg = odd ? db_g<R>(2 * j + 1) : db_g<R>(2 * j);
      v += hh * tr[0][km - j][cl] + gg * tr[1][km - j][cl];
    }
    out[(int64_t)m * ld + c] = v;
  }
  __syncthreads();
}

}  // namespace
}  // namespace rix
