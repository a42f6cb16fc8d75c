// Device-side building blocks of the FFT stages: in-register DFTs, Stockham
// passes in shared memory and the per-block bodies of the row and column
// passes.  Included by the translation units that launch them (each gets its
// own copy in an anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "rix_internal.cuh"

namespace rix {
namespace {

constexpr int kFftThreads = 256;

// complex values per thread per pass: the small setting keeps every pass in
// registers without spills; the large one is only used for lengths beyond it.
template <typename R> struct Vpt;
template <> struct Vpt<float> { static constexpr int kSmall = 16, kLarge = 32; };
template <> struct Vpt<double> { static constexpr int kSmall = 8, kLarge = 16; };
// Ping-pong CTAs hold kFftThreads * kPingPongVals complex values per buffer.
template <typename R> constexpr int kPingPongVals = std::is_same<R, float>::value ? 16 : 8;

__host__ __device__ constexpr int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4); }

// cos / sin of 2 pi m / 16
__device__ constexpr double kCos16[16] = {1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508978,
                                          0.0, -0.38268343236508978, -0.70710678118654752, -0.92387953251128674,
                                          -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508978,
                                          0.0, 0.38268343236508978, 0.70710678118654752, 0.92387953251128674};
__device__ constexpr double kSin16[16] = {0.0, 0.38268343236508978, 0.70710678118654752, 0.92387953251128674,
                                          1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508978,
                                          0.0, -0.38268343236508978, -0.70710678118654752, -0.92387953251128674,
                                          -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508978};

// exp(DIR * 2 pi i m / N) for N | 16
template <int N, int DIR, typename C>
__device__ __forceinline__ C wconst(int m) {
  const int k = (m * (16 / N)) & 15;
  return cmake<C>(kCos16[k], DIR * kSin16[k]);
}

template <int DIR, typename C>
__device__ __forceinline__ C rot90(C a) {   // a * exp(DIR i pi / 2)
  C r;
  if (DIR < 0) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
  return r;
}

template <int DIR, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot90<DIR>(a1 - a3);
  a0 = t0 + t2; a2 = t0 - t2; a1 = t1 + t3; a3 = t1 - t3;
}

// in-register DFT of size RAD, natural order in and out
template <int RAD, int DIR, typename C>
__device__ __forceinline__ void dft(C* v) {
  if constexpr (RAD == 2) {
    const C t = v[0]; v[0] = t + v[1]; v[1] = t - v[1];
  } else if constexpr (RAD == 4) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (RAD == 8) {
    // n = 2 n1 + n2: length-4 DFTs over n1, twiddle W8^(n2 k1), length-2 over n2
    dft4<DIR>(v[0], v[2], v[4], v[6]);
    dft4<DIR>(v[1], v[3], v[5], v[7]);
    C o[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      const C a = v[2 * k1];
      const C b = k1 ? cmul(v[2 * k1 + 1], wconst<8, DIR, C>(k1)) : v[2 * k1 + 1];
      o[k1] = a + b;
      o[k1 + 4] = a - b;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  } else {
    static_assert(RAD == 16, "radix");
    // n = 4 n1 + n2: length-4 DFTs over n1, twiddle W16^(n2 k1), length-4 over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    C y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) {
        const C t = v[4 * k1 + n2];
        y[4 * k1 + n2] = (n2 * k1) ? cmul(t, wconst<16, DIR, C>(n2 * k1)) : t;
      }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      dft4<DIR>(y[4 * k1], y[4 * k1 + 1], y[4 * k1 + 2], y[4 * k1 + 3]);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = y[4 * k1 + k2];
    }
  }
}

// One Stockham pass of radix RAD over B rows of length L in shared memory.
// Item i of a row (0 <= i < L/RAD), k = i mod p: inputs i + r L/RAD, twiddles
// exp(DIR 2 pi i r k / (p RAD)), outputs ((i - k) RAD + k) + r p.
template <typename R, int VPT, int DIR, int RAD>
__device__ __forceinline__ void fft_pass(cplx<R>* s, int B, int logL, int stride, int logp,
                                         const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  constexpr int K = VPT / RAD > 0 ? VPT / RAD : 1;
  constexpr int LR = RAD == 2 ? 1 : RAD == 4 ? 2 : RAD == 8 ? 3 : 4;
  const int logipr = logL - LR;
  const int ipr = 1 << logipr;
  const int total = B << logipr;
  const int p = 1 << logp;
  const int twshift = kTwLog - (logp + LR);
  C v[K][RAD];
  int ob[K];
#pragma unroll
  for (int it = 0; it < K; ++it) {
    const int g = threadIdx.x + it * kFftThreads;
    ob[it] = -1;
    if (g < total) {
      const int row = g >> logipr;
      const int i = g & (ipr - 1);
      const int k = i & (p - 1);
      const C* rs = s + row * stride;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[it][r] = rs[padi(i + r * ipr)];
      if (k) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          C w = tw[(r * k) << twshift];
          if (DIR > 0) w.y = -w.y;
          v[it][r] = cmul(v[it][r], w);
        }
      }
      dft<RAD, DIR>(v[it]);
      ob[it] = row * stride + (((i - k) << LR) + k);   // row base + first output index
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < K; ++it) {
    if (ob[it] >= 0) {
      const int g = threadIdx.x + it * kFftThreads;
      const int row = g >> logipr;
      const int o = ob[it] - row * stride;
      C* rs = s + row * stride;
#pragma unroll
      for (int r = 0; r < RAD; ++r) rs[padi(o + r * p)] = v[it][r];
    }
  }
  __syncthreads();
}

// In-place FFT of B rows of length L = 2^logL (unnormalised; DIR = -1 forward).
// Expects the data written and a __syncthreads() done by the caller.
template <typename R, int VPT, int DIR>
__device__ void fft_rows(cplx<R>* s, int B, int logL, int stride, const cplx<R>* __restrict__ tw) {
  // a thread holds whole radix items: the largest radix is min(16, VPT)
  constexpr int kMaxLr = VPT >= 16 ? 4 : 3;
  const int npass = (logL + kMaxLr - 1) / kMaxLr;
  int logp = 0;
  for (int ps = 0; ps < npass; ++ps) {
    const int rem = logL - logp, left = npass - ps;
    const int lr = (rem + left - 1) / left;
    if constexpr (kMaxLr == 4) {
      if (lr == 4) { fft_pass<R, VPT, DIR, 16>(s, B, logL, stride, logp, tw); logp += lr; continue; }
    }
    switch (lr) {
      case 3: fft_pass<R, VPT, DIR, 8>(s, B, logL, stride, logp, tw); break;
      case 2: fft_pass<R, VPT, DIR, 4>(s, B, logL, stride, logp, tw); break;
      default: fft_pass<R, VPT, DIR, 2>(s, B, logL, stride, logp, tw); break;
    }
    logp += lr;
  }
}

// v[r] *= w^r, w = exp(DIR 2 pi i k / (p RAD)): w, w^4 and w^8 come from the
// FP64-accurate table, the other powers from at most three products of them
// (a few ulp), instead of RAD - 1 dependent table loads.
template <typename R, int DIR, int RAD>
__device__ __forceinline__ void apply_twiddles(cplx<R>* v, const cplx<R>* __restrict__ tw, int k, int twshift) {
  using C = cplx<R>;
  C w[RAD];
  auto ld = [&](int m) {
    C t = tw[(m * k) << twshift];
    if (DIR > 0) t.y = -t.y;
    return t;
  };
  w[1] = ld(1);
  if constexpr (RAD >= 4) {
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
  }
  if constexpr (RAD >= 8) {
    w[4] = ld(4);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
  }
  if constexpr (RAD >= 16) {
    w[8] = ld(8);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
  }
#pragma unroll
  for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], w[r]);
}

// Out-of-place Stockham pass (ping-pong between two shared buffers): each
// thread carries one radix item at a time, so register use stays low.
template <typename R, int DIR, int RAD>
__device__ __forceinline__ void fft_pass_pp(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst, int B,
                                            int logL, int stride, int logp, const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  constexpr int LR = RAD == 2 ? 1 : RAD == 4 ? 2 : RAD == 8 ? 3 : 4;
  const int logipr = logL - LR;
  const int ipr = 1 << logipr;
  const int total = B << logipr;
  const int p = 1 << logp;
  const int twshift = kTwLog - (logp + LR);
  for (int g = threadIdx.x; g < total; g += kFftThreads) {
    const int row = g >> logipr;
    const int i = g & (ipr - 1);
    const int k = i & (p - 1);
    const C* rs = src + row * stride;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = rs[padi(i + r * ipr)];
    if (k) apply_twiddles<R, DIR, RAD>(v, tw, k, twshift);
    dft<RAD, DIR>(v);
    C* rd = dst + row * stride;
    const int o = ((i - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) rd[padi(o + r * p)] = v[r];
  }
  __syncthreads();
}

template <typename R, int DIR>
__device__ cplx<R>* fft_rows_pp(cplx<R>* a, cplx<R>* b, int B, int logL, int stride,
                                const cplx<R>* __restrict__ tw) {
  const int npass = (logL + 3) / 4;
  int logp = 0;
  for (int ps = 0; ps < npass; ++ps) {
    const int rem = logL - logp, left = npass - ps;
    const int lr = (rem + left - 1) / left;
    switch (lr) {
      case 4: fft_pass_pp<R, DIR, 16>(a, b, B, logL, stride, logp, tw); break;
      case 3: fft_pass_pp<R, DIR, 8>(a, b, B, logL, stride, logp, tw); break;
      case 2: fft_pass_pp<R, DIR, 4>(a, b, B, logL, stride, logp, tw); break;
      default: fft_pass_pp<R, DIR, 2>(a, b, B, logL, stride, logp, tw); break;
    }
    logp += lr;
    cplx<R>* t = a; a = b; b = t;
  }
  return a;
}

// VPT == 0: ping-pong between s and s2 (returns the buffer holding the
// result); VPT > 0: in place in s with VPT values per thread per pass.
template <typename R, int VPT, int DIR>
__device__ __forceinline__ cplx<R>* fft_any(cplx<R>* s, cplx<R>* s2, int B, int logL, int stride,
                                            const cplx<R>* __restrict__ tw) {
  if constexpr (VPT == 0) {
    return fft_rows_pp<R, DIR>(s, s2, B, logL, stride, tw);
  } else {
    fft_rows<R, VPT, DIR>(s, B, logL, stride, tw);
    return s;
  }
}

// ---------------------------------------------------------------- factors ----
template <typename R> __device__ __forceinline__ void sincos_pi(R x, R* s, R* c);
template <> __device__ __forceinline__ void sincos_pi<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void sincos_pi<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// exp(DIR 2 pi i w_p (n-1)) with the phase argument formed and reduced in FP64
template <typename R, int DIR>
__device__ __forceinline__ cplx<R> wscreen(double wp, double nm1) {
  const double ph = wp * nm1;
  const double fr = ph - rint(ph);
  R s, c;
  sincos_pi<R>((R)(2.0 * fr), &s, &c);
  return cmake<cplx<R>>(c, DIR * s);
}

struct KArgs {
  int M, L, logL, lo, S, nplanes, mode, B, stride, herm;
  const void* corr;
  const double* nm1;
  double w0, dw;
  const void* screen;   // tabulated corr x phase screen per plane, or null
  int pg;               // inverse rows: planes per grid row y (0: all planes, one image)
};

// Shared-memory layout of every transform kernel: s = B rows of padded_len(L)
// entries, followed (ping-pong variant, VPT == 0) by a second such buffer.
#define RIX_FFT_SMEM                                                     \
  extern __shared__ __align__(16) unsigned char smem_raw[];              \
  C* s = reinterpret_cast<C*>(smem_raw);                                 \
  C* s2 = s + (VPT == 0 ? a.B * a.stride : 0);

// ------------------------------------------------------------ row passes ----
template <typename R, int VPT>
__device__ __forceinline__ void fwd_rows_block(KArgs a, const R* __restrict__ img,
                                                          cplx<R>* __restrict__ T,
                                                          const cplx<R>* __restrict__ tw,
    cplx<R>* s, cplx<R>* s2, int bx, int by) {
  using C = cplx<R>;
  const int p = by;
  const int b0 = bx * a.B;
  const int L = a.L, M = a.M, half = M / 2;
  const R* corr = static_cast<const R*>(a.corr);
  const double wp = a.w0 + p * a.dw;
  const C* scr = a.mode == kFacPhase && a.screen ? static_cast<const C*>(a.screen) + (int64_t)p * M * M : nullptr;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < a.B * L; idx += kFftThreads) {
    const int r = idx >> a.logL, c = idx & (L - 1);
    const int b = b0 + r;
    const int ap = c < L / 2 ? c : c - L;       // a'
    C val = cmake<C>(0.0, 0.0);
    if (b < M && ap >= -half && ap < half) {
      const int aa = ap + half;
      const int64_t pix = (int64_t)b * M + aa;
      R x = img[pix];
      if ((aa + b) & 1) x = -x;
      if (scr) {
        val = scr[pix] * x;
      } else {
        if (a.mode != kFacNone) x *= corr[pix];
        if (a.mode == kFacPhase) val = wscreen<R, -1>(wp, a.nm1[pix]) * x;
        else val = cmake<C>(x, 0.0);
      }
    }
    s[r * a.stride + padi(c)] = val;
  }
  __syncthreads();
  const C* res = fft_any<R, VPT, -1>(s, s2, a.B, a.logL, a.stride, tw);
  // window columns, transposed: T[p][j][b]
  C* Tp = T + (int64_t)p * a.S * M;
  for (int idx = threadIdx.x; idx < a.B * a.S; idx += kFftThreads) {
    const int r = idx % a.B, j = idx / a.B;
    const int b = b0 + r;
    const int col = a.lo + j;
    if (b < M) Tp[(int64_t)j * M + b] = (col < L) ? res[r * a.stride + padi(col)] : cmake<C>(0.0, 0.0);
  }
  __syncthreads();
}


template <typename R, int VPT>
__device__ __forceinline__ void inv_rows_block(KArgs a, const cplx<R>* __restrict__ T,
                                                          R* __restrict__ img, double scale, int accumulate,
                                                          const cplx<R>* __restrict__ tw,
    cplx<R>* s, cplx<R>* s2, int bx, int by) {
  using C = cplx<R>;
  const int b0 = bx * a.B;
  const int L = a.L, M = a.M, half = M / 2;
  const int nout = a.B * M;
  const R* corr = static_cast<const R*>(a.corr);
  const R rscale = (R)scale;
  // planes [pb, pe) into image `by` of the output (a.pg > 0: one partial sum
  // per group of planes, summed by the caller)
  const int pb = a.pg > 0 ? by * a.pg : 0;
  const int pe = a.pg > 0 ? pb + a.pg : a.nplanes;
  if (a.pg > 0) img += (int64_t)by * M * M;
  // with several planes and at most KO outputs per thread, the sum over the
  // planes is kept in registers and the image written once
  constexpr int KO = VPT == 0 ? kPingPongVals<R> : 1;
  const bool regacc = VPT == 0 && pe - pb > 1 && nout <= kFftThreads * KO;
  R acc[KO];
#pragma unroll
  for (int k = 0; k < KO; ++k) acc[k] = R(0);
  for (int p = pb; p < pe; ++p) {
    const C* Tp = T + (int64_t)p * a.S * M;
  #pragma unroll 4
  for (int idx = threadIdx.x; idx < a.B * L; idx += kFftThreads) {
      const int r = idx >> a.logL, c = idx & (L - 1);
      s[r * a.stride + padi(c)] = cmake<C>(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int idx = threadIdx.x; idx < a.B * a.S; idx += kFftThreads) {
      const int r = idx % a.B, j = idx / a.B;
      const int b = b0 + r, col = a.lo + j;
      if (b < M && col < L) s[r * a.stride + padi(col)] = Tp[(int64_t)j * M + b];
    }
    if (a.herm) {
      // real output: the window holds k_u in [-L/2, 0] (columns 0 .. L/2);
      // column c > L/2 (k_u > 0) is the conjugate of column L - c
      for (int idx = threadIdx.x; idx < a.B * (L - a.S); idx += kFftThreads) {
        const int r = idx % a.B, c = a.S + idx / a.B;
        const int b = b0 + r;
        if (b < M) {
          C v = Tp[(int64_t)(L - c) * M + b];
          v.y = -v.y;
          s[r * a.stride + padi(c)] = v;
        }
      }
    }
    __syncthreads();
    const C* res = fft_any<R, VPT, +1>(s, s2, a.B, a.logL, a.stride, tw);
    const double wp = a.w0 + p * a.dw;
    const C* scr = a.mode == kFacPhase && a.screen ? static_cast<const C*>(a.screen) + (int64_t)p * M * M : nullptr;
    // plane p's contribution to output value idx of the CTA's rows
    auto plane_value = [&](int idx, int64_t& pix) -> R {
      const int r = idx / M, aa = idx - r * M;
      const int b = b0 + r;
      pix = (int64_t)b * M + aa;
      const C z = res[r * a.stride + padi((aa - half) & (L - 1))];
      R v;
      if (scr) {
        // Re(z conj(t)) with t = corr exp(-2 pi i w_p (n-1)): corr folded in
        const C t = scr[pix];
        v = z.x * t.x + z.y * t.y;
      } else if (a.mode == kFacPhase) {
        const C e = wscreen<R, +1>(wp, a.nm1[pix]);
        v = z.x * e.x - z.y * e.y;
      } else {
        v = z.x;
      }
      v *= rscale;
      if ((aa + b) & 1) v = -v;
      if (a.mode != kFacNone && !scr) v *= corr[pix];
      return v;
    };
    if (regacc) {
      // the planes' sum stays in registers (thread-owned outputs)
#pragma unroll
      for (int k = 0; k < KO; ++k) {
        const int idx = threadIdx.x + k * kFftThreads;
        if (idx < nout && b0 + idx / M < M) {
          int64_t pix;
          acc[k] += plane_value(idx, pix);
        }
      }
    } else {
      // the output image accumulates the planes; the first plane initialises it
      for (int idx = threadIdx.x; idx < nout; idx += kFftThreads) {
        if (b0 + idx / M >= M) continue;
        int64_t pix;
        const R v = plane_value(idx, pix);
        img[pix] = (p == pb && !accumulate) ? v : img[pix] + v;
      }
    }
    __syncthreads();
  }
  if (regacc) {
#pragma unroll
    for (int k = 0; k < KO; ++k) {
      const int idx = threadIdx.x + k * kFftThreads;
      const int r = idx / M, b = b0 + r;
      if (idx < nout && b < M) {
        const int64_t pix = (int64_t)b * M + (idx - r * M);
        img[pix] = accumulate ? img[pix] + acc[k] : acc[k];
      }
    }
  }
  __syncthreads();
}


// --------------------------------------------------------- column passes ----
template <typename R>
__device__ __forceinline__ void load_column_from_T(const KArgs& a, cplx<R>* s, const cplx<R>* __restrict__ Tp,
                                                   int j0) {
  using C = cplx<R>;
  const int L = a.L, M = a.M, half = M / 2;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < a.B * L; idx += kFftThreads) {
    const int r = idx >> a.logL, c = idx & (L - 1);
    const int j = j0 + r;
    const int bp = c < L / 2 ? c : c - L;
    C val = cmake<C>(0.0, 0.0);
    if (j < a.S && bp >= -half && bp < half) val = Tp[(int64_t)j * M + bp + half];
    s[r * a.stride + padi(c)] = val;
  }
}

template <typename R>
__device__ __forceinline__ void store_column_to_T(const KArgs& a, const cplx<R>* s, cplx<R>* __restrict__ Tp,
                                                  int j0) {
  const int L = a.L, M = a.M, half = M / 2;
  for (int idx = threadIdx.x; idx < a.B * M; idx += kFftThreads) {
    const int r = idx / M, b = idx - r * M;
    const int j = j0 + r;
    if (j < a.S) Tp[(int64_t)j * M + b] = s[r * a.stride + padi((b - half) & (L - 1))];
  }
}

template <typename R>
__device__ __forceinline__ cplx<R> spec_op(int op, cplx<R> x, const void* tab, const void* tab2, int64_t k) {
  using C = cplx<R>;
  if (op == kOpMulReal) {
    const R t = static_cast<const R*>(tab)[k];
    return x * t;
  } else if (op == kOpMulCplx) {
    return cmul(x, static_cast<const C*>(tab)[k]);
  } else if (op == kOpAxpyReal) {
    const R t = static_cast<const R*>(tab)[k];
    return x * t - static_cast<const C*>(tab2)[k];
  }
  return x;
}

template <typename R, int VPT>
__device__ __forceinline__ void fwd_cols_block(KArgs a, const cplx<R>* __restrict__ T,
                                                          cplx<R>* __restrict__ spec,
                                                          const cplx<R>* __restrict__ tw,
    cplx<R>* s, cplx<R>* s2, int bx, int by) {
  using C = cplx<R>;
  const int p = by;
  const int j0 = bx * a.B;
  load_column_from_T<R>(a, s, T + (int64_t)p * a.S * a.M, j0);
  __syncthreads();
  const C* res = fft_any<R, VPT, -1>(s, s2, a.B, a.logL, a.stride, tw);
  C* sp = spec + (int64_t)p * a.S * a.S;
  for (int idx = threadIdx.x; idx < a.B * a.S; idx += kFftThreads) {
    const int r = idx / a.S, i = idx - r * a.S;
    const int j = j0 + r, row = a.lo + i;
    if (j < a.S) sp[(int64_t)j * a.S + i] = (row < a.L) ? res[r * a.stride + padi(row)] : cmake<C>(0.0, 0.0);
  }
  __syncthreads();
}


template <typename R, int VPT>
__device__ __forceinline__ void inv_cols_block(KArgs a, const cplx<R>* __restrict__ spec, int op,
                                                          const void* tab, const void* tab2,
                                                          cplx<R>* __restrict__ T,
                                                          const cplx<R>* __restrict__ tw,
    cplx<R>* s, cplx<R>* s2, int bx, int by) {
  using C = cplx<R>;
  const int p = by;
  const int j0 = bx * a.B;
  const C* sp = spec + (int64_t)p * a.S * a.S;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < a.B * a.L; idx += kFftThreads) {
    const int r = idx >> a.logL, c = idx & (a.L - 1);
    const int j = j0 + r, i = c - a.lo;
    C val = cmake<C>(0.0, 0.0);
    if (j < a.S && i >= 0 && i < a.S) {
      const int64_t k = (int64_t)j * a.S + i;
      val = spec_op<R>(op, sp[k], tab, tab2, k);
    }
    s[r * a.stride + padi(c)] = val;
  }
  __syncthreads();
  const C* res = fft_any<R, VPT, +1>(s, s2, a.B, a.logL, a.stride, tw);
  store_column_to_T<R>(a, res, T + (int64_t)p * a.S * a.M, j0);
  __syncthreads();
}


template <typename R, int VPT>
__device__ __forceinline__ void conv_cols_block(KArgs a, const cplx<R>* __restrict__ Tin, int op,
                                                           const void* tab, const void* tab2,
                                                           cplx<R>* __restrict__ Tout,
                                                           const cplx<R>* __restrict__ tw,
    cplx<R>* s, cplx<R>* s2, int bx, int by) {
  using C = cplx<R>;
  const int j0 = bx * a.B;
  load_column_from_T<R>(a, s, Tin, j0);
  __syncthreads();
  C* res = fft_any<R, VPT, -1>(s, s2, a.B, a.logL, a.stride, tw);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < a.B * a.L; idx += kFftThreads) {
    const int r = idx >> a.logL, c = idx & (a.L - 1);
    const int j = j0 + r;
    if (j < a.S) {
      C* e = &res[r * a.stride + padi(c)];
      *e = spec_op<R>(op, *e, tab, tab2, (int64_t)j * a.L + c);
    }
  }
  __syncthreads();
  C* other = (res == s) ? s2 : s;
  const C* res2 = fft_any<R, VPT, +1>(res, other, a.B, a.logL, a.stride, tw);
  store_column_to_T<R>(a, res2, Tout, j0);
  __syncthreads();
}



// ------------------------------------------------------ host-side setup ----
template <typename R>
const cplx<R>* twiddles(const Ctx* ctx) {
  return std::is_same<R, float>::value ? static_cast<const cplx<R>*>(ctx->tw32.p)
                                       : static_cast<const cplx<R>*>(ctx->tw64.p);
}

template <typename R>
KArgs make_args(const XformGeom& g, int B) {
  KArgs a{};
  a.M = g.M; a.L = g.L; a.logL = g.logL; a.lo = g.lo; a.S = g.S; a.nplanes = g.nplanes;
  a.mode = g.mode; a.B = B; a.stride = padded_len(g.L); a.herm = g.herm;
  a.corr = g.corr; a.nm1 = g.nm1; a.w0 = g.w0; a.dw = g.dw;
  a.screen = g.screen;
  a.pg = g.pg;
  return a;
}


// Ping-pong (VPT = 0) whenever two buffers of one row fit; otherwise in place
// with the large values-per-thread setting.
constexpr size_t kSmemCap = 200 * 1024;
template <typename R>
bool use_inplace(int L) { return 2 * (size_t)padded_len(L) * sizeof(cplx<R>) > kSmemCap; }

}  // namespace
}  // namespace rix
