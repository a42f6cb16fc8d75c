// FFT passes with the transform length, the batch and the radix plan fixed at
// compile time, for the persistent minor-cycle loop.  Same Stockham
// (autosort) ping-pong scheme, shared-memory padding and FP64-accurate
// twiddle table as the run-time passes of fft_device.cuh; with every size a
// constant, the 16 operand addresses of a radix item are one base register
// plus immediate offsets and the item loops unroll.
#pragma once

#include "fft_device.cuh"

namespace rix {
namespace {

// radix (log2) of pass `ps` of a length-2^LOGL transform split into
// ceil(LOGL / 4) passes of radix <= 16, the larger radices first
__host__ __device__ constexpr int ct_npass(int logl) { return (logl + 3) / 4; }
__host__ __device__ constexpr int ct_lr(int logl, int ps) {
  int logp = 0, lr = 0;
  for (int q = 0; q <= ps; ++q) {
    const int rem = logl - logp, left = ct_npass(logl) - q;
    lr = (rem + left - 1) / left;
    logp += lr;
  }
  return lr;
}
__host__ __device__ constexpr int ct_logp(int logl, int ps) {
  int logp = 0;
  for (int q = 0; q < ps; ++q) logp += ct_lr(logl, q);
  return logp;
}

// One Stockham pass of radix 2^LR over B rows of length 2^LOGL (row stride
// padded_len(L)): item i of a row, k = i mod p, reads i + r L/RAD, applies
// exp(DIR 2 pi i r k / (p RAD)), writes ((i - k) RAD + k) + r p.
template <typename R, int DIR, int LR, int LOGL, int LOGP, int B>
__device__ __forceinline__ void pass_ct(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                                        const cplx<R>* __restrict__ tw) {
  using C = cplx<R>;
  constexpr int RAD = 1 << LR;
  constexpr int L = 1 << LOGL;
  constexpr int IPR = L / RAD;               // items per row
  constexpr int P = 1 << LOGP;
  constexpr int TOTAL = B * IPR;
  constexpr int NIT = (TOTAL + kFftThreads - 1) / kFftThreads;
  constexpr int STRIDE = padded_len(L);
  constexpr int TWSHIFT = kTwLog - (LOGP + LR);
  // padi(x + r c) == padi(x) + r (c + c / 16) when c is a multiple of 16
  constexpr bool kLinIn = (IPR % 16) == 0;
  // outputs o + r P: linear when P is a multiple of 16, or when all RAD of
  // them stay inside one 16-entry group (P RAD <= 16 and P RAD | 16)
  constexpr bool kLinOut16 = (P % 16) == 0;
  constexpr bool kLinOutSmall = (P * RAD <= 16) && (16 % (P * RAD) == 0);
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int g = threadIdx.x + it * kFftThreads;
    if ((TOTAL % kFftThreads) != 0 && g >= TOTAL) break;
    const int row = g / IPR;
    const int i = g % IPR;
    const int k = i % P;
    const C* rs = src + row * STRIDE;
    C v[RAD];
    if constexpr (kLinIn) {
      const C* b = rs + padi(i);
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[r] = b[r * (IPR + IPR / 16)];
    } else {
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[r] = rs[padi(i + r * IPR)];
    }
    if constexpr (LOGP > 0) {
      if (k) apply_twiddles<R, DIR, RAD>(v, tw, k, TWSHIFT);
    }
    dft<RAD, DIR>(v);
    C* rd = dst + row * STRIDE;
    const int o = ((i - k) << LR) + k;
    if constexpr (kLinOut16) {
      C* b = rd + padi(o);
#pragma unroll
      for (int r = 0; r < RAD; ++r) b[r * (P + P / 16)] = v[r];
    } else if constexpr (kLinOutSmall) {
      C* b = rd + padi(o);
#pragma unroll
      for (int r = 0; r < RAD; ++r) b[r * P] = v[r];
    } else {
#pragma unroll
      for (int r = 0; r < RAD; ++r) rd[padi(o + r * P)] = v[r];
    }
  }
  __syncthreads();
}

template <typename R, int DIR, int LOGL, int B, int PS>
__device__ __forceinline__ void passes_ct(cplx<R>* a, cplx<R>* b, const cplx<R>* __restrict__ tw) {
  if constexpr (PS < ct_npass(LOGL)) {
    pass_ct<R, DIR, ct_lr(LOGL, PS), LOGL, ct_logp(LOGL, PS), B>(a, b, tw);
    passes_ct<R, DIR, LOGL, B, PS + 1>(b, a, tw);
  }
}

// FFT (unnormalised, DIR = -1 forward) of B rows held in `a`; the result ends
// in the buffer returned (a after an even number of passes, else b).  The
// caller has written `a` and synchronised.
template <typename R, int DIR, int LOGL, int B>
__device__ __forceinline__ cplx<R>* fft_ct(cplx<R>* a, cplx<R>* b, const cplx<R>* __restrict__ tw) {
  passes_ct<R, DIR, LOGL, B, 0>(a, b, tw);
  return (ct_npass(LOGL) & 1) ? b : a;
}

}  // namespace
}  // namespace rix
