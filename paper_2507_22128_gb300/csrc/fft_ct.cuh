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

// Pruning for the centred, zero-padded transforms of the minor cycle: the
// data of an N-long row sits at positions [0, L/4) and [3L/4, L) of the
// L = 2N transform (centred) and the rest is zero (kPruneIn), or only those
// positions of the result are read (kPruneOut).  In the first pass (p = 1)
// item i < L/RAD reads i + r L/RAD, which is in the zero half exactly when
// RAD/4 <= r < 3 RAD/4; in the last pass (p = L/RAD) item i writes i + r p,
// needed exactly when r < RAD/4 or r >= 3 RAD/4.  So the loads and stores
// skipped are known at compile time for RAD >= 4.
template <int RAD>
__host__ __device__ constexpr bool ct_outer(int r) { return r < RAD / 4 || r >= 3 * RAD / 4; }

// dft4 with a1 = a2 = 0 (their values are not read)
template <int DIR, typename C>
__device__ __forceinline__ void dft4_z12(C& a0, C& a1, C& a2, C& a3) {
  const C x = a0, r = rot90<DIR>(a3);
  a0 = x + a3; a2 = x - a3; a1 = x - r; a3 = x + r;
}

// dft<RAD, DIR> of v with v[r] = 0 for RAD/4 <= r < 3 RAD/4 (not read): the
// first stage of each decomposition meets those zeros as a1 = a2 of its
// length-4 transforms
template <int RAD, int DIR, typename C>
__device__ __forceinline__ void dft_zin(C* v) {
  if constexpr (RAD == 4) {
    dft4_z12<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (RAD == 8) {
    dft4_z12<DIR>(v[0], v[2], v[4], v[6]);
    dft4_z12<DIR>(v[1], v[3], v[5], v[7]);
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
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4_z12<DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
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

// Input and output hooks of a transform.  The first pass takes its values
// from ld(row, pos) and the last pass hands its results to st(row, pos, v)
// (pos in natural order), instead of reading / writing the ping-pong
// buffers, so loads, scatters and epilogues fuse into the passes; pre() runs
// in every thread before the barrier that ends the second-to-last pass (to
// complete asynchronous copies that the last pass reads).  SmemIO / NoHook
// keep the buffers.
struct SmemIO {};
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// One Stockham pass of radix 2^LR over B rows of length 2^LOGL (row stride
// padded_len(L)): item i of a row, k = i mod p, reads i + r L/RAD, applies
// exp(DIR 2 pi i r k / (p RAD)), writes ((i - k) RAD + k) + r p.
template <typename R, int DIR, int LR, int LOGL, int LOGP, int B, bool kPruneIn = false, bool kPruneOut = false,
          class LD = SmemIO, class ST = SmemIO, class PRE = NoHook, bool kPre = false>
__device__ __forceinline__ void pass_ct(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                                        const cplx<R>* __restrict__ tw, const LD& ld = LD{}, const ST& st = ST{},
                                        const PRE& pre = PRE{}) {
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
  constexpr bool kZin = kPruneIn && LOGP == 0 && RAD >= 4;
  constexpr bool kZout = kPruneOut && LOGP + LR == LOGL && RAD >= 4;
  constexpr bool kLd = LOGP == 0 && !std::is_same<LD, SmemIO>::value;
  constexpr bool kSt = LOGP + LR == LOGL && !std::is_same<ST, SmemIO>::value;
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int g = threadIdx.x + it * kFftThreads;
    if ((TOTAL % kFftThreads) != 0 && g >= TOTAL) break;
    const int row = g / IPR;
    const int i = g % IPR;
    const int k = i % P;
    const C* rs = src + row * STRIDE;
    C v[RAD];
    if constexpr (kLd) {
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZin || ct_outer<RAD>(r)) v[r] = ld(row, i + r * IPR);
    } else if constexpr (kLinIn) {
      const C* b = rs + padi(i);
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZin || ct_outer<RAD>(r)) v[r] = b[r * (IPR + IPR / 16)];
    } else {
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZin || ct_outer<RAD>(r)) v[r] = rs[padi(i + r * IPR)];
    }
    if constexpr (LOGP > 0) {
      if (k) apply_twiddles<R, DIR, RAD>(v, tw, k, TWSHIFT);
    }
    if constexpr (kZin) dft_zin<RAD, DIR>(v);
    else dft<RAD, DIR>(v);
    C* rd = dst + row * STRIDE;
    const int o = ((i - k) << LR) + k;
    if constexpr (kSt) {
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZout || ct_outer<RAD>(r)) st(row, o + r * P, v[r]);
    } else if constexpr (kLinOut16) {
      C* b = rd + padi(o);
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZout || ct_outer<RAD>(r)) b[r * (P + P / 16)] = v[r];
    } else if constexpr (kLinOutSmall) {
      C* b = rd + padi(o);
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZout || ct_outer<RAD>(r)) b[r * P] = v[r];
    } else {
#pragma unroll
      for (int r = 0; r < RAD; ++r)
        if (!kZout || ct_outer<RAD>(r)) rd[padi(o + r * P)] = v[r];
    }
  }
  if constexpr (kPre) pre();
  __syncthreads();
}

template <typename R, int DIR, int LOGL, int B, int PS, bool kPruneIn, bool kPruneOut, class LD, class ST, class PRE>
__device__ __forceinline__ void passes_ct(cplx<R>* a, cplx<R>* b, const cplx<R>* __restrict__ tw, const LD& ld,
                                          const ST& st, const PRE& pre) {
  if constexpr (PS < ct_npass(LOGL)) {
    pass_ct<R, DIR, ct_lr(LOGL, PS), LOGL, ct_logp(LOGL, PS), B, kPruneIn, kPruneOut, LD, ST, PRE,
            PS == ct_npass(LOGL) - 2>(a, b, tw, ld, st, pre);
    passes_ct<R, DIR, LOGL, B, PS + 1, kPruneIn, kPruneOut>(b, a, tw, ld, st, pre);
  }
}

// FFT (unnormalised, DIR = -1 forward) of B rows held in `a`; the result ends
// in the buffer returned (a after an even number of passes, else b).  The
// caller has written `a` and synchronised.  kPruneIn: only the centred
// positions [0, L/4) and [3L/4, L) of `a` hold data (the rest is zero and
// need not be written); kPruneOut: only those positions of the result are
// valid.
// With hooks (ld, st, pre as described above pass_ct), `a` need not be
// written before the call when ld is given, and the result buffer is not
// written when st is given.
template <typename R, int DIR, int LOGL, int B, bool kPruneIn = false, bool kPruneOut = false, class LD = SmemIO,
          class ST = SmemIO, class PRE = NoHook>
__device__ __forceinline__ cplx<R>* fft_ct(cplx<R>* a, cplx<R>* b, const cplx<R>* __restrict__ tw, const LD& ld = LD{},
                                           const ST& st = ST{}, const PRE& pre = PRE{}) {
  static_assert(!(kPruneIn || kPruneOut) || (ct_lr(LOGL, 0) >= 2 && ct_lr(LOGL, ct_npass(LOGL) - 1) >= 2),
                "pruning needs radix >= 4 at both ends");
  static_assert(ct_npass(LOGL) >= 2, "hooks assume at least two passes");
  passes_ct<R, DIR, LOGL, B, 0, kPruneIn, kPruneOut>(a, b, tw, ld, st, pre);
  return (ct_npass(LOGL) & 1) ? b : a;
}

}  // namespace
}  // namespace rix
