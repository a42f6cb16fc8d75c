// a10: the FISTA minor cycles (Eq. 4-5) of one or more partitions as one
// persistent cooperative kernel per call, compiled for each transform length
// 2N and dictionary.
//
// Every iteration is a chain of phases; k_fista_loop separates them by a
// bounded grid barrier, k_fista_flow (a batch of Db4 loops) by per-loop
// stage counters in a dataflow schedule:
//   synthesis   x = W y, coarsest level first: with Db4, levels levels-1 .. 1
//               in one phase (syn_chain_tile) and the finest inside the row
//               phase (rows_fwd_syn_unit); otherwise one phase per level;
//   rows        F of the rows of pad(x), two real rows per complex transform,
//               window columns k_u in [-N, 0] written transposed (ta);
//   columns     per window column: F, Mx X, F^-1, crop  (ta -> tb; tb in
//               blocks of the 2B image rows of one row unit, tb_index);
//   rows        F^-1 of the rows (Hermitian completion, two real rows per
//               complex transform), crop, minus the constant image d:
//               g = 2 crop F^-1 [Mx F pad x] - d,  d = 2 crop F^-1 C,
//               which equals 2 crop F^-1 [Mx F pad x - C] (the transforms
//               and the crop are linear); d is formed once per launch, by
//               the column and row phases run on C before the first
//               iteration, so the iterations read N^2 values of d instead of
//               (N + 1) 2N values of C.
//   analysis    W^T g, one phase per level, with the thresholded,
//               momentum-accelerated step fused into the final coefficients.
// Phases hand their units (wavelet tiles, row pairs, column batches) out over
// the CTAs.  All image-sized buffers stay in L2 between phases.
//
// With the concatenated dictionary (db1 .. db8, scaled by 1/sqrt 8) every
// wavelet phase runs the levels of all eight members at once (units =
// member x tile), the row phase sums the members' syntheses, and a last
// synthesis of alpha writes the minor cycle's image.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fft_ct.cuh"
#include "grid_sync.cuh"
#include "wavelet_device.cuh"

namespace rix {
namespace {

// analysis block side: 32 at the fine levels with FP32 and Db4 (at least 256
// blocks per loop; with fewer, the smaller blocks keep more CTAs busy), kTB
// otherwise
template <typename R, int DICT>
__host__ __device__ constexpr int ana_fine_block() {
  return sizeof(R) == 4 && DICT == RIX_DICT_DB4 ? 32 : kTB;
}
// block side of the chained coarse synthesis (the level-1 output per unit)
template <typename R>
__host__ __device__ constexpr int chain_block() {
  return 32;
}

template <typename R, int DICT>
__device__ __forceinline__ int ana_block(int h) {
  constexpr int TBF = ana_fine_block<R, DICT>();
  return (TBF != kTB && (h / TBF) * (h / TBF) >= 256) ? TBF : kTB;
}

template <typename R, int LOGL, int DICT = RIX_DICT_DB4>
struct FistaShape {
  static constexpr int L = 1 << LOGL;
  static constexpr int N = L / 2;          // image side
  static constexpr int H = N / 2;
  static constexpr int S = N + 1;          // window columns k_u = -N .. 0
  static constexpr int STRIDE = padded_len(L);
  static constexpr int kVals = kPingPongVals<R> * kFftThreads;
  // complex rows per unit: one pass of the ping-pong FFT holds kVals values;
  // the row phases pack two real rows into each, so 2 B <= N
  static constexpr int B0 = kVals / L > 0 ? kVals / L : 1;
  static constexpr int B = B0 < N / 2 ? B0 : N / 2;
  static constexpr int kRowUnits = N / (2 * B);
  static constexpr int kColUnits = (S + B - 1) / B;
  static constexpr size_t kFftSmem = 2 * (size_t)B * STRIDE * sizeof(cplx<R>);
  // a unit's slice of Mx (B window columns of length L) or of d (2B rows of
  // N), copied asynchronously while the unit's transform runs
  static constexpr size_t kStage = (size_t)B * L * sizeof(R);
  static constexpr int KMAX = DICT == RIX_DICT_DB4 ? 8 : kMaxTaps;
  // analysis block side of the fine levels (kTB at the coarse ones; and with
  // FP64, for shared memory)
  static constexpr int TBF = ana_fine_block<R, DICT>();
  static constexpr size_t kDwtSmem = sizeof(DwtSmem<R, TBF, KMAX>) > sizeof(DwtSmem<R, kTB, KMAX>)
                                         ? sizeof(DwtSmem<R, TBF, KMAX>)
                                         : sizeof(DwtSmem<R, kTB, KMAX>);
  static constexpr size_t kIdwtSmem = sizeof(IdwtSmem<R, KMAX>) > chain_smem_bytes<R, chain_block<R>(), 8>()
                                          ? sizeof(IdwtSmem<R, KMAX>)
                                          : chain_smem_bytes<R, chain_block<R>(), 8>();
  static constexpr size_t kWavSmem = kDwtSmem > kIdwtSmem ? kDwtSmem : kIdwtSmem;
  static constexpr size_t kSmem = kFftSmem + kStage > kWavSmem ? kFftSmem + kStage : kWavSmem;
};

template <typename C> __device__ __forceinline__ C cpx(typename std::conditional<sizeof(C) == 8, float, double>::type re,
                                                       typename std::conditional<sizeof(C) == 8, float, double>::type im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}

// Layout of tb (the column phase's output, the inverse row phase's input):
// blocks of the 2B image rows that one row unit transforms, each block
// [window column j][row b mod 2B], so that a row unit reads one contiguous
// block; the column phase writes 2B-element runs instead.
template <typename F>
__device__ __forceinline__ int64_t tb_index(int j, int b) {
  constexpr int RB = 2 * F::B;
  return (int64_t)(b / RB) * (F::S * RB) + j * RB + (b % RB);
}

// a pair of complex values at 16-byte-aligned memory (one 16-byte access in
// FP32)
template <typename C>
__device__ __forceinline__ void ld_pair(const C* p, C& a, C& b) {
  if constexpr (sizeof(C) == 8) {
    const float4 w = *reinterpret_cast<const float4*>(p);
    a.x = w.x; a.y = w.y; b.x = w.z; b.y = w.w;
  } else {
    a = p[0];
    b = p[1];
  }
}
template <typename C>
__device__ __forceinline__ void st_pair(C* p, const C& a, const C& b) {
  if constexpr (sizeof(C) == 8) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// `bytes` (a multiple of 16; both addresses 16-byte aligned) from src to dst
__device__ __forceinline__ void stage_async(void* dst, const void* src, int bytes) {
  for (int o = threadIdx.x * 16; o < bytes; o += kFftThreads * 16)
    cp_async16(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o);
}

// rows b0 .. b0 + 2B of x -> window columns of their spectra, T[j][b];
// x = xscale * (sum of NSUM images xstride apart) when NSUM > 1
template <typename R, int LOGL, int NSUM = 1>
__device__ __forceinline__ void rows_fwd_unit(const R* __restrict__ x, int64_t xstride, R xscale,
                                              cplx<R>* __restrict__ T, const cplx<R>* __restrict__ tw, cplx<R>* s,
                                              cplx<R>* s2, int u) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL>;
  constexpr int L = F::L, N = F::N, H = F::H, B = F::B, STRIDE = F::STRIDE;
  const int b0 = u * 2 * B;
  // complex row q = x[b0 + 2q] + i x[b0 + 2q + 1], centred: pixel a sits at
  // grid column (a - N/2) mod L with sign (-1)^(a + b)
  constexpr int NE = B * N;
  constexpr int NLD = (NE + kFftThreads - 1) / kFftThreads;
  R va[NLD], vb[NLD];
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int e = threadIdx.x + k * kFftThreads;
    if (NE % kFftThreads == 0 || e < NE) {
      const int q = e / N, a = e % N;
      const int64_t row = b0 + 2 * q;
      if constexpr (NSUM == 1) {
        va[k] = x[row * N + a];
        vb[k] = x[(row + 1) * N + a];
      } else {
        R sa = R(0), sb = R(0);
#pragma unroll
        for (int m = 0; m < NSUM; ++m) {
          sa += x[m * xstride + row * N + a];
          sb += x[m * xstride + (row + 1) * N + a];
        }
        va[k] = xscale * sa;
        vb[k] = xscale * sb;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int e = threadIdx.x + k * kFftThreads;
    if (NE % kFftThreads == 0 || e < NE) {
      const int q = e / N, a = e % N;
      const bool odd = (a + b0) & 1;               // b0 + 2q has the parity of b0
      s[q * STRIDE + padi((a - H) & (L - 1))] = cpx<C>(odd ? -va[k] : va[k], odd ? vb[k] : -vb[k]);
    }
  }
  __syncthreads();
  // the zero padding (columns N/2 .. 3N/2 - 1) is never read: pruned input
  const C* res = fft_ct<R, -1, LOGL, B, true, false>(s, s2, tw);
  // X_a[j] = (Z[j] + conj Z[-j]) / 2,  X_b[j] = (Z[j] - conj Z[-j]) / 2i
  constexpr int NO = B * F::S;
  for (int e = threadIdx.x; e < NO; e += kFftThreads) {
    const int q = e % B, j = e / B;
    const C z = res[q * STRIDE + padi(j)];
    const C w = res[q * STRIDE + padi((L - j) & (L - 1))];
    const R h = R(0.5);
    st_pair(T + (int64_t)j * N + b0 + 2 * q, cpx<C>(h * (z.x + w.x), h * (z.y - w.y)),
            cpx<C>(h * (z.y + w.y), h * (w.x - z.x)));
  }
  __syncthreads();
}

// rows_fwd_unit with the finest synthesis level fused in (Db4): rows b0 ..
// b0 + 2B of x = W y are synthesised from the level-1 LL block `ll` and the
// level-0 detail subbands of `coef` (N x N buffers, Mallat layout) straight
// into the transform's input, so x is never written.  The level is separable
// and its two passes commute; the columns go first, into tv (shared memory):
//   tv[cx][r][k] = sum_j lo(2j + m&1) Q(0,cx)[(m>>1) - j][k]
//                      + hi(2j + m&1) Q(1,cx)[(m>>1) - j][k],   m = b0 + r,
// then the rows: x[m][c] = sum_j lo(2j + c&1) tv[0][r][(c>>1) - j]
//                               + hi(2j + c&1) tv[1][r][(c>>1) - j],
// indices periodic modulo N/2; Q(cy,cx) is subband (cy, cx) of the level.
template <typename R, int LOGL>
__device__ __forceinline__ void rows_fwd_syn_unit(const R* __restrict__ ll, const R* __restrict__ coef,
                                                  cplx<R>* __restrict__ T, const cplx<R>* __restrict__ tw, cplx<R>* s,
                                                  cplx<R>* s2, R* tv, int u) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL>;
  constexpr int L = F::L, N = F::N, H = F::H, B = F::B, STRIDE = F::STRIDE;
  static_assert(2 * B * N * sizeof(R) <= F::kStage, "tv exceeds the stage");
  const Db4Taps<R> tp;
  const int b0 = u * 2 * B;
  const int k0 = b0 >> 1;
  // columns: thread per (cx, k), a window of four coefficient rows per
  // subband sliding down the unit's row pairs
  for (int col = threadIdx.x; col < N; col += kFftThreads) {
    const int cx = col / H, k = col - cx * H;
    const R* q0 = cx == 0 ? ll + k : coef + H + k;              // Q(0, cx), row km at km N
    const R* q1 = coef + (int64_t)H * N + cx * H + k;           // Q(1, cx)
    R w0[4], w1[4];                                             // rows k0 + pr - 3 .. k0 + pr
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int km = (k0 - 3 + i) & (H - 1);
      w0[i] = q0[(int64_t)km * N];
      w1[i] = q1[(int64_t)km * N];
    }
#pragma unroll
    for (int pr = 0; pr < B; ++pr) {
      const int km = (k0 + pr) & (H - 1);
      w0[3] = q0[(int64_t)km * N];
      w1[3] = q1[(int64_t)km * N];
      R ev = R(0), od = R(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ev += tp.lo(2 * j) * w0[3 - j] + tp.hi(2 * j) * w1[3 - j];
        od += tp.lo(2 * j + 1) * w0[3 - j] + tp.hi(2 * j + 1) * w1[3 - j];
      }
      tv[(cx * 2 * B + 2 * pr) * H + k] = ev;
      tv[(cx * 2 * B + 2 * pr + 1) * H + k] = od;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        w0[i] = w0[i + 1];
        w1[i] = w1[i + 1];
      }
    }
  }
  __syncthreads();
  // rows, computed by the transform's first pass as it loads them: complex
  // row q = x[b0 + 2q] + i x[b0 + 2q + 1], centred as in rows_fwd_unit
  // (position p holds column (p + N/2) mod L; the pruned half is zero)
  auto ld_x = [&](int q, int p) -> C {
    const int c = (p + H) & (L - 1);
    const int kc = c >> 1;
    const bool oc = c & 1;
    const R* t0a = tv + (2 * q) * H;                  // cx = 0, row 2q
    const R* t1a = tv + (2 * B + 2 * q) * H;          // cx = 1, row 2q
    R va = R(0), vb = R(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int kk = (kc - j) & (H - 1);
      const R lo = oc ? tp.lo(2 * j + 1) : tp.lo(2 * j);
      const R hi = oc ? tp.hi(2 * j + 1) : tp.hi(2 * j);
      va += lo * t0a[kk] + hi * t1a[kk];
      vb += lo * t0a[H + kk] + hi * t1a[H + kk];
    }
    const bool odd = (c + b0) & 1;
    return cpx<C>(odd ? -va : va, odd ? vb : -vb);
  };
  const C* res = fft_ct<R, -1, LOGL, B, true, false>(s, s2, tw, ld_x);
  constexpr int NO = B * F::S;
  for (int e = threadIdx.x; e < NO; e += kFftThreads) {
    const int q = e % B, j = e / B;
    const C z = res[q * STRIDE + padi(j)];
    const C w = res[q * STRIDE + padi((L - j) & (L - 1))];
    const R h = R(0.5);
    st_pair(T + (int64_t)j * N + b0 + 2 * q, cpx<C>(h * (z.x + w.x), h * (z.y - w.y)),
            cpx<C>(h * (z.y + w.y), h * (w.x - z.x)));
  }
  __syncthreads();
}

// window columns j0 .. j0 + B: F, Mx X, F^-1, crop to the image rows.  The
// forward transform's first pass reads the columns from Tin, the inverse's
// first pass multiplies by Mx as it loads and its last pass writes the
// cropped rows to Tout (tb_index layout); the unit's Mx (rows j0 .. j0 + B of the table,
// contiguous) is copied to shared memory during the forward transform.
template <typename R, int LOGL>
__device__ __forceinline__ void cols_conv_unit(const cplx<R>* __restrict__ Tin, const R* __restrict__ mx,
                                               cplx<R>* __restrict__ Tout, const cplx<R>* __restrict__ tw,
                                               cplx<R>* s, cplx<R>* s2, R* stage, int u) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL>;
  constexpr int L = F::L, N = F::N, H = F::H, B = F::B, S = F::S, STRIDE = F::STRIDE;
  const int j0 = u * B;
  // rows j0 .. j0 + B - 1 < L of the L x L table: in bounds even past S
  stage_async(stage, mx + (int64_t)j0 * L, (int)F::kStage);
  // centred: position p holds image row (p + N/2) mod L; the pruned half is zero
  auto ld_in = [&](int q, int p) -> C {
    const int j = j0 + q;
    return j < S ? Tin[(int64_t)j * N + ((p + H) & (L - 1))] : cpx<C>(R(0), R(0));
  };
  auto wait = [] { cp_async_wait_all(); };
  C* res = fft_ct<R, -1, LOGL, B, true, false>(s, s2, tw, ld_in, SmemIO{}, wait);
  const C* rin = res;
  auto ld_mul = [&](int q, int p) -> C {
    const C z = rin[q * STRIDE + padi(p)];
    const R m = stage[q * L + p];
    return cpx<C>(z.x * m, z.y * m);
  };
  auto st_out = [&](int q, int p, const C& v) {
    const int j = j0 + q;
    if (j < S) Tout[tb_index<F>(j, (p + H) & (L - 1))] = v;
  };
  C* other = (res == s) ? s2 : s;
  fft_ct<R, +1, LOGL, B, false, true>(res, other, tw, ld_mul, st_out);
}

// window columns j0 .. j0 + B of a full-length spectrum (C[j][c], c < L):
// F^-1, crop to the image rows (the first half of d = 2 crop F^-1 C)
template <typename R, int LOGL>
__device__ __forceinline__ void cols_inv_unit(const cplx<R>* __restrict__ Cs, cplx<R>* __restrict__ Tout,
                                              const cplx<R>* __restrict__ tw, cplx<R>* s, cplx<R>* s2, int u) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL>;
  constexpr int L = F::L, N = F::N, H = F::H, B = F::B, S = F::S;
  const int j0 = u * B;
  auto ld_c = [&](int q, int p) -> C {
    const int j = j0 + q;
    return j < S ? Cs[(int64_t)j * L + p] : cpx<C>(R(0), R(0));
  };
  auto st_out = [&](int q, int p, const C& v) {
    const int j = j0 + q;
    if (j < S) Tout[tb_index<F>(j, (p + H) & (L - 1))] = v;
  };
  fft_ct<R, +1, LOGL, B, false, true>(s, s2, tw, ld_c, st_out);
}

// rows b0 .. b0 + 2B of g = scale * crop F^-1 [spectrum] (minus the same rows
// of d when kSubD: they are staged in shared memory during the transform),
// the spectrum given by its window columns k_u in [-N, 0] (T, tb_index
// layout: the unit's block is contiguous) and Hermitian symmetry; the last
// pass writes g.
template <typename R, int LOGL, bool kSubD>
__device__ __forceinline__ void rows_inv_unit(const cplx<R>* __restrict__ T, R* __restrict__ g, R scale,
                                              const R* __restrict__ d, const cplx<R>* __restrict__ tw, cplx<R>* s,
                                              cplx<R>* s2, R* stage, int u) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL>;
  constexpr int L = F::L, N = F::N, H = F::H, B = F::B, S = F::S, STRIDE = F::STRIDE;
  const int b0 = u * 2 * B;
  static_assert(2 * B * N * sizeof(R) <= F::kStage, "d rows exceed the stage");
  if constexpr (kSubD) stage_async(stage, d + (int64_t)b0 * N, 2 * B * N * (int)sizeof(R));
  // Z = Y_a + i Y_b over all columns: Z[c] from window column c and
  // Z[L - c] = conj Y_a[c] + i conj Y_b[c]; the self-conjugate columns 0 and
  // N keep their real parts (the imaginary parts only feed Im F^-1 Y)
  const C* blk = T + tb_index<F>(0, b0);
  constexpr int NE = B * S;
  constexpr int NLD = (NE + kFftThreads - 1) / kFftThreads;
  C ya[NLD], yb[NLD];
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int e = threadIdx.x + k * kFftThreads;
    if (e < NE) ld_pair(blk + 2 * e, ya[k], yb[k]);   // column e / B, rows 2 (e % B) and 2 (e % B) + 1
  }
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int e = threadIdx.x + k * kFftThreads;
    if (e < NE) {
      const int q = e % B, c = e / B;
      C a = ya[k], b = yb[k];
      if (c == 0 || c == N) {
        a.y = R(0);
        b.y = R(0);
      }
      s[q * STRIDE + padi(c)] = cpx<C>(a.x - b.y, a.y + b.x);
      if (c != 0 && c != N) s[q * STRIDE + padi(L - c)] = cpx<C>(a.x + b.y, b.x - a.y);
    }
  }
  __syncthreads();
  // crop (position p holds column (p + N/2) mod L), centring sign, scale
  auto st_g = [&](int q, int p, const C& z) {
    const int a = (p + H) & (L - 1);
    const int64_t row = b0 + 2 * q;
    const bool odd = (a + b0) & 1;
    const R va = z.x * scale, vb = z.y * scale;
    R ga = odd ? -va : va, gb = odd ? vb : -vb;
    if constexpr (kSubD) {
      ga -= stage[2 * q * N + a];
      gb -= stage[(2 * q + 1) * N + a];
    }
    g[row * N + a] = ga;
    g[(row + 1) * N + a] = gb;
  };
  auto wait = [] {
    if constexpr (kSubD) cp_async_wait_all();
  };
  fft_ct<R, +1, LOGL, B, false, true>(s, s2, tw, SmemIO{}, st_g, wait);
}

// member MM of the concatenated dictionary (db_{MM+1}, 2 (MM + 1) taps),
// out of line: each member's tile gets its own register allocation
template <typename R, int MM>
__device__ __noinline__ void syn_member(const R* ll, const R* cm, int n, R* dst, int N, int bx, int by,
                                        unsigned char* smem, const R* taps) {
  auto& ism = *reinterpret_cast<IdwtSmem<R, 2 * (MM + 1)>*>(smem);
  idwt_tile<R>(ll, cm, n, dst, N, bx, by, ism, RefTaps<R, 2 * (MM + 1)>{taps});
}
template <typename R, int MM>
__device__ __noinline__ void ana_member(const R* src, int n, R* dst, int N, int last, const StepArgs<R>& sm,
                                        int bx, int by, unsigned char* smem, const R* taps) {
  auto& dsm = *reinterpret_cast<DwtSmem<R, kTB, 2 * (MM + 1)>*>(smem);
  dwt_tile<R, kTB, true>(src, N, n, nullptr, dst, N, last, sm, bx, by, dsm, RefTaps<R, 2 * (MM + 1)>{taps});
}

// iterations whose FISTA momentum travels in the launch arguments
constexpr int kMomTab = 256;

template <typename R>
struct FistaArgs {
  FistaLoop<R> f[kMaxPart];   // the batch's loops, [0, nb)
  int nb;
  R gscale;
  R taps[8][16];              // RIX_DICT_DB1_8: low-pass filters of db1 .. db8
  // dataflow schedule (k_fista_flow): ticket counter, completed units per
  // loop and stage ([loop][stage], zeroed before the launch), momentum per
  // iteration
  unsigned int* ticket;
  unsigned int* done;
  const R* mom;           // device table, or null: mom_tab holds the iterations
  R mom_tab[kMomTab];
};

// units of one wavelet level of one loop: tiles of side `tile` over an n x n
// block, times the eight members with the concatenated dictionary
template <int DICT>
__device__ __forceinline__ int level_units(int n, int tile) {
  const int nt = (n + tile - 1) / tile;
  return (DICT == RIX_DICT_DB4 ? 1 : 8) * nt * nt;
}

// unit t of synthesis level l of x = W c for loop f: level l of member m
// reads its level-l+1 output (or c's coarse block at the top level) and lands
// in (l odd ? B : A) (Db4: tmp : x)
template <typename R, int DICT, int N>
__device__ __forceinline__ void synthesis_unit(const FistaLoop<R>& f, const R* coef, int l, int t,
                                               unsigned char* smem, const R (&taps)[8][16]) {
  const int n = N >> l, nt = (n + kTS - 1) / kTS, per = nt * nt;
  const bool top = l == f.levels - 1;
  if constexpr (DICT == RIX_DICT_DB4) {
    const R* ll = top ? coef : (((l + 1) & 1) ? f.tmp : f.x);
    R* dst = (l & 1) ? f.tmp : f.x;
    auto& ism = *reinterpret_cast<IdwtSmem<R, 8>*>(smem);
    idwt_tile<R>(ll, coef, n, dst, N, t % nt, t / nt, ism, Db4Taps<R>{});
  } else {
    const int64_t NN = (int64_t)N * N;
    const int m = t / per, tt = t - m * per;
    const R* cm = coef + m * NN;
    R* am = f.xs + m * NN;
    R* bm = f.bs + m * NN;
    const R* ll = top ? cm : (((l + 1) & 1) ? bm : am);
    R* dst = (l & 1) ? bm : am;
    const int bx = tt % nt, by = tt / nt;
#define RIX_SYN(MM)                                                                                     \
  case MM: syn_member<R, MM>(ll, cm, n, dst, N, bx, by, smem, taps[MM]); break;
    switch (m) { RIX_SYN(0) RIX_SYN(1) RIX_SYN(2) RIX_SYN(3) RIX_SYN(4) RIX_SYN(5) RIX_SYN(6) RIX_SYN(7) }
#undef RIX_SYN
  }
}

// unit t of analysis level l of W^T g with the step fused into the final
// coefficients, for loop f: level l of member m reads g (l = 0) or its level
// l-1 LL and writes its LL into (l odd ? B : A) (Db4: tmp : x)
template <typename R, int DICT, int N>
__device__ __forceinline__ void analysis_unit(const FistaLoop<R>& f, int l, int t, const StepArgs<R>& sa,
                                              unsigned char* smem, const R (&taps)[8][16]) {
  const int n = N >> l, tb = ana_block<R, DICT>(n / 2), nt = (n / 2 + tb - 1) / tb, per = nt * nt;
  const int last = l == f.levels - 1;
  if constexpr (DICT == RIX_DICT_DB4) {
    const R* src = l == 0 ? f.g : (((l - 1) & 1) ? f.tmp : f.x);
    R* dst = (l & 1) ? f.tmp : f.x;
    constexpr int TBF = ana_fine_block<R, DICT>();
    if (TBF != kTB && tb == TBF) {
      auto& dsm = *reinterpret_cast<DwtSmem<R, TBF, 8>*>(smem);
      dwt_tile<R, TBF, true>(src, N, n, nullptr, dst, N, last, sa, t % nt, t / nt, dsm, Db4Taps<R>{});
    } else {
      auto& dsm = *reinterpret_cast<DwtSmem<R, kTB, 8>*>(smem);
      dwt_tile<R, kTB, true>(src, N, n, nullptr, dst, N, last, sa, t % nt, t / nt, dsm, Db4Taps<R>{});
    }
  } else {
    const int64_t NN = (int64_t)N * N;
    const int m = t / per, tt = t - m * per;
    R* am = f.xs + m * NN;
    R* bm = f.bs + m * NN;
    const R* src = l == 0 ? f.g : (((l - 1) & 1) ? bm : am);
    R* dst = (l & 1) ? bm : am;
    StepArgs<R> sm = sa;
    sm.alpha += m * NN;
    sm.y += m * NN;
    const int bx = tt % nt, by = tt / nt;
#define RIX_ANA(MM)                                                                                     \
  case MM: ana_member<R, MM>(src, n, dst, N, last, sm, bx, by, smem, taps[MM]); break;
    switch (m) { RIX_ANA(0) RIX_ANA(1) RIX_ANA(2) RIX_ANA(3) RIX_ANA(4) RIX_ANA(5) RIX_ANA(6) RIX_ANA(7) }
#undef RIX_ANA
  }
}

// step constants of one loop: L = 2 max Mx and lambda are fixed during the
// minor cycle (lambda absolute, or lambda_rel max |residual| of the first
// cycle, or the schedule a ||residual_n||_2 b^n); the concatenation's
// 1/sqrt 8 enters the analysis through 1/L.  Formed once per launch (FP64
// divisions): inv_l and thr per loop, 0 when L = 0 (the step is a no-op).
template <typename R, int DICT>
__device__ __forceinline__ void step_constants(const FistaLoop<R>& f, R* inv_l, R* thr) {
  const double lip = 2.0 * (double)f.state[0];
  const double lam = f.sched_a > 0.0   ? f.sched_a * sqrt((double)f.state[2]) * f.sched_bn
                     : f.lambda > 0.0 ? f.lambda
                                      : f.lambda_rel * (double)f.state[1];
  const double ascale = DICT == RIX_DICT_DB4 ? 1.0 : 1.0 / sqrt(8.0);
  *inv_l = lip > 0.0 ? (R)(ascale / lip) : R(0);
  *thr = lip > 0.0 ? (R)(lam / lip) : R(0);
}

// The loops of the batch advance together: every phase hands out the units
// of all loops (unit u: loop u / per, its unit u % per), so one grid barrier
// per phase serves the whole batch.
template <typename R, int LOGL, int DICT>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 && LOGL <= 12 ? 2 : 1)
    k_fista_loop(const __grid_constant__ FistaArgs<R> a) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL, DICT>;
  constexpr int N = F::N;
  constexpr bool kCat = DICT != RIX_DICT_DB4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  C* s2 = s + F::B * F::STRIDE;
  R* stage = reinterpret_cast<R*>(smem_raw + F::kFftSmem);
  const int nb = a.nb;
  const FistaLoop<R>& f0 = a.f[0];
  GridBarrier bar{f0.barrier, f0.status, 0u};
  const R sscale = (R)(1.0 / sqrt(8.0));
  const int64_t NN = (int64_t)N * N;
  const int levels = f0.levels;
  __shared__ R s_inv_l[kMaxPart], s_thr[kMaxPart];
  if (threadIdx.x < nb) step_constants<R, DICT>(a.f[threadIdx.x], &s_inv_l[threadIdx.x], &s_thr[threadIdx.x]);
  __syncthreads();
  // the constant image d = 2 crop F^-1 C of every loop
  for (int u = blockIdx.x; u < nb * F::kColUnits; u += gridDim.x) {
    const FistaLoop<R>& f = a.f[u / F::kColUnits];
    cols_inv_unit<R, LOGL>(f.c, f.tb, f.tw, s, s2, u % F::kColUnits);
  }
  if (!grid_barrier(bar)) return;
  for (int u = blockIdx.x; u < nb * F::kRowUnits; u += gridDim.x) {
    const FistaLoop<R>& f = a.f[u / F::kRowUnits];
    rows_inv_unit<R, LOGL, false>(f.tb, f.d, a.gscale, nullptr, f.tw, s, s2, stage, u % F::kRowUnits);
  }
  if (!grid_barrier(bar)) return;
  // FISTA's momentum: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, momentum
  // (t_k - 1) / t_{k+1}, each operation rounded on its own; one thread per
  // CTA forms it (FP64 square root and division at 1/64 of the FP32 rate),
  // at the start of the iteration: the grid barriers before the analysis
  // phases publish it to the CTA
  __shared__ R s_mom;
  double t = 1.0;
  for (int it = 0; it < f0.iters; ++it) {
    if (threadIdx.x == 0) {
      const double tn = __dmul_rn(0.5, __dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, t), t)))));
      s_mom = (R)__ddiv_rn(__dadd_rn(t, -1.0), tn);
      t = tn;
    }
    // x = W y, coarsest level first.  Db4: levels levels-1 .. 1 in one
    // phase (chained synthesis, into tmp), the finest level fused into the
    // row transforms
    if constexpr (kCat) {
      for (int l = levels - 1; l >= 0; --l) {
        const int per = level_units<DICT>(N >> l, kTS);
        for (int u = blockIdx.x; u < nb * per; u += gridDim.x) {
          const FistaLoop<R>& f = a.f[u / per];
          synthesis_unit<R, DICT, N>(f, f.y, l, u % per, smem_raw, a.taps);
        }
        if (!grid_barrier(bar)) return;
      }
    } else if (levels > 1) {
      constexpr int T1 = chain_block<R>();
      constexpr int nt = (N / 2 + T1 - 1) / T1, per = nt * nt;
      for (int u = blockIdx.x; u < nb * per; u += gridDim.x) {
        const FistaLoop<R>& f = a.f[u / per];
        syn_chain_tile<R, T1>(f.y, levels, N, f.tmp, (u % per) % nt, (u % per) / nt, smem_raw, Db4Taps<R>{});
      }
      if (!grid_barrier(bar)) return;
    }
    for (int u = blockIdx.x; u < nb * F::kRowUnits; u += gridDim.x) {
      const FistaLoop<R>& f = a.f[u / F::kRowUnits];
      if constexpr (kCat) rows_fwd_unit<R, LOGL, 8>(f.xs, NN, sscale, f.ta, f.tw, s, s2, u % F::kRowUnits);
      else rows_fwd_syn_unit<R, LOGL>(levels > 1 ? f.tmp : f.y, f.y, f.ta, f.tw, s, s2, stage, u % F::kRowUnits);
    }
    if (!grid_barrier(bar)) return;
    for (int u = blockIdx.x; u < nb * F::kColUnits; u += gridDim.x) {
      const FistaLoop<R>& f = a.f[u / F::kColUnits];
      cols_conv_unit<R, LOGL>(f.ta, f.mx, f.tb, f.tw, s, s2, stage, u % F::kColUnits);
    }
    if (!grid_barrier(bar)) return;
    for (int u = blockIdx.x; u < nb * F::kRowUnits; u += gridDim.x) {
      const FistaLoop<R>& f = a.f[u / F::kRowUnits];
      rows_inv_unit<R, LOGL, true>(f.tb, f.g, a.gscale, f.d, f.tw, s, s2, stage, u % F::kRowUnits);
    }
    if (!grid_barrier(bar)) return;
    const R mom = s_mom;
    for (int l = 0; l < levels; ++l) {
      const int per = level_units<DICT>((N >> l) / 2, ana_block<R, DICT>((N >> l) / 2));
      for (int u = blockIdx.x; u < nb * per; u += gridDim.x) {
        const FistaLoop<R>& f = a.f[u / per];
        const int b = u / per;
        const StepArgs<R> sa{f.alpha, f.y, s_inv_l[b], s_thr[b], s_inv_l[b] != R(0), mom};
        analysis_unit<R, DICT, N>(f, l, u % per, sa, smem_raw, a.taps);
      }
      if (!grid_barrier(bar)) return;
    }
  }
  if constexpr (kCat) {
    // each loop's image W alpha: the members' syntheses, summed
    for (int l = levels - 1; l >= 0; --l) {
      const int per = level_units<DICT>(N >> l, kTS);
      for (int u = blockIdx.x; u < nb * per; u += gridDim.x) {
        const FistaLoop<R>& f = a.f[u / per];
        synthesis_unit<R, DICT, N>(f, f.alpha, l, u % per, smem_raw, a.taps);
      }
      if (!grid_barrier(bar)) return;
    }
    for (int b = 0; b < nb; ++b) {
      const FistaLoop<R>& f = a.f[b];
      for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NN; i += (int64_t)gridDim.x * blockDim.x) {
        R acc = R(0);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc += f.xs[m * NN + i];
        f.delta[i] = sscale * acc;
      }
    }
  }
}

// ------------------------------------------------------ dataflow schedule --
// The loops of a batch are independent; only the phases of one loop are
// ordered.  Instead of one grid barrier per phase, the units of every phase
// of every loop form one ordered list: stage by stage (the two phases that
// form d, then the phases of each iteration), each stage's loops in turn.  A
// CTA takes the next unit with an atomic ticket and, before running it,
// waits until the previous stage of the unit's loop has completed (a counter
// per loop and stage); so a CTA that would idle at a barrier runs another
// loop's units instead.  Every dependency is on a smaller ticket, taken by a
// resident CTA (cooperative launch) that is running or waiting on a still
// smaller one, so the schedule always progresses; every wait is bounded as
// the grid barrier's is (2 s or 2^26 polls, then RIX_ETIMEOUT in the job's
// status word).

// completed units of a stage: release after the CTA's writes
__device__ __forceinline__ void flow_done(unsigned int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_gpu_add(ctr, 1u);
  }
}

// wait until *ctr reaches `target`, then acquire (every thread of the CTA
// sees the stage's writes); false when the wait gave up
__device__ __forceinline__ bool flow_wait(const unsigned int* ctr, unsigned int target, int* status) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned long long t0 = global_ns();
    unsigned int spins = 0;
    while (ld_acquire_gpu(ctr) < target) {
      if ((++spins & 63u) == 0) {
        if (*reinterpret_cast<volatile int*>(status) != 0) { good = 0; break; }
        if (spins >= kBarrierMaxSpins || global_ns() - t0 > kBarrierTimeoutNs) {
          atomicCAS(status, 0, RIX_ETIMEOUT);
          good = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// phase kinds of one iteration (Db4)
enum FlowKind : int { kFlowChain = 0, kFlowRowsFwd, kFlowCols, kFlowRowsInv, kFlowAna };

template <typename R, int LOGL>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 && LOGL <= 12 ? 2 : 1)
    k_fista_flow(const __grid_constant__ FistaArgs<R> a) {
  using C = cplx<R>;
  using F = FistaShape<R, LOGL, RIX_DICT_DB4>;
  constexpr int N = F::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  C* s2 = s + F::B * F::STRIDE;
  R* stage = reinterpret_cast<R*>(smem_raw + F::kFftSmem);
  const int nb = a.nb;
  const FistaLoop<R>& f0 = a.f[0];
  const int levels = f0.levels;
  constexpr int T1 = chain_block<R>();
  constexpr int kChainNt = (N / 2 + T1 - 1) / T1;
  // the phases of one iteration: kind, analysis level, units per loop
  __shared__ int ph_kind[kChainMaxLev + 4], ph_lev[kChainMaxLev + 4], ph_units[kChainMaxLev + 4];
  __shared__ int s_nph, s_iter_units;
  __shared__ R s_inv_l[kMaxPart], s_thr[kMaxPart];
  __shared__ unsigned int s_ticket;
  if (threadIdx.x == 0) {
    int k = 0;
    if (levels > 1) { ph_kind[k] = kFlowChain; ph_lev[k] = 0; ph_units[k++] = kChainNt * kChainNt; }
    ph_kind[k] = kFlowRowsFwd; ph_lev[k] = 0; ph_units[k++] = F::kRowUnits;
    ph_kind[k] = kFlowCols; ph_lev[k] = 0; ph_units[k++] = F::kColUnits;
    ph_kind[k] = kFlowRowsInv; ph_lev[k] = 0; ph_units[k++] = F::kRowUnits;
    for (int l = 0; l < levels; ++l) {
      const int h = (N >> l) / 2, tb = ana_block<R, RIX_DICT_DB4>(h), nt = (h + tb - 1) / tb;
      ph_kind[k] = kFlowAna; ph_lev[k] = l; ph_units[k++] = nt * nt;
    }
    int tot = 0;
    for (int i = 0; i < k; ++i) tot += ph_units[i];
    s_nph = k;
    s_iter_units = tot;
    s_ticket = atomicAdd(a.ticket, 1u);
  }
  if (threadIdx.x < nb)
    step_constants<R, RIX_DICT_DB4>(a.f[threadIdx.x], &s_inv_l[threadIdx.x], &s_thr[threadIdx.x]);
  __syncthreads();
  const int nph = s_nph;
  const int64_t nstage = 2 + (int64_t)f0.iters * nph;
  const int64_t pro0 = (int64_t)nb * F::kColUnits, pro1 = pro0 + (int64_t)nb * F::kRowUnits;
  const int64_t per_iter = (int64_t)nb * s_iter_units;
  const int64_t total = pro1 + per_iter * f0.iters;
  // thread 0 decodes each ticket for the CTA: stage, loop, unit, phase kind
  // and level, iteration, and the size of the stage before it
  __shared__ long long u_stg;
  __shared__ int u_b, u_u, u_kind, u_lev, u_it, u_prev, u_live;
  auto decode = [&](unsigned int t) {
    u_live = (int64_t)t < total;
    if (!u_live) return;
    int64_t stg;
    int b, u, kind = -1, lev = 0, it = 0, prev_units = 0;
    if ((int64_t)t < pro0) {
      stg = 0; b = (int)(t / F::kColUnits); u = (int)(t % F::kColUnits);
    } else if ((int64_t)t < pro1) {
      const int64_t r = t - pro0;
      stg = 1; b = (int)(r / F::kRowUnits); u = (int)(r % F::kRowUnits); prev_units = F::kColUnits;
    } else {
      const int64_t r0 = t - pro1;
      it = (int)(r0 / per_iter);
      int64_t r = r0 - (int64_t)it * per_iter;
      int k = 0;
      while (r >= (int64_t)nb * ph_units[k]) { r -= (int64_t)nb * ph_units[k]; ++k; }
      b = (int)(r / ph_units[k]);
      u = (int)(r % ph_units[k]);
      kind = ph_kind[k];
      lev = ph_lev[k];
      stg = 2 + (int64_t)it * nph + k;
      prev_units = k > 0 ? ph_units[k - 1] : (it > 0 ? ph_units[nph - 1] : F::kRowUnits);
    }
    u_stg = stg; u_b = b; u_u = u; u_kind = kind; u_lev = lev; u_it = it; u_prev = prev_units;
  };
  if (threadIdx.x == 0) decode(s_ticket);
  __syncthreads();
  while (u_live) {
    const int64_t stg = u_stg;
    const int b = u_b, u = u_u, kind = u_kind, lev = u_lev, it = u_it, prev_units = u_prev;
    unsigned int* done_b = a.done + (int64_t)b * nstage;
    if (stg > 0 && !flow_wait(done_b + stg - 1, (unsigned int)prev_units, f0.status)) return;
    // the next ticket, taken while this unit runs
    unsigned int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(a.ticket, 1u);
    const FistaLoop<R>& f = a.f[b];
    if (stg == 0) {
      cols_inv_unit<R, LOGL>(f.c, f.tb, f.tw, s, s2, u);
    } else if (stg == 1) {
      rows_inv_unit<R, LOGL, false>(f.tb, f.d, a.gscale, nullptr, f.tw, s, s2, stage, u);
    } else if (kind == kFlowChain) {
      syn_chain_tile<R, T1>(f.y, levels, N, f.tmp, u % kChainNt, u / kChainNt, smem_raw, Db4Taps<R>{});
    } else if (kind == kFlowRowsFwd) {
      rows_fwd_syn_unit<R, LOGL>(levels > 1 ? f.tmp : f.y, f.y, f.ta, f.tw, s, s2, stage, u);
    } else if (kind == kFlowCols) {
      cols_conv_unit<R, LOGL>(f.ta, f.mx, f.tb, f.tw, s, s2, stage, u);
    } else if (kind == kFlowRowsInv) {
      rows_inv_unit<R, LOGL, true>(f.tb, f.g, a.gscale, f.d, f.tw, s, s2, stage, u);
    } else {
      const StepArgs<R> sa{f.alpha, f.y, s_inv_l[b], s_thr[b], s_inv_l[b] != R(0), a.mom ? a.mom[it] : a.mom_tab[it]};
      analysis_unit<R, RIX_DICT_DB4, N>(f, lev, u, sa, smem_raw, a.taps);
    }
    flow_done(done_b + stg);
    if (threadIdx.x == 0) decode(next);
    __syncthreads();
  }
}

// FISTA's momentum per iteration: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
// momentum (t_k - 1) / t_{k+1}, each operation rounded on its own
template <typename R>
__global__ void k_mom_table(int iters, R* mom) {
  double t = 1.0;
  for (int it = 0; it < iters; ++it) {
    const double tn = __dmul_rn(0.5, __dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, t), t)))));
    mom[it] = (R)__ddiv_rn(__dadd_rn(t, -1.0), tn);
    t = tn;
  }
}

// the same sequence on the host, each operation rounded on its own
// (volatile temporaries keep the compiler from contracting them)
template <typename R>
void mom_host(int iters, R* mom) {
  double t = 1.0;
  for (int it = 0; it < iters; ++it) {
    volatile double a = 4.0 * t;
    volatile double b = a * t;
    volatile double c = 1.0 + b;
    volatile double q = std::sqrt((double)c);
    volatile double e = 1.0 + q;
    volatile double tn = 0.5 * e;
    volatile double num = t - 1.0;
    volatile double m = num / tn;
    mom[it] = (R)m;
    t = tn;
  }
}

template <typename R, int LOGL, int DICT>
int launch_fista_loop(const Ctx* ctx, const FistaLoop<R>* f, int nb, cudaStream_t st) {
  using F = FistaShape<R, LOGL, DICT>;
  if (nb < 1 || nb > kMaxPart) return set_error(RIX_EINVAL, "FISTA batch of %d loops", nb);
  for (int b = 1; b < nb; ++b)
    if (f[b].n != f[0].n || f[b].levels != f[0].levels || f[b].iters != f[0].iters || f[b].dict != f[0].dict)
      return set_error(RIX_EINVAL, "FISTA batch: the loops differ in size, levels, iterations or dictionary");
  auto kern = k_fista_loop<R, LOGL, DICT>;
  const size_t smem = F::kSmem;
  RIX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFftThreads, smem));
  if (per_sm < 1) return set_error(RIX_EINVAL, "FISTA loop does not fit on an SM (%zu B shared)", smem);
  // one CTA per SM for a single loop (another partition's loop or gridder fits
  // beside it); a batch of loops takes up to two
  const int nblk = ctx->num_sms * std::min(per_sm, nb > 1 ? 2 : 1);
  FistaArgs<R> args{};
  for (int b = 0; b < nb; ++b) args.f[b] = f[b];
  args.nb = nb;
  args.gscale = (R)(2.0 / (4.0 * (double)F::N * (double)F::N));
  if constexpr (DICT == RIX_DICT_DB1_8) {
    for (int m = 0; m < 8; ++m) {
      double h[16];
      const int k = daubechies_lowpass(m + 1, h);
      if (k != 2 * (m + 1)) return set_error(RIX_EINVAL, "daubechies filter %d", m + 1);
      for (int i = 0; i < 16; ++i) args.taps[m][i] = i < k ? (R)h[i] : R(0);
    }
  }
  if constexpr (DICT == RIX_DICT_DB4) {
    if (nb > 1) {
      // several loops (Db4): the dataflow schedule instead of grid barriers
      auto fk = k_fista_flow<R, LOGL>;
      RIX_CUDA(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int fper = 0;
      RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fper, fk, kFftThreads, smem));
      if (fper < 1) return set_error(RIX_EINVAL, "FISTA loop does not fit on an SM (%zu B shared)", smem);
      const int fblk = ctx->num_sms * std::min(fper, 2);
      const int levels = f[0].levels;
      const int64_t nph = (levels > 1 ? 1 : 0) + 3 + levels;
      const int64_t nctl = 1 + (int64_t)nb * (2 + (int64_t)f[0].iters * nph);
      unsigned int* ctl = nullptr;
      R* mom = nullptr;
      RIX_CUDA(::rix::malloc_async(&ctl, (size_t)nctl * sizeof(unsigned int), st));
      if (::rix::malloc_async(&mom, (size_t)std::max(f[0].iters, 1) * sizeof(R), st) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(ctl, st);
        return set_error(RIX_ENOMEM, "FISTA schedule tables");
      }
      int rc = RIX_OK;
      if (cudaMemsetAsync(ctl, 0, (size_t)nctl * sizeof(unsigned int), st) != cudaSuccess) {
        rc = set_error(RIX_ECUDA, "FISTA schedule reset");
      } else {
        args.ticket = ctl;
        args.done = ctl + 1;
        if (f[0].iters <= kMomTab) {
          mom_host<R>(f[0].iters, args.mom_tab);
          args.mom = nullptr;
        } else {
          ::rix::note_launch();
          k_mom_table<R><<<1, 1, 0, st>>>(f[0].iters, mom);
          args.mom = mom;
        }
        void* params[] = {&args};
        ::rix::note_launch();
        timing_mark(kTimeMinorLoop, st, true);
        const cudaError_t e =
            cudaLaunchCooperativeKernel((const void*)fk, dim3(fblk), dim3(kFftThreads), params, smem, st);
        timing_mark(kTimeMinorLoop, st, false);
        if (e != cudaSuccess) rc = set_error(RIX_ECUDA, "FISTA loop launch: %s", cudaGetErrorString(e));
      }
      cudaFreeAsync(ctl, st);
      cudaFreeAsync(mom, st);
      return rc;
    }
  }
  RIX_CUDA(cudaMemsetAsync(f[0].barrier, 0, sizeof(unsigned int), st));
  void* params[] = {&args};
  ::rix::note_launch();
  timing_mark(kTimeMinorLoop, st, true);
  RIX_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(nblk), dim3(kFftThreads), params, smem, st));
  timing_mark(kTimeMinorLoop, st, false);
  return RIX_OK;
}

// dispatch on the transform length 2N (N a power of two in [32, KMAXN])
template <typename R, int DICT, int LOGL, int LOGL_MAX>
int fista_loop_dispatch(const Ctx* ctx, const FistaLoop<R>* f, int nb, int logl, cudaStream_t st) {
  if (logl == LOGL) return launch_fista_loop<R, LOGL, DICT>(ctx, f, nb, st);
  if constexpr (LOGL < LOGL_MAX) return fista_loop_dispatch<R, DICT, LOGL + 1, LOGL_MAX>(ctx, f, nb, logl, st);
  return set_error(RIX_EINVAL, "FISTA loop: image side %d not supported", f[0].n);
}

}  // namespace

// the instances of one dictionary (k_fista_*.cu, one translation unit each)
template <typename R, int DICT>
int fista_loop_dict(const Ctx* ctx, const FistaLoop<R>* f, int nb, cudaStream_t st) {
  constexpr int kMaxLogL = std::is_same<R, float>::value ? 13 : 12;   // N <= 4096 (FP32), 2048 (FP64)
  return fista_loop_dispatch<R, DICT, 6, kMaxLogL>(ctx, f, nb, ilog2(2 * (int64_t)f[0].n), st);
}

}  // namespace rix
