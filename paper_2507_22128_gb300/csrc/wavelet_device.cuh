// Device code of the periodic orthonormal 2D Daubechies wavelet transforms
// (the dictionaries of the FISTA minor cycle, Eq. 4-5; Sec. 5.2): one tile of
// one analysis level (with the FISTA step fused into the final coefficients)
// and one tile of one synthesis level, for a filter of K taps.  Shared by the
// per-level kernels and the persistent minor-cycle loop.
//
// Transform (periodic, analysis by correlation), per level of an n x n block:
//   a[k] = sum_i h[i] x[(2k + i) mod n],  d[k] = sum_i g[i] x[(2k + i) mod n],
//   g[i] = (-1)^i h[K - 1 - i], along rows and then columns; subband layout
//   [Y][X] with Y < n/2 column-low, X < n/2 row-low (Mallat); synthesis is
//   the transpose.
#pragma once

#include <cuda_runtime.h>

#include "rix_internal.cuh"

namespace rix {
namespace {

// --------------------------------------------------------------- filters ----
// Daubechies 4-vanishing-moment low-pass filter (8 taps, minimum phase,
// normalised to sum sqrt(2)).  Compile-time constants: every use has a
// compile-time tap index, so the taps fold into immediates (no constant-bank
// loads or FP64 conversions).
__device__ constexpr double kDb4[8] = {0.23037781330885523,  0.7148465705525415,   0.6308807679295904,
                                       -0.02798376941698385, -0.18703481171888114, 0.030841381835986965,
                                       0.032883011666982945, -0.010597401784997278};

template <typename R>
struct Db4Taps {
  static constexpr int K = 8;
  __device__ __forceinline__ constexpr R lo(int i) const { return (R)kDb4[i]; }
  __device__ __forceinline__ constexpr R hi(int i) const {
    return (i & 1) ? -(R)kDb4[7 - i] : (R)kDb4[7 - i];
  }
};

// a filter of K taps read where it lives (a kernel parameter: the taps stay
// constant-bank operands instead of occupying registers across loops)
template <typename R, int KT>
struct RefTaps {
  static constexpr int K = KT;
  const R* h;
  __device__ __forceinline__ R lo(int i) const { return h[i]; }
  __device__ __forceinline__ R hi(int i) const { return (i & 1) ? -h[KT - 1 - i] : h[KT - 1 - i]; }
};

// ----------------------------------------------------- asynchronous copies --
// global -> shared copies that bypass the registers (cp.async); a thread's
// copies are complete after cp_async_wait_all, and everyone's after that and
// a CTA barrier.  BYTES = 4, 8 (cached in L1 and L2) or 16 (L2 only); both
// addresses aligned to BYTES.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
  } else {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(BYTES) : "memory");
  }
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) { cp_async<16>(sdst, gsrc); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------- fused analysis levels ----
// A CTA owns a TB x TB block of each of the four subbands of an n x n block
// (n a power of two), stages the periodic (2 TB + K - 2)^2 input tile and the
// step's inputs (y and alpha of the block) with asynchronous copies, filters
// the tile's rows (low and high) and then its columns.
constexpr int kTB = 16;                      // the smaller block side
constexpr int kMaxTaps = 16;                 // db8
template <int TB, int K> constexpr int tin_side() { return 2 * TB + K - 2; }

// FISTA step fused into the analysis of the gradient (Beck & Teboulle 2009):
// at each final coefficient c = s g:  a' = S_{lam/L}(y - c/L),
// y = a' + mom (a' - a),  a = a'   (s: the dictionary's scale; inv_l folds it)
template <typename R>
struct StepArgs {
  R* alpha;
  R* y;
  R inv_l, thr;         // s / L and lambda / L (both 0 when L = 0: the step is a no-op)
  bool active;
  R mom;
};

template <typename R, int TB, int K>
struct DwtSmem {
  static constexpr int TIN = tin_side<TB, K>();
  R tin[TIN][TIN + 1];
  R trow[TIN][2 * TB + 1];             // [input row][lo x | hi x]
  alignas(16) R ys[4][TB * TB];        // step inputs per quadrant, [row][column] of the block
  alignas(16) R as[4][TB * TB];
};

// one TB x TB output block (bx, by) of each subband; 256 threads
template <typename R, int TB, bool kStep, typename TAPS>
__device__ __forceinline__ void dwt_tile(const R* __restrict__ src, int lds, int n, R* __restrict__ coef,
                                         R* __restrict__ ll, int ld, int last, const StepArgs<R>& st, int bx, int by,
                                         DwtSmem<R, TB, TAPS::K>& sm, const TAPS& tp) {
  constexpr int K = TAPS::K;
  constexpr int TIN = tin_side<TB, K>();
  static_assert((TB * TB) % 256 == 0, "block side");
  auto& tin = sm.tin;
  auto& trow = sm.trow;
  const int h = n / 2;
  const int y0 = by * TB, x0 = bx * TB;
  // the coefficients this block updates: quadrants 1-3, and 0 at the last
  // level; 16-byte copies of whole block rows (h is a multiple of the chunk)
  if constexpr (kStep) {
    constexpr int CH = 16 / (int)sizeof(R);
    constexpr int CPR = TB / CH;
    for (int c = threadIdx.x; c < 4 * TB * CPR; c += blockDim.x) {
      const int q = c / (TB * CPR), rem = c - q * (TB * CPR);
      const int r = rem / CPR, k = rem - r * CPR;
      const int y = y0 + r, x = x0 + k * CH;
      if ((q != 0 || last) && y < h && x < h) {
        const int64_t i = (int64_t)((q >> 1) * h + y) * ld + (q & 1) * h + x;
        cp_async16(&sm.ys[q][r * TB + k * CH], st.y + i);
        cp_async16(&sm.as[q][r * TB + k * CH], st.alpha + i);
      }
    }
  }
  for (int t = threadIdx.x; t < TIN * TIN; t += blockDim.x) {
    const int r = t / TIN, c = t - r * TIN;
    cp_async<(int)sizeof(R)>(&tin[r][c], src + (int64_t)((2 * y0 + r) & (n - 1)) * lds + ((2 * x0 + c) & (n - 1)));
  }
  cp_async_wait_all();
  __syncthreads();
  for (int t = threadIdx.x; t < TIN * TB; t += blockDim.x) {
    const int r = t / TB, xx = t - r * TB;
    R a = R(0), d = R(0);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const R w = tin[r][2 * xx + i];
      a += tp.lo(i) * w;
      d += tp.hi(i) * w;
    }
    trow[r][xx] = a;
    trow[r][TB + xx] = d;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TB * TB / 256; ++k) {
    const int pidx = threadIdx.x + 256 * k;
    const int ty = pidx / TB, tx = pidx - ty * TB;
    const int y = y0 + ty, x = x0 + tx;
    if (y < h && x < h) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cy = q >> 1, cx = q & 1;
        R g = R(0);
#pragma unroll
        for (int i = 0; i < K; ++i) g += (cy ? tp.hi(i) : tp.lo(i)) * trow[2 * ty + i][cx * TB + tx];
        const int64_t idx = (int64_t)(cy * h + y) * ld + cx * h + x;
        if (q == 0 && !last) {
          ll[(int64_t)y * ld + x] = g;
        } else if (kStep) {
          const R z = sm.ys[q][pidx] - g * st.inv_l;
          const R az = fabs(z) - st.thr;
          const R an = (st.active && az > R(0)) ? copysign(az, z) : R(0);
          st.y[idx] = an + st.mom * (an - sm.as[q][pidx]);
          st.alpha[idx] = an;
        } else {
          coef[idx] = g;
        }
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------- synthesis level ----
// out (n x n, ld) from the LL block `llin` (ld) and the detail subbands of
// `coef` (ld); a CTA owns a kTS x kTS output block.
constexpr int kTS = 32;
template <int K> constexpr int rk_side() { return kTS / 2 + K / 2; }

template <typename R, int K>
struct IdwtSmem {
  static constexpr int RK = rk_side<K>();
  R cq[4][RK][RK + 1];         // quadrant tiles: LL, row-high, col-high, HH
  R tr[2][RK][kTS + 1];        // after row synthesis: [column half][coef row][c]
};

template <typename R, typename TAPS>
__device__ __forceinline__ void idwt_tile(const R* __restrict__ llin, const R* __restrict__ coef, int n,
                                          R* __restrict__ out, int ld, int bx, int by, IdwtSmem<R, TAPS::K>& sm,
                                          const TAPS& tp) {
  constexpr int K = TAPS::K;
  constexpr int RK = rk_side<K>();
  auto& cq = sm.cq;
  auto& tr = sm.tr;
  const int h = n / 2;
  const int m0 = by * kTS, c0 = bx * kTS;
  // output m uses coefficients (m - i) / 2 for the taps i of its parity
  const int kb_m = (m0 >> 1) - K / 2, kb_c = (c0 >> 1) - K / 2;
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
  // rows: tr[cy][rk][c] = sum over the K/2 taps of the parity of c
  for (int t = threadIdx.x; t < 2 * RK * kTS; t += blockDim.x) {
    const int cy = t / (RK * kTS), rem = t - cy * RK * kTS;
    const int rk = rem / kTS, cl = rem - rk * kTS;
    const int c = c0 + cl;
    const bool odd = c & 1;
    const int kc = (c >> 1) - kb_c;             // tap i = 2 j + (c & 1) reads coefficient (c - i) / 2
    R v2 = R(0);
#pragma unroll
    for (int j = 0; j < K / 2; ++j) {
      const R hh = odd ? tp.lo(2 * j + 1) : tp.lo(2 * j);
      const R gg = odd ? tp.hi(2 * j + 1) : tp.hi(2 * j);
      v2 += hh * cq[2 * cy][rk][kc - j] + gg * cq[2 * cy + 1][rk][kc - j];
    }
    tr[cy][rk][cl] = v2;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kTS * kTS; t += blockDim.x) {
    const int ml = t / kTS, cl = t - ml * kTS;
    const int m = m0 + ml, c = c0 + cl;
    if (m >= n || c >= n) continue;
    const bool odd = m & 1;
    const int km = (m >> 1) - kb_m;
    R v2 = R(0);
#pragma unroll
    for (int j = 0; j < K / 2; ++j) {
      const R hh = odd ? tp.lo(2 * j + 1) : tp.lo(2 * j);
      const R gg = odd ? tp.hi(2 * j + 1) : tp.hi(2 * j);
      v2 += hh * tr[0][km - j][cl] + gg * tr[1][km - j][cl];
    }
    out[(int64_t)m * ld + c] = v2;
  }
  __syncthreads();
}

// ------------------------------------------- chained coarse synthesis ----
// The level-1 output block [m0, m0 + T1) x [c0, c0 + T1) of x = W c depends,
// at each coarser level, only on the region of that level's output that the
// taps reach: output rows m of level l read coefficient rows (m >> 1) - j,
// j < K/2, of level l (periodic modulo the level's side), i.e. rows
// [(lo >> 1) - K/2 + 1, ((lo + len - 1) >> 1)] for a region [lo, lo + len).
// A unit loads the coefficients of all those regions at once (the top LL
// block and the three detail subbands of every level, with asynchronous
// copies) and synthesises the regions coarsest first in shared memory; so
// the levels levels-1 .. 1 take one grid phase instead of one each, at the
// price of recomputing the (small) coarse regions per unit.
constexpr int kChainMaxLev = 12;

// an upper bound of the region side at chain step s (s = 0: the block)
template <int T1, int K>
__host__ __device__ constexpr int chain_max_len(int step) {
  int n = T1;
  for (int i = 0; i < step; ++i) n = n / 2 + K / 2;
  return n;
}

// shared-memory elements of a chain of up to kChainMaxLev levels
template <int T1, int K>
__host__ __device__ constexpr int chain_smem_elems() {
  int e = 0;
  for (int s = 1; s <= kChainMaxLev; ++s) e += 3 * chain_max_len<T1, K>(s) * chain_max_len<T1, K>(s);   // details
  const int m2 = chain_max_len<T1, K>(1);
  e += m2 * m2;                  // top LL region
  e += 2 * m2 * m2;              // region ping-pong
  e += 2 * m2 * T1;              // row pass
  return e;
}
template <typename R, int T1, int K>
__host__ __device__ constexpr size_t chain_smem_bytes() {
  return 16 * sizeof(int) * (kChainMaxLev + 1) + (size_t)chain_smem_elems<T1, K>() * sizeof(R);
}

// block (bx, by) of the level-1 output (side n1 = N / 2, ld N) into dst,
// from the coefficients `coef` (N x N, Mallat layout, `levels` levels)
template <typename R, int T1, typename TAPS>
__device__ __forceinline__ void syn_chain_tile(const R* __restrict__ coef, int levels, int N, R* __restrict__ dst,
                                               int bx, int by, unsigned char* smem, const TAPS& tp) {
  constexpr int K = TAPS::K, HK = K / 2;
  // table per level l = 1 .. levels: region rows [lr, lr + nr), cols
  // [lc, lc + nc) of level l's output (l = levels: the top LL block), and the
  // offset of level l's details (the region of level l + 1)
  int* tab = reinterpret_cast<int*>(smem);
  int* lr = tab;
  int* nr = tab + (kChainMaxLev + 1);
  int* lc = tab + 2 * (kChainMaxLev + 1);
  int* nc = tab + 3 * (kChainMaxLev + 1);
  int* doff = tab + 4 * (kChainMaxLev + 1);
  R* pool = reinterpret_cast<R*>(smem + 16 * sizeof(int) * (kChainMaxLev + 1));
  constexpr int M2 = chain_max_len<T1, K>(1);
  if (threadIdx.x == 0) {
    lr[1] = by * T1; nr[1] = T1; lc[1] = bx * T1; nc[1] = T1;
    int off = 0;
    for (int l = 1; l < levels; ++l) {
      lr[l + 1] = (lr[l] >> 1) - (HK - 1);
      nr[l + 1] = ((lr[l] + nr[l] - 1) >> 1) - lr[l + 1] + 1;
      lc[l + 1] = (lc[l] >> 1) - (HK - 1);
      nc[l + 1] = ((lc[l] + nc[l] - 1) >> 1) - lc[l + 1] + 1;
      doff[l] = off;
      off += 3 * nr[l + 1] * nc[l + 1];
    }
    doff[levels] = off;          // the top LL region
  }
  __syncthreads();
  // threads as TC columns x (256 / TC) row groups: no divisions in the
  // loops, and a thread's column fixes its taps' parity
  constexpr int TC = T1;
  constexpr int RG = 256 / TC;
  static_assert(256 % TC == 0, "block side");
  const int tc = threadIdx.x % TC, tg = threadIdx.x / TC;
  // every coefficient the block needs, in one batch of asynchronous copies
  for (int l = 1; l < levels; ++l) {
    const int h = N >> (l + 1);                // side of level l's subbands
    const int r0 = lr[l + 1], c0 = lc[l + 1], rn = nr[l + 1], cn = nc[l + 1];
    R* dl = pool + doff[l];
    if (tc < cn) {
      const int col = (c0 + tc) & (h - 1);
      for (int rr = tg; rr < 3 * rn; rr += RG) {
        const int q = rr >= 2 * rn ? 3 : rr >= rn ? 2 : 1;
        const int row = (r0 + rr - (q - 1) * rn) & (h - 1);
        cp_async<(int)sizeof(R)>(dl + rr * cn + tc, coef + (int64_t)((q >> 1) * h + row) * N + (q & 1) * h + col);
      }
    }
  }
  {
    const int h = N >> levels;
    const int r0 = lr[levels], c0 = lc[levels], rn = nr[levels], cn = nc[levels];
    R* tl = pool + doff[levels];
    if (tc < cn) {
      const int col = (c0 + tc) & (h - 1);
      for (int rk = tg; rk < rn; rk += RG)
        cp_async<(int)sizeof(R)>(tl + rk * cn + tc, coef + (int64_t)((r0 + rk) & (h - 1)) * N + col);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  R* buf[2] = {pool + doff[levels] + M2 * M2, pool + doff[levels] + 2 * M2 * M2};
  R* tr = pool + doff[levels] + 3 * M2 * M2;
  const R* ll = pool + doff[levels];
  int llw = nc[levels];                         // row stride of ll
  const int n1 = N >> 1;
  for (int l = levels - 1; l >= 1; --l) {
    const int ir0 = lr[l + 1], irn = nr[l + 1], ic0 = lc[l + 1], icn = nc[l + 1];
    const int or0 = lr[l], orn = nr[l], oc0 = lc[l], ocn = nc[l];
    const R* d1 = pool + doff[l];               // (0, 1): row-high
    const R* d2 = d1 + irn * icn;               // (1, 0): column-high
    const R* d3 = d2 + irn * icn;               // (1, 1)
    // rows: tr[cy][rk][c] for the output columns c
    if (tc < ocn) {
      const int ca = oc0 + tc;
      const int kc = (ca >> 1) - ic0;
      const int par = ca & 1;
      R tl[HK], th[HK];
#pragma unroll
      for (int j = 0; j < HK; ++j) {
        tl[j] = par ? tp.lo(2 * j + 1) : tp.lo(2 * j);
        th[j] = par ? tp.hi(2 * j + 1) : tp.hi(2 * j);
      }
      for (int rr = tg; rr < 2 * irn; rr += RG) {
        const bool cy = rr >= irn;
        const int rk = cy ? rr - irn : rr;
        const R* q0 = cy ? d2 + rk * icn : ll + rk * llw;
        const R* q1 = (cy ? d3 : d1) + rk * icn;
        R v = R(0);
#pragma unroll
        for (int j = 0; j < HK; ++j) v += tl[j] * q0[kc - j] + th[j] * q1[kc - j];
        tr[rr * ocn + tc] = v;
      }
    }
    __syncthreads();
    // columns, into the next region (or the level-1 output)
    R* out = buf[l & 1];
    if (tc < ocn) {
      for (int r = tg; r < orn; r += RG) {
        const int ma = or0 + r;
        const int km = (ma >> 1) - ir0;
        const int par = ma & 1;
        R v = R(0);
#pragma unroll
        for (int j = 0; j < HK; ++j) {
          const R lo = par ? tp.lo(2 * j + 1) : tp.lo(2 * j);
          const R hi = par ? tp.hi(2 * j + 1) : tp.hi(2 * j);
          v += lo * tr[(km - j) * ocn + tc] + hi * tr[(irn + km - j) * ocn + tc];
        }
        if (l > 1) {
          out[r * ocn + tc] = v;
        } else if (ma < n1 && oc0 + tc < n1) {
          dst[(int64_t)ma * N + oc0 + tc] = v;
        }
      }
    }
    __syncthreads();
    ll = out;
    llw = ocn;
  }
}

}  // namespace
}  // namespace rix
