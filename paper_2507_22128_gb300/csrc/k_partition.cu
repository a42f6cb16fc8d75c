// a1-a3: per-sample FP64 grid coordinates, |uv| partition masks (Sec. 3),
// entry generation, stable LSD radix sort by tile key and gridder work items.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "rix_internal.cuh"

namespace rix {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kChunk = 2048;                          // entries per gridder work item

// ------------------------------------------------------------------ scan ----
__global__ void __launch_bounds__(kScanThreads) k_scan_block(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out, int64_t n,
                                                             uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    sum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0u;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = s - t;   // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1 && block_sums) block_sums[blockIdx.x] = s;
  }
  __syncthreads();
  uint32_t run = warp_tot[warp] + incl - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const uint32_t o = offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t j = i + (int64_t)k * kScanThreads;
    if (j < n) out[j] += o;
  }
}

__global__ void k_total(const uint32_t* in, const uint32_t* ex, int64_t n, uint32_t* total) {
  *total = (n > 0) ? in[n - 1] + ex[n - 1] : 0u;
}

// ----------------------------------------------------------- radix sort ----
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys, int64_t n,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of block b owns keys [b*4096 + w*512, +512) in 16
// rounds of 32; ranks within a round come from __match_any_sync, ranks across
// rounds from a warp-private digit histogram, ranks across warps from a
// per-digit prefix over the warps, ranks across blocks from the scanned
// (digit, block) histogram.
template <typename K, bool kVals>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t whist[kSortThreads / 32][256];
  for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortItems);
  K key[kSortItems];
  uint32_t val[kSortItems];
  uint32_t rank[kSortItems];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t idx = seg + r * 32 + lane;
    const bool valid = idx < n;
    key[r] = valid ? kin[idx] : K(0);
    if (kVals) val[r] = valid ? vin[idx] : 0u;
    const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
    uint32_t base_cnt = valid ? whist[warp][d] : 0u;
    rank[r] = base_cnt + __popc(peers & lt);
    __syncwarp();
    if (valid && (__ffs(peers) - 1) == lane) whist[warp][d] = base_cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread t turns the warps' counts of digit t into exclusive global offsets
    const int d = threadIdx.x;
    uint32_t run = offs[(int64_t)d * nblocks + blockIdx.x];
    for (int w = 0; w < kSortThreads / 32; ++w) {
      uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t idx = seg + r * 32 + lane;
    if (idx < n) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
      const uint32_t dst = whist[warp][d] + rank[r];
      kout[dst] = key[r];
      if (kVals) vout[dst] = val[r];
    }
  }
}

template <typename K, bool kVals>
int radix_sort_impl(K* keys, uint32_t* vals, K* keys_tmp, uint32_t* vals_tmp, int64_t n, int bits,
                    cudaStream_t st, bool* in_tmp) {
  *in_tmp = false;
  if (n <= 1 || bits <= 0) return RIX_OK;
  if (n > (int64_t)0xFFFFFFFFu) return set_error(RIX_EINVAL, "radix sort: too many keys");
  const int nblocks = (int)ceil_div(n, kSortTile);
  const int64_t hn = (int64_t)256 * nblocks;
  uint32_t* hist = nullptr;
  RIX_CUDA(::rix::malloc_async(&hist, 2 * hn * sizeof(uint32_t), st));
  K* a = keys; K* b = keys_tmp;
  uint32_t* va = vals; uint32_t* vb = vals_tmp;
  int rc = RIX_OK;
  for (int shift = 0; shift < bits; shift += 8) {
    ::rix::note_launch(); k_radix_hist<K><<<nblocks, kSortThreads, 0, st>>>(a, n, shift, hist, nblocks);
    rc = scan_exclusive_u32(hist, hist + hn, hn, nullptr, st);
    if (rc != RIX_OK) break;
    ::rix::note_launch(); k_radix_scatter<K, kVals><<<nblocks, kSortThreads, 0, st>>>(a, va, b, vb, n, shift, hist + hn,
                                                                 nblocks);
    std::swap(a, b);
    std::swap(va, vb);
    *in_tmp = !*in_tmp;
  }
  cudaFreeAsync(hist, st);
  if (rc != RIX_OK) return rc;
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

// ------------------------------------------------------- sample geometry ----
struct Thresholds {
  double lo[kMaxPart];   // ell_p - delta (p >= 1)
  double hi[kMaxPart];   // ell_{p+1} + delta (p <= P-2)
  int nparts;
};

struct Coords {
  int ju, jv;        // first taps on the 2N grid
  bool inside;
  double r;          // radius in N-grid Fourier pixels
  double ul, vl, wl;
};

__device__ __forceinline__ Coords sample_coords(const SampleGeomParams& g, int64_t s) {
  const int64_t row = s / g.nchan;
  const int ch = (int)(s - row * g.nchan);
  const double sc = g.inv_lambda[ch];
  Coords c;
  c.ul = __dmul_rn(g.uvw[row * 3 + 0], sc);
  c.vl = __dmul_rn(g.uvw[row * 3 + 1], sc);
  c.wl = __dmul_rn(g.uvw[row * 3 + 2], sc);
  const double x = __dadd_rn(__dmul_rn(c.ul, g.scale), g.half);
  const double y = __dadd_rn(__dmul_rn(c.vl, g.scale), g.half);
  const double xs = __dadd_rn(x, -0.5 * kW);
  const double ys = __dadd_rn(y, -0.5 * kW);
  const double cx = ceil(xs), cy = ceil(ys);
  const bool finite = fabs(cx) < 1e9 && fabs(cy) < 1e9;
  c.ju = finite ? (int)cx : -1;
  c.jv = finite ? (int)cy : -1;
  c.inside = finite && c.ju >= 0 && c.ju + kW <= g.ng && c.jv >= 0 && c.jv + kW <= g.ng;
  const double pu = __dmul_rn(c.ul, g.ndl);
  const double pv = __dmul_rn(c.vl, g.ndl);
  c.r = __dsqrt_rn(__dadd_rn(__dmul_rn(pu, pu), __dmul_rn(pv, pv)));
  return c;
}

__device__ __forceinline__ int sample_plane(const SampleGeomParams& g, double wl) {
  if (g.nw <= 0) return 0;
  const double tw = __ddiv_rn(__dadd_rn(wl, -g.w_min), g.dw);
  double p0 = ceil(tw);
  p0 = fmin(fmax(p0, 0.0), (double)(g.nw - g.ww));
  return (int)p0;
}

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_w_minmax(SampleGeomParams g, int64_t ns, unsigned long long* mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = s / g.nchan;
    const int ch = (int)(s - row * g.nchan);
    const unsigned long long b = ordered_bits(__dmul_rn(g.uvw[row * 3 + 2], g.inv_lambda[ch]));
    lo = min(lo, b);
    hi = max(hi, b);
  }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

__global__ void k_radius_bits(SampleGeomParams g, int64_t ns, uint64_t* out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    Coords c = sample_coords(g, s);
    out[s] = (uint64_t)__double_as_longlong(c.r);   // r >= 0: bit order = value order
  }
}

// Radix select of the ring radii: the order statistics k_i = i (ns - 1) / P,
// i = 1 .. P-1, of the 64-bit radius keys, one 8-bit digit per pass from the
// most significant: each pass histograms the digit of the keys that match
// target i's prefix so far, then k_select_step finds the digit value holding
// rank k_i and extends the prefix.  After eight passes the prefix is the
// key of rank k_i itself, the same value a full sort would put there.
struct SelectState {
  uint64_t prefix[kMaxPart];
  int64_t rank[kMaxPart];
  unsigned int hist[kMaxPart][256];
};

__global__ void k_select_init(SelectState* st, int64_t ns, int nparts) {
  const int i = threadIdx.x;
  if (i < kMaxPart) {
    st->prefix[i] = 0ull;
    st->rank[i] = (i + 1 < nparts) ? ((int64_t)(i + 1) * (ns - 1)) / nparts : 0;
  }
  for (int j = threadIdx.x; j < kMaxPart * 256; j += blockDim.x) (&st->hist[0][0])[j] = 0u;
}

// keys matching each target's prefix of the bits above `shift`: histogram of
// bits [shift, shift + 8)
__global__ void k_select_hist(const uint64_t* __restrict__ keys, int64_t n, int ntg, int shift, SelectState* st) {
  __shared__ unsigned int h[kMaxPart][256];
  for (int j = threadIdx.x; j < kMaxPart * 256; j += blockDim.x) (&h[0][0])[j] = 0u;
  __shared__ uint64_t pre[kMaxPart];
  if (threadIdx.x < kMaxPart) pre[threadIdx.x] = st->prefix[threadIdx.x];
  __syncthreads();
  // the early digits take few values: lanes with equal digits add once
  // (warp-aggregated), so the shared atomics do not serialise
  const int lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = b + threadIdx.x;
    const bool valid = e < n;
    const uint64_t k = valid ? keys[e] : 0ull;
    const uint64_t hi = shift + 8 < 64 ? (k >> (shift + 8)) : 0ull;
    const unsigned d = (unsigned)(k >> shift) & 255u;
    for (int t = 0; t < ntg; ++t) {
      const bool m = valid && hi == pre[t];
      const unsigned act = __ballot_sync(0xffffffffu, m);
      if (m) {
        const unsigned grp = __match_any_sync(act, d);
        if (lane == __ffs(grp) - 1) atomicAdd(&h[t][d], (unsigned)__popc(grp));
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ntg * 256; j += blockDim.x) {
    const unsigned v = (&h[0][0])[j];
    if (v) atomicAdd(&(&st->hist[0][0])[j], v);
  }
}

// one thread per target: the digit holding rank k, the rank within it; the
// histograms are cleared for the next pass
__global__ void k_select_step(SelectState* st, int ntg) {
  const int t = threadIdx.x;
  if (t < ntg) {
    int64_t k = st->rank[t];
    unsigned d = 0;
    for (; d < 255u; ++d) {
      const int64_t c = st->hist[t][d];
      if (k < c) break;
      k -= c;
    }
    st->rank[t] = k;
    st->prefix[t] = (st->prefix[t] << 8) | d;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kMaxPart * 256; j += blockDim.x) (&st->hist[0][0])[j] = 0u;
}

__global__ void k_select_out(const SelectState* st, int ntg, double* ells) {
  const int t = threadIdx.x;
  if (t < ntg) ells[t] = __longlong_as_double((long long)st->prefix[t]);
}

// Uniform weighting: density of the natural weights on the N x N uv grid
// (nearest cell of each sample inside the grid and its Hermitian mirror),
// accumulated in FP64, then w / D(cell) in FP64 rounded to float32.
__device__ __forceinline__ void uniform_cell(const SampleGeomParams& g, const Coords& c, int& a, int& b) {
  a = (int)floor(__dadd_rn(__dmul_rn(c.ul, g.ndl), 0.5));
  b = (int)floor(__dadd_rn(__dmul_rn(c.vl, g.ndl), 0.5));
}

__global__ void k_uniform_density(SampleGeomParams g, int64_t ns, const float* __restrict__ w, int n,
                                  double* __restrict__ dens) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const Coords c = sample_coords(g, s);
    if (!c.inside) continue;
    const double ws = w ? (double)w[s] : 1.0;
    int a, b;
    uniform_cell(g, c, a, b);
    const int h = n / 2;
    if (a + h >= 0 && a + h < n && b + h >= 0 && b + h < n) atomicAdd(&dens[(int64_t)(a + h) * n + (b + h)], ws);
    if (h - a >= 0 && h - a < n && h - b >= 0 && h - b < n) atomicAdd(&dens[(int64_t)(h - a) * n + (h - b)], ws);
  }
}

__global__ void k_uniform_apply(SampleGeomParams g, int64_t ns, const float* __restrict__ w_in, int n,
                                const double* __restrict__ dens, float* __restrict__ w_out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const Coords c = sample_coords(g, s);
    const double ws = w_in ? (double)w_in[s] : 1.0;
    double out = ws;
    if (c.inside) {
      int a, b;
      uniform_cell(g, c, a, b);
      const int h = n / 2;
      if (a + h >= 0 && a + h < n && b + h >= 0 && b + h < n) {
        const double d = dens[(int64_t)(a + h) * n + (b + h)];
        if (d > 0.0) out = __ddiv_rn(ws, d);
      }
    }
    w_out[s] = (float)out;
  }
}

struct ClassifyOut {
  uint8_t* mask_out;       // may be null
  uint32_t* counts;        // per sample: number of partitions
  int* win;                // [kMaxPart][4]: min j, max j on 2N grid; min j', max j' on 4N grid
  unsigned long long* part_count;   // [kMaxPart]
  double* wsum;            // [kMaxPart]
  unsigned long long* n_outside;
  const float* weight;     // may be null
};

__global__ void k_classify(SampleGeomParams g, int64_t ns, Thresholds th, ClassifyOut o) {
  // per-block partial results (shared-memory atomics), merged into the
  // global ones once per block: a global atomic per warp on the same dozen
  // addresses serialised the kernel
  __shared__ int s_win[kMaxPart * 4];
  __shared__ unsigned long long s_cnt[kMaxPart];
  __shared__ double s_w[kMaxPart];
  __shared__ unsigned long long s_out;
  for (int i = threadIdx.x; i < kMaxPart * 4; i += blockDim.x) s_win[i] = (i & 1) ? INT_MIN : INT_MAX;
  for (int i = threadIdx.x; i < kMaxPart; i += blockDim.x) {
    s_cnt[i] = 0ull;
    s_w[i] = 0.0;
  }
  if (threadIdx.x == 0) s_out = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < ns; s0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = s0 + threadIdx.x;
    const bool live = s < ns;
    Coords c;
    uint32_t mask = 0;
    int pju = 0, pjv = 0;
    float wt = 0.f;
    if (live) {
      c = sample_coords(g, s);
      if (c.inside) {
        for (int p = 0; p < th.nparts; ++p) {
          bool ok = true;
          if (p > 0) ok = ok && (c.r >= th.lo[p]);
          if (p < th.nparts - 1) ok = ok && (c.r <= th.hi[p]);
          mask |= (ok ? 1u : 0u) << p;
        }
        // first taps on the 4N PSF grid (image 2N): x' = u_l * (dl * 4N) + 2N
        const double x2 = __dadd_rn(__dmul_rn(c.ul, 2.0 * g.scale), 2.0 * g.half);
        const double y2 = __dadd_rn(__dmul_rn(c.vl, 2.0 * g.scale), 2.0 * g.half);
        pju = (int)ceil(__dadd_rn(x2, -0.5 * kW));
        pjv = (int)ceil(__dadd_rn(y2, -0.5 * kW));
      }
      wt = o.weight ? o.weight[s] : 1.0f;
      if (o.mask_out) o.mask_out[s] = (uint8_t)mask;
      o.counts[s] = __popc(mask);
    }
    const unsigned outside = __ballot_sync(0xffffffffu, live && !c.inside);
    if (lane == 0 && outside) atomicAdd(&s_out, (unsigned long long)__popc(outside));
    for (int p = 0; p < th.nparts; ++p) {
      const bool in = (mask >> p) & 1u;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (!bal) continue;
      int mn = in ? min(c.ju, c.jv) : INT_MAX;
      int mx = in ? max(c.ju, c.jv) : INT_MIN;
      int pmn = in ? min(pju, pjv) : INT_MAX;
      int pmx = in ? max(pju, pjv) : INT_MIN;
      double w = in ? (double)wt : 0.0;
      mn = __reduce_min_sync(0xffffffffu, mn);
      mx = __reduce_max_sync(0xffffffffu, mx);
      pmn = __reduce_min_sync(0xffffffffu, pmn);
      pmx = __reduce_max_sync(0xffffffffu, pmx);
      for (int off = 16; off; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
      if (lane == 0) {
        atomicMin(&s_win[p * 4 + 0], mn);
        atomicMax(&s_win[p * 4 + 1], mx);
        atomicMin(&s_win[p * 4 + 2], pmn);
        atomicMax(&s_win[p * 4 + 3], pmx);
        atomicAdd(&s_cnt[p], (unsigned long long)__popc(bal));
        atomicAdd(&s_w[p], w);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < th.nparts && s_cnt[threadIdx.x] > 0ull) {
    const int p = threadIdx.x;
    atomicMin(&o.win[p * 4 + 0], s_win[p * 4 + 0]);
    atomicMax(&o.win[p * 4 + 1], s_win[p * 4 + 1]);
    atomicMin(&o.win[p * 4 + 2], s_win[p * 4 + 2]);
    atomicMax(&o.win[p * 4 + 3], s_win[p * 4 + 3]);
    atomicAdd(&o.part_count[p], s_cnt[p]);
    atomicAdd(&o.wsum[p], s_w[p]);
  }
  if (threadIdx.x == 0 && s_out) atomicAdd(o.n_outside, s_out);
}

struct KeyLayout {
  int bt, bw, logT;
};

__global__ void k_scatter_entries(SampleGeomParams g, int64_t ns, int nparts, Thresholds th,
                                  KeyLayout kl, const uint32_t* __restrict__ off,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ samples) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    Coords c = sample_coords(g, s);
    if (!c.inside) continue;
    const int p0 = sample_plane(g, c.wl);
    uint32_t e = off[s];
    const uint32_t tile = ((uint32_t)p0 << (2 * kl.bt)) | ((uint32_t)(c.jv >> kl.logT) << kl.bt) |
                          (uint32_t)(c.ju >> kl.logT);
    for (int p = 0; p < nparts; ++p) {
      bool ok = true;
      if (p > 0) ok = ok && (c.r >= th.lo[p]);
      if (p < nparts - 1) ok = ok && (c.r <= th.hi[p]);
      if (!ok) continue;
      keys[e] = ((uint32_t)p << (2 * kl.bt + kl.bw)) | tile;
      samples[e] = (uint32_t)s;
      ++e;
    }
  }
}

__global__ void k_seg_flags(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ f) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    f[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1u : 0u;
}

__global__ void k_seg_starts(const uint32_t* __restrict__ f, const uint32_t* __restrict__ ex, int64_t n,
                             uint32_t* __restrict__ starts) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (f[e]) starts[ex[e]] = (uint32_t)e;
}

__global__ void k_seg_chunks(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ nseg_p,
                             int64_t n, uint32_t* __restrict__ chunks) {
  const uint32_t nseg = *nseg_p;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t end = (i + 1 < nseg) ? starts[i + 1] : n;
    chunks[i] = (uint32_t)((end - starts[i] + kChunk - 1) / kChunk);
  }
}

__global__ void k_items(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ nseg_p,
                        const uint32_t* __restrict__ chunks, const uint32_t* __restrict__ coff,
                        int64_t n, uint32_t* __restrict__ items, const uint32_t* __restrict__ nitems_p) {
  const uint32_t nseg = *nseg_p;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += (int64_t)gridDim.x * blockDim.x) {
    for (uint32_t c = 0; c < chunks[i]; ++c) items[coff[i] + c] = starts[i] + c * (uint32_t)kChunk;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) items[*nitems_p] = (uint32_t)n;
}

__global__ void k_item_ranges(const uint32_t* __restrict__ items, const uint32_t* __restrict__ nitems_p,
                              const int64_t* __restrict__ ent_begin, int nparts, int64_t* __restrict__ out) {
  const int p = threadIdx.x;
  if (p > nparts) return;
  const int64_t target = ent_begin[p];
  int64_t lo = 0, hi = *nitems_p;   // first item with begin >= target
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if ((int64_t)items[mid] < target) lo = mid + 1; else hi = mid;
  }
  out[p] = lo;
}

}  // namespace

// exported helpers ----------------------------------------------------------
int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, cudaStream_t st) {
  if (n <= 0) {
    if (total_dev) RIX_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st));
    return RIX_OK;
  }
  const int64_t nb = ceil_div(n, kScanTile);
  if (nb > 0x7fffffff) return set_error(RIX_EINVAL, "scan too large");
  if (nb == 1) {
    ::rix::note_launch(); k_scan_block<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
  } else {
    uint32_t* sums = nullptr;
    RIX_CUDA(::rix::malloc_async(&sums, 2 * nb * sizeof(uint32_t), st));
    ::rix::note_launch(); k_scan_block<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
    int rc = scan_exclusive_u32(sums, sums + nb, nb, nullptr, st);
    if (rc == RIX_OK) { ::rix::note_launch(); k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, sums + nb); }
    cudaFreeAsync(sums, st);
    if (rc != RIX_OK) return rc;
  }
  if (total_dev) { ::rix::note_launch(); k_total<<<1, 1, 0, st>>>(in, out, n, total_dev); }
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

int radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp, int64_t n,
                   int bits, cudaStream_t st, bool* in_tmp) {
  return radix_sort_impl<uint32_t, true>(keys, vals, keys_tmp, vals_tmp, n, bits, st, in_tmp);
}



static int grid_blocks(const Ctx* ctx, int64_t n, int threads) {
  int64_t b = ceil_div(std::max<int64_t>(n, 1), threads);
  return (int)std::min<int64_t>(b, (int64_t)ctx->num_sms * 16);
}

int partition_job(Job* job, const double* uvw, int64_t nrow, const float* weight, const double* ell_px,
                  double delta, uint8_t* mask_out, cudaStream_t st) {
  Ctx* ctx = job->ctx;
  const int P = job->n_part;
  const int nchan = job->desc.nchan;
  const int64_t ns = nrow * nchan;
  if (nrow < 0 || nrow > job->max_rows) return set_error(RIX_EINVAL, "nrow %lld outside [0, %lld]", (long long)nrow, (long long)job->max_rows);
  if (ns > (int64_t)0x7fffffff) return set_error(RIX_EINVAL, "too many samples (%lld)", (long long)ns);
  if (!(delta >= 0.0)) return set_error(RIX_EINVAL, "delta must be >= 0");
  if (nrow > 0 && !uvw) return set_error(RIX_EINVAL, "uvw is NULL");

  // resident copies of the inputs
  RIX_TRY(job->uvw.alloc(ctx, std::max<int64_t>(nrow, 1) * 3 * sizeof(double)));
  if (nrow > 0) RIX_CUDA(cudaMemcpyAsync(job->uvw.p, uvw, nrow * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (weight) {
    RIX_TRY(job->weight.alloc(ctx, std::max<int64_t>(ns, 1) * sizeof(float)));
    if (ns > 0) RIX_CUDA(cudaMemcpyAsync(job->weight.p, weight, ns * sizeof(float), cudaMemcpyDeviceToDevice, st));
  } else {
    job->weight.release();
  }

  SampleGeomParams g{};
  g.uvw = job->uvw.as<double>();
  g.inv_lambda = job->inv_lambda.as<double>();
  g.nrow = nrow;
  g.nchan = nchan;
  g.ng = job->ng;
  g.scale = job->desc.cell_rad * (double)job->ng;
  g.half = 0.5 * job->ng;
  g.ndl = job->desc.cell_rad * (double)job->desc.n;
  g.nw = job->nw;
  g.ww = job->ww;
  g.w_min = 0.0;
  g.dw = 1.0;

  // small device scratch block: [0,16) u64 minmax/counters, doubles, ints
  struct Small {
    unsigned long long wmm[2];
    unsigned long long part_count[kMaxPart];
    unsigned long long n_outside;
    double wsum[kMaxPart];
    double ells[kMaxPart];
    int win[kMaxPart * 4];
    uint32_t totals[4];
    int64_t ent_begin[kMaxPart + 1];
    int64_t item_range[kMaxPart + 1];
  };
  Small* sm_d = nullptr;
  RIX_CUDA(::rix::malloc_async(&sm_d, sizeof(Small), st));
  Small sm_h;
  std::memset(&sm_h, 0, sizeof(sm_h));
  sm_h.wmm[0] = ~0ull;
  for (int p = 0; p < kMaxPart; ++p) {
    sm_h.win[p * 4 + 0] = INT_MAX; sm_h.win[p * 4 + 1] = INT_MIN;
    sm_h.win[p * 4 + 2] = INT_MAX; sm_h.win[p * 4 + 3] = INT_MIN;
  }
  RIX_CUDA(cudaMemcpyAsync(sm_d, &sm_h, sizeof(Small), cudaMemcpyHostToDevice, st));
  auto fail = [&](int rc) { cudaFreeAsync(sm_d, st); return rc; };

  const int blocks = grid_blocks(ctx, ns, 256);
  // --- w-plane parameters ------------------------------------------------
  double w_min = 0.0, dw = 1.0;
  if (job->nw > 0 && ns > 0) {
    ::rix::note_launch(); k_w_minmax<<<blocks, 256, 0, st>>>(g, ns, sm_d->wmm);
    if (cudaGetLastError() != cudaSuccess) return fail(set_error(RIX_ECUDA, "k_w_minmax launch"));
    unsigned long long mm[2];
    if (cudaMemcpyAsync(mm, sm_d->wmm, sizeof(mm), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(set_error(RIX_ECUDA, "w range readback"));
    auto unord = [](unsigned long long b) {
      unsigned long long v = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
      double d; std::memcpy(&d, &v, sizeof(d)); return d;
    };
    const double wmin = unord(mm[0]), wmax = unord(mm[1]);
    w_min = wmin;
    dw = (wmax > wmin) ? (wmax - wmin) / (double)(job->nw - job->ww) : 1.0;
  }
  g.w_min = w_min;
  g.dw = dw;

  // --- uniform weighting (before the weight sums and every gridding) ------
  if (job->desc.weighting == RIX_WEIGHT_UNIFORM && ns > 0) {
    const int n = job->desc.n;
    double* dens = nullptr;
    if (::rix::malloc_async(&dens, (size_t)n * n * sizeof(double), st) != cudaSuccess)
      return fail(set_error(RIX_ENOMEM, "uniform weighting density"));
    const bool had = job->weight.p != nullptr;
    if (!had) {
      const int rc = job->weight.alloc(ctx, ns * sizeof(float));
      if (rc != RIX_OK) { cudaFreeAsync(dens, st); return fail(rc); }
    }
    const float* w_in = had ? job->weight.as<float>() : nullptr;
    if (cudaMemsetAsync(dens, 0, (size_t)n * n * sizeof(double), st) != cudaSuccess) {
      cudaFreeAsync(dens, st);
      return fail(set_error(RIX_ECUDA, "uniform weighting memset"));
    }
    ::rix::note_launch(); k_uniform_density<<<blocks, 256, 0, st>>>(g, ns, w_in, n, dens);
    ::rix::note_launch(); k_uniform_apply<<<blocks, 256, 0, st>>>(g, ns, w_in, n, dens, job->weight.as<float>());
    cudaFreeAsync(dens, st);
    if (cudaGetLastError() != cudaSuccess) return fail(set_error(RIX_ECUDA, "uniform weighting launch"));
  }

  // --- ring radii ---------------------------------------------------------
  double ells[kMaxPart] = {};
  if (P > 1) {
    if (ell_px) {
      for (int i = 0; i < P - 1; ++i) ells[i] = ell_px[i];
      for (int i = 1; i < P - 1; ++i)
        if (!(ells[i] > ells[i - 1])) return fail(set_error(RIX_EINVAL, "ell_px must be ascending"));
    } else if (ns > 0) {
      uint64_t* rb = nullptr;
      SelectState* sel = nullptr;
      if (::rix::malloc_async(&rb, ns * sizeof(uint64_t), st) != cudaSuccess ||
          ::rix::malloc_async(&sel, sizeof(SelectState), st) != cudaSuccess) {
        if (rb) cudaFreeAsync(rb, st);
        return fail(set_error(RIX_ENOMEM, "radius select scratch"));
      }
      ::rix::note_launch(); k_radius_bits<<<blocks, 256, 0, st>>>(g, ns, rb);
      ::rix::note_launch(); k_select_init<<<1, 256, 0, st>>>(sel, ns, P);
      const int hb = std::min(blocks, 4 * ctx->num_sms);
      for (int shift = 56; shift >= 0; shift -= 8) {
        ::rix::note_launch(); k_select_hist<<<hb, 256, 0, st>>>(rb, ns, P - 1, shift, sel);
        ::rix::note_launch(); k_select_step<<<1, 256, 0, st>>>(sel, P - 1);
      }
      ::rix::note_launch(); k_select_out<<<1, 32, 0, st>>>(sel, P - 1, sm_d->ells);
      cudaFreeAsync(rb, st);
      cudaFreeAsync(sel, st);
      if (cudaGetLastError() != cudaSuccess) return fail(set_error(RIX_ECUDA, "radius select launch"));
      if (cudaMemcpyAsync(ells, sm_d->ells, sizeof(ells), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail(set_error(RIX_ECUDA, "quantile readback"));
    }
  }
  Thresholds th{};
  th.nparts = P;
  for (int p = 0; p < P; ++p) {
    th.lo[p] = (p > 0) ? ells[p - 1] - delta : 0.0;
    th.hi[p] = (p < P - 1) ? ells[p] + delta : 0.0;
  }

  // --- classify -----------------------------------------------------------
  uint32_t* counts = nullptr;
  uint32_t* offs = nullptr;
  if (::rix::malloc_async(&counts, std::max<int64_t>(ns, 1) * sizeof(uint32_t), st) != cudaSuccess ||
      ::rix::malloc_async(&offs, std::max<int64_t>(ns, 1) * sizeof(uint32_t), st) != cudaSuccess)
    return fail(set_error(RIX_ENOMEM, "classify scratch"));
  ClassifyOut co{mask_out, counts, sm_d->win, sm_d->part_count, sm_d->wsum, &sm_d->n_outside,
                 job->weight.as<float>()};
  if (ns > 0) { ::rix::note_launch(); k_classify<<<blocks, 256, 0, st>>>(g, ns, th, co); }
  int rc = scan_exclusive_u32(counts, offs, ns, &sm_d->totals[0], st);
  if (rc != RIX_OK) return fail(rc);
  if (cudaMemcpyAsync(&sm_h, sm_d, sizeof(Small), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(set_error(RIX_ECUDA, "classify readback: %s", cudaGetErrorString(cudaGetLastError())));
  const int64_t n_ent = sm_h.totals[0];

  // --- entries and sort ---------------------------------------------------
  const int logT = ilog2(job->tile);
  KeyLayout kl{};
  kl.logT = logT;
  kl.bt = ilog2(job->ng / job->tile);
  const int nblk = job->nw > 0 ? job->nw - job->ww + 1 : 1;
  kl.bw = nblk > 1 ? ilog2(nblk) : 0;
  const int bp = P > 1 ? ilog2(P) : 0;
  job->bt = kl.bt; job->bw = kl.bw; job->bp = bp;
  const int key_bits = 2 * kl.bt + kl.bw + bp;
  if (key_bits > 32) return fail(set_error(RIX_EINVAL, "sort key needs %d bits", key_bits));

  RIX_TRY(job->keys.alloc(ctx, std::max<int64_t>(n_ent, 1) * sizeof(uint32_t)));
  RIX_TRY(job->samples.alloc(ctx, std::max<int64_t>(n_ent, 1) * sizeof(uint32_t)));
  uint32_t *kt = nullptr, *vt = nullptr;
  if (::rix::malloc_async(&kt, std::max<int64_t>(n_ent, 1) * sizeof(uint32_t), st) != cudaSuccess ||
      ::rix::malloc_async(&vt, std::max<int64_t>(n_ent, 1) * sizeof(uint32_t), st) != cudaSuccess)
    return fail(set_error(RIX_ENOMEM, "sort scratch"));
  if (ns > 0) {
    ::rix::note_launch(); 
    k_scatter_entries<<<blocks, 256, 0, st>>>(g, ns, P, th, kl, offs, job->keys.as<uint32_t>(),
                                              job->samples.as<uint32_t>());
  }
  bool in_tmp = false;
  rc = radix_sort_u32(job->keys.as<uint32_t>(), job->samples.as<uint32_t>(), kt, vt, n_ent, key_bits, st, &in_tmp);
  if (rc != RIX_OK) return fail(rc);
  if (in_tmp) {
    RIX_CUDA(cudaMemcpyAsync(job->keys.p, kt, n_ent * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    RIX_CUDA(cudaMemcpyAsync(job->samples.p, vt, n_ent * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  }

  // --- work items ----------------------------------------------------------
  // scratch: flags -> kt, exclusive scan -> vt, segment starts -> wa, chunk counts -> wb
  int64_t ent_begin[kMaxPart + 1];
  ent_begin[0] = 0;
  for (int p = 0; p < P; ++p) ent_begin[p + 1] = ent_begin[p] + (int64_t)sm_h.part_count[p];
  int64_t n_items = 0;
  uint32_t *wa = nullptr, *wb = nullptr;
  if (n_ent > 0) {
    if (::rix::malloc_async(&wa, n_ent * sizeof(uint32_t), st) != cudaSuccess ||
        ::rix::malloc_async(&wb, n_ent * sizeof(uint32_t), st) != cudaSuccess)
      return fail(set_error(RIX_ENOMEM, "work-item scratch"));
    const int eb = grid_blocks(ctx, n_ent, 256);
    ::rix::note_launch(); k_seg_flags<<<eb, 256, 0, st>>>(job->keys.as<uint32_t>(), n_ent, kt);
    rc = scan_exclusive_u32(kt, vt, n_ent, &sm_d->totals[1], st);
    if (rc != RIX_OK) return fail(rc);
    uint32_t* starts = wa;
    ::rix::note_launch(); k_seg_starts<<<eb, 256, 0, st>>>(kt, vt, n_ent, starts);
    uint32_t* chunks = wb;
    ::rix::note_launch(); k_seg_chunks<<<eb, 256, 0, st>>>(starts, &sm_d->totals[1], n_ent, chunks);
    // chunk offsets into kt (flags no longer needed)
    uint32_t nseg_h = 0;
    RIX_CUDA(cudaMemcpyAsync(&nseg_h, &sm_d->totals[1], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RIX_CUDA(cudaStreamSynchronize(st));
    rc = scan_exclusive_u32(chunks, kt, nseg_h, &sm_d->totals[2], st);
    if (rc != RIX_OK) return fail(rc);
    uint32_t nit_h = 0;
    RIX_CUDA(cudaMemcpyAsync(&nit_h, &sm_d->totals[2], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RIX_CUDA(cudaStreamSynchronize(st));
    n_items = nit_h;
    RIX_TRY(job->items.alloc(ctx, (n_items + 1) * sizeof(uint32_t)));
    ::rix::note_launch(); k_items<<<grid_blocks(ctx, nseg_h, 256), 256, 0, st>>>(starts, &sm_d->totals[1], chunks, kt, n_ent,
                                                         job->items.as<uint32_t>(), &sm_d->totals[2]);
    RIX_CUDA(cudaMemcpyAsync(sm_d->ent_begin, ent_begin, sizeof(ent_begin), cudaMemcpyHostToDevice, st));
    ::rix::note_launch(); k_item_ranges<<<1, 32, 0, st>>>(job->items.as<uint32_t>(), &sm_d->totals[2], sm_d->ent_begin, P,
                                    sm_d->item_range);
  } else {
    RIX_TRY(job->items.alloc(ctx, sizeof(uint32_t)));
    RIX_CUDA(cudaMemsetAsync(job->items.p, 0, sizeof(uint32_t), st));
    RIX_CUDA(cudaMemsetAsync(sm_d->item_range, 0, sizeof(sm_d->item_range), st));
  }
  RIX_CUDA(cudaMemcpyAsync(&sm_h, sm_d, sizeof(Small), cudaMemcpyDeviceToHost, st));
  RIX_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(kt, st);
  cudaFreeAsync(vt, st);
  if (wa) cudaFreeAsync(wa, st);
  if (wb) cudaFreeAsync(wb, st);
  cudaFreeAsync(counts, st);
  cudaFreeAsync(offs, st);
  cudaFreeAsync(sm_d, st);
  RIX_LAUNCH_CHECK();

  // --- host-side bookkeeping -----------------------------------------------
  job->n_entries = n_ent;
  job->n_items = n_items;
  std::memset(&job->stats, 0, sizeof(job->stats));
  rix_job_stats& S = job->stats;
  S.nrow = nrow;
  S.n_samples = ns;
  S.n_outside = (int64_t)sm_h.n_outside;
  S.n_entries = n_ent;
  S.delta_px = delta;
  S.w_min = w_min;
  S.dw = dw;
  S.n_work_items = n_items;
  for (int i = 0; i < P - 1; ++i) { S.ell_px[i] = ells[i]; job->ells[i] = ells[i]; }
  const int T = job->tile;
  for (int p = 0; p < P; ++p) {
    Part& pt = job->part[p];
    pt.ent_begin = ent_begin[p];
    pt.ent_count = (int64_t)sm_h.part_count[p];
    pt.item_begin = sm_h.item_range[p];
    pt.item_count = sm_h.item_range[p + 1] - sm_h.item_range[p];
    pt.wsum = sm_h.wsum[p];
    S.part_count[p] = pt.ent_count;
    S.part_weight[p] = pt.wsum;
    if (pt.ent_count > 0) {
      const int mn = sm_h.win[p * 4 + 0], mx = sm_h.win[p * 4 + 1];
      int lo = (mn / T) * T;
      int hi = (mx / T + 1) * T + kW;
      hi = std::min(job->ng, (hi + 7) / 8 * 8);
      pt.win_lo = lo;
      pt.win_n = hi - lo;
      const int pmn = sm_h.win[p * 4 + 2], pmx = sm_h.win[p * 4 + 3];
      int plo = std::max(0, (pmn / 8) * 8);
      int phi = std::min(2 * job->ng, (pmx + kW + 7) / 8 * 8);
      pt.pwin_lo = plo;
      pt.pwin_n = phi - plo;
    } else {
      pt.win_lo = job->ng / 2; pt.win_n = 8;
      pt.pwin_lo = job->ng; pt.pwin_n = 8;
    }
    S.window_lo[p] = pt.win_lo;
    S.window_size[p] = pt.win_n;
  }
  return RIX_OK;
}

}  // namespace rix
