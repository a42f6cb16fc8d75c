// a4-a7: G^dagger F and F^dagger G of Eq. 2 for one uv partition.
//
// Model image -> w-planes (correction, phase screen, pruned FFT; k_fft.cu)
// -> per work item (one uv tile of one w-plane block, at most 2048 sorted
// samples): stage the tile (+ kernel halo) of the 8 model planes it touches
// into shared memory, degrid each sample with a warp (32 lanes x 16 taps,
// warp-shuffle reduction), form the weighted residual, spread it into a
// shared-memory sub-grid, and flush that sub-grid once per work item with
// vector atomics -> residual planes -> inverse pruned FFT, conjugate phase
// screen, sum over planes, correction -> residual image.
//
// Precision: sample coordinates, the kernel argument offsets and the w-plane
// phases are formed in FP64; kernel weights, accumulation and FFTs in the
// job's precision (FP32 or FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <type_traits>
#include <vector>

#include "rix_internal.cuh"

namespace rix {
namespace {


// ----------------------------------------------------------- host tables ----
// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// Fourier transform of the ES kernel over cell units,
//   Phi(f) = (W/2) int_{-1}^{1} phi(z) cos(pi W z f) dz,
// with z = sin(t) (analytic integrand), by Gauss-Legendre quadrature in t.
struct EsFourier {
  std::vector<double> st, wt;
  EsFourier() {
    std::vector<double> x, w;
    gauss_legendre(96, x, w);
    st.resize(x.size());
    wt.resize(x.size());
    for (size_t k = 0; k < x.size(); ++k) {
      const double t = 0.5 * M_PI * x[k];
      st[k] = std::sin(t);
      wt[k] = 0.5 * M_PI * w[k] * std::exp(kBeta * (std::cos(t) - 1.0)) * std::cos(t);
    }
  }
  double operator()(double f) const {
    double acc = 0.0;
    for (size_t k = 0; k < st.size(); ++k) acc += wt[k] * std::cos(M_PI * kW * f * st[k]);
    return 0.5 * kW * acc;
  }
};

// Chebyshev coefficients of Phi on [lo, hi] (degree kCheb - 1): Phi is entire
// and |pi W f| <= 2 pi over the w-correction's range, so 40 terms reach
// double precision.
constexpr int kCheb = 40;
void chebyshev_fit(const EsFourier& phi, double lo, double hi, double* c) {
  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  double f[kCheb];
  for (int k = 0; k < kCheb; ++k) f[k] = phi(mid + half * std::cos(M_PI * (k + 0.5) / kCheb));
  for (int j = 0; j < kCheb; ++j) {
    double acc = 0.0;
    for (int k = 0; k < kCheb; ++k) acc += f[k] * std::cos(M_PI * j * (k + 0.5) / kCheb);
    c[j] = 2.0 * acc / kCheb;
  }
  c[0] *= 0.5;
}

struct CorrArgs {
  int M;
  int ox, oy;           // pixel offset of the table's centre from the phase centre
  double cell;
  const double* p1;     // Phi((a - M/2) / Ng), [M]
  int wstack;
  double dw, lo, hi;    // Chebyshev interval of dw (n - 1)
  double cheb[kCheb];
};

// corr[b][a] = 1 / (Phi(a'/Ng) Phi(b'/Ng) [n Phi(dw (n-1))]),  nm1[b][a] = n - 1,
// with a' = a - M/2, b' = b - M/2 the offsets from the table's centre and n at
// the sky position (a' + ox, b' + oy) cells from the phase centre
template <typename R>
__global__ void k_corrections(CorrArgs a, R* __restrict__ corr, double* __restrict__ nm1) {
  const int64_t tot = (int64_t)a.M * a.M;
  const int h = a.M / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / a.M), c = (int)(i - (int64_t)b * a.M);
    double v = 1.0 / (a.p1[c] * a.p1[b]);
    if (a.wstack) {
      const double l = (double)(c - h + a.ox) * a.cell, m = (double)(b - h + a.oy) * a.cell;
      const double r2 = __dadd_rn(__dmul_rn(l, l), __dmul_rn(m, m));
      const double n = __dsqrt_rn(1.0 - r2);
      const double d = -r2 / (1.0 + n);
      double phw;
      if (a.hi > a.lo) {
        // Clenshaw recurrence for sum_j c_j T_j(x)
        const double x = (2.0 * a.dw * d - (a.lo + a.hi)) / (a.hi - a.lo);
        double b1 = 0.0, b2 = 0.0;
        for (int j = kCheb - 1; j >= 1; --j) {
          const double t = 2.0 * x * b1 - b2 + a.cheb[j];
          b2 = b1;
          b1 = t;
        }
        phw = x * b1 - b2 + a.cheb[0];
      } else {
        phw = a.cheb[0];
      }
      v /= n * phw;
      nm1[i] = d;
    }
    corr[i] = (R)v;
  }
}

// dw (n - 1) -> n Phi(dw (n - 1)) and n - 1 at squared radius r2 (a Clenshaw
// sum of the Chebyshev fit of Phi)
__device__ __forceinline__ double wfactor(const CorrArgs& a, double r2, double* nm1_out) {
  const double n = __dsqrt_rn(1.0 - r2);
  const double d = -r2 / (1.0 + n);
  double phw;
  if (a.hi > a.lo) {
    const double x = (2.0 * a.dw * d - (a.lo + a.hi)) / (a.hi - a.lo);
    double b1 = 0.0, b2 = 0.0;
    for (int j = kCheb - 1; j >= 1; --j) {
      const double t = 2.0 * x * b1 - b2 + a.cheb[j];
      b2 = b1;
      b1 = t;
    }
    phw = x * b1 - b2 + a.cheb[0];
  } else {
    phw = a.cheb[0];
  }
  *nm1_out = d;
  return n * phw;
}

// k_corrections for a table centred on the phase centre (ox = oy = 0): the
// w-factor depends on l^2 + m^2 only, so one thread per pixel of the quadrant
// [0, M/2]^2 evaluates it once and writes the up to four pixels (b, c),
// (b, M - c), (M - b, c), (M - b, M - c) that share it
template <typename R>
__global__ void k_corrections_sym(CorrArgs a, R* __restrict__ corr, double* __restrict__ nm1) {
  const int h = a.M / 2;
  const int64_t q = (int64_t)(h + 1) * (h + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / (h + 1)), c = (int)(i - (int64_t)b * (h + 1));
    double wf = 1.0, d = 0.0;
    if (a.wstack) {
      const double l = (double)(c - h) * a.cell, m = (double)(b - h) * a.cell;
      wf = wfactor(a, __dadd_rn(__dmul_rn(l, l), __dmul_rn(m, m)), &d);
    }
    const int bs[2] = {b, 2 * h - b}, cs[2] = {c, 2 * h - c};
    for (int u = 0; u < 2; ++u) {
      const int bb = bs[u];
      if (bb >= a.M || (u == 1 && bb == b)) continue;
      for (int w = 0; w < 2; ++w) {
        const int cc = cs[w];
        if (cc >= a.M || (w == 1 && cc == c)) continue;
        const int64_t pix = (int64_t)bb * a.M + cc;
        corr[pix] = (R)(1.0 / (a.p1[cc] * a.p1[bb] * wf));
        if (a.wstack) nm1[pix] = d;
      }
    }
  }
}

// Fills the M x M tables corr and nm1 (w-stacked jobs) for grid side ng,
// centred ox, oy cells from the phase centre; the w-correction's Chebyshev
// fit covers a field of half side `half_px` cells about the phase centre.
template <typename R>
int fill_correction(Job* job, int M, int ng, int ox, int oy, int half_px, R* corr, double* nm1, cudaStream_t st) {
  static const EsFourier phi;
  const bool ws = job->nw > 0;
  const double cell = job->desc.cell_rad, dw = job->stats.dw;
  std::vector<double> p1(M);
  for (int a = 0; a < M; ++a) p1[a] = phi((double)(a - M / 2) / ng);
  CorrArgs ca{};
  ca.M = M;
  ca.ox = ox;
  ca.oy = oy;
  ca.cell = cell;
  ca.wstack = ws;
  ca.dw = dw;
  if (ws) {
    // the most negative dw (n - 1) is at the field's corner
    const double l = (double)(-half_px) * cell;
    const double r2 = 2.0 * l * l;
    const double n = std::sqrt(1.0 - r2);
    const double dmin = dw * (-r2 / (1.0 + n));
    ca.lo = std::min(dmin, 0.0) * (1.0 + 1e-12);
    ca.hi = 0.0;
    if (ca.hi > ca.lo) chebyshev_fit(phi, ca.lo, ca.hi, ca.cheb);
    else ca.cheb[0] = phi(0.0);
    job->stats.max_dw_nm1 = std::max(job->stats.max_dw_nm1, std::fabs(dmin));
  }
  double* p1d = nullptr;
  RIX_CUDA(::rix::malloc_async((void**)&p1d, M * sizeof(double), st));
  RIX_CUDA(cudaMemcpyAsync(p1d, p1.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
  ca.p1 = p1d;
  const int64_t tot = (int64_t)M * M;
  const int blocks = (int)std::min<int64_t>(ceil_div(tot, 256), (int64_t)job->ctx->num_sms * 16);
  ::rix::note_launch();
  if (ox == 0 && oy == 0) k_corrections_sym<R><<<blocks, 256, 0, st>>>(ca, corr, ws ? nm1 : nullptr);
  else k_corrections<R><<<blocks, 256, 0, st>>>(ca, corr, ws ? nm1 : nullptr);
  cudaFreeAsync(p1d, st);
  RIX_LAUNCH_CHECK();
  RIX_CUDA(cudaStreamSynchronize(st));   // p1 is a host temporary
  return RIX_OK;
}

template <typename R>
int build_correction(Job* job, int M, int ng, DevBuf& corr, DevBuf& nm1, cudaStream_t st) {
  RIX_TRY(corr.alloc(job->ctx, (size_t)M * M * sizeof(R)));
  if (job->nw > 0) RIX_TRY(nm1.alloc(job->ctx, (size_t)M * M * sizeof(double)));
  return fill_correction<R>(job, M, ng, 0, 0, M / 2, corr.as<R>(), job->nw > 0 ? nm1.as<double>() : nullptr, st);
}

// --------------------------------------------------------------- kernels ----

struct TileArgs {
  const uint32_t* keys;
  const uint32_t* samples;
  const uint32_t* items;
  int64_t item_begin, item_count;
  const double* uvw;
  const double* inv_lambda;
  int nchan;
  double scale, half;       // grid coordinate x = u_l * scale + half
  int nw, ww;
  double w_min, dw;
  int bt, bw, logT;
  int win_lo, S;            // plane window [win_lo, win_lo + S)^2
  const void* model;        // cplx [planes][S][S], u-major
  void* out;                // cplx [planes][S][S]
  const void* vis_in;       // cplx per sample
  void* vis_out;            // cplx per sample
  const float* weight;      // per sample or null
  const void* geom;         // EntryGeom<R> per sorted entry, from entry geom_off on
  int64_t geom_off;
  int64_t ent_begin, ent_count;   // the partition's entries
  int* status;              // the job's status word (RIX_EINTERNAL on a failed check)
};

// On the PSF's 2N grid (x_psf = 2 x exactly), an image-grid tile of side T
// at tx T maps to first taps in [2 tx T + 3, 2 tx T + 2 T + 2]: the staged
// region starts kPsfOrg cells after 2 tx T and has side 2 T + 9.
constexpr int kPsfOrg = 2;
template <int T> constexpr int psf_staged_side() { return 2 * T + 9; }

template <int T, int MODE> struct TileGeom {
  // staged side and origin offset (in grid cells) relative to the tile origin
  static constexpr int SP = (MODE == kPsf) ? psf_staged_side<T>() : T + kW - 1;
  static constexpr int ORG = (MODE == kPsf) ? kPsfOrg : 0;
  // plane stride in elements, == 8 (mod 16) so that the two plane halves of a
  // half-warp land on disjoint banks
  static constexpr int PL = ((SP * SP + 7) / 16) * 16 + 8;
};

// geometry of the sorted entries [e_off, e_off + n) into out[0, n): on the
// image grid (first tap relative to the tile origin tx T) or, kPsfGrid, on the
// PSF's 2N grid (a.scale, a.half of that grid; relative to 2 tx T + kPsfOrg)
template <typename R, bool kPsfGrid, int T>
__global__ void k_entry_geom(TileArgs a, int64_t e_off, int64_t n, EntryGeom<R>* __restrict__ out) {
  const uint32_t tmask = (1u << a.bt) - 1u;
  constexpr int kLim = kPsfGrid ? psf_staged_side<T>() - kW : T - 1;   // largest first-tap offset
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = e_off + i;
    const uint32_t key = a.keys[e];
    const int tx = (int)(key & tmask), ty = (int)((key >> a.bt) & tmask);
    const int gu0 = kPsfGrid ? 2 * tx * T + kPsfOrg : tx * T;
    const int gv0 = kPsfGrid ? 2 * ty * T + kPsfOrg : ty * T;
    const uint32_t s = a.samples[e];
    const int64_t row = s / (uint32_t)a.nchan;
    const int ch = (int)(s - row * a.nchan);
    const double sc = a.inv_lambda[ch];
    const double ul = __dmul_rn(a.uvw[row * 3 + 0], sc);
    const double vl = __dmul_rn(a.uvw[row * 3 + 1], sc);
    const double x = __dadd_rn(__dmul_rn(ul, a.scale), a.half);
    const double y = __dadd_rn(__dmul_rn(vl, a.scale), a.half);
    const double xs = __dadd_rn(x, -0.5 * kW), ys = __dadd_rn(y, -0.5 * kW);
    const double cx = ceil(xs), cy = ceil(ys);
    int ou = (int)cx - gu0, ov = (int)cy - gv0;
    EntryGeom<R> g;
    g.du = (R)__dadd_rn(cx, -xs);
    g.dv = (R)__dadd_rn(cy, -ys);
    g.dw = R(0);
    if (a.nw > 0) {
      const double wl = __dmul_rn(a.uvw[row * 3 + 2], sc);
      const double tw = __ddiv_rn(__dadd_rn(wl, -a.w_min), a.dw);
      const double pc = fmin(fmax(ceil(tw), 0.0), (double)(a.nw - a.ww));
      g.dw = (R)__dadd_rn(pc, -tw);
    }
    // the first tap lies in the entry's tile (staged region) by construction
    // of the key; an entry that does not is flagged (RIX_EINTERNAL at the
    // next rix_job_sync) and its offsets are kept in range so that no access
    // leaves the staged tile
    if (ou < 0 || ov < 0 || ou > kLim || ov > kLim) {
      atomicCAS(a.status, 0, RIX_EINTERNAL);
      ou = min(max(ou, 0), kLim);
      ov = min(max(ov, 0), kLim);
    }
    g.ouv = (uint32_t)ou | ((uint32_t)ov << 8);
    out[i] = g;
  }
}

template <typename R, int WW, int T, int MODE>
__global__ void __launch_bounds__(256) k_tiles(TileArgs a) {
  using C = cplx<R>;
  using TG = TileGeom<T, MODE>;
  constexpr int SP = TG::SP, PL = TG::PL;
  constexpr int G = (WW == 1) ? 8 : 32;       // lanes per sample
  constexpr int SPW = 32 / G;                 // samples per warp at once
  constexpr int RPL = WW * kW / G;            // rows of 8 taps per lane
  constexpr bool kUseModel = (MODE == kDegrid || MODE == kResid);
  constexpr bool kUseGrid = (MODE != kDegrid);
  extern __shared__ __align__(32) unsigned char smem_raw[];
  C* sm_model = reinterpret_cast<C*>(smem_raw);
  C* sm_grid = sm_model + (kUseModel ? WW * PL : 0);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int gl = lane % G, grp = lane / G;
  const int64_t SS = (int64_t)a.S * a.S;
  const C* model = static_cast<const C*>(a.model);
  C* out = static_cast<C*>(a.out);
  const C* vin = static_cast<const C*>(a.vis_in);
  C* vout = static_cast<C*>(a.vis_out);
  const uint32_t tmask = (1u << a.bt) - 1u;

  for (int64_t it = blockIdx.x; it < a.item_count; it += gridDim.x) {
    const int64_t item = a.item_begin + it;
    const uint32_t e0 = a.items[item], e1 = a.items[item + 1];
    const uint32_t key = a.keys[e0];
    const int tx = (int)(key & tmask), ty = (int)((key >> a.bt) & tmask);
    const int p0 = (WW > 1) ? (int)((key >> (2 * a.bt)) & ((1u << a.bw) - 1u)) : 0;
    const int gu0 = (MODE == kPsf ? 2 * tx * T : tx * T) + TG::ORG;   // grid coords of smem (0, 0)
    const int gv0 = (MODE == kPsf ? 2 * ty * T : ty * T) + TG::ORG;
    const int u0 = gu0 - a.win_lo, v0 = gv0 - a.win_lo;

    for (int idx = threadIdx.x; idx < WW * SP * SP; idx += blockDim.x) {
      const int pl = idx / (SP * SP), rem = idx - pl * (SP * SP);
      const int iu = rem / SP, iv = rem - iu * SP;
      if (kUseModel) {
        const int u = u0 + iu, v = v0 + iv;
        C val = cmake<C>(0.0, 0.0);
        if (u >= 0 && u < a.S && v >= 0 && v < a.S) val = model[(p0 + pl) * SS + (int64_t)u * a.S + v];
        sm_model[pl * PL + iu * SP + iv] = val;
      }
      if (kUseGrid) sm_grid[pl * PL + iu * SP + iv] = cmake<C>(0.0, 0.0);
    }
    __syncthreads();

    for (uint32_t base = e0 + warp * 32; base < e1; base += nwarps * 32) {
      const int nvalid = (int)min(32u, e1 - base);
      const bool valid = lane < nvalid;
      // ---- per-lane sample geometry ----
      const uint32_t s = valid ? a.samples[base + lane] : 0u;
      int ou = 0, ov = 0;
      R du = R(0), dv = R(0), dwo = R(0);
      // precomputed per entry (image grid: at partition time; PSF: before
      // the PSF's launch)
      if (valid) {
        const EntryGeom<R> g = static_cast<const EntryGeom<R>*>(a.geom)[base + lane - a.geom_off];
        ou = (int)(g.ouv & 0xffu);
        ov = (int)(g.ouv >> 8);
        du = g.du; dv = g.dv; dwo = g.dw;
      }
      if (!valid) { ou = 0; ov = 0; }
      // guard against any sample outside the staged region (never expected)
      if (ou < 0 || ov < 0 || ou > SP - kW || ov > SP - kW) { ou = 0; ov = 0; }
      R vre = R(0), vim = R(0), wt = R(0);
      if (valid) {
        wt = a.weight ? (R)a.weight[s] : R(1);
        if (MODE == kGrid || MODE == kResid) { const C v = vin[s]; vre = v.x; vim = v.y; }
        if (MODE == kPsf) vre = R(1);
      }

      for (int k0 = 0; k0 < nvalid; k0 += SPW) {
        const int k = k0 + grp;
        const bool kvalid = k < nvalid;
        const int src = kvalid ? k : 0;
        const int kou = __shfl_sync(0xffffffffu, ou, src);
        const int kov = __shfl_sync(0xffffffffu, ov, src);
        const R kdu = __shfl_sync(0xffffffffu, du, src);
        const R kdv = __shfl_sync(0xffffffffu, dv, src);
        // ---- kernel weights, computed lane-parallel and broadcast ----
        R wu[kW];
        R wvr[RPL];          // v weight times w weight of each row this lane owns
        int rbase[RPL];      // smem offset of (plane, v row) of each row
        if constexpr (G == 32) {
          const R kdw = __shfl_sync(0xffffffffu, dwo, src);
          // lanes 0-7: u weights, 8-15: v weights, 16 .. 16 + WW - 1: w weights
          const R kd = gl < 8 ? kdu : (gl < 16 ? kdv : kdw);
          const R myw = gl < 16 + WW ? es_weight<R>(kd, gl & 7) : R(0);
#pragma unroll
          for (int i = 0; i < kW; ++i) wu[i] = __shfl_sync(0xffffffffu, myw, i);
          const int vrow = gl & 7, plh = gl >> 3;
          const R wv = __shfl_sync(0xffffffffu, myw, 8 + vrow);
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            const int pl = plh + 4 * r;
            const R ww = __shfl_sync(0xffffffffu, myw, 16 + pl);
            wvr[r] = wv * ww;
            rbase[r] = pl * PL + kou * SP + kov + vrow;
          }
        } else {
          const R myu = es_weight<R>(kdu, gl);
          const R myv = es_weight<R>(kdv, gl);
#pragma unroll
          for (int i = 0; i < kW; ++i) wu[i] = __shfl_sync(0xffffffffu, myu, grp * G + i);
          wvr[0] = myv;
          rbase[0] = kou * SP + kov + gl;
        }
        // ---- degrid ----
        R accr = R(0), acci = R(0);
        if constexpr (kUseModel) {
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int i = 0; i < kW; ++i) {
              const C g = sm_model[rbase[r] + i * SP];
              sr += wu[i] * g.x;
              si += wu[i] * g.y;
            }
            accr += wvr[r] * sr;
            acci += wvr[r] * si;
          }
#pragma unroll
          for (int o = G / 2; o; o >>= 1) {
            accr += __shfl_xor_sync(0xffffffffu, accr, o);
            acci += __shfl_xor_sync(0xffffffffu, acci, o);
          }
        }
        if constexpr (MODE == kDegrid) {
          const uint32_t ks = __shfl_sync(0xffffffffu, s, src);
          if (kvalid && gl == 0) vout[ks] = cmake<C>(accr, acci);
        } else {
          // ---- grid the weighted (residual) visibility ----
          const R kvr = __shfl_sync(0xffffffffu, vre, src);
          const R kvi = __shfl_sync(0xffffffffu, vim, src);
          const R kwt = __shfl_sync(0xffffffffu, wt, src);
          R yr = kwt * kvr, yi = kwt * kvi;
          if (MODE == kResid) { yr = kwt * (kvr - accr); yi = kwt * (kvi - acci); }
          if (kvalid) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              const R cr = yr * wvr[r], ci = yi * wvr[r];
#pragma unroll
              for (int i = 0; i < kW; ++i) {
                C* g = &sm_grid[rbase[r] + i * SP];
                atomicAdd(&g->x, cr * wu[i]);
                if (MODE != kPsf) atomicAdd(&g->y, ci * wu[i]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    if constexpr (kUseGrid) {
      for (int idx = threadIdx.x; idx < WW * SP * SP; idx += blockDim.x) {
        const int pl = idx / (SP * SP), rem = idx - pl * (SP * SP);
        const int iu = rem / SP, iv = rem - iu * SP;
        const int u = u0 + iu, v = v0 + iv;
        const C val = sm_grid[pl * PL + iu * SP + iv];
        if ((val.x != R(0) || val.y != R(0)) && u >= 0 && u < a.S && v >= 0 && v < a.S) {
          C* dst = &out[(p0 + pl) * SS + (int64_t)u * a.S + v];
          if constexpr (sizeof(R) == 4) {
            atomicAdd(reinterpret_cast<float2*>(dst), *reinterpret_cast<const float2*>(&val));
          } else {
            atomicAdd(&dst->x, val.x);
            atomicAdd(&dst->y, val.y);
          }
        }
      }
      __syncthreads();
    }
  }
}

template <typename R, int WW, int T, int MODE>
int launch_tiles_impl(const Ctx* ctx, const TileArgs& a, cudaStream_t st) {
  using TG = TileGeom<T, MODE>;
  constexpr bool kUseModel = (MODE == kDegrid || MODE == kResid);
  constexpr bool kUseGrid = (MODE != kDegrid);
  const size_t sm = (size_t)(int(kUseModel) + int(kUseGrid)) * WW * TG::PL * sizeof(cplx<R>);
  auto kern = k_tiles<R, WW, T, MODE>;
  RIX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm));
  per_sm = std::max(per_sm, 1);
  const int64_t blocks = std::min<int64_t>(a.item_count, (int64_t)ctx->num_sms * per_sm);
  if (blocks <= 0) return RIX_OK;
  timing_mark(kTimeTiles, st, true);
  ::rix::note_launch(); kern<<<(unsigned)blocks, 256, sm, st>>>(a);
  timing_mark(kTimeTiles, st, false);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

// ---- w-stacked gridding without shared-memory atomics ----------------------
// Phase A: each warp degrids 4 samples of a 32-sample batch (32 lanes x 16
// taps, shuffle reduction) and stores per-sample records (weighted residual,
// tap origin, the 24 kernel weights).  Phase B: warp w owns w-plane w of the
// staged sub-grid and applies every record of the batch to it with plain
// read-modify-writes: lane (v row = lane & 7, u taps lane >> 3 and +4) touches
// distinct cells, warps touch distinct planes, so nothing races.
template <int T, int MODE> struct WsGeom {
  static constexpr int SP = (MODE == kPsf) ? psf_staged_side<T>() : T + kW - 1;       // staged side
  static constexpr int ORG = (MODE == kPsf) ? kPsfOrg : 0;
  static constexpr int SPP = (MODE == kPsf) ? SP : ((SP + 7) / 16) * 16 + 8;   // row stride, 8 mod 16
  static constexpr int PL = ((SP * SPP + 7) / 16) * 16 + 8;                // plane stride, 8 mod 16
};

template <typename R>
struct alignas(4 * sizeof(R)) WsRecord {
  // header, one vector load: weighted residual and the tap origin (ou | ov << 8)
  R yr, yi;
  uint32_t ouv;
  uint32_t pad[sizeof(R) == 8 ? 3 : 1];   // the weights start on a 4 sizeof(R) boundary
  // u weights in pairs (u_i, u_{i+4}) at [2i, 2i + 1] for i < 4, then the 8
  // v weights and the 8 w weights
  R w[3 * kW];
};

// header of a record as loaded by phase B
static_assert(offsetof(WsRecord<float>, w) == 16 && sizeof(WsRecord<float>) % 16 == 0, "record layout");
static_assert(offsetof(WsRecord<double>, w) == 32 && sizeof(WsRecord<double>) % 32 == 0, "record layout");
template <typename R> struct WsHead { R yr, yi; uint32_t ouv; };
__device__ __forceinline__ WsHead<float> ws_head(const WsRecord<float>& r) {
  const float4 h = *reinterpret_cast<const float4*>(&r);
  return {h.x, h.y, __float_as_uint(h.z)};
}
__device__ __forceinline__ WsHead<double> ws_head(const WsRecord<double>& r) {
  const double2 h = *reinterpret_cast<const double2*>(&r);
  return {h.x, h.y, r.ouv};
}

constexpr int kWsBatch = 32;

template <typename R, int T, int MODE>
__global__ void __launch_bounds__(256) k_tiles_ws(TileArgs a) {
  using C = cplx<R>;
  using TG = WsGeom<T, MODE>;
  constexpr int SP = TG::SP, SPP = TG::SPP, PL = TG::PL;
  constexpr bool kUseModel = (MODE == kResid);
  extern __shared__ __align__(32) unsigned char smem_raw[];
  C* sm_model = reinterpret_cast<C*>(smem_raw);
  C* sm_grid = sm_model + (kUseModel ? kW * PL : 0);
  WsRecord<R>* rec = reinterpret_cast<WsRecord<R>*>(sm_grid + kW * PL);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int64_t SS = (int64_t)a.S * a.S;
  const C* model = static_cast<const C*>(a.model);
  C* out = static_cast<C*>(a.out);
  const C* vin = static_cast<const C*>(a.vis_in);
  const uint32_t tmask = (1u << a.bt) - 1u;
  const int per_warp = kWsBatch / nwarps;

  for (int64_t it = blockIdx.x; it < a.item_count; it += gridDim.x) {
    const int64_t item = a.item_begin + it;
    const uint32_t e0 = a.items[item], e1 = a.items[item + 1];
    const uint32_t key = a.keys[e0];
    const int tx = (int)(key & tmask), ty = (int)((key >> a.bt) & tmask);
    const int p0 = (int)((key >> (2 * a.bt)) & ((1u << a.bw) - 1u));
    const int gu0 = (MODE == kPsf ? 2 * tx * T : tx * T) + TG::ORG;
    const int gv0 = (MODE == kPsf ? 2 * ty * T : ty * T) + TG::ORG;
    const int u0 = gu0 - a.win_lo, v0 = gv0 - a.win_lo;

    for (int idx = threadIdx.x; idx < kW * SP * SP; idx += blockDim.x) {
      const int pl = idx / (SP * SP), rem = idx - pl * (SP * SP);
      const int iu = rem / SP, iv = rem - iu * SP;
      if (kUseModel) {
        const int u = u0 + iu, v = v0 + iv;
        C val = cmake<C>(0.0, 0.0);
        if (u >= 0 && u < a.S && v >= 0 && v < a.S) val = model[(p0 + pl) * SS + (int64_t)u * a.S + v];
        sm_model[pl * PL + iu * SPP + iv] = val;
      }
      sm_grid[pl * PL + iu * SPP + iv] = cmake<C>(0.0, 0.0);
    }
    __syncthreads();

    for (uint32_t base = e0; base < e1; base += kWsBatch) {
      const int nb = (int)min((uint32_t)kWsBatch, e1 - base);
      // ---------------- phase A: weights, degrid, records ----------------------
      {
        const int j0 = warp * per_warp;
        const bool valid = lane < per_warp && j0 + lane < nb;
        const uint32_t s = valid ? a.samples[base + j0 + lane] : 0u;
        int ou = 0, ov = 0;
        R du = R(0), dv = R(0), dwo = R(0);
        if (valid) {
          // precomputed per entry (image grid: at partition time; PSF: before
          // the PSF's launch)
          const EntryGeom<R> g = static_cast<const EntryGeom<R>*>(a.geom)[base + j0 + lane - a.geom_off];
          ou = (int)(g.ouv & 0xffu);
          ov = (int)(g.ouv >> 8);
          du = g.du; dv = g.dv; dwo = g.dw;
        }
        if (!valid || ou < 0 || ov < 0 || ou > SP - kW || ov > SP - kW) { ou = 0; ov = 0; }
        R vre = R(0), vim = R(0), wt = R(0);
        if (valid) {
          wt = a.weight ? (R)a.weight[s] : R(1);
          if (MODE == kGrid || MODE == kResid) { const C v = vin[s]; vre = v.x; vim = v.y; }
          if (MODE == kPsf) vre = R(1);
        }
        for (int j = 0; j < per_warp && j0 + j < nb; ++j) {
          const int kou = __shfl_sync(0xffffffffu, ou, j);
          const int kov = __shfl_sync(0xffffffffu, ov, j);
          const R kdu = __shfl_sync(0xffffffffu, du, j);
          const R kdv = __shfl_sync(0xffffffffu, dv, j);
          const R kdw = __shfl_sync(0xffffffffu, dwo, j);
          // lanes 0-7: u weights, 8-15: v weights, 16-23: w weights
          const R kd = lane < 8 ? kdu : (lane < 16 ? kdv : kdw);
          const R myw = lane < 24 ? es_weight<R>(kd, lane & 7) : R(0);
          WsRecord<R>& rc = rec[j0 + j];
          if (lane < 24) rc.w[lane < 8 ? 2 * (lane & 3) + (lane >> 2) : lane] = myw;
          R accr = R(0), acci = R(0);
          if constexpr (kUseModel) {
            R wu[kW];
#pragma unroll
            for (int i = 0; i < kW; ++i) wu[i] = __shfl_sync(0xffffffffu, myw, i);
            const int vrow = lane & 7, plh = lane >> 3;
            const R wv = __shfl_sync(0xffffffffu, myw, 8 + vrow);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const int pl = plh + 4 * r;
              const R wvw = wv * __shfl_sync(0xffffffffu, myw, 16 + pl);
              const C* gp = sm_model + pl * PL + kou * SPP + kov + vrow;
              R sr = R(0), si = R(0);
#pragma unroll
              for (int i = 0; i < kW; ++i) {
                const C g = gp[i * SPP];
                sr += wu[i] * g.x;
                si += wu[i] * g.y;
              }
              accr += wvw * sr;
              acci += wvw * si;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
              accr += __shfl_xor_sync(0xffffffffu, accr, o);
              acci += __shfl_xor_sync(0xffffffffu, acci, o);
            }
          }
          const R kvr = __shfl_sync(0xffffffffu, vre, j);
          const R kvi = __shfl_sync(0xffffffffu, vim, j);
          const R kwt = __shfl_sync(0xffffffffu, wt, j);
          if (lane == 0) {
            rc.yr = kwt * (kvr - accr);
            rc.yi = kwt * (kvi - acci);
            rc.ouv = (uint32_t)kou | ((uint32_t)kov << 8);
          }
        }
      }
      __syncthreads();
      // ---------------- phase B: warp w applies the batch to plane w ----------
      {
        const int vrow = lane & 7, ig = lane >> 3;
        C* gpl = sm_grid + warp * PL;
        for (int k = 0; k < nb; ++k) {
          const WsRecord<R>& rc = rec[k];
          const WsHead<R> hd = ws_head(rc);
          const R f = rc.w[2 * kW + warp] * rc.w[kW + vrow];
          const R cr = hd.yr * f, ci = hd.yi * f;
          C* cell = gpl + ((int)(hd.ouv & 0xffu) + ig) * SPP + (int)(hd.ouv >> 8) + vrow;
          using R2 = cplx<R>;
          const R2 wp = *reinterpret_cast<const R2*>(&rc.w[2 * ig]);
          const R w0 = wp.x, w1 = wp.y;
          C g0 = cell[0], g1 = cell[4 * SPP];
          g0.x += cr * w0; g0.y += ci * w0;
          g1.x += cr * w1; g1.y += ci * w1;
          cell[0] = g0;
          cell[4 * SPP] = g1;
        }
      }
      __syncthreads();
    }

    for (int idx = threadIdx.x; idx < kW * SP * SP; idx += blockDim.x) {
      const int pl = idx / (SP * SP), rem = idx - pl * (SP * SP);
      const int iu = rem / SP, iv = rem - iu * SP;
      const int u = u0 + iu, v = v0 + iv;
      const C val = sm_grid[pl * PL + iu * SPP + iv];
      if ((val.x != R(0) || val.y != R(0)) && u >= 0 && u < a.S && v >= 0 && v < a.S) {
        C* dst = &out[(p0 + pl) * SS + (int64_t)u * a.S + v];
        if constexpr (sizeof(R) == 4) {
          atomicAdd(reinterpret_cast<float2*>(dst), *reinterpret_cast<const float2*>(&val));
        } else {
          atomicAdd(&dst->x, val.x);
          atomicAdd(&dst->y, val.y);
        }
      }
    }
    __syncthreads();
  }
}

template <typename R, int T, int MODE>
int launch_tiles_ws(const Ctx* ctx, const TileArgs& a, cudaStream_t st) {
  using TG = WsGeom<T, MODE>;
  constexpr bool kUseModel = (MODE == kResid);
  const size_t sm = (size_t)(int(kUseModel) + 1) * kW * TG::PL * sizeof(cplx<R>) + kWsBatch * sizeof(WsRecord<R>);
  auto kern = k_tiles_ws<R, T, MODE>;
  RIX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm));
  per_sm = std::max(per_sm, 1);
  const int64_t blocks = std::min<int64_t>(a.item_count, (int64_t)ctx->num_sms * per_sm);
  if (blocks <= 0) return RIX_OK;
  timing_mark(kTimeTiles, st, true);
  ::rix::note_launch(); kern<<<(unsigned)blocks, 256, sm, st>>>(a);
  timing_mark(kTimeTiles, st, false);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

template <typename R, int MODE>
int launch_tiles(const Job* job, const TileArgs& a, cudaStream_t st) {
  const bool ws = job->nw > 0;
  if constexpr (std::is_same<R, float>::value && (MODE == kGrid || MODE == kResid)) {
    // FP32 w-stacked gridding on the image grid: register-resident
    // footprints (k_tiles_fp.cu)
    if (ws && job->tile == 16)
      return launch_tiles_fp(job, MODE, a.item_begin, a.item_count, a.ent_begin, a.ent_count, a.win_lo, a.S, a.model,
                             a.out, a.vis_in, st);
  }
  if constexpr (MODE != kDegrid) {
    // w-stacked gridding: plane-owned shared-memory sub-grid (tile 16 only)
    if (ws) return launch_tiles_ws<R, 16, MODE>(job->ctx, a, st);
  }
  if (job->tile == 16) {
    return ws ? launch_tiles_impl<R, kW, 16, MODE>(job->ctx, a, st) : launch_tiles_impl<R, 1, 16, MODE>(job->ctx, a, st);
  }
  return ws ? launch_tiles_impl<R, kW, 32, MODE>(job->ctx, a, st) : launch_tiles_impl<R, 1, 32, MODE>(job->ctx, a, st);
}

TileArgs base_args(const Job* job, const Part& pt) {
  TileArgs a{};
  a.keys = job->keys.as<uint32_t>();
  a.samples = job->gsamples.as<uint32_t>();   // gridder order, matching egeom
  a.items = job->items.as<uint32_t>();
  a.item_begin = pt.item_begin;
  a.item_count = pt.item_count;
  a.uvw = job->uvw.as<double>();
  a.inv_lambda = job->inv_lambda.as<double>();
  a.nchan = job->desc.nchan;
  a.scale = job->desc.cell_rad * (double)job->ng;
  a.half = 0.5 * job->ng;
  a.nw = job->nw;
  a.ww = job->ww;
  a.w_min = job->stats.w_min;
  a.dw = job->stats.dw;
  a.bt = job->bt;
  a.bw = job->bw;
  a.logT = ilog2(job->tile);
  a.win_lo = pt.win_lo;
  a.S = pt.win_n;
  a.weight = job->weight.as<float>();
  a.geom = job->egeom.p;
  a.geom_off = 0;
  a.ent_begin = pt.ent_begin;
  a.ent_count = pt.ent_count;
  a.status = job->status.as<int>();
  return a;
}

XformGeom plane_geom(const Job* job, const Part& pt, bool psf) {
  XformGeom g{};
  const int n = job->desc.n;
  g.M = psf ? 2 * n : n;
  g.L = psf ? 2 * job->ng : job->ng;
  g.logL = ilog2(g.L);
  g.lo = psf ? pt.pwin_lo : pt.win_lo;
  g.S = psf ? pt.pwin_n : pt.win_n;
  g.nplanes = job->nw > 0 ? job->nw : 1;
  g.mode = job->nw > 0 ? kFacPhase : kFacReal;
  g.corr = psf ? job->corr_psf.p : job->corr_img.p;
  g.nm1 = psf ? job->nm1_psf.as<double>() : job->nm1_img.as<double>();
  g.w0 = job->stats.w_min - 0.5 * job->ww * job->stats.dw;
  g.dw = job->stats.dw;
  // the image grid's factors are tabulated once per job (the PSF's grid is
  // transformed once per job: it forms them on the fly)
  if (!psf && g.mode == kFacPhase && job->screen_img.p) g.screen = job->screen_img.p;
  return g;
}

template <typename R>
int ensure_plane_buffers(Job* job, Part& pt) {
  const int np = job->nw > 0 ? job->nw : 1;
  const size_t plane = (size_t)pt.win_n * pt.win_n * sizeof(cplx<R>);
  if (pt.model_planes.bytes < np * plane) RIX_TRY(pt.model_planes.alloc(job->ctx, np * plane));
  if (pt.resid_planes.bytes < np * plane) RIX_TRY(pt.resid_planes.alloc(job->ctx, np * plane));
  const size_t tb = (size_t)np * pt.win_n * job->desc.n * sizeof(cplx<R>);
  if (pt.tbuf.bytes < tb) RIX_TRY(pt.tbuf.alloc(job->ctx, tb));
  return RIX_OK;
}

// image -> model planes of partition p
template <typename R>
int image_to_planes(Job* job, Part& pt, const R* image, cudaStream_t st) {
  RIX_TRY(ensure_plane_buffers<R>(job, pt));
  const XformGeom g = plane_geom(job, pt, false);
  RIX_TRY(fwd_rows<R>(job->ctx, g, image, pt.tbuf.as<cplx<R>>(), st));
  RIX_TRY(fwd_cols<R>(job->ctx, g, pt.tbuf.as<cplx<R>>(), pt.model_planes.as<cplx<R>>(), st));
  return RIX_OK;
}

// residual planes -> image (scaled by 1 / W_p); the plane-group images of the
// inverse row pass are the partition's own, allocated at the first call
template <typename R>
int planes_to_image(Job* job, Part& pt, R* image, cudaStream_t st) {
  const XformGeom g = plane_geom(job, pt, false);
  RIX_TRY(inv_cols<R>(job->ctx, g, pt.resid_planes.as<cplx<R>>(), kOpNone, nullptr, nullptr,
                      pt.tbuf.as<cplx<R>>(), st));
  const double sc = pt.wsum > 0.0 ? 1.0 / pt.wsum : 0.0;
  const int G = inv_rows_groups<R>(job->ctx, g, 16);
  if (G < 0) return G;
  const size_t gb = (size_t)G * g.M * g.M * sizeof(R);
  if (G > 1 && pt.groups.bytes < gb) RIX_TRY(pt.groups.alloc(job->ctx, gb));
  RIX_TRY(inv_rows<R>(job->ctx, g, pt.tbuf.as<cplx<R>>(), image, sc, 0, st, pt.groups.as<R>(), G));
  return RIX_OK;
}

}  // namespace

template <typename R>
int grid_build_corrections(Job* job, cudaStream_t st) {
  const int n = job->desc.n;
  job->stats.max_dw_nm1 = 0.0;
  RIX_TRY(build_correction<R>(job, n, job->ng, job->corr_img, job->nm1_img, st));
  RIX_TRY(build_correction<R>(job, 2 * n, 2 * job->ng, job->corr_psf, job->nm1_psf, st));
  if (job->nw > 0) {
    // corr x phase screen of every w-plane on the image grid: read by the
    // row passes of every major cycle instead of forming them in FP64
    XformGeom g = plane_geom(job, job->part[0], false);
    g.screen = nullptr;
    const size_t bytes = (size_t)g.nplanes * g.M * g.M * sizeof(cplx<R>);
    RIX_TRY(job->screen_img.alloc(job->ctx, bytes));
    RIX_TRY(build_screen_table<R>(job->ctx, g, job->screen_img.as<cplx<R>>(), st));
  }
  return RIX_OK;
}

template <typename R>
int op_degrid(Job* job, int p, const R* image, cplx<R>* vis_out, cudaStream_t st) {
  Part& pt = job->part[p];
  if (pt.ent_count == 0) return RIX_OK;
  RIX_TRY(image_to_planes<R>(job, pt, image, st));
  TileArgs a = base_args(job, pt);
  a.model = pt.model_planes.p;
  a.vis_out = vis_out;
  return launch_tiles<R, kDegrid>(job, a, st);
}

template <typename R>
int op_grid(Job* job, int p, const cplx<R>* vis, R* image_out, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  if (pt.ent_count == 0) {
    RIX_CUDA(cudaMemsetAsync(image_out, 0, (size_t)n * n * sizeof(R), st));
    return RIX_OK;
  }
  RIX_TRY(ensure_plane_buffers<R>(job, pt));
  const int np = job->nw > 0 ? job->nw : 1;
  RIX_CUDA(cudaMemsetAsync(pt.resid_planes.p, 0, (size_t)np * pt.win_n * pt.win_n * sizeof(cplx<R>), st));
  TileArgs a = base_args(job, pt);
  a.out = pt.resid_planes.p;
  a.vis_in = vis;
  RIX_TRY(launch_tiles<R, kGrid>(job, a, st));
  return planes_to_image<R>(job, pt, image_out, st);
}

template <typename R>
int op_major(Job* job, int p, const cplx<R>* vis, R* residual, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  if (pt.ent_count == 0) {
    RIX_CUDA(cudaMemsetAsync(residual, 0, (size_t)n * n * sizeof(R), st));
    return RIX_OK;
  }
  RIX_TRY(image_to_planes<R>(job, pt, pt.model.as<R>(), st));
  const int np = job->nw > 0 ? job->nw : 1;
  RIX_CUDA(cudaMemsetAsync(pt.resid_planes.p, 0, (size_t)np * pt.win_n * pt.win_n * sizeof(cplx<R>), st));
  TileArgs a = base_args(job, pt);
  a.model = pt.model_planes.p;
  a.out = pt.resid_planes.p;
  a.vis_in = vis;
  RIX_TRY(launch_tiles<R, kResid>(job, a, st));
  return planes_to_image<R>(job, pt, residual, st);
}

// pt.hspec = the centred spectrum of the 2N x 2N PSF on the 2N grid; `tt`
// ([2N][2N] complex) is the transpose buffer, a temporary when null
template <typename R>
int psf_spectrum(Job* job, Part& pt, cudaStream_t st, cplx<R>* tt = nullptr) {
  const int n = job->desc.n;
  const size_t img2 = (size_t)4 * n * n;
  cplx<R>* tmp = nullptr;
  if (!tt) {
    RIX_CUDA(::rix::malloc_async(&tmp, img2 * sizeof(cplx<R>), st));
    tt = tmp;
  }
  XformGeom h{};
  h.M = 2 * n; h.L = 2 * n; h.logL = ilog2(h.L); h.lo = 0; h.S = 2 * n; h.nplanes = 1; h.mode = kFacNone;
  int rc = fwd_rows<R>(job->ctx, h, pt.psf.as<R>(), tt, st);
  if (rc == RIX_OK) rc = fwd_cols<R>(job->ctx, h, tt, pt.hspec.as<cplx<R>>(), st);
  if (tmp) cudaFreeAsync(tmp, st);
  return rc;
}

// vis[s] = exp(2 pi i (u_s l0 + v_s m0)) for every sample s = row * nchan + ch
// (u, v in wavelengths, FP64 argument): unit visibilities with the phase
// centre moved to (l0, m0)
template <typename R>
__global__ void k_psf_phase(const double* __restrict__ uvw, const double* __restrict__ inv_lambda, int nchan,
                            int64_t ns, double l0, double m0, cplx<R>* __restrict__ vis) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / nchan;
    const int ch = (int)(i - row * nchan);
    const double sc = inv_lambda[ch];
    const double u = __dmul_rn(uvw[row * 3 + 0], sc), v = __dmul_rn(uvw[row * 3 + 1], sc);
    double sn, cs;
    sincospi(2.0 * __dadd_rn(__dmul_rn(u, l0), __dmul_rn(v, m0)), &sn, &cs);
    cplx<R> y;
    y.x = (R)cs;
    y.y = (R)sn;
    vis[i] = y;
  }
}

// The 2N x 2N PSF as four N x N tiles on the image grid (Ng = 2N), for jobs
// whose PSF grid (2 Ng) is longer than the transforms support.  By the shift
// theorem the tile whose centre sits (ox, oy) cells from the phase centre is
// the dirty image of the unit visibilities exp(2 pi i (u l0 + v m0)),
// (l0, m0) = (ox, oy) dl, with the image-domain factors (1/n, the w-screens
// and the w-correction) taken at the sky position of each pixel:
//   PSF(l0 + l', m0 + m') = Re sum_k w_k n^-1 exp(2 pi i (u_k (l0 + l')
//                           + v_k (m0 + m') + w_k (n - 1))) / W_p.
// The gridding kernel's correction is the image's own (it depends on l', m').
template <typename R>
int op_psf_tiled(Job* job, int p, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  const bool ws = job->nw > 0;
  const int64_t ns = job->stats.n_samples;
  const size_t npix = (size_t)n * n;
  RIX_TRY(ensure_plane_buffers<R>(job, pt));
  cplx<R>* vis = nullptr;
  R* tile = nullptr;
  R* corr = nullptr;
  double* nm1 = nullptr;
  int rc = RIX_OK;
  if (::rix::malloc_async(&vis, (size_t)std::max<int64_t>(ns, 1) * sizeof(cplx<R>), st) != cudaSuccess ||
      ::rix::malloc_async(&tile, npix * sizeof(R), st) != cudaSuccess ||
      (ws && (::rix::malloc_async(&corr, npix * sizeof(R), st) != cudaSuccess ||
              ::rix::malloc_async(&nm1, npix * sizeof(double), st) != cudaSuccess))) {
    cudaGetLastError();
    rc = set_error(RIX_ENOMEM, "PSF tiles");
  }
  const XformGeom g0 = plane_geom(job, pt, false);
  const int G = inv_rows_groups<R>(job->ctx, g0, 16);
  if (rc == RIX_OK && G < 0) rc = G;
  if (rc == RIX_OK && G > 1 && pt.groups.bytes < (size_t)G * npix * sizeof(R))
    rc = pt.groups.alloc(job->ctx, (size_t)G * npix * sizeof(R));
  const double sc = pt.wsum > 0.0 ? 1.0 / pt.wsum : 0.0;
  const int np = ws ? job->nw : 1;
  for (int t = 0; t < 4 && rc == RIX_OK; ++t) {
    const int tx = t & 1, ty = t >> 1;
    const int ox = tx * n - n / 2, oy = ty * n - n / 2;
    ::rix::note_launch();
    k_psf_phase<R><<<(int)std::min<int64_t>(ceil_div(std::max<int64_t>(ns, 1), 256), (int64_t)job->ctx->num_sms * 16),
                     256, 0, st>>>(job->uvw.as<double>(), job->inv_lambda.as<double>(), job->desc.nchan, ns,
                                   ox * job->desc.cell_rad, oy * job->desc.cell_rad, vis);
    if (cudaGetLastError() != cudaSuccess) { rc = set_error(RIX_ECUDA, "PSF phase launch"); break; }
    XformGeom g = g0;
    g.screen = nullptr;
    if (ws) {
      if ((rc = fill_correction<R>(job, n, job->ng, ox, oy, n, corr, nm1, st)) != RIX_OK) break;
      g.corr = corr;
      g.nm1 = nm1;
    }
    if (cudaMemsetAsync(pt.resid_planes.p, 0, (size_t)np * pt.win_n * pt.win_n * sizeof(cplx<R>), st) != cudaSuccess) {
      rc = set_error(RIX_ECUDA, "memset");
      break;
    }
    TileArgs a = base_args(job, pt);
    a.out = pt.resid_planes.p;
    a.vis_in = vis;
    if ((rc = launch_tiles<R, kGrid>(job, a, st)) != RIX_OK) break;
    if ((rc = inv_cols<R>(job->ctx, g, pt.resid_planes.as<cplx<R>>(), kOpNone, nullptr, nullptr,
                          pt.tbuf.as<cplx<R>>(), st)) != RIX_OK)
      break;
    if ((rc = inv_rows<R>(job->ctx, g, pt.tbuf.as<cplx<R>>(), tile, sc, 0, st, pt.groups.as<R>(), G)) != RIX_OK) break;
    if (cudaMemcpy2DAsync(pt.psf.as<R>() + (size_t)ty * n * 2 * n + (size_t)tx * n, 2 * n * sizeof(R), tile,
                          n * sizeof(R), n * sizeof(R), n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      rc = set_error(RIX_ECUDA, "PSF tile copy");
  }
  if (vis) cudaFreeAsync(vis, st);
  if (tile) cudaFreeAsync(tile, st);
  if (corr) cudaFreeAsync(corr, st);
  if (nm1) cudaFreeAsync(nm1, st);
  return rc;
}

// whether partition PSFs of this job are formed by op_psf_tiled
template <typename R>
bool psf_uses_tiles(const Job* job) {
  if (job->psf_method == RIX_PSF_TILES) return true;
  if (job->psf_method == RIX_PSF_DOUBLE_GRID) return false;
  return 2 * job->ng > fft_max_len<R>();
}

template <typename R>
int op_psf(Job* job, int p, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  const int np = job->nw > 0 ? job->nw : 1;
  const size_t img2 = (size_t)4 * n * n;
  if (pt.psf.bytes < img2 * sizeof(R)) RIX_TRY(pt.psf.alloc(job->ctx, img2 * sizeof(R)));
  if (pt.hspec.bytes < img2 * sizeof(cplx<R>)) RIX_TRY(pt.hspec.alloc(job->ctx, img2 * sizeof(cplx<R>)));
  if (pt.ent_count == 0) {
    RIX_CUDA(cudaMemsetAsync(pt.psf.p, 0, img2 * sizeof(R), st));
    RIX_CUDA(cudaMemsetAsync(pt.hspec.p, 0, img2 * sizeof(cplx<R>), st));
    pt.psf_ready = true;
    return RIX_OK;
  }
  if (psf_uses_tiles<R>(job)) {
    RIX_TRY(op_psf_tiled<R>(job, p, st));
    RIX_TRY(psf_spectrum<R>(job, pt, st));
    pt.psf_ready = true;
    return RIX_OK;
  }
  // temporary PSF planes and transpose buffer
  const size_t planes = (size_t)np * pt.pwin_n * pt.pwin_n;
  // also holds the [2N][2N] transpose of the PSF spectrum below
  const size_t tb = std::max((size_t)np * pt.pwin_n * 2 * n, (size_t)4 * n * n);
  cplx<R>* pp = nullptr;
  cplx<R>* tt = nullptr;
  EntryGeom<R>* pg = nullptr;
  RIX_CUDA(::rix::malloc_async(&pp, planes * sizeof(cplx<R>), st));
  if (::rix::malloc_async(&tt, tb * sizeof(cplx<R>), st) != cudaSuccess) {
    cudaFreeAsync(pp, st);
    return set_error(RIX_ENOMEM, "PSF transpose buffer");
  }
  int rc = RIX_OK;
  do {
    if (cudaMemsetAsync(pp, 0, planes * sizeof(cplx<R>), st) != cudaSuccess) { rc = set_error(RIX_ECUDA, "memset"); break; }
    TileArgs a = base_args(job, pt);
    a.scale = job->desc.cell_rad * (double)(2 * job->ng);
    a.half = (double)job->ng;
    a.win_lo = pt.pwin_lo;
    a.S = pt.pwin_n;
    a.out = pp;
    if (std::is_same<R, float>::value && job->nw > 0 && job->tile == 16) {
      // FP32 w-stacked: the register-resident gridder on 16 x 16 tiles of the
      // PSF grid (k_tiles_fp.cu)
      if ((rc = launch_psf_fp(job, p, a.scale, a.half, pp, st)) != RIX_OK) break;
    } else {
      // the partition's entries' geometry on the 2N grid, in FP64 (one thread
      // per entry), for the one PSF launch
      if (::rix::malloc_async(&pg, (size_t)pt.ent_count * sizeof(EntryGeom<R>), st) != cudaSuccess) {
        rc = set_error(RIX_ENOMEM, "PSF entry geometry");
        break;
      }
      {
        const int blocks = (int)std::min<int64_t>(ceil_div(pt.ent_count, 256), (int64_t)job->ctx->num_sms * 16);
        ::rix::note_launch();
        if (job->tile == 16) k_entry_geom<R, true, 16><<<blocks, 256, 0, st>>>(a, pt.ent_begin, pt.ent_count, pg);
        else k_entry_geom<R, true, 32><<<blocks, 256, 0, st>>>(a, pt.ent_begin, pt.ent_count, pg);
        RIX_LAUNCH_CHECK();
      }
      a.geom = pg;
      a.geom_off = pt.ent_begin;
      if ((rc = launch_tiles<R, kPsf>(job, a, st)) != RIX_OK) break;
    }
    const XformGeom g = plane_geom(job, pt, true);
    if ((rc = inv_cols<R>(job->ctx, g, pp, kOpNone, nullptr, nullptr, tt, st)) != RIX_OK) break;
    const double sc = pt.wsum > 0.0 ? 1.0 / pt.wsum : 0.0;
    if ((rc = inv_rows<R>(job->ctx, g, tt, pt.psf.as<R>(), sc, 0, st)) != RIX_OK) break;
    // centred spectrum of the 2N x 2N PSF on the 2N grid
    rc = psf_spectrum<R>(job, pt, st, tt);
  } while (0);
  cudaFreeAsync(pp, st);
  cudaFreeAsync(tt, st);
  if (pg) cudaFreeAsync(pg, st);
  if (rc == RIX_OK) pt.psf_ready = true;
  return rc;
}

// Gridding of partition p (as op_grid) with its w-planes, transpose buffer
// and the inverse row pass's plane-group images in caller-provided device
// scratch instead of the job's own buffers; FP32 jobs.  Allocates nothing.
// The plane groups take what the scratch has left after the planes and the
// transpose buffer (one group, no group images, when nothing is left).
// Returns RIX_EINVAL when the planes and transpose buffer do not fit.
int op_grid_into_scratch(Job* job, int p, const float2* vis, float* image_out, float2* scratch,
                         size_t scratch_elems, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  if (pt.ent_count == 0) {
    RIX_CUDA(cudaMemsetAsync(image_out, 0, (size_t)n * n * sizeof(float), st));
    return RIX_OK;
  }
  const size_t np = job->nw > 0 ? (size_t)job->nw : 1;
  const size_t plane_elems = np * pt.win_n * pt.win_n;
  const size_t t_elems = np * pt.win_n * n;
  if (plane_elems + t_elems > scratch_elems)
    return set_error(RIX_EINVAL, "partition %d needs %zu bytes of scratch, the fixed scratch holds %zu", p,
                     (plane_elems + t_elems) * sizeof(float2), scratch_elems * sizeof(float2));
  float2* planes = scratch;
  float2* tbuf = scratch + plane_elems;
  float* group_imgs = reinterpret_cast<float*>(scratch + plane_elems + t_elems);
  const size_t left_floats = 2 * (scratch_elems - plane_elems - t_elems);
  const int max_groups = (int)std::min<size_t>(16, left_floats / ((size_t)n * n));
  RIX_CUDA(cudaMemsetAsync(planes, 0, plane_elems * sizeof(float2), st));   // the sub-grids accumulate
  TileArgs a = base_args(job, pt);
  a.out = planes;
  a.vis_in = vis;
  RIX_TRY(launch_tiles<float, kGrid>(job, a, st));
  const XformGeom g = plane_geom(job, pt, false);
  RIX_TRY(inv_cols<float>(job->ctx, g, planes, kOpNone, nullptr, nullptr, tbuf, st));
  const double sc = pt.wsum > 0.0 ? 1.0 / pt.wsum : 0.0;
  return inv_rows<float>(job->ctx, g, tbuf, image_out, sc, 0, st, group_imgs, std::max(max_groups, 1));
}

int ensure_planes_f32(Job* job, int p) { return ensure_plane_buffers<float>(job, job->part[p]); }

// The major cycles of the batch's pairs (each as op_major) with one gridder
// launch: the caller's stream forks to the batch's streams for every pair's
// model -> planes transform, residual-plane clearing and visibility gather,
// joins for the gridder, and forks again for the planes -> residual
// transforms.
int op_major_batch(Batch* b, const float2* const* vis, cudaStream_t st) {
  const int ns = Batch::kStreams;
  auto fork = [&]() -> int {
    RIX_CUDA(cudaEventRecord(b->ev_fork, st));
    for (int k = 0; k < ns; ++k) RIX_CUDA(cudaStreamWaitEvent(b->streams[k], b->ev_fork, 0));
    return RIX_OK;
  };
  auto join = [&]() -> int {
    for (int k = 0; k < ns; ++k) {
      RIX_CUDA(cudaEventRecord(b->ev_join[k], b->streams[k]));
      RIX_CUDA(cudaStreamWaitEvent(st, b->ev_join[k], 0));
    }
    return RIX_OK;
  };
  RIX_TRY(fork());
  for (int i = 0; i < b->n; ++i) {
    Job* job = b->jobs[i];
    Part& pt = job->part[b->parts[i]];
    cudaStream_t s = b->streams[i % ns];
    if (pt.ent_count == 0) {
      RIX_CUDA(cudaMemsetAsync(pt.resid.p, 0, (size_t)job->desc.n * job->desc.n * sizeof(float), s));
      continue;
    }
    RIX_TRY(image_to_planes<float>(job, pt, pt.model.as<float>(), s));
    const size_t np = (size_t)job->nw;
    RIX_CUDA(cudaMemsetAsync(pt.resid_planes.p, 0, np * pt.win_n * pt.win_n * sizeof(float2), s));
    RIX_TRY(gather_y(job, pt.ent_begin, pt.ent_count, vis[i], s));
  }
  RIX_TRY(join());
  RIX_TRY(batch_gridder(b, st));
  RIX_TRY(fork());
  for (int i = 0; i < b->n; ++i) {
    Job* job = b->jobs[i];
    Part& pt = job->part[b->parts[i]];
    if (pt.ent_count > 0) RIX_TRY(planes_to_image<float>(job, pt, pt.resid.as<float>(), b->streams[i % ns]));
  }
  return join();
}

template <typename R>
int grid_entry_geometry(Job* job, cudaStream_t st) {
  const int64_t n = job->n_entries;
  RIX_TRY(job->egeom.alloc(job->ctx, (size_t)std::max<int64_t>(n, 1) * sizeof(EntryGeom<R>)));
  if (n == 0) return RIX_OK;
  TileArgs a = base_args(job, job->part[0]);   // job-level fields only
  a.samples = job->samples.as<uint32_t>();      // the sorted order (grid_work_order reorders both after)
  job->gorder = false;
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)job->ctx->num_sms * 16);
  ::rix::note_launch();
  if (job->tile == 16) k_entry_geom<R, false, 16><<<blocks, 256, 0, st>>>(a, 0, n, job->egeom.as<EntryGeom<R>>());
  else k_entry_geom<R, false, 32><<<blocks, 256, 0, st>>>(a, 0, n, job->egeom.as<EntryGeom<R>>());
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

#define RIX_GRID_INST(R)                                                               \
  template int grid_build_corrections<R>(Job*, cudaStream_t);                          \
  template int grid_entry_geometry<R>(Job*, cudaStream_t);                             \
  template int op_degrid<R>(Job*, int, const R*, cplx<R>*, cudaStream_t);              \
  template int op_grid<R>(Job*, int, const cplx<R>*, R*, cudaStream_t);                \
  template int op_major<R>(Job*, int, const cplx<R>*, R*, cudaStream_t);               \
  template int op_psf<R>(Job*, int, cudaStream_t);
RIX_GRID_INST(float)
RIX_GRID_INST(double)

}  // namespace rix
