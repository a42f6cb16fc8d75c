// a8-a11: the fill of each partition's missing spatial frequencies from the
// other partitions' previous-cycle images (Sec. 3-4, Eq. 5 and 7), the
// minor cycles (FISTA with a Db4 dictionary, Eq. 4-5; multi-scale CLEAN,
// Eq. 6-7), the image update (Eq. 3) and the equal-weight combine (Sec. 5.2).
//
// All image-domain operators are applied on the 2N-padded grid through the
// transforms of k_fft.cu; spectra are centred and stored u-major, (2N)^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rix_internal.cuh"
#include "fft_device.cuh"
#include "wavelet_device.cuh"
#include "grid_sync.cuh"

namespace rix {
namespace {

// ------------------------------------------------------------ transforms ----
XformGeom fill_geom(int n) {
  XformGeom g{};
  g.M = n; g.L = 2 * n; g.logL = ilog2(g.L); g.lo = 0; g.S = 2 * n; g.nplanes = 1; g.mode = kFacNone;
  return g;
}

// centred spectrum of the 2N-padded image x
template <typename R>
int img_spectrum(Job* job, Part& pt, const R* x, cplx<R>* spec, cudaStream_t st) {
  const XformGeom g = fill_geom(job->desc.n);
  RIX_TRY(fwd_rows<R>(job->ctx, g, x, pt.ft_a.as<cplx<R>>(), st));
  return fwd_cols<R>(job->ctx, g, pt.ft_a.as<cplx<R>>(), spec, st);
}

// out (+)= scale * crop F^-1 [op(spec)]
template <typename R>
int spec_to_img(Job* job, Part& pt, const cplx<R>* spec, int op, const void* tab, R* out, double scale,
                int accumulate, cudaStream_t st) {
  const XformGeom g = fill_geom(job->desc.n);
  RIX_TRY(inv_cols<R>(job->ctx, g, spec, op, tab, nullptr, pt.ft_a.as<cplx<R>>(), st));
  return inv_rows<R>(job->ctx, g, pt.ft_a.as<cplx<R>>(), out, scale, accumulate, st);
}

// out (+)= scale * crop F^-1 [op(F pad x)]   (three passes; the spectral op is
// fused between the forward and inverse column transforms)
// The image and the result are real and every spectral operator used here
// preserves Hermitian symmetry, so only the columns k_u in [-N, 0] of the
// spectrum are formed and transformed; the inverse row pass completes the
// others by conjugation.
template <typename R>
int convolve(Job* job, Part& pt, const R* x, int op, const void* tab, const void* tab2, R* out, double scale,
             int accumulate, cudaStream_t st) {
  XformGeom g = fill_geom(job->desc.n);
  g.S = job->desc.n + 1;
  g.herm = 1;
  RIX_TRY(fwd_rows<R>(job->ctx, g, x, pt.ft_a.as<cplx<R>>(), st));
  RIX_TRY(conv_cols<R>(job->ctx, g, pt.ft_a.as<cplx<R>>(), op, tab, tab2, pt.ft_b.as<cplx<R>>(), st));
  return inv_rows<R>(job->ctx, g, pt.ft_b.as<cplx<R>>(), out, scale, accumulate, st);
}

// ---------------------------------------------------------------- kernels ----
int blocks_for(const Ctx* ctx, int64_t n, int threads = 256) {
  return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads), (int64_t)ctx->num_sms * 8);
}

// Gamma_p = Lambda_{p+1} - Lambda_p, Lambda_i(r) = clip((ell_i + delta - r) / (2 delta), 0, 1),
// r = |k| / 2 on the centred 2N grid (u-major index [ju][jv]).
struct GammaArgs {
  int n, nparts;
  double ells[kMaxPart];
  double delta;
};

__device__ __forceinline__ double ramp(double ell, double delta, double r) {
  if (delta <= 0.0) return r < ell ? 1.0 : (r > ell ? 0.0 : 0.5);
  return fmin(fmax((ell + delta - r) / (2.0 * delta), 0.0), 1.0);
}

template <typename R>
__global__ void k_gamma(GammaArgs a, R* __restrict__ gam) {
  const int L = 2 * a.n;
  const int64_t tot = (int64_t)L * L;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int ju = (int)(i / L), jv = (int)(i - (int64_t)ju * L);
    const double ku = ju - a.n, kv = jv - a.n;
    const double r = sqrt(ku * ku + kv * kv) / 2.0;
    double lam_lo = 0.0;
    for (int p = 0; p < a.nparts; ++p) {
      const double lam_hi = (p == a.nparts - 1) ? 1.0 : ramp(a.ells[p], a.delta, r);
      gam[(int64_t)p * tot + i] = (R)(lam_hi - lam_lo);
      lam_lo = lam_hi;
    }
  }
}

// rho += phi - ibar
template <typename R>
__global__ void k_rho_sub(R* __restrict__ rho, const R* __restrict__ phi, const R* __restrict__ ibar, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] += phi[i] - ibar[i];
}

template <typename R>
__global__ void k_axpy(R* __restrict__ y, const R* __restrict__ x, R alpha, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += alpha * x[i];
}

// ---- band-limited exchange (Sec. 6.3, Sec. 7 item a) ----------------------
// flags of the half plane ju <= N (k_u <= 0) of a partition's ring support,
// Gamma_p > 0 (flat u-major index ju * 2N + jv)
template <typename R>
__global__ void k_ring_flags(const R* __restrict__ gam_p, int64_t nhalf, uint32_t* __restrict__ flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nhalf; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = gam_p[i] > R(0) ? 1u : 0u;
}
__global__ void k_ring_index(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos, int64_t nhalf,
                             uint32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nhalf; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) idx[pos[i]] = (uint32_t)i;
}
// the exchanged coefficients Gamma_p X at the support
template <typename R>
__global__ void k_phi_pack(const R* __restrict__ gam_p, const cplx<R>* __restrict__ spec,
                           const uint32_t* __restrict__ idx, int64_t count, cplx<R>* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = idx[i];
    const R g = gam_p[j];
    const cplx<R> x = spec[j];
    out[i] = cmake<cplx<R>>(g * x.x, g * x.y);
  }
}
// the spectrum rebuilt from the coefficients (zeroed by the caller) and
// their conjugate mirrors k -> -k (index j -> 2N - j mod 2N) off the
// self-mirrored columns ju = 0 and ju = N
template <typename R>
__global__ void k_phi_unpack(const cplx<R>* __restrict__ coef, const uint32_t* __restrict__ idx, int64_t count,
                             int n, cplx<R>* __restrict__ spec) {
  const int n2 = 2 * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = idx[i];
    const int ju = (int)(j / (uint32_t)n2), jv = (int)(j - (uint32_t)ju * n2);
    const cplx<R> c = coef[i];
    spec[j] = c;
    if (ju > 0 && ju < n) spec[(int64_t)((n2 - ju) % n2) * n2 + (n2 - jv) % n2] = cmake<cplx<R>>(c.x, -c.y);
  }
}

template <typename R>
__global__ void k_mean(R* __restrict__ out, const R* const* __restrict__ imgs, int nimg, int64_t n) {
  const R inv = R(1) / (R)nimg;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R s = R(0);
    for (int k = 0; k < nimg; ++k) s += imgs[k][i];
    out[i] = s * inv;
  }
}

// max |x| into *out (out pre-set to 0); values are >= 0 so the bit pattern
// order of the IEEE encoding matches the value order
__device__ __forceinline__ void atomic_max_nonneg(float* out, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* out, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(v));
}

template <typename R>
__global__ void k_absmax(const R* __restrict__ x, int64_t n, R* __restrict__ out) {
  R m = R(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// out += sum of x^2 (per warp, then atomically)
template <typename R>
__global__ void k_sumsq(const R* __restrict__ x, int64_t n, R* __restrict__ out) {
  R a = R(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += x[i] * x[i];
  for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, a);
}

// ------------------------------------------------------------ fill kernels ----
// ms-CLEAN composite dirty spectrum and PSF spectrum (Eq. 7):
//   D = g Gam_p I_p + sum_q mu_q H_q Rho_q,   P = g Gam_p H_p + sum_q mu_q Gam_q H_q
struct FillArgs {
  int64_t tot;
  int p, nparts;
  double g, mu[kMaxPart];
  const void* gam;                 // R [P][tot]
  const void* h[kMaxPart];         // cplx [tot]
  const void* rho[kMaxPart];       // cplx [tot] (spectra), null for q == p
  const void* ispec;               // cplx [tot]
};

template <typename R>
__global__ void k_fill_msclean(FillArgs a, cplx<R>* __restrict__ dspec, cplx<R>* __restrict__ pspec) {
  using C = cplx<R>;
  const R* gam = static_cast<const R*>(a.gam);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.tot; i += (int64_t)gridDim.x * blockDim.x) {
    const R gp = gam[(int64_t)a.p * a.tot + i] * (R)a.g;
    const C hp = static_cast<const C*>(a.h[a.p])[i];
    C d = static_cast<const C*>(a.ispec)[i] * gp;
    C ps = hp * gp;
    for (int q = 0; q < a.nparts; ++q) {
      if (q == a.p || a.mu[q] == 0.0) continue;
      const C hq = static_cast<const C*>(a.h[q])[i];
      const C rq = static_cast<const C*>(a.rho[q])[i];
      d = d + cmul(hq, rq) * (R)a.mu[q];
      ps = ps + hq * (gam[(int64_t)q * a.tot + i] * (R)a.mu[q]);
    }
    dspec[i] = d;
    pspec[i] = ps;
  }
}

// FISTA quadratic form (Eq. 5): Mx = Gam_p^2 |H_p|^2 + gn sum_q Gam_q^2,
// C = Gam_p^2 conj(H_p) I_p + gn sum_q Gam_q Rho_q; also max(Mx) for L.
template <typename R>
__global__ void k_fill_fista(FillArgs a, double gn, R* __restrict__ mx, cplx<R>* __restrict__ c,
                             R* __restrict__ mxmax) {
  using C = cplx<R>;
  const R* gam = static_cast<const R*>(a.gam);
  R m = R(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.tot; i += (int64_t)gridDim.x * blockDim.x) {
    const R gp = gam[(int64_t)a.p * a.tot + i];
    const R g2 = gp * gp;
    const C hp = static_cast<const C*>(a.h[a.p])[i];
    const C ip = static_cast<const C*>(a.ispec)[i];
    R mv = g2 * (hp.x * hp.x + hp.y * hp.y);
    C cv = cmulc(ip, hp) * g2;
    for (int q = 0; q < a.nparts; ++q) {
      if (q == a.p) continue;
      const R gq = gam[(int64_t)q * a.tot + i];
      mv += (R)gn * gq * gq;
      cv = cv + static_cast<const C*>(a.rho[q])[i] * ((R)gn * gq);
    }
    mx[i] = mv;
    c[i] = cv;
    m = fmax(m, mv);
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(mxmax, m);
}

}  // namespace

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_idwt_level(const R* __restrict__ llin, const R* __restrict__ coef, int n,
                                                    R* __restrict__ out, int ld) {
  __shared__ IdwtSmem<R, 8> sm;
  idwt_tile<R>(llin, coef, n, out, ld, blockIdx.x, blockIdx.y, sm, Db4Taps<R>{});
}

// coefficients c (N x N) -> image out; tmp: N x N scratch.  Levels are
// synthesised coarsest first, alternating out / tmp so the finest lands in out.
template <typename R>
int idwt2(const Ctx* ctx, const R* c, R* out, R* tmp, int N, int levels, cudaStream_t s) {
  const R* ll = c;
  for (int l = levels - 1; l >= 0; --l) {
    const int n = N >> l;
    R* dst = ((l & 1) == 0) ? out : tmp;
    dim3 grid((unsigned)ceil_div(n, kTS), (unsigned)ceil_div(n, kTS));
    note_launch();
    k_idwt_level<R><<<grid, 256, 0, s>>>(ll, c, n, dst, N);
    ll = dst;
  }
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

}  // namespace

namespace {

// --------------------------------------------------------------- ms-CLEAN ----
template <typename R>
struct Cand {
  R val;       // b_s |R_s(p)| / P_ss(0); -1 = none
  R rval;      // R_s(p), signed
  int s, pix;
  R r0max;     // max |R_0| over the image
};

template <typename R>
__device__ __forceinline__ bool better(const Cand<R>& a, const Cand<R>& b) {
  if (a.val != b.val) return a.val > b.val;
  if (a.s != b.s) return a.s < b.s;
  return a.pix < b.pix;
}

template <typename R>
__device__ __forceinline__ Cand<R> shfl_cand(const Cand<R>& c, int o) {
  Cand<R> r;
  r.val = __shfl_xor_sync(0xffffffffu, c.val, o);
  r.rval = __shfl_xor_sync(0xffffffffu, c.rval, o);
  r.s = __shfl_xor_sync(0xffffffffu, c.s, o);
  r.pix = __shfl_xor_sync(0xffffffffu, c.pix, o);
  r.r0max = __shfl_xor_sync(0xffffffffu, c.r0max, o);
  return r;
}

template <typename R>
__device__ __forceinline__ Cand<R> merge(const Cand<R>& a, const Cand<R>& b) {
  Cand<R> r = better(b, a) ? b : a;
  r.r0max = fmax(a.r0max, b.r0max);
  return r;
}

// block-wide reduction; the result is valid in every thread
template <typename R>
__device__ Cand<R> block_reduce(Cand<R> c, Cand<R>* sh) {
  for (int o = 16; o; o >>= 1) c = merge(c, shfl_cand(c, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = c;
  __syncthreads();
  if (warp == 0) {
    Cand<R> d = lane < nw ? sh[lane] : Cand<R>{R(-1), R(0), 0x7fffffff, 0x7fffffff, R(0)};
    for (int o = 16; o; o >>= 1) d = merge(d, shfl_cand(d, o));
    if (lane == 0) sh[0] = d;
  }
  __syncthreads();
  return sh[0];
}

struct CleanArgs {
  int n, ns, niter;
  double gain, threshold;
  double bias[kMaxScales];
  int allowed;                 // bit mask of scales usable this cycle
  void* R;                     // [ns][n][n]
  const void* P;               // [ns][ns][2n][2n]
  void* model;                 // [n][n]
  const void* stencil;         // concatenated (2r+1)^2 stencils of B_s
  int st_off[kMaxScales], st_rad[kMaxScales];
  void* slots;                 // Cand<R> [2][gridDim]
  int* comp_s;                 // [niter]
  int* comp_pix;
  double* comp_amp;
  int* count;
  unsigned int* barrier;       // arrival counter, zeroed before the launch
  int* status;                 // the job's status word
};

// The whole minor cycle in one cooperative launch: each iteration subtracts
// the previous component from every scale residual and, in the same sweep,
// finds the next peak; one bounded grid barrier per iteration separates the
// sweep from the global reduction (double-buffered candidate slots).  A
// barrier that gives up (RIX_ETIMEOUT in the status word) ends every CTA.
// NS = the number of scales, fixed at compile time so that a sweep issues
// the loads of every scale of a pixel together.
template <typename R, int NS>
__global__ void __launch_bounds__(256) k_msclean(CleanArgs a) {
  GridBarrier bar{a.barrier, a.status, 0u};
  __shared__ Cand<R> sh[32];
  const int n = a.n, n2 = 2 * a.n;
  const int64_t npix = (int64_t)n * n;
  R* __restrict__ Rs = static_cast<R*>(a.R);
  const R* __restrict__ P = static_cast<const R*>(a.P);
  Cand<R>* slots = static_cast<Cand<R>*>(a.slots);
  __shared__ R peak[kMaxScales], scl[kMaxScales];
  if (threadIdx.x < NS) {
    const int s = threadIdx.x;
    peak[s] = P[((int64_t)(s * NS + s) * n2 + n) * n2 + n];
    // the candidate value b_s |R_s| / P_ss(0) as |R_s| times b_s / P_ss(0)
    // (a scale whose peak is 0 never wins: 0; the loop stops if it is chosen)
    scl[s] = peak[s] != R(0) ? (R)a.bias[s] / peak[s] : R(0);
  }
  __syncthreads();
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int logn = 31 - __clz(n);   // n is a power of two
  const int64_t n2sq = (int64_t)n2 * n2;

  // sweep with the subtraction of component (sc, py, px, amp) (amp = 0: none)
  auto sweep = [&](int sc, int py, int px, R amp) {
    Cand<R> c{R(-1), R(0), 0x7fffffff, 0x7fffffff, R(0)};
    const R* __restrict__ psc = P + (int64_t)sc * n2sq;   // P_{s, sc} = psc + s NS (2n)^2
    for (int64_t i = gtid; i < npix; i += gstride) {
      const int y = (int)(i >> logn), x = (int)(i & (n - 1));
      // P_{s,sc}(y - py, x - px) on the centred 2n grid
      const int64_t pp = (int64_t)(n + y - py) * n2 + (n + x - px);
      R v[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) v[s] = Rs[s * npix + i];
      if (amp != R(0)) {
        R q[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) q[s] = psc[(int64_t)s * NS * n2sq + pp];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          v[s] -= amp * q[s];
          Rs[s * npix + i] = v[s];
        }
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const R av = fabs(v[s]);
        if (s == 0) c.r0max = fmax(c.r0max, av);
        if ((a.allowed >> s) & 1) {
          const R val = av * scl[s];
          if (val > c.val || (val == c.val && (s < c.s || (s == c.s && (int)i < c.pix)))) {
            c.val = val;
            c.rval = v[s];
            c.s = s;
            c.pix = (int)i;
          }
        }
      }
    }
    return block_reduce(c, sh);
  };

  Cand<R> loc = sweep(0, 0, 0, R(0));
  if (threadIdx.x == 0) slots[blockIdx.x] = loc;
  int it = 0;
  for (;; ++it) {
    if (!grid_barrier(bar)) return;
    const Cand<R>* cur = slots + (int64_t)(it & 1) * gridDim.x;
    Cand<R> c{R(-1), R(0), 0x7fffffff, 0x7fffffff, R(0)};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) c = merge(c, cur[b]);
    const Cand<R> best = block_reduce(c, sh);
    if (it >= a.niter || best.r0max < (R)a.threshold || best.val < R(0) || peak[best.s] == R(0)) break;
    const R amp = (R)a.gain * best.rval / peak[best.s];
    const int py = best.pix / n, px = best.pix - py * n;
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) {
        a.comp_s[it] = best.s;
        a.comp_pix[it] = best.pix;
        a.comp_amp[it] = (double)amp;
      }
      // model += amp * B_s(. - p*), clipped to the image
      const int rad = a.st_rad[best.s], w = 2 * rad + 1;
      const R* stn = static_cast<const R*>(a.stencil) + a.st_off[best.s];
      R* model = static_cast<R*>(a.model);
      for (int k = threadIdx.x; k < w * w; k += blockDim.x) {
        const int dy = k / w - rad, dx = k % w - rad;
        const int yy = py + dy, xx = px + dx;
        if (yy >= 0 && yy < n && xx >= 0 && xx < n) model[(int64_t)yy * n + xx] += amp * stn[k];
      }
    }
    loc = sweep(best.s, py, px, amp);
    if (threadIdx.x == 0) slots[(int64_t)((it + 1) & 1) * gridDim.x + blockIdx.x] = loc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count = it;
}

// elementwise product of two complex spectra times a third: out = a * b * c
template <typename R>
__global__ void k_cmul3(const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y, const cplx<R>* __restrict__ z,
                        cplx<R>* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cmul(cmul(x[i], y[i]), z[i]);
}

}  // namespace

// ================================================================== host ====
namespace {

template <typename R>
int alloc_zero(Job* job, DevBuf& b, size_t bytes, cudaStream_t st) {
  if (b.bytes < bytes) RIX_TRY(b.alloc(job->ctx, bytes));
  RIX_CUDA(cudaMemsetAsync(b.p, 0, bytes, st));
  return RIX_OK;
}

template <typename R>
int ensure(Job* job, DevBuf& b, size_t bytes) {
  if (b.bytes < bytes) RIX_TRY(b.alloc(job->ctx, bytes));
  return RIX_OK;
}

// Phi_p from its exchanged coefficients: out (+)= scale * crop F^-1[spectrum]
// with the spectrum rebuilt in `spec` ((2N)^2) and `T` as the transpose
// buffer ([2N][N] complex)
template <typename R>
int phi_from_coef(Job* job, int p, const cplx<R>* coef, cplx<R>* spec, cplx<R>* T, R* out, double scale,
                  int accumulate, cudaStream_t st) {
  const int n = job->desc.n;
  const int64_t tot = (int64_t)4 * n * n;
  const Part& pt = job->part[p];
  RIX_CUDA(cudaMemsetAsync(spec, 0, tot * sizeof(cplx<R>), st));
  ::rix::note_launch();
  k_phi_unpack<R><<<blocks_for(job->ctx, pt.ring_count), 256, 0, st>>>(coef, pt.ring_idx.as<uint32_t>(),
                                                                       pt.ring_count, n, spec);
  RIX_LAUNCH_CHECK();
  const XformGeom g = fill_geom(n);
  RIX_TRY(inv_cols<R>(job->ctx, g, spec, kOpNone, nullptr, nullptr, T, st));
  return inv_rows<R>(job->ctx, g, T, out, scale, accumulate, st);
}

// rho_{q->p} += Phi_q^{n-1} for every other partition (cycle n >= 2); with
// the spectral exchange Phi_q arrives as its ring-support coefficients
template <typename R>
int ingest(Job* job, int p, int cycle, cudaStream_t st) {
  if (cycle < 2) return RIX_OK;
  const int64_t npix = (int64_t)job->desc.n * job->desc.n;
  if (job->desc.exchange == RIX_EXCHANGE_SPECTRAL) {
    Part& pt = job->part[p];
    const double inv = 1.0 / (double)(4 * npix);
    for (int q = 0; q < job->n_part; ++q)
      if (q != p)
        RIX_TRY(phi_from_coef<R>(job, q, job->part[q].outbox[(cycle - 1) & 1].as<cplx<R>>(), pt.fs_a.as<cplx<R>>(),
                                 pt.ft_a.as<cplx<R>>(), pt.rho[q].as<R>(), inv, 1, st));
    return RIX_OK;
  }
  for (int q = 0; q < job->n_part; ++q) {
    if (q == p) continue;
    ::rix::note_launch(); k_axpy<R><<<blocks_for(job->ctx, npix), 256, 0, st>>>(job->part[p].rho[q].as<R>(),
                                                          job->part[q].outbox[(cycle - 1) & 1].as<R>(), R(1), npix);
  }
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

// spectra of the own residual (slot p) and of the aggregates rho_{q->p}
template <typename R>
int fill_spectra(Job* job, int p, cudaStream_t st) {
  Part& pt = job->part[p];
  const int64_t tot = (int64_t)4 * job->desc.n * job->desc.n;
  cplx<R>* sp = pt.fspec.as<cplx<R>>();
  RIX_TRY(img_spectrum<R>(job, pt, pt.resid.as<R>(), sp + p * tot, st));
  for (int q = 0; q < job->n_part; ++q)
    if (q != p) RIX_TRY(img_spectrum<R>(job, pt, pt.rho[q].as<R>(), sp + q * tot, st));
  return RIX_OK;
}

template <typename R>
FillArgs fill_args(Job* job, int p) {
  FillArgs a{};
  const int64_t tot = (int64_t)4 * job->desc.n * job->desc.n;
  a.tot = tot;
  a.p = p;
  a.nparts = job->n_part;
  a.gam = job->gam.p;
  for (int q = 0; q < job->n_part; ++q) {
    a.h[q] = job->part[q].hspec.p;
    a.rho[q] = (q == p) ? nullptr : job->part[p].fspec.as<cplx<R>>() + q * tot;
  }
  a.ispec = job->part[p].fspec.as<cplx<R>>() + p * tot;
  return a;
}

// Eq. 3 and the exchange: model += i_bar; Phi_p = Gamma_p i_bar (outbox of
// this cycle's parity); rho_{q->p} -= Gamma_q i_bar.
template <typename R>
int publish(Job* job, int p, int cycle, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  const int64_t npix = (int64_t)n * n, tot = 4 * npix;
  const double inv = 1.0 / (double)tot;
  const R* ibar = pt.delta.as<R>();
  ::rix::note_launch(); k_axpy<R><<<blocks_for(job->ctx, npix), 256, 0, st>>>(pt.model.as<R>(), ibar, R(1), npix);
  RIX_LAUNCH_CHECK();
  const R* gam = job->gam.as<R>();
  if (job->desc.exchange == RIX_EXCHANGE_SPECTRAL) {
    // the message is Gamma_p F pad i_bar on the ring support (half plane)
    RIX_TRY(img_spectrum<R>(job, pt, ibar, pt.fs_a.as<cplx<R>>(), st));
    ::rix::note_launch();
    k_phi_pack<R><<<blocks_for(job->ctx, pt.ring_count), 256, 0, st>>>(gam + p * tot, pt.fs_a.as<cplx<R>>(),
                                                                       pt.ring_idx.as<uint32_t>(), pt.ring_count,
                                                                       pt.outbox[cycle & 1].as<cplx<R>>());
    RIX_LAUNCH_CHECK();
  } else {
    RIX_TRY(convolve<R>(job, pt, ibar, kOpMulReal, gam + p * tot, nullptr, pt.outbox[cycle & 1].as<R>(), inv, 0, st));
    if (job->n_part == 2) {
      // Gamma_q = 1 - Gamma_p and crop F^-1 F pad = identity, so
      // Gamma_q i_bar = i_bar - Phi_p: rho_{q->p} += Phi_p - i_bar
      const int q = 1 - p;
      ::rix::note_launch();
      k_rho_sub<R><<<blocks_for(job->ctx, npix), 256, 0, st>>>(pt.rho[q].as<R>(), pt.outbox[cycle & 1].as<R>(), ibar,
                                                               npix);
      RIX_LAUNCH_CHECK();
      return RIX_OK;
    }
  }
  for (int q = 0; q < job->n_part; ++q)
    if (q != p) RIX_TRY(convolve<R>(job, pt, ibar, kOpMulReal, gam + q * tot, nullptr, pt.rho[q].as<R>(), -inv, 1, st));
  return RIX_OK;
}

// B_s: 1 - (r/s)^2 for r < s pixels, unit sum; B_0 = delta.  Stencil of
// (2 rad + 1)^2 values, rad = ceil(s) - 1 (0 for s = 0).
void scale_stencil(double s, std::vector<double>& st, int& rad) {
  if (s <= 0.0) {
    rad = 0;
    st.assign(1, 1.0);
    return;
  }
  rad = (int)std::ceil(s) - 1;
  const int w = 2 * rad + 1;
  st.assign((size_t)w * w, 0.0);
  double sum = 0.0;
  for (int dy = -rad; dy <= rad; ++dy)
    for (int dx = -rad; dx <= rad; ++dx) {
      const double r2 = (double)(dx * dx + dy * dy);
      const double v = r2 < s * s ? 1.0 - r2 / (s * s) : 0.0;
      st[(size_t)(dy + rad) * w + (dx + rad)] = v;
      sum += v;
    }
  for (double& v : st) v /= sum;
}

template <typename R>
__global__ void k_place_stencil(const R* __restrict__ stn, int rad, R* __restrict__ img, int n2) {
  const int w = 2 * rad + 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < w * w; k += gridDim.x * blockDim.x) {
    const int dy = k / w - rad, dx = k % w - rad;
    img[(int64_t)(n2 / 2 + dy) * n2 + (n2 / 2 + dx)] = stn[k];
  }
}

}  // namespace

template <typename R>
int fill_init(Job* job, cudaStream_t st) {
  const int n = job->desc.n, P = job->n_part;
  const int64_t npix = (int64_t)n * n, tot = 4 * npix;
  RIX_TRY(ensure<R>(job, job->gam, (size_t)P * tot * sizeof(R)));
  GammaArgs ga{};
  ga.n = n;
  ga.nparts = P;
  for (int i = 0; i < P - 1; ++i) ga.ells[i] = job->ells[i];
  ga.delta = job->stats.delta_px;
  ::rix::note_launch(); k_gamma<R><<<blocks_for(job->ctx, tot), 256, 0, st>>>(ga, job->gam.as<R>());
  RIX_LAUNCH_CHECK();
  // ring support of every partition's filter on the half plane ju <= N
  {
    const int64_t nhalf = (int64_t)(n + 1) * 2 * n;
    uint32_t *flags = nullptr, *pos = nullptr, *total = nullptr;
    int rc = RIX_OK;
    if (malloc_async(&flags, nhalf * sizeof(uint32_t), st) != cudaSuccess ||
        malloc_async(&pos, nhalf * sizeof(uint32_t), st) != cudaSuccess ||
        malloc_async(&total, sizeof(uint32_t), st) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(RIX_ENOMEM, "ring support scratch");
    }
    for (int p = 0; p < P && rc == RIX_OK; ++p) {
      Part& pt = job->part[p];
      ::rix::note_launch();
      k_ring_flags<R><<<blocks_for(job->ctx, nhalf), 256, 0, st>>>(job->gam.as<R>() + p * tot, nhalf, flags);
      if ((rc = scan_exclusive_u32(flags, pos, nhalf, total, st)) != RIX_OK) break;
      uint32_t cnt = 0;
      if (cudaMemcpyAsync(&cnt, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = set_error(RIX_ECUDA, "ring support count");
        break;
      }
      pt.ring_count = cnt;
      if ((rc = ensure<R>(job, pt.ring_idx, std::max<size_t>(cnt, 1) * sizeof(uint32_t))) != RIX_OK) break;
      ::rix::note_launch();
      k_ring_index<<<blocks_for(job->ctx, nhalf), 256, 0, st>>>(flags, pos, nhalf, pt.ring_idx.as<uint32_t>());
      if (cudaGetLastError() != cudaSuccess) rc = set_error(RIX_ECUDA, "ring index launch");
    }
    if (flags) cudaFreeAsync(flags, st);
    if (pos) cudaFreeAsync(pos, st);
    if (total) cudaFreeAsync(total, st);
    if (rc != RIX_OK) return rc;
  }
  for (int p = 0; p < P; ++p) {
    Part& pt = job->part[p];
    RIX_TRY(ensure<R>(job, pt.fs_a, tot * sizeof(cplx<R>)));
    RIX_TRY(ensure<R>(job, pt.fs_b, tot * sizeof(cplx<R>)));
    RIX_TRY(ensure<R>(job, pt.ft_a, (size_t)2 * n * n * sizeof(cplx<R>)));
    RIX_TRY(ensure<R>(job, pt.ft_b, (size_t)2 * n * n * sizeof(cplx<R>)));
    RIX_TRY(ensure<R>(job, pt.fimg, npix * sizeof(R)));
    RIX_TRY(ensure<R>(job, pt.fspec, (size_t)P * tot * sizeof(cplx<R>)));
    // the exchanged message per cycle parity: the image, or its ring-support
    // coefficients
    const size_t ob = job->desc.exchange == RIX_EXCHANGE_SPECTRAL
                          ? std::max<size_t>(pt.ring_count, 1) * sizeof(cplx<R>) : npix * sizeof(R);
    RIX_TRY(alloc_zero<R>(job, pt.outbox[0], ob, st));
    RIX_TRY(alloc_zero<R>(job, pt.outbox[1], ob, st));
    for (int q = 0; q < P; ++q)
      if (q != p) RIX_TRY(alloc_zero<R>(job, pt.rho[q], npix * sizeof(R), st));
    RIX_TRY(alloc_zero<R>(job, pt.fi_state, 4 * sizeof(R), st));
  }
  return RIX_OK;
}

template <typename R>
int op_msclean(Job* job, int p, const rix_msclean_params* prm, R* delta_out, cudaStream_t st) {
  Part& pt = job->part[p];
  const Ctx* ctx = job->ctx;
  const int n = job->desc.n, P = job->n_part, ns = prm->n_scales;
  const int cycle = pt.cycle;
  const int64_t npix = (int64_t)n * n, tot = 4 * npix;
  const double inv = 1.0 / (double)tot;
  RIX_TRY(ingest<R>(job, p, cycle, st));
  // (gamma, mu) of Eq. 7: (1, 0) at cycle 1, then the partitions' weight fractions
  double wtot = 0.0;
  for (int q = 0; q < P; ++q) wtot += job->part[q].wsum;
  FillArgs fa = fill_args<R>(job, p);
  fa.g = 1.0;
  for (int q = 0; q < P; ++q) fa.mu[q] = 0.0;
  if (cycle > 1 && wtot > 0.0) {
    fa.g = pt.wsum / wtot;
    for (int q = 0; q < P; ++q) fa.mu[q] = (q == p) ? 0.0 : job->part[q].wsum / wtot;
  }
  RIX_TRY(fill_spectra<R>(job, p, st));
  cplx<R>* dspec = pt.fs_a.as<cplx<R>>();
  cplx<R>* pspec = pt.fs_b.as<cplx<R>>();
  ::rix::note_launch(); k_fill_msclean<R><<<blocks_for(ctx, tot), 256, 0, st>>>(fa, dspec, pspec);
  RIX_LAUNCH_CHECK();

  // scale functions: stencils, their 2N-grid spectra B_s
  std::vector<double> stn_all;
  CleanArgs ca{};
  for (int s = 0; s < ns; ++s) {
    std::vector<double> stn;
    int rad = 0;
    scale_stencil((double)prm->scales[s], stn, rad);
    ca.st_off[s] = (int)stn_all.size();
    ca.st_rad[s] = rad;
    stn_all.insert(stn_all.end(), stn.begin(), stn.end());
  }
  // the composite PSF of cycles >= 2 is the same: reuse the scale spectra
  // and cross PSFs of an earlier such cycle with the same scales
  const std::vector<float> scales(prm->scales, prm->scales + ns);
  const bool reuse = cycle >= 3 && pt.ms_p_cycle >= 2 && pt.ms_p_scales == scales &&
                     pt.ms_P.bytes >= (size_t)ns * ns * tot * sizeof(R);
  if (!reuse) pt.ms_p_cycle = 0;
  RIX_TRY(ensure<R>(job, pt.ms_B, (size_t)ns * tot * sizeof(cplx<R>) + stn_all.size() * sizeof(R) + 64));
  cplx<R>* bspec = pt.ms_B.as<cplx<R>>();
  R* stn_dev = reinterpret_cast<R*>(bspec + ns * tot);
  if (!reuse) {
    std::vector<R> tmp(stn_all.begin(), stn_all.end());
    RIX_CUDA(cudaMemcpyAsync(stn_dev, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice, st));
    RIX_CUDA(cudaStreamSynchronize(st));   // tmp is a host temporary
  }
  // scratch 2N x 2N image and [2N][2N] transpose buffer
  R* img2 = nullptr;
  cplx<R>* t2 = nullptr;
  RIX_CUDA(::rix::malloc_async(&img2, tot * sizeof(R), st));
  if (::rix::malloc_async(&t2, tot * sizeof(cplx<R>), st) != cudaSuccess) {
    cudaFreeAsync(img2, st);
    return set_error(RIX_ENOMEM, "ms-CLEAN scratch");
  }
  int rc = RIX_OK;
  XformGeom g2{};
  g2.M = 2 * n; g2.L = 2 * n; g2.logL = ilog2(g2.L); g2.lo = 0; g2.S = 2 * n; g2.nplanes = 1; g2.mode = kFacNone;
  for (int s = 0; s < ns && rc == RIX_OK && !reuse; ++s) {
    if (cudaMemsetAsync(img2, 0, tot * sizeof(R), st) != cudaSuccess) { rc = set_error(RIX_ECUDA, "memset"); break; }
    ::rix::note_launch(); k_place_stencil<R><<<4, 256, 0, st>>>(stn_dev + ca.st_off[s], ca.st_rad[s], img2, 2 * n);
    if ((rc = fwd_rows<R>(ctx, g2, img2, t2, st)) != RIX_OK) break;
    rc = fwd_cols<R>(ctx, g2, t2, bspec + s * tot, st);
  }
  // scale residuals R_s = crop F^-1[B_s D] and cross PSFs P_st = F^-1[B_s B_t P]
  if (rc == RIX_OK) rc = ensure<R>(job, pt.ms_R, (size_t)ns * npix * sizeof(R));
  if (rc == RIX_OK) rc = ensure<R>(job, pt.ms_P, (size_t)ns * ns * tot * sizeof(R));
  for (int s = 0; s < ns && rc == RIX_OK; ++s)
    rc = spec_to_img<R>(job, pt, dspec, kOpMulCplx, bspec + s * tot, pt.ms_R.as<R>() + s * npix, inv, 0, st);
  // P_ts = P_st (B_s B_t = B_t B_s): the upper triangle is transformed, the
  // lower one copied
  for (int s = 0; s < ns && rc == RIX_OK && !reuse; ++s)
    for (int t = s; t < ns && rc == RIX_OK; ++t) {
      R* pst = pt.ms_P.as<R>() + (int64_t)(s * ns + t) * tot;
      ::rix::note_launch(); k_cmul3<R><<<blocks_for(ctx, tot), 256, 0, st>>>(bspec + s * tot, bspec + t * tot, pspec, dspec, tot);
      if ((rc = inv_cols<R>(ctx, g2, dspec, kOpNone, nullptr, nullptr, t2, st)) != RIX_OK) break;
      if ((rc = inv_rows<R>(ctx, g2, t2, pst, inv, 0, st)) != RIX_OK) break;
      if (t != s && cudaMemcpyAsync(pt.ms_P.as<R>() + (int64_t)(t * ns + s) * tot, pst, tot * sizeof(R),
                                    cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = set_error(RIX_ECUDA, "cross PSF copy");
    }
  cudaFreeAsync(img2, st);
  cudaFreeAsync(t2, st);
  if (rc != RIX_OK) return rc;
  if (!reuse && cycle >= 2) {
    pt.ms_p_cycle = cycle;
    pt.ms_p_scales = scales;
  }

  // scales present at cycle 1 (psi^1 of Eq. 7): partition 0 keeps all; p > 0
  // keeps s = 0 and the scales with N / (2 s) >= ell_p - delta
  int allowed = 0;
  float smax = 0.f;
  for (int s = 0; s < ns; ++s) smax = std::max(smax, prm->scales[s]);
  for (int s = 0; s < ns; ++s) {
    const double sc = prm->scales[s];
    bool ok = true;
    if (cycle == 1 && p > 0 && sc > 0.0) ok = (double)n / (2.0 * sc) >= job->ells[p - 1] - job->stats.delta_px;
    if (ok) allowed |= 1 << s;
    ca.bias[s] = smax > 0.f ? 1.0 - 0.6 * sc / (double)smax : 1.0;
  }
  // state: delta image, components, slots
  const int cap = std::max(prm->niter, 1);
  int per_sm = 0;
  void (*kern)(CleanArgs) = nullptr;
  switch (ns) {
    case 1: kern = k_msclean<R, 1>; break;
    case 2: kern = k_msclean<R, 2>; break;
    case 3: kern = k_msclean<R, 3>; break;
    case 4: kern = k_msclean<R, 4>; break;
    case 5: kern = k_msclean<R, 5>; break;
    case 6: kern = k_msclean<R, 6>; break;
    case 7: kern = k_msclean<R, 7>; break;
    case 8: kern = k_msclean<R, 8>; break;
    default: return set_error(RIX_EINVAL, "%d scales", ns);
  }
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
  // at most four CTAs per SM: enough loads in flight for the sweeps, and
  // every CTA reads every CTA's candidate at each iteration
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * std::min(std::max(per_sm, 1), 4),
                                                                 ceil_div(npix, 256)));
  const size_t comp_bytes = (size_t)cap * (2 * sizeof(int) + sizeof(double)) + 16;
  RIX_TRY(ensure<R>(job, pt.ms_comp, comp_bytes));
  RIX_TRY(ensure<R>(job, pt.ms_state, 2 * (size_t)nblk * sizeof(Cand<R>) + 64));
  pt.ms_ncomp_cap = cap;
  RIX_CUDA(cudaMemsetAsync(pt.delta.p, 0, npix * sizeof(R), st));
  RIX_CUDA(cudaMemsetAsync(pt.ms_comp.p, 0, comp_bytes, st));
  char* cb = pt.ms_comp.as<char>();
  ca.n = n;
  ca.ns = ns;
  ca.niter = prm->niter;
  ca.gain = prm->gain;
  ca.threshold = prm->threshold;
  ca.allowed = allowed;
  ca.R = pt.ms_R.p;
  ca.P = pt.ms_P.p;
  ca.model = pt.delta.p;
  ca.stencil = stn_dev;
  ca.slots = pt.ms_state.p;
  ca.comp_amp = reinterpret_cast<double*>(cb);
  ca.comp_s = reinterpret_cast<int*>(cb + (size_t)cap * sizeof(double));
  ca.comp_pix = ca.comp_s + cap;
  ca.count = ca.comp_pix + cap;
  RIX_TRY(ensure<R>(job, pt.sync, 16));
  RIX_CUDA(cudaMemsetAsync(pt.sync.p, 0, sizeof(unsigned int), st));
  ca.barrier = pt.sync.as<unsigned int>();
  ca.status = job->status.as<int>();
  void* args[] = {&ca};
  ::rix::note_launch();
  timing_mark(kTimeMinorLoop, st, true);
  RIX_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(nblk), dim3(256), args, 0, st));
  timing_mark(kTimeMinorLoop, st, false);
  RIX_TRY(publish<R>(job, p, cycle, st));
  if (delta_out) RIX_CUDA(cudaMemcpyAsync(delta_out, pt.delta.p, npix * sizeof(R), cudaMemcpyDeviceToDevice, st));
  return RIX_OK;
}

// Everything of partition p's FISTA minor cycle before the iteration loop:
// ingest the received images, the fill tables (Mx, C), lambda's reference,
// the coefficient buffers; *f receives the loop's description.
template <typename R>
int fista_prepare(Job* job, int p, const rix_fista_params* prm, FistaLoop<R>* f, cudaStream_t st) {
  Part& pt = job->part[p];
  const Ctx* ctx = job->ctx;
  const int n = job->desc.n;
  const int cycle = pt.cycle;
  const int64_t npix = (int64_t)n * n, tot = 4 * npix;
  RIX_TRY(ingest<R>(job, p, cycle, st));
  if (!pt.lambda_set) {
    // lambda_rel refers to max |residual| of the partition's first cycle
    RIX_CUDA(cudaMemsetAsync(pt.fi_state.as<R>() + 1, 0, sizeof(R), st));
    ::rix::note_launch(); k_absmax<R><<<blocks_for(ctx, npix), 256, 0, st>>>(pt.resid.as<R>(), npix, pt.fi_state.as<R>() + 1);
    RIX_LAUNCH_CHECK();
    pt.lambda_set = true;
  }
  RIX_TRY(fill_spectra<R>(job, p, st));
  RIX_TRY(ensure<R>(job, pt.fi_mx, tot * sizeof(R)));
  RIX_TRY(ensure<R>(job, pt.fi_c, tot * sizeof(cplx<R>)));
  FillArgs fa = fill_args<R>(job, p);
  const double gn = cycle == 1 ? 0.0 : 1.0;
  RIX_CUDA(cudaMemsetAsync(pt.fi_state.p, 0, sizeof(R), st));
  ::rix::note_launch(); k_fill_fista<R><<<blocks_for(ctx, tot), 256, 0, st>>>(fa, gn, pt.fi_mx.as<R>(), pt.fi_c.as<cplx<R>>(),
                                                        pt.fi_state.as<R>());
  RIX_LAUNCH_CHECK();
  const bool cat = prm->dictionary == RIX_DICT_DB1_8;
  const int64_t ncoef = (cat ? 8 : 1) * npix;
  RIX_TRY(alloc_zero<R>(job, pt.fi_alpha, ncoef * sizeof(R), st));
  RIX_TRY(alloc_zero<R>(job, pt.fi_y, ncoef * sizeof(R), st));
  RIX_TRY(ensure<R>(job, pt.fi_x, (cat ? 8 : 1) * npix * sizeof(R)));
  RIX_TRY(ensure<R>(job, pt.fi_alpha_prev, (cat ? 8 : 1) * npix * sizeof(R)));
  RIX_TRY(ensure<R>(job, pt.fi_d, npix * sizeof(R)));
  double sched_bn = 0.0;
  if (prm->sched_a > 0.0) {
    // lambda_n = a ||residual of cycle n||_2 b^n: the squared norm goes to state[2]
    RIX_CUDA(cudaMemsetAsync(pt.fi_state.as<R>() + 2, 0, sizeof(R), st));
    ::rix::note_launch(); k_sumsq<R><<<blocks_for(ctx, npix), 256, 0, st>>>(pt.resid.as<R>(), npix, pt.fi_state.as<R>() + 2);
    RIX_LAUNCH_CHECK();
    sched_bn = std::pow(prm->sched_b, (double)cycle);
  }
  RIX_TRY(ensure<R>(job, pt.sync, 16));
  *f = FistaLoop<R>{};
  f->alpha = pt.fi_alpha.as<R>();
  f->y = pt.fi_y.as<R>();
  f->x = pt.fi_x.as<R>();
  f->g = pt.fimg.as<R>();
  f->tmp = pt.fi_alpha_prev.as<R>();
  f->ta = pt.ft_a.as<cplx<R>>();
  f->tb = pt.ft_b.as<cplx<R>>();
  f->mx = pt.fi_mx.as<R>();
  f->c = pt.fi_c.as<cplx<R>>();
  f->d = pt.fi_d.as<R>();
  f->state = pt.fi_state.as<R>();
  f->tw = twiddles<R>(ctx);
  f->barrier = pt.sync.as<unsigned int>();
  f->status = job->status.as<int>();
  f->lambda = prm->lambda;
  f->lambda_rel = prm->lambda_rel;
  f->n = n;
  f->levels = prm->levels;
  f->iters = prm->iters;
  f->dict = prm->dictionary;
  f->sched_a = prm->sched_a;
  f->sched_bn = sched_bn;
  if (cat) {
    // member level buffers: A in fi_x, B in fi_alpha_prev, 8 N^2 each
    f->xs = f->x;
    f->bs = f->tmp;
    f->delta = pt.delta.as<R>();
  }
  return RIX_OK;
}

// the loops of f[0 .. nb) in one launch
template <typename R>
int fista_run(const Ctx* ctx, const FistaLoop<R>* f, int nb, const rix_fista_params* prm, cudaStream_t st) {
  if (prm->iters <= 0 || nb <= 0) return RIX_OK;
  if (prm->dictionary == RIX_DICT_DB1_8) return fista_loop_dict<R, RIX_DICT_DB1_8>(ctx, f, nb, st);
  return fista_loop_dict<R, RIX_DICT_DB4>(ctx, f, nb, st);
}

// Everything after the loop: i_bar_p = W alpha, the image update and the
// Phi / rho exchange terms (publish).
template <typename R>
int fista_finish(Job* job, int p, const rix_fista_params* prm, R* delta_out, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  const int64_t npix = (int64_t)n * n;
  if (prm->dictionary == RIX_DICT_DB1_8) {
    // the loop wrote W alpha into delta; with no iteration alpha = 0
    if (prm->iters == 0) RIX_CUDA(cudaMemsetAsync(pt.delta.p, 0, npix * sizeof(R), st));
  } else {
    RIX_TRY(idwt2<R>(job->ctx, pt.fi_alpha.as<R>(), pt.delta.as<R>(), pt.fi_alpha_prev.as<R>(), n, prm->levels, st));
  }
  RIX_TRY(publish<R>(job, p, pt.cycle, st));
  if (delta_out) RIX_CUDA(cudaMemcpyAsync(delta_out, pt.delta.p, npix * sizeof(R), cudaMemcpyDeviceToDevice, st));
  return RIX_OK;
}

template <typename R>
int op_fista(Job* job, int p, const rix_fista_params* prm, R* delta_out, cudaStream_t st) {
  FistaLoop<R> f;
  RIX_TRY(fista_prepare<R>(job, p, prm, &f, st));
  RIX_TRY(fista_run<R>(job->ctx, &f, 1, prm, st));
  return fista_finish<R>(job, p, prm, delta_out, st);
}

template <typename R>
int op_fista_batch(Job* job, int nb, const int* parts, const rix_fista_params* prm, cudaStream_t st,
                   const cudaStream_t* ps) {
  FistaLoop<R> f[kMaxPart];
  // each partition's preparation on its own stream, the loop after all of them
  for (int i = 0; i < nb; ++i) {
    Part& pt = job->part[parts[i]];
    RIX_TRY(fista_prepare<R>(job, parts[i], prm, &f[i], ps[i]));
    RIX_CUDA(cudaEventRecord(pt.ev_prep, ps[i]));
    RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_prep, 0));
  }
  RIX_TRY(fista_run<R>(job->ctx, f, nb, prm, st));
  RIX_CUDA(cudaEventRecord(job->ev_batch, st));
  // each partition's finish on its own stream, `st` after all of them
  for (int i = 0; i < nb; ++i) {
    Part& pt = job->part[parts[i]];
    RIX_CUDA(cudaStreamWaitEvent(ps[i], job->ev_batch, 0));
    RIX_TRY(fista_finish<R>(job, parts[i], prm, nullptr, ps[i]));
    RIX_CUDA(cudaEventRecord(pt.ev_done, ps[i]));
    RIX_CUDA(cudaStreamWaitEvent(st, pt.ev_done, 0));
  }
  return RIX_OK;
}

template <typename R>
int op_combine(Job* job, R* out, cudaStream_t st) {
  const int64_t npix = (int64_t)job->desc.n * job->desc.n;
  const R* ptrs[kMaxPart];
  for (int q = 0; q < job->n_part; ++q) ptrs[q] = job->part[q].model.as<R>();
  const R** dptrs = nullptr;
  RIX_CUDA(::rix::malloc_async((void**)&dptrs, sizeof(ptrs), st));
  RIX_CUDA(cudaMemcpyAsync(dptrs, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, st));
  ::rix::note_launch(); k_mean<R><<<blocks_for(job->ctx, npix), 256, 0, st>>>(out, dptrs, job->n_part, npix);
  cudaFreeAsync(dptrs, st);
  RIX_LAUNCH_CHECK();
  RIX_CUDA(cudaStreamSynchronize(st));   // ptrs is a host temporary
  return RIX_OK;
}

#define RIX_MINOR_INST(R)                                                                   \
  template int fill_init<R>(Job*, cudaStream_t);                                            \
  template int op_msclean<R>(Job*, int, const rix_msclean_params*, R*, cudaStream_t);       \
  template int op_fista<R>(Job*, int, const rix_fista_params*, R*, cudaStream_t);           \
  template int op_fista_batch<R>(Job*, int, const int*, const rix_fista_params*, cudaStream_t,          \
                                 const cudaStream_t*);                                                     \
  template int op_combine<R>(Job*, R*, cudaStream_t);
RIX_MINOR_INST(float)
RIX_MINOR_INST(double)

int get_components(Job* job, int part, int32_t* count, int32_t capacity, int32_t* scale_out,
                   int32_t* pixel_out, double* amp_out, cudaStream_t st) {
  Job& J = *job;
  if (part < 0 || part >= J.n_part) return set_error(RIX_EINVAL, "partition out of range");
  Part& pt = J.part[part];
  *count = 0;
  if (pt.ms_ncomp_cap == 0 || !pt.ms_comp.p) return RIX_OK;
  const int cap = pt.ms_ncomp_cap;
  char* cb = pt.ms_comp.as<char>();
  const double* amp = reinterpret_cast<const double*>(cb);
  const int* sc = reinterpret_cast<const int*>(cb + (size_t)cap * sizeof(double));
  const int* px = sc + cap;
  const int* cnt = px + cap;
  int c = 0;
  RIX_CUDA(cudaMemcpyAsync(&c, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
  RIX_CUDA(cudaStreamSynchronize(st));
  *count = c;
  const int k = std::min(c, (int)std::max(capacity, 0));
  if (k > 0) {
    if (scale_out) RIX_CUDA(cudaMemcpyAsync(scale_out, sc, k * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (pixel_out) RIX_CUDA(cudaMemcpyAsync(pixel_out, px, k * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (amp_out) RIX_CUDA(cudaMemcpyAsync(amp_out, amp, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    RIX_CUDA(cudaStreamSynchronize(st));
  }
  return RIX_OK;
}

// ---- band-limited exchange calls ---------------------------------------------
// Gamma_p F pad i_bar_p of the partition's last minor cycle on its ring
// support (half plane), ring_count coefficients, into `out`
template <typename R>
int op_phi_pack(Job* job, int p, cplx<R>* out, cudaStream_t st) {
  Part& pt = job->part[p];
  const int n = job->desc.n;
  const int64_t tot = (int64_t)4 * n * n;
  cplx<R>* spec = nullptr;
  cplx<R>* T = nullptr;
  int rc = RIX_OK;
  if (malloc_async(&spec, tot * sizeof(cplx<R>), st) != cudaSuccess ||
      malloc_async(&T, (size_t)2 * n * n * sizeof(cplx<R>), st) != cudaSuccess) {
    cudaGetLastError();
    rc = set_error(RIX_ENOMEM, "pack scratch");
  }
  if (rc == RIX_OK) {
    const XformGeom g = fill_geom(n);
    rc = fwd_rows<R>(job->ctx, g, pt.delta.as<R>(), T, st);
    if (rc == RIX_OK) rc = fwd_cols<R>(job->ctx, g, T, spec, st);
  }
  if (rc == RIX_OK) {
    ::rix::note_launch();
    k_phi_pack<R><<<blocks_for(job->ctx, pt.ring_count), 256, 0, st>>>(job->gam.as<R>() + p * tot, spec,
                                                                       pt.ring_idx.as<uint32_t>(), pt.ring_count, out);
    if (cudaGetLastError() != cudaSuccess) rc = set_error(RIX_ECUDA, "pack launch");
  }
  if (spec) cudaFreeAsync(spec, st);
  if (T) cudaFreeAsync(T, st);
  return rc;
}

// Phi_p = crop F^-1 of the spectrum rebuilt from partition p's coefficients
template <typename R>
int op_phi_unpack(Job* job, int p, const cplx<R>* coef, R* out, cudaStream_t st) {
  const int n = job->desc.n;
  const int64_t tot = (int64_t)4 * n * n;
  cplx<R>* spec = nullptr;
  cplx<R>* T = nullptr;
  int rc = RIX_OK;
  if (malloc_async(&spec, tot * sizeof(cplx<R>), st) != cudaSuccess ||
      malloc_async(&T, (size_t)2 * n * n * sizeof(cplx<R>), st) != cudaSuccess) {
    cudaGetLastError();
    rc = set_error(RIX_ENOMEM, "unpack scratch");
  }
  if (rc == RIX_OK) rc = phi_from_coef<R>(job, p, coef, spec, T, out, 1.0 / (double)tot, 0, st);
  if (spec) cudaFreeAsync(spec, st);
  if (T) cudaFreeAsync(T, st);
  return rc;
}

template int op_phi_pack<float>(Job*, int, float2*, cudaStream_t);
template int op_phi_pack<double>(Job*, int, double2*, cudaStream_t);
template int op_phi_unpack<float>(Job*, int, const float2*, float*, cudaStream_t);
template int op_phi_unpack<double>(Job*, int, const double2*, double*, cudaStream_t);

}  // namespace rix
