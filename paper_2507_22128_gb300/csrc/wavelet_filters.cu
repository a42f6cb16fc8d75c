// Daubechies low-pass filters db1 .. db8 for the concatenated dictionary of
// the FISTA minor cycle (Sec. 5.2), computed on the host.
//
// Daubechies' construction: |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)) with
// P(y) = sum_{k<p} binom(p-1+k, k) y^k.  Each root y_j of P (degree p-1, found
// here by the Weierstrass / Durand-Kerner simultaneous iteration in long
// double, then Newton-polished) gives, through y = (2 - z - 1/z)/4, the pair
// of z-roots of z^2 - (2 - 4y) z + 1; the root inside the unit circle is kept
// (spectral factorisation).  The filter is the polynomial with those roots
// and a p-fold root at z = -1, scaled to sum sqrt(2) and ordered with the
// larger energy first (minimum phase).
#include <cmath>
#include <complex>
#include <vector>

#include "rix_internal.cuh"

namespace rix {

int daubechies_lowpass(int p, double* h) {
  if (p < 1 || p > 8 || !h) return set_error(RIX_EINVAL, "daubechies order %d outside 1..8", p);
  using cl = std::complex<long double>;
  const int deg = p - 1;
  std::vector<long double> c(p);          // P(y) coefficients, c[k] of y^k
  for (int k = 0; k < p; ++k) {
    long double b = 1.0L;                   // binom(p - 1 + k, k)
    for (int j = 1; j <= k; ++j) b = b * (long double)(p - 1 + j) / (long double)j;
    c[k] = b;
  }
  auto P = [&](cl y) {
    cl v = 0.0L;
    for (int k = deg; k >= 0; --k) v = v * y + c[k];
    return v;
  };
  auto dP = [&](cl y) {
    cl v = 0.0L;
    for (int k = deg; k >= 1; --k) v = v * y + (long double)k * c[k];
    return v;
  };
  std::vector<cl> y(deg);
  const cl seed(0.4L, 0.9L);
  cl s = 1.0L;
  for (int i = 0; i < deg; ++i) { y[i] = s; s *= seed; }
  for (int it = 0; it < 500 && deg > 0; ++it) {
    long double moved = 0.0L;
    for (int i = 0; i < deg; ++i) {
      cl den = c[deg];
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (y[i] - y[j]);
      const cl step = P(y[i]) / den;
      y[i] -= step;
      moved = std::max(moved, std::abs(step));
    }
    if (moved < 1e-30L) break;
  }
  for (int i = 0; i < deg; ++i)
    for (int it = 0; it < 4; ++it) y[i] -= P(y[i]) / dP(y[i]);
  // polynomial coefficients, highest power first, of prod (z - r)
  std::vector<cl> poly(1, cl(1.0L));
  auto mul = [&](cl r) {
    std::vector<cl> q(poly.size() + 1, cl(0.0L));
    for (size_t i = 0; i < poly.size(); ++i) {
      q[i] += poly[i];
      q[i + 1] -= r * poly[i];
    }
    poly.swap(q);
  };
  for (int i = 0; i < deg; ++i) {
    const cl b = 2.0L - 4.0L * y[i];
    const cl d = std::sqrt(b * b - 4.0L);
    const cl z1 = 0.5L * (b + d), z2 = 0.5L * (b - d);
    mul(std::abs(z1) < 1.0L ? z1 : z2);
  }
  for (int i = 0; i < p; ++i) mul(cl(-1.0L));
  const int K = 2 * p;
  std::vector<long double> hr(K);
  long double sum = 0.0L;
  for (int i = 0; i < K; ++i) {
    hr[i] = poly[i].real();
    sum += hr[i];
  }
  const long double scale = std::sqrt(2.0L) / sum;
  long double head = 0.0L, tail = 0.0L;
  for (int i = 0; i < K; ++i) hr[i] *= scale;
  for (int i = 0; i <= p && i < K; ++i) {
    head += hr[i] * hr[i];
    tail += hr[K - 1 - i] * hr[K - 1 - i];
  }
  for (int i = 0; i < K; ++i) h[i] = (double)(tail > head ? hr[K - 1 - i] : hr[i]);
  return K;
}

}  // namespace rix

extern "C" int rix_daubechies_lowpass(int p, double* h_out) { return rix::daubechies_lowpass(p, h_out); }
