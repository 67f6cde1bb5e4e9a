// Host-side set-up shared by every entry point that runs the transverse solve phases: the
// FFT plan of a grid axis, the twiddle and wavenumber tables (built in FP64 on the host,
// stored in the working precision), and the map from the device status word to qsa_status.
#pragma once
#include <cmath>
#include <vector>

#include "../../include/qsa.h"
#include "qsa_common.cuh"

namespace qsa {

// Stages of the Stockham transform of n = 2^a 3^b points: radix 4 while it divides, then
// radix 2, then radix 3; per stage the product of the earlier radices and the shifts that
// replace divisions when a count is a power of two.
inline FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  while (m % 4 == 0) { p.radix[p.nstages++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[p.nstages++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.nstages++] = 3; m /= 3; }
  auto log2_or_neg = [](int v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
  };
  int ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    p.ns[s] = ns;
    p.nbsh[s] = log2_or_neg(n / p.radix[s]);
    p.nssh[s] = log2_or_neg(ns);
    ns *= p.radix[s];
  }
  return p;
}

// Twiddles exp(-2 pi i m / n) of the x axis (m < nx) followed by those of the y axis.
template <typename R>
std::vector<C<R>> twiddle_table(int nx, int ny) {
  std::vector<C<R>> tw((size_t)nx + ny);
  for (int m = 0; m < nx; ++m) {
    const double t = -2.0 * M_PI * m / nx;
    tw[m] = C<R>{R(std::cos(t)), R(std::sin(t))};
  }
  for (int m = 0; m < ny; ++m) {
    const double t = -2.0 * M_PI * m / ny;
    tw[(size_t)nx + m] = C<R>{R(std::cos(t)), R(std::sin(t))};
  }
  return tw;
}

// Wavenumber table of the k-space solves: [k_x (nxh)][k_x derivative symbol (nxh)][k_y (ny)]
// [k_y derivative symbol (ny)], with k_x = 2 pi m / Lx (m = 0..nx/2), k_y = 2 pi m / Ly in
// numpy.fft order, and the derivative symbols zero at the Nyquist index of an even grid.
template <typename R>
std::vector<R> wavenumber_table(int nx, int ny, double Lx, double Ly) {
  const int nxh = nx / 2 + 1;
  std::vector<R> kt((size_t)2 * nxh + 2 * ny);
  for (int m = 0; m < nxh; ++m) {
    const double k = 2.0 * M_PI * m / Lx;
    kt[m] = R(k);
    kt[(size_t)nxh + m] = (nx % 2 == 0 && 2 * m == nx) ? R(0) : R(k);
  }
  for (int m = 0; m < ny; ++m) {
    const int mm = (m <= ny / 2) ? m : m - ny;
    const double k = 2.0 * M_PI * mm / Ly;
    kt[(size_t)2 * nxh + m] = R(k);
    kt[(size_t)2 * nxh + ny + m] = (ny % 2 == 0 && 2 * m == ny) ? R(0) : R(k);
  }
  return kt;
}

// qsa_status of a device status word: errors take precedence over the floor warning.
inline int status_code(int st) {
  if (st & ST_TIMEOUT) return QSA_ERR_TIMEOUT;
  if (st & ST_NONFINITE) return QSA_ERR_NONFINITE;
  if (st & ST_FLOOR) return QSA_WARN_PSI_FLOOR;
  return QSA_OK;
}

// Text of a negative status_code.
inline const char* status_text(int rc) {
  return rc == QSA_ERR_TIMEOUT ? "device wait exceeded spin_limit"
                               : rc == QSA_ERR_NONFINITE ? "non-finite field value"
                                                         : "device error";
}

}  // namespace qsa
