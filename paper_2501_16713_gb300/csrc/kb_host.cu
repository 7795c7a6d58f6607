// Interpolation kernel and deapodization function in FP64 on the host.
//
// The kernel is the Kaiser-Bessel function used by the paper's gridding
// (Notations: c(x) and C(k_x); deapodization divides by the transform of the
// interpolation kernel), minus its edge value so that it is continuous at
// +-W/2:  c(u) = I0(beta sqrt(1 - (2u/W)^2)) - 1 for |u| < W/2.  Its Fourier
// transform C(nu) = W [sinh(z)/z - sin(pi W nu)/(pi W nu)],
// z = sqrt(beta^2 - (pi W nu)^2), is evaluated with libm sinh/sin/sqrt.
//
// The GPU evaluates c through one polynomial per tap: for fractional offset f
// of the first tap, tap t sits at distance u = f + W/2 - 1 - t and
//   c(f + W/2 - 1 - t) ~= sum_k a[t][k] s^k,   s = 2f - 1 in [-1, 1],
// interpolated at Chebyshev nodes in FP64 (the approach of piecewise
// polynomial kernel evaluation by Horner's rule; Barnett, Magland & af
// Klinteberg, SIAM J. Sci. Comput. 2019).
#include <cmath>
#include <cstring>

#include "kb_host.h"

namespace nrs {

double bessel_i0m1(double z) {
  const double q = 0.25 * z * z;
  double term = q, sum = q;
  for (int k = 2; k < 500; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

double beatty_beta(int width, double osf) {
  const double r = double(width) / osf;
  return M_PI * std::sqrt(r * r * (osf - 0.5) * (osf - 0.5) - 0.8);
}

double kb_kernel(double u, int width, double beta) {
  const double x = 2.0 * u / double(width);
  if (!(std::fabs(x) < 1.0)) return 0.0;
  return bessel_i0m1(beta * std::sqrt(1.0 - x * x));
}

double kb_kernel_ft(double nu, int width, double beta) {
  const double a = M_PI * double(width) * nu;
  const double z2 = beta * beta - a * a;
  double first;
  if (z2 > 0) {
    const double z = std::sqrt(z2);
    first = std::sinh(z) / z;
  } else if (z2 < 0) {
    const double y = std::sqrt(-z2);
    first = std::sin(y) / y;
  } else {
    first = 1.0;
  }
  const double second = (a == 0.0) ? 1.0 : std::sin(a) / a;
  return double(width) * (first - second);
}

namespace {

// Solve the n x n system V a = b in place (Gaussian elimination, partial pivoting).
void solve_dense(double* V, double* b, int n) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(V[r * n + col]) > std::fabs(V[piv * n + col])) piv = r;
    if (piv != col) {
      for (int c = 0; c < n; ++c) std::swap(V[col * n + c], V[piv * n + c]);
      std::swap(b[col], b[piv]);
    }
    for (int r = col + 1; r < n; ++r) {
      const double f = V[r * n + col] / V[col * n + col];
      for (int c = col; c < n; ++c) V[r * n + c] -= f * V[col * n + c];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < n; ++c) s -= V[r * n + c] * b[c];
    b[r] = s / V[r * n + r];
  }
}

}  // namespace

double fit_kernel_polys(int width, double beta, KernelCoefs* out) {
  std::memset(out, 0, sizeof(*out));
  const int n = kNumCoef;
  double worst = 0.0;
  const double peak = kb_kernel(0.0, width, beta);
  for (int t = 0; t < width; ++t) {
    double V[kNumCoef * kNumCoef], b[kNumCoef];
    for (int i = 0; i < n; ++i) {
      const double s = std::cos(M_PI * (i + 0.5) / n);
      const double f = 0.5 * (s + 1.0);
      double p = 1.0;
      for (int k = 0; k < n; ++k) {
        V[i * n + k] = p;
        p *= s;
      }
      b[i] = kb_kernel(f + 0.5 * width - 1.0 - t, width, beta);
    }
    solve_dense(V, b, n);
    for (int k = 0; k < n; ++k) out->c[t][k] = float(b[k]);
    // error of the FP32 Horner evaluation (as on the GPU) against FP64 c
    for (int i = 0; i <= 4000; ++i) {
      const float f = float(i) / 4000.0f;
      const float s = std::fmaf(2.0f, f, -1.0f);
      float acc = out->c[t][n - 1];
      for (int k = n - 2; k >= 0; --k) acc = std::fmaf(acc, s, out->c[t][k]);
      const double ref = kb_kernel(double(f) + 0.5 * width - 1.0 - t, width, beta);
      worst = std::fmax(worst, std::fabs(double(acc) - ref) / peak);
    }
  }
  return worst;
}

}  // namespace nrs
