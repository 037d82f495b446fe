// FP64 host building blocks of the 1D tables of the box FGT (Section 2.4 and
// Section 4.1): Gauss-Legendre rule, Legendre values, values -> Legendre
// coefficients (Definition val2poldef), the Gaussian integrals J_lambda[P_n]
// (eq. (gsintegrals), seeds in closed form, five-term recurrence
// eq. (Jnrecurrence)), spherical Bessel functions and the Fourier integrals
// I[P_n] (eq. (pwintegrals2)).
#include "fgt_tables.h"

#include <cmath>

static constexpr double kPi = 3.14159265358979323846264338327950288;

namespace fgt {

void gl_rule(int n, double *x, double *w) {
  // Newton iteration on P_n from the asymptotic root estimate; roots placed in ascending order.
  const int half = (n + 1) / 2;
  for (int i = 0; i < half; ++i) {
    double z = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, pc = z;  // P_0, P_1
      for (int m = 2; m <= n; ++m) {
        const double pn = ((2 * m - 1) * z * pc - (m - 1) * pm) / m;
        pm = pc;
        pc = pn;
      }
      if (n == 1) { pc = z; pm = 1.0; }
      dp = n * (pm - z * pc) / (1.0 - z * z);
      const double step = pc / dp;
      z -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    {
      double pm = 1.0, pc = z;
      for (int m = 2; m <= n; ++m) {
        const double pn = ((2 * m - 1) * z * pc - (m - 1) * pm) / m;
        pm = pc;
        pc = pn;
      }
      if (n == 1) { pc = z; pm = 1.0; }
      dp = n * (pm - z * pc) / (1.0 - z * z);
    }
    const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;             // smallest first
    x[n - 1 - i] = z;
    w[i] = wi;
    w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

void legendre_values(int nmax, double x, double *P) {
  P[0] = 1.0;
  if (nmax >= 1) P[1] = x;
  for (int n = 1; n < nmax; ++n) P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1);
}

void val_to_pol(int k, const double *eta, const double *w, double *T) {
  double P[64];
  for (int j = 0; j < k; ++j) {
    legendre_values(k - 1, eta[j], P);
    for (int n = 0; n < k; ++n) T[n * k + j] = 0.5 * (2 * n + 1) * w[j] * P[n];
  }
}

// erf(b) - erf(a) for a <= b without cancellation when both have the same sign
static double erf_diff(double a, double b) {
  if (a >= 0) return std::erfc(a) - std::erfc(b);
  if (b <= 0) return std::erfc(-b) - std::erfc(-a);
  return std::erf(b) - std::erf(a);
}

void gauss_legendre_integrals(double lam, double t, int nmax, double *J) {
  if (lam <= 0.125) {
    const double a = (-1.0 - t) / lam, b = (1.0 - t) / lam;
    const double ea = std::exp(-a * a), eb = std::exp(-b * b);
    const double l2 = lam * lam;
    double Jl[72];
    Jl[0] = 0.5 * std::sqrt(kPi) * lam * erf_diff(a, b);
    const double D = -0.5 * l2 * (eb - ea);                 // int (x - t) g
    Jl[1] = t * Jl[0] + D;
    const double V2 = -0.5 * l2 * ((1.0 - t) * eb + (1.0 + t) * ea) + 0.5 * l2 * Jl[0];  // int (x - t)^2 g
    const double M2 = V2 + 2.0 * t * D + t * t * Jl[0];     // int x^2 g
    Jl[2] = 0.5 * (3.0 * M2 - Jl[0]);
    // (n+2)/(2n+3) J_{n+2} = t (J_{n+1} - J_{n-1}) + (n-1)/(2n-1) J_{n-2}
    //                        + (2n+1) (lam^2/2 + 1/((2n+3)(2n-1))) J_n,   n >= 1
    for (int n = 1; n + 2 <= nmax; ++n) {
      const double jm2 = (n >= 2) ? Jl[n - 2] : 0.0;
      const double rhs = t * (Jl[n + 1] - Jl[n - 1]) + (double)(n - 1) / (2 * n - 1) * jm2 +
                         (2 * n + 1) * (0.5 * l2 + 1.0 / ((2.0 * n + 3.0) * (2.0 * n - 1.0))) * Jl[n];
      Jl[n + 2] = rhs * (2.0 * n + 3.0) / (n + 2.0);
    }
    for (int n = 0; n <= nmax; ++n) J[n] = Jl[n];
    return;
  }
  // smooth integrand: composite Gauss-Legendre, 8 panels x 24 nodes
  static thread_local double qx[24], qw[24];
  static thread_local bool init = false;
  if (!init) { gl_rule(24, qx, qw); init = true; }
  for (int n = 0; n <= nmax; ++n) J[n] = 0.0;
  double P[72];
  for (int pnl = 0; pnl < 8; ++pnl) {
    const double lo = -1.0 + 0.25 * pnl;
    for (int q = 0; q < 24; ++q) {
      const double x = lo + 0.125 * (qx[q] + 1.0);
      const double g = std::exp(-(t - x) * (t - x) / (lam * lam)) * 0.125 * qw[q];
      legendre_values(nmax, x, P);
      for (int n = 0; n <= nmax; ++n) J[n] += g * P[n];
    }
  }
}

void spherical_bessel(double x, int nmax, double *out) {
  if (x == 0.0) {
    out[0] = 1.0;
    for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
    return;
  }
  const double ax = std::fabs(x);
  const int nb = nmax > 1 ? nmax : 1;                  // keep j_1 for the sign test
  const int N = (nb > (int)ax ? nb : (int)ax) + 60;    // start far above both n and x
  // Miller backward recurrence j_{n-1} = (2n+1)/x j_n - j_{n+1} from (j_{N+1}, j_N) = (0, tiny),
  // normalised with sum_n (2n+1) j_n^2 = 1; rescaled against overflow.
  double buf[80];
  double jp = 0.0, jc = 1e-30, norm = 0.0;
  for (int n = N; n >= 1; --n) {
    if (n <= nb) buf[n] = jc;
    norm += (2.0 * n + 1.0) * jc * jc;
    const double jm = (2.0 * n + 1.0) / ax * jc - jp;
    jp = jc;
    jc = jm;
    if (std::fabs(jc) > 1e150) {
      const double sc = 1e-150;
      jc *= sc;
      jp *= sc;
      norm *= sc * sc;
      for (int m = n; m <= nb; ++m) buf[m] *= sc;
    }
  }
  buf[0] = jc;
  norm += jc * jc;
  double s = 1.0 / std::sqrt(norm);
  // overall sign from j_0 = sin(x)/x, or from j_1 = sin(x)/x^2 - cos(x)/x near the zeros of sin
  const double j0 = std::sin(ax) / ax;
  const double j1 = std::sin(ax) / (ax * ax) - std::cos(ax) / ax;
  if (std::fabs(j0) >= std::fabs(j1)) {
    if (j0 * buf[0] < 0) s = -s;
  } else {
    if (j1 * buf[1] < 0) s = -s;
  }
  for (int n = 0; n <= nmax; ++n) out[n] = buf[n] * s;
  if (x < 0)
    for (int n = 1; n <= nmax; n += 2) out[n] = -out[n];
}

void legendre_fourier_integrals(double t, int nmax, double *re, double *im) {
  double j[80];
  spherical_bessel(t, nmax, j);
  // 2 i^n j_n(t): i^0 = 1, i^1 = i, i^2 = -1, i^3 = -i
  for (int n = 0; n <= nmax; ++n) {
    const double v = 2.0 * j[n];
    switch (n & 3) {
      case 0: re[n] = v; im[n] = 0; break;
      case 1: re[n] = 0; im[n] = v; break;
      case 2: re[n] = -v; im[n] = 0; break;
      default: re[n] = 0; im[n] = -v; break;
    }
  }
}

}  // namespace fgt
