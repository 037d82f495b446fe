// Host FP64 building blocks of the box FGT's 1D tables (Section 2.4).
#pragma once

namespace fgt {

// n-point Gauss-Legendre rule on [-1, 1], ascending nodes (n <= 64).
void gl_rule(int n, double *x, double *w);
// P_0..P_nmax at x (three-term recurrence).
void legendre_values(int nmax, double x, double *P);
// T[n*k + j] = (2n+1)/2 w_j P_n(eta_j): node values -> Legendre coefficients (Definition val2poldef,
// with the row = coefficient, column = node reading).
void val_to_pol(int k, const double *eta, const double *w, double *T);
// J_lambda[P_n](t), n = 0..nmax (nmax <= 70), eq. (gsintegrals).
void gauss_legendre_integrals(double lambda, double t, int nmax, double *J);
// j_n(x), n = 0..nmax (nmax <= 70).
void spherical_bessel(double x, int nmax, double *out);
// I[P_n](t) = 2 i^n j_n(t), eq. (pwintegrals2).
void legendre_fourier_integrals(double t, int nmax, double *re, double *im);

}  // namespace fgt
