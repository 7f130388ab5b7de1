// spmc_tables.cpp -- host-side node and transform tables of the CUDA library.
//
// Gauss-type nodes (Section 2.3): Jacobi-Gauss (1,1) in space; shifted
// Legendre-Gauss-Lobatto or left Gauss-Radau in time.  Zeros are found as zeros
// of Jacobi polynomials P^{(a,b)}_n by Newton's method with deflation:
//   JG(1,1) interior nodes      = zeros of P^{(1,1)}_n,
//   LGL interior nodes          = zeros of P^{(1,1)}_{M-1}  (= zeros of L_M'),
//   left-Radau interior nodes   = zeros of P^{(0,1)}_M     (with -1 added).
// Analysis matrices: a_pj of Eq. spacelag and b_qk of Eq. timeLag.
#include "spmc_tables.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace spmc {

static const double kPi = 3.14159265358979323846;

// P^{(a,b)}_0..P^{(a,b)}_m at x by the standard three-term recurrence.
void jacobi_values(int m, double a, double b, double x, double* P) {
  P[0] = 1.0;
  if (m == 0) return;
  P[1] = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int n = 2; n <= m; ++n) {
    double c = 2.0 * n + a + b;
    double a1 = 2.0 * n * (n + a + b) * (c - 2.0);
    double a2 = (c - 1.0) * (a * a - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (n + a - 1.0) * (n + b - 1.0) * c;
    P[n] = ((a2 + a3 * x) * P[n - 1] - a4 * P[n - 2]) / a1;
  }
}

// P^{(a,b)}_n and its derivative (d/dx P^{(a,b)}_n = (n+a+b+1)/2 P^{(a+1,b+1)}_{n-1}).
static void jacobi_and_derivative(int n, double a, double b, double x, double* val, double* der) {
  std::vector<double> P(n + 1), Q(std::max(n, 1));
  jacobi_values(n, a, b, x, P.data());
  *val = P[n];
  if (n == 0) { *der = 0.0; return; }
  jacobi_values(n - 1, a + 1.0, b + 1.0, x, Q.data());
  *der = 0.5 * (n + a + b + 1.0) * Q[n - 1];
}

// The n zeros of P^{(a,b)}_n in ascending order.
void jacobi_zeros(int n, double a, double b, double* z) {
  for (int k = 0; k < n; ++k) {
    // guess between Chebyshev points of the first kind
    double x = -std::cos((2.0 * k + 1.0) * kPi / (2.0 * n + 1.0));
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi_and_derivative(n, a, b, x, &p, &dp);
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += 1.0 / (x - z[i]);
      double dx = p / (dp - s * p);
      x -= dx;
      if (std::fabs(dx) <= 4e-16 * std::max(1.0, std::fabs(x))) {
        // two polishing steps
        for (int pol = 0; pol < 2; ++pol) {
          jacobi_and_derivative(n, a, b, x, &p, &dp);
          s = 0.0;
          for (int i = 0; i < k; ++i) s += 1.0 / (x - z[i]);
          x -= p / (dp - s * p);
        }
        break;
      }
    }
    z[k] = x;
  }
  std::sort(z, z + n);
}

void legendre_values(int m, double x, double* L) { jacobi_values(m, 0.0, 0.0, x, L); }

void space_nodes(int n, double* x) { jacobi_zeros(n, 1.0, 1.0, x); }

void time_nodes(int family, int M, double* xi) {
  xi[0] = -1.0;
  if (family == 2) {   // Chebyshev-Gauss-Lobatto -cos(pi k / M)
    for (int k = 1; k < M; ++k) xi[k] = -std::cos(kPi * k / M);
    xi[M] = 1.0;
    return;
  }
  if (family == 0) {
    xi[M] = 1.0;
    if (M >= 2) jacobi_zeros(M - 1, 1.0, 1.0, xi + 1);
  } else {
    jacobi_zeros(M, 0.0, 1.0, xi + 1);
  }
}

void time_weights(int family, int M, const double* xi, double* w) {
  std::vector<double> L(M + 1);
  for (int k = 0; k <= M; ++k) {
    legendre_values(M, xi[k], L.data());
    double LM = L[M];
    if (family == 0) w[k] = 2.0 / (M * (M + 1.0) * LM * LM);
    else w[k] = (k == 0) ? 2.0 / ((M + 1.0) * (M + 1.0)) : (1.0 - xi[k]) / ((M + 1.0) * (M + 1.0) * LM * LM);
  }
}

// a_pj (row-major [p][j]) of Eq. spacelag with the JG(1,1) weights
// w_j = 8(n+1) / ((n+2) (1-x_j^2) P_n'(x_j)^2).
void space_analysis(int n, double* A) {
  std::vector<double> x(n), P(n + 1);
  space_nodes(n, x.data());
  for (int j = 0; j < n; ++j) {
    double pn, dpn;
    jacobi_and_derivative(n, 1.0, 1.0, x[j], &pn, &dpn);
    double one_m = 1.0 - x[j] * x[j];
    double wj = 8.0 * (n + 1.0) / ((n + 2.0) * one_m * dpn * dpn);
    jacobi_values(n - 1, 1.0, 1.0, x[j], P.data());
    for (int p = 0; p < n; ++p) {
      double gt = 8.0 * (p + 1.0) / ((2.0 * p + 3.0) * (p + 2.0));
      A[p * n + j] = wj * P[p] / (one_m * gt);
    }
  }
}

// b_qk (row-major [q][k]) of Eq. timeLag on the reference interval; gamma_q =
// 2/(2q+1) for q < M and the discrete norm sum_k L_M(xi_k)^2 w_k for q = M.
void time_analysis(int family, int M, double* B) {
  if (family == 2) {
    // the DCT-I at the CGL points: B[q][k] = 2 T_q(xi_k) / (M c_q c_k), c = 2 at the ends
    std::vector<double> xi(M + 1);
    time_nodes(2, M, xi.data());
    for (int q = 0; q <= M; ++q)
      for (int k = 0; k <= M; ++k) {
        const double cq = (q == 0 || q == M) ? 2.0 : 1.0, ck = (k == 0 || k == M) ? 2.0 : 1.0;
        B[q * (M + 1) + k] = 2.0 * std::cos(q * std::acos(xi[k])) / (M * cq * ck);
      }
    return;
  }
  std::vector<double> xi(M + 1), w(M + 1), L(M + 1), Lk((M + 1) * (M + 1));
  time_nodes(family, M, xi.data());
  time_weights(family, M, xi.data(), w.data());
  for (int k = 0; k <= M; ++k) {
    legendre_values(M, xi[k], L.data());
    for (int q = 0; q <= M; ++q) Lk[q * (M + 1) + k] = L[q];
  }
  double gM = 0.0;
  for (int k = 0; k <= M; ++k) gM += Lk[M * (M + 1) + k] * Lk[M * (M + 1) + k] * w[k];
  for (int q = 0; q <= M; ++q) {
    double g = (q < M) ? 2.0 / (2.0 * q + 1.0) : gM;
    for (int k = 0; k <= M; ++k) B[q * (M + 1) + k] = Lk[q * (M + 1) + k] * w[k] / g;
  }
}

// The fractional case (generalised Jacobi functions (1-x^2)^a P^{(a,a)}_p,
// a = alpha/2): nodes = zeros of P^{(a,a)}_n; analysis
// A[p][j] = w_j P_p(x_j) / ((1-x_j^2)^a gamma_p) with the Gauss-Jacobi weights
// w_j = 2^{2a+1} Gamma(n+a+1)^2 / (n! Gamma(n+2a+1) (1-x_j^2) P_n'(x_j)^2) and
// gamma_p = 2^{2a+1} Gamma(p+a+1)^2 / ((2p+2a+1) p! Gamma(p+2a+1)).
static double gj_norm(double a, int p) {
  return std::exp((2.0 * a + 1.0) * std::log(2.0) + 2.0 * std::lgamma(p + a + 1.0) - std::lgamma(p + 1.0) -
                  std::lgamma(p + 2.0 * a + 1.0)) / (2.0 * p + 2.0 * a + 1.0);
}
static void gj_weights(int n, double a, const double* x, double* w) {
  const double c = std::exp((2.0 * a + 1.0) * std::log(2.0) + 2.0 * std::lgamma(n + a + 1.0) - std::lgamma(n + 1.0) -
                            std::lgamma(n + 2.0 * a + 1.0));
  for (int j = 0; j < n; ++j) {
    double pn, dpn;
    jacobi_and_derivative(n, a, a, x[j], &pn, &dpn);
    w[j] = c / ((1.0 - x[j] * x[j]) * dpn * dpn);
  }
}
void space_nodes_frac(int n, double alpha, double* x) { jacobi_zeros(n, 0.5 * alpha, 0.5 * alpha, x); }
void space_analysis_frac(int n, double alpha, double* A) {
  const double a = 0.5 * alpha;
  std::vector<double> x(n), w(n), P(n + 1);
  space_nodes_frac(n, alpha, x.data());
  gj_weights(n, a, x.data(), w.data());
  for (int j = 0; j < n; ++j) {
    jacobi_values(n - 1, a, a, x[j], P.data());
    for (int p = 0; p < n; ++p) A[p * n + j] = w[j] * P[p] / (std::pow(1.0 - x[j] * x[j], a) * gj_norm(a, p));
  }
}

// Device table of the fractional case (layout in spmc_tables.h): recurrence
// P_p = ra_p x P_{p-1} - rb_p P_{p-2} of P^{(a,a)} (p >= 2), the eigenvalues
// lam_p = Gamma(alpha+p+1)/p! of (-Delta)^{alpha/2} on the basis, and the
// coefficients s_p of sin(x) = sum_p s_p P^{(a,a)}_p(x) (40-point Gauss-Jacobi
// quadrature: exact for the sine's Taylor polynomial to degree 79).
void frac_table(double alpha, double* T) {
  const double a = 0.5 * alpha;
  for (int i = 0; i < kFracTable; ++i) T[i] = 0.0;
  for (int p = 2; p < kFracModes; ++p) {
    const double c = 2.0 * p + 2.0 * a;
    T[kFracRa + p] = (c - 1.0) * c / (2.0 * p * (p + 2.0 * a));
    T[kFracRb + p] = (p + a - 1.0) * (p + a - 1.0) * c / (p * (p + 2.0 * a) * (c - 2.0));
  }
  for (int p = 0; p < kFracModes; ++p) T[kFracLam + p] = std::exp(std::lgamma(alpha + p + 1.0) - std::lgamma(p + 1.0));
  const int nq = kFracModes;
  std::vector<double> x(nq), w(nq), P(nq + 1);
  jacobi_zeros(nq, a, a, x.data());
  gj_weights(nq, a, x.data(), w.data());
  for (int j = 0; j < nq; ++j) {
    jacobi_values(nq - 1, a, a, x[j], P.data());
    for (int p = 0; p < nq; ++p) T[kFracSin + p] += w[j] * std::sin(x[j]) * P[p];
  }
  for (int p = 0; p < nq; ++p) T[kFracSin + p] /= gj_norm(a, p);
  T[kFracA] = a;
  T[kFracAlpha] = alpha;
  T[kFracGamma] = std::exp(std::lgamma(1.0 + alpha));
  // the jump law U ~ Beta(a, 1-a): ln B(a, 1-a) and the term ratios of the series
  // I_x(p,q) = x^p (1-x)^q / (p B) sum_k prod_{i<k} x (p+q+i)/(p+1+i) for (p,q) = (a, 1-a), (1-a, a)
  T[kFracLnB] = std::lgamma(a) + std::lgamma(1.0 - a);
  for (int k = 0; k < kFracSeries; ++k) {
    T[kFracRp + k] = (1.0 + k) / (a + 1.0 + k);
    T[kFracRq + k] = (1.0 + k) / (2.0 - a + k);
  }
}

// The Chebyshev basis: interior CGL points -cos(pi j / (n+1)), j = 1..n; the
// analysis matrix maps nodal values to coefficients of phi_p = T_p - T_{p+2}:
// a_k = 2 / ((n+1) c_k) sum_j u_j T_k(x_j) (c_0 = 2), c_p = a_p + c_{p-2}.
void space_nodes_cheb(int n, double* x) {
  for (int j = 0; j < n; ++j) x[j] = -std::cos(kPi * (j + 1) / (n + 1));
}
void space_analysis_cheb(int n, double* A) {
  std::vector<double> x(n);
  space_nodes_cheb(n, x.data());
  const int N = n + 1;
  for (int j = 0; j < n; ++j) {
    const double th = std::acos(x[j]);
    for (int p = 0; p < n; ++p) {
      double acc = 0.0;
      for (int k = p; k >= 0; k -= 2) acc += 2.0 * std::cos(k * th) / (N * (k == 0 ? 2.0 : 1.0));
      A[p * n + j] = acc;
    }
  }
}

// phi_p(x) = (1-x^2) P^{(1,1)}_p(x), p < n (u0 from coefficients).
void phi_values(int n, double x, double* phi) {
  std::vector<double> P(n);
  jacobi_values(n - 1, 1.0, 1.0, x, P.data());
  for (int p = 0; p < n; ++p) phi[p] = (1.0 - x * x) * P[p];
}

}  // namespace spmc
