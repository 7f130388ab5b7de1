// spmc_tables.h -- host-side Gauss-type node and transform tables (Section 2.3).
#pragma once

namespace spmc {
void jacobi_values(int m, double a, double b, double x, double* P);
void jacobi_zeros(int n, double a, double b, double* z);
void legendre_values(int m, double x, double* L);
void space_nodes(int n, double* x);                               // JG(1,1), ascending
void time_nodes(int family, int M, double* xi);                   // LGL (0), left Radau (1), CGL (2)
void time_weights(int family, int M, const double* xi, double* w);
void space_analysis(int n, double* A);                            // a_pj, [p][j]
void time_analysis(int family, int M, double* B);                 // b_qk, [q][k]
void phi_values(int n, double x, double* phi);                    // phi_0..phi_{n-1}
// fractional case (alpha in (0, 2), a = alpha / 2)
void space_nodes_frac(int n, double alpha, double* x);            // zeros of P^{(a,a)}_n
void space_analysis_frac(int n, double alpha, double* A);         // [p][j]
constexpr int kFracModes = 40;
constexpr int kFracRa = 0, kFracRb = 40, kFracLam = 80, kFracSin = 120, kFracA = 160, kFracAlpha = 161,
              kFracGamma = 162, kFracLnB = 163, kFracRp = 164, kFracRq = 244, kFracSeries = 80,
              kFracTable = 324;   // Gamma(1+alpha); ln B(a, 1-a); the jump law's series ratios
void frac_table(double alpha, double* T);
// Chebyshev basis (time family 2: Chebyshev-Gauss-Lobatto)
void space_nodes_cheb(int n, double* x);                          // interior CGL points, ascending
void space_analysis_cheb(int n, double* A);                       // coefficients of T_p - T_{p+2}
}  // namespace spmc
