/*
 * spmc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, serial FP64 CPU restatement of the hp-version time-stepping
 * spectral Monte Carlo method (residual iteration, Section 2.4 and Algorithm 1),
 * written from the paper for checking the CUDA path.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Every routine follows the definition it cites, term by term: no blocking, no
 * sum factorisation, no precomputed time slices.  The residual at a walker point
 * is the direct sum over all coefficients of Eq. (u_N).  OpenMP is used only to
 * run independent nodes side by side; every per-node sum is sequential, so the
 * result does not depend on the thread count.
 *
 * Readings of points where the paper is silent or garbled (each listed with its
 * reason in the design notes):
 *   - spatial nodes are Jacobi-Gauss (1,1) interior nodes (Section 2.3);
 *   - time nodes are shifted LGL, or left Gauss-Radau (includes t_{n-1});
 *   - b_qk uses reference-interval weights with gamma_q = 2/(2q+1), q < M_n, and
 *     the discrete norm for q = M_n (Eq. timeLag);
 *   - -d^2/dx^2 phi_p = (p+1)(p+2) P_p^{(1,1)}, not the printed (p+1) (Eq. u_N);
 *   - the d/dt coefficients sum over l > q with l+q odd and keep the spatial basis
 *     phi_p (Legendre derivative identity; the printed P_p^{(1,1)} is garbled);
 *   - along a walk the integrand time runs backward from t_{n,l} to t_{n-1}
 *     (Feynman-Kac for the backward heat semigroup, Eq. fkx_2);
 *   - N_* = max(1, ceil(N_ref (t_{n,l}-t_{n-1})/h_n)) (Eq. time division);
 *   - walk_mode 0 (the solver's walk): balls inside Omega ("a ball B_r(x_j)
 *     inside the domain", Section 2.2) of radius min(J, dist to the boundary),
 *     each step weighted by the ball's mean exit time, the step integral
 *     estimated at a Green-function point of the ball (the representation
 *     W(x) E_{Q_r}[f(Y, t_q)] of Lemma 3.3's proof) and a random sub-step time;
 *     the fixed-radius walk with point evaluation at the centres is unstable
 *     for the spectral degrees used here;
 *   - walk_mode 1 (the walk of Table 1): fixed radius J, Q_L sums q = 0..L-1
 *     with L from Eq. indexL, so L = 0 when X_1 exits;
 *   - directions: d=1 one sign bit; d=2 angle 2 pi U; d>=3 normalised Box-Muller
 *     Gaussians (Lemma Xlocation only asks for a uniform direction);
 *   - the first iterate is the constant-in-time extension of row 0 (Remark 2.1);
 *   - Philox4x32-10 keyed by the 64-bit seed, counter (word block, sample, node,
 *     instance|interval|iteration): the paper does not name a generator.
 *
 * Parity pins (tests under tests/): Gauss tables against scipy, analysis matrices
 * against Legendre-form basis values from numpy, reconstruction and derivative
 * maps against numpy polynomial calculus, the polynomial fixed point (r == 0),
 * the fixed-step walk mean against an exact lattice Markov-chain computation,
 * the inside-ball walk against Dynkin's formula, Philox against an independent
 * implementation, exit probabilities against Table 1, and convergence to
 * closed-form solutions.  The adjoint is checked by forward-mode
 * tangents (orc_solve_tangent) and central differences on common random numbers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAXD 5
#define ORC_MAXN 64

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with a     */
/* Weyl-sequence key schedule.                                                */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod1;
    uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The random words of one walk.  Word w of the walk of (sample, node) in
 * (instance, interval, iteration) is lane w%4 of Philox at counter
 * (w/4, sample, node, instance<<20 | interval<<10 | iteration). */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t block[4];
  int64_t cached;
} orc_stream;

static void stream_init(orc_stream* s, uint64_t seed, uint32_t sample, uint32_t node,
                        int instance, int interval, int iteration) {
  s->key[0] = (uint32_t)(seed & 0xffffffffu);
  s->key[1] = (uint32_t)(seed >> 32);
  s->ctr[0] = 0;
  s->ctr[1] = sample;
  s->ctr[2] = node;
  s->ctr[3] = ((uint32_t)(instance & 0xfff) << 20) | ((uint32_t)(interval & 0x3ff) << 10) |
              (uint32_t)(iteration & 0x3ff);
  s->cached = -1;
}

static uint32_t stream_word(orc_stream* s, int64_t w) {
  int64_t blk = w / 4;
  if (blk != s->cached) {
    s->ctr[0] = (uint32_t)blk;
    orc_philox4x32_10(s->ctr, s->key, s->block);
    s->cached = blk;
  }
  return s->block[w % 4];
}

/* Uniform on (0,1) from two words, 53 bits: ((a>>5) 2^26 + (b>>6) + 1/2) 2^-53. */
double orc_u01_pair(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Words drawn per walk step for dimension d. */
int orc_words_per_step(int d) {
  if (d == 1) return 1;
  if (d == 2) return 2;
  return 4 * ((d + 1) / 2);
}

/* Direction theta_q, uniform on S^{d-1} (Lemma Xlocation), from the step's words. */
static void draw_direction(orc_stream* s, int d, int64_t step_index, double* theta) {
  int64_t w0 = step_index * (int64_t)orc_words_per_step(d);
  if (d == 1) {
    uint32_t a = stream_word(s, w0);
    theta[0] = (a >> 31) ? -1.0 : 1.0;
    return;
  }
  if (d == 2) {
    double U = orc_u01_pair(stream_word(s, w0), stream_word(s, w0 + 1));
    theta[0] = cos(2.0 * ORC_PI * U);
    theta[1] = sin(2.0 * ORC_PI * U);
    return;
  }
  double z[ORC_MAXD + 1];
  int npairs = (d + 1) / 2;
  for (int k = 0; k < npairs; ++k) {
    double U1 = orc_u01_pair(stream_word(s, w0 + 4 * k), stream_word(s, w0 + 4 * k + 1));
    double U2 = orc_u01_pair(stream_word(s, w0 + 4 * k + 2), stream_word(s, w0 + 4 * k + 3));
    double R = sqrt(-2.0 * log(U1));
    z[2 * k] = R * cos(2.0 * ORC_PI * U2);
    z[2 * k + 1] = R * sin(2.0 * ORC_PI * U2);
  }
  double nrm = 0.0;
  for (int e = 0; e < d; ++e) nrm += z[e] * z[e];
  nrm = sqrt(nrm);
  for (int e = 0; e < d; ++e) theta[e] = z[e] / nrm;
}

/* Inside-ball walk (walk_mode 0): the words of one step, padded to whole
 * Philox blocks.  d <= 2, one word per uniform, 8 words (2 blocks):
 *   [next-step direction | Green point direction | time sub-point word |
 *    roulette word | Green radius uniform(s) (d = 2: two) | unused].
 * d >= 3, uniforms from word pairs:
 *   [next-step direction | Green point direction | Green radius uniform (a pair) |
 *    time sub-point word | roulette word].
 * The paper leaves the random stream open; with d <= 2 a 32-bit word per
 * uniform (resolution 2^-32) is far below the Monte Carlo error, and the words
 * the walk needs at every step (direction, sub-point, roulette) share one
 * block. */
int orc_ball_words_per_step(int d) {
  if (d <= 2) return 8;
  int wd = orc_words_per_step(d);
  int w = 2 * wd + 2 + 2;
  return (w + 3) / 4 * 4;
}
static int64_t ball_gdir_index(int d) { return d <= 2 ? 1 : orc_words_per_step(d); }
static int64_t ball_radius_index(int d) { return d <= 2 ? 4 : 2 * orc_words_per_step(d); }
static int64_t ball_gword_index(int d) { return d <= 2 ? 2 : 2 * orc_words_per_step(d) + 2; }
static int64_t ball_rword_index(int d) { return ball_gword_index(d) + 1; }

/* Uniform on (0,1) from one word: (a + 1/2) 2^-32. */
double orc_u01_word(uint32_t a) { return ((double)a + 0.5) * (1.0 / 4294967296.0); }

/* Direction from the words starting at w0 (same laws as draw_direction; the
 * d = 2 angle from one word). */
static void direction_at(orc_stream* s, int d, int64_t w0, double* theta) {
  if (d == 1) {
    theta[0] = (stream_word(s, w0) >> 31) ? -1.0 : 1.0;
    return;
  }
  if (d == 2) {
    double U = orc_u01_word(stream_word(s, w0));
    theta[0] = cos(2.0 * ORC_PI * U);
    theta[1] = sin(2.0 * ORC_PI * U);
    return;
  }
  double z[ORC_MAXD + 1];
  int npairs = (d + 1) / 2;
  for (int k = 0; k < npairs; ++k) {
    double U1 = orc_u01_pair(stream_word(s, w0 + 4 * k), stream_word(s, w0 + 4 * k + 1));
    double U2 = orc_u01_pair(stream_word(s, w0 + 4 * k + 2), stream_word(s, w0 + 4 * k + 3));
    double R = sqrt(-2.0 * log(U1));
    z[2 * k] = R * cos(2.0 * ORC_PI * U2);
    z[2 * k + 1] = R * sin(2.0 * ORC_PI * U2);
  }
  double nrm = 0.0;
  for (int e = 0; e < d; ++e) nrm += z[e] * z[e];
  nrm = sqrt(nrm);
  for (int e = 0; e < d; ++e) theta[e] = z[e] / nrm;
}

/* Radial law of the ball's Green function G_r(0, y) (the expected occupation
 * density of Brownian motion started at the centre and killed on the sphere),
 * as a fraction v = |y|/r: d=1: density 2(1-v); d=2: density 4 v log(1/v);
 * d>=3: density proportional to v - v^{d-1}. */
double orc_green_radius(int d, double U1, double U2) {
  if (d == 1) return 1.0 - sqrt(U1);
  if (d == 2) return sqrt(U1 * U2);
  /* CDF F(v) = (d v^2 - 2 v^d)/(d-2), solved for F(v) = U1 by bisection */
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 60; ++it) {
    double v = 0.5 * (lo + hi);
    double vd = 1.0;
    for (int k = 0; k < d; ++k) vd *= v;
    double F = (d * v * v - 2.0 * vd) / (d - 2.0);
    if (F < U1) lo = v; else hi = v;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------- */
/* Orthogonal polynomials (Section 2.3).                                      */
/* ------------------------------------------------------------------------- */
/* Legendre L_0..L_m at x by the three-term recurrence. */
void orc_legendre(int m, double x, double* L) {
  L[0] = 1.0;
  if (m >= 1) L[1] = x;
  for (int k = 1; k < m; ++k) L[k + 1] = ((2.0 * k + 1.0) * x * L[k] - k * L[k - 1]) / (k + 1.0);
}

/* Jacobi P_0^{(1,1)}..P_m^{(1,1)} at x:
 * n(n+2) P_n = (2n+1)(n+1) x P_{n-1} - n(n+1) P_{n-2}, P_0 = 1, P_1 = 2x. */
void orc_jacobi11(int m, double x, double* P) {
  P[0] = 1.0;
  if (m >= 1) P[1] = 2.0 * x;
  for (int n = 2; n <= m; ++n)
    P[n] = ((2.0 * n + 1.0) * (n + 1.0) * x * P[n - 1] - n * (n + 1.0) * P[n - 2]) / (n * (n + 2.0));
}

/* Babuska-Shen basis phi_p = (1-x^2) P_p^{(1,1)}, p = 0..m (Section 2.3). */
void orc_phi(int m, double x, double* phi) {
  double P[ORC_MAXN + 2];
  orc_jacobi11(m, x, P);
  for (int p = 0; p <= m; ++p) phi[p] = (1.0 - x * x) * P[p];
}

/* Jacobi P_0^{(a,a)}..P_m^{(a,a)} at x (the general three-term recurrence with
 * both parameters a):
 * 2n(n+2a)(2n+2a-2) P_n = (2n+2a-1)(2n+2a)(2n+2a-2) x P_{n-1} - 2(n+a-1)^2(2n+2a) P_{n-2},
 * P_0 = 1, P_1 = (a+1) x. */
void orc_jacobi_aa(int m, double a, double x, double* P) {
  P[0] = 1.0;
  if (m >= 1) P[1] = (a + 1.0) * x;
  for (int n = 2; n <= m; ++n) {
    double c = 2.0 * n + 2.0 * a;
    P[n] = ((c - 1.0) * c * (c - 2.0) * x * P[n - 1] - 2.0 * (n + a - 1.0) * (n + a - 1.0) * c * P[n - 2]) /
           (2.0 * n * (n + 2.0 * a) * (c - 2.0));
  }
}

/* The fractional case (Section 4, Ex. 2; the remark on generalised Jacobi
 * functions): basis phi_p = (1-x^2)_+^a P_p^{(a,a)}, a = alpha/2, with
 * (-Delta)^{alpha/2} phi_p = lam_p P_p^{(a,a)} on (-1,1), lam_p = Gamma(alpha+p+1)/p!
 * (the hypersingular integral with the standard constant
 * C_{1,alpha} = alpha 2^{alpha-1} Gamma((1+alpha)/2) / (sqrt(pi) Gamma(1-alpha/2))).
 * For alpha = 2 these are the Babuska-Shen basis and (p+1)(p+2). */
double orc_frac_lambda(double alpha, int p) { return exp(lgamma(alpha + p + 1.0) - lgamma(p + 1.0)); }

/* int_{-1}^{1} (1-x^2)^a P_p^{(a,a)}(x)^2 dx */
static double jacobi_aa_norm(double a, int p) {
  return exp((2.0 * a + 1.0) * log(2.0) + 2.0 * lgamma(p + a + 1.0) - lgamma(p + 1.0) - lgamma(p + 2.0 * a + 1.0)) /
         (2.0 * p + 2.0 * a + 1.0);
}

/* ------------------------------------------------------------------------- */
/* Gauss-type nodes and weights.                                              */
/* ------------------------------------------------------------------------- */
/* Jacobi-Gauss (a,a): the n zeros of P_n^{(a,a)}, weights for (1-x^2)^a:
 * w_j = 2^{2a+1} Gamma(n+a+1)^2 / (Gamma(n+1) Gamma(n+2a+1) (1-x_j^2) P_n'(x_j)^2),
 * with (1-x^2) P_n' = (n+a) P_{n-1} - n x P_n.  Newton with deflation. */
void orc_gj_nodes(int n, double a, double* x, double* w) {
  double P[ORC_MAXN + 2];
  for (int j = 0; j < n; ++j) {
    double z = -cos(ORC_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 200; ++it) {
      orc_jacobi_aa(n, a, z, P);
      double dP = ((n + a) * P[n - 1] - n * z * P[n]) / (1.0 - z * z);
      double defl = 0.0;
      for (int k = 0; k < j; ++k) defl += 1.0 / (z - x[k]);
      double step = P[n] / (dP - P[n] * defl);
      z -= step;
      if (fabs(step) < 1e-16 * (1.0 + fabs(z))) break;
    }
    x[j] = z;
  }
  for (int u = 0; u < n; ++u)
    for (int v = u + 1; v < n; ++v)
      if (x[v] < x[u]) { double t = x[u]; x[u] = x[v]; x[v] = t; }
  double cst = exp((2.0 * a + 1.0) * log(2.0) + 2.0 * lgamma(n + a + 1.0) - lgamma(n + 1.0) - lgamma(n + 2.0 * a + 1.0));
  for (int j = 0; j < n; ++j) {
    orc_jacobi_aa(n, a, x[j], P);
    double dP = ((n + a) * P[n - 1] - n * x[j] * P[n]) / (1.0 - x[j] * x[j]);
    w[j] = cst / ((1.0 - x[j] * x[j]) * dP * dP);
  }
}
/* Jacobi-Gauss (1,1): the n zeros of P_n^{(1,1)} and the weights for the
 * weight function (1-x^2):  w_j = 8(n+1)/((n+2)(1-x_j^2) P_n'(x_j)^2), with
 * (1-x^2) P_n' = (n+1) P_{n-1} - n x P_n.  Newton with deflation of the roots
 * already found, started from Chebyshev-type guesses. */
void orc_jg11_nodes(int n, double* x, double* w) {
  double P[ORC_MAXN + 2];
  for (int j = 0; j < n; ++j) {
    double z = -cos(ORC_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      orc_jacobi11(n, z, P);
      double dP = ((n + 1.0) * P[n - 1] - n * z * P[n]) / (1.0 - z * z);
      double defl = 0.0;
      for (int k = 0; k < j; ++k) defl += 1.0 / (z - x[k]);
      double step = P[n] / (dP - P[n] * defl);
      z -= step;
      if (fabs(step) < 1e-16 * (1.0 + fabs(z))) break;
    }
    x[j] = z;
  }
  /* sort ascending */
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (x[b] < x[a]) { double t = x[a]; x[a] = x[b]; x[b] = t; }
  for (int j = 0; j < n; ++j) {
    orc_jacobi11(n, x[j], P);
    double dP = ((n + 1.0) * P[n - 1] - n * x[j] * P[n]) / (1.0 - x[j] * x[j]);
    w[j] = 8.0 * (n + 1.0) / ((n + 2.0) * (1.0 - x[j] * x[j]) * dP * dP);
  }
}

/* Legendre-Gauss-Lobatto, M+1 points: -1, the zeros of L_M' (which are the
 * Jacobi-Gauss (1,1) nodes of order M-1), +1; w_k = 2/(M(M+1) L_M(x_k)^2). */
void orc_lgl_nodes(int M, double* xi, double* w) {
  double L[ORC_MAXN + 2], dummy[ORC_MAXN + 2];
  xi[0] = -1.0;
  xi[M] = 1.0;
  if (M >= 2) orc_jg11_nodes(M - 1, xi + 1, dummy);
  for (int k = 0; k <= M; ++k) {
    orc_legendre(M, xi[k], L);
    w[k] = 2.0 / (M * (M + 1.0) * L[M] * L[M]);
  }
}

/* Left Gauss-Radau, M+1 points including -1: the zeros of L_M + L_{M+1};
 * w_0 = 2/(M+1)^2, w_k = (1-x_k)/((M+1)^2 L_M(x_k)^2). */
void orc_radau_left_nodes(int M, double* xi, double* w) {
  double L[ORC_MAXN + 3];
  xi[0] = -1.0;
  for (int j = 1; j <= M; ++j) {
    double z = -cos(ORC_PI * (2.0 * j) / (2.0 * M + 1.0));
    for (int it = 0; it < 100; ++it) {
      orc_legendre(M + 1, z, L);
      double F = L[M] + L[M + 1];
      /* (1-z^2) L_m' = m (L_{m-1} - z L_m) */
      double dLM = M * (L[M - 1] - z * L[M]) / (1.0 - z * z);
      double dLM1 = (M + 1.0) * (L[M] - z * L[M + 1]) / (1.0 - z * z);
      double dF = dLM + dLM1;
      double defl = 0.0;
      for (int k = 0; k < j; ++k) defl += 1.0 / (z - xi[k]);
      double step = F / (dF - F * defl);
      z -= step;
      if (fabs(step) < 1e-16 * (1.0 + fabs(z))) break;
    }
    xi[j] = z;
  }
  for (int a = 1; a <= M; ++a)
    for (int b = a + 1; b <= M; ++b)
      if (xi[b] < xi[a]) { double t = xi[a]; xi[a] = xi[b]; xi[b] = t; }
  for (int k = 0; k <= M; ++k) {
    orc_legendre(M, xi[k], L);
    w[k] = (k == 0) ? 2.0 / ((M + 1.0) * (M + 1.0))
                    : (1.0 - xi[k]) / ((M + 1.0) * (M + 1.0) * L[M] * L[M]);
  }
}

/* Chebyshev polynomials T_0..T_m at x and their second derivatives:
 * T_{k+1} = 2x T_k - T_{k-1}, T'_{k+1} = 2 T_k + 2x T'_k - T'_{k-1},
 * T''_{k+1} = 4 T'_k + 2x T''_k - T''_{k-1}. */
void orc_cheb(int m, double x, double* T, double* T2) {
  double T1[ORC_MAXN + 4];
  T[0] = 1.0; T1[0] = 0.0; T2[0] = 0.0;
  if (m >= 1) { T[1] = x; T1[1] = 1.0; T2[1] = 0.0; }
  for (int k = 1; k < m; ++k) {
    T[k + 1] = 2.0 * x * T[k] - T[k - 1];
    T1[k + 1] = 2.0 * T[k] + 2.0 * x * T1[k] - T1[k - 1];
    T2[k + 1] = 4.0 * T1[k] + 2.0 * x * T2[k] - T2[k - 1];
  }
}

/* Chebyshev-Gauss-Lobatto points -cos(pi k / M), k = 0..M (the Chebyshev
 * basis of the remark on quasi-linear reconstruction after Algorithm 1). */
void orc_cgl_nodes(int M, double* xi) {
  for (int k = 0; k <= M; ++k) xi[k] = -cos(ORC_PI * k / M);
  xi[0] = -1.0;
  xi[M] = 1.0;
}

void orc_time_nodes(int family, int M, double* xi, double* w) {
  if (family == 0) orc_lgl_nodes(M, xi, w);
  else if (family == 1) orc_radau_left_nodes(M, xi, w);
  else {
    orc_cgl_nodes(M, xi);
    for (int k = 0; k <= M; ++k) w[k] = 0.0;   /* not used by the Chebyshev transform */
  }
}

/* ------------------------------------------------------------------------- */
/* Analysis matrices (Eqs. spacelag, timeLag).                                */
/* ------------------------------------------------------------------------- */
/* A[p*n + j] = omega_j P_p^{(1,1)}(x_j) / ((1-x_j^2) gamma~_p),
 * gamma~_p = 8(p+1)/((2p+3)(p+2)). */
void orc_space_analysis(int n, double* A) {
  double x[ORC_MAXN], w[ORC_MAXN], P[ORC_MAXN + 2];
  orc_jg11_nodes(n, x, w);
  for (int j = 0; j < n; ++j) {
    orc_jacobi11(n - 1, x[j], P);
    for (int p = 0; p < n; ++p) {
      double gt = 8.0 * (p + 1.0) / ((2.0 * p + 3.0) * (p + 2.0));
      A[p * n + j] = w[j] * P[p] / ((1.0 - x[j] * x[j]) * gt);
    }
  }
}

/* B[q*(M+1) + k] = L_q(xi_k) w_k / gamma_q on the reference interval:
 * gamma_q = 2/(2q+1) for q < M, gamma_M = sum_k L_M(xi_k)^2 w_k.
 * Chebyshev family (2): the discrete Chebyshev transform (DCT-I) of the
 * values at the CGL points, B[q][k] = 2 T_q(xi_k) / (M c_q c~_k), c_q = 2 for
 * q = 0, M (else 1), c~_k likewise (the end values count half). */
void orc_time_analysis(int family, int M, double* B) {
  double xi[ORC_MAXN + 1], w[ORC_MAXN + 1], L[ORC_MAXN + 2];
  if (family == 2) {
    double T[ORC_MAXN + 4], T2[ORC_MAXN + 4];
    orc_cgl_nodes(M, xi);
    for (int k = 0; k <= M; ++k) {
      orc_cheb(M, xi[k], T, T2);
      double ck = (k == 0 || k == M) ? 2.0 : 1.0;
      for (int q = 0; q <= M; ++q) {
        double cq = (q == 0 || q == M) ? 2.0 : 1.0;
        B[q * (M + 1) + k] = 2.0 * T[q] / (M * cq * ck);
      }
    }
    return;
  }
  double Lv[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
  orc_time_nodes(family, M, xi, w);
  for (int k = 0; k <= M; ++k) {
    orc_legendre(M, xi[k], L);
    for (int q = 0; q <= M; ++q) Lv[q * (M + 1) + k] = L[q];
  }
  for (int q = 0; q <= M; ++q) {
    double gamma;
    if (q < M) gamma = 2.0 / (2.0 * q + 1.0);
    else {
      gamma = 0.0;
      for (int k = 0; k <= M; ++k) gamma += Lv[q * (M + 1) + k] * Lv[q * (M + 1) + k] * w[k];
    }
    for (int k = 0; k <= M; ++k) B[q * (M + 1) + k] = Lv[q * (M + 1) + k] * w[k] / gamma;
  }
}

/* ------------------------------------------------------------------------- */
/* Problem description.                                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  int dim;          /* d, Omega = (-1,1)^d */
  int n_space;      /* JG(1,1) nodes per dimension = spatial modes per dimension */
  int time_family;  /* 0 = LGL, 1 = left Gauss-Radau */
  int n_ref;        /* N_* rule: N_* = max(1, ceil(n_ref (t_l - t_{n-1}) / h_n)) */
  int64_t M;        /* samples per node */
  double kappa;     /* diffusion coefficient: L = -kappa Delta */
  uint64_t seed;
  int instance;
  int f_kind;       /* 0: f = s (c0 + c1 u + c2 u^2 + c3 u^3); 1: f = s sin(u) */
  double f_coef[4];
  double f_scale;   /* s */
  int ex_kind;      /* 0: none; 1: e^{-beta t} prod sin(pi x_e); 2: e^{-beta t} prod cos(pi x_e/2);
                       3: (1+t+t^2) prod (1-x_e^2)(1+x_e) */
  double ex_beta;
  int n_threads;
  int walk_mode;    /* 0: balls inside Omega (radius min(J, dist)), 1: fixed radius J (Lemma Xlocation) */
  double shell;     /* inside-ball walk: absorbed once dist(X, boundary) < shell */
  int max_steps;    /* inside-ball walk: cap on the number of quadrature terms */
  int n_sub;        /* inside-ball walk: time sub-points per full step (a power of two) */
  int bc_kind;      /* boundary data g = trace of the exact solution: 0 g = 0; 1 homogenised by the
                       Gordon-Hall lifting G of g (the unknown is w = u - G); 2 g applied where the
                       walk is absorbed (direct estimator only) */
  int estimator;    /* 0: residual iteration (Eqs. ufg_ep1, varepsilon_1); 1: the direct estimator
                       S_i of Eq. Phi_ast (Picard iteration, Eq. linearized_func) */
  double alpha;     /* 0: L = -kappa Delta; in (0, 2): L = kappa (-Delta)^{alpha/2} (d = 1, walk_mode 2,
                       generalised Jacobi functions with a = alpha/2) */
  int basis;        /* 0: Jacobi/Legendre (Section 2.3); 1: Chebyshev in space and time (time_family 2):
                       CGL points, phi_p = T_p - T_{p+2}, T_q in time, coefficients by the DCT-I */
} orc_problem;

static int is_frac(const orc_problem* pb) { return pb->alpha > 0.0 && pb->alpha < 2.0; }

/* Spatial nodes of the problem: Jacobi-Gauss (1,1), or (a,a) in the fractional case. */
void orc_space_nodes(const orc_problem* pb, double* x, double* w) {
  if (is_frac(pb)) orc_gj_nodes(pb->n_space, 0.5 * pb->alpha, x, w);
  else if (pb->basis == 1) {
    /* the interior Chebyshev-Gauss-Lobatto points -cos(pi j / (n+1)), j = 1..n */
    double xx[ORC_MAXN + 2];
    orc_cgl_nodes(pb->n_space + 1, xx);
    for (int j = 0; j < pb->n_space; ++j) { x[j] = xx[j + 1]; w[j] = 0.0; }
  } else orc_jg11_nodes(pb->n_space, x, w);
}

/* The space analysis matrix of the problem: (1,1) as above, or in the
 * fractional case A[p*n + j] = w_j P_p^{(a,a)}(x_j) / ((1-x_j^2)^a gamma_p^{(a)})
 * (Gauss-Jacobi (a,a) quadrature of u (1-x^2)^{-a} P_p against the weight). */
void orc_space_analysis_pb(const orc_problem* pb, double* A) {
  int n = pb->n_space;
  if (pb->basis == 1) {
    /* Chebyshev: the DCT-I of (0, u_1..u_n, 0) at the N+1 = n+2 CGL points gives
     * a_k = (2 / (N c_k)) sum_j u_j T_k(x_j) (c_0 = c_N = 2); the interpolant
     * vanishes at +-1, so a = sum c_p (T_p - T_{p+2}) with c_p = a_p + c_{p-2}. */
    int N = n + 1;
    double x[ORC_MAXN], w[ORC_MAXN], T[ORC_MAXN + 4], T2[ORC_MAXN + 4];
    orc_space_nodes(pb, x, w);
    for (int j = 0; j < n; ++j) {
      orc_cheb(N, x[j], T, T2);
      for (int p = 0; p < n; ++p) {
        double acc = 0.0;
        for (int k = p; k >= 0; k -= 2) acc += 2.0 * T[k] / (N * (k == 0 ? 2.0 : 1.0));
        A[p * n + j] = acc;
      }
    }
    return;
  }
  if (!is_frac(pb)) { orc_space_analysis(n, A); return; }
  double a = 0.5 * pb->alpha, x[ORC_MAXN], w[ORC_MAXN], P[ORC_MAXN + 2];
  orc_gj_nodes(n, a, x, w);
  for (int j = 0; j < n; ++j) {
    orc_jacobi_aa(n - 1, a, x[j], P);
    for (int p = 0; p < n; ++p) A[p * n + j] = w[j] * P[p] / (pow(1.0 - x[j] * x[j], a) * jacobi_aa_norm(a, p));
  }
}

static int64_t ipow(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

double orc_f(const orc_problem* pb, double u) {
  if (pb->f_kind == 1) return pb->f_scale * sin(u);
  return pb->f_scale * (pb->f_coef[0] + u * (pb->f_coef[1] + u * (pb->f_coef[2] + u * pb->f_coef[3])));
}

double orc_df(const orc_problem* pb, double u) {
  if (pb->f_kind == 1) return pb->f_scale * cos(u);
  return pb->f_scale * (pb->f_coef[1] + u * (2.0 * pb->f_coef[2] + 3.0 * u * pb->f_coef[3]));
}

/* d f / d s (the reaction scale), used by the tangent solve. */
static double orc_df_ds(const orc_problem* pb, double u) {
  if (pb->f_kind == 1) return sin(u);
  return pb->f_coef[0] + u * (pb->f_coef[1] + u * (pb->f_coef[2] + u * pb->f_coef[3]));
}

/* Manufactured exact solution and its derivatives. */
double orc_exact(const orc_problem* pb, const double* x, double t) {
  int d = pb->dim;
  double v = 1.0;
  if (pb->ex_kind == 1) {
    for (int e = 0; e < d; ++e) v *= sin(ORC_PI * x[e]);
    return exp(-pb->ex_beta * t) * v;
  }
  if (pb->ex_kind == 2) {
    for (int e = 0; e < d; ++e) v *= cos(0.5 * ORC_PI * x[e]);
    return exp(-pb->ex_beta * t) * v;
  }
  if (pb->ex_kind == 3) {
    for (int e = 0; e < d; ++e) v *= (1.0 - x[e] * x[e]) * (1.0 + x[e]);
    return (1.0 + t + t * t) * v;
  }
  if (pb->ex_kind == 4) {
    for (int e = 0; e < d; ++e) v *= cos(ORC_PI * (x[e] - 0.3) / 3.0);
    return exp(-pb->ex_beta * t) * v;
  }
  if (pb->ex_kind == 5) {
    for (int e = 0; e < d; ++e) v *= sin(ORC_PI * x[e]);
    return exp(-pb->ex_beta * t) * v + 0.5 * t;
  }
  if (pb->ex_kind == 6 || pb->ex_kind == 7) {
    /* fractional examples (1-D, zero outside Omega), a = alpha/2:
     * 6: (1-x^2)_+^a sin(x) e^{cos t} / (1+t^2)   (Section 4, Ex. 2)
     * 7: (1+t) (1-x^2)_+^a (1 + P_1^{(a,a)}(x)/2)  (in the approximation space) */
    double a = 0.5 * pb->alpha;
    if (!(fabs(x[0]) < 1.0)) return 0.0;
    double wgt = pow(1.0 - x[0] * x[0], a);
    if (pb->ex_kind == 6) return wgt * sin(x[0]) * exp(cos(t)) / (1.0 + t * t);
    return (1.0 + t) * wgt * (1.0 + 0.5 * (a + 1.0) * x[0]);
  }
  return 0.0;
}

/* Coefficients s_n of sin(x) = sum_n s_n P_n^{(a,a)}(x), n < 40, by Gauss-Jacobi
 * (a,a) quadrature with 40 nodes (exact for the polynomial part up to degree
 * 79; the remainder of the sine's Taylor series is below 1e-40). */
static void frac_sin_coef(double a, double* s) {
  double x[40], w[40], P[41];
  orc_gj_nodes(40, a, x, w);
  for (int k = 0; k < 40; ++k) s[k] = 0.0;
  for (int j = 0; j < 40; ++j) {
    orc_jacobi_aa(39, a, x[j], P);
    for (int k = 0; k < 40; ++k) s[k] += w[j] * sin(x[j]) * P[k];
  }
  for (int k = 0; k < 40; ++k) s[k] /= jacobi_aa_norm(a, k);
}

/* (-Delta)^{alpha/2} of the fractional exact solutions at (x, t), |x| < 1:
 * kind 6: T(t) sum_n s_n lam_n P_n(x); kind 7: (1+t)(lam_0 + lam_1 P_1(x)/2). */
static double frac_op_exact(const orc_problem* pb, double x, double t) {
  static _Thread_local double cache_alpha = -1.0, s[40];
  double a = 0.5 * pb->alpha, P[41];
  if (pb->ex_kind == 7) {
    orc_jacobi_aa(1, a, x, P);
    return (1.0 + t) * (orc_frac_lambda(pb->alpha, 0) + 0.5 * orc_frac_lambda(pb->alpha, 1) * P[1]);
  }
  if (cache_alpha != pb->alpha) { frac_sin_coef(a, s); cache_alpha = pb->alpha; }
  orc_jacobi_aa(39, a, x, P);
  double acc = 0.0;
  for (int n = 0; n < 40; ++n) acc += s[n] * orc_frac_lambda(pb->alpha, n) * P[n];
  return acc * exp(cos(t)) / (1.0 + t * t);
}

/* The exact solutions with non-zero boundary values, with their derivatives:
 * u, d_t u and the second derivatives d^2 u / d x_e^2 (e < d) at (x, t).
 *   4: u = e^{-beta t} prod cos(pi (x_e - 0.3) / 3)   (different non-zero values on opposite faces)
 *   5: u = e^{-beta t} prod sin(pi x_e) + t / 2     (u(., 0) = 0 on the boundary, g = t / 2)  */
static void exact_parts(const orc_problem* pb, const double* x, double t, double* u, double* ut, double* uxx) {
  int d = pb->dim;
  double T = exp(-pb->ex_beta * t), prod = 1.0;
  if (pb->ex_kind == 4) {
    for (int e = 0; e < d; ++e) prod *= cos(ORC_PI * (x[e] - 0.3) / 3.0);
    *u = T * prod;
    *ut = -pb->ex_beta * T * prod;
    for (int e = 0; e < d; ++e) uxx[e] = -(ORC_PI * ORC_PI / 9.0) * T * prod;
    return;
  }
  for (int e = 0; e < d; ++e) prod *= sin(ORC_PI * x[e]);
  *u = T * prod + 0.5 * t;
  *ut = -pb->ex_beta * T * prod + 0.5;
  for (int e = 0; e < d; ++e) uxx[e] = -(ORC_PI * ORC_PI) * T * prod;
}

/* Source added to f so that the exact solution solves
 * d_t u + kappa (-Delta) u = f(u) + f_add: f_add = d_t u - kappa Delta u - f(u). */
double orc_source(const orc_problem* pb, const double* x, double t) {
  if (pb->ex_kind == 0) return 0.0;
  int d = pb->dim;
  if (pb->ex_kind == 6 || pb->ex_kind == 7) {
    /* d_t u + kappa (-Delta)^{alpha/2} u - f(u) */
    double u = orc_exact(pb, x, t), ut;
    if (pb->ex_kind == 6) ut = u * (-sin(t) - 2.0 * t / (1.0 + t * t));
    else ut = u / (1.0 + t);
    return ut + pb->kappa * frac_op_exact(pb, x[0], t) - orc_f(pb, u);
  }
  if (pb->ex_kind >= 4) {
    double u, ut, uxx[ORC_MAXD], lap = 0.0;
    exact_parts(pb, x, t, &u, &ut, uxx);
    for (int e = 0; e < d; ++e) lap += uxx[e];
    return ut - pb->kappa * lap - orc_f(pb, u);
  }
  double u = orc_exact(pb, x, t);
  double dtu, mlap;
  if (pb->ex_kind == 1) { dtu = -pb->ex_beta * u; mlap = d * ORC_PI * ORC_PI * u; }
  else if (pb->ex_kind == 2) { dtu = -pb->ex_beta * u; mlap = d * 0.25 * ORC_PI * ORC_PI * u; }
  else {
    /* u = T(t) prod g(x_e), g = (1-x^2)(1+x) = 1 + x - x^2 - x^3, -g'' = 2 + 6x */
    double T = 1.0 + t + t * t, g[ORC_MAXD];
    for (int e = 0; e < d; ++e) g[e] = (1.0 - x[e] * x[e]) * (1.0 + x[e]);
    double prod = 1.0;
    for (int e = 0; e < d; ++e) prod *= g[e];
    dtu = (1.0 + 2.0 * t) * prod;
    mlap = 0.0;
    for (int e = 0; e < d; ++e) {
      double term = 2.0 + 6.0 * x[e];
      for (int e2 = 0; e2 < d; ++e2) if (e2 != e) term *= g[e2];
      mlap += term;
    }
    mlap *= T;
  }
  return dtu + pb->kappa * mlap - orc_f(pb, u);
}

/* Homogenisation of non-zero boundary data g (the remark on non-homogeneous
 * boundary conditions in Section 2.3): u = w + G with G a lifting of g, and
 *   d_t w - kappa Delta w = f(w + G) + f_add - (d_t G - kappa Delta G),  w = 0 on the boundary,
 * w(., 0) = u0 - G(., 0).  G is the Gordon-Hall transfinite interpolant of g,
 *   G = sum over non-empty axis sets A of (-1)^(|A|+1) P_A g,
 *   P_A g(x) = sum over s in {-1,1}^A of prod_{e in A} (1 + s_e x_e)/2  g(x with x_e = s_e, e in A),
 * which uses g on the faces only and equals g on the boundary.  Its blending
 * factors are linear in their own axes, so d_t G and Delta G need g_t and the
 * second derivatives of g along the free axes of each face.  The boundary data
 * here is the trace of the exact solution (kinds 4 and 5; zero for kinds 1-3).
 * G, d_t G and Delta G at (x, t); zeros unless bc_kind == 1. */
void orc_lift(const orc_problem* pb, const double* x, double t, double* G, double* Gt, double* lapG) {
  *G = 0.0; *Gt = 0.0; *lapG = 0.0;
  if (pb->bc_kind != 1 || (pb->ex_kind != 4 && pb->ex_kind != 5)) return;
  int d = pb->dim;
  for (int A = 1; A < (1 << d); ++A) {
    int na = 0, idx[ORC_MAXD];
    for (int e = 0; e < d; ++e) if (A & (1 << e)) idx[na++] = e;
    double sgn = (na % 2 == 1) ? 1.0 : -1.0;
    for (int sbits = 0; sbits < (1 << na); ++sbits) {
      double z[ORC_MAXD], wgt = 1.0;
      for (int e = 0; e < d; ++e) z[e] = x[e];
      for (int a = 0; a < na; ++a) {
        double se = (sbits & (1 << a)) ? 1.0 : -1.0;
        z[idx[a]] = se;
        wgt *= 0.5 * (1.0 + se * x[idx[a]]);
      }
      double u, ut, uxx[ORC_MAXD], lapf = 0.0;
      exact_parts(pb, z, t, &u, &ut, uxx);
      for (int e = 0; e < d; ++e) if (!(A & (1 << e))) lapf += uxx[e];
      *G += sgn * wgt * u;
      *Gt += sgn * wgt * ut;
      *lapG += sgn * wgt * lapf;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Reconstruction (Eq. u_N and the Remark on tensor products).                */
/* U[l * S + j]: nodal values, l = 0..Mt time nodes, j spatial linear index   */
/* with x_1 fastest, S = n^d.  cu[q * S + p], ct[q * S + p]: coefficients of  */
/* u* in phi_{p_1}..phi_{p_d} L_q and of d_t u* in the same basis.           */
/* ------------------------------------------------------------------------- */
void orc_reconstruct(const orc_problem* pb, int Mt, double h, const double* U, double* cu, double* ct) {
  int d = pb->dim, n = pb->n_space;
  int64_t S = ipow(n, d);
  double* A = (double*)malloc(sizeof(double) * n * n);
  double* B = (double*)malloc(sizeof(double) * (Mt + 1) * (Mt + 1));
  orc_space_analysis_pb(pb, A);
  orc_time_analysis(pb->time_family, Mt, B);
  int64_t tot = S * (Mt + 1);
  double* cur = (double*)malloc(sizeof(double) * tot);
  double* nxt = (double*)malloc(sizeof(double) * tot);
  /* time axis: cur[q][j] = sum_k b_qk U[k][j] */
  for (int q = 0; q <= Mt; ++q)
    for (int64_t j = 0; j < S; ++j) {
      double acc = 0.0;
      for (int k = 0; k <= Mt; ++k) acc += B[q * (Mt + 1) + k] * U[k * S + j];
      cur[q * S + j] = acc;
    }
  /* each spatial axis e: contract j_e with a_{p_e j_e} */
  for (int e = 0; e < d; ++e) {
    int64_t stride = ipow(n, e);
    for (int q = 0; q <= Mt; ++q)
      for (int64_t idx = 0; idx < S; ++idx) {
        int pe = (int)((idx / stride) % n);
        int64_t base = idx - (int64_t)pe * stride;
        double acc = 0.0;
        for (int je = 0; je < n; ++je) acc += A[pe * n + je] * cur[q * S + base + je * stride];
        nxt[q * S + idx] = acc;
      }
    double* t = cur; cur = nxt; nxt = t;
  }
  memcpy(cu, cur, sizeof(double) * tot);
  /* d/dt: ct_q = (2/h)(2q+1) sum_{l>q, l+q odd} cu_l  (Legendre derivative identity);
   * Chebyshev: ct_q = (2/h)(2/c_q) sum_{l>q, l+q odd} l cu_l, c_0 = 2, else 1 */
  for (int q = 0; q <= Mt; ++q)
    for (int64_t p = 0; p < S; ++p) {
      double acc = 0.0;
      if (pb->basis == 1) {
        for (int l = q + 1; l <= Mt; l += 2) acc += l * cu[l * S + p];
        ct[q * S + p] = (2.0 / h) * (q == 0 ? 1.0 : 2.0) * acc;
      } else {
        for (int l = q + 1; l <= Mt; l += 2) acc += cu[l * S + p];
        ct[q * S + p] = (2.0 / h) * (2.0 * q + 1.0) * acc;
      }
    }
  free(A); free(B); free(cur); free(nxt);
}

/* Values of u*, d_t u* and -Delta u* at (x, xi) by the direct sum over all
 * coefficients (Eq. u_N, with -d^2 phi_p = (p+1)(p+2) P_p^{(1,1)} per axis; in
 * the fractional case (-Delta)^{alpha/2} u* with lam_p = Gamma(alpha+p+1)/p!). */
void orc_eval(const orc_problem* pb, int Mt, const double* cu, const double* ct, const double* x,
              double xi, double* u_out, double* dtu_out, double* mlap_out) {
  int d = pb->dim, n = pb->n_space;
  int64_t S = ipow(n, d);
  double phi[ORC_MAXD][ORC_MAXN + 2], P[ORC_MAXD][ORC_MAXN + 2], L[ORC_MAXN + 2], lam[ORC_MAXN + 2];
  for (int p = 0; p < n; ++p) lam[p] = is_frac(pb) ? orc_frac_lambda(pb->alpha, p) : (p + 1.0) * (p + 2.0);
  for (int e = 0; e < d; ++e) {
    if (pb->basis == 1) {
      /* phi_p = T_p - T_{p+2}; -phi_p'' = T''_{p+2} - T''_p, kept in P with lam = 1 */
      double T[ORC_MAXN + 4], T2[ORC_MAXN + 4];
      orc_cheb(n + 1, x[e], T, T2);
      for (int p = 0; p < n; ++p) { phi[e][p] = T[p] - T[p + 2]; P[e][p] = T2[p + 2] - T2[p]; }
      for (int p = 0; p < n; ++p) lam[p] = 1.0;
    } else if (is_frac(pb)) {
      /* phi_p = (1-x^2)^a P_p^{(a,a)}; (-Delta)^{alpha/2} phi_p = lam_p P_p^{(a,a)} */
      double a = 0.5 * pb->alpha;
      orc_jacobi_aa(n - 1, a, x[e], P[e]);
      double wgt = fabs(x[e]) < 1.0 ? pow(1.0 - x[e] * x[e], a) : 0.0;
      for (int p = 0; p < n; ++p) phi[e][p] = wgt * P[e][p];
    } else {
      orc_jacobi11(n - 1, x[e], P[e]);
      orc_phi(n - 1, x[e], phi[e]);
    }
  }
  if (pb->basis == 1) { double T2[ORC_MAXN + 4]; orc_cheb(Mt, xi, L, T2); }
  else orc_legendre(Mt, xi, L);
  double u = 0.0, dtu = 0.0, mlap = 0.0;
  for (int q = 0; q <= Mt; ++q)
    for (int64_t idx = 0; idx < S; ++idx) {
      int p[ORC_MAXD];
      int64_t r = idx;
      for (int e = 0; e < d; ++e) { p[e] = (int)(r % n); r /= n; }
      double prod = L[q];
      for (int e = 0; e < d; ++e) prod *= phi[e][p[e]];
      double lap = 0.0;
      for (int e = 0; e < d; ++e) {
        double term = L[q] * lam[p[e]] * P[e][p[e]];
        for (int e2 = 0; e2 < d; ++e2) if (e2 != e) term *= phi[e2][p[e2]];
        lap += term;
      }
      u += cu[q * S + idx] * prod;
      dtu += ct[q * S + idx] * prod;
      mlap += cu[q * S + idx] * lap;
    }
  *u_out = u; *dtu_out = dtu; *mlap_out = mlap;
}

/* Residual of the error equation (Eq. ufg_ep1):
 * r = f(u*) + f_add - d_t u* + kappa Delta u*.
 * With lifted boundary data (bc_kind 1) the equation is the one for w:
 * r = f(u* + G) + f_add - d_t G + kappa Delta G - d_t u* + kappa Delta u*.
 * The direct estimator (estimator 1) integrates the right-hand side of the
 * Picard step (Eq. linearized_func) instead: r without -d_t u* + kappa Delta u*. */
double orc_residual(const orc_problem* pb, int Mt, double t0, double h, const double* cu,
                    const double* ct, const double* x, double tau) {
  double xi = (2.0 * tau - t0 - (t0 + h)) / h;
  double u, dtu, mlap;
  orc_eval(pb, Mt, cu, ct, x, xi, &u, &dtu, &mlap);
  double G, Gt, lapG;
  orc_lift(pb, x, tau, &G, &Gt, &lapG);
  double r = orc_f(pb, u + G) + orc_source(pb, x, tau) - Gt + pb->kappa * lapG;
  if (pb->estimator == 0) r += -dtu - pb->kappa * mlap;
  return r;
}

/* N_* for a time node at s = t_{n,l} - t_{n-1} in an interval of length h. */
int orc_nstar(int n_ref, double s, double h) {
  double v = ceil((double)n_ref * s / h - 1e-9);
  return v < 1.0 ? 1 : (int)v;
}

/* ------------------------------------------------------------------------- */
/* One walk (Lemma Xlocation, Eqs. indexL and interIQ), as the list of its    */
/* quadrature terms: Q = sum_i w_i r(Y_i, tau_i).                             */
/* ------------------------------------------------------------------------- */
typedef struct {
  int Mt; double t0, h; const double* cu; const double* ct;
  int interval, iteration;
} orc_interval_ctx;

/* The quadrature points of one walk: for term i, the point pts[i*d..], the
 * time taus[i] and the weight wts[i] (at most cap terms).  Returns L. */
/* Regularised incomplete beta function I_x(p, q) from its hypergeometric form
 * I_x(p,q) = x^p (1-x)^q / (p B(p,q)) F(p+q, 1; p+1; x), summed for x <= 1/2,
 * with I_x(p,q) = 1 - I_{1-x}(q,p) above. */
double orc_ibeta(double x, double p, double q) {
  if (!(x > 0.0)) return 0.0;
  if (!(x < 1.0)) return 1.0;
  if (x > 0.5) return 1.0 - orc_ibeta(1.0 - x, q, p);
  double pre = exp(p * log(x) + q * log1p(-x) - (lgamma(p) + lgamma(q) - lgamma(p + q))) / p;
  double term = 1.0, sum = 1.0;
  for (int k = 0; k < 4000; ++k) {
    term *= (p + q + k) / (p + 1.0 + k) * x;
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return pre * sum;
}

/* Its inverse in x by bisection (I_x is increasing in x). */
double orc_ibeta_inv(double w, double p, double q) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 100; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_ibeta(mid, p, q) < w) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Jump length of the alpha-stable process out of a ball of radius r around
 * its centre (d = 1), from the uniform omega: the exit point lies at distance
 * r / sqrt(U), U ~ Beta(alpha/2, 1 - alpha/2) (the Blumenthal-Getoor-Ray exit
 * law).  Section 4, Ex. 2 writes U = 1 - X, X = I^{-1}_omega(1 - alpha/2, alpha/2);
 * the same number is U = I^{-1}_{1-omega}(alpha/2, 1 - alpha/2), computed so to
 * avoid the cancellation in 1 - X for omega near 1. */
double orc_stable_jump(double r, double alpha, double omega) {
  double a = 0.5 * alpha;
  double U = orc_ibeta_inv(1.0 - omega, a, 1.0 - a);
  return r / sqrt(U);
}

int orc_walk_points_end(const orc_problem* pb, const orc_interval_ctx* ic, uint32_t node_lin, uint32_t sample,
                        const double* x_start, double t_node, int nstar, double* pts, double* taus, double* wts,
                        int cap, double* x_end, int* end_kind, double* t_end) {
  int d = pb->dim;
  orc_stream st;
  stream_init(&st, pb->seed, sample, node_lin, pb->instance, ic->interval, ic->iteration);
  double s = t_node - ic->t0;
  double delta = s / nstar;
  double J = sqrt(2.0 * d * pb->kappa * delta);
  double X[ORC_MAXD], Xn[ORC_MAXD], theta[ORC_MAXD];
  for (int e = 0; e < d; ++e) X[e] = x_start[e];
  int L = 0;
  if (pb->walk_mode == 2) {
    /* The alpha-stable walk (Section 4, Ex. 2, d = 1): steps of time Delta, each
     * the exit from the ball of radius r = (kappa Delta Gamma(1+alpha))^{1/alpha}
     * around X_q (its mean exit time C r^alpha / kappa is Delta, C = 1/Gamma(1+alpha));
     * the jump J_q = r / sqrt(1 - I^{-1}_omega(1-alpha/2, alpha/2)) in direction
     * theta_q = +-1.  Words 2q (direction, top bit) and 2q+1 (omega).  As in the
     * fixed-radius walk, the walk ends at the first point outside Omega and the
     * term q (the residual at X_q, time t_node - q Delta, weight Delta) counts
     * when X_{q+1} is inside. */
    double r = pow(pb->kappa * delta * exp(lgamma(1.0 + pb->alpha)), 1.0 / pb->alpha);
    for (int q = 0; q < nstar && q < pb->max_steps; ++q) {
      uint32_t wd = stream_word(&st, 2 * (int64_t)q), wo = stream_word(&st, 2 * (int64_t)q + 1);
      double th = (wd >> 31) ? -1.0 : 1.0;
      double J = orc_stable_jump(r, pb->alpha, orc_u01_word(wo));
      double Xn = X[0] + J * th;
      if (!(Xn > -1.0 && Xn < 1.0)) break;
      if (L < cap) {
        pts[L] = X[0];
        taus[L] = t_node - q * delta;
        wts[L] = delta;
      }
      L = q + 1;
      X[0] = Xn;
    }
    if (x_end) x_end[0] = X[0];
    if (end_kind) *end_kind = 0;
    return L;
  }
  if (pb->walk_mode == 1) {
    /* Fixed radius J; the walk ends at the first step centre outside Omega
     * (Eq. indexL); the term q counts when X_{q+1} is still inside. */
    for (int q = 0; q < nstar; ++q) {
      draw_direction(&st, d, q, theta);
      int inside = 1;
      for (int e = 0; e < d; ++e) {
        Xn[e] = X[e] + J * theta[e];
        if (!(Xn[e] > -1.0 && Xn[e] < 1.0)) inside = 0;
      }
      if (!inside) break;
      if (L < cap) {
        for (int e = 0; e < d; ++e) pts[L * d + e] = X[e];
        taus[L] = t_node - q * delta;
        wts[L] = delta;
      }
      L = q + 1;
      for (int e = 0; e < d; ++e) X[e] = Xn[e];
    }
    if (x_end) for (int e = 0; e < d; ++e) x_end[e] = X[e];
    return L;
  }
  /* Balls inside Omega (walk-on-spheres).  The ball around X_q has radius
   * r_q = min(J, dist(X_q, boundary)), so it lies in Omega, and weight w_q equal
   * to its mean exit time: Delta for a full ball, r_q^2/(2 d kappa) for a shrunk
   * one, cut to the time left.  The per-step integral of the residual is
   * estimated at one point Y_q of the ball drawn from its Green function G_r
   * (the per-step representation W E_{Q_r}[f(Y, t_q)] of the error analysis)
   * and at one of n_sub sub-step midpoints of the step, drawn uniformly: path
   * time runs on the grid tau_m = t_{n,l} - (m + 1/2) delta, delta = Delta/n_sub.
   * The clock is (k sub-steps done, fraction f of the next): a full ball
   * advances k by n_sub; a shrunk ball is evaluated at the sub-step it sits in
   * and advances f.  The walk is absorbed once dist < shell and ends when the
   * time s is used up.  Q = sum_q w_q r(Y_q, tau_{m_q}). */
  int64_t W = orc_ball_words_per_step(d);
  int G = pb->n_sub;
  int gbits = 0;
  while ((1 << gbits) < G) ++gbits;
  int64_t Ktot = (int64_t)G * nstar;
  double sub = delta / G;
  double shell = pb->shell;
  if (!(shell > 0.0)) {
    /* half the distance of the outermost JG(1,1) node to the boundary, at most 2e-3 */
    double xs[ORC_MAXN], ws[ORC_MAXN];
    orc_space_nodes(pb, xs, ws);
    shell = 0.5 * (1.0 - fabs(xs[0]));
    if (shell > 2e-3) shell = 2e-3;
  }
  int64_t k = 0;
  double f = 0.0;
  int ended = 0;   /* 1: the time ran out (survived), 2: absorbed at the boundary */
  for (int q = 0; q < pb->max_steps; ++q) {
    double dist = 1.0;
    int near = 0;
    for (int e = 0; e < d; ++e) {
      double de = 1.0 - fabs(X[e]);
      if (de < dist) { dist = de; near = e; }
    }
    if (dist < shell) {
      /* absorbed: for the direct estimator, the boundary point is the walk's
       * position moved onto its nearest face, at the path time reached so far */
      ended = 2;
      if (t_end) *t_end = t_node - ((double)k * sub + f);
      if (pb->estimator == 1) X[near] = X[near] < 0.0 ? -1.0 : 1.0;
      break;
    }
    int64_t w0 = (int64_t)q * W;
    uint32_t gword = stream_word(&st, w0 + ball_gword_index(d));
    int g = gbits ? (int)(gword >> (32 - gbits)) : 0;
    double left = (double)(Ktot - k) * sub - f;
    double w;
    int64_t m;
    int last = 0;
    double r;
    if (J <= dist) {
      r = J;
      w = delta;
      if (k + G >= Ktot) {
        /* the last (possibly partial) full step: the sub-points still ahead */
        int64_t ahead = Ktot - k;
        m = k + (gbits ? (int64_t)(((uint64_t)gword * (uint64_t)ahead) >> 32) : 0);
        w = left;
        last = 1;
      } else {
        m = k + g;
        k += G;
      }
    } else {
      r = dist;
      w = (r * r) / (2.0 * d * pb->kappa);
      m = k;
      if (w >= left) { w = left; last = 1; }
      else {
        f += w;
        while (f >= sub) { f -= sub; ++k; }
        if (k >= Ktot) last = 1;
      }
    }
    double thg[ORC_MAXD], Y[ORC_MAXD];
    direction_at(&st, d, w0 + ball_gdir_index(d), thg);
    int64_t wr = w0 + ball_radius_index(d);
    double U1 = (d <= 2) ? orc_u01_word(stream_word(&st, wr)) : orc_u01_pair(stream_word(&st, wr), stream_word(&st, wr + 1));
    double U2 = (d == 2) ? orc_u01_word(stream_word(&st, wr + 1)) : 0.0;
    double v = orc_green_radius(d, U1, U2);
    for (int e = 0; e < d; ++e) Y[e] = X[e] + r * v * thg[e];
    double tau = t_node - ((double)m + 0.5) * sub;
    /* A shrunk ball's term (weight w < Delta) is evaluated with probability
     * w/Delta and then weighted Delta (unbiased Russian roulette): most of the
     * many small steps that approach the boundary cost no evaluation. */
    double wq = w;
    if (r < J && w > 0.0) {
      uint32_t rword = stream_word(&st, w0 + ball_rword_index(d));
      double Ur = ((double)(rword >> 8) + 0.5) * (1.0 / 16777216.0);
      double pi = w / delta;
      wq = (Ur < pi) ? delta : 0.0;
    }
    if (L < cap) {
      for (int e = 0; e < d; ++e) pts[L * d + e] = Y[e];
      taus[L] = tau;
      wts[L] = wq;
    }
    L = q + 1;
    if (last) {
      ended = 1;
      if (pb->estimator == 1) {
        /* the direct estimator needs the position at t_{n-1}: the last step moves
         * by sqrt(2 d kappa w) for the time w it took (Lemma Xlocation's increment;
         * at most the ball's radius, so X stays in Omega), in the step's own
         * direction words.  Earlier steps move by r = sqrt(2 d kappa w) as well. */
        direction_at(&st, d, w0, theta);
        double rl = sqrt(2.0 * d * pb->kappa * w);
        for (int e = 0; e < d; ++e) X[e] = X[e] + rl * theta[e];
      }
      if (t_end) *t_end = ic->t0;
      break;
    }
    direction_at(&st, d, w0, theta);
    for (int e = 0; e < d; ++e) X[e] = X[e] + r * theta[e];
  }
  if (x_end) for (int e = 0; e < d; ++e) x_end[e] = X[e];
  if (end_kind) *end_kind = ended;
  return L;
}

int orc_walk_points(const orc_problem* pb, const orc_interval_ctx* ic, uint32_t node_lin, uint32_t sample,
                    const double* x_start, double t_node, int nstar, double* pts, double* taus, double* wts,
                    int cap, double* x_end) {
  return orc_walk_points_end(pb, ic, node_lin, sample, x_start, t_node, nstar, pts, taus, wts, cap, x_end, NULL,
                             NULL);
}

#define ORC_WALK_CAP 8192

/* One walk's Q = sum_i w_i r(Y_i, tau_i) (integrand 1 when ic->cu == NULL). */
double orc_walk(const orc_problem* pb, const orc_interval_ctx* ic, uint32_t node_lin, uint32_t sample,
                const double* x_start, double t_node, int nstar, int* L_out, double* x_end) {
  int d = pb->dim;
  double* pts = (double*)malloc(sizeof(double) * ORC_WALK_CAP * d);
  double* taus = (double*)malloc(sizeof(double) * ORC_WALK_CAP);
  double* wts = (double*)malloc(sizeof(double) * ORC_WALK_CAP);
  double xe[ORC_MAXD], te = 0.0;
  int kind = 0;
  int L = orc_walk_points_end(pb, ic, node_lin, sample, x_start, t_node, nstar, pts, taus, wts, ORC_WALK_CAP, xe,
                              &kind, &te);
  double sum = 0.0;
  for (int i = 0; i < L && i < ORC_WALK_CAP; ++i) {
    if (wts[i] == 0.0) continue;
    double r = ic->cu ? orc_residual(pb, ic->Mt, ic->t0, ic->h, ic->cu, ic->ct, pts + i * d, taus[i]) : 1.0;
    sum += wts[i] * r;
  }
  if (pb->estimator == 1 && ic->cu) {
    /* Eq. Phi_ast: u*^{n-1}(X, t_{n-1}) for a walk that reached t_{n-1} (the
     * interval's expansion at xi = -1 is the interpolant of the hand-off row),
     * g(X, t) where it was absorbed (raw boundary data; zero once homogenised) */
    if (kind == 1) {
      double u, dtu, mlap;
      orc_eval(pb, ic->Mt, ic->cu, ic->ct, xe, -1.0, &u, &dtu, &mlap);
      sum += u;
    } else if (kind == 2 && pb->bc_kind == 2) {
      sum += orc_exact(pb, xe, te);
    }
  }
  if (x_end) for (int e = 0; e < d; ++e) x_end[e] = xe[e];
  free(pts); free(taus); free(wts);
  if (L_out) *L_out = L;
  return sum;
}

/* Spatial node coordinates of linear index j. */
static void node_coords(int d, int n, const double* xs, int64_t j, double* x) {
  for (int e = 0; e < d; ++e) { x[e] = xs[j % n]; j /= n; }
}

/* eps at one node (Eq. varepsilon_1): Neumaier-compensated sum of Q_L over the
 * samples in order, divided by M.  For the direct estimator: the mean of S_i
 * (Eq. Phi_ast); the iteration subtracts the node's current value. */
double orc_node_eps(const orc_problem* pb, const orc_interval_ctx* ic, int64_t j, int l) {
  int d = pb->dim, n = pb->n_space;
  double xs[ORC_MAXN], ws[ORC_MAXN], xi[ORC_MAXN + 1], wt[ORC_MAXN + 1], x[ORC_MAXD];
  orc_space_nodes(pb, xs, ws);
  orc_time_nodes(pb->time_family, ic->Mt, xi, wt);
  node_coords(d, n, xs, j, x);
  double s = (xi[l] + 1.0) * 0.5 * ic->h;
  double t_node = ic->t0 + s;
  int nstar = orc_nstar(pb->n_ref, s, ic->h);
  int64_t S = ipow(n, d);
  uint32_t node_lin = (uint32_t)(l * S + j);
  double sum = 0.0, comp = 0.0;
  for (int64_t i = 0; i < pb->M; ++i) {
    double Q = orc_walk(pb, ic, node_lin, (uint32_t)i, x, t_node, nstar, NULL, NULL);
    double t = sum + Q;
    if (fabs(sum) >= fabs(Q)) comp += (sum - t) + Q; else comp += (Q - t) + sum;
    sum = t;
  }
  return (sum + comp) / (double)pb->M;
}

/* ------------------------------------------------------------------------- */
/* Residual iterations on one interval (Algorithm 1, Steps 1-3).             */
/* U is updated in place; eps_out (optional) receives eps for every node.    */
/* Returns the number of iterations run; max_eps[k] per iteration.           */
/* ------------------------------------------------------------------------- */
int orc_iterate(const orc_problem* pb, int interval, double t0, double t1, int Mt, double* U,
                int first_iteration, int n_iter, double tol, double* max_eps, double* eps_out) {
  int d = pb->dim, n = pb->n_space;
  int64_t S = ipow(n, d);
  double h = t1 - t0;
  double* cu = (double*)malloc(sizeof(double) * S * (Mt + 1));
  double* ct = (double*)malloc(sizeof(double) * S * (Mt + 1));
  double* eps = (double*)malloc(sizeof(double) * S * (Mt + 1));
  int done = 0;
  for (int k = 0; k < n_iter; ++k) {
    orc_reconstruct(pb, Mt, h, U, cu, ct);
    orc_interval_ctx ic = {Mt, t0, h, cu, ct, interval, first_iteration + k};
    int64_t nn = S * Mt;
#ifdef _OPENMP
    int nt = pb->n_threads > 0 ? pb->n_threads : 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t a = 0; a < nn; ++a) {
      int l = 1 + (int)(a / S);
      int64_t j = a % S;
      eps[l * S + j] = orc_node_eps(pb, &ic, j, l);
      if (pb->estimator == 1) eps[l * S + j] -= U[l * S + j];
    }
    double mx = 0.0;
    for (int l = 1; l <= Mt; ++l)
      for (int64_t j = 0; j < S; ++j) {
        U[l * S + j] += eps[l * S + j];
        if (fabs(eps[l * S + j]) > mx) mx = fabs(eps[l * S + j]);
      }
    if (max_eps) max_eps[k] = mx;
    if (eps_out) {
      for (int64_t j = 0; j < S; ++j) eps_out[j] = 0.0;
      memcpy(eps_out + S, eps + S, sizeof(double) * S * Mt);
    }
    ++done;
    if (tol > 0.0 && mx < tol) break;
  }
  free(cu); free(ct); free(eps);
  return done;
}

/* ------------------------------------------------------------------------- */
/* Aitken acceleration (the Remark after Algorithm 1: Aitken-weighted Picard  */
/* iteration).  The paper gives no formula; this follows Aitken's dynamic     */
/* relaxation of a fixed-point iteration U <- G(U) with residual r = G(U) - U */
/* (here r = eps): U_{k+1} = U_k + omega_k r_k, omega_1 = 1 and               */
/*   omega_k = -omega_{k-1} <r_{k-1}, r_k - r_{k-1}> / |r_k - r_{k-1}|^2,      */
/* the secant estimate of the iteration's contraction along the last step,   */
/* kept in [1/2, 2]: once r_k is Monte Carlo noise, successive residuals are  */
/* uncorrelated and the unbounded factor would halve at every step.          */
/* ------------------------------------------------------------------------- */
double orc_aitken_omega(int64_t n, const double* r_prev, const double* r_cur, double omega_prev) {
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double dr = r_cur[i] - r_prev[i];
    num += r_prev[i] * dr;
    den += dr * dr;
  }
  if (!(den > 0.0)) return omega_prev;
  double w = -omega_prev * num / den;
  if (w < 0.5) w = 0.5;
  if (w > 2.0) w = 2.0;
  return w;
}

/* orc_iterate with Aitken relaxation.  eps_prev (Mt S values, rows l >= 1) and
 * *omega carry the previous iteration's residual and factor between calls;
 * first_iteration == 1 starts a fresh sequence (omega = 1).  max_eps[k] is
 * the largest |eps| (the residual), not the applied step. */
int orc_iterate_aitken(const orc_problem* pb, int interval, double t0, double t1, int Mt, double* U,
                       int first_iteration, int n_iter, double* eps_prev, double* omega, double* max_eps) {
  int d = pb->dim, n = pb->n_space;
  int64_t S = ipow(n, d);
  double h = t1 - t0;
  int64_t nn = S * Mt;
  double* cu = (double*)malloc(sizeof(double) * S * (Mt + 1));
  double* ct = (double*)malloc(sizeof(double) * S * (Mt + 1));
  double* eps = (double*)malloc(sizeof(double) * nn);
  for (int k = 0; k < n_iter; ++k) {
    int it = first_iteration + k;
    orc_reconstruct(pb, Mt, h, U, cu, ct);
    orc_interval_ctx ic = {Mt, t0, h, cu, ct, interval, it};
#ifdef _OPENMP
    int nt = pb->n_threads > 0 ? pb->n_threads : 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t a = 0; a < nn; ++a) {
      eps[a] = orc_node_eps(pb, &ic, a % S, 1 + (int)(a / S));
      if (pb->estimator == 1) eps[a] -= U[S + a];
    }
    double w = (it == 1) ? 1.0 : orc_aitken_omega(nn, eps_prev, eps, *omega);
    double mx = 0.0;
    for (int64_t a = 0; a < nn; ++a) {
      U[S + a] += w * eps[a];
      if (fabs(eps[a]) > mx) mx = fabs(eps[a]);
      eps_prev[a] = eps[a];
    }
    *omega = w;
    if (max_eps) max_eps[k] = mx;
  }
  free(cu); free(ct); free(eps);
  return n_iter;
}

/* Value of the interval's expansion at t_n (xi = 1) at every spatial node:
 * u*(x_j, t_n) = sum_q sum_k b_qk U[k][j] L_q(1)  (Algorithm 1, Step 4). */
void orc_handoff(const orc_problem* pb, int Mt, const double* U, double* row) {
  int64_t S = ipow(pb->n_space, pb->dim);
  double* B = (double*)malloc(sizeof(double) * (Mt + 1) * (Mt + 1));
  orc_time_analysis(pb->time_family, Mt, B);
  for (int64_t j = 0; j < S; ++j) {
    double acc = 0.0;
    for (int q = 0; q <= Mt; ++q)
      for (int k = 0; k <= Mt; ++k) acc += B[q * (Mt + 1) + k] * U[k * S + j];
    row[j] = acc;
  }
  free(B);
}

/* hp solve (Algorithm 1): n_int intervals with breaks t[0..n_int] and degrees
 * Mt[0..n_int-1]; u0 holds the initial nodal values (S of them).  U_all
 * receives, interval after interval, the (Mt+1) x S nodal blocks.  iters_out
 * (optional) receives the iteration count per interval. */
void orc_solve(const orc_problem* pb, int n_int, const double* t, const int* Mt, int K, double tol,
               const double* u0, double* U_all, int* iters_out) {
  int64_t S = ipow(pb->n_space, pb->dim);
  double* row = (double*)malloc(sizeof(double) * S);
  memcpy(row, u0, sizeof(double) * S);
  if (pb->bc_kind == 1) {
    /* w(., 0) = u0 - G(., 0) at the nodes */
    double xs[ORC_MAXN], ws[ORC_MAXN], x[ORC_MAXD], G, Gt, lapG;
    orc_space_nodes(pb, xs, ws);
    for (int64_t j = 0; j < S; ++j) {
      node_coords(pb->dim, pb->n_space, xs, j, x);
      orc_lift(pb, x, t[0], &G, &Gt, &lapG);
      row[j] -= G;
    }
  }
  int64_t off = 0;
  for (int m = 0; m < n_int; ++m) {
    double* U = U_all + off;
    for (int l = 0; l <= Mt[m]; ++l) memcpy(U + l * S, row, sizeof(double) * S);
    int it = orc_iterate(pb, m, t[m], t[m + 1], Mt[m], U, 1, K, tol, NULL, NULL);
    if (iters_out) iters_out[m] = it;
    orc_handoff(pb, Mt[m], U, row);
    off += (int64_t)(Mt[m] + 1) * S;
  }
  free(row);
}

/* ------------------------------------------------------------------------- */
/* Forward-mode tangent of the hp solve, for checking gradients.             */
/* Direction: ds (reaction scale) and du0 (nodal tangent of u0).  The walks  */
/* do not depend on the parameters (common random numbers), so the tangent   */
/* of eps is the sample mean of Delta sum r_dot along the same paths, with   */
/* r_dot = f'(u*) u_dot* + (df/ds) ds - d_t u_dot* - kappa (-Delta u_dot*).   */
/* dU_all receives the tangent of U_all (same layout).                        */
/* ------------------------------------------------------------------------- */
static double walk_tangent(const orc_problem* pb, const orc_interval_ctx* ic, const double* cdu,
                           const double* cdt, double ds, uint32_t node_lin, uint32_t sample,
                           const double* x_start, double t_node, int nstar) {
  int d = pb->dim;
  double* pts = (double*)malloc(sizeof(double) * ORC_WALK_CAP * d);
  double* taus = (double*)malloc(sizeof(double) * ORC_WALK_CAP);
  double* wts = (double*)malloc(sizeof(double) * ORC_WALK_CAP);
  int L = orc_walk_points(pb, ic, node_lin, sample, x_start, t_node, nstar, pts, taus, wts, ORC_WALK_CAP, NULL);
  double sum = 0.0;
  for (int i = 0; i < L && i < ORC_WALK_CAP; ++i) {
    if (wts[i] == 0.0) continue;
    double xi = (2.0 * taus[i] - ic->t0 - (ic->t0 + ic->h)) / ic->h;
    double u, dtu, mlap, ud, dtud, mlapd;
    orc_eval(pb, ic->Mt, ic->cu, ic->ct, pts + i * d, xi, &u, &dtu, &mlap);
    orc_eval(pb, ic->Mt, cdu, cdt, pts + i * d, xi, &ud, &dtud, &mlapd);
    /* the source f_add = d_t u_ex - kappa Delta u_ex - f(u_ex) depends on s through f(u_ex) */
    double dsrc = (pb->ex_kind != 0) ? -orc_df_ds(pb, orc_exact(pb, pts + i * d, taus[i])) * ds : 0.0;
    sum += wts[i] * (orc_df(pb, u) * ud + orc_df_ds(pb, u) * ds + dsrc - dtud - pb->kappa * mlapd);
  }
  free(pts); free(taus); free(wts);
  return sum;
}

void orc_solve_tangent(const orc_problem* pb, int n_int, const double* t, const int* Mt, int K,
                       const double* u0, const double* du0, double ds, double* U_all, double* dU_all) {
  int d = pb->dim, n = pb->n_space;
  int64_t S = ipow(n, d);
  double* row = (double*)malloc(sizeof(double) * S);
  double* drow = (double*)malloc(sizeof(double) * S);
  memcpy(row, u0, sizeof(double) * S);
  memcpy(drow, du0, sizeof(double) * S);
  double xs[ORC_MAXN], ws[ORC_MAXN];
  orc_space_nodes(pb, xs, ws);
  int64_t off = 0;
  for (int m = 0; m < n_int; ++m) {
    int M_t = Mt[m];
    double t0 = t[m], h = t[m + 1] - t[m];
    double* U = U_all + off;
    double* dU = dU_all + off;
    for (int l = 0; l <= M_t; ++l) {
      memcpy(U + l * S, row, sizeof(double) * S);
      memcpy(dU + l * S, drow, sizeof(double) * S);
    }
    double* cu = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double* ct = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double* cdu = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double* cdt = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double* eps = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double* deps = (double*)malloc(sizeof(double) * S * (M_t + 1));
    double xi[ORC_MAXN + 1], wt[ORC_MAXN + 1];
    orc_time_nodes(pb->time_family, M_t, xi, wt);
    for (int k = 0; k < K; ++k) {
      orc_reconstruct(pb, M_t, h, U, cu, ct);
      orc_reconstruct(pb, M_t, h, dU, cdu, cdt);
      orc_interval_ctx ic = {M_t, t0, h, cu, ct, m, 1 + k};
      int64_t nn = S * M_t;
#ifdef _OPENMP
      int nt = pb->n_threads > 0 ? pb->n_threads : 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
      for (int64_t a = 0; a < nn; ++a) {
        int l = 1 + (int)(a / S);
        int64_t j = a % S;
        double x[ORC_MAXD];
        node_coords(d, n, xs, j, x);
        double s = (xi[l] + 1.0) * 0.5 * h;
        int nstar = orc_nstar(pb->n_ref, s, h);
        uint32_t node_lin = (uint32_t)(l * S + j);
        double sv = 0.0, sd = 0.0;
        for (int64_t i = 0; i < pb->M; ++i) {
          sv += orc_walk(pb, &ic, node_lin, (uint32_t)i, x, t0 + s, nstar, NULL, NULL);
          sd += walk_tangent(pb, &ic, cdu, cdt, ds, node_lin, (uint32_t)i, x, t0 + s, nstar);
        }
        eps[l * S + j] = sv / (double)pb->M;
        deps[l * S + j] = sd / (double)pb->M;
      }
      for (int l = 1; l <= M_t; ++l)
        for (int64_t j = 0; j < S; ++j) {
          U[l * S + j] += eps[l * S + j];
          dU[l * S + j] += deps[l * S + j];
        }
    }
    orc_handoff(pb, M_t, U, row);
    orc_handoff(pb, M_t, dU, drow);
    free(cu); free(ct); free(cdu); free(cdt); free(eps); free(deps);
    off += (int64_t)(M_t + 1) * S;
  }
  free(row); free(drow);
}
