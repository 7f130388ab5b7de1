// spmc_kernels.cuh -- kernels of one residual iteration (Algorithm 1, Steps 1-3)
// and of the interval hand-off (Step 4), for a batch of instances.
//
//   reconstruct_kernel  Step 1: nodal -> modal (Eq. u_N), FP64
//   slice_kernel        time contraction of the coefficients at every path time
//                       of every node's walk grid, FP64 or FP32
//   sweep_kernel        Step 2: M walks per node, residual quadrature per walk,
//                       per-block FP64 sums of Q (Eqs. interIQ, varepsilon_1)
//   update_kernel       Step 3: eps = sum / M (compensated, FP64), u += eps
//   init/handoff        Step 4 and the first iterate (Remark 2.1)
#pragma once
#include "spmc_device.cuh"

namespace spmc {

// One sampled time node (l >= 1) of one instance in the current interval.
struct TimeNode {
  int inst;
  int ell;
  int nstar;        // N_* of Eq. time division
  int Mt;           // time degree of the interval
  long long slice_base;  // first slice (sub-point m = 0) of this node
  long long u_off;  // offset of the instance's nodal block of this interval
  double t_node, t0, h;
};

// Per active instance in the current interval.
struct InstInterval {
  int inst;
  int Mt;
  long long u_off;     // nodal block (Mt+1) x S
  long long c_off;     // coefficient blocks cu, ct ((Mt+1) x S each)
  long long b_off;     // time analysis matrix (Mt+1)^2
  long long h_off;     // hand-off weights sum_q b_qk (Mt+1)
  long long next_u_off;  // nodal block of the next interval (-1 if none)
  int next_Mt;
  double t0, h;
};

struct SliceInfo {
  double tau;       // path time of the sub-point
  double Tt, dTt;   // exact-solution time factor and its derivative at tau
  int kind;         // 0: a sub-point of the walk grid; the direct estimator's two extra slots
                    // per time node: 1 the initial term at t_{n-1}, 2 the boundary term
};

// ----------------------------------------------------------------- Step 1
// cu = (B_n x A x ... x A) U, ct_q = (2/h)(2q+1) sum_{l>q, l+q odd} cu_l.
// One block per active instance; the nodal block lives in shared memory.
// `abort` (may be null): a failed earlier launch of the same iteration sequence
// set it; every launch of the sequence then returns without work.
template <int D>
__global__ void reconstruct_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ U,
                                   const double* __restrict__ A, const double* __restrict__ Bt,
                                   double* __restrict__ coef, int n, const int* __restrict__ abort) {
  extern __shared__ double sm[];
  if (abort && *abort) return;
  const InstInterval w = ii[blockIdx.x];
  int S = 1;
  for (int e = 0; e < D; ++e) S *= n;
  const int T = w.Mt + 1;
  const int tot = T * S;
  double* a = sm;
  double* b = sm + tot;
  const double* B = Bt + w.b_off;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) a[i] = U[w.u_off + i];
  __syncthreads();
  // time axis
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    int q = i / S, j = i - q * S;
    double acc = 0.0;
    for (int k = 0; k < T; ++k) acc += B[q * T + k] * a[k * S + j];
    b[i] = acc;
  }
  __syncthreads();
  double* src = b;
  double* dst = a;
  int stride = 1;
  for (int e = 0; e < D; ++e) {
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      int q = i / S, idx = i - q * S;
      int pe = (idx / stride) % n;
      int base = q * S + idx - pe * stride;
      double acc = 0.0;
      for (int je = 0; je < n; ++je) acc += A[pe * n + je] * src[base + je * stride];
      dst[i] = acc;
    }
    __syncthreads();
    double* t = src; src = dst; dst = t;
    stride *= n;
  }
  double* cu = coef + w.c_off;
  double* ct = cu + tot;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    int q = i / S, p = i - q * S;
    cu[i] = src[i];
    double acc = 0.0;
    for (int l = q + 1; l < T; l += 2) acc += src[l * S + p];
    ct[i] = (2.0 / w.h) * (2.0 * q + 1.0) * acc;
  }
}

// The Chebyshev basis (the remark on quasi-linear reconstruction after
// Algorithm 1): coefficients from the discrete Chebyshev transform (DCT-I) of
// the values at Chebyshev-Gauss-Lobatto points, per axis.  dct1 returns
// F_k = f_0 + (-1)^k f_N + 2 sum_{0<j<N} f_j cos(pi j k / N), k = 0..N, through
// the FFT of the even extension (length 2N) when N is a power of two, by the
// direct sum otherwise (N <= 40).  cs[m], sn[m] = cos, sin(pi m / N), m < 2N
// (the twiddles of the FFT and the cosines of the direct sum).
__device__ __forceinline__ void dct1(const double* f, double* F, int N, const double* cs, const double* sn) {
  const int L = 2 * N;
  if ((N & (N - 1)) == 0 && N <= 32) {
    double re[64], im[64];
    for (int j = 0; j <= N; ++j) re[j] = f[j];
    for (int j = N + 1; j < L; ++j) re[j] = f[L - j];
    for (int j = 0; j < L; ++j) im[j] = 0.0;
    // bit-reversal permutation
    for (int i = 1, j = 0; i < L; ++i) {
      int bit = L >> 1;
      for (; j & bit; bit >>= 1) j ^= bit;
      j ^= bit;
      if (i < j) { double t = re[i]; re[i] = re[j]; re[j] = t; t = im[i]; im[i] = im[j]; im[j] = t; }
    }
    // radix-2 butterflies, twiddles e^{-2 pi i k / len} = cs[m] - i sn[m], m = k L / len
    for (int len = 2; len <= L; len <<= 1) {
      const int hl = len >> 1, step = L / len;
      for (int k = 0; k < hl; ++k) {
        const double c = cs[k * step], sg = -sn[k * step];
        for (int i = 0; i < L; i += len) {
          const double vr = re[i + k + hl] * c - im[i + k + hl] * sg;
          const double vi = re[i + k + hl] * sg + im[i + k + hl] * c;
          re[i + k + hl] = re[i + k] - vr; im[i + k + hl] = im[i + k] - vi;
          re[i + k] += vr; im[i + k] += vi;
        }
      }
    }
    for (int k = 0; k <= N; ++k) F[k] = re[k];
    return;
  }
  for (int k = 0; k <= N; ++k) {
    double acc = f[0] + ((k & 1) ? -f[N] : f[N]);
    for (int j = 1; j < N; ++j) acc += 2.0 * f[j] * cs[(j * k) % L];
    F[k] = acc;
  }
}

// Reconstruction in the Chebyshev basis, one block per active instance: the
// time axis (CGL points -cos(pi k / M)) gives T_q coefficients
// e_q = (-1)^q F_q / (M c_q) (c_0 = c_M = 2, else 1); each space axis the DCT of
// (0, u_1..u_n, 0) at the n+2 CGL points, a_k = (-1)^k F_k / ((n+1) c_k), turned
// into coefficients of phi_p = T_p - T_{p+2} by c_p = a_p + c_{p-2}.  The time
// derivative by ct_q = (2/h)(2/c_q) sum_{l>q, l+q odd} l cu_l.
template <int D>
__global__ void cheb_reconstruct_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ U,
                                        double* __restrict__ coef, int n, const int* __restrict__ abort) {
  extern __shared__ double sm[];
  if (abort && *abort) return;
  const InstInterval w = ii[blockIdx.x];
  int S = 1;
  for (int e = 0; e < D; ++e) S *= n;
  const int T = w.Mt + 1, M = w.Mt;
  const int tot = T * S;
  double* a = sm;
  double* b = sm + tot;
  __shared__ double tcs[80], tsn[80], xcs[80], xsn[80];   // cos, sin(pi m / M) and (pi m / (n+1))
  const int N = n + 1;
  for (int m = threadIdx.x; m < 2 * M; m += blockDim.x) sincospi((double)m / M, &tsn[m], &tcs[m]);
  for (int m = threadIdx.x; m < 2 * N; m += blockDim.x) sincospi((double)m / N, &xsn[m], &xcs[m]);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) a[i] = U[w.u_off + i];
  __syncthreads();
  double f[41], F[41];
  // time axis: one line per spatial node
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    for (int k = 0; k < T; ++k) f[k] = a[k * S + j];
    dct1(f, F, M, tcs, tsn);
    for (int q = 0; q < T; ++q) b[q * S + j] = ((q & 1) ? -F[q] : F[q]) / (M * ((q == 0 || q == M) ? 2.0 : 1.0));
  }
  __syncthreads();
  double* src = b;
  double* dst = a;
  int stride = 1;
  for (int e = 0; e < D; ++e) {
    // one line per (q, the other indices)
    const int lines = tot / n;
    for (int li = threadIdx.x; li < lines; li += blockDim.x) {
      const int q = li / (S / n), rest = li - q * (S / n);
      const int lo = rest % stride, hi = rest / stride;
      const int base = q * S + hi * stride * n + lo;
      f[0] = 0.0;
      f[N] = 0.0;
      for (int j = 0; j < n; ++j) f[j + 1] = src[base + j * stride];
      dct1(f, F, N, xcs, xsn);
      double cm2 = 0.0, cm1 = 0.0;
      for (int p = 0; p < n; ++p) {
        const double ak = ((p & 1) ? -F[p] : F[p]) / (N * (p == 0 ? 2.0 : 1.0));
        const double cp = ak + cm2;
        dst[base + p * stride] = cp;
        cm2 = cm1;
        cm1 = cp;
      }
    }
    __syncthreads();
    double* t = src; src = dst; dst = t;
    stride *= n;
  }
  double* cu = coef + w.c_off;
  double* ct = cu + tot;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int q = i / S, p = i - q * S;
    cu[i] = src[i];
    double acc = 0.0;
    for (int l = q + 1; l < T; l += 2) acc += l * src[l * S + p];
    ct[i] = (2.0 / w.h) * (q == 0 ? 1.0 : 2.0) * acc;
  }
}

// ----------------------------------------------------------------- slices
// For every node's walk grid tau_m = t_node - (m + t_off) delta / n_sub (t_off =
// 1/2: the sub-step midpoints of the inside-ball walk; 0 with n_sub = 1: the step
// centres t_node - m Delta of the fixed-radius walk):
//   C_m[p] = sum_q cu[q][p] L_q(xi(tau_m)),  H_m[p] = -sum_q ct[q][p] L_q(xi(tau_m)).
// d=2 slices are stored [p_x][p_y] (p_y contiguous).  One block per slice.
// Slice layout: C then H, each n rows (d = 2) or one row (d = 1) of `row`
// entries (row >= n, zero padded), slices `sl_stride` entries apart.
template <int D, typename R>
__global__ void slice_kernel(const TimeNode* __restrict__ tn, const long long* __restrict__ slice_node,
                             const InstInterval* __restrict__ inst_of_node, const double* __restrict__ coef,
                             const InstanceParams* __restrict__ ip, R* __restrict__ slices,
                             SliceInfo* __restrict__ sinfo, int n, int n_sub, int row, long long sl_stride,
                             double t_off, const int* __restrict__ abort, int cheb = 0) {
  __shared__ double L[41];
  if (abort && *abort) return;
  long long s = blockIdx.x;
  long long ti = slice_node[s];
  const TimeNode node = tn[ti];
  const InstInterval w = inst_of_node[ti];
  int m = (int)(s - node.slice_base);
  int S = 1;
  for (int e = 0; e < D; ++e) S *= n;
  const double sdur = __dsub_rn(node.t_node, node.t0);
  const double delta = __ddiv_rn(sdur, (double)node.nstar);
  const double sub = __ddiv_rn(delta, (double)n_sub);
  const int Ktot = n_sub * node.nstar;
  // the direct estimator's slots after the walk grid: the expansion at t_{n-1}
  const int kind = m < Ktot ? 0 : 1 + (m - Ktot);
  const double tau = kind ? node.t0 : __dsub_rn(node.t_node, __dmul_rn((double)m + t_off, sub));
  if (threadIdx.x == 0) {
    double xi = (2.0 * tau - node.t0 - (node.t0 + node.h)) / node.h;
    L[0] = 1.0;
    if (node.Mt >= 1) L[1] = xi;
    // Legendre L_q, or Chebyshev T_q for the Chebyshev basis
    for (int k = 1; k < node.Mt; ++k)
      L[k + 1] = cheb ? 2.0 * xi * L[k] - L[k - 1] : ((2.0 * k + 1.0) * xi * L[k] - k * L[k - 1]) / (k + 1.0);
    const InstanceParams P = ip[node.inst];
    SliceInfo si;
    si.tau = tau;
    si.kind = kind;
    if (P.ex_kind == 3) { si.Tt = 1.0 + tau + tau * tau; si.dTt = 1.0 + 2.0 * tau; }
    else if (P.ex_kind == 6) {   // e^{cos t} / (1 + t^2)
      si.Tt = exp(cos(tau)) / (1.0 + tau * tau);
      si.dTt = si.Tt * (-sin(tau) - 2.0 * tau / (1.0 + tau * tau));
    } else if (P.ex_kind == 7) { si.Tt = 1.0 + tau; si.dTt = 1.0; }
    else if (P.ex_kind >= 1) { si.Tt = exp(-P.ex_beta * tau); si.dTt = -P.ex_beta * si.Tt; }
    else { si.Tt = 0.0; si.dTt = 0.0; }
    sinfo[s] = si;
  }
  __syncthreads();
  const double* cu = coef + w.c_off;
  const double* ct = cu + (long long)(node.Mt + 1) * S;
  R* out = slices + s * sl_stride;
  const int half = (D == 2) ? n * row : row;
  for (int i = threadIdx.x; i < 2 * half; i += blockDim.x) out[i] = R(0);
  __syncthreads();
  for (int p = threadIdx.x; p < S; p += blockDim.x) {
    double c = 0.0, h = 0.0;
    for (int q = 0; q <= node.Mt; ++q) {
      c += cu[q * S + p] * L[q];
      h -= ct[q * S + p] * L[q];
    }
    int dstp = p;
    if (D == 2) { int px = p % n, py = p / n; dstp = px * row + py; }
    out[dstp] = (R)c;
    out[half + dstp] = (R)h;
  }
}

// ----------------------------------------------------------------- Step 2
struct SweepArgs {
  const TimeNode* tn;
  const InstanceParams* ip;
  const double* xnodes;     // JG(1,1) nodes (n)
  const void* slices;       // R[2 S] per slice
  const SliceInfo* sinfo;
  double* partial;          // per (time node, j, chunk) sum of Q
  unsigned long long* counters;  // [0] points evaluated, [1] walks capped
  int* status;
  int n, S, n_chunks, chunk, n_sub, gbits, max_steps;
  long long M;              // samples per node (the last chunk may be partial)
  long long sl_stride;      // entries between consecutive slices (global and shared)
  int half;                 // entries of C (= of H) in a slice
  double kappa, shell;
  uint32_t k0, k1;
  int interval, iteration;
  int walk_mode;            // 0: inside-ball walk; 1: fixed-radius walk with centre points;
                            // 2: the alpha-stable walk of the fractional case (d = 1)
  const double* frac;       // walk_mode 2: the plan's fractional table (kFrac* layout)
  // adjoint sweep only
  const double* lambda;     // adjoint of the nodal values (layout of U)
  double* gT;               // per slice: 3 S accumulators (coefficient order)
  double* gds;              // per instance: derivative in the reaction scale
};

// Per-sample walk state, kept in shared memory (structure of arrays).
template <int D, typename R>
struct WalkState {
  R* X[D];
  R* f;       // fraction of the current sub-step used by shrunk balls
  R* w;       // weight of the pending step
  R* r;       // ball radius of the pending step
  R* S;       // running sum of w r(Y, tau) for the walk
  int* k;     // whole sub-steps used
  int* q;     // step counter
  int* mnext; // sub-point of the pending evaluation; -1 once the walk has ended
  int* last;  // the pending step ends the walk
};

// Prepare step q of sample s (the ball, its weight and its sub-point) as the
// CPU reference does: absorb in the shell, shrink the ball to the distance to
// the boundary, cut the last step to the time left.
//
// walk_mode 1 (the fixed-radius walk of Lemma Xlocation, Eqs. indexL and
// interIQ): step q moves the centre by J theta_q; the term of step q (the
// residual at the centre X_q, time t_node - q Delta, weight Delta) counts only if
// X_{q+1} is still inside Omega, and the walk ends at the first centre outside
// or after N_* steps.  The slices then hold the step-centre times (n_sub = 1).
template <int D, typename R>
__device__ __forceinline__ void prepare_step(const WalkState<D, R>& st, int s, const WalkStream& ws, R J, R delta,
                                             R sub, int Ktot, int G, int gbits, R shell, R kappa, int max_steps,
                                             double& acc, unsigned long long& capped, int walk_mode = 0,
                                             const double* frac = nullptr, double r_stable = 0.0) {
  int q = st.q[s];
  if (walk_mode == 2) {
    // the alpha-stable walk (d = 1): step q jumps out of the ball of radius
    // r_stable around X_q, by J_q = r_stable / sqrt(U_q) in direction +-1 (words
    // 2q and 2q + 1 of one Philox block); the term of step q counts if X_{q+1}
    // is still inside.  st.r holds the signed jump.
    if (q >= max_steps || q >= Ktot) {
      if (q >= max_steps && q < Ktot) ++capped;
      st.mnext[s] = -1;
      return;
    }
    const Philox4 b = ws.block((uint32_t)q >> 1);
    const uint32_t wd = b.v[(2 * q) & 3], wo = b.v[(2 * q + 1) & 3];
    const double omega = U01<double>::one(wo);
    const double Jq = (double)stable_jump<R, double>((R)r_stable, (R)frac[kFracAD], (R)frac[kFracLnBD],
                                                     frac + kFracRpD, frac + kFracRqD, omega);
    const double step = (wd >> 31) ? -Jq : Jq;
    const double xn = (double)st.X[0][s] + step;
    if (!(xn > -1.0 && xn < 1.0)) { st.mnext[s] = -1; return; }
    st.w[s] = delta;
    st.r[s] = (R)step;
    st.mnext[s] = q;
    st.last[s] = (q + 1 >= Ktot) ? 1 : 0;
    return;
  }
  if (walk_mode == 1) {
    if (q >= max_steps || q >= Ktot) {
      if (q >= max_steps && q < Ktot) ++capped;
      st.mnext[s] = -1;
      return;
    }
    R th[D];
    literal_direction<D, R>(ws, q, th);
    bool inside = true;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      const R xn = Ar<R>::add(st.X[e][s], Ar<R>::mul(J, th[e]));
      if (!(xn > R(-1) && xn < R(1))) inside = false;
    }
    if (!inside) { st.mnext[s] = -1; return; }
    st.w[s] = delta;
    st.r[s] = J;
    st.mnext[s] = q;
    st.last[s] = (q + 1 >= Ktot) ? 1 : 0;
    return;
  }
  R dist = R(1);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    R de = Ar<R>::sub(R(1), fabs(st.X[e][s]));
    if (de < dist) dist = de;
  }
  if (q >= max_steps || dist < shell) {
    if (q >= max_steps) ++capped;
    st.mnext[s] = -1;   // the walk's Q stays in st.S[s]
    return;
  }
  constexpr int W = step_words(D);
  uint32_t gword = stream_word(ws, (uint32_t)q * W + gword_index(D));
  int g = gbits ? (int)(gword >> (32 - gbits)) : 0;
  int k = st.k[s];
  R f = st.f[s];
  R left = Ar<R>::sub(Ar<R>::mul((R)(Ktot - k), sub), f);
  R w, r;
  int m, last = 0;
  if (J <= dist) {
    r = J;
    w = delta;
    if (k + G >= Ktot) {
      int ahead = Ktot - k;
      m = k + (gbits ? (int)(((unsigned long long)gword * (unsigned long long)ahead) >> 32) : 0);
      w = left;
      last = 1;
    } else {
      m = k + g;
      k += G;
    }
  } else {
    r = dist;
    const R two_dk = Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa);
    w = Ar<R>::divr(Ar<R>::mul(r, r), two_dk, Ar<R>::div(R(1), two_dk));
    m = k;
    if (w >= left) { w = left; last = 1; }
    else {
      f = Ar<R>::add(f, w);
      while (f >= sub) { f = Ar<R>::sub(f, sub); ++k; }
      if (k >= Ktot) last = 1;
    }
  }
  st.k[s] = k;
  st.f[s] = f;
  st.w[s] = w;
  st.r[s] = r;
  st.mnext[s] = m;
  st.last[s] = last;
}

// Persistent sweep.  A cohort is a tile of JT spatial nodes of one sampled time
// node times one chunk of CC samples per node: W = JT CC walks that share the
// time node's slices.  Each block takes cohorts from a global counter and runs
// them pass by pass: a pass handles the window of n_sub sub-points
// [m0, m0 + n_sub) whose slices are staged in shared memory; every walk whose
// pending evaluation lies in the window is evaluated and keeps stepping while
// its next evaluation stays in the window.  Walk state lives in a block-private
// global region (L2 resident); the pending sub-points and the active and ready
// lists live in shared memory.  When every walk of the cohort has ended, the
// block sums each node's walks in sample order (FP64) into the node's chunk sum.
template <int D, typename R>
struct StateRegion {
  // block-private global arrays of W entries each
  R* X[D];
  R *f, *w, *r, *S;
  int *k, *q, *last;
};

template <int D, int NMAX, typename R, bool ADJ = false>
__global__ void __launch_bounds__(256, (sizeof(R) == 4) ? 2 : 1)
sweep_kernel(SweepArgs a, int JT, int CC, long long n_cohorts, int* __restrict__ work_counter,
             void* __restrict__ state_base, long long state_stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int S = a.S, n = a.n;
  const int G = a.n_sub;
  const long long slst = a.sl_stride;
  const int half = a.half;
  const int W = JT * CC;
  const int n_jt = (S + JT - 1) / JT;
  R* sSl = reinterpret_cast<R*>(smraw);                       // [G][slst]
  unsigned char* p = smraw + ((G * slst * sizeof(R) + 15) / 16) * 16;
  int* mnext = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* act = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* ready = reinterpret_cast<int*>(p); p += W * sizeof(int);
  double* sAcc = reinterpret_cast<double*>(p);   // adjoint: [G][3][S] accumulators of the window
  __shared__ int red[64];
  __shared__ double dred[32];
  __shared__ int s_next, s_nact;
  __shared__ double s_Tt[16], s_dTt[16];

  // block-private walk state (structure of arrays)
  unsigned char* gb = reinterpret_cast<unsigned char*>(state_base) + (long long)blockIdx.x * state_stride;
  WalkState<D, R> st;
#pragma unroll
  for (int e = 0; e < D; ++e) { st.X[e] = reinterpret_cast<R*>(gb); gb += W * sizeof(R); }
  st.f = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.w = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.r = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.S = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.k = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.q = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.last = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.mnext = mnext;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const R kappa = (R)a.kappa;
  const R shell = (R)a.shell;
  const R* slices = reinterpret_cast<const R*>(a.slices);
  unsigned long long capped = 0, points = 0;
  double dummy_acc = 0.0;
  double ds_acc = 0.0;   // adjoint: derivative in the reaction scale (this thread's terms)

  // block-wide exclusive scan of one count per thread; returns the total
  auto block_scan = [&](int cnt, int& base) -> int {
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int wv = 0; wv < nwarps; ++wv) {
      if (wv < warp) wbase += red[wv];
      total += red[wv];
    }
    __syncthreads();
    base = wbase + incl - cnt;
    return total;
  };

  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(work_counter, 1);
    __syncthreads();
    const long long id = s_next;
    __syncthreads();
    if (id >= n_cohorts) break;
    long long b = id;
    const int chunk = (int)(b % a.n_chunks);
    b /= a.n_chunks;
    const int jt = (int)(b % n_jt);
    const long long ti = b / n_jt;
    const TimeNode node = a.tn[ti];
    const InstanceParams ip = a.ip[node.inst];
    const int j0 = jt * JT;
    const R sdur = Ar<R>::sub((R)node.t_node, (R)node.t0);
    const R delta = Ar<R>::div(sdur, (R)node.nstar);
    const R J = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), delta));
    const R sub = Ar<R>::div(delta, (R)G);
    const int Ktot = G * node.nstar;
    // the alpha-stable walk's ball radius: its mean exit time r^alpha / (kappa Gamma(1+alpha)) is Delta
    double r_stable = 0.0;
    if (a.walk_mode == 2) {
      const double dd = (node.t_node - node.t0) / (double)node.nstar;
      r_stable = pow(a.kappa * dd * a.frac[kFracGammaD], 1.0 / a.frac[kFracAlphaD]);
    }
    const uint32_t tag = ((uint32_t)(node.inst & 0xfff) << 20) | ((uint32_t)(a.interval & 0x3ff) << 10) |
                         (uint32_t)(a.iteration & 0x3ff);
    const long long sample0 = (long long)chunk * CC;
    WalkStream ws;
    ws.k0 = a.k0; ws.k1 = a.k1; ws.tag = tag;

    // start the cohort's walks
    int cnt = 0;
    for (int wk = threadIdx.x; wk < W; wk += blockDim.x) {
      const int jj = wk / CC, s = wk - jj * CC;
      const int j = j0 + jj;
      st.S[wk] = R(0);
      if (j >= S || sample0 + s >= a.M) { mnext[wk] = -1; continue; }
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { st.X[e][wk] = (R)a.xnodes[jr % n]; jr /= n; }
      st.f[wk] = R(0); st.k[wk] = 0; st.q[wk] = 0;
      ws.node = (uint32_t)(node.ell * S + j);
      ws.sample = (uint32_t)(sample0 + s);
      prepare_step<D, R>(st, wk, ws, J, delta, sub, Ktot, G, a.gbits, shell, kappa, a.max_steps, dummy_acc, capped,
                         a.walk_mode, a.frac, r_stable);
      if (mnext[wk] >= 0) ++cnt;
    }
    __syncthreads();
    {
      int base;
      const int tot = block_scan(cnt, base);
      for (int wk = threadIdx.x; wk < W; wk += blockDim.x)
        if (mnext[wk] >= 0) act[base++] = wk;
      if (threadIdx.x == 0) s_nact = tot;
      __syncthreads();
    }
    int m0 = 0;
    const int max_passes = 2 * Ktot + 8;
    int passes = 0;
    while (s_nact > 0) {
      const int nact = s_nact;
      if (++passes > max_passes) {  // cannot happen for consistent inputs: report and end the walks
        if (threadIdx.x == 0) { atomicOr(a.status, 2); s_nact = 0; }
        for (int i = threadIdx.x; i < nact; i += blockDim.x) mnext[act[i]] = -1;
        __syncthreads();
        break;
      }
      // ready list: active walks pending in the window; smallest pending beyond it
      int rc = 0, mn = 0x7fffffff;
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int mv = mnext[act[i]];
        if (mv < m0 + G) ++rc; else mn = min(mn, mv);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      if (lane == 0) red[32 + warp] = mn;
      int rbase;
      const int nready = block_scan(rc, rbase);
      int gmin = 0x7fffffff;
      for (int wv = 0; wv < nwarps; ++wv) gmin = min(gmin, red[32 + wv]);
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int wk = act[i];
        if (mnext[wk] < m0 + G) ready[rbase++] = wk;
      }
      if (nready == 0) {
        __syncthreads();
        m0 = gmin;
        continue;
      }
      if (ADJ)
        for (int i = threadIdx.x; i < G * 3 * S; i += blockDim.x) sAcc[i] = 0.0;
      // stage the window's slices (16-byte vector copies) and time factors
      {
        const int nsl = min(G, Ktot - m0);
        const R* src = slices + (node.slice_base + m0) * slst;
        const int vec = (int)(16 / sizeof(R));
        const long long nv = (long long)nsl * slst / vec;
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(sSl);
        for (long long i = threadIdx.x; i < nv; i += blockDim.x) d4[i] = s4[i];
        if (threadIdx.x < nsl) {
          SliceInfo si = a.sinfo[node.slice_base + m0 + threadIdx.x];
          s_Tt[threadIdx.x] = si.Tt; s_dTt[threadIdx.x] = si.dTt;
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nready; i += blockDim.x) {
        const int wk = ready[i];
        const int jj = wk / CC;
        ws.node = (uint32_t)(node.ell * S + j0 + jj);
        ws.sample = (uint32_t)(sample0 + (wk - jj * CC));
        int mv = mnext[wk];
        while (mv >= m0 && mv < m0 + G) {
          const int q = st.q[wk];
          constexpr int WS = step_words(D);
          const uint32_t w0 = (uint32_t)q * WS;
          const R r = st.r[wk];
          R Y[D];
          R w = st.w[wk];
          if (a.walk_mode >= 1) {
            // fixed-radius and alpha-stable walks: the residual at the step centre
#pragma unroll
            for (int e = 0; e < D; ++e) Y[e] = st.X[e][wk];
          } else {
            // Green-function point of the pending ball
            R thg[D];
            direction<D, R>(ws, w0 + gdir_index(D), thg);
            R U1, U2;
            green_uniforms<D, R>(ws, w0, U1, U2);
            const R v = green_radius<D, R>(U1, U2);
            const R rv = Ar<R>::mul(r, v);
#pragma unroll
            for (int e = 0; e < D; ++e) Y[e] = Ar<R>::add(st.X[e][wk], Ar<R>::mul(rv, thg[e]));
            // a shrunk ball's term is evaluated with probability w / Delta and
            // then weighted Delta (unbiased Russian roulette)
            if (r < J && w > R(0)) {
              const uint32_t rw = stream_word(ws, w0 + rword_index(D));
              w = roulette_keep<R>(rw, Ar<R>::divr(w, delta, Ar<R>::div(R(1), delta))) ? delta : R(0);
            }
          }
          if (w > R(0)) {
            const int bsl = mv - m0;
            const R* sc = sSl + bsl * slst;
            if (ADJ) {
              const double cw = a.lambda[node.u_off + (long long)node.ell * S + j0 + jj] * (double)w / (double)a.M;
              ds_acc += adjoint_at<D, NMAX, R>(ip, n, sc, Y, cw, sAcc + (long long)bsl * 3 * S, S, (R)s_Tt[bsl]);
            } else {
              R res;
              if (D == 1 && a.walk_mode == 2)
                res = residual_frac<R>(ip, kappa, n, sc, sc + half, Y[0], (R)s_Tt[bsl], (R)s_dTt[bsl], a.frac);
              else
                res = residual_at<D, NMAX, R>(ip, kappa, n, sc, sc + half, Y, (R)s_Tt[bsl], (R)s_dTt[bsl]);
              st.S[wk] += w * res;
            }
            ++points;
          }
          if (st.last[wk]) { mnext[wk] = -1; break; }
          // step to the sphere of the ball (fixed-radius walk: to the next centre)
          R th[D];
          if (a.walk_mode == 2) th[0] = R(1);   // st.r holds the signed jump
          else if (a.walk_mode == 1) literal_direction<D, R>(ws, q, th);
          else direction<D, R>(ws, w0, th);
#pragma unroll
          for (int e = 0; e < D; ++e) st.X[e][wk] = Ar<R>::add(st.X[e][wk], Ar<R>::mul(r, th[e]));
          st.q[wk] = q + 1;
          prepare_step<D, R>(st, wk, ws, J, delta, sub, Ktot, G, a.gbits, shell, kappa, a.max_steps,
                             dummy_acc, capped, a.walk_mode, a.frac, r_stable);
          mv = mnext[wk];
        }
      }
      __syncthreads();
      if (ADJ) {
        const int nsl = min(G, Ktot - m0);
        for (int i = threadIdx.x; i < nsl * 3 * S; i += blockDim.x) {
          const double v = sAcc[i];
          if (v != 0.0) atomicAdd(&a.gT[(node.slice_base + m0) * 3 * S + i], v);
        }
      }
      // compact the active list
      int kc = 0;
      for (int i = threadIdx.x; i < nact; i += blockDim.x) kc += (mnext[act[i]] >= 0);
      int kbase;
      const int nkeep = block_scan(kc, kbase);
      // stable compaction through the ready buffer
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int wk = act[i];
        if (mnext[wk] >= 0) ready[kbase++] = wk;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nkeep; i += blockDim.x) act[i] = ready[i];
      if (threadIdx.x == 0) s_nact = nkeep;
      __syncthreads();
      m0 += G;
    }
    if (ADJ) {
      // derivative in the reaction scale: block sum of this cohort's terms
      double t = ds_acc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) dred[warp] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int wv = 0; wv < nwarps; ++wv) tt += dred[wv];
        if (tt != 0.0) atomicAdd(&a.gds[node.inst], tt);
      }
      __syncthreads();
      ds_acc = 0.0;
      continue;   // no chunk sums in the adjoint sweep
    }
    // every walk of the cohort has ended: each node's chunk sum in sample order
    for (int jj = 0; jj < JT; ++jj) {
      const int j = j0 + jj;
      if (j >= S) break;
      double t = 0.0;
      for (int s = threadIdx.x; s < CC; s += blockDim.x) t += (double)st.S[jj * CC + s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) dred[warp] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int wv = 0; wv < nwarps; ++wv) tt += dred[wv];
        a.partial[(ti * S + j) * a.n_chunks + chunk] = tt;
      }
      __syncthreads();
    }
  }

#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    points += __shfl_xor_sync(0xffffffffu, points, o);
    capped += __shfl_xor_sync(0xffffffffu, capped, o);
  }
  if (lane == 0) {
    if (points) atomicAdd(&a.counters[0], points);
    if (capped) atomicAdd(&a.counters[1], capped);
  }
}

// ----------------------------------------------------------------- Step 3
// eps = (Neumaier sum of the chunk sums, in chunk order) / M;  u += eps.
__global__ void update_kernel(const TimeNode* __restrict__ tn, const double* __restrict__ partial,
                              double* __restrict__ U, double* __restrict__ eps_out,
                              unsigned long long* __restrict__ max_eps_bits, int* status, long long n_nodes,
                              int S, int n_chunks, double inv_M) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  int inst = -1;
  if (i < n_nodes) {
    long long ti = i / S;
    int j = (int)(i - ti * S);
    const TimeNode node = tn[ti];
    inst = node.inst;
    const double* pp = partial + i * n_chunks;
    double sum = 0.0, comp = 0.0;
    for (int c = 0; c < n_chunks; ++c) {
      double x = pp[c];
      double t = sum + x;
      if (fabs(sum) >= fabs(x)) comp += (sum - t) + x; else comp += (x - t) + sum;
      sum = t;
    }
    e = (sum + comp) * inv_M;
    if (!isfinite(e)) atomicOr(status, 1);
    U[node.u_off + (long long)node.ell * S + j] += e;
    if (eps_out) eps_out[i] = e;
    unsigned long long bits = __double_as_longlong(fabs(e));
    atomicMax(&max_eps_bits[inst], bits);
  }
}

// eps = (exact fixed-point sum of the node's terms, rounded once to FP64) / M;
// u += eps.  acc holds four limb counters per (time node, node).
__global__ void update_fixed_kernel(const TimeNode* __restrict__ tn, const unsigned long long* __restrict__ acc,
                                    double* __restrict__ U, double* __restrict__ eps_out,
                                    unsigned long long* __restrict__ max_eps_bits, int* status, long long n_nodes,
                                    int S, double inv_M, int direct, const int* __restrict__ abort) {
  if (abort && *abort) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const long long ti = i / S;
  const int j = (int)(i - ti * S);
  const TimeNode node = tn[ti];
  const long long ui = node.u_off + (long long)node.ell * S + j;
  // residual iteration: eps = mean of Q; direct estimator: eps = mean of S_i - u
  double e = fix_value(acc + 4 * i) * inv_M;
  if (direct) e -= U[ui];
  if (!isfinite(e)) atomicOr(status, 1);
  U[ui] += e;
  if (eps_out) eps_out[i] = e;
  atomicMax(&max_eps_bits[node.inst], (unsigned long long)__double_as_longlong(fabs(e)));
}

// The node-sharded iteration: eps of the pairs i in [lo, hi) from their exact
// sums (no update), and the update of every pair from a gathered eps array.
__global__ void eps_out_kernel(const unsigned long long* __restrict__ acc, double* __restrict__ eps, long long lo,
                               long long hi, double inv_M, int* status, const TimeNode* __restrict__ tn,
                               const double* __restrict__ U, int S, int direct, const int* __restrict__ abort) {
  if (*abort) return;
  const long long i = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  double e = fix_value(acc + 4 * i) * inv_M;
  if (direct) {   // the direct estimator's value minus the node's current value
    const long long ti = i / S;
    const TimeNode node = tn[ti];
    e -= U[node.u_off + (long long)node.ell * S + (i - ti * S)];
  }
  if (!isfinite(e)) atomicOr(status, 1);
  eps[i] = e;
}
__global__ void apply_eps_kernel(const TimeNode* __restrict__ tn, const double* __restrict__ eps,
                                 double* __restrict__ U, unsigned long long* __restrict__ max_eps_bits, int* status,
                                 long long n_nodes, int S) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const long long ti = i / S;
  const int j = (int)(i - ti * S);
  const TimeNode node = tn[ti];
  const double e = eps[i];
  if (!isfinite(e)) atomicOr(status, 1);
  U[node.u_off + (long long)node.ell * S + j] += e;
  atomicMax(&max_eps_bits[node.inst], (unsigned long long)__double_as_longlong(fabs(e)));
}

// eps of every pair from the cohort kernel's chunk sums (Neumaier, chunk order).
__global__ void eps_from_partial_kernel(const double* __restrict__ partial, double* __restrict__ eps,
                                        long long n_pairs, int n_chunks, double inv_M, int* status) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pairs) return;
  const double* pp = partial + i * n_chunks;
  double sum = 0.0, comp = 0.0;
  for (int c = 0; c < n_chunks; ++c) {
    const double x = pp[c], t = sum + x;
    if (fabs(sum) >= fabs(x)) comp += (sum - t) + x; else comp += (x - t) + sum;
    sum = t;
  }
  const double e = (sum + comp) * inv_M;
  if (!isfinite(e)) atomicOr(status, 1);
  eps[i] = e;
}

// Aitken relaxation (the Remark after Algorithm 1), one block per active
// instance over its pairs [first[b], first[b+1]) x S: omega = -omega_prev
// <r_prev, r - r_prev> / |r - r_prev|^2 kept in [1/2, 2] (omega = 1 on an
// interval's first iteration), then u += omega r, r_prev = r.  The dot
// products are summed in a fixed order (per-thread strided sums, then a
// fixed tree), so the factor does not depend on scheduling.
__global__ void aitken_apply_kernel(const InstInterval* __restrict__ ii, const TimeNode* __restrict__ tn,
                                    const long long* __restrict__ first_tn, const double* __restrict__ eps,
                                    double* __restrict__ eps_prev, double* __restrict__ omega, double* __restrict__ U,
                                    unsigned long long* __restrict__ max_eps_bits, int S, int first_iteration,
                                    const int* __restrict__ abort) {
  __shared__ double s_num[256], s_den[256];
  __shared__ double s_w;
  if (abort && *abort) return;
  const int b = blockIdx.x;
  const long long p0 = first_tn[b] * S, p1 = first_tn[b + 1] * S;
  const int inst = ii[b].inst;
  double num = 0.0, den = 0.0;
  if (!first_iteration)
    for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const double dr = eps[p] - eps_prev[p];
      num += eps_prev[p] * dr;
      den += dr * dr;
    }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { s_num[threadIdx.x] += s_num[threadIdx.x + o]; s_den[threadIdx.x] += s_den[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double w = 1.0;
    if (!first_iteration) {
      w = omega[inst];
      if (s_den[0] > 0.0) w = fmin(fmax(-w * s_num[0] / s_den[0], 0.5), 2.0);
    }
    omega[inst] = w;
    s_w = w;
  }
  __syncthreads();
  const double w = s_w;
  double mx = 0.0;
  for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const long long ti = p / S;
    const int j = (int)(p - ti * S);
    const TimeNode node = tn[ti];
    const double e = eps[p];
    U[node.u_off + (long long)node.ell * S + j] += w * e;
    eps_prev[p] = e;
    mx = fmax(mx, fabs(e));
  }
  atomicMax(&max_eps_bits[inst], (unsigned long long)__double_as_longlong(mx));
}

// ----------------------------------------------------------------- Step 4 and first iterate
// row 0 of interval 0 from u0; every other row equal to row 0.
// With lifted boundary data the unknown starts from w(., t_0) = u0 - G(., t_0).
template <int D>
__global__ void init_first_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ u0,
                                  double* __restrict__ U, int S, const InstanceParams* __restrict__ ipt,
                                  const double* __restrict__ xnodes, int n) {
  const InstInterval w = ii[blockIdx.x];
  const InstanceParams ip = ipt[w.inst];
  const int T = w.Mt + 1;
  const double Tt = exp(-ip.ex_beta * w.t0);
  for (int i = threadIdx.x; i < T * S; i += blockDim.x) {
    const int j = i % S;
    double v = u0[(long long)w.inst * S + j];
    if (ip.bc_kind == 1) {
      double y[D], G, Gt, lapG;
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { y[e] = xnodes[jr % n]; jr /= n; }
      lift_bv<D, double>(ip, y, Tt, w.t0, G, Gt, lapG);
      v -= G;
    }
    U[w.u_off + i] = v;
  }
}

// The solution at the nodes of one instance's interval: the nodal values plus
// the lifting G(x_j, t_{n,l}) for lifted boundary data.  `times` holds t_{n,l}.
template <int D>
__global__ void solution_kernel(const double* __restrict__ U, double* __restrict__ out,
                                const InstanceParams* __restrict__ ipt, int inst, const double* __restrict__ times,
                                const double* __restrict__ xnodes, int n, int S, int T) {
  const InstanceParams ip = ipt[inst];
  const long long tot = (long long)T * S;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(i / S), j = (int)(i - (long long)l * S);
    double v = U[i];
    if (ip.bc_kind == 1) {
      double y[D], G, Gt, lapG;
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { y[e] = xnodes[jr % n]; jr /= n; }
      lift_bv<D, double>(ip, y, exp(-ip.ex_beta * times[l]), times[l], G, Gt, lapG);
      v += G;
    }
    out[i] = v;
  }
}

// u*(x_j, t_n) = sum_k hw_k U[k][j] with hw_k = sum_q b_qk L_q(1); the next
// interval starts from it in every row.
__global__ void handoff_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ hw,
                               double* __restrict__ U, int S) {
  const InstInterval w = ii[blockIdx.x];
  if (w.next_u_off < 0) return;
  const int T = w.Mt + 1, Tn = w.next_Mt + 1;
  const double* h = hw + w.h_off;
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < T; ++k) acc += h[k] * U[w.u_off + (long long)k * S + j];
    for (int l = 0; l < Tn; ++l) U[w.next_u_off + (long long)l * S + j] = acc;
  }
}

}  // namespace spmc

namespace spmc {

// ----------------------------------------------------------------- adjoint
// lambda of interval r before its last iteration: lambda[k][j] = hw_k g_j with
// g = dL/du(T) (the instance's last interval) or mu of the next interval.
__global__ void adj_lambda_init_kernel(const InstInterval* __restrict__ ii, const int* __restrict__ last_of_inst,
                                       const double* __restrict__ hw, const double* __restrict__ dLdz,
                                       const double* __restrict__ mu, double* __restrict__ lambda, int r, int S) {
  const InstInterval w = ii[blockIdx.x];
  const int T = w.Mt + 1;
  const double* src = (last_of_inst[w.inst] == r ? dLdz : mu) + (long long)w.inst * S;
  const double* h = hw + w.h_off;
  for (int i = threadIdx.x; i < T * S; i += blockDim.x) {
    const int k = i / S, j = i - k * S;
    lambda[w.u_off + i] = h[k] * src[j];
  }
}

// Transposed time contraction of the adjoint slice accumulators:
// Lam[c][q][p] = sum over the instance's slices s of L_q(xi(tau_s)) gT[s][c][p],
// c in {alpha Phi, beta Phi, beta Psi}.  One block per active instance.
__global__ void adj_time_kernel(const InstInterval* __restrict__ ii, const TimeNode* __restrict__ tn,
                                const long long* __restrict__ first_tn, const SliceInfo* __restrict__ sinfo,
                                const double* __restrict__ gT, double* __restrict__ lam, int S, int n_sub) {
  __shared__ double L[41];
  const InstInterval w = ii[blockIdx.x];
  const int T = w.Mt + 1;
  double* out = lam + 3LL * w.c_off / 2;   // c_off counts two (Mt+1) S blocks per instance
  for (int i = threadIdx.x; i < 3 * T * S; i += blockDim.x) out[i] = 0.0;
  __syncthreads();
  for (long long t = first_tn[blockIdx.x]; t < first_tn[blockIdx.x + 1]; ++t) {
    const TimeNode nd = tn[t];
    const long long ns = (long long)n_sub * nd.nstar;
    for (long long m = 0; m < ns; ++m) {
      const long long sidx = nd.slice_base + m;
      __syncthreads();
      if (threadIdx.x == 0) {
        const double tau = sinfo[sidx].tau;
        const double xi = (2.0 * tau - w.t0 - (w.t0 + w.h)) / w.h;
        L[0] = 1.0;
        if (w.Mt >= 1) L[1] = xi;
        for (int q = 1; q < w.Mt; ++q) L[q + 1] = ((2.0 * q + 1.0) * xi * L[q] - q * L[q - 1]) / (q + 1.0);
      }
      __syncthreads();
      const double* g = gT + sidx * 3 * S;
      for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) {
        const double v = g[i];
        if (v == 0.0) continue;
        const int c = i / S, p = i - c * S;
        for (int q = 0; q < T; ++q) out[((long long)c * T + q) * S + p] += L[q] * v;
      }
    }
  }
}

// lambda += R^T (Lam_alpha - Dt^T Lam_betaPhi - kappa Lam_betaPsi), R = B x A x ... x A,
// (Dt^T X)_l = sum_{q < l, l+q odd} (2/h)(2q+1) X_q.  One block per active instance.
template <int D>
__global__ void adj_combine_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ lam,
                                   const double* __restrict__ A, const double* __restrict__ Bt,
                                   double* __restrict__ lambda, int n, double kappa) {
  extern __shared__ double sm[];
  const InstInterval w = ii[blockIdx.x];
  int S = 1;
  for (int e = 0; e < D; ++e) S *= n;
  const int T = w.Mt + 1, tot = T * S;
  const double* la = lam + 3LL * w.c_off / 2;
  const double* lb = la + tot;
  const double* lp = lb + tot;
  double* x = sm;
  double* y = sm + tot;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int l = i / S, p = i - l * S;
    double dt = 0.0;
    for (int q = l - 1; q >= 0; q -= 2) dt += (2.0 / w.h) * (2.0 * q + 1.0) * lb[q * S + p];
    x[i] = la[i] - dt - kappa * lp[i];
  }
  __syncthreads();
  // spatial axes: x[..p_e..] -> y[..j_e..] = sum_{p_e} A[p_e][j_e] x
  double* src = x;
  double* dst = y;
  int stride = 1;
  for (int e = 0; e < D; ++e) {
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int q = i / S, idx = i - q * S;
      const int je = (idx / stride) % n;
      const int base = q * S + idx - je * stride;
      double acc = 0.0;
      for (int pe = 0; pe < n; ++pe) acc += A[pe * n + je] * src[base + pe * stride];
      dst[i] = acc;
    }
    __syncthreads();
    double* t = src; src = dst; dst = t;
    stride *= n;
  }
  // time axis: lambda[k][j] += sum_q B[q][k] src[q][j]
  const double* B = Bt + w.b_off;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int kk = i / S, j = i - kk * S;
    double acc = 0.0;
    for (int q = 0; q < T; ++q) acc += B[q * T + kk] * src[q * S + j];
    lambda[w.u_off + i] += acc;
  }
}

// mu_j = sum_l lambda[l][j]: the adjoint of the interval's first row.
__global__ void adj_mu_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ lambda,
                              double* __restrict__ mu, int S) {
  const InstInterval w = ii[blockIdx.x];
  const int T = w.Mt + 1;
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < T; ++l) acc += lambda[w.u_off + (long long)l * S + j];
    mu[(long long)w.inst * S + j] = acc;
  }
}

}  // namespace spmc

namespace spmc {

// ----------------------------------------------------------------- d >= 3
// Reconstruction in global memory, one axis per launch: out = M x_axis in, for
// every active instance (blockIdx.y).  axis 0 is time (matrix B_n, row-major
// [q][k]); axis e >= 1 is space axis e-1 (matrix A, [p][j]).  Blocks are
// (M_n+1) x n^d FP64, time slowest, x_1 fastest.
__global__ void mode_product_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ in_base,
                                    long long in_is_U, double* __restrict__ out_base, const double* __restrict__ A,
                                    const double* __restrict__ Bt, int n, int S, int axis) {
  const InstInterval w = ii[blockIdx.y];
  const int T = w.Mt + 1;
  const long long tot = (long long)T * S;
  const double* in = in_is_U ? in_base + w.u_off : in_base + w.c_off / 2;
  double* out = out_base + w.c_off / 2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / S);
    const int idx = (int)(i - (long long)q * S);
    double acc = 0.0;
    if (axis == 0) {
      const double* B = Bt + w.b_off;
      for (int k = 0; k < T; ++k) acc += B[q * T + k] * in[(long long)k * S + idx];
    } else {
      int stride = 1;
      for (int e = 1; e < axis; ++e) stride *= n;
      const int pe = (idx / stride) % n;
      const long long base = (long long)q * S + idx - (long long)pe * stride;
      for (int je = 0; je < n; ++je) acc += A[pe * n + je] * in[base + (long long)je * stride];
    }
    out[i] = acc;
  }
}

// cu (final mode product) -> coefficient blocks: cu copied, ct by the
// Legendre derivative identity.
__global__ void coef_finish_kernel(const InstInterval* __restrict__ ii, const double* __restrict__ src_base,
                                   double* __restrict__ coef, int S) {
  const InstInterval w = ii[blockIdx.y];
  const int T = w.Mt + 1;
  const long long tot = (long long)T * S;
  const double* src = src_base + w.c_off / 2;
  double* cu = coef + w.c_off;
  double* ct = cu + tot;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / S);
    const long long p = i - (long long)q * S;
    cu[i] = src[i];
    double acc = 0.0;
    for (int l = q + 1; l < T; l += 2) acc += src[(long long)l * S + p];
    ct[i] = (2.0 / w.h) * (2.0 * q + 1.0) * acc;
  }
}

// Residual at y (d = 5, n <= 8) from a slice streamed through shared memory one
// x_5 mode at a time: the caller stages tile t (C and H for p_5 = t, n^4 each,
// x_1 fastest) and calls accumulate for every tile, then finish.  The
// contraction is sum-factorised from x_1 to x_5 with three running states:
// S0 (all phi), S1 (one psi, the Laplacian) and H (all phi, d_t part).
template <typename R>
struct Eval5 {
  R ph[5][8], ps[5][8];
  R s0, s1, hh;   // final contractions
  __device__ __forceinline__ void init(int n, const R* y) {
#pragma unroll
    for (int e = 0; e < 5; ++e) basis<8, R>(n, y[e], ph[e], ps[e]);
    s0 = R(0); s1 = R(0); hh = R(0);
  }
  // entry idx of a register array (runtime index without local memory)
  static __device__ __forceinline__ R pick(const R* v, int idx) {
    R out = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) out = (idx == k) ? v[k] : out;
    return out;
  }
  // tile of p_5 = t: C[p1 + n p2 + n^2 p3 + n^3 p4], H likewise
  __device__ __forceinline__ void accumulate(int n, int t, const R* __restrict__ C, const R* __restrict__ H) {
    R a0 = R(0), a1 = R(0), ah = R(0);          // level 4 (over p4)
    for (int p4 = 0; p4 < n; ++p4) {
      R b0 = R(0), b1 = R(0), bh = R(0);        // level 3 (over p3)
#pragma unroll
      for (int p3 = 0; p3 < 8; ++p3) {
        if (p3 < n) {
          R c0 = R(0), c1 = R(0), ch = R(0);    // level 2 (over p2)
#pragma unroll
          for (int p2 = 0; p2 < 8; ++p2) {
            if (p2 < n) {
              const R* cr = C + ((p4 * n + p3) * n + p2) * n;
              const R* hr = H + ((p4 * n + p3) * n + p2) * n;
              R d0 = R(0), d1 = R(0), dh = R(0);   // level 1 (over p1)
#pragma unroll
              for (int p1 = 0; p1 < 8; ++p1) {
                if (p1 < n) {
                  const R cv = cr[p1];
                  d0 += cv * ph[0][p1];
                  d1 += cv * ps[0][p1];
                  dh += hr[p1] * ph[0][p1];
                }
              }
              c0 += d0 * ph[1][p2];
              c1 += d1 * ph[1][p2] + d0 * ps[1][p2];
              ch += dh * ph[1][p2];
            }
          }
          b0 += c0 * ph[2][p3];
          b1 += c1 * ph[2][p3] + c0 * ps[2][p3];
          bh += ch * ph[2][p3];
        }
      }
      const R f4 = pick(ph[3], p4), g4 = pick(ps[3], p4);
      a0 += b0 * f4;
      a1 += b1 * f4 + b0 * g4;
      ah += bh * f4;
    }
    const R f5 = pick(ph[4], t), g5 = pick(ps[4], t);
    s0 += a0 * f5;
    s1 += a1 * f5 + a0 * g5;
    hh += ah * f5;
  }
  // r = f(u*) + f_add + H - kappa (-Delta u*)
  __device__ __forceinline__ R finish(const InstanceParams& ip, R kappa, const R* y, R Tt, R dTt) const {
    return reaction<R>(ip, s0) + source<5, R>(ip, kappa, y, Tt, dTt) + hh - kappa * s1;
  }
};

}  // namespace spmc

namespace spmc {

// Persistent sweep for d = 5 (n <= 8).  Cohorts, windows and walks as in
// sweep_kernel; the evaluation differs: a slice (2 n^5 entries) does not fit in
// shared memory, so each window runs rounds of
//   (a) the pending evaluation point (Green point, roulette) of every walk
//       pending in the window,
//   (b) for each of the window's slices, all walks pending at it together: the
//       slice streams through shared memory one x_5 mode (2 n^4 entries) at a
//       time and every walk accumulates its sum-factorised contraction,
//   (c) one step of every walk pending in the window,
// until no walk is pending in the window.
template <typename R>
__global__ void __launch_bounds__(256)
sweep5_kernel(SweepArgs a, int JT, int CC, long long n_cohorts, int* __restrict__ work_counter,
              void* __restrict__ state_base, long long state_stride) {
  constexpr int D = 5;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int S = a.S, n = a.n;
  const int G = a.n_sub;
  const long long slst = a.sl_stride;
  const int half = a.half;
  const int W = JT * CC;
  const int n_jt = (S + JT - 1) / JT;
  const int n4 = n * n * n * n;
  R* tC = reinterpret_cast<R*>(smraw);                       // [2][n^4] tile
  unsigned char* p = smraw + ((2 * n4 * sizeof(R) + 15) / 16) * 16;
  int* mnext = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* act = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* ready = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* elist = reinterpret_cast<int*>(p); p += W * sizeof(int);
  int* eb = reinterpret_cast<int*>(p); p += W * sizeof(int);
  R* ew = reinterpret_cast<R*>(p); p += W * sizeof(R);
  R* eY = reinterpret_cast<R*>(p); p += 5 * W * sizeof(R);
  __shared__ int red[64];
  __shared__ double dred[32];
  __shared__ int s_next, s_nact;
  __shared__ double s_Tt[16], s_dTt[16];

  unsigned char* gb = reinterpret_cast<unsigned char*>(state_base) + (long long)blockIdx.x * state_stride;
  WalkState<D, R> st;
#pragma unroll
  for (int e = 0; e < D; ++e) { st.X[e] = reinterpret_cast<R*>(gb); gb += W * sizeof(R); }
  st.f = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.w = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.r = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.S = reinterpret_cast<R*>(gb); gb += W * sizeof(R);
  st.k = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.q = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.last = reinterpret_cast<int*>(gb); gb += W * sizeof(int);
  st.mnext = mnext;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const R kappa = (R)a.kappa;
  const R shell = (R)a.shell;
  const R* slices = reinterpret_cast<const R*>(a.slices);
  unsigned long long capped = 0, points = 0;
  double dummy_acc = 0.0;

  auto block_scan = [&](int cnt, int& base) -> int {
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int wv = 0; wv < nwarps; ++wv) {
      if (wv < warp) wbase += red[wv];
      total += red[wv];
    }
    __syncthreads();
    base = wbase + incl - cnt;
    return total;
  };

  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(work_counter, 1);
    __syncthreads();
    const long long id = s_next;
    __syncthreads();
    if (id >= n_cohorts) break;
    long long b = id;
    const int chunk = (int)(b % a.n_chunks);
    b /= a.n_chunks;
    const int jt = (int)(b % n_jt);
    const long long ti = b / n_jt;
    const TimeNode node = a.tn[ti];
    const InstanceParams ip = a.ip[node.inst];
    const int j0 = jt * JT;
    const R sdur = Ar<R>::sub((R)node.t_node, (R)node.t0);
    const R delta = Ar<R>::div(sdur, (R)node.nstar);
    const R J = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), delta));
    const R sub = Ar<R>::div(delta, (R)G);
    const int Ktot = G * node.nstar;
    const uint32_t tag = ((uint32_t)(node.inst & 0xfff) << 20) | ((uint32_t)(a.interval & 0x3ff) << 10) |
                         (uint32_t)(a.iteration & 0x3ff);
    const long long sample0 = (long long)chunk * CC;
    WalkStream ws;
    ws.k0 = a.k0; ws.k1 = a.k1; ws.tag = tag;

    int cnt = 0;
    for (int wk = threadIdx.x; wk < W; wk += blockDim.x) {
      const int jj = wk / CC, s = wk - jj * CC;
      const int j = j0 + jj;
      st.S[wk] = R(0);
      if (j >= S || sample0 + s >= a.M) { mnext[wk] = -1; continue; }
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { st.X[e][wk] = (R)a.xnodes[jr % n]; jr /= n; }
      st.f[wk] = R(0); st.k[wk] = 0; st.q[wk] = 0;
      ws.node = (uint32_t)(node.ell * S + j);
      ws.sample = (uint32_t)(sample0 + s);
      prepare_step<D, R>(st, wk, ws, J, delta, sub, Ktot, G, a.gbits, shell, kappa, a.max_steps, dummy_acc, capped);
      if (mnext[wk] >= 0) ++cnt;
    }
    __syncthreads();
    {
      int base;
      const int tot = block_scan(cnt, base);
      for (int wk = threadIdx.x; wk < W; wk += blockDim.x)
        if (mnext[wk] >= 0) act[base++] = wk;
      if (threadIdx.x == 0) s_nact = tot;
      __syncthreads();
    }
    int m0 = 0;
    const int max_passes = 2 * Ktot + 8;
    int passes = 0;
    while (s_nact > 0) {
      const int nact = s_nact;
      if (++passes > max_passes) {
        if (threadIdx.x == 0) { atomicOr(a.status, 2); s_nact = 0; }
        for (int i = threadIdx.x; i < nact; i += blockDim.x) mnext[act[i]] = -1;
        __syncthreads();
        break;
      }
      int rc = 0, mn = 0x7fffffff;
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int mv = mnext[act[i]];
        if (mv < m0 + G) ++rc; else mn = min(mn, mv);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      if (lane == 0) red[32 + warp] = mn;
      int rbase;
      const int nready = block_scan(rc, rbase);
      int gmin = 0x7fffffff;
      for (int wv = 0; wv < nwarps; ++wv) gmin = min(gmin, red[32 + wv]);
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int wk = act[i];
        if (mnext[wk] < m0 + G) ready[rbase++] = wk;
      }
      if (nready == 0) {
        __syncthreads();
        m0 = gmin;
        continue;
      }
      if (threadIdx.x < G && m0 + (int)threadIdx.x < Ktot) {
        SliceInfo si = a.sinfo[node.slice_base + m0 + threadIdx.x];
        s_Tt[threadIdx.x] = si.Tt; s_dTt[threadIdx.x] = si.dTt;
      }
      __syncthreads();
      int rounds = 0;
      while (true) {
        if (++rounds > a.max_steps + 8) {  // cannot happen: each round advances every pending walk by a step
          if (threadIdx.x == 0) atomicOr(a.status, 2);
          for (int i = threadIdx.x; i < nready; i += blockDim.x) mnext[ready[i]] = -1;
          __syncthreads();
          break;
        }
        // (a) pending evaluation points
        for (int i = threadIdx.x; i < nready; i += blockDim.x) {
          const int wk = ready[i];
          const int mv = mnext[wk];
          eb[wk] = -1;
          if (!(mv >= m0 && mv < m0 + G)) continue;
          const int jj = wk / CC;
          ws.node = (uint32_t)(node.ell * S + j0 + jj);
          ws.sample = (uint32_t)(sample0 + (wk - jj * CC));
          const int q = st.q[wk];
          constexpr int WS = step_words(D);
          const uint32_t w0 = (uint32_t)q * WS;
          const R r = st.r[wk];
          R w = st.w[wk];
          if (r < J && w > R(0)) {
            const uint32_t rw = stream_word(ws, w0 + rword_index(D));
            w = roulette_keep<R>(rw, Ar<R>::divr(w, delta, Ar<R>::div(R(1), delta))) ? delta : R(0);
          }
          if (w > R(0)) {
            R thg[D];
            direction<D, R>(ws, w0 + gdir_index(D), thg);
            R U1, U2;
            green_uniforms<D, R>(ws, w0, U1, U2);
            const R v = green_radius<D, R>(U1, U2);
            const R rv = Ar<R>::mul(r, v);
#pragma unroll
            for (int e = 0; e < D; ++e) eY[e * W + wk] = Ar<R>::add(st.X[e][wk], Ar<R>::mul(rv, thg[e]));
            ew[wk] = w;
            eb[wk] = mv - m0;
          }
        }
        __syncthreads();
        // (b) evaluations, slice by slice
        for (int bs = 0; bs < G; ++bs) {
          if (m0 + bs >= Ktot) break;
          int ec = 0;
          for (int i = threadIdx.x; i < nready; i += blockDim.x) ec += (eb[ready[i]] == bs);
          int ebase;
          const int ne = block_scan(ec, ebase);
          for (int i = threadIdx.x; i < nready; i += blockDim.x)
            if (eb[ready[i]] == bs) elist[ebase++] = ready[i];
          __syncthreads();
          if (ne == 0) continue;
          const R* sl = slices + (node.slice_base + m0 + bs) * slst;
          for (int c0 = 0; c0 < ne; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            const bool has = i < ne;
            const int wk = has ? elist[i] : 0;
            Eval5<R> ev;
            R Y[D];
            if (has) {
#pragma unroll
              for (int e = 0; e < D; ++e) Y[e] = eY[e * W + wk];
              ev.init(n, Y);
            }
            for (int t5 = 0; t5 < n; ++t5) {
              __syncthreads();
              for (int x = threadIdx.x; x < n4; x += blockDim.x) {
                tC[x] = sl[(long long)t5 * n4 + x];
                tC[n4 + x] = sl[half + (long long)t5 * n4 + x];
              }
              __syncthreads();
              if (has) ev.accumulate(n, t5, tC, tC + n4);
            }
            if (has) {
              const R res = ev.finish(ip, kappa, Y, (R)s_Tt[bs], (R)s_dTt[bs]);
              st.S[wk] += ew[wk] * res;
              ++points;
            }
          }
          __syncthreads();
        }
        // (c) one step of every walk pending in the window
        int pend = 0;
        for (int i = threadIdx.x; i < nready; i += blockDim.x) {
          const int wk = ready[i];
          int mv = mnext[wk];
          if (!(mv >= m0 && mv < m0 + G)) continue;
          if (st.last[wk]) { mnext[wk] = -1; continue; }
          const int jj = wk / CC;
          ws.node = (uint32_t)(node.ell * S + j0 + jj);
          ws.sample = (uint32_t)(sample0 + (wk - jj * CC));
          const int q = st.q[wk];
          constexpr int WS = step_words(D);
          const uint32_t w0 = (uint32_t)q * WS;
          const R r = st.r[wk];
          R th[D];
          direction<D, R>(ws, w0, th);
#pragma unroll
          for (int e = 0; e < D; ++e) st.X[e][wk] = Ar<R>::add(st.X[e][wk], Ar<R>::mul(r, th[e]));
          st.q[wk] = q + 1;
          prepare_step<D, R>(st, wk, ws, J, delta, sub, Ktot, G, a.gbits, shell, kappa, a.max_steps,
                             dummy_acc, capped);
          mv = mnext[wk];
          pend += (mv >= m0 && mv < m0 + G);
        }
        if (!__syncthreads_or(pend)) break;
      }
      // compact the active list
      int kc = 0;
      for (int i = threadIdx.x; i < nact; i += blockDim.x) kc += (mnext[act[i]] >= 0);
      int kbase;
      const int nkeep = block_scan(kc, kbase);
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int wk = act[i];
        if (mnext[wk] >= 0) ready[kbase++] = wk;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nkeep; i += blockDim.x) act[i] = ready[i];
      if (threadIdx.x == 0) s_nact = nkeep;
      __syncthreads();
      m0 += G;
    }
    for (int jj = 0; jj < JT; ++jj) {
      const int j = j0 + jj;
      if (j >= S) break;
      double t = 0.0;
      for (int s = threadIdx.x; s < CC; s += blockDim.x) t += (double)st.S[jj * CC + s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) dred[warp] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int wv = 0; wv < nwarps; ++wv) tt += dred[wv];
        a.partial[(ti * S + j) * a.n_chunks + chunk] = tt;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    points += __shfl_xor_sync(0xffffffffu, points, o);
    capped += __shfl_xor_sync(0xffffffffu, capped, o);
  }
  if (lane == 0) {
    if (points) atomicAdd(&a.counters[0], points);
    if (capped) atomicAdd(&a.counters[1], capped);
  }
}

}  // namespace spmc
