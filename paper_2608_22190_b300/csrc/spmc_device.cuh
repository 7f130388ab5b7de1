// spmc_device.cuh -- device building blocks of the sweep (sm_103a).
//
//  * Philox4x32-10 (Salmon et al., SC'11) counter-based generator;
//  * Jacobi/Babuska-Shen basis values by recurrence (Section 2.3);
//  * the inside-ball walk step of the residual estimator (Section 2.2,
//    Lemma Xlocation, Eqs. indexL, interIQ, with walk-on-spheres balls that stay
//    inside Omega and Green-function quadrature points per ball);
//  * the residual r = f(u*) + f_add - d_t u* + kappa Delta u* at a point from a
//    time-contracted coefficient slice (Eqs. u_N, ufg_ep1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spmc {

constexpr double kPiD = 3.14159265358979323846;

// ------------------------------------------------------------------ Philox
struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  Philox4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// ------------------------------------------------------------------ division
// Quotient of a 32-bit unsigned n by a divisor d fixed for a launch, by one
// high multiply, a subtract, an add and two shifts (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Sec. 4):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n),
// exact for every n < 2^32 and 1 <= d < 2^32.
struct FastDiv {
  uint32_t d = 1, m = 1, s1 = 0, s2 = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t dd) : d(dd) {
    int l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)dd) ++l;
    m = (uint32_t)((((1ull << l) - dd) << 32) / dd + 1);
    s1 = l < 1 ? (uint32_t)l : 1u;
    s2 = l > 1 ? (uint32_t)(l - 1) : 0u;
  }
  __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(m, n);
#else
    const uint32_t t = (uint32_t)(((unsigned long long)m * n) >> 32);
#endif
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// The stream of one walk: key = seed, counter = (block, sample, node, tag).
struct WalkStream {
  uint32_t k0, k1, sample, node, tag;
  __device__ __forceinline__ Philox4 block(uint32_t b) const { return philox4x32_10(b, sample, node, tag, k0, k1); }
};

template <typename R> struct U01;
template <> struct U01<double> {
  // 53-bit uniform on (0,1) from a pair of words
  static __device__ __forceinline__ double pair(uint32_t a, uint32_t b) {
    return __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)), 0.5),
                     1.0 / 9007199254740992.0);
  }
  // 32-bit uniform on (0,1) from one word: (a + 1/2) 2^-32 (exact in FP64)
  static __device__ __forceinline__ double one(uint32_t a) {
    return __dmul_rn(__dadd_rn((double)a, 0.5), 1.0 / 4294967296.0);
  }
};
template <> struct U01<float> {
  // 24-bit uniform on (0,1) from the first word of the pair
  static __device__ __forceinline__ float pair(uint32_t a, uint32_t) {
    return ((float)(a >> 8) + 0.5f) * (1.0f / 16777216.0f);
  }
  static __device__ __forceinline__ float one(uint32_t a) { return pair(a, 0u); }
};

// exact-rounding arithmetic helpers (no FMA contraction where the walk
// decides control flow: the FP64 walk must match the CPU step for step)
template <typename R> struct Ar;
template <> struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double abs_(double a) { return ::fabs(a); }
  // a / b given inv_b = 1 / b: the FP64 walk divides (step for step as the CPU reference)
  static __device__ __forceinline__ double divr(double a, double b, double) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double log_(double a) { return log(a); }
  static __device__ __forceinline__ void sincos2pi(double U, double* s, double* c) { sincospi(2.0 * U, s, c); }
  static __device__ __forceinline__ double sinpi_(double x) { return sinpi(x); }
  static __device__ __forceinline__ double cospi_(double x) { return cospi(x); }
  static __device__ __forceinline__ double sin_(double x) { return sin(x); }
  static __device__ __forceinline__ double cos_(double x) { return cos(x); }
  static constexpr int kBisect = 60;
};
template <> struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float abs_(float a) { return fabsf(a); }
  // a / b given inv_b = 1 / b: the FP32 walk multiplies by the reciprocal
  static __device__ __forceinline__ float divr(float a, float, float inv_b) { return __fmul_rn(a, inv_b); }
  static __device__ __forceinline__ float log_(float a) { return logf(a); }
  static __device__ __forceinline__ void sincos2pi(float U, float* s, float* c) { sincospif(2.0f * U, s, c); }
  static __device__ __forceinline__ float sinpi_(float x) { return sinpif(x); }
  static __device__ __forceinline__ float cospi_(float x) { return cospif(x); }
  static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
  static __device__ __forceinline__ float cos_(float x) { return cosf(x); }
  static constexpr int kBisect = 24;
};

// ------------------------------------------------------------------ word layout
// Words of one step of the inside-ball walk, padded to whole Philox blocks:
// [next-step direction wd | Green direction wd | Green radius 2 (d=2: 4) |
//  sub-point 1 | evaluation roulette 1]
__host__ __device__ constexpr int dir_words(int d) { return d == 1 ? 1 : (d == 2 ? 2 : 4 * ((d + 1) / 2)); }
__host__ __device__ constexpr int radius_words(int d) { return d == 2 ? 4 : 2; }
// Words of one walk step, padded to whole Philox blocks.  d <= 2 (one word per
// uniform, 8 words): [step direction | Green direction | sub-point word |
// roulette word | Green radius uniform(s) | unused], so the words every step
// needs share the first block.  d >= 3 (uniforms from word pairs):
// [step direction | Green direction | Green radius pair | sub-point | roulette].
__host__ __device__ constexpr int step_words(int d) {
  return d <= 2 ? 8 : ((2 * dir_words(d) + radius_words(d) + 2) + 3) / 4 * 4;
}
__host__ __device__ constexpr int gdir_index(int d) { return d <= 2 ? 1 : dir_words(d); }
__host__ __device__ constexpr int radius_index(int d) { return d <= 2 ? 4 : 2 * dir_words(d); }
__host__ __device__ constexpr int gword_index(int d) { return d <= 2 ? 2 : 2 * dir_words(d) + radius_words(d); }
__host__ __device__ constexpr int rword_index(int d) { return gword_index(d) + 1; }

// fetch word w of the walk (one Philox evaluation per call)
__device__ __forceinline__ uint32_t stream_word(const WalkStream& s, uint32_t w) {
  Philox4 b = s.block(w >> 2);
  return b.v[w & 3];
}

// Uniform direction on S^{d-1} from the words starting at w0 (Lemma Xlocation):
// d=1 sign bit; d=2 angle 2 pi U (U from one word); d>=3 normalised Box-Muller
// Gaussians (uniforms from word pairs).
template <int D, typename R>
__device__ __forceinline__ void direction(const WalkStream& s, uint32_t w0, R* th) {
  if (D == 1) {
    th[0] = (stream_word(s, w0) >> 31) ? R(-1) : R(1);
  } else if (D == 2) {
    R U = U01<R>::one(stream_word(s, w0));
    R sn, cs;
    Ar<R>::sincos2pi(U, &sn, &cs);
    th[0] = cs; th[1] = sn;
  } else {
    constexpr int NP = (D + 1) / 2;
    R z[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      Philox4 b = s.block((w0 >> 2) + k);  // w0 is a multiple of 4 for d >= 3
      R U1 = U01<R>::pair(b.v[0], b.v[1]);
      R U2 = U01<R>::pair(b.v[2], b.v[3]);
      R Rr = Ar<R>::sqrt_(Ar<R>::mul(R(-2), Ar<R>::log_(U1)));
      R sn, cs;
      Ar<R>::sincos2pi(U2, &sn, &cs);
      z[2 * k] = Ar<R>::mul(Rr, cs);
      z[2 * k + 1] = Ar<R>::mul(Rr, sn);
    }
    R nrm = R(0);
#pragma unroll
    for (int e = 0; e < D; ++e) nrm = Ar<R>::add(nrm, Ar<R>::mul(z[e], z[e]));
    nrm = Ar<R>::sqrt_(nrm);
#pragma unroll
    for (int e = 0; e < D; ++e) th[e] = Ar<R>::div(z[e], nrm);
  }
}

// Direction of step q of the fixed-radius walk (Lemma Xlocation as printed):
// words per step d = 1: one (its sign bit); d = 2: two (a 53-bit / 24-bit
// uniform angle from the pair); d >= 3: normalised Box-Muller Gaussians from
// dir_words(d) words.
template <int D, typename R>
__device__ __forceinline__ void literal_direction(const WalkStream& s, int q, R* th) {
  if (D == 1) {
    th[0] = (stream_word(s, (uint32_t)q) >> 31) ? R(-1) : R(1);
  } else if (D == 2) {
    const Philox4 b = s.block((uint32_t)q >> 1);   // words 2q, 2q + 1 share a block
    const R U = U01<R>::pair(b.v[(2 * q) & 3], b.v[(2 * q + 1) & 3]);
    R sn, cs;
    Ar<R>::sincos2pi(U, &sn, &cs);
    th[0] = cs; th[1] = sn;
  } else {
    direction<D, R>(s, (uint32_t)q * (uint32_t)dir_words(D), th);
  }
}

// The Green radius uniforms of the step whose words start at w0 (U2 is used for d = 2 only).
template <int D, typename R>
__device__ __forceinline__ void green_uniforms(const WalkStream& s, uint32_t w0, R& U1, R& U2) {
  const uint32_t wr = w0 + radius_index(D);   // a multiple of 4
  const Philox4 b = s.block(wr >> 2);
  if (D <= 2) {
    U1 = U01<R>::one(b.v[0]);
    U2 = (D == 2) ? U01<R>::one(b.v[1]) : R(0);
  } else {
    U1 = U01<R>::pair(b.v[0], b.v[1]);
    U2 = R(0);
  }
}

// Radial law of the ball's Green function as a fraction v of the radius:
// d=1 density 2(1-v); d=2 density 4 v log(1/v); d>=3 density prop. to v - v^{d-1}.
template <int D, typename R>
__device__ __forceinline__ R green_radius(R U1, R U2) {
  if (D == 1) return Ar<R>::sub(R(1), Ar<R>::sqrt_(U1));
  if (D == 2) return Ar<R>::sqrt_(Ar<R>::mul(U1, U2));
  R lo = R(0), hi = R(1);
  for (int it = 0; it < Ar<R>::kBisect; ++it) {
    R v = Ar<R>::mul(R(0.5), Ar<R>::add(lo, hi));
    R vd = R(1);
#pragma unroll
    for (int k = 0; k < D; ++k) vd = Ar<R>::mul(vd, v);
    R F = Ar<R>::div(Ar<R>::sub(Ar<R>::mul(Ar<R>::mul(R(D), v), v), Ar<R>::mul(R(2), vd)), R(D - 2.0));
    if (F < U1) lo = v; else hi = v;
  }
  return Ar<R>::mul(R(0.5), Ar<R>::add(lo, hi));
}

// Russian-roulette decision of a shrunk ball: keep the term iff the uniform
// ((rw >> 8) + 1/2) 2^-24 is below p = w / Delta.  Decided in integers: with
// a = rw >> 8, (a + 1/2) 2^-24 < p  <=>  2a + 1 < 2^25 p  <=>  2a + 1 < ceil(2^25 p)
// (an integer n is below x iff it is below ceil(x)); 2^25 p is exact in R, so
// the decision is the same as the FP64 comparison for both precisions and the
// FP32 sweep issues no FP64 instruction for it.
template <typename R>
__device__ __forceinline__ bool roulette_keep(uint32_t rw, R p) {
  const R P = p * R(33554432.0);            // exact (a power-of-two scale)
  if (P >= R(33554432.0)) return true;      // p >= 1: every uniform is below it
  if (!(P >= R(0))) return false;           // negative or NaN: never below it
  int c;                                    // ceil(P), exact: an integer in [0, 2^25]
  if constexpr (sizeof(R) == 4) c = __float2int_ru(P);
  else c = __double2int_ru(P);
  return (int)(2u * (rw >> 8) + 1u) < c;
}

// ------------------------------------------------------------------ exact sums
// Order-independent per-node sums.  A term x is rounded once to the signed
// fixed-point integer N = round(x 2^80) (magnitude below 2^126, so |x| < 2^46)
// by integer operations on its bits; sums of N are exact, so a node's total
// does not depend on the order in which events or blocks add to it.  The
// global accumulator of a node holds four 64-bit counters of 32-bit limbs of N
// (limb 3 signed); limbs are added without carries, so each counter has room
// for 2^32 additions.  FixedAcc::value() assembles the 128-bit total and rounds
// it to FP64 once.
constexpr int kFixFrac = 80;

// N for a double or float term; returns false if |x| >= 2^46 or x is not finite.
__device__ __forceinline__ bool fix_from_double(double x, __int128& N) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E >= 1023 + 46) { N = 0; return false; }
  const unsigned long long m = (b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int s = (E ? E : 1) - 1075 + kFixFrac;   // x = m 2^(E - 1075), N = m 2^s
  unsigned __int128 v;
  if (s >= 0) v = (unsigned __int128)m << s;
  else if (s > -54) v = (unsigned __int128)((m + (1ull << (-s - 1))) >> (-s));
  else v = 0;
  N = (b >> 63) ? -(__int128)v : (__int128)v;
  return true;
}
__device__ __forceinline__ bool fix_from_float(float x, __int128& N) {
  const uint32_t b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xff);
  if (E >= 127 + 46) { N = 0; return false; }
  const uint32_t m = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  const int s = (E ? E : 1) - 150 + kFixFrac;    // x = m 2^(E - 150)
  unsigned __int128 v;
  if (s >= 0) v = (unsigned __int128)m << s;
  else if (s > -25) v = (unsigned __int128)((m + (1u << (-s - 1))) >> (-s));
  else v = 0;
  N = (b >> 31) ? -(__int128)v : (__int128)v;
  return true;
}
// The same fixed-point value of an FP32 term as five signed 26-bit limbs,
// N = sum_k L[k] 2^(26 k): the (rounded) 24-bit significand shifted to its
// place spans two adjacent limbs, the others are zero.  Each |L[k]| < 2^26, so
// 32 of them sum exactly in an int32 (a warp reduction per limb), and the
// limb sums reassemble the exact 128-bit total.
__device__ __forceinline__ bool fix_limbs_float(float x, int (&L)[5]) {
  const uint32_t b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xff);
#pragma unroll
  for (int k = 0; k < 5; ++k) L[k] = 0;
  if (E >= 127 + 46) return false;
  uint32_t m = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  int s = (E ? E : 1) - 150 + kFixFrac;           // x = m 2^(E - 150): N = m 2^s
  if (s < 0) { m = s > -25 ? (m + (1u << (-s - 1))) >> (-s) : 0u; s = 0; }
  const int li = s / 26;                           // s <= 102: li <= 3
  const unsigned long long t = (unsigned long long)m << (s - 26 * li);   // < 2^50
  int lo = (int)(t & 0x3ffffffull), hi = (int)(t >> 26);
  if (b >> 31) { lo = -lo; hi = -hi; }
#pragma unroll
  for (int k = 0; k < 5; ++k) L[k] = (k == li) ? lo : ((k == li + 1) ? hi : 0);
  return true;
}
__device__ __forceinline__ __int128 fix_from_limbs(const int (&L)[5]) {
  __int128 N = 0;
#pragma unroll
  for (int k = 4; k >= 0; --k) N = N * ((__int128)1 << 26) + (__int128)L[k];
  return N;
}

template <typename R> __device__ __forceinline__ bool fix_from(R x, __int128& N);
template <> __device__ __forceinline__ bool fix_from<double>(double x, __int128& N) { return fix_from_double(x, N); }
template <> __device__ __forceinline__ bool fix_from<float>(float x, __int128& N) { return fix_from_float(x, N); }

// add N to a node's four limb counters (no return value: fire-and-forget atomics)
__device__ __forceinline__ void fix_atomic_add(unsigned long long* acc, __int128 N) {
  const unsigned __int128 u = (unsigned __int128)N;
  const unsigned long long l0 = (unsigned long long)(u & 0xffffffffull);
  const unsigned long long l1 = (unsigned long long)((u >> 32) & 0xffffffffull);
  const unsigned long long l2 = (unsigned long long)((u >> 64) & 0xffffffffull);
  const long long l3 = (long long)(N >> 96);   // arithmetic shift: signed top limb
  if (l0) atomicAdd(acc + 0, l0);
  if (l1) atomicAdd(acc + 1, l1);
  if (l2) atomicAdd(acc + 2, l2);
  if (l3) atomicAdd(acc + 3, (unsigned long long)l3);
}

// the FP64 value of a node's counters: sum_k c_k 2^(32 k) 2^-80, rounded once
__device__ __forceinline__ double fix_value(const unsigned long long* acc) {
  __int128 T = (__int128)(unsigned __int128)acc[0];
  T += (__int128)((unsigned __int128)acc[1] << 32);
  T += (__int128)((unsigned __int128)acc[2] << 64);
  T += (__int128)((unsigned __int128)acc[3] << 96);   // wraps like the signed limb it holds
  const bool neg = T < 0;
  unsigned __int128 a = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  // round a to 53 significant bits, then scale: exact except for that one rounding
  int nb = 0;
  for (unsigned __int128 t = a; t; t >>= 1) ++nb;
  double v;
  if (nb <= 53) v = (double)(unsigned long long)a;
  else {
    const int sh = nb - 53;
    unsigned __int128 q = a >> sh;
    const unsigned __int128 rem = a - (q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;   // nearest, ties to even
    v = ldexp((double)(unsigned long long)q, sh);
  }
  v = ldexp(v, -kFixFrac);
  return neg ? -v : v;
}

// ------------------------------------------------------------------ problem
struct InstanceParams {
  int f_kind;      // 0: s (c0 + c1 u + c2 u^2 + c3 u^3), 1: s sin(u)
  int ex_kind;     // 0 none, 1 sin product, 2 half-cos product, 3 polynomial,
                   // 4 shifted third-cos product, 5 sin product + t/2 (non-zero boundary values)
  double fc[4];
  double f_scale;
  double ex_beta;
  int bc_kind;     // 0 g = 0, 1 lifted (the unknown is w = u - G), 2 g at absorption
};

template <typename R>
__device__ __forceinline__ R reaction(const InstanceParams& ip, R u) {
  if (ip.f_kind == 1) return R(ip.f_scale) * Ar<R>::sin_(u);
  return R(ip.f_scale) * (R(ip.fc[0]) + u * (R(ip.fc[1]) + u * (R(ip.fc[2]) + u * R(ip.fc[3]))));
}

// Manufactured source f_add = d_t u_ex - kappa Delta u_ex - f(u_ex) at (y, tau);
// Tt = time factor of u_ex at tau, dTt its derivative (polynomial kind).
template <int D, typename R>
__device__ __forceinline__ R source(const InstanceParams& ip, R kappa, const R* y, R Tt, R dTt) {
  if (ip.ex_kind == 0) return R(0);
  if (ip.ex_kind == 1 || ip.ex_kind == 2) {
    R prod = R(1);
#pragma unroll
    for (int e = 0; e < D; ++e)
      prod *= (ip.ex_kind == 1) ? Ar<R>::sinpi_(y[e]) : Ar<R>::cospi_(R(0.5) * y[e]);
    R ue = Tt * prod;
    R cl = (ip.ex_kind == 1) ? R(D * kPiD * kPiD) : R(D * 0.25 * kPiD * kPiD);
    return (R(-ip.ex_beta) + kappa * cl) * ue - reaction<R>(ip, ue);
  }
  R g[D];
  R prod = R(1);
#pragma unroll
  for (int e = 0; e < D; ++e) { g[e] = (R(1) - y[e] * y[e]) * (R(1) + y[e]); prod *= g[e]; }
  R mlap = R(0);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    R term = R(2) + R(6) * y[e];
#pragma unroll
    for (int e2 = 0; e2 < D; ++e2) if (e2 != e) term *= g[e2];
    mlap += term;
  }
  R ue = Tt * prod;
  return dTt * prod + kappa * Tt * mlap - reaction<R>(ip, ue);
}

// Closed forms with non-zero boundary values (the remark on non-homogeneous
// boundary conditions in Section 2.3), T = e^{-beta t}:
//   4: u = T prod c(y_e),  c(y) = cos(pi (y - 0.3) / 3)   (different values on opposite faces)
//   5: u = T prod sin(pi y_e) + t / 2                      (u(., 0) = 0 on the boundary)
template <int D, typename R>
__device__ __forceinline__ R exact_bv(const InstanceParams& ip, const R* y, R Tt, R t) {
  R prod = R(1);
  if (ip.ex_kind == 4) {
#pragma unroll
    for (int e = 0; e < D; ++e) prod *= Ar<R>::cospi_((y[e] - R(0.3)) / R(3));
    return Tt * prod;
  }
#pragma unroll
  for (int e = 0; e < D; ++e) prod *= Ar<R>::sinpi_(y[e]);
  return Tt * prod + R(0.5) * t;
}

// The Gordon-Hall transfinite lifting G of the boundary trace of kinds 4 and 5
// and its d_t G, Delta G at (y, t).  For a product trace T prod c(y_e) the
// lifting is T (prod c - prod (c - c_b)), c_b the linear interpolant of c
// between the faces; kind 5's trace t/2 lifts to the constant t/2.  Zero
// unless bc_kind == 1.
template <int D, typename R>
__device__ __forceinline__ void lift_bv(const InstanceParams& ip, const R* y, R Tt, R t, R& G, R& Gt, R& lapG) {
  G = R(0); Gt = R(0); lapG = R(0);
  if (ip.bc_kind != 1 || (ip.ex_kind != 4 && ip.ex_kind != 5)) return;
  if (ip.ex_kind == 5) { G = R(0.5) * t; Gt = R(0.5); return; }
  const R cm = R(0.20791169081775945), cp = R(0.7431448254773942);   // c(-1), c(1)
  R c[D], dl[D], pc = R(1), pd = R(1);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    c[e] = Ar<R>::cospi_((y[e] - R(0.3)) / R(3));
    dl[e] = c[e] - (R(0.5) * (R(1) - y[e]) * cm + R(0.5) * (R(1) + y[e]) * cp);
    pc *= c[e];
    pd *= dl[e];
  }
  G = Tt * (pc - pd);
  Gt = R(-ip.ex_beta) * G;
  // c'' = -(pi/3)^2 c and (c - c_b)'' = c''
  R s = R(0);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    R term = c[e];
#pragma unroll
    for (int f = 0; f < D; ++f) if (f != e) term *= dl[f];
    s += term;
  }
  lapG = R(-kPiD * kPiD / 9.0) * Tt * (R(D) * pc - s);
}

// The forcing of the equation the iteration solves at (y, tau) for the current
// u* there: f(u*) + f_add, or with lifted boundary data (bc_kind 1)
// f(u* + G) + f_add - d_t G + kappa Delta G (the equation for w = u - G).
// Kinds 0-3 evaluate exactly reaction + source.
template <int D, typename R>
__device__ __forceinline__ R forcing(const InstanceParams& ip, R kappa, const R* y, R Tt, R dTt, R tau, R u) {
  if (ip.ex_kind <= 3) return reaction<R>(ip, u) + source<D, R>(ip, kappa, y, Tt, dTt);
  R G, Gt, lapG;
  lift_bv<D, R>(ip, y, Tt, tau, G, Gt, lapG);
  const R ue = exact_bv<D, R>(ip, y, Tt, tau);
  R fadd;
  if (ip.ex_kind == 4) {
    fadd = (R(-ip.ex_beta) + kappa * R(D * kPiD * kPiD / 9.0)) * ue - reaction<R>(ip, ue);
  } else {
    const R sp = ue - R(0.5) * tau;   // the sine part
    fadd = (R(-ip.ex_beta) + kappa * R(D * kPiD * kPiD)) * sp + R(0.5) - reaction<R>(ip, ue);
  }
  return reaction<R>(ip, u + G) + fadd - Gt + kappa * lapG;
}

// Recurrence coefficients of P^{(1,1)}: P_p = ra_p x P_{p-1} - rb_p P_{p-2},
// ra_p = (2p+1)(p+1)/(p(p+2)), rb_p = (p+1)/(p+2); lam_p = (p+1)(p+2)
// (tables filled once by the host, read through the constant cache).
constexpr int kMaxModes = 64;
__constant__ double c_ra_d[kMaxModes], c_rb_d[kMaxModes], c_lam_d[kMaxModes];
__constant__ float c_ra_f[kMaxModes], c_rb_f[kMaxModes], c_lam_f[kMaxModes];
template <typename R> __device__ __forceinline__ R jac_ra(int p);
template <typename R> __device__ __forceinline__ R jac_rb(int p);
template <typename R> __device__ __forceinline__ R jac_lam(int p);
template <> __device__ __forceinline__ double jac_ra<double>(int p) { return c_ra_d[p]; }
template <> __device__ __forceinline__ double jac_rb<double>(int p) { return c_rb_d[p]; }
template <> __device__ __forceinline__ double jac_lam<double>(int p) { return c_lam_d[p]; }
template <> __device__ __forceinline__ float jac_ra<float>(int p) { return c_ra_f[p]; }
template <> __device__ __forceinline__ float jac_rb<float>(int p) { return c_rb_f[p]; }
template <> __device__ __forceinline__ float jac_lam<float>(int p) { return c_lam_f[p]; }

// Basis values phi_p(y) = (1-y^2) P_p(y) and psi_p(y) = (p+1)(p+2) P_p(y), p < n.
template <int NMAX, typename R>
__device__ __forceinline__ void basis(int n, R y, R* phi, R* psi) {
  R om = R(1) - y * y;
  R pm2 = R(1), pm1 = R(2) * y;
#pragma unroll
  for (int p = 0; p < NMAX; ++p) {
    R P;
    if (p == 0) P = R(1);
    else if (p == 1) P = R(2) * y;
    else { P = jac_ra<R>(p) * y * pm1 - jac_rb<R>(p) * pm2; pm2 = pm1; pm1 = P; }
    phi[p] = (p < n) ? om * P : R(0);
    psi[p] = (p < n) ? jac_lam<R>(p) * P : R(0);
  }
}

// u* and G = -d_t u* + kappa Delta u* at y from one slice (slice_parts), and
// the residual there (residual_at): C = time-contracted coefficients of u*,
// H = time-contracted coefficients of -d_t u* (both in the phi basis; for d=2
// stored [p_x][p_y] with p_y contiguous).
//   u* = sum_p C_p Phi_p(y),
//   G  = sum_p H_p Phi_p(y) - kappa sum_p C_p Psi_p(y)   (= -d_t u* + kappa Delta u*)
//   r  = f(u*) + f_add + G
template <int D, int NMAX, typename R>
__device__ __forceinline__ void slice_parts(R kappa, int n, const R* __restrict__ sC, const R* __restrict__ sH,
                                            const R* y, R& u_out, R& G_out) {
  R u = R(0), G = R(0);
  if (D == 1) {
    R om = R(1) - y[0] * y[0];
    R pm2 = R(1), pm1 = R(2) * y[0];
    R cpsi = R(0);
#pragma unroll
    for (int p = 0; p < NMAX; ++p) {
      if (p < n) {
        R P;
        if (p == 0) P = R(1);
        else if (p == 1) P = R(2) * y[0];
        else { P = jac_ra<R>(p) * y[0] * pm1 - jac_rb<R>(p) * pm2; pm2 = pm1; pm1 = P; }
        R phi = om * P;
        R c = sC[p];
        u += c * phi;
        G += sH[p] * phi;
        cpsi += c * jac_lam<R>(p) * P;
      }
    }
    G -= kappa * cpsi;
  } else if (D == 2) {
    R phy[NMAX], psy[NMAX];
    basis<NMAX, R>(n, y[1], phy, psy);
    R omx = R(1) - y[0] * y[0];
    R pm2 = R(1), pm1 = R(2) * y[0];
    R cpsi = R(0);
    for (int p1 = 0; p1 < n; ++p1) {
      R P;
      if (p1 == 0) P = R(1);
      else if (p1 == 1) P = R(2) * y[0];
      else { P = jac_ra<R>(p1) * y[0] * pm1 - jac_rb<R>(p1) * pm2; pm2 = pm1; pm1 = P; }
      R phx = omx * P, psx = jac_lam<R>(p1) * P;
      const R* c = sC + p1 * NMAX;     // rows padded to NMAX entries
      const R* hh = sH + p1 * NMAX;
      // rows are 16-byte aligned and padded to NMAX: vector loads, two partial
      // sums per quantity (independent FMA chains)
      R a1 = R(0), a2 = R(0), a3 = R(0), b1 = R(0), b2 = R(0), b3 = R(0);
      if (sizeof(R) == 4) {
        const float4* c4 = reinterpret_cast<const float4*>(c);
        const float4* h4 = reinterpret_cast<const float4*>(hh);
#pragma unroll
        for (int v = 0; v < NMAX / 4; ++v) {
          const float4 cv = c4[v], hv = h4[v];
          const int p2 = 4 * v;
          a1 += (R)cv.x * phy[p2];     a2 += (R)cv.x * psy[p2];     a3 += (R)hv.x * phy[p2];
          b1 += (R)cv.y * phy[p2 + 1]; b2 += (R)cv.y * psy[p2 + 1]; b3 += (R)hv.y * phy[p2 + 1];
          a1 += (R)cv.z * phy[p2 + 2]; a2 += (R)cv.z * psy[p2 + 2]; a3 += (R)hv.z * phy[p2 + 2];
          b1 += (R)cv.w * phy[p2 + 3]; b2 += (R)cv.w * psy[p2 + 3]; b3 += (R)hv.w * phy[p2 + 3];
        }
      } else {
        const double2* c2 = reinterpret_cast<const double2*>(c);
        const double2* h2 = reinterpret_cast<const double2*>(hh);
#pragma unroll
        for (int v = 0; v < NMAX / 2; ++v) {
          const double2 cv = c2[v], hv = h2[v];
          const int p2 = 2 * v;
          a1 += (R)cv.x * phy[p2];     a2 += (R)cv.x * psy[p2];     a3 += (R)hv.x * phy[p2];
          b1 += (R)cv.y * phy[p2 + 1]; b2 += (R)cv.y * psy[p2 + 1]; b3 += (R)hv.y * phy[p2 + 1];
        }
      }
      a1 += b1; a2 += b2; a3 += b3;
      u += phx * a1;
      G += phx * a3;
      cpsi += psx * a1 + phx * a2;
    }
    G -= kappa * cpsi;
  }
  u_out = u;
  G_out = G;
}
// The Chebyshev basis phi_p = T_p - T_{p+2} (p < n) and its second derivatives
// at y, from T_{k+1} = 2y T_k - T_{k-1} and the recurrences of T' and T''.
template <int NMAX, typename R>
__device__ __forceinline__ void cheb_basis(int n, R y, R* phi, R* phi2) {
  R T[NMAX + 2], T2[NMAX + 2];
  R t1m = R(0), t1 = R(1);   // T'_{k-1}, T'_k
  T[0] = R(1); T2[0] = R(0);
  T[1] = y; T2[1] = R(0);
#pragma unroll
  for (int k = 1; k < NMAX + 1; ++k) {
    T[k + 1] = R(2) * y * T[k] - T[k - 1];
    const R t1n = R(2) * T[k] + R(2) * y * t1 - t1m;
    T2[k + 1] = R(4) * t1 + R(2) * y * T2[k] - T2[k - 1];
    t1m = t1;
    t1 = t1n;
  }
#pragma unroll
  for (int p = 0; p < NMAX; ++p) {
    phi[p] = (p < n) ? T[p] - T[p + 2] : R(0);
    phi2[p] = (p < n) ? T2[p] - T2[p + 2] : R(0);
  }
}

// u* and G = -d_t u* + kappa Delta u* at y from a slice in the Chebyshev basis
// (same layout as the Jacobi slices: C, H as coefficients of phi, d = 2 rows [p_x][p_y]).
template <int D, int NMAX, typename R>
__device__ __forceinline__ void slice_parts_cheb(R kappa, int n, const R* __restrict__ sC,
                                                 const R* __restrict__ sH, const R* y, R& u_out, R& G_out) {
  R px[NMAX], px2[NMAX];
  cheb_basis<NMAX, R>(n, y[0], px, px2);
  R u = R(0), G = R(0), lap = R(0);
  if (D == 1) {
#pragma unroll
    for (int p = 0; p < NMAX; ++p) {
      u += sC[p] * px[p];
      G += sH[p] * px[p];
      lap += sC[p] * px2[p];
    }
  } else {
    R py[NMAX], py2[NMAX];
    cheb_basis<NMAX, R>(n, y[1], py, py2);
    for (int p1 = 0; p1 < n; ++p1) {
      const R* c = sC + p1 * NMAX;
      const R* hh = sH + p1 * NMAX;
      R cu = R(0), cl = R(0), ch = R(0);
#pragma unroll
      for (int p2 = 0; p2 < NMAX; ++p2) {
        cu += c[p2] * py[p2];
        cl += c[p2] * py2[p2];
        ch += hh[p2] * py[p2];
      }
      u += px[p1] * cu;
      G += px[p1] * ch;
      lap += px2[p1] * cu + px[p1] * cl;
    }
  }
  u_out = u;
  G_out = G + kappa * lap;
}

template <int D, int NMAX, typename R>
__device__ __forceinline__ R residual_at(const InstanceParams& ip, R kappa, int n, const R* __restrict__ sC,
                                         const R* __restrict__ sH, const R* y, R Tt, R dTt) {
  R u, G;
  slice_parts<D, NMAX, R>(kappa, n, sC, sH, y, u, G);
  return reaction<R>(ip, u) + source<D, R>(ip, kappa, y, Tt, dTt) + G;
}

// ---------------------------------------------------------------- fractional
// The fractional case (Section 4, Ex. 2; d = 1): L = kappa (-Delta)^{alpha/2},
// basis phi_p = (1-y^2)^a P_p^{(a,a)} (a = alpha/2) with
// (-Delta)^{alpha/2} phi_p = lam_p P_p^{(a,a)}.  `tab` is the plan's table
// (recurrence coefficients, lam_p, the sine series of Ex. 2's solution; layout
// kFrac* in spmc_tables.h).
constexpr int kFracRaD = 0, kFracRbD = 40, kFracLamD = 80, kFracSinD = 120, kFracAD = 160, kFracAlphaD = 161,
              kFracGammaD = 162, kFracLnBD = 163, kFracRpD = 164, kFracRqD = 244, kFracSeriesD = 80,
              kFracModesD = 40;

// I_u(a, 1-a) of the jump law, regularised incomplete beta by its series
// I_x(p,q) = x^p (1-x)^q / (p B(p,q)) sum_k prod_{i<k} x (p+q+i)/(p+1+i)
// (x <= 1/2; 1 - I_{1-x}(q, p) above); rp, rq hold the ratios (p+q+i)/(p+1+i)
// for (p, q) = (a, 1-a) and (1-a, a) (the plan's table, or a copy of it in
// the sweep's precision), lnB = ln B(a, 1-a).  R = double for the FP64 sweep,
// float for the FP32 one.
template <typename R, typename T>
__device__ __forceinline__ R ibeta_jump(R x, R a, R lnB, const T* __restrict__ rp, const T* __restrict__ rq) {
  const bool flip = x > R(0.5);
  const R p = flip ? R(1) - a : a, q = flip ? a : R(1) - a;
  const T* r = flip ? rq : rp;
  if (flip) x = R(1) - x;
  if (!(x > R(0))) return flip ? R(1) : R(0);
  const R pre = exp(p * log(x) + q * log1p(-x) - lnB) / p;
  const R eps = sizeof(R) == 8 ? R(1e-18) : R(1e-9);
  R term = R(1), sum = R(1);
  for (int k = 0; k < kFracSeriesD; ++k) {
    term *= (R)r[k] * x;
    sum += term;
    if (term < eps * sum) break;
  }
  const R v = pre * sum;
  return flip ? R(1) - v : v;
}

// Exit distance from a ball of radius r of the alpha-stable process started at
// its centre: r / sqrt(U), U ~ Beta(a, 1-a) (the Blumenthal-Getoor-Ray law),
// U = I^{-1}_{1-omega}(a, 1-a) by Newton's method kept inside a bisection bracket.
template <typename R, typename T>
__device__ __forceinline__ R stable_jump(R r, R a, R lnB, const T* __restrict__ rp, const T* __restrict__ rq,
                                         double omega) {
  const R p = a, q = R(1) - a;
  const R target = (R)(1.0 - omega);
  const R tol = sizeof(R) == 8 ? R(1e-16) : R(1e-7);
  R lo = R(0), hi = R(1);
  // start from the leading term at the nearer end
  R x = exp((log(target) + log(p) + lnB) / p);
  if (!(x < R(0.5))) x = R(1) - exp((log1p(-target) + log(q) + lnB) / q);
  if (!(x > R(0) && x < R(1))) x = R(0.5);
  for (int it = 0; it < 100; ++it) {
    const R F = ibeta_jump<R, T>(x, a, lnB, rp, rq) - target;
    if (F < R(0)) lo = x; else hi = x;
    const R dF = exp((p - R(1)) * log(x) + (q - R(1)) * log1p(-x) - lnB);
    R xn = x - F / dF;
    if (!(xn > lo && xn < hi)) xn = R(0.5) * (lo + hi);
    const bool done = fabs(xn - x) <= tol * xn || hi - lo <= tol * R(0.1);
    x = xn;
    if (done) break;
  }
  return r / sqrt(x);
}

// The residual at y (|y| < 1) from a slice of the fractional case:
//   u* = sum C_p phi_p(y),  G = sum H_p phi_p(y) - kappa sum C_p lam_p P_p(y),
//   r = f(u*) + f_add + G,
// f_add of the fractional examples: 6, u = (1-y^2)^a sin(y) T(t) (Ex. 2),
// (-Delta)^{alpha/2} u = T sum s_p lam_p P_p; 7, u = T (1-y^2)^a (1 + P_1/2), T = 1+t.
template <typename R>
__device__ __forceinline__ R residual_frac(const InstanceParams& ip, R kappa, int n, const R* __restrict__ sC,
                                           const R* __restrict__ sH, R y, R Tt, R dTt,
                                           const double* __restrict__ tab) {
  const R a = (R)tab[kFracAD];
  const R wgt = pow(R(1) - y * y, a);
  R pm2 = R(1), pm1 = (a + R(1)) * y;
  R u = R(0), G = R(0), cl = R(0), fr = R(0);
  const bool sine = ip.ex_kind == 6;
  const int top = sine ? kFracModesD : n;
  for (int p = 0; p < top; ++p) {
    R P;
    if (p == 0) P = R(1);
    else if (p == 1) P = pm1;
    else { P = (R)tab[kFracRaD + p] * y * pm1 - (R)tab[kFracRbD + p] * pm2; pm2 = pm1; pm1 = P; }
    const R lam = (R)tab[kFracLamD + p];
    if (p < n) {
      u += sC[p] * P;
      G += sH[p] * P;
      cl += sC[p] * lam * P;
    }
    if (sine) fr += (R)tab[kFracSinD + p] * lam * P;
  }
  u *= wgt;
  G = G * wgt - kappa * cl;
  R fadd = R(0);
  if (sine) {
    const R ws = wgt * sin(y);
    fadd = dTt * ws + kappa * Tt * fr - reaction<R>(ip, Tt * ws);
  } else if (ip.ex_kind == 7) {
    const R P1 = (a + R(1)) * y;
    const R lam0 = (R)tab[kFracLamD], lam1 = (R)tab[kFracLamD + 1];
    const R shape = wgt * (R(1) + R(0.5) * P1);
    fadd = dTt * shape + kappa * Tt * (lam0 + R(0.5) * lam1 * P1) - reaction<R>(ip, Tt * shape);
  }
  return reaction<R>(ip, u) + fadd + G;
}

}  // namespace spmc

namespace spmc {

// g(u) = df/ds and g'(u) for f = s g(u).
__device__ __forceinline__ void reaction_g(const InstanceParams& ip, double u, double* g, double* dg) {
  if (ip.f_kind == 1) { *g = sin(u); *dg = cos(u); return; }
  *g = ip.fc[0] + u * (ip.fc[1] + u * (ip.fc[2] + u * ip.fc[3]));
  *dg = ip.fc[1] + u * (2.0 * ip.fc[2] + 3.0 * u * ip.fc[3]);
}

// Adjoint of one quadrature term at y with weight cw = lambda_i w_p / M:
// u* from the forward slice C, then the rank-1 scatters
//   acc[0] += cw s g'(u*) Phi(y),  acc[1] += cw Phi(y),  acc[2] += cw Psi(y)
// in coefficient order (x_1 fastest), Phi = prod phi, Psi = sum over one axis of
// psi with phi on the others.  Returns cw (g(u*) - g(u_ex)) = the term's
// derivative in the reaction scale s (the source f_add depends on s through
// f(u_ex)).
template <int D, int NMAX, typename R>
__device__ __forceinline__ double adjoint_at(const InstanceParams& ip, int n, const R* __restrict__ sC, const R* y,
                                             double cw, double* acc, int S, R Tt) {
  R phx[NMAX], psx[NMAX];
  basis<NMAX, R>(n, y[0], phx, psx);
  double u = 0.0;
  if (D == 1) {
    for (int p = 0; p < n; ++p) u += (double)sC[p] * (double)phx[p];
  } else {
    R phy[NMAX], psy[NMAX];
    basis<NMAX, R>(n, y[1], phy, psy);
    for (int p1 = 0; p1 < n; ++p1) {
      double a = 0.0;
      for (int p2 = 0; p2 < n; ++p2) a += (double)sC[p1 * NMAX + p2] * (double)phy[p2];
      u += (double)phx[p1] * a;
    }
  }
  double g, dg;
  reaction_g(ip, u, &g, &dg);
  const double al = cw * ip.f_scale * dg;
  if (D == 1) {
    for (int p = 0; p < n; ++p) {
      atomicAdd(&acc[p], al * (double)phx[p]);
      atomicAdd(&acc[S + p], cw * (double)phx[p]);
      atomicAdd(&acc[2 * S + p], cw * (double)psx[p]);
    }
  } else {
    R phy[NMAX], psy[NMAX];
    basis<NMAX, R>(n, y[1], phy, psy);
    for (int p2 = 0; p2 < n; ++p2)
      for (int p1 = 0; p1 < n; ++p1) {
        const int p = p1 + n * p2;
        const double ff = (double)phx[p1] * (double)phy[p2];
        atomicAdd(&acc[p], al * ff);
        atomicAdd(&acc[S + p], cw * ff);
        atomicAdd(&acc[2 * S + p], cw * ((double)psx[p1] * (double)phy[p2] + (double)phx[p1] * (double)psy[p2]));
      }
  }
  double gex = 0.0;
  if (ip.ex_kind != 0) {
    // u_ex at y: time factor Tt times the spatial closed form
    double prod = 1.0;
    for (int e = 0; e < D; ++e) {
      const double ye = (double)y[e];
      if (ip.ex_kind == 1) prod *= sinpi(ye);
      else if (ip.ex_kind == 2) prod *= cospi(0.5 * ye);
      else prod *= (1.0 - ye * ye) * (1.0 + ye);
    }
    double dgx;
    reaction_g(ip, (double)Tt * prod, &gex, &dgx);
  }
  return cw * (g - gex);
}

}  // namespace spmc
