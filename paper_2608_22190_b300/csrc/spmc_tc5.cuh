// spmc_tc5.cuh -- the 5-D residual evaluation of the event sweep on the tensor
// cores (tcgen05, TMEM, bulk copies), FP32 sweep.
//
// With P_a the Jacobi P^{(1,1)} polynomials, o_e = 1 - y_e^2, phi_a = o P_a and
// psi_a = lam_a P_a (lam_a = (a+1)(a+2)), the residual at a point y of the
// tensor-product expansion (Eq. u_N and the Remark on tensor products) needs
//     T0 = <C, P(y1) x ... x P(y5)>,  T_e = the same with lam on axis e,
//     TH = <H, P(y1) x ... x P(y5)>,
// from which u* = prod o T0, -d_t u* = prod o TH and
// -Delta u* = sum_e (prod_{e' != e} o_e') T_e.  The contraction is
// sum-factorised: stage 1 contracts the axes (p1, p2) -- a K = 64 product of
// the event's row A = P(y1) x P(y2) with the slice's tensors viewed as 512 rows
// (p3, p4, p5) of 64 -- on the tensor cores, for the four tensors
// [C | Lam_1 C | Lam_2 C | H] (the lam weights of axes 1 and 2 folded into the
// tensors); stage 2 contracts (p3, p4, p5) on the FP32 pipe, with the lam
// weights of axes 3-5 applied there.  TF32 with the 3-term split
// (A_hi B_hi + A_hi B_lo + A_lo B_hi), FP32 accumulation in TMEM.
//
// Tensors of every slice are written once per iteration by slice5_tc_kernel in
// the no-swizzle K-major core-matrix layout (spmc_tc.cuh), hi and lo parts
// apart, so that 128 rows of one tensor part are 32 KB of contiguous memory and
// arrive in shared memory by one bulk copy.  Modes are padded to 8 per axis.
#pragma once
#include <cstdint>

#include "spmc_tc.cuh"

namespace spmc {

struct Tc5 {
  static constexpr int NP = 8;                        // modes per axis (padded)
  static constexpr int K = 64;                        // (p1, p2)
  static constexpr int KC = K / 4;                    // 16-byte chunks per row
  static constexpr uint32_t SBO = KC * 128;           // bytes between 8-row groups
  static constexpr uint32_t LBO = 128;
  static constexpr int ROWS = 512;                    // (p3, p4, p5)
  static constexpr int CROWS = 128;                   // rows of one chunk = the MMA's N
  static constexpr int NCHUNK = 16;                   // 4 tensors x 4 chunks
  static constexpr uint32_t PART = ROWS * K * 4;      // one tensor, hi or lo: 128 KB
  static constexpr uint32_t CHUNK_BYTES = CROWS * K * 4;   // 32 KB
  static constexpr size_t SLICE_BYTES = 8 * (size_t)PART;  // [tensor][hi, lo]: 1 MB
  static constexpr uint32_t A_BYTES = 128 * K * 4;    // 32 KB (hi or lo)
  static constexpr int SMEM = 2 * A_BYTES + 4 * CHUNK_BYTES + 256 + 128;   // A, B[2][hi, lo], barriers, alignment
  static constexpr int EV_CHUNK = 2048;               // events per block
  static constexpr int TM_COLS = 256;                 // two 128-column accumulators
};

// One block per slice: C = sum_q cu_q L_q(xi(tau)), H = -sum_q ct_q L_q(xi(tau))
// (FP64), then C, lam_{p1} C, lam_{p2} C and H rounded to FP32 and split into
// TF32 hi + lo, in the core-matrix layout of a [512 x 64] K-major tile each.
__global__ void __launch_bounds__(256) slice5_tc_kernel(const TimeNode* __restrict__ tn,
                                                        const long long* __restrict__ slice_node,
                                                        const InstInterval* __restrict__ inst_of_node,
                                                        const double* __restrict__ coef,
                                                        const InstanceParams* __restrict__ ip,
                                                        unsigned char* __restrict__ tcs,
                                                        SliceInfo* __restrict__ sinfo, int n, int n_sub,
                                                        double t_off, const int* __restrict__ abort) {
  __shared__ double L[41];
  if (abort && *abort) return;
  const long long s = blockIdx.x;
  const long long ti = slice_node[s];
  const TimeNode node = tn[ti];
  const InstInterval w = inst_of_node[ti];
  const int m = (int)(s - node.slice_base);
  const int S = n * n * n * n * n;
  const double sdur = __dsub_rn(node.t_node, node.t0);
  const double delta = __ddiv_rn(sdur, (double)node.nstar);
  const double sub = __ddiv_rn(delta, (double)n_sub);
  const double tau = __dsub_rn(node.t_node, __dmul_rn((double)m + t_off, sub));
  if (threadIdx.x == 0) {
    const double xi = (2.0 * tau - node.t0 - (node.t0 + node.h)) / node.h;
    L[0] = 1.0;
    if (node.Mt >= 1) L[1] = xi;
    for (int k = 1; k < node.Mt; ++k) L[k + 1] = ((2.0 * k + 1.0) * xi * L[k] - k * L[k - 1]) / (k + 1.0);
    const InstanceParams P = ip[node.inst];
    SliceInfo si;
    si.tau = tau;
    si.kind = 0;
    if (P.ex_kind == 3) { si.Tt = 1.0 + tau + tau * tau; si.dTt = 1.0 + 2.0 * tau; }
    else if (P.ex_kind == 1 || P.ex_kind == 2) { si.Tt = exp(-P.ex_beta * tau); si.dTt = -P.ex_beta * si.Tt; }
    else { si.Tt = 0.0; si.dTt = 0.0; }
    sinfo[s] = si;
  }
  __syncthreads();
  const double* cu = coef + w.c_off;
  const double* ct = cu + (long long)(node.Mt + 1) * S;
  unsigned char* out = tcs + (size_t)s * Tc5::SLICE_BYTES;
  for (int idx = threadIdx.x; idx < Tc5::ROWS * Tc5::K; idx += blockDim.x) {
    const int p1 = idx & 7, p2 = (idx >> 3) & 7, p3 = (idx >> 6) & 7, p4 = (idx >> 9) & 7, p5 = idx >> 12;
    double c = 0.0, h = 0.0;
    if (p1 < n && p2 < n && p3 < n && p4 < n && p5 < n) {
      const long long pl = p1 + (long long)n * (p2 + n * (p3 + n * (p4 + n * p5)));
      for (int q = 0; q <= node.Mt; ++q) {
        c += cu[(long long)q * S + pl] * L[q];
        h -= ct[(long long)q * S + pl] * L[q];
      }
    }
    const double vals[4] = {c, jac_lam<double>(p1) * c, jac_lam<double>(p2) * c, h};
    const uint32_t off = tc::kmajor_offset(idx >> 6, idx & 63, Tc5::KC);   // row (p3, p4, p5), k (p1, p2)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float hi, lo;
      tc::split_tf32((float)vals[t], hi, lo);
      *reinterpret_cast<float*>(out + (size_t)(2 * t) * Tc5::PART + off) = hi;
      *reinterpret_cast<float*>(out + (size_t)(2 * t + 1) * Tc5::PART + off) = lo;
    }
  }
}

namespace tc {
// 32 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// expect `bytes` more transaction bytes on the barrier (with this thread's arrival)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global memory to this CTA's shared memory, completing on the barrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}
}  // namespace tc

// Events in fixed chunks of EV_CHUNK (a chunk may span slices); per slice
// segment, tiles of 128 events (one per thread = one TMEM lane).  Per tile the
// 16 B chunks (4 tensors x 4 groups of 128 rows) flow through a two-stage
// pipeline: the bulk copy of chunk c + 1 and the MMAs of chunk c + 1 (into the
// other TMEM accumulator) run while the threads contract chunk c on the FP32 pipe.
// Every wait is bounded: on time-out the block records status bit 8, waits once
// more for what it issued, frees its TMEM and returns.
__global__ void __launch_bounds__(128, 1) eval5_tc_kernel(const long long* __restrict__ slice_node,
                                                          const TimeNode* __restrict__ tn,
                                                          const InstanceParams* __restrict__ ipt,
                                                          const unsigned char* __restrict__ tcs,
                                                          const SliceInfo* __restrict__ sinfo,
                                                          const unsigned int* __restrict__ starts,
                                                          const Event5<float>* __restrict__ events,
                                                          unsigned long long* __restrict__ acc, int n, int S,
                                                          long long n_slices, double kappa_d,
                                                          const unsigned long long* __restrict__ n_events_p,
                                                          int* status, const int* __restrict__ abort) {
  extern __shared__ unsigned char sm5raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*abort) return;
  const unsigned long long n_events = *n_events_p;
  const unsigned long long c0 = (unsigned long long)blockIdx.x * Tc5::EV_CHUNK;
  if (c0 >= n_events) return;
  const unsigned long long c1 = min(c0 + (unsigned long long)Tc5::EV_CHUNK, n_events);

  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm5raw) + 127) & ~uintptr_t(127));
  unsigned char* Ahi = base;
  unsigned char* Alo = base + Tc5::A_BYTES;
  unsigned char* Bb = base + 2 * Tc5::A_BYTES;       // [buffer][hi, lo]
  uint64_t* bar_b = reinterpret_cast<uint64_t*>(Bb + 4 * Tc5::CHUNK_BYTES);   // [2] chunk landed
  uint64_t* bar_m = bar_b + 2;                                                 // [2] MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_m + 2);

  if (warp == 0) {
    tc::tmem_alloc(tslot, Tc5::TM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar_b[0], 1); tc::mbar_init(&bar_b[1], 1);
    tc::mbar_init(&bar_m[0], 1); tc::mbar_init(&bar_m[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
  constexpr uint32_t idesc = tc::idesc_tf32(128, Tc5::CROWS);
  const uint32_t aH = tc::smem_u32(Ahi), aL = tc::smem_u32(Alo);
  const float kappa = (float)kappa_d;
  uint32_t ph_b[2] = {0u, 0u}, ph_m[2] = {0u, 0u};
  int pend_b[2] = {0, 0}, pend_m[2] = {0, 0};        // issued and not yet waited for
  bool ok = true;

  auto load_chunk = [&](const unsigned char* gsl, int c) {   // thread 0
    const int t = c >> 2, cc = c & 3, b = c & 1;
    unsigned char* dh = Bb + (2 * b) * Tc5::CHUNK_BYTES;
    unsigned char* dl = dh + Tc5::CHUNK_BYTES;
    const unsigned char* sh = gsl + (size_t)(2 * t) * Tc5::PART + (size_t)cc * Tc5::CHUNK_BYTES;
    const unsigned char* sl = gsl + (size_t)(2 * t + 1) * Tc5::PART + (size_t)cc * Tc5::CHUNK_BYTES;
    tc::mbar_expect_tx(&bar_b[b], 2 * Tc5::CHUNK_BYTES);
    tc::bulk_g2s(dh, sh, Tc5::CHUNK_BYTES, &bar_b[b]);
    tc::bulk_g2s(dl, sl, Tc5::CHUNK_BYTES, &bar_b[b]);
  };
  auto issue_mma = [&](int c) {   // thread 0: D[buffer c&1] = A B_c^T (3-term split)
    const int b = c & 1;
    const uint32_t bH = tc::smem_u32(Bb + (2 * b) * Tc5::CHUNK_BYTES), bL = bH + Tc5::CHUNK_BYTES;
    const uint32_t d = tbase + (uint32_t)(b * Tc5::CROWS);
    tc::fence_after();
#pragma unroll
    for (int s = 0; s < Tc5::K / 8; ++s) {
      const uint32_t ko = (uint32_t)s * 256;
      tc::mma_tf32(d, tc::sdesc(aL + ko, Tc5::LBO, Tc5::SBO), tc::sdesc(bH + ko, Tc5::LBO, Tc5::SBO), idesc,
                   s > 0 ? 1u : 0u);
      tc::mma_tf32(d, tc::sdesc(aH + ko, Tc5::LBO, Tc5::SBO), tc::sdesc(bL + ko, Tc5::LBO, Tc5::SBO), idesc, 1u);
      tc::mma_tf32(d, tc::sdesc(aH + ko, Tc5::LBO, Tc5::SBO), tc::sdesc(bH + ko, Tc5::LBO, Tc5::SBO), idesc, 1u);
    }
    tc::mma_commit(&bar_m[b]);
  };
  auto wait_b = [&](int b) {
    if (!tc::mbar_wait_bounded(&bar_b[b], ph_b[b])) ok = false;
    ph_b[b] ^= 1u;
    pend_b[b] = 0;
  };
  auto wait_m = [&](int b) {
    if (!tc::mbar_wait_bounded(&bar_m[b], ph_m[b])) ok = false;
    ph_m[b] ^= 1u;
    pend_m[b] = 0;
  };

  unsigned long long pos = c0;
  while (pos < c1 && ok) {
    // the slice holding event pos: the last s with starts[s S] <= pos
    long long lo_s = 0, hi_s = n_slices - 1;
    while (lo_s < hi_s) {
      const long long mid = (lo_s + hi_s + 1) >> 1;
      if ((unsigned long long)starts[mid * S] <= pos) lo_s = mid; else hi_s = mid - 1;
    }
    const long long sidx = lo_s;
    const unsigned long long s_end = (sidx + 1 < n_slices) ? (unsigned long long)starts[(sidx + 1) * S] : n_events;
    const unsigned long long g1 = min(c1, s_end);
    const unsigned char* gsl = tcs + (size_t)sidx * Tc5::SLICE_BYTES;
    const long long ti = slice_node[sidx];
    const TimeNode node = tn[ti];
    const InstanceParams ip = ipt[node.inst];
    const SliceInfo si = sinfo[sidx];
    const unsigned int key0 = (unsigned int)(sidx * S);

    for (unsigned long long t0 = pos; t0 < g1 && ok; t0 += 128) {
      const unsigned long long ei = t0 + tid;
      const bool has = ei < g1;
      float y[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, w = 0.f;
      unsigned int key = 0xffffffffu;
      if (has) {
        const Event5<float> e = events[ei];
#pragma unroll
        for (int d = 0; d < 5; ++d) y[d] = e.y[d];
        w = e.w;
        key = e.key;
      }
      // P_p(y_d), p < 8 (zero for p >= n)
      float P[5][8];
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        float pm2 = 1.f, pm1 = 2.f * y[d];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          float v;
          if (p == 0) v = 1.f;
          else if (p == 1) v = 2.f * y[d];
          else { v = jac_ra<float>(p) * y[d] * pm1 - jac_rb<float>(p) * pm2; pm2 = pm1; pm1 = v; }
          P[d][p] = p < n ? v : 0.f;
        }
      }
      // A row: P(y1) x P(y2), k = p1 + 8 p2, split hi / lo
#pragma unroll
      for (int c = 0; c < Tc5::KC; ++c) {
        float hv[4], lv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = 4 * c + q;
          tc::split_tf32(P[0][k & 7] * P[1][k >> 3], hv[q], lv[q]);
        }
        const uint32_t off = tc::kmajor_offset(tid, 4 * c, Tc5::KC);
        *reinterpret_cast<float4*>(Ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4*>(Alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) { load_chunk(gsl, 0); pend_b[0] = 1; }
      wait_b(0);
      if (tid == 0) { issue_mma(0); }
      pend_m[0] = 1;
      float T[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, TH = 0.f;   // T[0] = T0, T[1..5] = T_1..T_5
      for (int c = 0; c < Tc5::NCHUNK; ++c) {
        const int b = c & 1;
        if (c + 1 < Tc5::NCHUNK) {
          if (tid == 0) load_chunk(gsl, c + 1);   // its buffer's last MMA (chunk c - 1) has completed
          pend_b[b ^ 1] = 1;
        }
        wait_m(b);                                // MMA of chunk c done
        if (c + 1 < Tc5::NCHUNK) {
          wait_b(b ^ 1);
          if (tid == 0) issue_mma(c + 1);         // into the other accumulator, read by chunk c - 1's contraction
          pend_m[b ^ 1] = 1;
        }
        tc::fence_after();
        // stage 2 of chunk c: rows (p3, p4, p5) with p5 in {2 cc, 2 cc + 1}
        const int t = c >> 2, cc = c & 3;
        float c0v = 0.f, c3v = 0.f, c4v = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float v[32];
          tc::tmem_ld32(lane_base + (uint32_t)(b * Tc5::CROWS + 32 * j), v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int p4 = 4 * (j & 1) + q;
            float a = 0.f, bl = 0.f;
#pragma unroll
            for (int p3 = 0; p3 < 8; ++p3) {
              a = fmaf(v[8 * q + p3], P[2][p3], a);
              if (t == 0) bl = fmaf(v[8 * q + p3], jac_lam<float>(p3) * P[2][p3], bl);
            }
            c0v = fmaf(a, P[3][p4], c0v);
            if (t == 0) {
              c3v = fmaf(bl, P[3][p4], c3v);
              c4v = fmaf(a, jac_lam<float>(p4) * P[3][p4], c4v);
            }
          }
          if (j & 1) {   // both halves of p4 done: close this p5
            const int p5 = 2 * cc + (j >> 1);
            const float f5 = P[4][p5], g5 = jac_lam<float>(p5) * P[4][p5];
            if (t == 0) {
              T[0] = fmaf(c0v, f5, T[0]);
              T[3] = fmaf(c3v, f5, T[3]);
              T[4] = fmaf(c4v, f5, T[4]);
              T[5] = fmaf(c0v, g5, T[5]);
            } else if (t == 3) {
              TH = fmaf(c0v, f5, TH);
            } else {
              T[t] = fmaf(c0v, f5, T[t]);
            }
            c0v = c3v = c4v = 0.f;
          }
        }
        tc::fence_before();
        const bool all_ok = !__syncthreads_or(!ok);   // this accumulator may now be overwritten
        tc::fence_after();
        if (!all_ok) { ok = false; break; }
      }
      if (!ok) break;
      // the residual r = f(u*) + f_add + (-d_t u*) + kappa Delta u*
      __int128 val = 0;
      if (has) {
        float o[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) o[d] = 1.f - y[d] * y[d];
        const float po = o[0] * o[1] * o[2] * o[3] * o[4];
        float s1 = 0.f;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          float pr = T[d + 1];
#pragma unroll
          for (int d2 = 0; d2 < 5; ++d2) if (d2 != d) pr *= o[d2];
          s1 += pr;
        }
        const float u = po * T[0];
        const float res = reaction<float>(ip, u) + source<5, float>(ip, kappa, y, (float)si.Tt, (float)si.dTt) +
                          po * TH - kappa * s1;
        if (!fix_from_float(w * res, val)) atomicOr(status, 1);
      }
      // per-node sums (exact): events are sorted by key, so equal keys are adjacent lanes
      val = warp_run_sum(val, key, (unsigned int)lane);
      const unsigned int kprev = __shfl_up_sync(0xffffffffu, key, 1);
      if (has && (lane == 0 || kprev != key)) fix_atomic_add(acc + 4 * (ti * S + (long long)(key - key0)), val);
      __syncthreads();   // the A tile is rewritten by the next tile
    }
    pos = g1;
  }
  if (!__syncthreads_and(ok)) {
    // a copy or an MMA did not complete in time: report, give what is still
    // in flight one more bounded wait, stop
    if (tid == 0) atomicOr(status, 8);
    for (int b = 0; b < 2; ++b) {
      if (pend_b[b]) tc::mbar_wait_bounded(&bar_b[b], ph_b[b]);
      if (pend_m[b]) tc::mbar_wait_bounded(&bar_m[b], ph_m[b]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tbase, Tc5::TM_COLS);
  }
}

}  // namespace spmc
