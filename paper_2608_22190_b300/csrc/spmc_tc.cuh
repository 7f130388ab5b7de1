// spmc_tc.cuh -- 5th-generation tensor-core pieces (tcgen05, TMEM, mbarrier) in
// inline PTX for sm_103a, and the tensor-core evaluation of the event sweep.
//
// Operands are written by the CTA's threads straight into shared memory in the
// no-swizzle K-major core-matrix layout: a core matrix is 8 rows x 16 bytes
// (8 x 4 TF32 values) stored as 128 contiguous bytes; the core matrices of a
// row group follow each other along K (128 bytes apart), and row groups are
// KC * 128 bytes apart (KC = 16-byte chunks per row).  Element (row, k) of a
// K-major tile therefore sits at byte
//     (row / 8) * KC * 128 + (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4.
#pragma once
#include <cstdint>

#include "spmc_events.cuh"

namespace spmc {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// TMEM allocation (one full warp executes these)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ordering between thread barriers and tcgen05 operations
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of the barrier; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity, uint32_t max_tries = 1u << 24) {
  for (uint32_t t = 0; t < max_tries; ++t)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

// named barrier `id` (1..15) over `n` threads (a multiple of 32)
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// named barrier `id` over `n` threads that also ORs `pred` over them
__device__ __forceinline__ bool named_sync_or(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\n"
      "setp.ne.u32 p, %1, 0;\n"
      "bar.red.or.pred q, %2, %3, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// Shared-memory matrix descriptor: no swizzle, base offset 0, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, M x N x 8, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* m) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
               : "memory");
}

// 8 consecutive 32-bit columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Round to TF32 (nearest, ties away) and the FP32 remainder: x = hi + lo exactly.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  hi = __uint_as_float(u);
  lo = x - hi;
}

// byte offset of element (row, k) in a K-major no-swizzle tile with KC 16-byte chunks per row
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k, int KC) {
  return (uint32_t)((row >> 3) * KC * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Tensor-core evaluation of the events of one time slice (d = 2, FP32 sweep).
//
// With P_a the Jacobi P^{(1,1)} polynomials, phi_a(x) = (1 - x^2) P_a(x) and
// psi_a(x) = lam_a P_a(x) (lam_a = (a+1)(a+2)), the residual at an event
// (x, y) needs the four bilinear forms
//     sC = P(x)^T C P(y),  sH = P(x)^T H P(y),
//     sL = P(x)^T (Lam C) P(y),  sR = P(x)^T (C Lam) P(y),
// from which
//     u = ox oy sC,   G = ox oy sH - kappa (oy sL + ox sR),   ox = 1 - x^2, oy = 1 - y^2.
// For a tile of 128 events the left products P(x)^T [C | H | Lam C | C Lam]
// form one (128 x K) x (K x 4 NMAX) matrix product, run on the tensor cores in
// TF32 with the 3-term split (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32
// accumulation in TMEM), which keeps about FP32 accuracy.  Each thread owns one
// event = one TMEM lane: it writes its row of A, then contracts its TMEM row
// with P(y) on the FP32 pipe.
//
// One block per SM holds all 512 TMEM columns and NT tile groups of 128
// threads (five at NMAX <= 24: N columns each); each group has its own A rows,
// TMEM accumulator and mbarrier, and works through the tiles of the current
// slice segment independently of the others (named barriers), so that while one
// group waits for its products the others write rows or finish residuals.  The
// groups share the slice's B operand, rebuilt at segment boundaries.  The
// epilogue's dependent FP32 chains are what the warps wait on most, so the
// kernel is built for as many groups as TMEM holds (registers capped at 96).
template <int NMAX>
struct TcGeom {
  static constexpr int K = NMAX;                 // contraction length (a multiple of 8)
  static constexpr int N = 4 * NMAX;             // [C | H | Lam C | C Lam]
  static constexpr int KC = K / 4;               // 16-byte chunks per row
  static constexpr uint32_t SBO = KC * 128;      // bytes between 8-row groups
  static constexpr uint32_t LBO = 128;           // bytes between K-adjacent core matrices
  static constexpr int A_BYTES = 128 * K * 4;    // one tile's rows, hi or lo
  static constexpr int B_BYTES = N * K * 4;
  static constexpr int NT_FIT = 512 / N;         // accumulators that fit the SM's 512 TMEM columns
  static constexpr int NT = NT_FIT < 5 ? NT_FIT : 5;   // tile groups per block (one block per SM)
  static constexpr int THREADS = 128 * NT;
  static constexpr int TM_STRIDE = N;            // TMEM columns per group, inside one 512-column allocation
  static constexpr int TM_COLS = 512;
  static constexpr int BLOCKS_PER_SM = 1;
  static constexpr int SMEM = 2 * NT * A_BYTES + 2 * B_BYTES + 8 * NT + 16;   // A, B, mbarriers, TMEM slot
  static constexpr int CHUNK = 16384;            // events per block and step of the block loop
};

// row `row` of A: P_a(x), a < K (zero for a >= n unless FULL, n = K), split
// hi / lo, into the K-major tile pair (hi, lo)
template <int NMAX, bool FULL>
__device__ __forceinline__ void write_a_row(unsigned char* hi, unsigned char* lo, int row, float x, int n) {
  constexpr int KC = TcGeom<NMAX>::KC;
  float pm2 = 1.f, pm1 = 2.f * x;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    float hv[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = 4 * c + q;
      float P;
      if (a == 0) P = 1.f;
      else if (a == 1) P = 2.f * x;
      else { P = jac_ra<float>(a) * x * pm1 - jac_rb<float>(a) * pm2; pm2 = pm1; pm1 = P; }
      tc::split_tf32((FULL || a < n) ? P : 0.f, hv[q], lv[q]);
    }
    const uint32_t off = tc::kmajor_offset(row, 4 * c, KC);
    *reinterpret_cast<float4*>(hi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(lo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

// Events in chunks of CHUNK; block b takes chunks b, b + G, ... (G = grid
// size, a multiple of the SM count), so the grid is one resident wave.  A chunk
// may span slices: its slice segments are processed in turn, the tiles of a
// segment dealt round-robin to the block's groups.
template <int NMAX, bool FULL>
__global__ void __launch_bounds__(TcGeom<NMAX>::THREADS, TcGeom<NMAX>::BLOCKS_PER_SM) eval_events_tc_kernel(
    const long long* __restrict__ slice_node, const TimeNode* __restrict__ tn, const InstanceParams* __restrict__ ipt,
    const float* __restrict__ slices, const SliceInfo* __restrict__ sinfo, const unsigned int* __restrict__ starts,
    const Event<float>* __restrict__ events, unsigned long long* __restrict__ acc, int n, int S, long long n_slices,
    long long sl_stride, int half, double kappa_d, int direct, const unsigned long long* __restrict__ n_events_p,
    int* status, const int* __restrict__ abort) {
  using Gm = TcGeom<NMAX>;
  constexpr int K = Gm::K, N = Gm::N, KC = Gm::KC, NT = Gm::NT;
  extern __shared__ __align__(1024) unsigned char sm_tc[];
  unsigned char* Abuf = sm_tc;                                 // [group][hi, lo]
  unsigned char* Bhi = Abuf + 2 * NT * Gm::A_BYTES;
  unsigned char* Blo = Bhi + Gm::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + Gm::B_BYTES);   // [group]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + NT);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = tid >> 7, gt = tid & 127;
  if (*abort) return;
  const unsigned long long n_events = *n_events_p;
  if ((unsigned long long)blockIdx.x * Gm::CHUNK >= n_events) return;

  if (warp == 0) {
    tc::tmem_alloc(tslot, Gm::TM_COLS);
    tc::tmem_relinquish();
  }
  if (gt == 0) tc::mbar_init(mbar + grp, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tcol = *tslot + (uint32_t)(grp * Gm::TM_STRIDE);
  const uint32_t lane_base = tcol + ((uint32_t)((warp & 3) * 32) << 16);
  constexpr uint32_t idesc = tc::idesc_tf32(128, N);
  const uint32_t ah = tc::smem_u32(Abuf + 2 * grp * Gm::A_BYTES), al = ah + Gm::A_BYTES;
  const uint32_t bHi = tc::smem_u32(Bhi), bLo = tc::smem_u32(Blo);
  unsigned char* Ah = Abuf + 2 * grp * Gm::A_BYTES;
  unsigned char* Al = Ah + Gm::A_BYTES;
  const float kappa = (float)kappa_d;
  uint32_t phase = 0;
  bool ok = true;          // false: a time-out was seen (voted over the group, then over the block)
  bool timed_out = false;  // this group's last MMA did not complete in time

  for (unsigned long long c0 = (unsigned long long)blockIdx.x * Gm::CHUNK; c0 < n_events;
       c0 += (unsigned long long)gridDim.x * Gm::CHUNK) {
    const unsigned long long c1 = min(c0 + (unsigned long long)Gm::CHUNK, n_events);
    unsigned long long pos = c0;
    while (pos < c1) {
      // the slice holding event pos: the last s with starts[s S] <= pos
      long long lo_s = 0, hi_s = n_slices - 1;
      while (lo_s < hi_s) {
        const long long mid = (lo_s + hi_s + 1) >> 1;
        if ((unsigned long long)starts[mid * S] <= pos) lo_s = mid; else hi_s = mid - 1;
      }
      const long long sidx = lo_s;
      const unsigned long long s_end = (sidx + 1 < n_slices) ? (unsigned long long)starts[(sidx + 1) * S] : n_events;
      const unsigned long long g1 = min(c1, s_end);

      // every group is done with the previous segment's B; a failed group stops the block
      if (__syncthreads_or(!ok)) { ok = false; break; }
      // B = [C | H | Lam C | C Lam] of this slice as N rows of K, split hi / lo
      const float* src = slices + sidx * sl_stride;
      for (int idx = tid; idx < N * K; idx += Gm::THREADS) {
        const int nn = idx / K, a = idx - nn * K;
        const int blk = nn / NMAX, b = nn - blk * NMAX;
        float v = 0.f;
        if (FULL || (a < n && b < n)) {
          const float c = src[a * NMAX + b];
          if (blk == 0) v = c;
          else if (blk == 1) v = src[half + a * NMAX + b];
          else if (blk == 2) v = jac_lam<float>(a) * c;
          else v = c * jac_lam<float>(b);
        }
        float h, l;
        tc::split_tf32(v, h, l);
        const uint32_t off = tc::kmajor_offset(nn, a, KC);
        *reinterpret_cast<float*>(Bhi + off) = h;
        *reinterpret_cast<float*>(Blo + off) = l;
      }
      tc::fence_async_smem();
      __syncthreads();
      const long long ti = slice_node[sidx];
      const TimeNode node = tn[ti];
      const InstanceParams ip = ipt[node.inst];
      const SliceInfo si = sinfo[sidx];
      const float Tt = (float)si.Tt, dTt = (float)si.dTt, tau = (float)si.tau;
      const long long node0 = ti * S - (long long)(sidx * S);   // node index = node0 + key

      const int n_tiles = (int)((g1 - pos + 127) / 128);
      // the group's next event is loaded one tile ahead
      auto load_event = [&](int t, float4& e) {
        const unsigned long long i = pos + (unsigned long long)t * 128 + gt;
        e = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
        if (t < n_tiles && i < g1) e = *reinterpret_cast<const float4*>(events + i);
        return t < n_tiles && i < g1;
      };
      float4 ev_next;
      bool has_next = load_event(grp, ev_next);
      bool prev_done = true;   // this thread's wait for the group's previous tile completed
      for (int t = grp; t < n_tiles; t += NT) {
        const float4 ev = ev_next;
        const bool has = has_next;
        has_next = load_event(t + NT, ev_next);
        // the A rows are free: this thread waited for the previous tile's products
        write_a_row<NMAX, FULL>(Ah, Al, gt, ev.x, n);
        tc::fence_async_smem();
        tc::fence_before();
        // one barrier per tile: the rows are written and the previous tile's
        // accumulator has been read by every thread; the group agrees on a time-out
        if (tc::named_sync_or(1 + grp, 128, !prev_done)) { ok = false; timed_out = true; break; }
        if (gt == 0) {
          tc::fence_after();
#pragma unroll
          for (int s = 0; s < K / 8; ++s) {
            const uint32_t ko = (uint32_t)s * 256;   // 8 TF32 = two core matrices along K
            tc::mma_tf32(tcol, tc::sdesc(al + ko, Gm::LBO, Gm::SBO), tc::sdesc(bHi + ko, Gm::LBO, Gm::SBO), idesc,
                         s > 0 ? 1u : 0u);
            tc::mma_tf32(tcol, tc::sdesc(ah + ko, Gm::LBO, Gm::SBO), tc::sdesc(bLo + ko, Gm::LBO, Gm::SBO), idesc,
                         1u);
            tc::mma_tf32(tcol, tc::sdesc(ah + ko, Gm::LBO, Gm::SBO), tc::sdesc(bHi + ko, Gm::LBO, Gm::SBO), idesc,
                         1u);
          }
          tc::mma_commit(mbar + grp);
        }
        // P_b(y) while the products run
        const float y0 = ev.x, y1 = ev.y;
        float Py[NMAX];
        {
          float pm2 = 1.f, pm1 = 2.f * y1;
#pragma unroll
          for (int b = 0; b < NMAX; ++b) {
            float P;
            if (b == 0) P = 1.f;
            else if (b == 1) P = 2.f * y1;
            else { P = jac_ra<float>(b) * y1 * pm1 - jac_rb<float>(b) * pm2; pm2 = pm1; pm1 = P; }
            Py[b] = (FULL || b < n) ? P : 0.f;
          }
        }
        const bool done = tc::mbar_wait_bounded(mbar + grp, phase);
        phase ^= 1u;
        tc::fence_after();
        float sv[4];
#pragma unroll
        for (int blk = 0; blk < 4; ++blk) {
          float s = 0.f, s2 = 0.f;
#pragma unroll
          for (int c8 = 0; c8 < NMAX / 8; ++c8) {   // eight columns at a time: few live registers
            float v[8];
            tc::tmem_ld8(lane_base + (uint32_t)(blk * NMAX + c8 * 8), v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
              s = fmaf(v[q], Py[8 * c8 + q], s);
              s2 = fmaf(v[q + 1], Py[8 * c8 + q + 1], s2);
            }
          }
          sv[blk] = s + s2;
        }
        int L[5] = {0, 0, 0, 0, 0};
        const unsigned int key = has ? __float_as_uint(ev.w) : 0xffffffffu;
        if (has) {
          const float ox = 1.f - y0 * y0, oy = 1.f - y1 * y1;
          const float u = ox * oy * sv[0];
          const float G = ox * oy * sv[1] - kappa * (oy * sv[2] + ox * sv[3]);
          const float yy[2] = {y0, y1};
          float term;
          if (si.kind == 0) {
            float res = forcing<2, float>(ip, kappa, yy, Tt, dTt, tau, u);
            if (!direct) res += G;
            term = ev.z * res;
          } else if (si.kind == 1) {
            term = u;   // the direct estimator's initial term u*(X, t_{n-1})
          } else {
            term = exact_bv<2, float>(ip, yy, (float)exp(-ip.ex_beta * (double)ev.z), ev.z);   // g(X, t)
          }
          if (!fix_limbs_float(term, L)) atomicOr(status, 1);
        }
        // per-node sums (exact): events are sorted by key, so each key's lanes
        // form one run [start, end) of the warp, found from the run heads; each
        // run's limbs are summed by a warp reduction over its lanes
        const unsigned int kprev = __shfl_up_sync(0xffffffffu, key, 1);
        const unsigned int heads = __ballot_sync(0xffffffffu, lane == 0 || kprev != key);
        const unsigned int upto = 0xffffffffu >> (31 - lane);          // lanes 0..lane
        const int start = 31 - __clz(heads & upto);
        const unsigned int after = heads & ~upto;
        const unsigned int below_end = after ? (1u << (__ffs(after) - 1)) - 1u : 0xffffffffu;
        const unsigned int peers = below_end & ~((1u << start) - 1u);
#pragma unroll
        for (int k = 0; k < 5; ++k) L[k] = __reduce_add_sync(peers, L[k]);
        if (done && has && lane == start) fix_atomic_add(acc + 4 * (node0 + (long long)key), fix_from_limbs(L));
        prev_done = done;
      }
      // a time-out in the segment's last tile stops the block at the next block barrier
      if (!prev_done) { ok = false; timed_out = true; }
      pos = g1;
    }
    if (__syncthreads_or(!ok)) { ok = false; break; }
  }
  if (timed_out) {
    // an MMA of this group did not complete in time: report, give it one more bounded wait
    atomicOr(status, 8);
    tc::mbar_wait_bounded(mbar + grp, phase ^ 1u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(*tslot, Gm::TM_COLS);
  }
}

}  // namespace spmc
