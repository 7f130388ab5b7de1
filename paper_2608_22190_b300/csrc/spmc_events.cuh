// spmc_events.cuh -- the forward sweep as an event pipeline (d = 1, 2).
//
// The time slices depend only on (instance, time node, sub-point), not on the
// spatial node, so the residual evaluations of one slice can be done together
// for every node and sample of its time node.  Per batch of samples:
//   walk_events_kernel<COUNT>  every walk runs its steps (inside balls, Green
//                              points, roulette) and counts its evaluation
//                              events per (slice, spatial node);
//   scan kernels               exclusive offsets of the (slice, node) segments;
//   walk_events_kernel<FILL>   the same walks again (pure functions of their
//                              Philox streams) write each event (Green point,
//                              weight, key) into its segment;
//   eval_events_kernel         one block per slice stages the slice once in
//                              shared memory and evaluates all its events; the
//                              weighted residuals are summed per node exactly
//                              (fixed-point integers, see fix_from_double).
// The per-node sums feed the update kernel (eps = sum / M).  Nothing returns to
// the host between batches: the event buffer's capacity is set by the host from
// a measured high-water mark, the scan checks the batch's total against it on
// the device, and a batch that does not fit sets the abort word (the number of
// the iteration); every later launch of the iteration sequence then returns at
// once and the host, at its next synchronisation, grows the buffer and runs the
// iterations again from the one that failed.
#pragma once
#include <cooperative_groups.h>

#include "spmc_kernels.cuh"

namespace spmc {

template <typename R>
struct Event {
  R y[2];
  R w;
  unsigned int key;   // (slice, spatial node) = slice * S + j
};

struct EventArgs {
  const TimeNode* tn;
  const double* xnodes;
  unsigned int* counts;          // COUNT: (slice, node) histogram; FILL: placement cursors
  void* events;                  // Event<R>[cap] grouped by (slice, node) (FILL)
  unsigned long long cap;        // events the buffer holds (FILL)
  int* status;                   // bit 4: an event fell outside the buffer
  int* abort;                    // nonzero: an earlier batch did not fit; return at once
  int n, S, n_sub, gbits, max_steps, interval, iteration;
  long long n_tn;
  long long i0, nb;              // sample range of the batch
  double kappa, shell;
  uint32_t k0, k1;
  unsigned long long* counters;  // [0] points, [1] capped
};

// Every walk of the batch, lane by lane: a lane takes the next walk when its
// current one ends, so the lanes of a warp stay busy.  Walk ids run sample
// fastest (consecutive lanes share a node and mostly a slice); a thread steps
// through its walk ids by a fixed stride, kept as (time node, node, sample)
// counters.  COUNT counts the evaluation events per (slice, node); FILL runs
// the same walks again (pure functions of their Philox streams) and writes each
// event into its place.  Lanes with the same key share one atomic.
template <int D, typename R, bool FILL>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) walk_events_kernel(EventArgs a) {
  static_assert(D <= 2, "the event sweep reads a step's words from one Philox block (d <= 2 layout)");
  namespace cg = cooperative_groups;
  if (*a.abort) return;
  const int S = a.S, n = a.n, G = a.n_sub;
  const long long nb = a.nb;
  const R kappa = (R)a.kappa, shell = (R)a.shell;
  Event<R>* ev = reinterpret_cast<Event<R>*>(a.events);
  unsigned long long capped = 0, points = 0;

  // walk id = (ti * S + j) * nb + il; the stride decomposed the same way
  const long long total = a.n_tn * S * nb;
  long long wid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long per_tn = (long long)S * nb;
  long long ti = wid / per_tn;
  int j = (int)((wid - ti * per_tn) / nb);
  long long il = wid - ti * per_tn - (long long)j * nb;
  const long long st_t = stride / per_tn;
  const int st_j = (int)((stride - st_t * per_tn) / nb);
  const long long st_i = stride - st_t * per_tn - (long long)st_j * nb;

  // walk state
  bool live = false;
  R X[D], f = R(0), delta = R(0), J = R(0), sub = R(0);
  int k = 0, q = 0, Ktot = 0, key_j = 0;
  long long slice_base = 0, cached_ti = -1;
  uint32_t node_ell = 0;
  WalkStream ws;
  ws.k0 = a.k0; ws.k1 = a.k1;
  constexpr int WS = step_words(D);
  while (true) {
    if (!live) {
      if (wid >= total) break;
      if (ti != cached_ti) {   // time-node parameters, as the CPU reference computes them
        const TimeNode node = a.tn[ti];
        const R sdur = Ar<R>::sub((R)node.t_node, (R)node.t0);
        delta = Ar<R>::div(sdur, (R)node.nstar);
        J = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), delta));
        sub = Ar<R>::div(delta, (R)G);
        Ktot = G * node.nstar;
        slice_base = node.slice_base;
        node_ell = (uint32_t)node.ell;
        ws.tag = ((uint32_t)(node.inst & 0xfff) << 20) | ((uint32_t)(a.interval & 0x3ff) << 10) |
                 (uint32_t)(a.iteration & 0x3ff);
        cached_ti = ti;
      }
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { X[e] = (R)a.xnodes[jr % n]; jr /= n; }
      f = R(0); k = 0; q = 0;
      key_j = j;
      ws.node = node_ell * (uint32_t)S + (uint32_t)j;
      ws.sample = (uint32_t)(a.i0 + il);
      live = true;
      // advance to this thread's next walk id
      wid += stride;
      il += st_i;
      if (il >= nb) { il -= nb; ++j; }
      j += st_j;
      if (j >= S) { j -= S; ++ti; }
      ti += st_t;
    }
    // ---- one step, as the CPU reference: absorb, ball, weight, sub-point
    R dist = R(1);
#pragma unroll
    for (int e = 0; e < D; ++e) {
      R de = Ar<R>::sub(R(1), fabs(X[e]));
      if (de < dist) dist = de;
    }
    if (q >= a.max_steps || dist < shell) {
      if (q >= a.max_steps) ++capped;
      live = false;
      continue;
    }
    const uint32_t w0 = (uint32_t)q * WS;   // a multiple of 8 (d <= 2)
    // direction, Green direction, sub-point and roulette words: one block
    const Philox4 b0 = ws.block(w0 >> 2);
    const uint32_t gword = b0.v[gword_index(D)];
    const int g = a.gbits ? (int)(gword >> (32 - a.gbits)) : 0;
    R left = Ar<R>::sub(Ar<R>::mul((R)(Ktot - k), sub), f);
    R w, r;
    int m, last = 0;
    if (J <= dist) {
      r = J;
      w = delta;
      if (k + G >= Ktot) {
        const int ahead = Ktot - k;
        m = k + (a.gbits ? (int)(((unsigned long long)gword * (unsigned long long)ahead) >> 32) : 0);
        w = left;
        last = 1;
      } else {
        m = k + g;
        k += G;
      }
    } else {
      r = dist;
      w = Ar<R>::div(Ar<R>::mul(r, r), Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa));
      m = k;
      if (w >= left) { w = left; last = 1; }
      else {
        f = Ar<R>::add(f, w);
        while (f >= sub) { f = Ar<R>::sub(f, sub); ++k; }
        if (k >= Ktot) last = 1;
      }
    }
    // roulette for shrunk balls
    if (r < J && w > R(0)) w = roulette_keep<R>(b0.v[rword_index(D)], Ar<R>::div(w, delta)) ? delta : R(0);
    if (w > R(0)) {
      const unsigned int key = (unsigned int)((slice_base + m) * S + key_j);
      cg::coalesced_group grp = cg::coalesced_threads();
      cg::coalesced_group same = cg::labeled_partition(grp, key);
      if (!FILL) {
        if (same.thread_rank() == 0) atomicAdd(&a.counts[key], same.size());
      } else {
        unsigned int slot = 0;
        if (same.thread_rank() == 0) slot = atomicAdd(&a.counts[key], same.size());
        R thg[D];
        if (D == 1) {
          thg[0] = (b0.v[gdir_index(D)] >> 31) ? R(-1) : R(1);
        } else {
          const R U = U01<R>::one(b0.v[gdir_index(D)]);
          R sn, cs;
          Ar<R>::sincos2pi(U, &sn, &cs);
          thg[0] = cs; thg[1] = sn;
        }
        R U1, U2;
        green_uniforms<D, R>(ws, w0, U1, U2);
        const R v = green_radius<D, R>(U1, U2);
        const R rv = Ar<R>::mul(r, v);
        slot = same.shfl(slot, 0) + same.thread_rank();   // the atomic's round trip overlaps the Green point
        if ((unsigned long long)slot < a.cap) {
          Event<R> e;
          e.y[0] = Ar<R>::add(X[0], Ar<R>::mul(rv, thg[0]));
          e.y[1] = (D == 2) ? Ar<R>::add(X[1], Ar<R>::mul(rv, thg[1])) : R(0);
          e.w = w;
          e.key = key;
          ev[slot] = e;
        } else {
          atomicOr(a.status, 4);   // cannot happen: the scan checked the batch's total
          atomicCAS(a.abort, 0, a.iteration);
        }
        ++points;
      }
    }
    if (last) { live = false; continue; }
    // step to the sphere of the ball
    if (D == 1) {
      const R th = (b0.v[0] >> 31) ? R(-1) : R(1);
      X[0] = Ar<R>::add(X[0], Ar<R>::mul(r, th));
    } else {
      const R U = U01<R>::one(b0.v[0]);
      R sn, cs;
      Ar<R>::sincos2pi(U, &sn, &cs);
      X[0] = Ar<R>::add(X[0], Ar<R>::mul(r, cs));
      X[D - 1] = Ar<R>::add(X[D - 1], Ar<R>::mul(r, sn));
    }
    ++q;
  }
  if (FILL) {
    for (int o = 16; o > 0; o >>= 1) {
      points += __shfl_xor_sync(0xffffffffu, points, o);
      capped += __shfl_xor_sync(0xffffffffu, capped, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (points) atomicAdd(&a.counters[0], points);
      if (capped) atomicAdd(&a.counters[1], capped);
    }
  }
}

// Exclusive scan of n unsigned counts in place, in three launches (block scans
// of 1024 entries, a scan of the block totals, the add-back).
__global__ void scan_blocks_kernel(unsigned int* __restrict__ v, unsigned long long* __restrict__ bsum, long long n,
                                   const int* __restrict__ abort) {
  __shared__ unsigned int wsum[32];
  if (*abort) return;
  const long long base = (long long)blockIdx.x * 1024;
  unsigned int x[4];
  const int t = threadIdx.x;   // 256 threads x 4 entries
  unsigned int s = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = base + t * 4 + u;
    x[u] = i < n ? v[i] : 0u;
    s += x[u];
  }
  // inclusive scan of s over the block
  unsigned int incl = s;
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned int wbase = 0, tot = 0;
  for (int wv = 0; wv < 8; ++wv) { if (wv < warp) wbase += wsum[wv]; tot += wsum[wv]; }
  unsigned int run = wbase + incl - s;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = base + t * 4 + u;
    if (i < n) v[i] = run;
    run += x[u];
  }
  if (t == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of the block totals (one block, serial chunks).  The batch's
// total goes to *total; if it exceeds the event buffer's capacity, the largest
// total seen goes to *need and the abort word gets the iteration number.
__global__ void scan_totals_kernel(unsigned long long* __restrict__ bsum, long long nb, unsigned long long* total,
                                   unsigned long long cap, unsigned long long* need, int* abort, int iteration) {
  __shared__ unsigned long long carry;
  if (*abort) return;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ unsigned long long wsum[32];
  for (long long c0 = 0; c0 < nb; c0 += blockDim.x) {
    const long long i = c0 + threadIdx.x;
    const unsigned long long s = i < nb ? bsum[i] : 0ull;
    unsigned long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long wbase = 0, tot = 0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) { if (wv < warp) wbase += wsum[wv]; tot += wsum[wv]; }
    if (i < nb) bsum[i] = carry + wbase + incl - s;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry;
    atomicMax(need, carry);
    if (carry > cap) atomicCAS(abort, 0, iteration);
  }
}

__global__ void scan_add_kernel(unsigned int* __restrict__ v, const unsigned long long* __restrict__ bsum,
                                unsigned int* __restrict__ starts, long long n, const int* __restrict__ abort) {
  if (*abort) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const unsigned int o = v[i] + (unsigned int)bsum[i / 1024];
    v[i] = o;
    starts[i] = o;
  }
}

// Segmented warp sum of fixed-point terms over runs of equal keys (keys do not
// decrease across the lanes; lanes without a term carry key 0xffffffff and 0):
// each lane gets the sum of its run from itself to the run's end, so the run's
// first lane holds the run's total.  Exact, so independent of the lane order.
__device__ __forceinline__ __int128 warp_run_sum(__int128 v, unsigned int key, unsigned int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, d);
    const long long hi = __shfl_down_sync(0xffffffffu, (long long)(v >> 64), d);
    const unsigned int k2 = __shfl_down_sync(0xffffffffu, key, d);
    if (lane + d < 32 && k2 == key) v += (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
  }
  return v;
}

// One block per slice: stage the slice, evaluate its events, sum w r per node
// (exact fixed-point sums into four limb counters per (time node, node)).
template <int D, int NMAX, typename R>
__global__ void __launch_bounds__(256) eval_events_kernel(const long long* __restrict__ slice_node,
                                                          const TimeNode* __restrict__ tn,
                                                          const InstanceParams* __restrict__ ipt,
                                                          const void* __restrict__ slices_v,
                                                          const SliceInfo* __restrict__ sinfo,
                                                          const unsigned int* __restrict__ starts,
                                                          const void* __restrict__ events_v,
                                                          unsigned long long* __restrict__ acc, int n, int S,
                                                          long long sl_stride, int half, double kappa_d,
                                                          const unsigned long long* __restrict__ n_events_p,
                                                          int* status, const int* __restrict__ abort) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (*abort) return;
  const unsigned long long n_events = *n_events_p;
  R* sC = reinterpret_cast<R*>(smraw);
  const long long sidx = blockIdx.x;
  const unsigned int e0 = starts[sidx * S];
  const unsigned long long e1 = (sidx + 1 < (long long)gridDim.x) ? starts[(sidx + 1) * S] : n_events;
  if ((unsigned long long)e0 >= e1) return;
  const R* src = reinterpret_cast<const R*>(slices_v) + sidx * sl_stride;
  for (int i = threadIdx.x; i < (int)sl_stride; i += blockDim.x) sC[i] = src[i];
  const long long ti = slice_node[sidx];
  const TimeNode node = tn[ti];
  const InstanceParams ip = ipt[node.inst];
  const SliceInfo si = sinfo[sidx];
  const R kappa = (R)kappa_d;
  __syncthreads();
  const Event<R>* ev = reinterpret_cast<const Event<R>*>(events_v);
  const unsigned int lane = threadIdx.x & 31;
  for (unsigned long long base = e0; base < e1; base += blockDim.x) {
    const unsigned long long i = base + threadIdx.x;
    const bool has = i < e1;
    __int128 val = 0;
    unsigned int key = 0xffffffffu;
    if (has) {
      const Event<R> e = ev[i];
      R Y[D];
      Y[0] = e.y[0];
      if (D == 2) Y[1] = e.y[1];
      const R res = residual_at<D, NMAX, R>(ip, kappa, n, sC, sC + half, Y, (R)si.Tt, (R)si.dTt);
      if (!fix_from<R>(e.w * res, val)) atomicOr(status, 1);
      key = e.key;
    }
    // per-node sums: events are sorted by key, so equal keys are adjacent lanes
    val = warp_run_sum(val, key, lane);
    const unsigned int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    if (has && (lane == 0 || kprev != key))
      fix_atomic_add(acc + 4 * (ti * S + (long long)(key - (unsigned int)(sidx * S))), val);
  }
}

}  // namespace spmc
