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
#include "spmc_kernels.cuh"

namespace spmc {

template <typename R>
struct Event {
  R y[2];
  R w;
  unsigned int key;   // (slice, spatial node) = slice * S + j
};

// A 5-D event (Green point, weight, key).
template <typename R>
struct Event5 {
  R y[5];
  R w;
  unsigned int key;
};
template <int D, typename R> struct EventOf { using type = Event<R>; };
template <typename R> struct EventOf<5, R> { using type = Event5<R>; };

struct EventArgs {
  const TimeNode* tn;
  const InstanceParams* ip;
  const double* xnodes;
  const void* xy;                // coordinates of every spatial node in R: [j][e], S x D
  FastDiv div_nb, div_S;         // by the batch's samples and by the nodes per time node
  int fast32;                    // walk ids and (time node, node) indices below 2^32: the FastDiv decode
  unsigned int* counts;          // COUNT: (slice, node) histogram; FILL: placement cursors
  void* events;                  // Event<R>[cap] grouped by (slice, node) (FILL)
  unsigned long long cap;        // events the buffer holds (FILL)
  int* status;                   // bit 4: an event fell outside the buffer
  int* abort;                    // nonzero: an earlier batch did not fit; return at once
  int n, S, n_sub, gbits, max_steps, interval, iteration;
  long long n_tn;
  long long i0, nb;              // sample range of the batch
  long long node_lo, node_cnt;   // the (time node, spatial node) pairs walked: ti S + j in [node_lo, node_lo + node_cnt)
  double kappa, shell;
  uint32_t k0, k1;
  unsigned long long* counters;  // [0] points, [1] capped
  int direct;                    // the direct estimator (Eq. Phi_ast): initial- and boundary-term events
};

// Per-warp queue of pending evaluation events of the placing pass: what the
// Green point and the slot need (centre, radius, weight, key, the step's stream
// coordinates and its Green-direction word).
template <int D, typename R>
struct EmitQueue {
  static constexpr int CAP = 64;          // two warps' worth: 32 are flushed at a time
  R x[D][CAP], r[CAP], w[CAP];
  uint32_t key[CAP], w0[CAP], sample[CAP], node[CAP], tag[CAP], gdir[CAP];
};

// Every walk of the batch, lane by lane.  Walk ids are (node - node_lo) nb + il
// with node = ti S + j (sample fastest); block b owns the ids b, b + G, b + 2G, ... (G = grid size),
// an even mix of every time node and node, and its lanes take them one at a
// time from a shared counter as their walks end, so no lane waits for a fixed
// list of long walks.  COUNT counts the evaluation events per (slice, node);
// FILL runs the same walks again (pure functions of their Philox streams) and
// writes each event into its place.
//
// The loop is warp-synchronous: its condition is a warp vote, so every lane
// runs every iteration, and each iteration is a fixed sequence of predicated
// stages -- take a new walk (lanes whose walk ended), prepare the step (ball,
// weight, sub-point, roulette), record the event, move to the sphere.  COUNT
// adds each event to its (slice, node) count at once (one reduction per event,
// without a return value).  FILL appends it to its warp's queue; once 32 are queued
// the whole warp computes their Green points (a second Philox block, the radial
// law, the direction), claims their slots and stores them, all lanes together.
//
// Word layouts (one step): d <= 2, eight words -- [direction, Green direction,
// sub-point, roulette | Green radius uniforms] -- so the words every step needs
// sit in one Philox block; d = 5, 28 words -- [direction 12 | Green direction
// 12 | radius pair, sub-point, roulette] -- so a step reads its sub-point and
// roulette words from its seventh block and its direction from its first three.
template <int D, typename R, bool FILL>
__global__ void __launch_bounds__(256, (D <= 2 && sizeof(R) == 4) ? 4 : 2) walk_events_kernel(EventArgs a) {
  static_assert(D <= 2 || D == 5, "event sweep: d = 1, 2 or 5");
  using Ev = typename EventOf<D, R>::type;
  if (*a.abort) return;
  __shared__ unsigned long long s_next;
  __shared__ EmitQueue<D, R> s_q[FILL ? 8 : 1];   // one queue per warp of the 256-thread block
  const int S = a.S, G = a.n_sub;
  const long long nb = a.nb;
  const R kappa = (R)a.kappa, shell = (R)a.shell;
  Ev* ev = reinterpret_cast<Ev*>(a.events);
  unsigned long long capped = 0, points = 0;
  const unsigned int lane = threadIdx.x & 31;
  const unsigned int lt_mask = (1u << lane) - 1u;
  EmitQueue<D, R>& Q = s_q[FILL ? (threadIdx.x >> 5) : 0];
  int qn = 0;   // entries in this warp's queue (warp-uniform)

  const long long total = a.node_cnt * nb;
  const long long mine = total > (long long)blockIdx.x ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();

  // the placing pass's queue flush: lanes < cnt take entries 0..cnt-1
  auto flush = [&](int cnt) {
    __syncwarp();
    const bool has = (int)lane < cnt;
    const unsigned int fmask = __ballot_sync(0xffffffffu, has);
    if (has) {
      WalkStream w2;
      w2.k0 = a.k0; w2.k1 = a.k1;
      w2.sample = Q.sample[lane]; w2.node = Q.node[lane]; w2.tag = Q.tag[lane];
      const uint32_t key = Q.key[lane];
      const unsigned int peers = __match_any_sync(fmask, key);
      const int leader = __ffs(peers) - 1;
      unsigned int slot = 0;
      if ((int)lane == leader) slot = atomicAdd(&a.counts[key], (unsigned int)__popc(peers));
      R thg[D];
      const uint32_t gd = Q.gdir[lane];
      if constexpr (D == 1) {
        thg[0] = (gd >> 31) ? R(-1) : R(1);
      } else if constexpr (D == 2) {
        const R U = U01<R>::one(gd);
        R sn, cs;
        Ar<R>::sincos2pi(U, &sn, &cs);
        thg[0] = cs; thg[1] = sn;
      } else {
        direction<D, R>(w2, Q.w0[lane] + gdir_index(D), thg);
      }
      R U1, U2;
      green_uniforms<D, R>(w2, Q.w0[lane], U1, U2);
      const R v = green_radius<D, R>(U1, U2);
      const R rv = Ar<R>::mul(Q.r[lane], v);
      Ev e;
      if constexpr (D == 1) {
        e.y[0] = Ar<R>::add(Q.x[0][lane], Ar<R>::mul(rv, thg[0]));
        e.y[1] = R(0);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) e.y[d] = Ar<R>::add(Q.x[d][lane], Ar<R>::mul(rv, thg[d]));
      }
      e.w = Q.w[lane];
      e.key = key;
      slot = __shfl_sync(peers, slot, leader) + __popc(peers & lt_mask);   // the round trip overlaps the Green point
      if ((unsigned long long)slot < a.cap) {
        ev[slot] = e;
      } else {
        atomicOr(a.status, 4);   // cannot happen: the scan checked the batch's total
        atomicCAS(a.abort, 0, a.iteration);
      }
      ++points;
    }
    __syncwarp();
  };

  // walk state
  bool live = false, more = true;
  bool pend = false;     // direct estimator: the walk reached t_{n-1}; its initial-term event is next
  bool bc_raw = false;   // direct estimator with raw boundary data: absorbed walks emit the boundary term
  R X[D], f = R(0), delta = R(0), inv_delta = R(0), J = R(0), sub = R(0), t_node = R(0);
  const R two_dk = Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), inv_two_dk = Ar<R>::div(R(1), two_dk);
  int k = 0, q = 0, Ktot = 0, key_j = 0;
  long long slice_base = 0, cached_ti = -1;
  uint32_t node_ell = 0;
  WalkStream ws;
  ws.k0 = a.k0; ws.k1 = a.k1;
  constexpr int WS = step_words(D);
  while (__any_sync(0xffffffffu, live || more)) {
    // ---- stage 1: lanes without a walk take the block's next one
    const unsigned int need = __ballot_sync(0xffffffffu, !live && more);
    if (need) {
      unsigned long long base = 0;
      if ((int)lane == __ffs(need) - 1) base = atomicAdd(&s_next, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, __ffs(need) - 1);
      if (!live && more) {
        const unsigned long long kk = base + __popc(need & lt_mask);
        if ((long long)kk >= mine) {
          more = false;
        } else {
          const long long wid = (long long)blockIdx.x + (long long)kk * gridDim.x;
          long long node, il, ti;
          int j;
          if (a.fast32) {   // the usual case: about 2^25 walks per batch
            const uint32_t w32 = (uint32_t)wid;
            const uint32_t q32 = a.div_nb.div(w32);
            il = w32 - q32 * a.div_nb.d;
            const uint32_t nd = q32 + (uint32_t)a.node_lo;
            const uint32_t t32 = a.div_S.div(nd);
            node = nd; ti = t32; j = (int)(nd - t32 * (uint32_t)S);
          } else {
            node = wid / nb;
            il = wid - node * nb;
            node += a.node_lo;
            ti = node / S;
            j = (int)(node - ti * S);
          }
          if (ti != cached_ti) {   // time-node parameters, as the CPU reference computes them
            const TimeNode node = a.tn[ti];
            const R sdur = Ar<R>::sub((R)node.t_node, (R)node.t0);
            delta = Ar<R>::div(sdur, (R)node.nstar);
            inv_delta = Ar<R>::div(R(1), delta);
            J = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), delta));
            sub = Ar<R>::div(delta, (R)G);
            Ktot = G * node.nstar;
            slice_base = node.slice_base;
            node_ell = (uint32_t)node.ell;
            t_node = (R)node.t_node;
            bc_raw = a.direct && a.ip[node.inst].bc_kind == 2;
            ws.tag = ((uint32_t)(node.inst & 0xfff) << 20) | ((uint32_t)(a.interval & 0x3ff) << 10) |
                     (uint32_t)(a.iteration & 0x3ff);
            cached_ti = ti;
          }
          const R* xy = reinterpret_cast<const R*>(a.xy) + (size_t)j * D;
#pragma unroll
          for (int e = 0; e < D; ++e) X[e] = xy[e];
          f = R(0); k = 0; q = 0;
          key_j = j;
          ws.node = node_ell * (uint32_t)S + (uint32_t)j;
          ws.sample = (uint32_t)(a.i0 + il);
          live = true;
        }
      }
    }
    // ---- stage 2: the step, as the CPU reference: absorb, ball, weight, sub-point, roulette
    bool emit = false, last = false;
    R w = R(0), r = R(0), wstep = R(0);
    unsigned int key = 0;
    Philox4 b0{};
    uint32_t w0 = 0;
    if (live && pend) {
      // the direct estimator's initial term u*(X, t_{n-1}), weight 1, in the slot after the walk grid
      emit = true;
      w = R(1);
      key = ((uint32_t)slice_base + (uint32_t)Ktot) * (uint32_t)S + (uint32_t)key_j;
      pend = false;
      live = false;
    } else if (live) {
      R dist = R(1);
      int near = 0;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        const R de = Ar<R>::sub(R(1), Ar<R>::abs_(X[e]));
        if (de < dist) { dist = de; near = e; }
      }
      if (q >= a.max_steps || dist < shell) {
        if (q >= a.max_steps) {
          ++capped;
        } else if (bc_raw) {
          // absorbed: the boundary term g(X, t) at the nearest face and the path
          // time reached (carried in the weight field), in the second extra slot
#pragma unroll
          for (int e = 0; e < D; ++e)
            if (e == near) X[e] = X[e] < R(0) ? R(-1) : R(1);
          w = Ar<R>::sub(t_node, Ar<R>::add(Ar<R>::mul((R)k, sub), f));
          emit = true;
          key = ((uint32_t)slice_base + (uint32_t)Ktot + 1u) * (uint32_t)S + (uint32_t)key_j;
        }
        live = false;
      } else {
        w0 = (uint32_t)q * WS;   // a multiple of 4
        // the block of the sub-point and roulette words (d <= 2: also the
        // direction and Green-direction words)
        b0 = ws.block((w0 + gword_index(D)) >> 2);
        const uint32_t gword = b0.v[gword_index(D) & 3];
        const int g = a.gbits ? (int)(gword >> (32 - a.gbits)) : 0;
        const R left = Ar<R>::sub(Ar<R>::mul((R)(Ktot - k), sub), f);
        int m;
        if (J <= dist) {
          r = J;
          w = delta;
          if (k + G >= Ktot) {
            const int ahead = Ktot - k;
            m = k + (a.gbits ? (int)__umulhi(gword, (uint32_t)ahead) : 0);
            w = left;
            last = true;
          } else {
            m = k + g;
            k += G;
          }
        } else {
          r = dist;
          w = Ar<R>::divr(Ar<R>::mul(r, r), two_dk, inv_two_dk);
          m = k;
          if (w >= left) { w = left; last = true; }
          else {
            f = Ar<R>::add(f, w);
            while (f >= sub) { f = Ar<R>::sub(f, sub); ++k; }
            if (k >= Ktot) last = true;
          }
        }
        wstep = w;
        // roulette for shrunk balls
        if (r < J && w > R(0)) w = roulette_keep<R>(b0.v[rword_index(D) & 3], Ar<R>::divr(w, delta, inv_delta)) ? delta : R(0);
        emit = w > R(0);
        // keys fit 32 bits (the host checks n_slices S < 2^32)
        key = ((uint32_t)slice_base + (uint32_t)m) * (uint32_t)S + (uint32_t)key_j;
      }
    }
    // ---- stage 3: the event
    const unsigned int emask = __ballot_sync(0xffffffffu, emit);
    if (!FILL) {
      if (emit) atomicAdd(&a.counts[key], 1u);   // a reduction: the old value is not used
    } else if (emask) {
      if (emit) {
        const int pos = qn + __popc(emask & lt_mask);
#pragma unroll
        for (int d = 0; d < D; ++d) Q.x[d][pos] = X[d];
        Q.r[pos] = r; Q.w[pos] = w; Q.key[pos] = key; Q.w0[pos] = w0;
        Q.sample[pos] = ws.sample; Q.node[pos] = ws.node; Q.tag[pos] = ws.tag;
        Q.gdir[pos] = (D <= 2) ? b0.v[gdir_index(D) & 3] : 0u;
      }
      qn += __popc(emask);
      if (qn >= 32) {
        flush(32);
        // move the entries beyond the first 32 down
        const int rest = qn - 32;
        R tx[D], t2 = R(0), t3 = R(0);
        uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0, u4 = 0, u5 = 0;
        if ((int)lane < rest) {
          const int src = 32 + lane;
#pragma unroll
          for (int d = 0; d < D; ++d) tx[d] = Q.x[d][src];
          t2 = Q.r[src]; t3 = Q.w[src];
          u0 = Q.key[src]; u1 = Q.w0[src]; u2 = Q.sample[src]; u3 = Q.node[src]; u4 = Q.tag[src]; u5 = Q.gdir[src];
        }
        __syncwarp();
        if ((int)lane < rest) {
#pragma unroll
          for (int d = 0; d < D; ++d) Q.x[d][lane] = tx[d];
          Q.r[lane] = t2; Q.w[lane] = t3;
          Q.key[lane] = u0; Q.w0[lane] = u1; Q.sample[lane] = u2; Q.node[lane] = u3; Q.tag[lane] = u4;
          Q.gdir[lane] = u5;
        }
        __syncwarp();
        qn = rest;
      }
    }
    // ---- stage 4: the walk ends, or moves to the sphere of its ball.  For the
    // direct estimator the last step moves too, by sqrt(2 d kappa w) for the
    // time w it took (at most the ball's radius), and the walk's initial-term
    // event follows in the next round.
    if (live) {
      if (last && !a.direct) {
        live = false;
      } else {
        if (last) {
          r = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), wstep));
          pend = true;
        }
        if constexpr (D == 1) {
          const R th = (b0.v[0] >> 31) ? R(-1) : R(1);
          X[0] = Ar<R>::add(X[0], Ar<R>::mul(r, th));
        } else if constexpr (D == 2) {
          const R U = U01<R>::one(b0.v[0]);
          R sn, cs;
          Ar<R>::sincos2pi(U, &sn, &cs);
          X[0] = Ar<R>::add(X[0], Ar<R>::mul(r, cs));
          X[1] = Ar<R>::add(X[1], Ar<R>::mul(r, sn));
        } else {
          R th[D];
          direction<D, R>(ws, w0, th);
#pragma unroll
          for (int d = 0; d < D; ++d) X[d] = Ar<R>::add(X[d], Ar<R>::mul(r, th[d]));
        }
        ++q;
      }
    }
  }
  if (FILL) {
    if (qn > 0) flush(qn);
    for (int o = 16; o > 0; o >>= 1) {
      points += __shfl_xor_sync(0xffffffffu, points, o);
      capped += __shfl_xor_sync(0xffffffffu, capped, o);
    }
    if (lane == 0) {
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

// One block per slice: stage the slice, evaluate its events, sum their terms
// per node (exact fixed-point sums into four limb counters per (time node,
// node)).  A term is w r at a walk-grid slice (the residual, or for the direct
// estimator the forcing alone), u*(X, t_{n-1}) at the direct estimator's
// initial-term slot, g(X, t) at its boundary-term slot.
template <int D, int NMAX, typename R>
__global__ void __launch_bounds__(256) eval_events_kernel(const long long* __restrict__ slice_node,
                                                          const TimeNode* __restrict__ tn,
                                                          const InstanceParams* __restrict__ ipt,
                                                          const void* __restrict__ slices_v,
                                                          const SliceInfo* __restrict__ sinfo,
                                                          const unsigned int* __restrict__ starts,
                                                          const void* __restrict__ events_v,
                                                          unsigned long long* __restrict__ acc, int n, int S,
                                                          long long sl_stride, int half, double kappa_d, int direct,
                                                          int cheb, const unsigned long long* __restrict__ n_events_p,
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
      R u, G;
      if (cheb) slice_parts_cheb<D, NMAX, R>(kappa, n, sC, sC + half, Y, u, G);
      else slice_parts<D, NMAX, R>(kappa, n, sC, sC + half, Y, u, G);
      R term;
      if (si.kind == 0) {
        // w (f + f_add [+ lifting terms]) [+ w (-d_t u* + kappa Delta u*) for the residual iteration]
        R res = forcing<D, R>(ip, kappa, Y, (R)si.Tt, (R)si.dTt, (R)si.tau, u);
        if (!direct) res += G;
        term = e.w * res;
      } else if (si.kind == 1) {
        term = u;   // the initial term u*(X, t_{n-1})
      } else {
        term = exact_bv<D, R>(ip, Y, (R)exp(-ip.ex_beta * (double)e.w), e.w);   // g(X, t), t in the weight field
      }
      if (!fix_from<R>(term, val)) atomicOr(status, 1);
      key = e.key;
    }
    // per-node sums: events are sorted by key, so equal keys are adjacent lanes
    val = warp_run_sum(val, key, lane);
    const unsigned int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    if (has && (lane == 0 || kprev != key))
      fix_atomic_add(acc + 4 * (ti * S + (long long)(key - (unsigned int)(sidx * S))), val);
  }
}

// The fixed-radius walk (walk_mode 1, Lemma Xlocation, Eqs. indexL and
// interIQ) and the alpha-stable walk of the fractional case (walk_mode 2), one
// thread per walk: the walk's steps, the residual at each step centre X_q at
// time t_{n,l} - q Delta from the slice of step q (read through the cache), and
// the walk's Q = Delta sum_q r(X_q) counted while X_{q+1} stays inside Omega.
// Walk ids are node M + sample (sample fastest), node = ti S + j, so the walks of
// a node are adjacent lanes: their Q are summed exactly per node (fixed-point
// run sums, as in the event sweep) into the node's limb counters.
template <int D, int NMAX, typename R>
__global__ void __launch_bounds__(256) fixed_walk_kernel(SweepArgs a, long long n_walks,
                                                         unsigned long long* __restrict__ acc) {
  const int S = a.S, n = a.n;
  const R kappa = (R)a.kappa;
  const R* slices = reinterpret_cast<const R*>(a.slices);
  const unsigned int lane = threadIdx.x & 31;
  unsigned long long capped = 0, points = 0;
  // the alpha-stable jump law's series ratios in the sweep's precision
  __shared__ R s_rp[kFracSeriesD], s_rq[kFracSeriesD];
  R s_a = R(0), s_lnB = R(0);
  if (a.walk_mode == 2) {
    for (int k = threadIdx.x; k < kFracSeriesD; k += blockDim.x) {
      s_rp[k] = (R)a.frac[kFracRpD + k];
      s_rq[k] = (R)a.frac[kFracRqD + k];
    }
    s_a = (R)a.frac[kFracAD];
    s_lnB = (R)a.frac[kFracLnBD];
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long top = (n_walks + 31) / 32 * 32;   // whole warps: the run sums are warp-wide
  for (long long wid = (long long)blockIdx.x * blockDim.x + threadIdx.x; wid < top; wid += stride) {
    const bool has = wid < n_walks;
    __int128 val = 0;
    unsigned int key = 0xffffffffu;
    if (has) {
      const long long node = wid / a.M;
      const long long ti = node / S;
      const int j = (int)(node - ti * S);
      const TimeNode tn = a.tn[ti];
      const InstanceParams ip = a.ip[tn.inst];
      WalkStream ws;
      ws.k0 = a.k0; ws.k1 = a.k1;
      ws.tag = ((uint32_t)(tn.inst & 0xfff) << 20) | ((uint32_t)(a.interval & 0x3ff) << 10) |
               (uint32_t)(a.iteration & 0x3ff);
      ws.node = (uint32_t)(tn.ell * S + j);
      ws.sample = (uint32_t)(wid - node * a.M);
      const R sdur = Ar<R>::sub((R)tn.t_node, (R)tn.t0);
      const R delta = Ar<R>::div(sdur, (R)tn.nstar);
      const R J = Ar<R>::sqrt_(Ar<R>::mul(Ar<R>::mul(Ar<R>::mul(R(2), R(D)), kappa), delta));
      double r_stable = 0.0;
      if (a.walk_mode == 2)
        r_stable = pow(a.kappa * ((tn.t_node - tn.t0) / (double)tn.nstar) * a.frac[kFracGammaD],
                       1.0 / a.frac[kFracAlphaD]);
      R X[D];
      int jr = j;
#pragma unroll
      for (int e = 0; e < D; ++e) { X[e] = (R)a.xnodes[jr % n]; jr /= n; }
      R Q = R(0);
      for (int q = 0; q < tn.nstar; ++q) {
        if (q >= a.max_steps) { ++capped; break; }
        R Xn[D];
        bool inside = true;
        if (a.walk_mode == 2) {
          const Philox4 b = ws.block((uint32_t)q >> 1);
          const double Jq = (double)stable_jump<R, R>((R)r_stable, s_a, s_lnB, s_rp, s_rq,
                                                      U01<double>::one(b.v[(2 * q + 1) & 3]));
          const double xn = (double)X[0] + ((b.v[(2 * q) & 3] >> 31) ? -Jq : Jq);
          inside = xn > -1.0 && xn < 1.0;
          Xn[0] = (R)xn;
        } else {
          R th[D];
          literal_direction<D, R>(ws, q, th);
#pragma unroll
          for (int e = 0; e < D; ++e) {
            Xn[e] = Ar<R>::add(X[e], Ar<R>::mul(J, th[e]));
            if (!(Xn[e] > R(-1) && Xn[e] < R(1))) inside = false;
          }
        }
        if (!inside) break;
        const long long sl = tn.slice_base + q;
        const R* sc = slices + sl * a.sl_stride;
        const SliceInfo si = a.sinfo[sl];
        R res;
        if (D == 1 && a.walk_mode == 2)
          res = residual_frac<R>(ip, kappa, n, sc, sc + a.half, X[0], (R)si.Tt, (R)si.dTt, a.frac);
        else
          res = residual_at<D, NMAX, R>(ip, kappa, n, sc, sc + a.half, X, (R)si.Tt, (R)si.dTt);
        Q += delta * res;
        ++points;
#pragma unroll
        for (int e = 0; e < D; ++e) X[e] = Xn[e];
      }
      if (!fix_from<R>(Q, val)) atomicOr(a.status, 1);
      key = (unsigned int)node;
    }
    // per-node sums: walks of a node are adjacent lanes
    val = warp_run_sum(val, key, lane);
    const unsigned int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    if (has && (lane == 0 || kprev != key)) fix_atomic_add(acc + 4 * (long long)key, val);
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

// The adjoint of one iteration's sweep on the event pipeline (the forward
// iteration's own events: same walks, weights and points).  One block per
// slice.  Per event p at node i: cw = lambda_i w_p / M, u* from the slice's C,
// alpha = cw s g'(u*), beta = cw; the slice's three tensors
//   T_alpha = sum alpha Phi(Y),  T_beta = sum beta Phi(Y),  T_psi = sum beta Psi(Y)
// (Phi = prod phi, Psi = sum over one axis of psi with phi on the others) are
// outer-product sums over the events: per chunk of 128 events each event writes
//   a = [alpha ox oy P(x) | beta ox oy P(x) | beta oy lam P(x) | beta ox P(x)],
//   b = [P(y) | lam P(y)]
// to shared memory (d = 1: [alpha o P | beta o P | beta lam P]), and each thread
// accumulates its share of the 3 n^d outputs over the chunk in R, then in FP64
// across chunks; the slice's sums are added to gT (FP64) at the end, and the
// derivative in the reaction scale, sum cw (g(u*) - g(u_ex)), to gds.
template <int D, int NMAX, typename R>
__global__ void __launch_bounds__(256) adj_events_kernel(const long long* __restrict__ slice_node,
                                                         const TimeNode* __restrict__ tn,
                                                         const InstanceParams* __restrict__ ipt,
                                                         const void* __restrict__ slices_v,
                                                         const SliceInfo* __restrict__ sinfo,
                                                         const unsigned int* __restrict__ starts,
                                                         const void* __restrict__ events_v,
                                                         const double* __restrict__ lambda, double* __restrict__ gT,
                                                         double* __restrict__ gds, int n, int S, long long sl_stride,
                                                         long long M, const unsigned long long* __restrict__ n_events_p,
                                                         const int* __restrict__ abort) {
  constexpr int CH = 128;                       // events per chunk
  constexpr int NA = (D == 2) ? 4 * NMAX : 3 * NMAX, NB = (D == 2) ? 2 * NMAX : 1;
  constexpr int NOUT = (D == 2) ? 3 * NMAX * NMAX : 3 * NMAX;
  constexpr int KO = (NOUT + 255) / 256;        // outputs per thread
  extern __shared__ __align__(16) unsigned char smraw[];
  if (*abort) return;
  const unsigned long long n_events = *n_events_p;
  R* sC = reinterpret_cast<R*>(smraw);                        // the slice's C (sl_stride entries)
  R* sa = sC + ((sl_stride + 3) / 4) * 4;                     // [CH][NA]
  R* sb = sa + CH * NA;                                       // [CH][NB]
  __shared__ double dred[8];
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
  const Event<R>* ev = reinterpret_cast<const Event<R>*>(events_v);
  const double invM = 1.0 / (double)M;
  double acc[KO];
#pragma unroll
  for (int k = 0; k < KO; ++k) acc[k] = 0.0;
  double ds = 0.0;
  __syncthreads();
  for (unsigned long long base = e0; base < e1; base += CH) {
    if (threadIdx.x < CH) {
      const unsigned long long i = base + threadIdx.x;
      R* a = sa + threadIdx.x * NA;
      R* b = sb + threadIdx.x * NB;
      if (i < e1) {
        const Event<R> e = ev[i];
        const int j = (int)(e.key - (unsigned int)(sidx * S));
        const double cw = lambda[node.u_off + (long long)node.ell * S + j] * (double)e.w * invM;
        const R x = e.y[0], ox = R(1) - x * x;
        R Px[NMAX];
        {
          R pm2 = R(1), pm1 = R(2) * x;
#pragma unroll
          for (int p = 0; p < NMAX; ++p) {
            R v;
            if (p == 0) v = R(1);
            else if (p == 1) v = R(2) * x;
            else { v = jac_ra<R>(p) * x * pm1 - jac_rb<R>(p) * pm2; pm2 = pm1; pm1 = v; }
            Px[p] = p < n ? v : R(0);
          }
        }
        R u;
        R Py[NMAX], oy = R(1);
        if (D == 1) {
          R t = R(0);
#pragma unroll
          for (int p = 0; p < NMAX; ++p) t += sC[p] * Px[p];
          u = ox * t;
        } else {
          const R y = e.y[1];
          oy = R(1) - y * y;
          R pm2 = R(1), pm1 = R(2) * y;
#pragma unroll
          for (int p = 0; p < NMAX; ++p) {
            R v;
            if (p == 0) v = R(1);
            else if (p == 1) v = R(2) * y;
            else { v = jac_ra<R>(p) * y * pm1 - jac_rb<R>(p) * pm2; pm2 = pm1; pm1 = v; }
            Py[p] = p < n ? v : R(0);
          }
          R t = R(0);
          for (int p1 = 0; p1 < n; ++p1) {
            R r2 = R(0);
#pragma unroll
            for (int p2 = 0; p2 < NMAX; ++p2) r2 += sC[p1 * NMAX + p2] * Py[p2];
            t += Px[p1] * r2;
          }
          u = ox * oy * t;
        }
        double g, dg;
        reaction_g(ip, (double)u, &g, &dg);
        double gex = 0.0;
        if (ip.ex_kind != 0) {
          double prod = 1.0;
          for (int d = 0; d < D; ++d) {
            const double yd = (double)e.y[d];
            if (ip.ex_kind == 1) prod *= sinpi(yd);
            else if (ip.ex_kind == 2) prod *= cospi(0.5 * yd);
            else prod *= (1.0 - yd * yd) * (1.0 + yd);
          }
          double dgx;
          reaction_g(ip, si.Tt * prod, &gex, &dgx);
        }
        ds += cw * (g - gex);
        const R al = (R)(cw * ip.f_scale * dg), be = (R)cw;
#pragma unroll
        for (int p = 0; p < NMAX; ++p) {
          if (D == 2) {
            a[p] = al * ox * oy * Px[p];
            a[NMAX + p] = be * ox * oy * Px[p];
            a[2 * NMAX + p] = be * oy * jac_lam<R>(p) * Px[p];
            a[3 * NMAX + p] = be * ox * Px[p];
            b[p] = Py[p];
            b[NMAX + p] = jac_lam<R>(p) * Py[p];
          } else {
            a[p] = al * ox * Px[p];
            a[NMAX + p] = be * ox * Px[p];
            a[2 * NMAX + p] = be * jac_lam<R>(p) * Px[p];
          }
        }
      } else {
        for (int p = 0; p < NA; ++p) a[p] = R(0);
        for (int p = 0; p < NB; ++p) b[p] = R(0);
      }
    }
    __syncthreads();
    const int ne = (int)min((unsigned long long)CH, e1 - base);
#pragma unroll
    for (int k = 0; k < KO; ++k) {
      const int o = threadIdx.x + 256 * k;
      if (o < NOUT) {
        R s = R(0);
        if (D == 2) {
          const int c = o / (NMAX * NMAX), rem = o - c * NMAX * NMAX, p1 = rem / NMAX, p2 = rem - p1 * NMAX;
          if (c < 2) {
            for (int e = 0; e < ne; ++e) s += sa[e * NA + c * NMAX + p1] * sb[e * NB + p2];
          } else {
            for (int e = 0; e < ne; ++e)
              s += sa[e * NA + 2 * NMAX + p1] * sb[e * NB + p2] + sa[e * NA + 3 * NMAX + p1] * sb[e * NB + NMAX + p2];
          }
        } else {
          for (int e = 0; e < ne; ++e) s += sa[e * NA + o];
        }
        acc[k] += (double)s;
      }
    }
    __syncthreads();
  }
  // the slice's sums, in coefficient order (x_1 fastest): gT[s][c][p1 + n p2]
#pragma unroll
  for (int k = 0; k < KO; ++k) {
    const int o = threadIdx.x + 256 * k;
    if (o < NOUT && acc[k] != 0.0) {
      long long dst;
      if (D == 2) {
        const int c = o / (NMAX * NMAX), rem = o - c * NMAX * NMAX, p1 = rem / NMAX, p2 = rem - p1 * NMAX;
        if (p1 >= n || p2 >= n) continue;
        dst = (long long)c * S + p1 + (long long)n * p2;
      } else {
        const int c = o / NMAX, p = o - c * NMAX;
        if (p >= n) continue;
        dst = (long long)c * S + p;
      }
      atomicAdd(&gT[sidx * 3 * S + dst], acc[k]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
  if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = ds;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += dred[w];
    if (t != 0.0) atomicAdd(&gds[node.inst], t);
  }
}

}  // namespace spmc
