// spmc_lib.cu -- C-ABI of the B300 hp-version time-stepping spectral Monte
// Carlo library (declared in include/spmc.h): plans, problem set-up, the hp
// driver of Algorithm 1 and its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "spmc.h"
#include "spmc_kernels.cuh"
#include "spmc_events.cuh"
#include "spmc_tc.cuh"
#include "spmc_tc5.cuh"
#include "spmc_tables.h"

static_assert(spmc::kFracRa == spmc::kFracRaD && spmc::kFracRb == spmc::kFracRbD &&
                  spmc::kFracLam == spmc::kFracLamD && spmc::kFracSin == spmc::kFracSinD &&
                  spmc::kFracA == spmc::kFracAD && spmc::kFracAlpha == spmc::kFracAlphaD &&
                  spmc::kFracGamma == spmc::kFracGammaD && spmc::kFracModes == spmc::kFracModesD &&
                  spmc::kFracLnB == spmc::kFracLnBD && spmc::kFracRp == spmc::kFracRpD &&
                  spmc::kFracRq == spmc::kFracRqD && spmc::kFracSeries == spmc::kFracSeriesD,
              "the fractional table's host and device layouts agree");

using namespace spmc;

namespace {

struct HostProblem {
  bool set = false;
  int n_int = 0;
  std::vector<double> t;
  std::vector<int> deg;
  InstanceParams ip{};
  std::vector<double> u0;       // nodal
  int u0_kind = 0, n_coef = 0;
  std::vector<double> u0_coef;  // phi coefficients (for the gradient)
};

struct Round {
  // work tables of interval index r across instances (host and device copies)
  std::vector<TimeNode> tn;
  std::vector<InstInterval> ii;           // active instances
  std::vector<InstInterval> ii_of_node;   // per time node
  std::vector<long long> slice_node;      // per slice -> time node
  long long n_slices = 0;
  TimeNode* d_tn = nullptr;
  InstInterval* d_ii = nullptr;
  InstInterval* d_ii_of_node = nullptr;
  long long* d_slice_node = nullptr;
  long long* d_first = nullptr;           // per active instance: its first time node (and the end)
  long long coef_total = 0;
  int iteration = 0;                      // iterations run so far on this interval
};

}  // namespace

struct spmc_plan_s {
  spmc_plan_desc d{};
  std::string err;
  int S = 1;
  int chunk = 512, threads = 256;   // chunk = samples per node in a cohort
  int JT = 12;                       // spatial nodes per cohort
  int* d_work = nullptr;             // persistent-kernel work counter
  void* d_state = nullptr;           // block-private walk state regions
  size_t state_bytes = 0;
  // event pipeline (forward sweep, d <= 2)
  int sweep_mode = 0;                // 0: event pipeline, 1: cohort kernel
  long long ev_batch = 0;            // samples per batch (0: automatic)
  unsigned int* d_counts = nullptr;  // (slice, node) counters / cursors
  unsigned int* d_starts = nullptr;  // segment starts
  unsigned long long* d_bsum = nullptr;
  unsigned long long* d_total = nullptr;  // events of the batch (scan total)
  long long counts_cap = 0, bsum_cap = 0;
  void* d_events = nullptr;          // events grouped by (slice, node)
  size_t events_bytes = 0;
  unsigned long long ev_cap = 0;     // events the buffer holds (0: not sized yet)
  unsigned long long* d_need = nullptr;   // largest batch total seen
  int* d_abort = nullptr;            // 0, or the iteration whose batch did not fit
  unsigned long long* d_counters_bak = nullptr;  // counters at the start of the running iteration
  unsigned long long* d_acc = nullptr;    // per (time node, node) exact sums: four limb counters
  long long acc_cap = 0;
  std::map<void*, size_t> allocs;    // device memory the plan holds
  long long ws_bytes = 0;
  bool use_graphs = true;            // spmc_solve: each interval as one captured CUDA graph
  int accel = 0;                     // 1: Aitken relaxation of the update
  double *d_eps_cur = nullptr, *d_eps_prev = nullptr, *d_omega = nullptr;
  long long eps_cap = 0;
  void* d_tc5 = nullptr;             // d = 5 mixed event sweep: slices in the tensor-core layout
  size_t tc5_bytes = 0;
  cudaStream_t cap_stream = nullptr; // the plan's own stream for capturing (any caller stream may launch)
  std::vector<HostProblem> probs;
  bool built = false;
  std::vector<double> xnodes;
  // device
  double* d_x = nullptr;
  double* d_xyd = nullptr;       // coordinates of every spatial node, [j][e] (S x dim), FP64
  float* d_xyf = nullptr;        // the same rounded to FP32
  double* d_times = nullptr;     // t_{n,l} of one interval (spmc_get_solution)
  double* d_frac = nullptr;      // the fractional case's table (kFrac* layout of spmc_tables.h)
  double* d_A = nullptr;
  double* d_B = nullptr;
  double* d_hw = nullptr;
  InstanceParams* d_ip = nullptr;
  double* d_u0 = nullptr;
  double* d_U = nullptr;
  double* d_coef = nullptr;
  double* d_rec = nullptr;       // d >= 3: two reconstruction buffers of coef_cap / 2 each
  void* d_slices = nullptr;
  SliceInfo* d_sinfo = nullptr;
  double* d_partial = nullptr;
  unsigned long long* d_counters = nullptr;
  unsigned long long* d_maxeps = nullptr;
  int* d_status = nullptr;
  long long U_total = 0;
  std::vector<long long> inst_off, inst_count;
  std::vector<std::vector<long long>> int_off;
  std::vector<Round> rounds;
  long long slice_cap = 0, partial_cap = 0, coef_cap = 0;
  int row = 32, half = 64;       // slice geometry: row width, entries of C (= of H)
  double shell = 1e-4;           // absorption shell in use
  long long sl_stride = 132;     // entries between slices (bank-spread)
  spmc_stats stats{};
  bool solved = false;
  bool timing = false;
  bool params_dirty = false;   // instance parameters / u0 changed, layout unchanged
  // adjoint workspace (spmc_grad)
  double *d_lambda = nullptr, *d_Ubak = nullptr, *d_iter = nullptr, *d_gT = nullptr, *d_lam = nullptr;
  double *d_mu = nullptr, *d_dLdz = nullptr, *d_gds = nullptr, *d_phi = nullptr;
  int* d_last = nullptr;
  std::vector<long long*> d_first_tn;   // per round: instance ranges of the time-node table
  bool grad_ready = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;  // recorded, not yet read
  std::vector<int> ev_cat;           // per pending pair: 0 sweep, 1 count walks + scan, 2 evaluation, 3 fill walks
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
};

namespace {

const char* kVersion = "spmc-b300 0.1 (sm_103a)";

#define SPMC_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      plan->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return e_ == cudaErrorMemoryAllocation ? SPMC_ERR_OOM : SPMC_ERR_CUDA;         \
    }                                                                                \
  } while (0)

spmc_status fail(spmc_plan_t plan, spmc_status st, const std::string& msg) {
  if (plan) plan->err = msg;
  return st;
}

// Device memory of a plan: every allocation is recorded, so that the plan can
// report the bytes it holds (spmc_stats.workspace_bytes) and free them all.
cudaError_t pmalloc(spmc_plan_t plan, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) { plan->allocs[*p] = bytes; plan->ws_bytes += (long long)bytes; }
  return e;
}
void pfree(spmc_plan_t plan, void* p) {
  if (!p) return;
  auto it = plan->allocs.find(p);
  if (it != plan->allocs.end()) { plan->ws_bytes -= (long long)it->second; plan->allocs.erase(it); }
  cudaFree(p);
}

int nstar_of(int n_ref, double s, double h) {
  double v = std::ceil((double)n_ref * s / h - 1e-9);
  return v < 1.0 ? 1 : (int)v;
}

template <typename T>
spmc_status upload(spmc_plan_t plan, T** dptr, const std::vector<T>& v) {
  if (*dptr) { pfree(plan, *dptr); *dptr = nullptr; }
  if (v.empty()) return SPMC_OK;
  SPMC_CUDA(pmalloc(plan, (void**)dptr, sizeof(T) * v.size()));
  SPMC_CUDA(cudaMemcpy(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return SPMC_OK;
}

size_t sweep_smem(int G, long long sl_stride, int W, size_t rsz) {
  return ((G * sl_stride * rsz + 15) / 16) * 16 + 3 * (size_t)W * sizeof(int);
}

size_t state_stride_bytes(int D, int W, size_t rsz) {
  size_t b = (size_t)W * ((D + 4) * rsz + 3 * sizeof(int));
  return (b + 255) / 256 * 256;
}

// Slice geometry: rows padded to the template width of the sweep (16-byte
// vector loads), consecutive slices offset by 4 banks (conflict-free reads of
// the n_sub slices of a window).
void slice_geometry(spmc_plan_t plan) {
  const int n = plan->d.n_space;
  int row = 32;
  if (plan->d.dim == 2) row = n <= 8 ? 8 : (n <= 16 ? 16 : (n <= 24 ? 24 : 32));
  if (plan->d.dim >= 3) row = plan->S;
  plan->row = row;
  plan->half = plan->d.dim == 2 ? n * row : row;
  long long SL = 2LL * plan->half;
  if (plan->d.precision == SPMC_FP64) plan->sl_stride = SL + ((2 - SL % 16) + 16) % 16;
  else plan->sl_stride = SL + ((4 - SL % 32) + 32) % 32;
}

// Build the per-interval work tables, the nodal layout and the workspace once
// every instance is set.
spmc_status build(spmc_plan_t plan) {
  const spmc_plan_desc& d = plan->d;
  const int S = plan->S, B = d.batch;
  for (int i = 0; i < B; ++i)
    if (!plan->probs[i].set) return fail(plan, SPMC_ERR_INVALID, "instance " + std::to_string(i) + " not set");
  // nodal layout: instance-major, interval blocks of (M_n+1) x S
  plan->inst_off.assign(B, 0);
  plan->inst_count.assign(B, 0);
  plan->int_off.assign(B, {});
  long long off = 0;
  for (int i = 0; i < B; ++i) {
    plan->inst_off[i] = off;
    for (int m = 0; m < plan->probs[i].n_int; ++m) {
      plan->int_off[i].push_back(off);
      off += (long long)(plan->probs[i].deg[m] + 1) * S;
    }
    plan->inst_count[i] = off - plan->inst_off[i];
  }
  plan->U_total = off;
  // time analysis matrices and hand-off weights per degree
  std::map<int, std::pair<long long, long long>> bmap;
  std::vector<double> Bh, Hh;
  std::vector<std::vector<double>> xi_of(d.max_degree + 1);
  for (int i = 0; i < B; ++i)
    for (int m = 0; m < plan->probs[i].n_int; ++m) {
      int Mt = plan->probs[i].deg[m];
      if (bmap.count(Mt)) continue;
      std::vector<double> Bm((Mt + 1) * (Mt + 1));
      time_analysis(d.time_family, Mt, Bm.data());
      long long bo = Bh.size(), ho = Hh.size();
      Bh.insert(Bh.end(), Bm.begin(), Bm.end());
      for (int k = 0; k <= Mt; ++k) {
        double s = 0.0;
        for (int q = 0; q <= Mt; ++q) s += Bm[q * (Mt + 1) + k];
        Hh.push_back(s);
      }
      bmap[Mt] = {bo, ho};
      xi_of[Mt].resize(Mt + 1);
      time_nodes(d.time_family, Mt, xi_of[Mt].data());
    }
  spmc_status st;
  if ((st = upload(plan, &plan->d_B, Bh)) != SPMC_OK) return st;
  if ((st = upload(plan, &plan->d_hw, Hh)) != SPMC_OK) return st;
  // rounds
  int R = 0;
  for (int i = 0; i < B; ++i) R = std::max(R, plan->probs[i].n_int);
  for (auto& r : plan->rounds) {
    pfree(plan, r.d_tn); pfree(plan, r.d_ii); pfree(plan, r.d_ii_of_node); pfree(plan, r.d_slice_node);
    pfree(plan, r.d_first);
  }
  plan->rounds.assign(R, Round());
  long long slice_cap = 0, partial_cap = 0, coef_cap = 0;
  const int n_chunks = (int)((d.M + plan->chunk - 1) / plan->chunk);
  for (int r = 0; r < R; ++r) {
    Round& rd = plan->rounds[r];
    long long coef_off = 0, slice_off = 0;
    for (int i = 0; i < B; ++i) {
      const HostProblem& P = plan->probs[i];
      if (r >= P.n_int) continue;
      int Mt = P.deg[r];
      InstInterval w{};
      w.inst = i; w.Mt = Mt; w.u_off = plan->int_off[i][r]; w.c_off = coef_off;
      w.b_off = bmap[Mt].first; w.h_off = bmap[Mt].second;
      w.next_u_off = (r + 1 < P.n_int) ? plan->int_off[i][r + 1] : -1;
      w.next_Mt = (r + 1 < P.n_int) ? P.deg[r + 1] : 0;
      w.t0 = P.t[r]; w.h = P.t[r + 1] - P.t[r];
      coef_off += 2LL * (Mt + 1) * S;
      rd.ii.push_back(w);
      const std::vector<double>& xi = xi_of[Mt];
      for (int l = 1; l <= Mt; ++l) {
        TimeNode t{};
        t.inst = i; t.ell = l; t.Mt = Mt; t.u_off = w.u_off; t.t0 = w.t0; t.h = w.h;
        double s = (xi[l] + 1.0) * 0.5 * w.h;
        t.t_node = w.t0 + s;
        t.nstar = nstar_of(d.n_ref, s, w.h);
        t.slice_base = slice_off;
        // the direct estimator's two slots after the walk grid: initial term, boundary term
        long long ns = (long long)d.n_sub * t.nstar + (d.estimator == SPMC_EST_DIRECT ? 2 : 0);
        for (long long m = 0; m < ns; ++m) rd.slice_node.push_back((long long)rd.tn.size());
        slice_off += ns;
        rd.tn.push_back(t);
        rd.ii_of_node.push_back(w);
      }
    }
    rd.n_slices = slice_off;
    rd.coef_total = coef_off;
    slice_cap = std::max(slice_cap, slice_off);
    partial_cap = std::max(partial_cap, (long long)rd.tn.size() * S * n_chunks);
    coef_cap = std::max(coef_cap, coef_off);
    if ((st = upload(plan, &rd.d_tn, rd.tn)) != SPMC_OK) return st;
    if ((st = upload(plan, &rd.d_ii, rd.ii)) != SPMC_OK) return st;
    if ((st = upload(plan, &rd.d_ii_of_node, rd.ii_of_node)) != SPMC_OK) return st;
    if ((st = upload(plan, &rd.d_slice_node, rd.slice_node)) != SPMC_OK) return st;
    std::vector<long long> first(rd.ii.size() + 1, 0);
    for (size_t a = 0; a < rd.ii.size(); ++a) first[a + 1] = first[a] + rd.ii[a].Mt;   // time nodes l = 1..M_n
    if ((st = upload(plan, &rd.d_first, first)) != SPMC_OK) return st;
  }
  // workspace
  pfree(plan, plan->d_U); pfree(plan, plan->d_coef); pfree(plan, plan->d_slices); pfree(plan, plan->d_sinfo);
  pfree(plan, plan->d_partial);
  plan->d_U = nullptr; plan->d_coef = nullptr; plan->d_slices = nullptr; plan->d_sinfo = nullptr; plan->d_partial = nullptr;
  size_t rsz = d.precision == SPMC_FP64 ? sizeof(double) : sizeof(float);
  SPMC_CUDA(pmalloc(plan, (void**)&plan->d_U, sizeof(double) * std::max(1LL, plan->U_total)));
  SPMC_CUDA(pmalloc(plan, (void**)&plan->d_coef, sizeof(double) * std::max(1LL, coef_cap)));
  pfree(plan, plan->d_rec);
  plan->d_rec = nullptr;
  if (d.dim >= 3) SPMC_CUDA(pmalloc(plan, (void**)&plan->d_rec, sizeof(double) * std::max(1LL, coef_cap)));
  slice_geometry(plan);
  SPMC_CUDA(pmalloc(plan, &plan->d_slices, rsz * plan->sl_stride * std::max(1LL, slice_cap)));
  SPMC_CUDA(pmalloc(plan, (void**)&plan->d_sinfo, sizeof(SliceInfo) * std::max(1LL, slice_cap)));
  SPMC_CUDA(pmalloc(plan, (void**)&plan->d_partial, sizeof(double) * std::max(1LL, partial_cap)));
  plan->slice_cap = slice_cap; plan->partial_cap = partial_cap; plan->coef_cap = coef_cap;
  std::vector<InstanceParams> ips(B);
  std::vector<double> u0(B * (size_t)S);
  for (int i = 0; i < B; ++i) {
    ips[i] = plan->probs[i].ip;
    std::copy(plan->probs[i].u0.begin(), plan->probs[i].u0.end(), u0.begin() + (size_t)i * S);
  }
  if ((st = upload(plan, &plan->d_ip, ips)) != SPMC_OK) return st;
  if ((st = upload(plan, &plan->d_u0, u0)) != SPMC_OK) return st;
  plan->built = true;
  plan->grad_ready = false;
  return SPMC_OK;
}

// Re-upload instance parameters and initial values (same partition and degrees).
spmc_status refresh_params(spmc_plan_t plan, cudaStream_t stream) {
  const int B = plan->d.batch, S = plan->S;
  static thread_local std::vector<InstanceParams> ips;
  static thread_local std::vector<double> u0;
  ips.resize(B);
  u0.resize((size_t)B * S);
  for (int i = 0; i < B; ++i) {
    ips[i] = plan->probs[i].ip;
    std::copy(plan->probs[i].u0.begin(), plan->probs[i].u0.end(), u0.begin() + (size_t)i * S);
  }
  SPMC_CUDA(cudaMemcpyAsync(plan->d_ip, ips.data(), sizeof(InstanceParams) * B, cudaMemcpyHostToDevice, stream));
  SPMC_CUDA(cudaMemcpyAsync(plan->d_u0, u0.data(), sizeof(double) * u0.size(), cudaMemcpyHostToDevice, stream));
  SPMC_CUDA(cudaStreamSynchronize(stream));
  plan->params_dirty = false;
  return SPMC_OK;
}

bool uses_events(spmc_plan_t plan);

// Non-zero boundary data and the direct estimator run on the event sweep only.
spmc_status check_event_only(spmc_plan_t plan) {
  bool need = plan->d.estimator == SPMC_EST_DIRECT || plan->d.basis == SPMC_BASIS_CHEB;
  for (const HostProblem& P : plan->probs) need = need || P.ip.bc_kind != SPMC_BC_ZERO;
  if (need && (plan->d.dim > 2 || !uses_events(plan)))
    return fail(plan, SPMC_ERR_UNSUPPORTED,
                "boundary data, the direct estimator and the Chebyshev basis need the event sweep (d <= 2, "
                "inside-ball walk)");
  return SPMC_OK;
}

spmc_status ensure_ready(spmc_plan_t plan, cudaStream_t stream) {
  spmc_status st = SPMC_OK;
  if (!plan->built) st = build(plan);
  else if (plan->params_dirty) st = refresh_params(plan, stream);
  if (st != SPMC_OK) return st;
  return check_event_only(plan);
}

// Arguments of the cohort sweep kernels for one iteration of round rd.
SweepArgs sweep_args(spmc_plan_t plan, const Round& rd, int interval, int iteration) {
  const spmc_plan_desc& d = plan->d;
  SweepArgs a{};
  a.tn = rd.d_tn; a.ip = plan->d_ip; a.xnodes = plan->d_x; a.slices = plan->d_slices; a.sinfo = plan->d_sinfo;
  a.partial = plan->d_partial; a.counters = plan->d_counters; a.status = plan->d_status;
  a.n = d.n_space; a.S = plan->S;
  a.chunk = plan->chunk;
  a.n_chunks = (int)((d.M + plan->chunk - 1) / plan->chunk);
  a.n_sub = d.n_sub;
  int gb = 0;
  while ((1 << gb) < d.n_sub) ++gb;
  a.gbits = gb; a.max_steps = d.max_steps; a.kappa = d.kappa; a.shell = plan->shell;
  a.k0 = (uint32_t)(d.seed & 0xffffffffULL); a.k1 = (uint32_t)(d.seed >> 32);
  a.interval = interval; a.iteration = iteration;
  a.walk_mode = d.walk_mode;
  a.frac = plan->d_frac;
  a.M = d.M;
  a.sl_stride = plan->sl_stride;
  a.half = plan->half;
  return a;
}

template <int D, int NMAX, typename R>
spmc_status launch_sweep(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const spmc_plan_desc& d = plan->d;
  SweepArgs a = sweep_args(plan, rd, interval, iteration);
  const int JT = std::min(plan->JT, plan->S);
  const int W = JT * plan->chunk;
  const long long n_jt = (plan->S + JT - 1) / JT;
  const long long n_cohorts = (long long)rd.tn.size() * n_jt * a.n_chunks;
  if (n_cohorts <= 0) return SPMC_OK;
  size_t smem = sweep_smem(d.n_sub, plan->sl_stride, W, sizeof(R));
  auto kern = sweep_kernel<D, NMAX, R>;
  SPMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, occ = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, plan->threads, smem));
  if (occ < 1) return fail(plan, SPMC_ERR_UNSUPPORTED, "sweep configuration does not fit on an SM");
  long long grid = std::min<long long>(n_cohorts, (long long)sms * occ);
  const size_t stride = state_stride_bytes(D, W, sizeof(R));
  if (plan->state_bytes < stride * grid) {
    pfree(plan, plan->d_state);
    plan->d_state = nullptr;
    plan->state_bytes = 0;
    SPMC_CUDA(pmalloc(plan, &plan->d_state, stride * grid));
    plan->state_bytes = stride * grid;
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_work, 0, sizeof(int), stream));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (plan->timing) {
    if (!plan->ev_free.empty()) { ev = plan->ev_free.back(); plan->ev_free.pop_back(); }
    else { SPMC_CUDA(cudaEventCreate(&ev.first)); SPMC_CUDA(cudaEventCreate(&ev.second)); }
    SPMC_CUDA(cudaEventRecord(ev.first, stream));
  }
  kern<<<(unsigned)grid, plan->threads, smem, stream>>>(a, JT, plan->chunk, n_cohorts, plan->d_work, plan->d_state,
                                                         (long long)stride);
  SPMC_CUDA(cudaGetLastError());
  if (plan->timing) {
    SPMC_CUDA(cudaEventRecord(ev.second, stream));
    plan->ev_pending.push_back(ev);
    plan->ev_cat.push_back(0);
  }
  return SPMC_OK;
}

template <typename R>
spmc_status launch_sweep5(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const spmc_plan_desc& d = plan->d;
  SweepArgs a = sweep_args(plan, rd, interval, iteration);
  const int JT = std::max(1, std::min(plan->JT, plan->S));
  const int W = JT * plan->chunk;
  const long long n_jt = (plan->S + JT - 1) / JT;
  const long long n_cohorts = (long long)rd.tn.size() * n_jt * a.n_chunks;
  if (n_cohorts <= 0) return SPMC_OK;
  const int n4 = d.n_space * d.n_space * d.n_space * d.n_space;
  size_t smem = ((2 * (size_t)n4 * sizeof(R) + 15) / 16) * 16 + (size_t)W * (5 * sizeof(int) + 6 * sizeof(R)) + 16;
  auto kern = sweep5_kernel<R>;
  SPMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, occ = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, plan->threads, smem));
  if (occ < 1) return fail(plan, SPMC_ERR_UNSUPPORTED, "5-D sweep configuration does not fit on an SM");
  long long grid = std::min<long long>(n_cohorts, (long long)sms * occ);
  const size_t stride = state_stride_bytes(5, W, sizeof(R));
  if (plan->state_bytes < stride * grid) {
    pfree(plan, plan->d_state);
    plan->d_state = nullptr;
    plan->state_bytes = 0;
    SPMC_CUDA(pmalloc(plan, &plan->d_state, stride * grid));
    plan->state_bytes = stride * grid;
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_work, 0, sizeof(int), stream));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (plan->timing) {
    if (!plan->ev_free.empty()) { ev = plan->ev_free.back(); plan->ev_free.pop_back(); }
    else { SPMC_CUDA(cudaEventCreate(&ev.first)); SPMC_CUDA(cudaEventCreate(&ev.second)); }
    SPMC_CUDA(cudaEventRecord(ev.first, stream));
  }
  kern<<<(unsigned)grid, plan->threads, smem, stream>>>(a, JT, plan->chunk, n_cohorts, plan->d_work, plan->d_state,
                                                         (long long)stride);
  SPMC_CUDA(cudaGetLastError());
  if (plan->timing) {
    SPMC_CUDA(cudaEventRecord(ev.second, stream));
    plan->ev_pending.push_back(ev);
    plan->ev_cat.push_back(0);
  }
  return SPMC_OK;
}

template <typename R>
spmc_status dispatch_sweep(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const int n = plan->d.n_space;
  if (plan->d.dim == 5) return launch_sweep5<R>(plan, stream, rd, interval, iteration);
  if (plan->d.dim == 1) return launch_sweep<1, 32, R>(plan, stream, rd, interval, iteration);
  if (plan->d.dim == 2) {
    if (n <= 8) return launch_sweep<2, 8, R>(plan, stream, rd, interval, iteration);
    if (n <= 16) return launch_sweep<2, 16, R>(plan, stream, rd, interval, iteration);
    if (n <= 24) return launch_sweep<2, 24, R>(plan, stream, rd, interval, iteration);
    return launch_sweep<2, 32, R>(plan, stream, rd, interval, iteration);
  }
  return fail(plan, SPMC_ERR_UNSUPPORTED, "dimension not built");
}

// The forward sweep is the event pipeline: d <= 2, or d = 5 in mixed precision
// (tensor-core evaluation), with the inside-ball walk and unless the cohort
// kernel is chosen.
bool uses_events(spmc_plan_t plan) {
  const spmc_plan_desc& d = plan->d;
  return (d.dim <= 2 || (d.dim == 5 && d.precision == SPMC_MIXED)) && plan->sweep_mode != SPMC_SWEEP_COHORT &&
         d.walk_mode == 0;
}

// Reconstruction (Step 1) and time slices of the current nodal values of round rd.
spmc_status prepare_slices(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  const int S = plan->S, n = plan->d.n_space, D = plan->d.dim;
  if (rd.ii.empty()) return SPMC_OK;
  const double t_off = plan->d.walk_mode >= 1 ? 0.0 : 0.5;   // step centres / sub-step midpoints
  const int* ab = plan->d_abort;
  if (D >= 3) {
    // reconstruction in global memory: time axis, then each space axis
    const long long half_cap = plan->coef_cap / 2;
    double* buf[2] = {plan->d_rec, plan->d_rec + half_cap};
    dim3 grid(256, (unsigned)rd.ii.size());
    mode_product_kernel<<<grid, 256, 0, stream>>>(rd.d_ii, plan->d_U, 1, buf[0], plan->d_A, plan->d_B, n, S, 0);
    int cur = 0;
    for (int e = 1; e <= D; ++e) {
      mode_product_kernel<<<grid, 256, 0, stream>>>(rd.d_ii, buf[cur], 0, buf[1 - cur], plan->d_A, plan->d_B, n, S, e);
      cur = 1 - cur;
    }
    coef_finish_kernel<<<grid, 256, 0, stream>>>(rd.d_ii, buf[cur], plan->d_coef, S);
    SPMC_CUDA(cudaGetLastError());
    if (rd.n_slices > 0 && uses_events(plan)) {
      // the slices of the tensor-core evaluation: [C | Lam_1 C | Lam_2 C | H], TF32 hi / lo
      const size_t need = Tc5::SLICE_BYTES * (size_t)rd.n_slices;
      if (plan->tc5_bytes < need) {
        pfree(plan, plan->d_tc5);
        plan->d_tc5 = nullptr;
        plan->tc5_bytes = 0;
        SPMC_CUDA(pmalloc(plan, &plan->d_tc5, need));
        plan->tc5_bytes = need;
      }
      slice5_tc_kernel<<<(unsigned)rd.n_slices, 256, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node,
                                                                   plan->d_coef, plan->d_ip,
                                                                   (unsigned char*)plan->d_tc5, plan->d_sinfo, n,
                                                                   plan->d.n_sub, t_off, ab);
      SPMC_CUDA(cudaGetLastError());
      return SPMC_OK;
    }
    if (rd.n_slices > 0) {
      if (plan->d.precision == SPMC_FP64)
        slice_kernel<5, double><<<(unsigned)rd.n_slices, 256, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (double*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
      else
        slice_kernel<5, float><<<(unsigned)rd.n_slices, 256, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (float*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
      SPMC_CUDA(cudaGetLastError());
    }
    return SPMC_OK;
  }
  int maxT = 0;
  for (auto& w : rd.ii) maxT = std::max(maxT, w.Mt + 1);
  size_t smem = sizeof(double) * 2 * (size_t)maxT * S;
  if (plan->d.basis == SPMC_BASIS_CHEB) {
    // the discrete Chebyshev transforms (FFT of the even extension for power-of-two lengths)
    if (D == 1) {
      SPMC_CUDA(cudaFuncSetAttribute(cheb_reconstruct_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      cheb_reconstruct_kernel<1><<<(unsigned)rd.ii.size(), 256, smem, stream>>>(rd.d_ii, plan->d_U, plan->d_coef, n, ab);
    } else {
      SPMC_CUDA(cudaFuncSetAttribute(cheb_reconstruct_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      cheb_reconstruct_kernel<2><<<(unsigned)rd.ii.size(), 256, smem, stream>>>(rd.d_ii, plan->d_U, plan->d_coef, n, ab);
    }
  } else if (D == 1) {
    SPMC_CUDA(cudaFuncSetAttribute(reconstruct_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    reconstruct_kernel<1><<<(unsigned)rd.ii.size(), 256, smem, stream>>>(rd.d_ii, plan->d_U, plan->d_A, plan->d_B,
                                                                          plan->d_coef, n, ab);
  } else {
    SPMC_CUDA(cudaFuncSetAttribute(reconstruct_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    reconstruct_kernel<2><<<(unsigned)rd.ii.size(), 256, smem, stream>>>(rd.d_ii, plan->d_U, plan->d_A, plan->d_B,
                                                                          plan->d_coef, n, ab);
  }
  SPMC_CUDA(cudaGetLastError());
  const bool fp64 = plan->d.precision == SPMC_FP64;
  if (rd.n_slices > 0) {
    if (D == 1) {
      if (fp64) slice_kernel<1, double><<<(unsigned)rd.n_slices, 128, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (double*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
      else slice_kernel<1, float><<<(unsigned)rd.n_slices, 128, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (float*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
    } else {
      if (fp64) slice_kernel<2, double><<<(unsigned)rd.n_slices, 256, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (double*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
      else slice_kernel<2, float><<<(unsigned)rd.n_slices, 256, 0, stream>>>(rd.d_tn, rd.d_slice_node, rd.d_ii_of_node, plan->d_coef, plan->d_ip, (float*)plan->d_slices, plan->d_sinfo, n, plan->d.n_sub, plan->row, plan->sl_stride, t_off, ab, plan->d.basis);
    }
    SPMC_CUDA(cudaGetLastError());
  }
  return SPMC_OK;
}

// The adjoint sweep of iteration `iteration` of round rd (same walks as the forward sweep).
template <int D, int NMAX, typename R>
spmc_status launch_adjoint_sweep(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const spmc_plan_desc& d = plan->d;
  SweepArgs a = sweep_args(plan, rd, interval, iteration);
  a.lambda = plan->d_lambda; a.gT = plan->d_gT; a.gds = plan->d_gds;
  const int JT = std::min(4, plan->S);
  const int W = JT * plan->chunk;
  const long long n_jt = (plan->S + JT - 1) / JT;
  const long long n_cohorts = (long long)rd.tn.size() * n_jt * a.n_chunks;
  if (n_cohorts <= 0) return SPMC_OK;
  size_t smem = sweep_smem(d.n_sub, plan->sl_stride, W, sizeof(R)) + (size_t)d.n_sub * 3 * plan->S * sizeof(double);
  auto kern = sweep_kernel<D, NMAX, R, true>;
  SPMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, occ = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, plan->threads, smem));
  if (occ < 1) return fail(plan, SPMC_ERR_UNSUPPORTED, "adjoint sweep configuration does not fit on an SM");
  long long grid = std::min<long long>(n_cohorts, (long long)sms * occ);
  const size_t stride = state_stride_bytes(D, W, sizeof(R));
  if (plan->state_bytes < stride * grid) {
    pfree(plan, plan->d_state);
    plan->d_state = nullptr;
    plan->state_bytes = 0;
    SPMC_CUDA(pmalloc(plan, &plan->d_state, stride * grid));
    plan->state_bytes = stride * grid;
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_work, 0, sizeof(int), stream));
  kern<<<(unsigned)grid, plan->threads, smem, stream>>>(a, JT, plan->chunk, n_cohorts, plan->d_work, plan->d_state,
                                                         (long long)stride);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

template <typename R>
spmc_status dispatch_adjoint(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const int n = plan->d.n_space;
  if (plan->d.dim == 1) return launch_adjoint_sweep<1, 32, R>(plan, stream, rd, interval, iteration);
  if (plan->d.dim == 2) {
    if (n <= 8) return launch_adjoint_sweep<2, 8, R>(plan, stream, rd, interval, iteration);
    if (n <= 16) return launch_adjoint_sweep<2, 16, R>(plan, stream, rd, interval, iteration);
    if (n <= 24) return launch_adjoint_sweep<2, 24, R>(plan, stream, rd, interval, iteration);
    return launch_adjoint_sweep<2, 32, R>(plan, stream, rd, interval, iteration);
  }
  return fail(plan, SPMC_ERR_UNSUPPORTED, "dimension not built");
}

spmc_status timer_begin(spmc_plan_t plan, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t>& ev);
spmc_status timer_end(spmc_plan_t plan, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t>& ev, int cat);

// Grow a device buffer to at least `need` bytes (contents are not kept).
spmc_status grow(spmc_plan_t plan, void** p, size_t* have, size_t need) {
  if (*have >= need) return SPMC_OK;
  pfree(plan, *p);
  *p = nullptr;
  *have = 0;
  SPMC_CUDA(pmalloc(plan, p, need));
  *have = need;
  return SPMC_OK;
}

template <int D, int NMAX, typename R>
void launch_eval(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  const size_t esmem = sizeof(R) * (size_t)plan->sl_stride;
  eval_events_kernel<D, NMAX, R><<<(unsigned)rd.n_slices, 256, esmem, stream>>>(
      rd.d_slice_node, rd.d_tn, plan->d_ip, plan->d_slices, plan->d_sinfo, plan->d_starts, plan->d_events,
      plan->d_acc, plan->d.n_space, plan->S, plan->sl_stride, plan->half, plan->d.kappa, plan->d.estimator,
      plan->d.basis, plan->d_total, plan->d_status, plan->d_abort);
}

// Tensor-core evaluation (d = 2, FP32 sweep).  The dynamic shared memory is
// padded so that at most 512 / TM_COLS blocks share an SM: their TMEM
// allocations then always fit and tcgen05.alloc never waits.  The grid is one
// resident wave (BLOCKS_PER_SM x the SM count, fewer for a small buffer); the
// blocks loop over the batch's event chunks (the total stays on the device).
template <int NMAX, bool FULL>
spmc_status launch_eval_tc_t(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  using Gm = TcGeom<NMAX>;
  const int smem = std::max(Gm::SMEM, 233472 / (Gm::BLOCKS_PER_SM + 1) + 1024);
  static bool attr_set[64] = {};
  int dev = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && !attr_set[dev]) {
    SPMC_CUDA(cudaFuncSetAttribute(eval_events_tc_kernel<NMAX, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
    attr_set[dev] = true;
  }
  int n_sm = 0;
  SPMC_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned long long chunks = (plan->ev_cap + Gm::CHUNK - 1) / Gm::CHUNK;
  const unsigned long long blocks = std::max(1ULL, std::min(chunks, (unsigned long long)Gm::BLOCKS_PER_SM * n_sm));
  eval_events_tc_kernel<NMAX, FULL><<<(unsigned)blocks, Gm::THREADS, smem, stream>>>(
      rd.d_slice_node, rd.d_tn, plan->d_ip, reinterpret_cast<const float*>(plan->d_slices), plan->d_sinfo,
      plan->d_starts, reinterpret_cast<const Event<float>*>(plan->d_events), plan->d_acc, plan->d.n_space, plan->S,
      rd.n_slices, plan->sl_stride, plan->half, plan->d.kappa, plan->d.estimator, plan->d_total, plan->d_status,
      plan->d_abort);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}
template <int NMAX>
spmc_status launch_eval_tc(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  return plan->d.n_space == NMAX ? launch_eval_tc_t<NMAX, true>(plan, stream, rd)
                                 : launch_eval_tc_t<NMAX, false>(plan, stream, rd);
}

// Give the event buffer room for `events` events plus a quarter (the batches of
// later iterations differ a little from the one measured).
// bytes of one event record of the plan's event sweep
size_t event_bytes(spmc_plan_t plan) {
  if (plan->d.dim == 5) return sizeof(Event5<float>);
  return plan->d.precision == SPMC_FP64 ? sizeof(Event<double>) : sizeof(Event<float>);
}

spmc_status size_event_buffer(spmc_plan_t plan, unsigned long long events) {
  if (events > 0xffffffffULL)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "event sweep: a batch holds 2^32 events or more; use a smaller batch");
  const size_t eb = event_bytes(plan);
  unsigned long long cap = events + events / 4 + (1ull << 16);
  cap = std::min<unsigned long long>(cap, 0xffffffffULL);
  if (grow(plan, &plan->d_events, &plan->events_bytes, eb * (size_t)cap) != SPMC_OK) return SPMC_ERR_OOM;
  plan->ev_cap = std::max<unsigned long long>(cap, plan->events_bytes / eb);
  plan->ev_cap = std::min<unsigned long long>(plan->ev_cap, 0xffffffffULL);
  return SPMC_OK;
}

// The 5-D tensor-core evaluation: one block per SM (196 KB of shared memory,
// 256 TMEM columns); the grid covers the event buffer's capacity.
spmc_status launch_eval5_tc(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  static bool attr_set[64] = {};
  int dev = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && !attr_set[dev]) {
    SPMC_CUDA(cudaFuncSetAttribute(eval5_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc5::SMEM));
    attr_set[dev] = true;
  }
  const unsigned long long blocks = (plan->ev_cap + Tc5::EV_CHUNK - 1) / Tc5::EV_CHUNK;
  if (blocks > 0x7fffffffULL) return fail(plan, SPMC_ERR_UNSUPPORTED, "event batch too large for one evaluation launch");
  eval5_tc_kernel<<<(unsigned)blocks, 128, Tc5::SMEM, stream>>>(
      rd.d_slice_node, rd.d_tn, plan->d_ip, reinterpret_cast<const unsigned char*>(plan->d_tc5), plan->d_sinfo,
      plan->d_starts, reinterpret_cast<const Event5<float>*>(plan->d_events), plan->d_acc, plan->d.n_space, plan->S,
      rd.n_slices, plan->d.kappa, plan->d_total, plan->d_status, plan->d_abort);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

// The forward sweep of one iteration as an event pipeline, batch after batch,
// with no return to the host: the event buffer was sized from a measured batch
// (the plan's first batch is measured here, once) and the scan checks every
// batch's total against it on the device (see the abort word in
// spmc_events.cuh).
// The adjoint evaluation of one batch's events (spmc_grad): gT, gds.
template <int D, int NMAX, typename R>
spmc_status launch_adj_eval(spmc_plan_t plan, cudaStream_t stream, const Round& rd) {
  constexpr int NA = (D == 2) ? 4 * NMAX : 3 * NMAX, NB = (D == 2) ? 2 * NMAX : 1;
  const size_t smem = sizeof(R) * ((((size_t)plan->sl_stride + 3) / 4) * 4 + 128 * (size_t)(NA + NB));
  SPMC_CUDA(cudaFuncSetAttribute(adj_events_kernel<D, NMAX, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  adj_events_kernel<D, NMAX, R><<<(unsigned)rd.n_slices, 256, smem, stream>>>(
      rd.d_slice_node, rd.d_tn, plan->d_ip, plan->d_slices, plan->d_sinfo, plan->d_starts, plan->d_events,
      plan->d_lambda, plan->d_gT, plan->d_gds, plan->d.n_space, plan->S, plan->sl_stride, plan->d.M, plan->d_total,
      plan->d_abort);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

template <int D, typename R>
spmc_status event_sweep_t(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration,
                          long long node_lo, long long node_cnt, bool adjoint = false) {
  const spmc_plan_desc& d = plan->d;
  const int S = plan->S;
  const long long n_tn = (long long)rd.tn.size();
  const long long nkeys = rd.n_slices * S;
  if (n_tn == 0 || nkeys == 0) return SPMC_OK;
  if (nkeys > 0xffffffffLL) return fail(plan, SPMC_ERR_UNSUPPORTED, "event sweep: more than 2^32 (slice, node) pairs");
  // the exact per-node sums take at most 2^32 additions per counter
  if ((double)d.M * (double)d.max_steps >= 4294967296.0)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "event sweep: M x max_steps reaches 2^32; use the cohort sweep");
  // workspace
  if (plan->counts_cap < nkeys) {
    pfree(plan, plan->d_counts); pfree(plan, plan->d_starts);
    plan->d_counts = nullptr; plan->d_starts = nullptr; plan->counts_cap = 0;
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_counts, sizeof(unsigned int) * nkeys));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_starts, sizeof(unsigned int) * nkeys));
    plan->counts_cap = nkeys;
  }
  const long long nblk = (nkeys + 1023) / 1024;
  if (plan->bsum_cap < nblk) {
    pfree(plan, plan->d_bsum);
    plan->d_bsum = nullptr; plan->bsum_cap = 0;
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_bsum, sizeof(unsigned long long) * nblk));
    plan->bsum_cap = nblk;
  }
  if (!plan->d_total) SPMC_CUDA(pmalloc(plan, (void**)&plan->d_total, sizeof(unsigned long long)));
  if (plan->acc_cap < n_tn * S) {
    pfree(plan, plan->d_acc);
    plan->d_acc = nullptr; plan->acc_cap = 0;
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_acc, 4 * sizeof(unsigned long long) * n_tn * S));
    plan->acc_cap = n_tn * S;
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_acc, 0, 4 * sizeof(unsigned long long) * n_tn * S, stream));
  EventArgs a;
  a.tn = rd.d_tn; a.ip = plan->d_ip; a.xnodes = plan->d_x; a.counts = plan->d_counts;
  a.xy = sizeof(R) == 4 ? (const void*)plan->d_xyf : (const void*)plan->d_xyd;
  a.div_S = FastDiv((uint32_t)S);
  a.direct = d.estimator == SPMC_EST_DIRECT ? 1 : 0;
  a.status = plan->d_status;
  a.abort = plan->d_abort;
  a.events = nullptr; a.cap = 0;
  a.n = d.n_space; a.S = S; a.n_sub = d.n_sub;
  int gb = 0;
  while ((1 << gb) < d.n_sub) ++gb;
  a.gbits = gb; a.max_steps = d.max_steps; a.interval = interval; a.iteration = iteration;
  a.n_tn = n_tn; a.kappa = d.kappa; a.shell = plan->shell;
  a.k0 = (uint32_t)(d.seed & 0xffffffffULL); a.k1 = (uint32_t)(d.seed >> 32);
  a.counters = plan->d_counters;
  a.node_lo = node_lo; a.node_cnt = node_cnt;
  int dev = 0, sms = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one wave of resident blocks: every thread then gets the same number of walks
  int occ_c = 0, occ_f = 0;
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, walk_events_kernel<D, R, false>, 256, 0));
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, walk_events_kernel<D, R, true>, 256, 0));
  const unsigned wgrid_c = (unsigned)(sms * std::max(1, occ_c));
  const unsigned wgrid_f = (unsigned)(sms * std::max(1, occ_f));
  // samples per batch: about 2^25 walks per batch
  long long nb = plan->ev_batch > 0 ? plan->ev_batch : std::max(1LL, (1LL << 25) / (n_tn * S));
  nb = std::min<long long>(nb, d.M);
  const int NMAXv = (D == 1) ? 32 : plan->row;
  for (long long i0 = 0; i0 < d.M; i0 += nb) {
    a.i0 = i0;
    a.nb = std::min<long long>(nb, d.M - i0);
    a.div_nb = FastDiv((uint32_t)std::min<long long>(a.nb, 0xffffffffLL));
    a.fast32 = (node_cnt * a.nb < (1LL << 32) && node_lo + node_cnt < (1LL << 32)) ? 1 : 0;
    std::pair<cudaEvent_t, cudaEvent_t> tw{nullptr, nullptr}, te{nullptr, nullptr};
    if (timer_begin(plan, stream, tw) != SPMC_OK) return SPMC_ERR_CUDA;
    SPMC_CUDA(cudaMemsetAsync(plan->d_counts, 0, sizeof(unsigned int) * nkeys, stream));
    walk_events_kernel<D, R, false><<<wgrid_c, 256, 0, stream>>>(a);
    SPMC_CUDA(cudaGetLastError());
    const bool measure = plan->ev_cap == 0;   // the plan's first batch sizes the event buffer
    scan_blocks_kernel<<<(unsigned)nblk, 256, 0, stream>>>(plan->d_counts, plan->d_bsum, nkeys, plan->d_abort);
    scan_totals_kernel<<<1, 1024, 0, stream>>>(plan->d_bsum, nblk, plan->d_total,
                                               measure ? ~0ull : plan->ev_cap, plan->d_need, plan->d_abort,
                                               iteration);
    scan_add_kernel<<<(unsigned)((nkeys + 255) / 256), 256, 0, stream>>>(plan->d_counts, plan->d_bsum,
                                                                          plan->d_starts, nkeys, plan->d_abort);
    SPMC_CUDA(cudaGetLastError());
    if (timer_end(plan, stream, tw, 1) != SPMC_OK) return SPMC_ERR_CUDA;
    if (measure) {
      unsigned long long total = 0;
      SPMC_CUDA(cudaMemcpyAsync(&total, plan->d_total, sizeof(total), cudaMemcpyDeviceToHost, stream));
      SPMC_CUDA(cudaStreamSynchronize(stream));
      spmc_status st = size_event_buffer(plan, std::max(total, 1ull));
      if (st != SPMC_OK) return st;
    }
    a.events = plan->d_events;
    a.cap = plan->ev_cap;
    std::pair<cudaEvent_t, cudaEvent_t> tf{nullptr, nullptr};
    if (timer_begin(plan, stream, tf) != SPMC_OK) return SPMC_ERR_CUDA;
    walk_events_kernel<D, R, true><<<wgrid_f, 256, 0, stream>>>(a);
    SPMC_CUDA(cudaGetLastError());
    if (timer_end(plan, stream, tf, 3) != SPMC_OK) return SPMC_ERR_CUDA;
    if (timer_begin(plan, stream, te) != SPMC_OK) return SPMC_ERR_CUDA;
    const bool tensor = D == 2 && sizeof(R) == 4 && plan->sweep_mode == SPMC_SWEEP_EVENTS &&
                        plan->d.basis != SPMC_BASIS_CHEB;
    if (adjoint) {
      if constexpr (D <= 2) {
        spmc_status as = D == 1 ? launch_adj_eval<1, 32, R>(plan, stream, rd)
                         : NMAXv == 8 ? launch_adj_eval<2, 8, R>(plan, stream, rd)
                         : NMAXv == 16 ? launch_adj_eval<2, 16, R>(plan, stream, rd)
                         : NMAXv == 24 ? launch_adj_eval<2, 24, R>(plan, stream, rd)
                                       : launch_adj_eval<2, 32, R>(plan, stream, rd);
        if (as != SPMC_OK) return as;
      }
    } else if constexpr (D == 5) {
      spmc_status ts = launch_eval5_tc(plan, stream, rd);
      if (ts != SPMC_OK) return ts;
    } else if (tensor) {
      spmc_status ts = NMAXv == 8 ? launch_eval_tc<8>(plan, stream, rd)
                       : NMAXv == 16 ? launch_eval_tc<16>(plan, stream, rd)
                       : NMAXv == 24 ? launch_eval_tc<24>(plan, stream, rd)
                                     : launch_eval_tc<32>(plan, stream, rd);
      if (ts != SPMC_OK) return ts;
    } else if constexpr (D == 1) launch_eval<1, 32, R>(plan, stream, rd);
    else if (NMAXv == 8) launch_eval<2, 8, R>(plan, stream, rd);
    else if (NMAXv == 16) launch_eval<2, 16, R>(plan, stream, rd);
    else if (NMAXv == 24) launch_eval<2, 24, R>(plan, stream, rd);
    else launch_eval<2, 32, R>(plan, stream, rd);
    SPMC_CUDA(cudaGetLastError());
    if (timer_end(plan, stream, te, 2) != SPMC_OK) return SPMC_ERR_CUDA;
  }
  return SPMC_OK;
}

// The event sweep over the (time node, spatial node) pairs ti S + j in
// [node_lo, node_lo + node_cnt) of round rd (node_cnt < 0: all of them).
spmc_status event_sweep(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration,
                        long long node_lo = 0, long long node_cnt = -1, bool adjoint = false) {
  if (node_cnt < 0) node_cnt = (long long)rd.tn.size() * plan->S - node_lo;
  const bool fp64 = plan->d.precision == SPMC_FP64;
  const long long a = node_lo, c = node_cnt;
  if (plan->d.dim == 5) return event_sweep_t<5, float>(plan, stream, rd, interval, iteration, a, c, adjoint);
  if (plan->d.dim == 1) return fp64 ? event_sweep_t<1, double>(plan, stream, rd, interval, iteration, a, c, adjoint)
                                    : event_sweep_t<1, float>(plan, stream, rd, interval, iteration, a, c, adjoint);
  return fp64 ? event_sweep_t<2, double>(plan, stream, rd, interval, iteration, a, c, adjoint)
              : event_sweep_t<2, float>(plan, stream, rd, interval, iteration, a, c, adjoint);
}

// Copy the point / capped counters aside at the start of an iteration (unless
// an earlier launch of the sequence aborted), so that an iteration that is run
// again does not also count its aborted batches.
__global__ void counters_snapshot_kernel(const unsigned long long* __restrict__ c, unsigned long long* __restrict__ bak,
                                         const int* __restrict__ abort) {
  if (*abort) return;
  if (threadIdx.x < 2) bak[threadIdx.x] = c[threadIdx.x];
}

// One residual iteration on interval r for every instance that has it,
// enqueued without synchronising the stream.
// The fixed-radius and alpha-stable walks (walk_mode 1, 2; d <= 2) run one
// thread per walk unless the cohort kernel is chosen.
bool uses_fixed_walk(spmc_plan_t plan) {
  return plan->d.dim <= 2 && plan->d.walk_mode >= 1 && plan->sweep_mode != SPMC_SWEEP_COHORT;
}

template <typename R>
spmc_status fixed_sweep_t(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval, int iteration) {
  const long long n_tn = (long long)rd.tn.size(), S = plan->S;
  if (plan->acc_cap < n_tn * S) {
    pfree(plan, plan->d_acc);
    plan->d_acc = nullptr; plan->acc_cap = 0;
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_acc, 4 * sizeof(unsigned long long) * n_tn * S));
    plan->acc_cap = n_tn * S;
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_acc, 0, 4 * sizeof(unsigned long long) * n_tn * S, stream));
  if (n_tn * S > 0xffffffffLL) return fail(plan, SPMC_ERR_UNSUPPORTED, "fixed walks: too many nodes");
  const SweepArgs a = sweep_args(plan, rd, interval, iteration);
  const long long n_walks = n_tn * S * plan->d.M;
  int dev = 0, sms = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)std::max(1LL, std::min((n_walks + 255) / 256, (long long)sms * 16));
  const int n = plan->d.n_space;
  if (plan->d.dim == 1) fixed_walk_kernel<1, 32, R><<<blocks, 256, 0, stream>>>(a, n_walks, plan->d_acc);
  else if (n <= 8) fixed_walk_kernel<2, 8, R><<<blocks, 256, 0, stream>>>(a, n_walks, plan->d_acc);
  else if (n <= 16) fixed_walk_kernel<2, 16, R><<<blocks, 256, 0, stream>>>(a, n_walks, plan->d_acc);
  else if (n <= 24) fixed_walk_kernel<2, 24, R><<<blocks, 256, 0, stream>>>(a, n_walks, plan->d_acc);
  else fixed_walk_kernel<2, 32, R><<<blocks, 256, 0, stream>>>(a, n_walks, plan->d_acc);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

spmc_status iterate_once(spmc_plan_t plan, cudaStream_t stream, int r) {
  Round& rd = plan->rounds[r];
  const int S = plan->S;
  const int iteration = ++rd.iteration;
  if (rd.ii.empty()) return SPMC_OK;
  counters_snapshot_kernel<<<1, 32, 0, stream>>>(plan->d_counters, plan->d_counters_bak, plan->d_abort);
  spmc_status pst = prepare_slices(plan, stream, rd);
  if (pst != SPMC_OK) return pst;
  bool fp64 = plan->d.precision == SPMC_FP64;
  const bool events = uses_events(plan);
  const bool fixed = uses_fixed_walk(plan);
  const bool exact_sums = events || fixed;   // per-node limb counters (else per-chunk FP64 sums)
  std::pair<cudaEvent_t, cudaEvent_t> tev{nullptr, nullptr};
  if (events && plan->timing) {
    if (!plan->ev_free.empty()) { tev = plan->ev_free.back(); plan->ev_free.pop_back(); }
    else { SPMC_CUDA(cudaEventCreate(&tev.first)); SPMC_CUDA(cudaEventCreate(&tev.second)); }
    SPMC_CUDA(cudaEventRecord(tev.first, stream));
  }
  spmc_status st = events ? event_sweep(plan, stream, rd, r, iteration)
                   : fixed ? (fp64 ? fixed_sweep_t<double>(plan, stream, rd, r, iteration)
                                   : fixed_sweep_t<float>(plan, stream, rd, r, iteration))
                           : (fp64 ? dispatch_sweep<double>(plan, stream, rd, r, iteration)
                                   : dispatch_sweep<float>(plan, stream, rd, r, iteration));
  if (st != SPMC_OK) return st;
  if (events && plan->timing) {
    SPMC_CUDA(cudaEventRecord(tev.second, stream));
    plan->ev_pending.push_back(tev);
    plan->ev_cat.push_back(0);
  }
  SPMC_CUDA(cudaMemsetAsync(plan->d_maxeps, 0, sizeof(unsigned long long) * plan->d.batch, stream));
  long long nn = (long long)rd.tn.size() * S;
  if (nn > 0 && plan->accel) {
    // Aitken relaxation: eps of every pair, then one block per instance
    if (plan->eps_cap < nn) {
      pfree(plan, plan->d_eps_cur); pfree(plan, plan->d_eps_prev);
      plan->d_eps_cur = plan->d_eps_prev = nullptr; plan->eps_cap = 0;
      SPMC_CUDA(pmalloc(plan, (void**)&plan->d_eps_cur, sizeof(double) * nn));
      SPMC_CUDA(pmalloc(plan, (void**)&plan->d_eps_prev, sizeof(double) * nn));
      plan->eps_cap = nn;
    }
    if (!plan->d_omega) SPMC_CUDA(pmalloc(plan, (void**)&plan->d_omega, sizeof(double) * plan->d.batch));
    if (exact_sums)
      eps_out_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(
          plan->d_acc, plan->d_eps_cur, 0, nn, 1.0 / (double)plan->d.M, plan->d_status, rd.d_tn, plan->d_U, S,
          plan->d.estimator, plan->d_abort);
    else
      eps_from_partial_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(
          plan->d_partial, plan->d_eps_cur, nn, (int)((plan->d.M + plan->chunk - 1) / plan->chunk),
          1.0 / (double)plan->d.M, plan->d_status);
    aitken_apply_kernel<<<(unsigned)rd.ii.size(), 256, 0, stream>>>(rd.d_ii, rd.d_tn, rd.d_first, plan->d_eps_cur,
                                                                    plan->d_eps_prev, plan->d_omega, plan->d_U,
                                                                    plan->d_maxeps, S, iteration == 1 ? 1 : 0,
                                                                    plan->d_abort);
    SPMC_CUDA(cudaGetLastError());
  } else if (nn > 0) {
    if (exact_sums)
      update_fixed_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(
          rd.d_tn, plan->d_acc, plan->d_U, nullptr, plan->d_maxeps, plan->d_status, nn, S, 1.0 / (double)plan->d.M,
          plan->d.estimator, plan->d_abort);
    else
      update_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(
          rd.d_tn, plan->d_partial, plan->d_U, nullptr, plan->d_maxeps, plan->d_status, nn, S,
          (int)((plan->d.M + plan->chunk - 1) / plan->chunk), 1.0 / (double)plan->d.M);
    SPMC_CUDA(cudaGetLastError());
  }
  return SPMC_OK;
}

spmc_status size_events(spmc_plan_t plan, unsigned long long events) { return size_event_buffer(plan, events); }

// If a batch of the sequence just synchronised did not fit the event buffer,
// grow the buffer to the largest batch seen, clear the abort word and restore
// the counters of the failed iteration's start; *failed gets that iteration
// (0: nothing aborted).  The stream must be synchronised.
spmc_status recover_abort(spmc_plan_t plan, cudaStream_t stream, int* failed) {
  int ab = 0;
  SPMC_CUDA(cudaMemcpyAsync(&ab, plan->d_abort, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SPMC_CUDA(cudaStreamSynchronize(stream));
  *failed = ab;
  if (ab == 0) return SPMC_OK;
  unsigned long long need = 0;
  SPMC_CUDA(cudaMemcpyAsync(&need, plan->d_need, sizeof(need), cudaMemcpyDeviceToHost, stream));
  SPMC_CUDA(cudaMemcpyAsync(plan->d_counters, plan->d_counters_bak, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, stream));
  SPMC_CUDA(cudaMemsetAsync(plan->d_abort, 0, sizeof(int), stream));
  SPMC_CUDA(cudaStreamSynchronize(stream));
  return size_events(plan, need);
}

// n_iter iterations of interval r, enqueued back to back; the stream is
// synchronised once at the end.  An iteration whose batch outgrew the event
// buffer (and everything after it, which returned at once) is run again with
// a larger buffer.
spmc_status run_iterations(spmc_plan_t plan, cudaStream_t stream, int r, int n_iter) {
  Round& rd = plan->rounds[r];
  const int last = rd.iteration + n_iter;
  for (int attempt = 0; attempt < 4; ++attempt) {
    while (rd.iteration < last) {
      spmc_status st = iterate_once(plan, stream, r);
      if (st != SPMC_OK) return st;
    }
    int failed = 0;
    spmc_status st = recover_abort(plan, stream, &failed);
    if (st != SPMC_OK) return st;
    if (failed == 0) return SPMC_OK;
    rd.iteration = failed - 1;
  }
  return fail(plan, SPMC_ERR_CUDA, "event sweep: the event buffer kept overflowing");
}

spmc_status begin_interval(spmc_plan_t plan, cudaStream_t stream, int r);

// One interval of spmc_solve -- the hand-off (or first iterate) and K
// iterations, about a thousand launches -- captured as one CUDA graph and
// launched at once.  Used for the event sweep once the plan's buffers hold this
// round (nothing is allocated or synchronised while capturing); otherwise, or
// if the capture fails, *done stays false and the caller runs the interval
// launch by launch.  A batch that outgrows the event buffer is handled as in
// run_iterations: the iterations from the failed one on run again eagerly.
spmc_status run_interval_graph(spmc_plan_t plan, cudaStream_t s, int r, int K, bool* done) {
  *done = false;
  Round& rd = plan->rounds[r];
  const spmc_plan_desc& d = plan->d;
  const bool events = d.dim <= 2 && plan->sweep_mode != SPMC_SWEEP_COHORT && d.walk_mode == 0;
  if (!plan->use_graphs || plan->timing || !events || rd.ii.empty() || plan->ev_cap == 0 ||
      plan->counts_cap < rd.n_slices * plan->S || plan->acc_cap < (long long)rd.tn.size() * plan->S ||
      plan->bsum_cap < (rd.n_slices * plan->S + 1023) / 1024 || !plan->d_total)
    return SPMC_OK;
  // capture on the plan's own stream (the caller's may be the legacy default
  // stream, which cannot be captured); nothing runs while capturing, and the
  // graph is launched on the caller's stream
  if (!plan->cap_stream && cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    plan->cap_stream = nullptr;
    return SPMC_OK;
  }
  cudaStream_t cs = plan->cap_stream;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) { cudaGetLastError(); return SPMC_OK; }
  spmc_status st = begin_interval(plan, cs, r);
  for (int k = 0; k < K && st == SPMC_OK; ++k) st = iterate_once(plan, cs, r);
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t x = nullptr;
  if (st != SPMC_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    plan->err.clear();
    rd.iteration = 0;
    return SPMC_OK;   // run it launch by launch instead
  }
  cudaGraphDestroy(g);
  const cudaError_t le = cudaGraphLaunch(x, s);
  cudaGraphExecDestroy(x);   // freed once the launch completes
  if (le != cudaSuccess) return fail(plan, SPMC_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(le));
  plan->stats.graph_launches += 1;
  *done = true;
  int failed = 0;
  if ((st = recover_abort(plan, s, &failed)) != SPMC_OK) return st;
  if (failed == 0) return SPMC_OK;
  rd.iteration = failed - 1;
  return run_iterations(plan, s, r, K - (failed - 1));
}

// Copy the round's nodal blocks between U and a contiguous buffer (offsets c_off/2).
__global__ void round_copy_kernel(const InstInterval* __restrict__ ii, double* __restrict__ U,
                                  double* __restrict__ buf, int S, int to_buf) {
  const InstInterval w = ii[blockIdx.x];
  const long long tot = (long long)(w.Mt + 1) * S;
  double* b = buf + w.c_off / 2;
  for (long long i = threadIdx.x; i < tot; i += blockDim.x) {
    if (to_buf) b[i] = U[w.u_off + i];
    else U[w.u_off + i] = b[i];
  }
}

// grad of the u0 coefficients: dL/dc_{c} = sum_j mu_j prod_e phi_{c_e}(x_{j_e}).
__global__ void u0_coef_grad_kernel(const double* __restrict__ mu, const double* __restrict__ phi,
                                    const int* __restrict__ ncoef, double* __restrict__ out, long long out_stride,
                                    int n, int S, int D) {
  const int inst = blockIdx.x;
  const int nc = ncoef[inst];
  if (nc <= 0) return;
  int NC = 1;
  for (int e = 0; e < D; ++e) NC *= nc;
  for (int c = threadIdx.x; c < NC; c += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < S; ++j) {
      double prod = mu[(long long)inst * S + j];
      int jj = j, cc = c;
      for (int e = 0; e < D; ++e) { prod *= phi[(jj % n) * n + (cc % nc)]; jj /= n; cc /= nc; }
      acc += prod;
    }
    out[(long long)inst * out_stride + c] = acc;
  }
}

spmc_status begin_interval(spmc_plan_t plan, cudaStream_t stream, int r) {
  Round& rd = plan->rounds[r];
  rd.iteration = 0;
  if (r == 0) {
    if (!rd.ii.empty()) {
      const unsigned g = (unsigned)rd.ii.size();
      const int n = plan->d.n_space;
      if (plan->d.dim == 1) init_first_kernel<1><<<g, 256, 0, stream>>>(rd.d_ii, plan->d_u0, plan->d_U, plan->S, plan->d_ip, plan->d_x, n);
      else if (plan->d.dim == 2) init_first_kernel<2><<<g, 256, 0, stream>>>(rd.d_ii, plan->d_u0, plan->d_U, plan->S, plan->d_ip, plan->d_x, n);
      else init_first_kernel<5><<<g, 256, 0, stream>>>(rd.d_ii, plan->d_u0, plan->d_U, plan->S, plan->d_ip, plan->d_x, n);
    }
  } else {
    Round& prev = plan->rounds[r - 1];
    if (!prev.ii.empty())
      handoff_kernel<<<(unsigned)prev.ii.size(), 256, 0, stream>>>(prev.d_ii, plan->d_hw, plan->d_U, plan->S);
  }
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

spmc_status read_status(spmc_plan_t plan, cudaStream_t stream) {
  int h = 0;
  SPMC_CUDA(cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SPMC_CUDA(cudaStreamSynchronize(stream));
  if (h & 1) return fail(plan, SPMC_ERR_NONFINITE, "a non-finite eps was produced");
  if (h & 2) return fail(plan, SPMC_ERR_TIMEOUT, "a sweep block exceeded its round budget");
  if (h & 4) return fail(plan, SPMC_ERR_CUDA, "event sweep: an event fell outside its segment");
  if (h & 8) return fail(plan, SPMC_ERR_TIMEOUT, "tensor-core evaluation: an MMA did not complete in time");
  return SPMC_OK;
}

spmc_status read_max_eps(spmc_plan_t plan, cudaStream_t stream, double* out) {
  std::vector<unsigned long long> bits(plan->d.batch);
  SPMC_CUDA(cudaMemcpyAsync(bits.data(), plan->d_maxeps, sizeof(unsigned long long) * bits.size(),
                            cudaMemcpyDeviceToHost, stream));
  SPMC_CUDA(cudaStreamSynchronize(stream));
  double mx = 0.0;
  for (auto b : bits) { double v; std::memcpy(&v, &b, sizeof v); mx = std::max(mx, v); }
  *out = mx;
  return SPMC_OK;
}

void drain_timing(spmc_plan_t plan) {
  for (size_t i = 0; i < plan->ev_pending.size(); ++i) {
    auto& ev = plan->ev_pending[i];
    const int cat = i < plan->ev_cat.size() ? plan->ev_cat[i] : 0;
    float ms = 0.f;
    if (cudaEventSynchronize(ev.second) == cudaSuccess && cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
      if (cat == 0) { plan->stats.sweep_ms += ms; plan->stats.sweep_launches += 1; }
      else if (cat == 1) plan->stats.walk_ms += ms;
      else if (cat == 3) plan->stats.fill_ms += ms;
      else { plan->stats.eval_ms += ms; plan->stats.eval_launches += 1; }
    }
    plan->ev_free.push_back(ev);
  }
  plan->ev_pending.clear();
  plan->ev_cat.clear();
}

// Start / end a timed region on the stream (no-op unless timing is on).
spmc_status timer_begin(spmc_plan_t plan, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t>& ev) {
  if (!plan->timing) return SPMC_OK;
  if (!plan->ev_free.empty()) { ev = plan->ev_free.back(); plan->ev_free.pop_back(); }
  else { SPMC_CUDA(cudaEventCreate(&ev.first)); SPMC_CUDA(cudaEventCreate(&ev.second)); }
  SPMC_CUDA(cudaEventRecord(ev.first, s));
  return SPMC_OK;
}
spmc_status timer_end(spmc_plan_t plan, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t>& ev, int cat) {
  if (!plan->timing) return SPMC_OK;
  SPMC_CUDA(cudaEventRecord(ev.second, s));
  plan->ev_pending.push_back(ev);
  plan->ev_cat.push_back(cat);
  return SPMC_OK;
}

void sync_counters(spmc_plan_t plan) {
  drain_timing(plan);
  unsigned long long c[2] = {0, 0};
  if (cudaMemcpy(c, plan->d_counters, sizeof c, cudaMemcpyDeviceToHost) == cudaSuccess) {
    plan->stats.points = (long long)c[0];
    plan->stats.capped = (long long)c[1];
  }
}

}  // namespace

// ------------------------------------------------------------------ static scratch
// Device scratch of spmc_iterate_static: one array per GPU, for callers that
// cannot allocate at the call.  Host code must not use g_static_scratch as an
// address (it is a host-side stand-in); its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current.
static __device__ __align__(256) unsigned char g_static_scratch[SPMC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

spmc_status static_scratch(spmc_plan_t plan, void** out) {
  int dev = -1;
  SPMC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(plan, SPMC_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      plan->err = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
      return SPMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SPMC_OK;
}

// The sweep of one iteration with its scratch in the static array: one cohort of
// one node x chunk per block, as many resident blocks as the array holds.
template <int D, int NMAX, typename R>
spmc_status launch_sweep_static(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval,
                                int iteration, unsigned char* scratch, double* partial, size_t partial_bytes) {
  const spmc_plan_desc& d = plan->d;
  SweepArgs a = sweep_args(plan, rd, interval, iteration);
  a.partial = partial;
  const int JT = 1;
  const int W = plan->chunk;
  const long long n_cohorts = (long long)rd.tn.size() * plan->S * a.n_chunks;
  if (n_cohorts <= 0) return SPMC_OK;
  size_t smem = sweep_smem(d.n_sub, plan->sl_stride, W, sizeof(R));
  auto kern = sweep_kernel<D, NMAX, R>;
  SPMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, occ = 0;
  SPMC_CUDA(cudaGetDevice(&dev));
  SPMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, plan->threads, smem));
  if (occ < 1) return fail(plan, SPMC_ERR_UNSUPPORTED, "sweep configuration does not fit on an SM");
  const size_t stride = state_stride_bytes(D, W, sizeof(R));
  const size_t head = 256 + partial_bytes;                    // counter, then chunk sums, then walk state
  const long long fit = (long long)((SPMC_STATIC_SCRATCH_BYTES - head) / stride);
  long long grid = std::min<long long>(n_cohorts, std::min<long long>((long long)sms * occ, fit));
  if (grid < 1) return fail(plan, SPMC_ERR_UNSUPPORTED, "static scratch too small for one block's walk state");
  int* work = reinterpret_cast<int*>(scratch);
  SPMC_CUDA(cudaMemsetAsync(work, 0, sizeof(int), stream));
  kern<<<(unsigned)grid, plan->threads, smem, stream>>>(a, JT, plan->chunk, n_cohorts, work, scratch + head,
                                                         (long long)stride);
  SPMC_CUDA(cudaGetLastError());
  return SPMC_OK;
}

template <typename R>
spmc_status dispatch_sweep_static(spmc_plan_t plan, cudaStream_t stream, const Round& rd, int interval,
                                  int iteration, unsigned char* scratch, double* partial, size_t pb) {
  const int n = plan->d.n_space;
  if (plan->d.dim == 1) return launch_sweep_static<1, 32, R>(plan, stream, rd, interval, iteration, scratch, partial, pb);
  if (plan->d.dim == 2) {
    if (n <= 8) return launch_sweep_static<2, 8, R>(plan, stream, rd, interval, iteration, scratch, partial, pb);
    if (n <= 16) return launch_sweep_static<2, 16, R>(plan, stream, rd, interval, iteration, scratch, partial, pb);
    if (n <= 24) return launch_sweep_static<2, 24, R>(plan, stream, rd, interval, iteration, scratch, partial, pb);
    return launch_sweep_static<2, 32, R>(plan, stream, rd, interval, iteration, scratch, partial, pb);
  }
  return fail(plan, SPMC_ERR_UNSUPPORTED, "dimension not built");
}

}  // namespace

// =================================================================== C-ABI
extern "C" {

const char* spmc_version(void) { return kVersion; }

spmc_status spmc_plan(const spmc_plan_desc* desc, spmc_plan_t* out) {
  if (!out) return SPMC_ERR_INVALID;
  *out = nullptr;
  if (!desc) return SPMC_ERR_INVALID;
  const spmc_plan_desc& d = *desc;
  if (d.dim < 1 || d.dim > 5 || d.n_space < 2 || d.n_space > 32 || d.max_intervals < 1 || d.max_degree < 1 ||
      d.max_degree > 39 || d.M < 1 || d.K < 1 || d.n_ref < 1 || d.n_sub < 1 || d.n_sub > 16 ||
      (d.n_sub & (d.n_sub - 1)) || !(d.shell >= 0.0) || d.shell >= 0.5 || d.max_steps < 1 || !(d.kappa > 0.0) || d.batch < 1 ||
      (d.time_family != SPMC_TIME_LGL && d.time_family != SPMC_TIME_RADAU_LEFT && d.time_family != SPMC_TIME_CHEB) ||
      (d.basis != SPMC_BASIS_JACOBI && d.basis != SPMC_BASIS_CHEB) ||
      ((d.basis == SPMC_BASIS_CHEB) != (d.time_family == SPMC_TIME_CHEB)) ||
      (d.precision != SPMC_FP64 && d.precision != SPMC_MIXED) || d.M > 0x7fffffffLL ||
      (d.walk_mode < 0 || d.walk_mode > 2) || (d.estimator != SPMC_EST_RESIDUAL && d.estimator != SPMC_EST_DIRECT) ||
      (d.walk_mode == 2) != (d.alpha > 0.0 && d.alpha < 2.0))
    return SPMC_ERR_INVALID;
  if (d.dim != 1 && d.dim != 2 && d.dim != 5) return SPMC_ERR_UNSUPPORTED;
  if (d.dim == 5 && d.n_space > 8) return SPMC_ERR_UNSUPPORTED;
  if (d.dim <= 2) {
    // the reconstruction keeps two (M_n+1) x n^d FP64 blocks in shared memory
    double S = std::pow((double)d.n_space, d.dim);
    if (2.0 * (d.max_degree + 1) * S * 8.0 > 227.0 * 1024.0) return SPMC_ERR_UNSUPPORTED;
  }
  if (d.tol > 0.0 && d.batch > 1) return SPMC_ERR_UNSUPPORTED;
  if (d.walk_mode == 1 && d.dim > 2) return SPMC_ERR_UNSUPPORTED;
  if (d.walk_mode == 2 && d.dim != 1) return SPMC_ERR_UNSUPPORTED;   // the fractional case: d = 1
  if (d.basis == SPMC_BASIS_CHEB && (d.dim > 2 || d.walk_mode != 0)) return SPMC_ERR_UNSUPPORTED;
  if (d.estimator == SPMC_EST_DIRECT && (d.dim > 2 || d.walk_mode != 0)) return SPMC_ERR_UNSUPPORTED;
  spmc_plan_t plan = new spmc_plan_s();
  plan->d = d;
  if (d.walk_mode >= 1) plan->d.n_sub = 1;   // one evaluation time per step: its centre
  plan->S = 1;
  for (int e = 0; e < d.dim; ++e) plan->S *= d.n_space;
  plan->probs.assign(d.batch, HostProblem());
  plan->chunk = (int)std::min<long long>(d.precision == SPMC_FP64 ? 256 : 512, ((d.M + 31) / 32) * 32);
  plan->JT = (d.precision == SPMC_FP64 ? 4096 : 6144) / plan->chunk;
  if (d.dim == 5) {
    plan->chunk = (int)std::min<long long>(256, ((d.M + 31) / 32) * 32);
    plan->JT = 4;
  }
  slice_geometry(plan);
  plan->threads = 256;
  // tables
  const int n = d.n_space;
  const bool frac = d.walk_mode == 2;
  plan->xnodes.resize(n);
  if (frac) space_nodes_frac(n, d.alpha, plan->xnodes.data());
  else if (d.basis == SPMC_BASIS_CHEB) space_nodes_cheb(n, plan->xnodes.data());
  else space_nodes(n, plan->xnodes.data());
  // shell == 0: half the distance of the outermost node to the boundary, at most 2e-3
  plan->shell = d.shell > 0.0 ? d.shell : std::min(2e-3, 0.5 * (1.0 - std::fabs(plan->xnodes[0])));
  std::vector<double> A(n * n);
  if (frac) space_analysis_frac(n, d.alpha, A.data());
  else if (d.basis == SPMC_BASIS_CHEB) space_analysis_cheb(n, A.data());
  else space_analysis(n, A.data());
  spmc_status st;
  if ((st = upload(plan, &plan->d_x, plan->xnodes)) != SPMC_OK) { spmc_destroy(plan); return st; }
  {
    // node j's coordinates: digit e of j in base n (x fastest) picks xnodes
    std::vector<double> xyd((size_t)plan->S * d.dim);
    std::vector<float> xyf(xyd.size());
    for (long long j = 0; j < plan->S; ++j) {
      long long jr = j;
      for (int e = 0; e < d.dim; ++e) {
        xyd[(size_t)j * d.dim + e] = plan->xnodes[jr % n];
        xyf[(size_t)j * d.dim + e] = (float)plan->xnodes[jr % n];
        jr /= n;
      }
    }
    if ((st = upload(plan, &plan->d_xyd, xyd)) != SPMC_OK) { spmc_destroy(plan); return st; }
    if ((st = upload(plan, &plan->d_xyf, xyf)) != SPMC_OK) { spmc_destroy(plan); return st; }
  }
  if ((st = upload(plan, &plan->d_A, A)) != SPMC_OK) { spmc_destroy(plan); return st; }
  if (frac) {
    std::vector<double> T(kFracTable);
    frac_table(d.alpha, T.data());
    if ((st = upload(plan, &plan->d_frac, T)) != SPMC_OK) { spmc_destroy(plan); return st; }
  }
  double ra[kMaxModes], rb[kMaxModes], lam[kMaxModes];
  float raf[kMaxModes], rbf[kMaxModes], lamf[kMaxModes];
  for (int p = 0; p < kMaxModes; ++p) {
    ra[p] = p >= 2 ? (2.0 * p + 1.0) * (p + 1.0) / (p * (p + 2.0)) : 0.0;
    rb[p] = p >= 2 ? (p + 1.0) / (p + 2.0) : 0.0;
    lam[p] = (p + 1.0) * (p + 2.0);
    raf[p] = (float)ra[p]; rbf[p] = (float)rb[p]; lamf[p] = (float)lam[p];
  }
  cudaError_t e = cudaMemcpyToSymbol(c_ra_d, ra, sizeof ra);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rb_d, rb, sizeof rb);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_lam_d, lam, sizeof lam);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ra_f, raf, sizeof raf);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rb_f, rbf, sizeof rbf);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_lam_f, lamf, sizeof lamf);
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_counters, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(plan->d_counters, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_maxeps, sizeof(unsigned long long) * d.batch);
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_status, sizeof(int));
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_work, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(plan->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_abort, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(plan->d_abort, 0, sizeof(int));
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_need, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(plan->d_need, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = pmalloc(plan, (void**)&plan->d_counters_bak, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(plan->d_counters_bak, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    spmc_status r = (e == cudaErrorMemoryAllocation) ? SPMC_ERR_OOM : SPMC_ERR_CUDA;
    spmc_destroy(plan);
    return r;
  }
  *out = plan;
  return SPMC_OK;
}

spmc_status spmc_set_problem(spmc_plan_t plan, int instance, const spmc_problem* prob) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!prob || instance < 0 || instance >= plan->d.batch) return fail(plan, SPMC_ERR_INVALID, "bad instance or problem");
  const spmc_plan_desc& d = plan->d;
  const spmc_problem& p = *prob;
  if (p.n_intervals < 1 || p.n_intervals > d.max_intervals || !p.t_breaks || !p.degrees || !p.u0)
    return fail(plan, SPMC_ERR_INVALID, "bad interval count or null array");
  for (int m = 0; m < p.n_intervals; ++m) {
    if (!(p.t_breaks[m + 1] > p.t_breaks[m])) return fail(plan, SPMC_ERR_INVALID, "t_breaks not increasing");
    if (p.degrees[m] < 1 || p.degrees[m] > d.max_degree) return fail(plan, SPMC_ERR_INVALID, "degree out of range");
  }
  if (p.f_kind != SPMC_F_POLY3 && p.f_kind != SPMC_F_SIN) return fail(plan, SPMC_ERR_INVALID, "bad f_kind");
  if (p.ex_kind < SPMC_EX_NONE || p.ex_kind > SPMC_EX_FRAC_POLY) return fail(plan, SPMC_ERR_INVALID, "bad ex_kind");
  if (p.bc_kind < SPMC_BC_ZERO || p.bc_kind > SPMC_BC_RAW) return fail(plan, SPMC_ERR_INVALID, "bad bc_kind");
  if ((p.ex_kind == SPMC_EX_COSTHIRD || p.ex_kind == SPMC_EX_SINPLUS) && p.bc_kind == SPMC_BC_ZERO)
    return fail(plan, SPMC_ERR_INVALID, "ex_kind 4 and 5 have non-zero boundary values: bc_kind LIFT or RAW");
  if (p.bc_kind == SPMC_BC_RAW && d.estimator != SPMC_EST_DIRECT)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "raw boundary data enters through the direct estimator only");
  if (p.bc_kind != SPMC_BC_ZERO && (d.dim > 2 || d.walk_mode != 0))
    return fail(plan, SPMC_ERR_UNSUPPORTED, "boundary data: d <= 2 and the inside-ball walk only");
  const bool frac_kind = p.ex_kind == SPMC_EX_FRAC_SIN || p.ex_kind == SPMC_EX_FRAC_POLY;
  if (d.walk_mode == 2 && !(frac_kind || p.ex_kind == SPMC_EX_NONE))
    return fail(plan, SPMC_ERR_INVALID, "the fractional case takes ex_kind 0, 6 or 7");
  if (d.walk_mode != 2 && frac_kind) return fail(plan, SPMC_ERR_INVALID, "ex_kind 6 and 7 need the fractional case");
  if ((d.walk_mode == 2 || d.basis != SPMC_BASIS_JACOBI) && p.u0_kind != SPMC_U0_NODAL)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "the fractional case and the Chebyshev basis take nodal initial values");
  HostProblem& H = plan->probs[instance];
  bool same_layout = H.set && H.n_int == p.n_intervals &&
                     std::equal(H.deg.begin(), H.deg.end(), p.degrees) &&
                     std::equal(H.t.begin(), H.t.end(), p.t_breaks);
  H.n_int = p.n_intervals;
  H.t.assign(p.t_breaks, p.t_breaks + p.n_intervals + 1);
  H.deg.assign(p.degrees, p.degrees + p.n_intervals);
  H.ip.f_kind = p.f_kind; H.ip.ex_kind = p.ex_kind;
  for (int k = 0; k < 4; ++k) H.ip.fc[k] = p.f_coef[k];
  H.ip.f_scale = p.f_scale; H.ip.ex_beta = p.ex_beta;
  H.ip.bc_kind = p.bc_kind;
  const int S = plan->S, n = d.n_space, D = d.dim;
  H.u0.assign(S, 0.0);
  H.u0_kind = p.u0_kind;
  if (p.u0_kind == SPMC_U0_NODAL) {
    H.u0.assign(p.u0, p.u0 + S);
  } else if (p.u0_kind == SPMC_U0_PHI_COEF) {
    if (p.n_coef < 1 || p.n_coef > n) return fail(plan, SPMC_ERR_INVALID, "n_coef out of range");
    H.n_coef = p.n_coef;
    int nc = 1;
    for (int e = 0; e < D; ++e) nc *= p.n_coef;
    H.u0_coef.assign(p.u0, p.u0 + nc);
    std::vector<double> ph((size_t)n * n);  // ph[j*n + p] = phi_p(x_j)
    for (int j = 0; j < n; ++j) phi_values(n, plan->xnodes[j], &ph[(size_t)j * n]);
    for (int j = 0; j < S; ++j) {
      double acc = 0.0;
      for (int c = 0; c < nc; ++c) {
        double prod = p.u0[c];
        int jj = j, cc = c;
        for (int e = 0; e < D; ++e) { prod *= ph[(size_t)(jj % n) * n + (cc % p.n_coef)]; jj /= n; cc /= p.n_coef; }
        acc += prod;
      }
      H.u0[j] = acc;
    }
  } else {
    return fail(plan, SPMC_ERR_INVALID, "bad u0_kind");
  }
  H.set = true;
  if (plan->built && same_layout) plan->params_dirty = true;
  else plan->built = false;
  plan->solved = false;
  return SPMC_OK;
}

spmc_status spmc_solution_layout(spmc_plan_t plan, int instance, long long* offset, long long* count) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) { spmc_status st = build(plan); if (st != SPMC_OK) return st; }
  if (instance < 0 || instance >= plan->d.batch || !offset || !count) return fail(plan, SPMC_ERR_INVALID, "bad instance");
  *offset = plan->inst_off[instance];
  *count = plan->inst_count[instance];
  return SPMC_OK;
}

spmc_status spmc_begin_interval(spmc_plan_t plan, void* cuda_stream, int interval) {
  if (!plan) return SPMC_ERR_INVALID;
  { spmc_status st = ensure_ready(plan, (cudaStream_t)cuda_stream); if (st != SPMC_OK) return st; }
  if (interval < 0 || interval >= (int)plan->rounds.size()) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  return begin_interval(plan, (cudaStream_t)cuda_stream, interval);
}

spmc_status spmc_iterate(spmc_plan_t plan, void* cuda_stream, int interval, int n_iter, double* max_eps_host) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) return fail(plan, SPMC_ERR_INVALID, "call spmc_begin_interval first");
  if (interval < 0 || interval >= (int)plan->rounds.size() || n_iter < 0) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  spmc_status st = check_event_only(plan);
  if (st != SPMC_OK) return st;
  st = run_iterations(plan, s, interval, n_iter);
  if (st != SPMC_OK) return st;
  st = read_status(plan, s);
  if (st != SPMC_OK) return st;
  double mx = 0.0;
  if ((st = read_max_eps(plan, s, &mx)) != SPMC_OK) return st;
  if (max_eps_host) *max_eps_host = mx;
  plan->stats.iterations_run = n_iter;
  plan->stats.last_max_eps = mx;
  sync_counters(plan);
  return SPMC_OK;
}

spmc_status spmc_solve(spmc_plan_t plan, void* cuda_stream, double* u_nodes) {
  if (!plan) return SPMC_ERR_INVALID;
  { spmc_status st = ensure_ready(plan, (cudaStream_t)cuda_stream); if (st != SPMC_OK) return st; }
  if (!u_nodes) return fail(plan, SPMC_ERR_INVALID, "null output");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const spmc_plan_desc& d = plan->d;
  int total_iters = 0;
  double mx = 0.0;
  for (int r = 0; r < (int)plan->rounds.size(); ++r) {
    spmc_status st;
    if (d.tol <= 0.0) {
      bool done = false;
      if ((st = run_interval_graph(plan, s, r, d.K, &done)) != SPMC_OK) return st;
      if (done) { total_iters += d.K; continue; }
    }
    st = begin_interval(plan, s, r);
    if (st != SPMC_OK) return st;
    if (d.tol > 0.0) {
      for (int k = 0; k < d.K; ++k) {
        if ((st = run_iterations(plan, s, r, 1)) != SPMC_OK) return st;
        ++total_iters;
        if ((st = read_max_eps(plan, s, &mx)) != SPMC_OK) return st;
        if (mx < d.tol) break;
      }
    } else {
      if ((st = run_iterations(plan, s, r, d.K)) != SPMC_OK) return st;
      total_iters += d.K;
    }
  }
  SPMC_CUDA(cudaMemcpyAsync(u_nodes, plan->d_U, sizeof(double) * plan->U_total, cudaMemcpyDefault, s));
  spmc_status st = read_status(plan, s);
  if (st != SPMC_OK) return st;
  plan->stats.iterations_run = total_iters;
  plan->solved = true;
  return SPMC_OK;
}

spmc_status spmc_get_nodes(spmc_plan_t plan, void* cuda_stream, int instance, int interval, double* dst) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) return fail(plan, SPMC_ERR_INVALID, "plan not built");
  if (instance < 0 || instance >= plan->d.batch || !dst) return fail(plan, SPMC_ERR_INVALID, "bad instance");
  const HostProblem& P = plan->probs[instance];
  if (interval < 0 || interval >= P.n_int) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  size_t cnt = (size_t)(P.deg[interval] + 1) * plan->S;
  SPMC_CUDA(cudaMemcpyAsync(dst, plan->d_U + plan->int_off[instance][interval], sizeof(double) * cnt,
                            cudaMemcpyDefault, (cudaStream_t)cuda_stream));
  return SPMC_OK;
}

spmc_status spmc_get_solution(spmc_plan_t plan, void* cuda_stream, int instance, int interval, double* dst) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) return fail(plan, SPMC_ERR_INVALID, "plan not built");
  if (instance < 0 || instance >= plan->d.batch || !dst) return fail(plan, SPMC_ERR_INVALID, "bad instance");
  const HostProblem& P = plan->probs[instance];
  if (interval < 0 || interval >= P.n_int) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int Mt = P.deg[interval], T = Mt + 1, S = plan->S;
  // t_{n,l} of the interval's time nodes
  std::vector<double> xi(T), tt(T);
  time_nodes(plan->d.time_family, Mt, xi.data());
  for (int l = 0; l < T; ++l) tt[l] = P.t[interval] + (xi[l] + 1.0) * 0.5 * (P.t[interval + 1] - P.t[interval]);
  if (!plan->d_times) SPMC_CUDA(pmalloc(plan, (void**)&plan->d_times, sizeof(double) * 64));
  SPMC_CUDA(cudaMemcpyAsync(plan->d_times, tt.data(), sizeof(double) * T, cudaMemcpyHostToDevice, s));
  const long long tot = (long long)T * S;
  const unsigned g = (unsigned)std::min(4096LL, (tot + 255) / 256);
  const double* U = plan->d_U + plan->int_off[instance][interval];
  const int n = plan->d.n_space;
  if (plan->d.dim == 1) solution_kernel<1><<<g, 256, 0, s>>>(U, dst, plan->d_ip, instance, plan->d_times, plan->d_x, n, S, T);
  else if (plan->d.dim == 2) solution_kernel<2><<<g, 256, 0, s>>>(U, dst, plan->d_ip, instance, plan->d_times, plan->d_x, n, S, T);
  else solution_kernel<5><<<g, 256, 0, s>>>(U, dst, plan->d_ip, instance, plan->d_times, plan->d_x, n, S, T);
  SPMC_CUDA(cudaGetLastError());
  // the host vector of times must outlive the copy
  SPMC_CUDA(cudaStreamSynchronize(s));
  return SPMC_OK;
}

spmc_status spmc_set_nodes(spmc_plan_t plan, void* cuda_stream, int instance, int interval, const double* src) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) { spmc_status st = build(plan); if (st != SPMC_OK) return st; }
  if (instance < 0 || instance >= plan->d.batch || !src) return fail(plan, SPMC_ERR_INVALID, "bad instance");
  const HostProblem& P = plan->probs[instance];
  if (interval < 0 || interval >= P.n_int) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  size_t cnt = (size_t)(P.deg[interval] + 1) * plan->S;
  SPMC_CUDA(cudaMemcpyAsync(plan->d_U + plan->int_off[instance][interval], src, sizeof(double) * cnt,
                            cudaMemcpyDefault, (cudaStream_t)cuda_stream));
  return SPMC_OK;
}

spmc_status spmc_iterate_static(spmc_plan_t plan, void* cuda_stream, int interval, double* max_eps_host) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built || plan->params_dirty)
    return fail(plan, SPMC_ERR_INVALID, "spmc_iterate_static needs a built plan: call spmc_begin_interval first");
  if (plan->d.dim > 2) return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_iterate_static: dimensions 1 and 2 only");
  for (const HostProblem& P : plan->probs)
    if (P.ip.bc_kind != SPMC_BC_ZERO || plan->d.estimator != SPMC_EST_RESIDUAL || plan->d.basis != SPMC_BASIS_JACOBI)
      return fail(plan, SPMC_ERR_UNSUPPORTED,
                  "spmc_iterate_static: zero boundary data, the residual iteration and the Jacobi basis only");
  if (interval < 0 || interval >= (int)plan->rounds.size()) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  Round& rd = plan->rounds[interval];
  const int S = plan->S;
  const int n_chunks = (int)((plan->d.M + plan->chunk - 1) / plan->chunk);
  const long long nn = (long long)rd.tn.size() * S;
  const size_t partial_bytes = ((size_t)nn * n_chunks * sizeof(double) + 255) / 256 * 256;
  if (partial_bytes + 256 >= SPMC_STATIC_SCRATCH_BYTES)
    return fail(plan, SPMC_ERR_UNSUPPORTED,
                "spmc_iterate_static: the chunk sums of this problem exceed the 16 MiB static scratch");
  void* base = nullptr;
  spmc_status st = static_scratch(plan, &base);
  if (st != SPMC_OK) return st;
  unsigned char* scratch = reinterpret_cast<unsigned char*>(base);
  double* partial = reinterpret_cast<double*>(scratch + 256);
  const int iteration = rd.iteration + 1;
  if (!rd.ii.empty()) {
    // reconstruction and slices as in spmc_iterate (these launches allocate nothing)
    st = prepare_slices(plan, stream, rd);
    if (st != SPMC_OK) return st;
    const bool fp64 = plan->d.precision == SPMC_FP64;
    st = fp64 ? dispatch_sweep_static<double>(plan, stream, rd, interval, iteration, scratch, partial, partial_bytes)
              : dispatch_sweep_static<float>(plan, stream, rd, interval, iteration, scratch, partial, partial_bytes);
    if (st != SPMC_OK) return st;
    SPMC_CUDA(cudaMemsetAsync(plan->d_maxeps, 0, sizeof(unsigned long long) * plan->d.batch, stream));
    if (nn > 0) {
      update_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(rd.d_tn, partial, plan->d_U, nullptr,
                                                                      plan->d_maxeps, plan->d_status, nn, S,
                                                                      n_chunks, 1.0 / (double)plan->d.M);
      SPMC_CUDA(cudaGetLastError());
    }
  }
  rd.iteration = iteration;
  // status, counters and max |eps| through fixed host buffers (no allocation)
  int hs = 0;
  unsigned long long cnt2[2] = {0, 0};
  SPMC_CUDA(cudaMemcpyAsync(&hs, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SPMC_CUDA(cudaMemcpyAsync(cnt2, plan->d_counters, sizeof cnt2, cudaMemcpyDeviceToHost, stream));
  double mx = 0.0;
  unsigned long long bits[64];
  for (int b0 = 0; b0 < plan->d.batch; b0 += 64) {
    const int cnt = std::min(64, plan->d.batch - b0);
    SPMC_CUDA(cudaMemcpyAsync(bits, plan->d_maxeps + b0, sizeof(unsigned long long) * cnt, cudaMemcpyDeviceToHost,
                              stream));
    SPMC_CUDA(cudaStreamSynchronize(stream));
    for (int i = 0; i < cnt; ++i) { double v; std::memcpy(&v, &bits[i], sizeof v); mx = std::max(mx, v); }
  }
  if (hs & 1) return fail(plan, SPMC_ERR_NONFINITE, "a non-finite eps was produced");
  if (hs & 2) return fail(plan, SPMC_ERR_TIMEOUT, "a sweep block exceeded its pass budget");
  plan->stats.points = (long long)cnt2[0];
  plan->stats.capped = (long long)cnt2[1];
  plan->stats.iterations_run = 1;
  plan->stats.last_max_eps = mx;
  if (max_eps_host) *max_eps_host = mx;
  return SPMC_OK;
}

spmc_status spmc_round_nodes(spmc_plan_t plan, int interval, long long* n_pairs) {
  if (!plan || !n_pairs) return SPMC_ERR_INVALID;
  if (!plan->built) return fail(plan, SPMC_ERR_INVALID, "plan not built");
  if (interval < 0 || interval >= (int)plan->rounds.size()) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  *n_pairs = (long long)plan->rounds[interval].tn.size() * plan->S;
  return SPMC_OK;
}

spmc_status spmc_iterate_shard(spmc_plan_t plan, void* cuda_stream, int interval, int rank, int world,
                               double* eps_pairs) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built || plan->params_dirty) return fail(plan, SPMC_ERR_INVALID, "call spmc_begin_interval first");
  if (interval < 0 || interval >= (int)plan->rounds.size() || world < 1 || rank < 0 || rank >= world || !eps_pairs)
    return fail(plan, SPMC_ERR_INVALID, "bad interval, rank or output");
  if (plan->d.dim > 2 || plan->sweep_mode == SPMC_SWEEP_COHORT || plan->d.walk_mode != 0)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_iterate_shard: the event sweep only (d <= 2, inside-ball walk)");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Round& rd = plan->rounds[interval];
  const long long n = (long long)rd.tn.size() * plan->S;
  const long long lo = n * rank / world, hi = n * (rank + 1) / world;
  if (rd.ii.empty() || hi <= lo) return SPMC_OK;
  const int iteration = rd.iteration + 1;   // spmc_apply_eps advances the count
  for (int attempt = 0; attempt < 4; ++attempt) {
    counters_snapshot_kernel<<<1, 32, 0, s>>>(plan->d_counters, plan->d_counters_bak, plan->d_abort);
    spmc_status st = prepare_slices(plan, s, rd);
    if (st == SPMC_OK) st = event_sweep(plan, s, rd, interval, iteration, lo, hi - lo);
    if (st != SPMC_OK) return st;
    eps_out_kernel<<<(unsigned)((hi - lo + 255) / 256), 256, 0, s>>>(plan->d_acc, eps_pairs, lo, hi,
                                                                   1.0 / (double)plan->d.M, plan->d_status, rd.d_tn,
                                                                   plan->d_U, plan->S, plan->d.estimator,
                                                                   plan->d_abort);
    SPMC_CUDA(cudaGetLastError());
    int failed = 0;
    if ((st = recover_abort(plan, s, &failed)) != SPMC_OK) return st;
    if (failed == 0) return read_status(plan, s);
  }
  return fail(plan, SPMC_ERR_CUDA, "event sweep: the event buffer kept overflowing");
}

spmc_status spmc_apply_eps(spmc_plan_t plan, void* cuda_stream, int interval, const double* eps_pairs,
                           double* max_eps_host) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built) return fail(plan, SPMC_ERR_INVALID, "call spmc_begin_interval first");
  if (interval < 0 || interval >= (int)plan->rounds.size() || !eps_pairs)
    return fail(plan, SPMC_ERR_INVALID, "bad interval or input");
  if (plan->accel) return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_apply_eps: Aitken relaxation is not sharded");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Round& rd = plan->rounds[interval];
  rd.iteration += 1;
  const long long n = (long long)rd.tn.size() * plan->S;
  SPMC_CUDA(cudaMemsetAsync(plan->d_maxeps, 0, sizeof(unsigned long long) * plan->d.batch, s));
  if (n > 0) {
    apply_eps_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rd.d_tn, eps_pairs, plan->d_U, plan->d_maxeps,
                                                                 plan->d_status, n, plan->S);
    SPMC_CUDA(cudaGetLastError());
  }
  spmc_status st = read_status(plan, s);
  if (st != SPMC_OK) return st;
  double mx = 0.0;
  if ((st = read_max_eps(plan, s, &mx)) != SPMC_OK) return st;
  if (max_eps_host) *max_eps_host = mx;
  plan->stats.iterations_run = 1;
  plan->stats.last_max_eps = mx;
  return SPMC_OK;
}

spmc_status spmc_grad(spmc_plan_t plan, void* cuda_stream, const double* dloss_du_T, double* grad_f_scale,
                      double* grad_u0_coef) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->solved) return fail(plan, SPMC_ERR_INVALID, "spmc_grad needs a prior spmc_solve on this plan");
  if (!dloss_du_T) return fail(plan, SPMC_ERR_INVALID, "null dL/du(T)");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const spmc_plan_desc& d = plan->d;
  const int S = plan->S, n = d.n_space, D = d.dim, B = d.batch, K = d.K;
  const int R = (int)plan->rounds.size();
  if (d.tol > 0.0) return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_grad needs a fixed iteration count (tol <= 0)");
  if (d.dim > 2) return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_grad: dimensions 1 and 2 only");
  if (d.walk_mode == 2 || d.basis != SPMC_BASIS_JACOBI)
    return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_grad: not for the fractional case or the Chebyshev basis");
  for (const HostProblem& P : plan->probs)
    if (P.ip.bc_kind != SPMC_BC_ZERO || d.estimator != SPMC_EST_RESIDUAL)
      return fail(plan, SPMC_ERR_UNSUPPORTED, "spmc_grad: zero boundary data and the residual iteration only");
  // workspace (first call)
  if (!plan->grad_ready) {
    pfree(plan, plan->d_lambda); pfree(plan, plan->d_Ubak); pfree(plan, plan->d_iter); pfree(plan, plan->d_gT);
    pfree(plan, plan->d_lam); pfree(plan, plan->d_mu); pfree(plan, plan->d_dLdz); pfree(plan, plan->d_gds);
    pfree(plan, plan->d_phi); pfree(plan, plan->d_last);
    for (auto p : plan->d_first_tn) pfree(plan, p);
    plan->d_lambda = plan->d_Ubak = plan->d_iter = plan->d_gT = plan->d_lam = nullptr;
    plan->d_mu = plan->d_dLdz = plan->d_gds = plan->d_phi = nullptr;
    plan->d_last = nullptr;
    long long maxblk = 0;
    for (auto& rd : plan->rounds) maxblk = std::max(maxblk, rd.coef_total / 2);
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_lambda, sizeof(double) * std::max(1LL, plan->U_total)));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_Ubak, sizeof(double) * std::max(1LL, plan->U_total)));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_iter, sizeof(double) * std::max(1LL, maxblk * K)));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_gT, sizeof(double) * 3 * S * std::max(1LL, plan->slice_cap)));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_lam, sizeof(double) * std::max(1LL, 3 * plan->coef_cap / 2)));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_mu, sizeof(double) * (size_t)B * S));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_dLdz, sizeof(double) * (size_t)B * S));
    SPMC_CUDA(pmalloc(plan, (void**)&plan->d_gds, sizeof(double) * B));
    std::vector<int> last(B);
    for (int i = 0; i < B; ++i) last[i] = plan->probs[i].n_int - 1;
    spmc_status st;
    if ((st = upload(plan, &plan->d_last, last)) != SPMC_OK) return st;
    std::vector<double> ph((size_t)n * n);
    for (int j = 0; j < n; ++j) phi_values(n, plan->xnodes[j], &ph[(size_t)j * n]);
    if ((st = upload(plan, &plan->d_phi, ph)) != SPMC_OK) return st;
    plan->d_first_tn.assign(R, nullptr);
    for (int r = 0; r < R; ++r) {
      const Round& rd = plan->rounds[r];
      std::vector<long long> first(rd.ii.size() + 1, 0);
      long long t = 0;
      for (size_t a = 0; a < rd.ii.size(); ++a) {
        first[a] = t;
        while (t < (long long)rd.tn.size() && rd.tn[t].inst == rd.ii[a].inst) ++t;
      }
      first[rd.ii.size()] = t;
      if ((st = upload(plan, &plan->d_first_tn[r], first)) != SPMC_OK) return st;
    }
    plan->grad_ready = true;
  }
  SPMC_CUDA(cudaMemcpyAsync(plan->d_dLdz, dloss_du_T, sizeof(double) * (size_t)B * S, cudaMemcpyDefault, s));
  SPMC_CUDA(cudaMemsetAsync(plan->d_gds, 0, sizeof(double) * B, s));
  SPMC_CUDA(cudaMemsetAsync(plan->d_mu, 0, sizeof(double) * (size_t)B * S, s));
  SPMC_CUDA(cudaMemcpyAsync(plan->d_Ubak, plan->d_U, sizeof(double) * plan->U_total, cudaMemcpyDeviceToDevice, s));
  const bool fp64 = d.precision == SPMC_FP64;
  spmc_status st = SPMC_OK;
  for (int r = R - 1; r >= 0 && st == SPMC_OK; --r) {
    Round& rd = plan->rounds[r];
    if (rd.ii.empty()) continue;
    const unsigned nb = (unsigned)rd.ii.size();
    const long long blk = rd.coef_total / 2;
    // recompute the interval's iterates U^(0..K-1) from its first iterate
    if ((st = begin_interval(plan, s, r)) != SPMC_OK) break;
    for (int k = 0; k < K; ++k) {
      round_copy_kernel<<<nb, 256, 0, s>>>(rd.d_ii, plan->d_U, plan->d_iter + (long long)k * blk, S, 1);
      if (k + 1 < K && (st = run_iterations(plan, s, r, 1)) != SPMC_OK) break;
    }
    if (st != SPMC_OK) break;
    adj_lambda_init_kernel<<<nb, 256, 0, s>>>(rd.d_ii, plan->d_last, plan->d_hw, plan->d_dLdz, plan->d_mu,
                                              plan->d_lambda, r, S);
    SPMC_CUDA(cudaGetLastError());
    int maxT = 0;
    for (auto& w : rd.ii) maxT = std::max(maxT, w.Mt + 1);
    const size_t csm = sizeof(double) * 2 * (size_t)maxT * S;
    for (int k = K; k >= 1; --k) {
      round_copy_kernel<<<nb, 256, 0, s>>>(rd.d_ii, plan->d_U, plan->d_iter + (long long)(k - 1) * blk, S, 0);
      if ((st = prepare_slices(plan, s, rd)) != SPMC_OK) break;
      SPMC_CUDA(cudaMemsetAsync(plan->d_gT, 0, sizeof(double) * 3 * S * std::max(1LL, rd.n_slices), s));
      if (uses_events(plan)) {
        // the iteration's own events (same walks), adjoint evaluation per slice.  The
        // forward run of this iteration sized the event buffer for these very
        // batches, so none can overflow; if one did, the gradient is refused.
        st = event_sweep(plan, s, rd, r, k, 0, -1, true);
        if (st != SPMC_OK) break;
        int failed = 0;
        if ((st = recover_abort(plan, s, &failed)) != SPMC_OK) break;
        if (failed) { st = fail(plan, SPMC_ERR_CUDA, "adjoint event sweep: a batch outgrew the event buffer"); break; }
      } else {
        st = fp64 ? dispatch_adjoint<double>(plan, s, rd, r, k) : dispatch_adjoint<float>(plan, s, rd, r, k);
      }
      if (st != SPMC_OK) break;
      adj_time_kernel<<<nb, 256, 0, s>>>(rd.d_ii, rd.d_tn, plan->d_first_tn[r], plan->d_sinfo, plan->d_gT,
                                         plan->d_lam, S, d.n_sub);
      if (D == 1) {
        SPMC_CUDA(cudaFuncSetAttribute(adj_combine_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        adj_combine_kernel<1><<<nb, 256, csm, s>>>(rd.d_ii, plan->d_lam, plan->d_A, plan->d_B, plan->d_lambda, n, d.kappa);
      } else {
        SPMC_CUDA(cudaFuncSetAttribute(adj_combine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        adj_combine_kernel<2><<<nb, 256, csm, s>>>(rd.d_ii, plan->d_lam, plan->d_A, plan->d_B, plan->d_lambda, n, d.kappa);
      }
      SPMC_CUDA(cudaGetLastError());
    }
    if (st != SPMC_OK) break;
    adj_mu_kernel<<<nb, 256, 0, s>>>(rd.d_ii, plan->d_lambda, plan->d_mu, S);
    SPMC_CUDA(cudaGetLastError());
  }
  // the forward solution is restored whatever happened
  SPMC_CUDA(cudaMemcpyAsync(plan->d_U, plan->d_Ubak, sizeof(double) * plan->U_total, cudaMemcpyDeviceToDevice, s));
  if (st != SPMC_OK) return st;
  if (grad_f_scale)
    SPMC_CUDA(cudaMemcpyAsync(grad_f_scale, plan->d_gds, sizeof(double) * B, cudaMemcpyDefault, s));
  if (grad_u0_coef) {
    int maxnc = 0;
    std::vector<int> nc(B);
    for (int i = 0; i < B; ++i) { nc[i] = plan->probs[i].u0_kind == SPMC_U0_PHI_COEF ? plan->probs[i].n_coef : 0; maxnc = std::max(maxnc, nc[i]); }
    if (maxnc > 0) {
      long long NC = 1;
      for (int e = 0; e < D; ++e) NC *= maxnc;
      int* d_nc = nullptr;
      if ((st = upload(plan, &d_nc, nc)) != SPMC_OK) return st;
      u0_coef_grad_kernel<<<(unsigned)B, 128, 0, s>>>(plan->d_mu, plan->d_phi, d_nc, grad_u0_coef, NC, n, S, D);
      SPMC_CUDA(cudaGetLastError());
      SPMC_CUDA(cudaStreamSynchronize(s));
      pfree(plan, d_nc);
    }
  }
  return read_status(plan, s);
}

spmc_status spmc_autotune(spmc_plan_t plan, void* cuda_stream, int interval, double* best_ms) {
  if (!plan) return SPMC_ERR_INVALID;
  if (!plan->built || plan->params_dirty)
    return fail(plan, SPMC_ERR_INVALID, "spmc_autotune needs a built plan: call spmc_begin_interval first");
  if (interval < 0 || interval >= (int)plan->rounds.size()) return fail(plan, SPMC_ERR_INVALID, "bad interval");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Round& rd = plan->rounds[interval];
  if (rd.ii.empty()) return SPMC_OK;
  const bool fp64 = plan->d.precision == SPMC_FP64;
  // reconstruction and slices of the current nodal values (left unchanged)
  spmc_status st = prepare_slices(plan, s, rd);
  if (st != SPMC_OK) return st;
  // the trial sweeps leave the points / capped counters as they were
  unsigned long long saved[2] = {0, 0};
  SPMC_CUDA(cudaMemcpyAsync(saved, plan->d_counters, sizeof saved, cudaMemcpyDeviceToHost, s));
  SPMC_CUDA(cudaStreamSynchronize(s));
  cudaEvent_t e0, e1;
  SPMC_CUDA(cudaEventCreate(&e0));
  SPMC_CUDA(cudaEventCreate(&e1));
  const bool timing = plan->timing;
  plan->timing = false;
  float best = 1e30f;
  if (uses_events(plan)) {
    // event sweep: samples per batch for 2^23 .. 2^26 walks per batch
    const long long keep = plan->ev_batch;
    long long best_nb = keep;
    const long long walks_per_sample = std::max<long long>(1, (long long)rd.tn.size() * plan->S);
    for (int lg = 23; lg <= 26; ++lg) {
      const long long nb = std::max<long long>(1, std::min<long long>(plan->d.M, (1LL << lg) / walks_per_sample));
      plan->ev_batch = nb;
      for (int attempt = 0; attempt < 3; ++attempt) {   // a larger batch may first outgrow the event buffer
        SPMC_CUDA(cudaEventRecord(e0, s));
        st = event_sweep(plan, s, rd, interval, rd.iteration + 1);
        if (st != SPMC_OK) break;
        SPMC_CUDA(cudaEventRecord(e1, s));
        SPMC_CUDA(cudaEventSynchronize(e1));
        int failed = 0;
        if ((st = recover_abort(plan, s, &failed)) != SPMC_OK || failed == 0) break;
      }
      if (st != SPMC_OK) break;
      float ms = 0.f;
      SPMC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; best_nb = nb; }
      if (nb >= plan->d.M) break;
    }
    plan->ev_batch = (st == SPMC_OK) ? best_nb : keep;
  } else {
    // candidate cohort widths that fit two blocks per SM (FP32) / one (FP64)
    const int wmax = plan->d.dim == 5 ? 2048 : (fp64 ? 4096 : 6144);
    const int cands[] = {1, 2, 4, 6, 8, 12, 16, 24, 32};
    const int keep = plan->JT;
    int best_jt = keep;
    for (int jt : cands) {
      if (jt * plan->chunk > wmax || (jt > plan->S && jt != 1)) continue;
      plan->JT = jt;
      SPMC_CUDA(cudaEventRecord(e0, s));
      st = fp64 ? dispatch_sweep<double>(plan, s, rd, interval, rd.iteration + 1)
                : dispatch_sweep<float>(plan, s, rd, interval, rd.iteration + 1);
      if (st != SPMC_OK) break;
      SPMC_CUDA(cudaEventRecord(e1, s));
      SPMC_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      SPMC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; best_jt = jt; }
    }
    plan->JT = (st == SPMC_OK) ? best_jt : keep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->timing = timing;
  if (st != SPMC_OK) return st;
  SPMC_CUDA(cudaMemcpyAsync(plan->d_counters, saved, sizeof saved, cudaMemcpyHostToDevice, s));
  SPMC_CUDA(cudaStreamSynchronize(s));
  if (best_ms) *best_ms = best;
  return SPMC_OK;
}

spmc_status spmc_set_sweep(spmc_plan_t plan, int mode, long long batch) {
  if (!plan) return SPMC_ERR_INVALID;
  if (mode != SPMC_SWEEP_EVENTS && mode != SPMC_SWEEP_COHORT && mode != SPMC_SWEEP_EVENTS_ALU)
    return fail(plan, SPMC_ERR_INVALID, "spmc_set_sweep: unknown mode");
  plan->sweep_mode = mode;
  plan->ev_batch = batch > 0 ? batch : 0;
  return SPMC_OK;
}

spmc_status spmc_set_acceleration(spmc_plan_t plan, int mode) {
  if (!plan) return SPMC_ERR_INVALID;
  if (mode != SPMC_ACCEL_NONE && mode != SPMC_ACCEL_AITKEN) return fail(plan, SPMC_ERR_INVALID, "unknown acceleration");
  plan->accel = mode;
  return SPMC_OK;
}

spmc_status spmc_set_graphs(spmc_plan_t plan, int enable) {
  if (!plan) return SPMC_ERR_INVALID;
  plan->use_graphs = enable != 0;
  return SPMC_OK;
}

spmc_status spmc_set_timing(spmc_plan_t plan, int enable) {
  if (!plan) return SPMC_ERR_INVALID;
  drain_timing(plan);
  plan->timing = enable != 0;
  if (plan->timing) {
    plan->stats.sweep_ms = 0.0; plan->stats.sweep_launches = 0;
    plan->stats.walk_ms = 0.0; plan->stats.fill_ms = 0.0; plan->stats.eval_ms = 0.0; plan->stats.eval_launches = 0;
  }
  return SPMC_OK;
}

spmc_status spmc_space_nodes(spmc_plan_t plan, double* x_host) {
  if (!plan || !x_host) return SPMC_ERR_INVALID;
  std::copy(plan->xnodes.begin(), plan->xnodes.end(), x_host);
  return SPMC_OK;
}

spmc_status spmc_get_stats(spmc_plan_t plan, spmc_stats* out) {
  if (!plan || !out) return SPMC_ERR_INVALID;
  sync_counters(plan);
  plan->stats.workspace_bytes = plan->ws_bytes;
  *out = plan->stats;
  return SPMC_OK;
}

const char* spmc_last_error(spmc_plan_t plan) { return plan ? plan->err.c_str() : "null plan"; }

void spmc_destroy(spmc_plan_t plan) {
  if (!plan) return;
  drain_timing(plan);
  for (auto& ev : plan->ev_free) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  for (auto& kv : plan->allocs) cudaFree(kv.first);   // every device allocation of the plan
  plan->allocs.clear();
  delete plan;
}

}  // extern "C"
