/*
 * spmc.h -- C-ABI of the B300 implementation of the hp-version time-stepping
 * spectral Monte Carlo method for semilinear parabolic equations
 *
 *     d_t u - kappa Delta u = f(u) + f_add(x, t)   in (-1,1)^d x (0, T],
 *     u = 0 on the boundary,  u(., 0) = u0                       (Eq. mainproblem)
 *
 * solved interval by interval over an hp time partition (Eq. mesh, Eq.
 * multischeme) by the residual iteration of Section 2.4 / Algorithm 1: on
 * interval n, iteration k reconstructs the space-time spectral expansion of the
 * nodal values (Eq. u_N), estimates the error eps at every space-time node by
 * Monte Carlo sampling of the Feynman-Kac representation of the error equation
 * (Eqs. ufg_ep1, varepsilon_1) and updates u <- u + eps (Algorithm 1, Step 3).
 *
 * Conventions
 *  - All entry points return spmc_status; no C++ exception crosses the ABI.
 *    On failure, spmc_last_error(plan) returns a message (valid until the next
 *    call on that plan).
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as void*;
 *    NULL means the legacy default stream).  Calls that return host values
 *    (max |eps|, statistics) synchronise that stream.
 *  - Device buffers passed in are owned by the caller; the plan owns its
 *    workspace and frees it in spmc_destroy.  Host arrays are read during the
 *    call only.
 *  - Spatial nodes are the Jacobi-Gauss (1,1) nodes (Section 2.3), n_space per
 *    axis, linear index j = j_1 + n_space (j_2 + n_space (...)) (x_1 fastest).
 *    Nodal arrays of one interval are (M_n + 1) rows (time nodes, row 0 at
 *    t_{n-1}) of n_space^d values.
 *  - A plan is not thread-safe: one host thread at a time per plan.
 */
#ifndef SPMC_H
#define SPMC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPMC_OK = 0,
  SPMC_ERR_INVALID = 1,      /* bad argument or plan state */
  SPMC_ERR_UNSUPPORTED = 2,  /* valid request outside what this library implements */
  SPMC_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  SPMC_ERR_OOM = 4,          /* device allocation failed */
  SPMC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  SPMC_ERR_NONFINITE = 6     /* a non-finite eps was produced */
} spmc_status;

enum { SPMC_TIME_LGL = 0, SPMC_TIME_RADAU_LEFT = 1, SPMC_TIME_CHEB = 2 };   /* time nodes per interval */
enum { SPMC_BASIS_JACOBI = 0, SPMC_BASIS_CHEB = 1 };       /* spectral basis */
enum { SPMC_FP64 = 0, SPMC_MIXED = 1 };                    /* sweep arithmetic */
enum { SPMC_F_POLY3 = 0, SPMC_F_SIN = 1 };                 /* reaction f(u) */
enum { SPMC_EX_NONE = 0, SPMC_EX_SIN = 1, SPMC_EX_COSHALF = 2, SPMC_EX_POLY = 3,
       SPMC_EX_COSTHIRD = 4, SPMC_EX_SINPLUS = 5,                   /* non-zero boundary values */
       SPMC_EX_FRAC_SIN = 6, SPMC_EX_FRAC_POLY = 7 };               /* the fractional case */
enum { SPMC_BC_ZERO = 0, SPMC_BC_LIFT = 1, SPMC_BC_RAW = 2 };       /* boundary data g */
enum { SPMC_EST_RESIDUAL = 0, SPMC_EST_DIRECT = 1 };               /* estimator */
enum { SPMC_U0_NODAL = 0, SPMC_U0_PHI_COEF = 1 };

typedef struct spmc_plan_s* spmc_plan_t;

/* Geometry, discretisation and sampling of a batch of instances.
 * Section 2.1 (notation), Eq. time division (N_*), Lemma Xlocation (walk). */
typedef struct {
  int dim;                  /* d: 1, 2 or 5 (n_space <= 8 for d = 5) */
  int n_space;              /* JG(1,1) nodes = spatial modes per axis, 2..32 */
  int time_family;          /* SPMC_TIME_LGL or SPMC_TIME_RADAU_LEFT */
  int max_intervals;        /* largest interval count of any instance */
  int max_degree;           /* largest time degree M_n of any interval, 1..39 */
  long long M;              /* samples per node, >= 1 */
  int K;                    /* iterations per interval (cap when tol > 0) */
  double tol;               /* stop an interval once max|eps| < tol; <= 0: run K */
  int n_ref;                /* N_* = max(1, ceil(n_ref (t_{n,l} - t_{n-1}) / h_n)) */
  int n_sub;                /* time sub-points per full walk step, power of two <= 16 */
  double shell;             /* the walk is absorbed within this distance of the boundary;
                               0: half the distance of the outermost node, at most 2e-3
                               (a shell wider than that distance freezes those nodes) */
  int max_steps;            /* cap on quadrature terms per walk */
  double kappa;             /* diffusion coefficient (> 0) */
  unsigned long long seed;  /* Philox4x32-10 key */
  int precision;            /* SPMC_FP64 or SPMC_MIXED (FP32 sweep, FP64 elsewhere) */
  int batch;                /* number of instances, >= 1 */
  int walk_mode;            /* SPMC_WALK_BALLS (0): balls inside Omega of radius min(J, dist),
                               the residual at a Green-function point of each ball and a
                               random sub-step time; SPMC_WALK_FIXED (1): the fixed-radius
                               walk of Lemma Xlocation with the residual at the step centres
                               (Eqs. indexL, interIQ; n_sub is then 1, d <= 2, cohort sweep).
                               The second diverges at high spectral degrees.  SPMC_WALK_STABLE (2):
                               the alpha-stable walk of the fractional case (see alpha). */
  int estimator;            /* SPMC_EST_RESIDUAL (0): the residual iteration of Algorithm 1 (u <- u + eps,
                               eps the mean of Q_L of the residual, Eq. varepsilon_1);
                               SPMC_EST_DIRECT (1): the direct estimator of Eq. Phi_ast, a Picard
                               iteration (Eq. linearized_func) u <- mean of S_i, S_i = u*^{n-1}(X, t_{n-1})
                               for a walk that reaches t_{n-1} (the walk's last step moves by
                               sqrt(2 d kappa w) for the time w it took), g(X_p, t_p) for one absorbed at
                               the boundary (raw boundary data), plus the quadrature of f(u*) + f_add.
                               Its sampling error does not fall with the iterations.  Event sweep only
                               (d <= 2, walk_mode 0). */
  double alpha;             /* 0 (or 2): L = -kappa Delta.  In (0, 2), with walk_mode SPMC_WALK_STABLE and
                               d = 1: the fractional case of Section 4, Ex. 2 and 3,
                               d_t u + kappa (-Delta)^{alpha/2} u = f(u) + f_add, u = 0 outside Omega:
                               spatial nodes are the Jacobi-Gauss (alpha/2, alpha/2) nodes, the basis
                               the generalised Jacobi functions (1-x^2)^{alpha/2} P_p^{(alpha/2,alpha/2)}
                               ((-Delta)^{alpha/2} of one is Gamma(alpha+p+1)/p! P_p), and the walk the
                               alpha-stable walk: steps of time Delta, each the exit from the ball of
                               radius r = (kappa Delta Gamma(1+alpha))^{1/alpha} around the current point,
                               at distance r / sqrt(U), U ~ Beta(alpha/2, 1-alpha/2), in direction +-1;
                               the residual at the step centres (Eqs. indexL, interIQ); the cohort sweep. */
  int basis;                /* SPMC_BASIS_JACOBI (0): Jacobi-Gauss (1,1) nodes, Babuska-Shen basis, Legendre
                               in time (Section 2.3).  SPMC_BASIS_CHEB (1): the Chebyshev basis of the remark
                               on quasi-linear reconstruction after Algorithm 1, with time_family
                               SPMC_TIME_CHEB: interior Chebyshev-Gauss-Lobatto points in space, phi_p =
                               T_p - T_{p+2}, T_q in time at the CGL points; coefficients by the discrete
                               Chebyshev transform (DCT-I, through the FFT of the even extension for
                               power-of-two lengths); d <= 2, the inside-ball walk, the event sweep with
                               the FP64/FP32 evaluation (not the tensor-core one). */
} spmc_plan_desc;
enum { SPMC_WALK_BALLS = 0, SPMC_WALK_FIXED = 1, SPMC_WALK_STABLE = 2 };

/* One instance: partition, degrees, reaction, manufactured source, boundary
 * data, u0.  Eq. mainproblem; f_add makes the closed form named by ex_kind an
 * exact solution (Section 4 examples); the boundary data g is that closed
 * form's trace (zero for kinds 1-3). */
typedef struct {
  int n_intervals;          /* 1..max_intervals */
  const double* t_breaks;   /* host, n_intervals + 1 strictly increasing values */
  const int* degrees;       /* host, n_intervals time degrees M_n, 1..max_degree */
  int f_kind;               /* SPMC_F_POLY3: s (c0 + c1 u + c2 u^2 + c3 u^3); SPMC_F_SIN: s sin(u) */
  double f_coef[4];
  double f_scale;           /* s */
  int ex_kind;              /* SPMC_EX_*: e^{-beta t} prod sin(pi x_e); e^{-beta t} prod cos(pi x_e / 2);
                               (1+t+t^2) prod (1-x_e^2)(1+x_e); or no source */
  double ex_beta;
  int u0_kind;              /* SPMC_U0_NODAL: u0 holds n_space^d nodal values;
                               SPMC_U0_PHI_COEF: u0 holds n_coef^d coefficients of
                               prod phi_{p_e}(x_e), p_e < n_coef (x_1 fastest) */
  int n_coef;
  const double* u0;         /* host */
  int bc_kind;              /* SPMC_BC_ZERO: g = 0 (kinds 0-3).  SPMC_BC_LIFT: homogenisation (Section 2.3,
                               remark on non-homogeneous boundary conditions): the plan solves for
                               w = u - G, G the Gordon-Hall transfinite lifting of g from its face values,
                               with the reaction f(w + G) and the source f_add - d_t G + kappa Delta G;
                               u0 is given for u and w(., 0) = u0 - G(., 0) is formed on the device;
                               spmc_get_nodes returns w, spmc_get_solution u.  SPMC_BC_RAW: g enters where
                               the walk is absorbed (SPMC_EST_DIRECT only).  Kinds 4, 5 need LIFT or RAW;
                               d <= 2 and the event sweep. */
} spmc_problem;

typedef struct {
  long long node_samples;   /* walks run */
  long long points;         /* residual evaluations */
  long long capped;         /* walks cut at max_steps */
  int iterations_run;       /* iterations of the last spmc_solve / spmc_iterate */
  double last_max_eps;
  long long sweep_launches; /* sweep kernel launches timed (spmc_set_timing) */
  double sweep_ms;          /* their summed duration, from CUDA events on the caller's stream */
  double walk_ms;           /* event sweep: the counting walk pass and the scan (part of sweep_ms) */
  double eval_ms;           /* event sweep: the per-slice evaluation launches (part of sweep_ms) */
  long long eval_launches;
  double fill_ms;           /* event sweep: the placing walk pass (part of sweep_ms) */
  long long workspace_bytes;/* device memory the plan holds (its own allocations) */
  long long graph_launches; /* intervals spmc_solve ran as one captured CUDA graph */
} spmc_stats;

/* Validate desc, build the node tables and allocate the workspace.
 * Errors: SPMC_ERR_INVALID (out-of-range field), SPMC_ERR_UNSUPPORTED (dim or
 * size this library does not implement), SPMC_ERR_OOM, SPMC_ERR_CUDA.
 * *out is NULL on failure. */
spmc_status spmc_plan(const spmc_plan_desc* desc, spmc_plan_t* out);

/* Set instance `instance` (0..batch-1).  Every instance must be set before
 * spmc_solve / spmc_begin_interval.  Copies the host arrays. */
spmc_status spmc_set_problem(spmc_plan_t plan, int instance, const spmc_problem* prob);

/* Number of doubles one instance's full solution occupies (sum over its
 * intervals of (M_n+1) n_space^d), and its offset in spmc_solve's output. */
spmc_status spmc_solution_layout(spmc_plan_t plan, int instance, long long* offset, long long* count);

/* Algorithm 1 for every instance: all intervals, K iterations each (or until
 * max|eps| < tol), hand-off of u*(., t_n) between intervals (Step 4).
 * u_nodes: caller-owned device buffer of spmc_solution_layout's total size;
 * receives every interval's nodal values.  With a fixed K, the event sweep,
 * timing off and graphs on (the default, spmc_set_graphs), every interval after
 * the first -- its hand-off and K iterations -- is captured on the caller's
 * stream as one CUDA graph and launched at once; the stream is synchronised once
 * per interval.  Results are the same bit for bit either way. */
spmc_status spmc_solve(spmc_plan_t plan, void* cuda_stream, double* u_nodes);

/* Stepwise driver.  spmc_begin_interval sets the first iterate of interval
 * `interval` (0-based) of every instance that has it: row 0 from u0 (interval
 * 0) or from the previous interval's expansion at its end, all rows equal to
 * row 0 (Remark 2.1).  spmc_iterate then runs n_iter iterations (iteration
 * numbers continue from the previous call on that interval) and returns the
 * largest |eps| of the last one over all instances.  The iterations are
 * enqueued back to back and the stream is synchronised once, at the end (the
 * plan's very first event-sweep batch also synchronises once to size the event
 * buffer).  If a batch outgrows the event buffer, the device skips the rest of
 * the sequence and the call grows the buffer and runs the skipped iterations
 * again, so results never depend on it. */
spmc_status spmc_begin_interval(spmc_plan_t plan, void* cuda_stream, int interval);
spmc_status spmc_iterate(spmc_plan_t plan, void* cuda_stream, int interval, int n_iter, double* max_eps_host);

/* Copy the current nodal values of (instance, interval) into dst (device
 * pointer, (M_n+1) n_space^d doubles). */
spmc_status spmc_get_nodes(spmc_plan_t plan, void* cuda_stream, int instance, int interval, double* dst);

/* The solution u at the nodes of (instance, interval) into dst (device
 * pointer, (M_n+1) n_space^d doubles): the nodal values plus, for lifted
 * boundary data (SPMC_BC_LIFT), the lifting G(x_j, t_{n,l}) (computed on the
 * device); otherwise the nodal values themselves. */
spmc_status spmc_get_solution(spmc_plan_t plan, void* cuda_stream, int instance, int interval, double* dst);

/* Overwrite the nodal values of (instance, interval) with src ((M_n+1)
 * n_space^d doubles, host or device pointer): checkpoint restore, or a chosen
 * iterate for checking.  A later spmc_iterate on that interval continues from it. */
spmc_status spmc_set_nodes(spmc_plan_t plan, void* cuda_stream, int instance, int interval, const double* src);

/* One residual iteration on `interval` (like spmc_iterate with n_iter = 1 with
 * the cohort sweep, whose results it reproduces bit for bit) that allocates
 * nothing.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory at the point of the call, e.g.
 * code running between the set-up of a real-time loop and its teardown, or a
 * host thread inside a region where cudaMalloc would synchronise the device or
 * is forbidden by the surrounding allocator policy.  The sweep kernel's scratch
 * (walk state, work counter, per-node chunk sums) lives in a file-scope device
 * array of SPMC_STATIC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until exit; nodal values, coefficients and slices stay in the plan,
 * which must already be built (spmc_begin_interval on it has run).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) for the current device; make that first call before
 *    any stream capture.
 *  - Every call shares the array and leaves its last contents there; the call
 *    clears what must start at zero.  Calls that overlap on the GPU (other
 *    streams, other plans, other host threads) race on it: serialise them.
 *  - A problem whose chunk sums and minimal walk state do not fit in the array
 *    is rejected with SPMC_ERR_UNSUPPORTED and a message naming the limit.
 * max_eps_host receives the largest |eps| (the stream is synchronised); the
 * statistics (points, capped, iterations_run, last_max_eps) are updated as by
 * spmc_iterate. */
#define SPMC_STATIC_SCRATCH_BYTES (16u << 20)
spmc_status spmc_iterate_static(spmc_plan_t plan, void* cuda_stream, int interval, double* max_eps_host);

/* Node-sharded iterations, for running one batch of instances on several GPUs
 * (the sampled nodes of a sweep are independent; Algorithm 1, Step 2 parallel
 * over nodes).  Every rank holds the same plan and nodal values and
 * reconstructs redundantly; each samples its share of the round's
 * (time node, spatial node) pairs and the eps of all pairs are exchanged once
 * per iteration.
 *  - spmc_round_nodes: the number of pairs of interval `interval`: n_pairs =
 *    (sum over its instances of M_n) x n_space^d; pair i = ti n_space^d + j, ti
 *    running over the instances (in order) and their time nodes l = 1..M_n.
 *  - spmc_iterate_shard: the sweep of the next iteration for the pairs
 *    [n rank / world, n (rank + 1) / world) only; writes their eps to
 *    eps_pairs[i] (device, n_pairs doubles; other entries untouched) and does
 *    not change the nodal values.  Event sweep only (d <= 2, inside-ball walk):
 *    SPMC_ERR_UNSUPPORTED otherwise.  Per-pair eps are exact sums, so the
 *    shards' eps equal those of an unsharded iteration bit for bit.
 *  - spmc_apply_eps: u += eps for every pair of the interval (eps_pairs on the
 *    device, e.g. after an all-reduce of the ranks' zero-filled buffers) and
 *    advance the iteration count; returns the largest |eps|.
 * The stream is synchronised by each call. */
spmc_status spmc_round_nodes(spmc_plan_t plan, int interval, long long* n_pairs);
spmc_status spmc_iterate_shard(spmc_plan_t plan, void* cuda_stream, int interval, int rank, int world,
                               double* eps_pairs);
spmc_status spmc_apply_eps(spmc_plan_t plan, void* cuda_stream, int interval, const double* eps_pairs,
                           double* max_eps_host);

/* Reverse-mode gradient of L(u(T)) for every instance: given dL/du at the
 * spatial nodes at t = T (device, batch x n_space^d doubles), returns
 * dL/d(f_scale) (device, batch doubles) and dL/d(u0 coefficients) (device,
 * batch x n_coef^d doubles; instances set with SPMC_U0_PHI_COEF).  The walks are
 * the forward solve's (common random numbers); iterations are recomputed from
 * per-interval checkpoints.  Requires a prior spmc_solve on the same plan. */
spmc_status spmc_grad(spmc_plan_t plan, void* cuda_stream, const double* dloss_du_T,
                      double* grad_f_scale, double* grad_u0_coef);

/* Forward-sweep strategy for d <= 2 (d = 5, spmc_grad and spmc_iterate_static
 * always use the cohort kernel):
 *   SPMC_SWEEP_EVENTS (default): per batch of `batch` samples, the walks run
 *     once and append their evaluation events (Green point, weight, slice and
 *     node); a counting sort groups them by (time slice, node); one block per
 *     slice then evaluates all of them against that slice.  With d = 2 and
 *     SPMC_MIXED the evaluation is a matrix product on the tensor cores
 *     (tcgen05, TF32 with a 3-term split, FP32 accumulation); otherwise it runs
 *     on the FP32 / FP64 pipes.  Per-event terms are summed in FP64.  Device
 *     memory: an event buffer of 16 (FP32) or 32 (FP64) bytes per event of a
 *     batch, sized from the largest batch seen (plus a quarter), allocated on
 *     first use and kept.  batch <= 0 picks about 2^25 walks per batch.
 *   SPMC_SWEEP_EVENTS_ALU: the same, with the evaluation always on the FP32 /
 *     FP64 pipes.
 *   SPMC_SWEEP_COHORT: the persistent cohort kernel; a walk's terms are summed
 *     in the sweep precision, then in FP64 per chunk.
 * The two give the same walks and the same points; only summation order and,
 * in SPMC_MIXED, the per-walk FP32 partial sums differ.  Both are bitwise
 * reproducible: the event sweep adds each term to its node as a fixed-point
 * integer (the term rounded once to a multiple of 2^-80), so its per-node sums
 * are exact and do not depend on the order of the atomics, and are rounded to
 * FP64 once; the cohort kernel sums each node's walks in sample order.  The
 * event sweep needs M x max_steps < 2^32 (SPMC_ERR_UNSUPPORTED otherwise).
 * Returns SPMC_ERR_INVALID for an unknown mode. */
#define SPMC_SWEEP_EVENTS 0
#define SPMC_SWEEP_COHORT 1
#define SPMC_SWEEP_EVENTS_ALU 2
spmc_status spmc_set_sweep(spmc_plan_t plan, int mode, long long batch);

/* Acceleration of the residual iteration (the Remark after Algorithm 1 on
 * Aitken-weighted Picard iteration; the paper gives no formula).
 * SPMC_ACCEL_AITKEN: Aitken's dynamic relaxation per instance,
 *   u_{k+1} = u_k + omega_k eps_k,  omega_1 = 1 on each interval,
 *   omega_k = -omega_{k-1} <eps_{k-1}, eps_k - eps_{k-1}> / |eps_k - eps_{k-1}|^2,
 * kept in [1/2, 2] (once eps is Monte Carlo noise, successive residuals are
 * uncorrelated and the unbounded factor would halve at each step).  The sums
 * run in a fixed order.  Not combined with the sharded iteration.
 * SPMC_ACCEL_NONE (default): u_{k+1} = u_k + eps_k. */
enum { SPMC_ACCEL_NONE = 0, SPMC_ACCEL_AITKEN = 1 };
spmc_status spmc_set_acceleration(spmc_plan_t plan, int mode);

/* Enable (1, the default) or disable (0) spmc_solve's capture of each interval
 * as a CUDA graph.  The caller's stream must not be capturing already. */
spmc_status spmc_set_graphs(spmc_plan_t plan, int enable);

/* Enable (1) or disable (0) CUDA-event timing of every sweep kernel launch; the
 * totals accumulate in spmc_stats.sweep_ms / sweep_launches (reset on enable). */
spmc_status spmc_set_timing(spmc_plan_t plan, int enable);

/* Autotuner: times the forward sweep of one iteration of `interval` (which must
 * have been started with spmc_begin_interval) for each candidate setting, keeps
 * the fastest for the plan and returns its time in *best_ms (may be NULL).  The
 * setting is the batch size (2^23 .. 2^26 walks per batch) of the event sweep,
 * or the cohort width (spatial nodes per cohort) of the cohort kernel.  The
 * nodal values and the points / capped counters are left unchanged: the
 * candidates run the reconstruction, slices and sweep but not the update.
 * Results of later iterations do not depend on the choice (the cohort kernel
 * sums per node in sample order whatever the width; the event sweep's per-node
 * sums are exact whatever the batch). */
spmc_status spmc_autotune(spmc_plan_t plan, void* cuda_stream, int interval, double* best_ms);

/* The n_space JG(1,1) node coordinates of one axis, ascending (host array). */
spmc_status spmc_space_nodes(spmc_plan_t plan, double* x_host);

spmc_status spmc_get_stats(spmc_plan_t plan, spmc_stats* out);
const char* spmc_last_error(spmc_plan_t plan);
void spmc_destroy(spmc_plan_t plan);

/* Library version string. */
const char* spmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPMC_H */
