"""Benchmark: node-samples/s of the hp-version time-stepping spectral Monte Carlo
hot path on the 2-D long-time workload (24 x 24 JG x 16 LGL nodes per interval,
T = 20 in 20 intervals of h = 1, M = 65536 samples per node, K = 8 iterations),
batched mixed precision (FP32 sweep; FP64 reconstruction, update and sums).

One step = one interval of the hp solve: the hand-off from the previous interval
(Algorithm 1, Step 4) and K residual iterations (Steps 1-3); consecutive steps
continue the solve interval after interval.  Inputs are resident in HBM; L2 is
flushed between steps outside the timed events.  The JSON
line also carries the FP64 path's throughput on a bounded run, the roofline
figures of the sweep's kernels (count walk, fill walk, evaluation; the
dominant one as `roofline`), an end-to-end figure through the C-ABI with host
buffers, and the CPU oracle's throughput on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--intervals", type=int, default=20, help="intervals of the workload (20 = full)")
    ap.add_argument("--M", type=int, default=65536)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, e2e and CPU legs")
    ap.add_argument("--case", default=None, choices=["iterate1", "iterate1_5d", "iterate1_frac", "iterate1_cheb"],
                    help="profiling case: build the plan and run one iteration of the first interval, untimed "
                         "(iterate1_5d: the 5-D workload; iterate1_frac: the fractional Allen-Cahn problem, "
                         "alpha = 0.4, h = 0.5; iterate1_cheb: the 2-D workload in the Chebyshev basis; all at "
                         "--M samples)")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([v.strip() for v in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --------------------------------------------------------------------------- helpers
def workload(args, rank=0):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=args.M, n_intervals=args.intervals)
    wl.seed = rank            # independent replica per rank (weak scaling)
    return wl


def max_over_ranks(ms, device):
    """The slowest rank's step time (ms): every rank's replica must finish
    before the job's step is done.  One process per GPU; a no-op without a
    process group of more than one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(units_per_rank_step, world, ms):
    """Whole-job units per second: every rank processes its own replica of the
    workload (weak scaling), so the job does world x the per-rank units in the
    slowest rank's time."""
    return units_per_rank_step * world / (ms / 1e3)


def node_samples_per_solve(wl):
    S = wl.n_space ** wl.dim
    tot = 0
    for inst in wl.instances:
        for Mt in inst.degrees:
            tot += int(Mt) * S * wl.M * wl.K
    return tot


def node_samples_per_interval(wl, r):
    S = wl.n_space ** wl.dim
    return sum(int(i.degrees[r]) * S * wl.M * wl.K for i in wl.instances if r < len(i.degrees))


def flops_per_point(dim, n):
    """Algorithmic FP32 flops of one residual evaluation (d = 2): three
    contractions of the n x n slice with the y-basis (3 n^2 FMA), the x-side
    accumulation (4 n FMA) and the two basis recurrences (about 5 n flops each)."""
    if dim == 2:
        return 2 * 3 * n * n + 2 * 4 * n + 2 * 5 * n
    return 2 * 3 * n + 10 * n


def walk_ops_per_event(dim, fill):
    """Algorithmic 32-bit operations of one walk step that ends in an evaluation
    event: Philox4x32-10 blocks (10 rounds x (2 32x32->64 multiplies = 4 ops,
    4 xors) + 9 key bumps x 2 adds = 98 ops) -- one per step (direction,
    sub-point and roulette words share it), a second for the Green radius words
    when the event is written (fill pass) -- plus the step's geometry
    (distance, ball, weight, sub-point, the sin/cos pairs and the Green radius,
    about 60 FP32 ops)."""
    blocks = 2 if fill else 1
    return 98 * blocks + 60


def sweep_roofline(wl, prec, points, st, peaks, steps, step_ms):
    """Per-kernel roofline figures of the event sweep and the dominant one."""
    from paper_2608_22190_b300 import _lib as L
    n = wl.n_space
    nmax = 8 if n <= 8 else (16 if n <= 16 else (24 if n <= 24 else 32))
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * sm_max * 1e6 / 1e12          # lane-ops/s (one FP32 or INT32 lane op per cycle)
    tf32_ratio = 1.1 / 2.25                               # nominal dense TF32 / BF16 (recipe table)
    # measured sustained cuBLAS BF16 rate; without the measurement file, the
    # recipe's fallback (1.4 PFLOP/s sustained on an earlier B300)
    bf16_sus = peaks.get("bf16_tflops_sustained", 1400.0)
    bf16_src = "bf16_tflops_sustained (MEASURED_PEAKS.json, of measured)" if "bf16_tflops_sustained" in peaks \
        else "fallback 1400 TFLOP/s sustained BF16 (no measured peaks file, of fallback)"
    kern = {}
    t_count, t_fill, t_eval = st["walk_ms"] / 1e3, st["fill_ms"] / 1e3, st["eval_ms"] / 1e3
    per_ev_c, per_ev_f = walk_ops_per_event(wl.dim, False), walk_ops_per_event(wl.dim, True)
    if t_count > 0:
        a = points * per_ev_c / t_count / 1e12
        kern["walk_count"] = {"bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s", "frac": a / alu_peak,
                              "ms": t_count * 1e3 / steps, "ops_per_event": per_ev_c}
    if t_fill > 0:
        a = points * per_ev_f / t_fill / 1e12
        kern["walk_fill"] = {"bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s", "frac": a / alu_peak,
                             "ms": t_fill * 1e3 / steps, "ops_per_event": per_ev_f}
    if t_eval > 0:
        if prec == L.MIXED and wl.dim == 2:
            fpe = 2 * nmax * 4 * nmax                     # one (1 x K)(K x 4 NMAX) product per event
            peak = bf16_sus * tf32_ratio
            a = points * fpe / t_eval / 1e12
            kern["eval_tc"] = {"bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                               "ms": t_eval * 1e3 / steps, "flops_per_event": fpe,
                               "executed_tensor_tflops": 3 * a,
                               "peak_source": bf16_src + " x nominal TF32/BF16 1.1/2.25"}
        else:
            fpe = flops_per_point(wl.dim, n)
            peak = 1.25 if prec == L.FP64 else alu_peak * 2
            a = points * fpe / t_eval / 1e12
            kern["eval_alu"] = {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                                "ms": t_eval * 1e3 / steps, "flops_per_event": fpe,
                                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)" if prec == L.FP64
                                else "148 SMs x 128 FP32 lanes x 2 x sm_max_mhz"}
    # DRAM bytes per event from one ncu capture of each kernel as it is now
    # (profiles/walk_events_w2_fullset.md, profiles/eval_tc_w2_fullset.md: M = 1024,
    # 1.0212e8 events), scaled by the events of one launch; traffic grows with the events
    per_event_bytes = {"walk_fill": (0.605840 + 2.131090) * 1e9 / 1.02118e8,
                       "eval_tc": (1.664608 + 0.005134) * 1e9 / 1.02118e8}
    # the counting pass reads its tables and keeps the counts in L2: its DRAM traffic
    # does not grow with the events (0.0118 GB read, nothing written, per launch)
    per_launch_bytes = {"walk_count": 0.011807e9}
    launches = max(1, st["eval_launches"])
    for k, v in kern.items():
        v["traffic"] = None
        if wl.dim == 2 and k in per_event_bytes:
            v["traffic"] = per_event_bytes[k] * points / launches
        elif wl.dim == 2 and k in per_launch_bytes:
            v["traffic"] = per_launch_bytes[k]
    name = max(kern, key=lambda k: kern[k]["ms"]) if kern else None
    roof = dict(kern[name]) if name else {}
    if name:
        roof["kernel"] = name
        roof["share_of_step"] = roof["ms"] / step_ms
    return roof, kern


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def cpu_baseline(wl, budget_s=12.0):
    """The oracle, as it stands, on a bounded sample of the workload: eps at a set
    of nodes of the first iteration of the first interval (independent nodes run
    on separate host threads; each node is the oracle's serial sum)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as O
    from paper_2608_22190_b300 import workloads as W
    inst = wl.instances[0]
    cores = os.cpu_count() or 1
    spec = O.Spec(dim=wl.dim, n_space=wl.n_space, time_family=wl.time_family, n_ref=wl.n_ref, M=16,
                  kappa=wl.kappa, seed=wl.seed, f_kind=inst.f_kind, f_coef=tuple(inst.f_coef),
                  f_scale=inst.f_scale, ex_kind=inst.ex_kind, ex_beta=inst.ex_beta, n_sub=wl.n_sub,
                  shell=wl.shell, max_steps=wl.max_steps, n_threads=1)
    u0 = W.u0_nodal(inst, O.space_nodes_grid(spec))
    Mt = int(inst.degrees[0])
    h = float(inst.t_breaks[1] - inst.t_breaks[0])
    cu, ct = O.reconstruct(spec, Mt, h, np.tile(u0, (Mt + 1, 1)))
    S = wl.n_space ** wl.dim
    rng = np.random.default_rng(0)

    def run(n_nodes, m):
        sp = O.Spec(**{**spec.__dict__, "M": m})
        nodes = [(int(rng.integers(0, S)), int(rng.integers(1, Mt + 1))) for _ in range(n_nodes)]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda jl: O.node_eps(sp, Mt, 0.0, h, cu, ct, jl[0], jl[1]), nodes))
        return time.perf_counter() - t0, n_nodes * m

    dt, ns = run(cores, 8)
    scale = max(1.0, budget_s / max(dt, 1e-3))
    m = int(min(4096, max(8, 8 * scale)))
    dt, ns = run(cores, m)
    return {"value": ns / dt, "unit": "node-samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} nodes x {m} samples, iteration 1 of interval 1 of the 2-D long-time workload "
                      f"({dt:.1f} s)"}


def flush_l2(buf):
    buf.fill_(1.0)


# --------------------------------------------------------------------------- arms
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300.api import Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    prec = L.MIXED if args.precision == "mixed" else L.FP64
    wl = workload(args, rank)
    plan = Plan.from_workload(wl, precision=prec)
    out = torch.empty(plan.total_size(), dtype=torch.float64, device="cuda")
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    n_int = max(len(i.degrees) for i in wl.instances)
    state = {"r": 0}
    plan.begin_interval(0)
    tune_ms = plan.autotune(0)

    def step():
        r = state["r"] % n_int
        plan.begin_interval(r)
        plan.iterate(r, wl.K)
        state["r"] += 1
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.set_timing(True)
    base_points = plan.stats()["points"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    done = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush_l2(l2)
            evs[i][0].record(stream)
            done.append(step())
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    st = plan.stats()
    plan.set_timing(False)
    ms = max_over_ranks(ms, "cuda")
    per_step = sum(node_samples_per_interval(wl, r) for r in done) / len(done)
    value = job_throughput(per_step, world, ms)

    # roofline of the dominant kernel of the sweep (by device time in the timed
    # region; every launch bracketed by CUDA events on the launching stream)
    points = st["points"] - base_points
    peaks = measured_peaks()
    roof, kernels = sweep_roofline(wl, prec, points, st, peaks, args.steps, ms)
    batches = st["eval_launches"]
    # per step: hand-off (or first iterate); per iteration: counter snapshot,
    # reconstruction, slices, update; per batch: count walk, three scan kernels,
    # fill walk, evaluation
    launches = args.steps * (1 + 4 * wl.K) + 6 * batches

    line = {"metric": "node-samples/sec & time to L-inf err 1e-6: batched mixed vs plain FP64, 1 B300",
            "value": value, "unit": "node-samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == L.MIXED else "f64",
            "data": "synthetic (manufactured solution u = e^{-0.1 t} sin(pi x) sin(pi y))",
            "config": {"workload": "w2-2d-long-time: 24x24 JG x 16 LGL, T=20 in 20 intervals, M=65536, K=8"
                       if args.intervals == 20 else f"w2-2d-long-time ({args.intervals} intervals)",
                       "precision": args.precision, "n_ref": wl.n_ref, "n_sub": wl.n_sub,
                       "l2": "flushed between steps (256 MB write, outside the timed events)",
                       "node_samples_per_step": per_step,
                       "step": "one interval of the hp solve: hand-off + K = 8 iterations",
                       "intervals_timed": done},
            "clocks": clk.summary(), "gpu_launches": launches, "roofline": roof, "kernels": kernels,
            "wall_s": t_wall, "autotune": {"sweep_ms": tune_ms}}

    if rank == 0 and not args.no_extras:
        line["e2e"] = e2e_leg(args, wl, prec)
        line["fp64_path"] = fp64_leg(args)
        line["fp64_path"]["ratio_mixed_over_fp64"] = value / line["fp64_path"]["value"]
        line["time_to_1e-6"] = time_to_tol_legs(args)
        line["batch_w3"] = batch_leg(args)
        line["w4_5d"] = w4_leg(args, peaks)
        line["w5_adjoint"] = w5_leg(args)
        line["boundary"] = boundary_leg(args)
        line["fractional"] = fractional_leg(args)
        line["chebyshev"] = chebyshev_leg(args)
        line["cpu_baseline"] = cpu_baseline(wl)
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def e2e_leg(args, wl, prec):
    """Same metric through the C-ABI with HOST buffers: every step uploads the
    instance (initial values, partition, parameters) from pinned host memory,
    runs one interval (hand-off + K iterations) and reads that interval's nodal
    values back into pinned host memory."""
    import numpy as np
    import torch
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    plan = Plan.from_workload(wl, precision=prec)
    inst = wl.instances[0]
    grid = plan.node_grid()
    u0 = torch.from_numpy(W.u0_nodal(inst, grid)).pin_memory()
    Mt = int(inst.degrees[0])
    host_out = torch.empty((Mt + 1) * plan.S, dtype=torch.float64).pin_memory()
    steps = max(1, min(args.steps, 2))

    def step(r):
        plan.set_problem(0, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, inst.f_scale, inst.ex_kind,
                         inst.ex_beta, u0.numpy())
        plan.begin_interval(r)
        plan.iterate(r, wl.K)
        plan.get_nodes_into(0, r, host_out)
        torch.cuda.current_stream().synchronize()

    step(0)
    t0 = time.perf_counter()
    for i in range(steps):
        step(0)
    dt = (time.perf_counter() - t0) / steps
    plan.close()
    return {"value": node_samples_per_interval(wl, 0) / dt, "unit": "node-samples/s",
            "h2d_bytes_per_step": int(u0.numel() * 8 + (len(inst.t_breaks) + len(inst.degrees)) * 8 + 96),
            "d2h_bytes_per_step": int(host_out.numel() * 8), "ms_per_step": dt * 1e3}


def fp64_leg(args):
    """The plain FP64 path on the headline's workload and M (2-D long-time, 24 x 24
    x 16, M = 65536), L2 flushed before the timed region.  One step here is one
    iteration of the first interval: a full interval of eight FP64 iterations
    takes several minutes on B300, whose FP64 pipe is 1/64 of its FP32 rate.
    Node-samples/s is per node-sample, so it compares with the headline."""
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    wl = W.w2(M=args.M, n_intervals=1, K=1)
    plan = Plan.from_workload(wl, precision=L.FP64)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    plan.begin_interval(0)
    flush_l2(l2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plan.iterate(0, 1)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    plan.close()
    ns = node_samples_per_interval(wl, 0)
    return {"value": ns / (ms / 1e3), "unit": "node-samples/s", "ms": ms,
            "config": {"workload": f"w2-2d-long-time: 24x24 JG x 16 LGL, h=1, M={args.M}",
                       "step": "one FP64 iteration of interval 1", "l2": "flushed before the timed region"}}


def hp_time_to_tol(wl, prec, tol, kmax, accel="none", estimator=0, sweep=None):
    """Time until every node of every interval is within tol of the closed form:
    the hp solve interval by interval (hand-off, then iterations until the
    interval's L-inf error <= tol, at most kmax).  GPU time of the hand-offs and
    iterations (CUDA events around each call); the error of the solution u (the
    nodal values, plus the lifting for lifted boundary data) is read between
    calls, outside the events."""
    import numpy as np
    import torch
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    inst = wl.instances[0]
    plan = Plan.from_workload(wl, precision=prec, estimator=estimator)
    plan.set_acceleration(accel)
    if sweep:
        plan.set_sweep(sweep)
    grid = plan.node_grid()
    ms_total, iters, errs = 0.0, [], []

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    for r in range(len(inst.degrees)):
        ex = W.exact_block(wl, inst, grid, r)
        ms_total += timed(lambda: plan.begin_interval(r))
        err, k = float("inf"), 0
        while k < kmax and err > tol:
            ms_total += timed(lambda: plan.iterate(r, 1))
            k += 1
            err = float(np.abs(plan.get_solution(0, r).cpu().numpy() - ex).max())
        iters.append(k)
        errs.append(err)
    plan.close()
    return {"reached": bool(max(errs) <= tol), "ms": ms_total, "linf": max(errs), "iterations": iters,
            "linf_by_interval": errs, "M": wl.M, "n_ref": wl.n_ref, "k_max": kmax}


def time_to_tol_legs(args, tol=1e-6):
    """Time to L-inf error 1e-6 against the closed form.
      w2_full_mixed / w2_full_mixed_M2048 / w2_full_fp64: the 2-D long-time
        workload, all 20 intervals; mixed at the headline's M = 65536 and at
        M = 2048, plain FP64 at M = 2048 (the FP64 pipe would take about an hour
        at 65536), so mixed and FP64 also compare at equal M;
      w2_full_mixed_M512 / _M1024 / _M4096: mixed at other sample counts (up
        to 50 iterations per interval), to find the fastest way to the tolerance;
      w1_mixed / w1_fp64: the 1-D single-interval workload at its full size
        (M = 4096), with the L-inf distance of every iterate from the FP64
        oracle's iterate on the same streams (computed on the host cores
        meanwhile); w1_mixed_aitken / w1_fp64_aitken: the same with Aitken's
        relaxation of the update."""
    import os
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    from oracle import oracle as O
    out = {}
    kmax1 = 12
    # the oracle's iterates of the 1-D workload, on the host cores while the GPU runs
    wl1 = W.w1()
    inst1 = wl1.instances[0]
    spec1 = O.Spec(dim=1, n_space=wl1.n_space, time_family=wl1.time_family, n_ref=wl1.n_ref, M=wl1.M,
                   kappa=wl1.kappa, seed=wl1.seed, f_kind=inst1.f_kind, f_coef=tuple(inst1.f_coef),
                   f_scale=inst1.f_scale, ex_kind=inst1.ex_kind, ex_beta=inst1.ex_beta, n_sub=wl1.n_sub,
                   shell=wl1.shell, max_steps=wl1.max_steps, n_threads=os.cpu_count() or 1)
    Mt1 = int(inst1.degrees[0])

    def oracle_iterates():
        U = np.tile(W.u0_nodal(inst1, O.space_nodes_grid(spec1)), (Mt1 + 1, 1)).copy()
        res = []
        for k in range(kmax1):
            O.iterate(spec1, 0, inst1.t_breaks[0], inst1.t_breaks[1], Mt1, U, k + 1, 1)
            res.append(U.copy())
        return res

    pool = ThreadPoolExecutor(1)
    fut = pool.submit(oracle_iterates)
    gpu_iterates = {}
    for name, prec, accel in (("w1_mixed", L.MIXED, "none"), ("w1_fp64", L.FP64, "none"),
                              ("w1_mixed_aitken", L.MIXED, "aitken"), ("w1_fp64_aitken", L.FP64, "aitken")):
        wl = W.w1()
        plan = Plan.from_workload(wl, precision=prec)
        plan.set_acceleration(accel)
        ex = W.exact_block(wl, wl.instances[0], plan.node_grid(), 0)
        plan.begin_interval(0)
        ms_total, errs, reached, its = 0.0, [], None, []
        for k in range(kmax1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.iterate(0, 1)
            b.record()
            torch.cuda.synchronize()
            ms_total += a.elapsed_time(b)
            U = plan.get_nodes(0, 0).cpu().numpy()
            its.append(U)
            errs.append(float(np.abs(U - ex).max()))
            if reached is None and errs[-1] <= tol:
                reached = {"iterations": k + 1, "ms": ms_total}
        gpu_iterates[name] = its
        out[name] = {"reached": reached, "linf_by_iteration": errs, "ms_per_iteration": ms_total / kmax1,
                     "n_ref": wl.n_ref, "M": wl.M}
        plan.close()
    out["w2_full_mixed"] = hp_time_to_tol(W.w2(M=args.M), L.MIXED, tol, 12)
    out["w2_full_mixed_M2048"] = hp_time_to_tol(W.w2(M=2048), L.MIXED, tol, 16)
    for m in (512, 1024, 4096):   # the samples per iteration that reach the tolerance fastest
        out[f"w2_full_mixed_M{m}"] = hp_time_to_tol(W.w2(M=m), L.MIXED, tol, 50)
    out["w2_full_mixed_M2048_aitken"] = hp_time_to_tol(W.w2(M=2048), L.MIXED, tol, 16, accel="aitken")
    out["w2_full_fp64"] = hp_time_to_tol(W.w2(M=2048), L.FP64, tol, 16)
    ref = fut.result()
    pool.shutdown()
    for name in ("w1_mixed", "w1_fp64"):
        out[name]["linf_vs_oracle_by_iteration"] = [float(np.abs(g - r).max())
                                                     for g, r in zip(gpu_iterates[name], ref)]
    fp = out["w2_full_fp64"]
    for name in ("w2_full_mixed", "w2_full_mixed_M2048", "w2_full_mixed_M2048_aitken", "w2_full_mixed_M512",
                 "w2_full_mixed_M1024", "w2_full_mixed_M4096"):
        if out[name]["reached"] and fp["reached"]:
            out[name]["speedup_over_fp64_M2048"] = fp["ms"] / out[name]["ms"]
    return out


def batch_leg(args):
    """The batched initial-singularity workload at its full size: 256 uneven
    instances (8-16 geometric intervals, degrees 4 + 2k, reaction scales in
    [0.5, 2]) in one plan, M = 32768, K = 8, mixed; the first round of intervals
    (every instance's interval 1, degree 4) in node-samples/s."""
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    wl = W.w3()
    plan = Plan.from_workload(wl, precision=L.MIXED)
    ns, ms = 0, 0.0
    for r in range(1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.begin_interval(r)
        plan.iterate(r, wl.K)
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        ns += sum(int(i.degrees[r]) * wl.n_space * wl.M * wl.K for i in wl.instances if r < len(i.degrees))
    plan.close()
    return {"value": ns / (ms / 1e3), "unit": "node-samples/s", "instances": len(wl.instances), "M": wl.M,
            "sample": "interval 1 of all 256 instances (full workload size), K = 8", "ms": ms}


def w4_leg(args, peaks, tol=1e-6):
    """The 5-D workload (8^5 JG nodes x 8 LGL, T = 0.5 in one interval, mixed:
    FP32 walks, tensor-core evaluation).  At M = 1024: iterations until the
    L-inf error against the closed form is <= tol (at most 12), GPU time of the
    iterations.  Then one iteration at the full M = 16384 for the throughput
    (node-samples/s) and the tensor-core roofline of the evaluation kernel: 4
    tensors x 2 x 64 x 512 = 262144 algorithmic flops per evaluation event
    (stage 1 of the sum-factorised contraction; the split executes 3x that)."""
    import numpy as np
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    out = {}
    wl = W.w4(M=1024, K=12)
    plan = Plan.from_workload(wl, precision=L.MIXED)
    ex = W.exact_block(wl, wl.instances[0], plan.node_grid(), 0)
    plan.begin_interval(0)
    ms_total, errs = 0.0, []
    while len(errs) < 12 and (not errs or errs[-1] > tol):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.iterate(0, 1)
        b.record()
        torch.cuda.synchronize()
        ms_total += a.elapsed_time(b)
        errs.append(float(np.abs(plan.get_nodes(0, 0).cpu().numpy() - ex).max()))
    plan.close()
    out["time_to_1e-6"] = {"reached": errs[-1] <= tol, "ms": ms_total, "iterations": len(errs),
                           "linf_by_iteration": errs, "M": 1024}
    wl = W.w4(M=16384, K=1)
    plan = Plan.from_workload(wl, precision=L.MIXED)
    plan.begin_interval(0)
    plan.set_timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plan.iterate(0, 1)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st = plan.stats()
    plan.close()
    ns = node_samples_per_interval(wl, 0)
    fpe = 4 * 2 * 64 * 512
    bf16_sus = peaks.get("bf16_tflops_sustained", 1400.0)
    peak = bf16_sus * 1.1 / 2.25
    ach = st["points"] * fpe / (st["eval_ms"] / 1e3) / 1e12 if st["eval_ms"] > 0 else None
    out["full_M"] = {"value": ns / (ms / 1e3), "unit": "node-samples/s", "ms_per_iteration": ms, "M": wl.M,
                     "events": st["points"], "eval_ms": st["eval_ms"], "fill_ms": st["fill_ms"],
                     "count_ms": st["walk_ms"],
                     "roofline_eval5_tc": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                           "frac": ach / peak if ach else None, "flops_per_event": fpe,
                                           "peak_source": ("bf16_tflops_sustained (of measured)" if
                                                           "bf16_tflops_sustained" in peaks else
                                                           "fallback 1400 TFLOP/s sustained BF16 (of fallback)")
                                           + " x nominal TF32/BF16 1.1/2.25"}}
    return out


def boundary_leg(args, tol=1e-6):
    """Non-homogeneous boundary data and the direct estimator (Eq. Phi_ast).
      w6_lifted_M2048: the 2-D boundary-data workload (lifted, f = sin u), mixed,
        all 20 intervals, time to L-inf 1e-6 of u = w + G;
      w6_lifted_interval: one interval (hand-off + K = 8 iterations) at the full
        M = 65536, node-samples/s;
      w7_*: the 1-D long-time problem (T = 20, f = sin u, boundary data t/2),
        FP64, M = 16384: the hp partition of 20 intervals with the residual
        iteration (lifted data) and with the direct estimator (raw data), and the
        classical single-interval solve over [0, 20] with each (degree 16): the
        L-inf error of u at every node after K iterations per interval."""
    import numpy as np
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    out = {}
    out["w6_lifted_M2048"] = hp_time_to_tol(W.w6(M=2048), L.MIXED, tol, 16)
    wl = W.w6(M=65536, K=8, n_intervals=1)
    plan = Plan.from_workload(wl, precision=L.MIXED)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.begin_interval(0)
    plan.iterate(0, 1)    # sizes the event buffer
    plan.begin_interval(0)
    a.record()
    plan.begin_interval(0)
    plan.iterate(0, 8)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    plan.close()
    out["w6_lifted_interval"] = {"value": node_samples_per_interval(wl, 0) / (ms / 1e3), "unit": "node-samples/s",
                                 "ms": ms, "M": wl.M, "K": 8}

    def solve_err(wl, estimator):
        plan = Plan.from_workload(wl, precision=L.FP64, estimator=estimator)
        grid = plan.node_grid()
        t0 = time.time()
        plan.solve()
        torch.cuda.synchronize()
        wall = time.time() - t0
        errs = [float(np.abs(plan.get_solution(0, m).cpu().numpy()
                             - W.exact_block(wl, wl.instances[0], grid, m)).max())
                for m in range(len(wl.instances[0].degrees))]
        plan.close()
        return {"linf": max(errs), "linf_last_interval": errs[-1], "wall_s": wall, "M": wl.M, "K": wl.K,
                "intervals": len(errs)}
    out["w7_hp_residual_lifted"] = solve_err(W.w7(bc_kind=W.BC_LIFT), 0)
    out["w7_hp_direct_raw"] = solve_err(W.w7(bc_kind=W.BC_RAW), 1)
    out["w7_classical_residual_lifted"] = solve_err(W.w7(bc_kind=W.BC_LIFT, n_intervals=1, degree=16, K=16), 0)
    out["w7_classical_direct_raw"] = solve_err(W.w7(bc_kind=W.BC_RAW, n_intervals=1, degree=16, K=16), 1)
    return out


def chebyshev_leg(args, tol=1e-6):
    """The Chebyshev basis (CGL points, DCT-I reconstruction) against the Jacobi
    basis on the 2-D long-time workload, all 20 intervals, mixed, M = 2048,
    both with the FP32 evaluation kernel (the tensor-core one is Jacobi-only):
    GPU time and iterations to L-inf 1e-6 against the closed form."""
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    out = {}
    out["w2_chebyshev_M2048"] = hp_time_to_tol(W.chebyshev(W.w2(M=2048)), L.MIXED, tol, 16)
    out["w2_jacobi_alu_M2048"] = hp_time_to_tol(W.w2(M=2048), L.MIXED, tol, 16, sweep="events_alu")
    return out


def fractional_leg(args):
    """The fractional Allen-Cahn problem of Section 4, Ex. 2 (alpha-stable walk,
    generalised Jacobi functions; 10 Jacobi-Gauss (alpha/2, alpha/2) nodes x 7 LGL,
    f = u - u^3 + source, exact u = (1-x^2)^{alpha/2} sin(x) e^{cos t}/(1+t^2)),
    mixed, M = 2048, K = 12 iterations per interval, T = 10: the L-inf error of
    every node against the closed form for time steps h = 1, 0.5, 0.25 (Fig.
    EX2, left) at alpha = 0.4 and 1.2, and the classical single interval over
    [0, 10] (degree 16, K = 24) at alpha = 0.4 (Fig. EX2, right); GPU time of
    the solve (CUDA events) and node-samples/s."""
    import numpy as np
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    out = {}

    def run(alpha, h, T=10.0, degree=6, K=12, M=2048):
        wl = W.w8(M=M, K=K, alpha=alpha, h=h, T=T, degree=degree)
        plan = Plan.from_workload(wl, precision=L.MIXED)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.solve()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        x = plan.space_nodes()
        inst = wl.instances[0]
        errs = []
        for m in range(len(inst.degrees)):
            xi = W.time_nodes_reference(wl.time_family, degree)
            t = inst.t_breaks[m] + (xi + 1) * 0.5 * (inst.t_breaks[m + 1] - inst.t_breaks[m])
            errs.append(float(np.abs(plan.get_nodes(0, m).cpu().numpy() - W.frac_exact(alpha, W.EX_FRAC_SIN, x, t)).max()))
        plan.close()
        ns = sum(int(d) * wl.n_space * M * K for d in inst.degrees)
        return {"linf": max(errs), "linf_final_interval": errs[-1], "ms": ms, "node_samples_per_s": ns / (ms / 1e3),
                "intervals": len(errs), "h": h, "alpha": alpha, "M": M, "K": K}
    for alpha in (0.4, 1.2):
        for h in (1.0, 0.5, 0.25):
            out[f"alpha{alpha}_h{h}"] = run(alpha, h)
    for T in (2.0, 10.0):
        try:
            out[f"alpha0.4_classical_single_interval_T{T:g}"] = run(0.4, T, T=T, degree=16, K=24)
        except L.SpmcError as e:   # the Picard iteration over one long interval does not contract
            out[f"alpha0.4_classical_single_interval_T{T:g}"] = {"diverged": True, "status": str(e)}
    return out


def w5_leg(args):
    """The adjoint workload at its full geometry and batch (128 instances of
    2-D Allen-Cahn, 16 x 16 JG x 12 LGL, T = 5 in 10 intervals, kappa = 0.01,
    K = 8), mixed, at M = 64 samples per node (the full M = 16384 means about
    1.9e13 evaluation events per forward solve, since kappa = 0.01 keeps every
    ball full): the forward solve and the reverse-mode gradient of
    L = 1/2 |u(T)|^2 w.r.t. the reaction scales and the 64 initial
    coefficients of every instance, wall time of each (synchronised)."""
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan
    wl = W.w5(M=64)
    plan = Plan.from_workload(wl, precision=L.MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    flat = plan.solve()
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    z = plan.final_values(flat)
    st = plan.stats()
    t0 = time.perf_counter()
    gs, gc = plan.grad(z, n_coef=8)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    plan.close()
    ns = node_samples_per_solve(wl)
    return {"forward_s": tf, "grad_s": tb, "node_samples_per_s_forward": ns / tf, "events_forward": st["points"],
            "graph_launches": st["graph_launches"], "M": wl.M, "instances": len(wl.instances),
            "grad_norm": float(torch.linalg.vector_norm(gs).item())}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on a bounded sample of the
    same workload, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args, 0)
    steps = []
    for _ in range(max(1, args.warmup) // 3 + args.steps):
        steps.append(cpu_baseline(wl, budget_s=6.0))
    vals = [s["value"] for s in steps[-args.steps:]]
    v = statistics.mean(vals)
    cb = dict(steps[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": "node-samples/sec & time to L-inf err 1e-6: batched mixed vs plain FP64, 1 B300",
            "value": v, "unit": "node-samples/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "w2-2d-long-time (bounded CPU sample)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "node-samples/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """A small untimed case for profilers: one iteration of the first interval."""
    import torch
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300.api import Plan
    torch.cuda.set_device(0)
    from paper_2608_22190_b300 import workloads as W
    if args.case == "iterate1_5d":
        wl = W.w4(M=args.M, K=1)
    elif args.case == "iterate1_frac":
        wl = W.w8(M=args.M, K=1, alpha=0.4, h=0.5, T=0.5)
    elif args.case == "iterate1_cheb":
        wl = W.chebyshev(workload(args, 0))
    else:
        wl = workload(args, 0)
    plan = Plan.from_workload(wl, precision=L.MIXED if args.precision == "mixed" else L.FP64)
    plan.begin_interval(0)
    plan.iterate(0, 1)
    print(json.dumps({"case": args.case, "M": wl.M, "stats": plan.stats()}))
    plan.close()


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
