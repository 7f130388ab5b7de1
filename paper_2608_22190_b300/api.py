"""Python front end of the CUDA library: plans over PyTorch device memory.

A Plan holds one batch of instances of Eq. mainproblem (homogeneous Dirichlet
data on (-1,1)^d) and runs Algorithm 1 on the caller's CUDA stream.  All
arithmetic of the method happens in libspmc.so; this module only marshals
arguments and allocates result tensors with torch.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from . import workloads as W


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    def __init__(self, dim, n_space, time_family, max_intervals, max_degree, M, K, tol=0.0, n_ref=80, n_sub=4,
                 shell=1e-4, max_steps=512, kappa=1.0, seed=0, precision=L.FP64, batch=1, walk_mode=L.WALK_BALLS,
                 estimator=L.EST_RESIDUAL, alpha=0.0, basis=L.BASIS_JACOBI):
        d = L.PlanDesc()
        d.dim, d.n_space, d.time_family = dim, n_space, time_family
        d.max_intervals, d.max_degree, d.M, d.K, d.tol = max_intervals, max_degree, M, K, tol
        d.n_ref, d.n_sub, d.shell, d.max_steps = n_ref, n_sub, shell, max_steps
        d.kappa, d.seed, d.precision, d.batch = kappa, seed, precision, batch
        d.walk_mode = walk_mode
        d.estimator = estimator
        d.alpha = alpha
        d.basis = basis
        self.desc = d
        self._h = C.c_void_p()
        L.check(L.lib.spmc_plan(C.byref(d), C.byref(self._h)))
        self.dim, self.n_space, self.batch = dim, n_space, batch
        self.S = n_space ** dim
        self.degrees = [None] * batch

    # ------------------------------------------------------------------ set-up
    def space_nodes(self) -> np.ndarray:
        x = np.zeros(self.n_space)
        L.check(L.lib.spmc_space_nodes(self._h, x.ctypes.data_as(C.POINTER(C.c_double))), self._h)
        return x

    def node_grid(self) -> np.ndarray:
        """(S, d) coordinates of the spatial nodes, x_1 fastest."""
        x = self.space_nodes()
        idx = np.arange(self.S)
        cols = []
        for e in range(self.dim):
            cols.append(x[(idx // self.n_space ** e) % self.n_space])
        return np.stack(cols, axis=1)

    def set_problem(self, instance, t_breaks, degrees, f_kind=L.F_POLY3, f_coef=(0, 0, 0, -1.0), f_scale=1.0,
                    ex_kind=L.EX_NONE, ex_beta=1.0, u0=None, u0_kind=L.U0_NODAL, n_coef=0, bc_kind=L.BC_ZERO):
        t = np.ascontiguousarray(t_breaks, dtype=np.float64)
        dg = np.ascontiguousarray(degrees, dtype=np.int32)
        u = np.ascontiguousarray(u0, dtype=np.float64).ravel()
        p = L.Problem()
        p.n_intervals = len(dg)
        p.t_breaks = t.ctypes.data_as(C.POINTER(C.c_double))
        p.degrees = dg.ctypes.data_as(C.POINTER(C.c_int))
        p.f_kind, p.f_scale, p.ex_kind, p.ex_beta = f_kind, f_scale, ex_kind, ex_beta
        for i, c in enumerate(f_coef):
            p.f_coef[i] = c
        p.u0_kind, p.n_coef = u0_kind, n_coef
        p.u0 = u.ctypes.data_as(C.POINTER(C.c_double))
        p.bc_kind = bc_kind
        L.check(L.lib.spmc_set_problem(self._h, instance, C.byref(p)), self._h)
        self.degrees[instance] = [int(v) for v in dg]

    @classmethod
    def from_workload(cls, wl: "W.Workload", precision=L.FP64, **overrides):
        insts = wl.instances
        kw = dict(dim=wl.dim, n_space=wl.n_space, time_family=wl.time_family,
                  max_intervals=max(len(i.degrees) for i in insts), max_degree=max(int(max(i.degrees)) for i in insts),
                  M=wl.M, K=wl.K, n_ref=wl.n_ref, n_sub=wl.n_sub, shell=wl.shell, max_steps=wl.max_steps,
                  kappa=wl.kappa, seed=wl.seed, precision=precision, batch=len(insts))
        if getattr(wl, "alpha", 0.0):
            kw.update(alpha=wl.alpha, walk_mode=L.WALK_STABLE)
        if wl.time_family == L.TIME_CHEB:
            kw.update(basis=L.BASIS_CHEB)
        kw.update(overrides)
        plan = cls(**kw)
        grid = plan.node_grid()
        for b, inst in enumerate(insts):
            if inst.u0_kind == "phi_coef":
                nc = inst.u0_coef.shape[0]
                # x_1 fastest: coefficient (i, j) of phi_i(x) phi_j(y) sits at i + nc j
                plan.set_problem(b, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, inst.f_scale,
                                 inst.ex_kind, inst.ex_beta, np.ascontiguousarray(inst.u0_coef.T).ravel(),
                                 L.U0_PHI_COEF, nc)
            else:
                u0 = (W.frac_exact(wl.alpha, inst.ex_kind, grid[:, 0], inst.t_breaks[0])[0]
                      if getattr(wl, "alpha", 0.0) else W.u0_nodal(inst, grid))
                plan.set_problem(b, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, inst.f_scale,
                                 inst.ex_kind, inst.ex_beta, u0, bc_kind=getattr(inst, "bc_kind", L.BC_ZERO))
        return plan

    # ------------------------------------------------------------------ layout
    def layout(self, instance):
        off, cnt = C.c_longlong(), C.c_longlong()
        L.check(L.lib.spmc_solution_layout(self._h, instance, C.byref(off), C.byref(cnt)), self._h)
        return off.value, cnt.value

    def total_size(self) -> int:
        o, c = self.layout(self.batch - 1)
        return o + c

    def blocks(self, flat: torch.Tensor, instance: int):
        """Split an instance's part of spmc_solve's output into per-interval (M_n+1, S) views."""
        off, _ = self.layout(instance)
        out = []
        for Mt in self.degrees[instance]:
            n = (Mt + 1) * self.S
            out.append(flat[off: off + n].view(Mt + 1, self.S))
            off += n
        return out

    # ------------------------------------------------------------------ run
    def solve(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.total_size(), dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.numel() >= self.total_size()
        L.check(L.lib.spmc_solve(self._h, C.c_void_p(_stream_ptr(stream)), C.c_void_p(out.data_ptr())), self._h)
        return out

    def begin_interval(self, interval: int, stream=None):
        L.check(L.lib.spmc_begin_interval(self._h, C.c_void_p(_stream_ptr(stream)), interval), self._h)

    def iterate(self, interval: int, n_iter: int = 1, stream=None) -> float:
        mx = C.c_double()
        L.check(L.lib.spmc_iterate(self._h, C.c_void_p(_stream_ptr(stream)), interval, n_iter, C.byref(mx)), self._h)
        return mx.value

    def round_nodes(self, interval: int) -> int:
        """Number of (time node, spatial node) pairs sampled on `interval`."""
        n = C.c_longlong()
        L.check(L.lib.spmc_round_nodes(self._h, interval, C.byref(n)), self._h)
        return n.value

    def iterate_shard(self, interval: int, rank: int, world: int, eps: torch.Tensor, stream=None):
        """The next iteration's sweep for this rank's share of the pairs; writes
        their eps into `eps` (float64, device, round_nodes(interval) entries)."""
        assert eps.dtype == torch.float64 and eps.is_cuda and eps.numel() >= self.round_nodes(interval)
        L.check(L.lib.spmc_iterate_shard(self._h, C.c_void_p(_stream_ptr(stream)), interval, rank, world,
                                         C.c_void_p(eps.data_ptr())), self._h)

    def apply_eps(self, interval: int, eps: torch.Tensor, stream=None) -> float:
        """u += eps for every pair of `interval`; returns max |eps|."""
        assert eps.dtype == torch.float64 and eps.is_cuda
        mx = C.c_double()
        L.check(L.lib.spmc_apply_eps(self._h, C.c_void_p(_stream_ptr(stream)), interval,
                                     C.c_void_p(eps.data_ptr()), C.byref(mx)), self._h)
        return mx.value

    def final_values(self, flat: torch.Tensor) -> torch.Tensor:
        """u(T) at the spatial nodes for every instance: the last row of each
        instance's last interval (LGL time nodes end at t_n), shape (batch, S)."""
        rows = []
        for b in range(self.batch):
            blk = self.blocks(flat, b)[-1]
            rows.append(blk[-1])
        return torch.stack(rows)

    def grad(self, dloss_du_T: torch.Tensor, n_coef: int = 0, stream=None):
        """Reverse-mode gradient after solve(): returns (dL/d f_scale (batch,),
        dL/d u0 coefficients (batch, n_coef^d) or None)."""
        g = dloss_du_T.contiguous().to(torch.float64)
        assert g.is_cuda and g.numel() == self.batch * self.S
        gs = torch.zeros(self.batch, dtype=torch.float64, device="cuda")
        gc = torch.zeros(self.batch, max(1, n_coef ** self.dim), dtype=torch.float64, device="cuda") if n_coef else None
        L.check(L.lib.spmc_grad(self._h, C.c_void_p(_stream_ptr(stream)), C.c_void_p(g.data_ptr()),
                                C.c_void_p(gs.data_ptr()), C.c_void_p(gc.data_ptr() if gc is not None else None)),
                self._h)
        return gs, gc

    def get_nodes(self, instance: int, interval: int, stream=None) -> torch.Tensor:
        Mt = self.degrees[instance][interval]
        out = torch.empty((Mt + 1, self.S), dtype=torch.float64, device="cuda")
        L.check(L.lib.spmc_get_nodes(self._h, C.c_void_p(_stream_ptr(stream)), instance, interval,
                                     C.c_void_p(out.data_ptr())), self._h)
        return out

    def get_solution(self, instance: int, interval: int, stream=None) -> torch.Tensor:
        """u at the nodes of (instance, interval): the nodal values plus the lifting
        of the boundary data where it is lifted (computed on the device)."""
        Mt = self.degrees[instance][interval]
        out = torch.empty((Mt + 1, self.S), dtype=torch.float64, device="cuda")
        L.check(L.lib.spmc_get_solution(self._h, C.c_void_p(_stream_ptr(stream)), instance, interval,
                                        C.c_void_p(out.data_ptr())), self._h)
        return out

    def get_nodes_into(self, instance: int, interval: int, dst: torch.Tensor, stream=None):
        """Copy (instance, interval)'s nodal values into dst (device or pinned host tensor)."""
        Mt = self.degrees[instance][interval]
        assert dst.dtype == torch.float64 and dst.is_contiguous() and dst.numel() >= (Mt + 1) * self.S
        L.check(L.lib.spmc_get_nodes(self._h, C.c_void_p(_stream_ptr(stream)), instance, interval,
                                     C.c_void_p(dst.data_ptr())), self._h)
        return dst

    def set_nodes(self, instance: int, interval: int, values: torch.Tensor, stream=None):
        v = values.contiguous()
        Mt = self.degrees[instance][interval]
        assert v.dtype == torch.float64 and v.numel() == (Mt + 1) * self.S
        L.check(L.lib.spmc_set_nodes(self._h, C.c_void_p(_stream_ptr(stream)), instance, interval,
                                     C.c_void_p(v.data_ptr())), self._h)
        if v.is_cuda:
            torch.cuda.current_stream().synchronize()

    def stats(self) -> dict:
        s = L.Stats()
        L.check(L.lib.spmc_get_stats(self._h, C.byref(s)), self._h)
        return {"points": s.points, "capped": s.capped, "iterations_run": s.iterations_run,
                "last_max_eps": s.last_max_eps, "sweep_launches": s.sweep_launches, "sweep_ms": s.sweep_ms,
                "walk_ms": s.walk_ms, "fill_ms": s.fill_ms, "eval_ms": s.eval_ms,
                "eval_launches": s.eval_launches, "workspace_bytes": s.workspace_bytes,
                "graph_launches": s.graph_launches}

    def autotune(self, interval: int = 0, stream=None) -> float:
        """Tune the forward sweep by timing one sweep per candidate setting: the
        event sweep's batch size, or the cohort kernel's width (nodal values and
        the point counters unchanged).  Returns the best sweep time in ms."""
        ms = C.c_double()
        L.check(L.lib.spmc_autotune(self._h, C.c_void_p(_stream_ptr(stream)), interval, C.byref(ms)), self._h)
        return ms.value

    def set_sweep(self, mode: str = "events", batch: int = 0):
        """Forward-sweep strategy for d <= 2: "events" (default; tensor-core
        evaluation for d = 2 in mixed precision), "events_alu" or "cohort"."""
        m = {"events": L.SPMC_SWEEP_EVENTS, "cohort": L.SPMC_SWEEP_COHORT,
             "events_alu": L.SPMC_SWEEP_EVENTS_ALU}[mode]
        L.check(L.lib.spmc_set_sweep(self._h, m, int(batch)), self._h)

    def set_acceleration(self, mode: str = "none"):
        """"aitken": Aitken's dynamic relaxation of the update (factor in [1/2, 2]); "none" (default)."""
        L.check(L.lib.spmc_set_acceleration(self._h, {"none": L.ACCEL_NONE, "aitken": L.ACCEL_AITKEN}[mode]),
                self._h)

    def set_graphs(self, enable: bool):
        """solve(): run each interval after the first as one captured CUDA graph (default on)."""
        L.check(L.lib.spmc_set_graphs(self._h, 1 if enable else 0), self._h)

    def set_timing(self, enable: bool):
        L.check(L.lib.spmc_set_timing(self._h, 1 if enable else 0), self._h)

    def close(self):
        if self._h:
            L.lib.spmc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SpmcFunction(torch.autograd.Function):
    """u(T) at the nodes as a differentiable function of the reaction scales
    (batch,) and the u0 phi-coefficients (batch, n_coef, n_coef) (2-D, LGL time
    nodes).  Forward: spmc_solve; backward: spmc_grad (adjoint sweeps on the
    forward walks, iterations recomputed from each interval's first iterate)."""

    @staticmethod
    def forward(ctx, f_scale, u0_coef, plan, wl):
        nc = u0_coef.shape[-1]
        for b, inst in enumerate(wl.instances):
            c = u0_coef[b].detach().cpu().numpy()
            plan.set_problem(b, inst.t_breaks, inst.degrees, inst.f_kind, inst.f_coef, float(f_scale[b]),
                             inst.ex_kind, inst.ex_beta, np.ascontiguousarray(c.T).ravel(), L.U0_PHI_COEF, nc)
        flat = plan.solve()
        ctx.plan, ctx.nc, ctx.dim = plan, nc, wl.dim
        ctx.devices = (f_scale.device, u0_coef.device)
        return plan.final_values(flat).clone().to(u0_coef.device)

    @staticmethod
    def backward(ctx, grad_out):
        gs, gc = ctx.plan.grad(grad_out.to("cuda"), n_coef=ctx.nc)
        nc = ctx.nc
        # coefficient (i, j) of phi_i(x) phi_j(y) sits at i + nc j
        gcoef = gc.view(-1, nc, nc).transpose(1, 2).contiguous()
        return gs.to(ctx.devices[0]), gcoef.to(ctx.devices[1]), None, None
