"""Shared helpers of the tests: the same problem set up for the CUDA path (through
the C-ABI) and for the CPU oracle."""
import os

import numpy as np

from paper_2608_22190_b300 import workloads as W


def oracle_spec(O, wl, inst, **over):
    kw = dict(dim=wl.dim, n_space=wl.n_space, time_family=wl.time_family, n_ref=wl.n_ref, M=wl.M,
              kappa=wl.kappa, seed=wl.seed, f_kind=inst.f_kind, f_coef=tuple(inst.f_coef), f_scale=inst.f_scale,
              ex_kind=inst.ex_kind, ex_beta=inst.ex_beta, n_sub=wl.n_sub, shell=wl.shell,
              max_steps=wl.max_steps, n_threads=os.cpu_count() or 1, bc_kind=getattr(inst, "bc_kind", 0),
              basis=1 if wl.time_family == 2 else 0)
    kw.update(over)
    return O.Spec(**kw)


def oracle_u0(O, wl, inst, spec):
    grid = O.space_nodes_grid(spec)
    if inst.u0_kind == "phi_coef":
        nc = inst.u0_coef.shape[0]
        x, _ = O.jg11_nodes(wl.n_space)
        ph = np.array([O.phi(wl.n_space - 1, xj)[:nc] for xj in x])   # [j, i]
        full = ph @ inst.u0_coef @ ph.T                                # [jx, jy]
        return np.ascontiguousarray(full.T).ravel()                     # x fastest
    return W.u0_nodal(inst, grid)


def parity_tol(ref):
    """|gpu - oracle| bound for the FP64 path: 1e-12 x max(|ref_i|, 1e-3 max|ref|).
    That is 1e-12 relative for every node whose magnitude is at least 1e-3 of the
    largest, and an absolute 1e-15 x max|ref| for the smaller ones (nodes near the
    boundary of a sine profile, whose relative error is dominated by the rounding
    of their larger neighbours' contributions).  The two sides differ only in
    summation order and in last-bit rounding of tables and transcendentals."""
    ref = np.asarray(ref)
    return 1e-12 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
