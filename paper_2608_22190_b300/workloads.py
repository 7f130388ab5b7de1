"""Seeded synthetic workloads shaped like the paper's experiments.

This module holds inputs only: problem shapes, meshes, degrees and the random
per-instance parameters (reaction scales, interval counts, initial-condition
coefficients, walk start points).  It contains none of the method's arithmetic
and serves the CUDA path and the CPU oracle alike.

Workloads (sizes as the benchmarks state them; Section 4 examples they stand in for):
  w1  1-D, u = e^{-t} sin(pi x), f = -u^3 + source, T = 1, one interval,
      14 interior JG(1,1) nodes (16 LGL points with the two fixed boundary
      points) x 16 left Gauss-Radau time nodes, M = 4096, K = 6     (Ex. 1 shape)
  w2  2-D long time, u = e^{-0.1 t} sin(pi x) sin(pi y), f = sin u + source,
      T = 20 in 20 intervals of h = 1, 24 x 24 JG x 16 LGL, M = 65536, K = 8
                                                                  (Ex. 2 shape)
  w3  1-D initial singularity, u0 = |x|^0.6 (1 - x^2), f = s (u - u^3),
      geometric mesh t_n = T 0.2^{N-n}, degree p_k = 4 + 2k, 32 JG nodes,
      M = 32768, K = 8; 256 instances, s ~ U[0.5, 2], N ~ U{8..16}  (Ex. 3 shape)
  w4  5-D, u = e^{-t} prod cos(pi x_e / 2), f = -u^3 + source, T = 0.5,
      8 JG nodes per axis x 8 LGL, M = 16384, K = 6              (Ex. 4 shape)
  w6  2-D non-homogeneous boundary data, u = e^{-0.1 t} prod cos(pi (x_e - 0.3) / 3)
      (different non-zero values on opposite faces), f = sin u + source, lifted,
      T = 20 in 20 intervals of h = 1, 24 x 24 JG x 16 LGL, M = 65536, K = 8
  w8  1-D fractional Allen-Cahn (Section 4, Ex. 2): d_t u + (-Delta)^{alpha/2} u + u^3 - u = f_add,
      u = (1-x^2)_+^{alpha/2} sin(x) e^{cos t}/(1+t^2), alpha = 0.4, 10 Jacobi-Gauss (alpha/2, alpha/2)
      nodes x 7 LGL (M_n = 6), h = 0.5 (0.1..1), alpha-stable walk with N_ref = 20
  w7  1-D long time for the direct estimator and the classical comparison,
      u = e^{-t/4} sin(pi x) + t/2 (boundary data t/2), f = sin u + source, kappa = 1/(4 pi^2),
      T = 20 in 20 intervals of degree 8 (or one interval: the classical single solve)
  w5  adjoint: 2-D u_t = 0.01 Delta u + a (u - u^3), T = 5 in 10 intervals,
      16 x 16 JG x 12 LGL, M = 16384, u0 = sum_{i,j<8} c_ij phi_i phi_j with
      c_ij = z_ij / (1+i+j)^2, z ~ N(0,1), scaled down to max |u0| = 1 where the
      draw exceeds it (the phase variable's range); 128 instances
The paper uses no public dataset; these synthetic inputs stand in for its
examples (its data is only available on request).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# enums shared by name with the C-ABI header (values fixed there)
TIME_LGL, TIME_RADAU_LEFT, TIME_CHEB = 0, 1, 2
F_POLY3, F_SIN = 0, 1
EX_NONE, EX_SIN, EX_COSHALF, EX_POLY, EX_COSTHIRD, EX_SINPLUS, EX_FRAC_SIN, EX_FRAC_POLY = range(8)
BC_ZERO, BC_LIFT, BC_RAW = 0, 1, 2


@dataclass
class Instance:
    t_breaks: np.ndarray            # n_intervals + 1 breakpoints
    degrees: np.ndarray             # time degree M_n per interval (M_n + 1 nodes)
    f_kind: int = F_POLY3
    f_coef: tuple = (0.0, 0.0, 0.0, -1.0)
    f_scale: float = 1.0
    ex_kind: int = EX_NONE
    ex_beta: float = 1.0
    u0_kind: str = "exact"          # "exact" (closed form at t=0), "singular", "phi_coef"
    u0_coef: Optional[np.ndarray] = None   # phi_i phi_j coefficients (u0_kind == "phi_coef")
    bc_kind: int = BC_ZERO          # boundary data: zero, lifted, or raw (direct estimator)


@dataclass
class Workload:
    name: str
    dim: int
    n_space: int
    time_family: int
    M: int
    K: int
    kappa: float = 1.0
    seed: int = 0
    n_ref: int = 80
    n_sub: int = 4
    shell: float = 0.0          # 0: half the outermost node's distance to the boundary
    max_steps: int = 512
    instances: List[Instance] = field(default_factory=list)
    alpha: float = 0.0          # (0, 2): the fractional case (alpha-stable walk, d = 1)

    @property
    def n_nodes_space(self) -> int:
        return self.n_space ** self.dim


def uniform_mesh(T: float, n: int) -> np.ndarray:
    return np.linspace(0.0, T, n + 1)


def geometric_mesh(T: float, n: int, ratio: float = 0.2) -> np.ndarray:
    t = np.zeros(n + 1)
    for k in range(1, n + 1):
        t[k] = T * ratio ** (n - k)
    return t


def w1(M: int = 4096, K: int = 6, seed: int = 0, n_space: int = 14, degree: int = 15) -> Workload:
    inst = Instance(t_breaks=uniform_mesh(1.0, 1), degrees=np.array([degree]), f_coef=(0, 0, 0, -1.0),
                    ex_kind=EX_SIN, ex_beta=1.0)
    return Workload("w1-1d-single-interval", 1, n_space, TIME_RADAU_LEFT, M, K, seed=seed, instances=[inst])


def w2(M: int = 65536, K: int = 8, seed: int = 0, n_space: int = 24, degree: int = 15,
       n_intervals: int = 20, h: float = 1.0) -> Workload:
    inst = Instance(t_breaks=uniform_mesh(h * n_intervals, n_intervals), degrees=np.full(n_intervals, degree),
                    f_kind=F_SIN, f_coef=(0, 0, 0, 0), ex_kind=EX_SIN, ex_beta=0.1)
    return Workload("w2-2d-long-time", 2, n_space, TIME_LGL, M, K, seed=seed, n_ref=160, instances=[inst])


def w3(M: int = 32768, K: int = 8, seed: int = 0, batch: int = 256, n_space: int = 32, param_seed: int = 1,
       fixed_intervals: Optional[int] = None) -> Workload:
    rng = np.random.default_rng(param_seed)
    insts = []
    for b in range(batch):
        s = float(rng.uniform(0.5, 2.0))
        n = int(rng.integers(8, 17)) if fixed_intervals is None else fixed_intervals
        deg = np.array([4 + 2 * k for k in range(n)])
        insts.append(Instance(t_breaks=geometric_mesh(1.0, n), degrees=deg, f_coef=(0, 1.0, 0, -1.0),
                              f_scale=s, ex_kind=EX_NONE, u0_kind="singular"))
    return Workload("w3-1d-initial-singularity-batch", 1, n_space, TIME_LGL, M, K, seed=seed, instances=insts)


def w4(M: int = 16384, K: int = 6, seed: int = 0, n_space: int = 8, degree: int = 7) -> Workload:
    inst = Instance(t_breaks=uniform_mesh(0.5, 1), degrees=np.array([degree]), f_coef=(0, 0, 0, -1.0),
                    ex_kind=EX_COSHALF, ex_beta=1.0)
    return Workload("w4-5d", 5, n_space, TIME_LGL, M, K, seed=seed, instances=[inst])


def w5(M: int = 16384, K: int = 8, seed: int = 0, batch: int = 128, n_space: int = 16, degree: int = 11,
       n_intervals: int = 10, T: float = 5.0, param_seed: int = 2, n_coef: int = 8) -> Workload:
    rng = np.random.default_rng(param_seed)
    insts = []
    i = np.arange(n_coef)
    decay = 1.0 / (1.0 + i[:, None] + i[None, :]) ** 2
    # u0 on a fine grid of the square, for the amplitude cap below
    g = np.linspace(-1.0, 1.0, 129)
    phi = np.stack([phi_values(p, g) for p in range(n_coef)])          # [p, point]
    for b in range(batch):
        c = rng.standard_normal((n_coef, n_coef)) * decay
        # Allen-Cahn's phase variable lies in [-1, 1]; draws whose initial data
        # leave it are scaled back to max |u0| = 1 (then |f'(u)| <= 2 and h |f'| <= 1)
        amp = np.abs(phi.T @ c @ phi).max()
        if amp > 1.0:
            c = c / amp
        insts.append(Instance(t_breaks=uniform_mesh(T, n_intervals), degrees=np.full(n_intervals, degree),
                              f_coef=(0, 1.0, 0, -1.0), f_scale=1.0, ex_kind=EX_NONE, u0_kind="phi_coef",
                              u0_coef=c))
    return Workload("w5-2d-adjoint-batch", 2, n_space, TIME_LGL, M, K, kappa=0.01, seed=seed, instances=insts)


def phi_values(p: int, x: np.ndarray) -> np.ndarray:
    """phi_p(x) = 2(p+1)/(2p+3) (L_p(x) - L_{p+2}(x)) (Section 2.3), for building
    initial data from coefficients."""
    from numpy.polynomial import legendre as npleg
    c = np.zeros(p + 3)
    c[p], c[p + 2] = 1.0, -1.0
    return 2.0 * (p + 1) / (2 * p + 3) * npleg.legval(x, c)


def uniform_points(n: int, dim: int, seed: int) -> np.ndarray:
    """Start points drawn uniformly in (-1,1)^dim (walk statistics, Table 1)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, dim))


def w6(M: int = 65536, K: int = 8, seed: int = 0, n_space: int = 24, degree: int = 15,
       n_intervals: int = 20, h: float = 1.0) -> Workload:
    inst = Instance(t_breaks=uniform_mesh(h * n_intervals, n_intervals), degrees=np.full(n_intervals, degree),
                    f_kind=F_SIN, f_coef=(0, 0, 0, 0), ex_kind=EX_COSTHIRD, ex_beta=0.1, bc_kind=BC_LIFT)
    return Workload("w6-2d-boundary-data", 2, n_space, TIME_LGL, M, K, seed=seed, n_ref=160, instances=[inst])


def w7(M: int = 16384, K: int = 4, seed: int = 0, n_space: int = 14, degree: int = 8, T: float = 20.0,
       n_intervals: int = 20, bc_kind: int = BC_RAW) -> Workload:
    inst = Instance(t_breaks=uniform_mesh(T, n_intervals), degrees=np.full(n_intervals, degree),
                    f_kind=F_SIN, f_coef=(0, 0, 0, 0), ex_kind=EX_SINPLUS, ex_beta=0.25, bc_kind=bc_kind)
    return Workload("w7-1d-direct-long-time", 1, n_space, TIME_LGL, M, K, kappa=0.25 / np.pi ** 2, seed=seed,
                    n_ref=40, instances=[inst])


def w8(M: int = 4096, K: int = 10, seed: int = 0, n_space: int = 10, degree: int = 6, alpha: float = 0.4,
       h: float = 0.5, T: float = 5.0, n_ref: int = 20) -> Workload:
    n_int = int(round(T / h))
    inst = Instance(t_breaks=uniform_mesh(n_int * h, n_int), degrees=np.full(n_int, degree),
                    f_coef=(0.0, 1.0, 0.0, -1.0), ex_kind=EX_FRAC_SIN, ex_beta=0.0)
    return Workload("w8-1d-fractional-allen-cahn", 1, n_space, TIME_LGL, M, K, seed=seed, n_ref=n_ref, n_sub=1,
                    instances=[inst], alpha=alpha)


def frac_nodes(n: int, alpha: float) -> np.ndarray:
    """Jacobi-Gauss (alpha/2, alpha/2) nodes (scipy), for the closed forms."""
    import scipy.special as sps
    return np.sort(sps.roots_jacobi(n, alpha / 2, alpha / 2)[0])


def u0_nodal(inst: Instance, grid: np.ndarray) -> np.ndarray:
    """Initial values at the spatial nodes (grid: (S, d) coordinates): the
    closed form at t = 0 of the manufactured solution, or the singular profile
    |x|^0.6 (1 - x^2) of the initial-singularity workload."""
    if inst.u0_kind == "singular":
        return np.prod(np.abs(grid) ** 0.6 * (1.0 - grid ** 2), axis=1)
    if inst.ex_kind == EX_SIN:
        return np.prod(np.sin(np.pi * grid), axis=1)
    if inst.ex_kind == EX_COSHALF:
        return np.prod(np.cos(0.5 * np.pi * grid), axis=1)
    if inst.ex_kind == EX_POLY:
        return np.prod((1.0 - grid ** 2) * (1.0 + grid), axis=1)
    if inst.ex_kind == EX_COSTHIRD:
        return np.prod(np.cos(np.pi * (grid - 0.3) / 3.0), axis=1)
    if inst.ex_kind == EX_SINPLUS:
        return np.prod(np.sin(np.pi * grid), axis=1)
    if inst.ex_kind in (EX_FRAC_SIN, EX_FRAC_POLY):
        raise ValueError("fractional kinds: use frac_exact with the workload's alpha")
    raise ValueError("instance has no closed-form initial condition")


def frac_exact(alpha: float, ex_kind: int, x: np.ndarray, t) -> np.ndarray:
    """The fractional examples' closed forms at points x (|x| < 1) and times t:
    6, (1-x^2)^{alpha/2} sin(x) e^{cos t}/(1+t^2) (Section 4, Ex. 2); 7,
    (1+t)(1-x^2)^{alpha/2}(1 + P_1^{(a,a)}(x)/2), P_1 = (alpha/2 + 1) x.
    Returns (len(t), len(x))."""
    a = alpha / 2
    t = np.atleast_1d(np.asarray(t, dtype=float))[:, None]
    w = (1 - x ** 2) ** a
    if ex_kind == EX_FRAC_SIN:
        return w * np.sin(x) * np.exp(np.cos(t)) / (1 + t ** 2)
    return (1 + t) * w * (1 + 0.5 * (a + 1) * x)


def chebyshev(wl: Workload) -> Workload:
    """The same workload in the Chebyshev basis (Chebyshev-Gauss-Lobatto points
    in space and time)."""
    return replace(wl, time_family=TIME_CHEB, name=wl.name + "-chebyshev")


def time_nodes_reference(family: int, Mt: int) -> np.ndarray:
    """Reference-interval time nodes (LGL, left Radau or Chebyshev-Gauss-Lobatto),
    for evaluating closed-form solutions at the nodes."""
    import scipy.special as sps
    if family == TIME_CHEB:
        return -np.cos(np.pi * np.arange(Mt + 1) / Mt)
    if family == TIME_LGL:
        inner = sps.roots_jacobi(Mt - 1, 1.0, 1.0)[0] if Mt >= 2 else np.zeros(0)
        return np.concatenate([[-1.0], inner, [1.0]])
    return np.concatenate([[-1.0], sps.roots_jacobi(Mt, 0.0, 1.0)[0]])


def exact_block(wl: Workload, inst: Instance, grid: np.ndarray, interval: int) -> np.ndarray:
    """The manufactured closed form at every node of one interval, (M_n+1, S)."""
    Mt = int(inst.degrees[interval])
    t0, t1 = inst.t_breaks[interval], inst.t_breaks[interval + 1]
    t = t0 + (time_nodes_reference(wl.time_family, Mt) + 1.0) * 0.5 * (t1 - t0)
    if inst.ex_kind == EX_SIN:
        return np.exp(-inst.ex_beta * t)[:, None] * np.prod(np.sin(np.pi * grid), axis=1)[None, :]
    if inst.ex_kind == EX_COSHALF:
        return np.exp(-inst.ex_beta * t)[:, None] * np.prod(np.cos(0.5 * np.pi * grid), axis=1)[None, :]
    if inst.ex_kind == EX_POLY:
        return (1.0 + t + t * t)[:, None] * np.prod((1.0 - grid ** 2) * (1.0 + grid), axis=1)[None, :]
    if inst.ex_kind == EX_COSTHIRD:
        return np.exp(-inst.ex_beta * t)[:, None] * np.prod(np.cos(np.pi * (grid - 0.3) / 3.0), axis=1)[None, :]
    if inst.ex_kind == EX_SINPLUS:
        return (np.exp(-inst.ex_beta * t)[:, None] * np.prod(np.sin(np.pi * grid), axis=1)[None, :]
                + 0.5 * t[:, None])
    raise ValueError("instance has no closed form")
