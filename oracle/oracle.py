"""Python access to the CPU oracle (spmc_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline leg may import
this module.  The product path never calls it.  Builds ``liboracle.so`` next to the
C source with gcc (FP64, no FMA contraction) and wraps its entry points with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n_space", C.c_int), ("time_family", C.c_int), ("n_ref", C.c_int),
        ("M", C.c_int64), ("kappa", C.c_double), ("seed", C.c_uint64), ("instance", C.c_int),
        ("f_kind", C.c_int), ("f_coef", C.c_double * 4), ("f_scale", C.c_double),
        ("ex_kind", C.c_int), ("ex_beta", C.c_double), ("n_threads", C.c_int),
        ("walk_mode", C.c_int), ("shell", C.c_double), ("max_steps", C.c_int), ("n_sub", C.c_int),
        ("bc_kind", C.c_int), ("estimator", C.c_int), ("alpha", C.c_double), ("basis", C.c_int),
    ]


class IntervalCtx(C.Structure):
    _fields_ = [
        ("Mt", C.c_int), ("t0", C.c_double), ("h", C.c_double),
        ("cu", C.POINTER(C.c_double)), ("ct", C.POINTER(C.c_double)),
        ("interval", C.c_int), ("iteration", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        D = C.POINTER(C.c_double)
        I = C.POINTER(C.c_int)
        U32 = C.POINTER(C.c_uint32)
        P = C.POINTER(Problem)
        sig = {
            "orc_philox4x32_10": (None, [U32, U32, U32]),
            "orc_u01_pair": (C.c_double, [C.c_uint32, C.c_uint32]),
            "orc_u01_word": (C.c_double, [C.c_uint32]),
            "orc_ball_words_per_step": (C.c_int, [C.c_int]),
            "orc_words_per_step": (C.c_int, [C.c_int]),
            "orc_legendre": (None, [C.c_int, C.c_double, D]),
            "orc_jacobi11": (None, [C.c_int, C.c_double, D]),
            "orc_phi": (None, [C.c_int, C.c_double, D]),
            "orc_jg11_nodes": (None, [C.c_int, D, D]),
            "orc_lgl_nodes": (None, [C.c_int, D, D]),
            "orc_radau_left_nodes": (None, [C.c_int, D, D]),
            "orc_space_analysis": (None, [C.c_int, D]),
            "orc_time_analysis": (None, [C.c_int, C.c_int, D]),
            "orc_f": (C.c_double, [P, C.c_double]),
            "orc_exact": (C.c_double, [P, D, C.c_double]),
            "orc_source": (C.c_double, [P, D, C.c_double]),
            "orc_lift": (None, [P, D, C.c_double, D, D, D]),
            "orc_jacobi_aa": (None, [C.c_int, C.c_double, C.c_double, D]),
            "orc_gj_nodes": (None, [C.c_int, C.c_double, D, D]),
            "orc_frac_lambda": (C.c_double, [C.c_double, C.c_int]),
            "orc_space_nodes": (None, [P, D, D]),
            "orc_space_analysis_pb": (None, [P, D]),
            "orc_ibeta": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_ibeta_inv": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_stable_jump": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_cheb": (None, [C.c_int, C.c_double, D, D]),
            "orc_cgl_nodes": (None, [C.c_int, D]),
            "orc_reconstruct": (None, [P, C.c_int, C.c_double, D, D, D]),
            "orc_eval": (None, [P, C.c_int, D, D, D, C.c_double, D, D, D]),
            "orc_residual": (C.c_double, [P, C.c_int, C.c_double, C.c_double, D, D, D, C.c_double]),
            "orc_nstar": (C.c_int, [C.c_int, C.c_double, C.c_double]),
            "orc_walk": (C.c_double, [P, C.POINTER(IntervalCtx), C.c_uint32, C.c_uint32, D,
                                      C.c_double, C.c_int, I, D]),
            "orc_node_eps": (C.c_double, [P, C.POINTER(IntervalCtx), C.c_int64, C.c_int]),
            "orc_iterate": (C.c_int, [P, C.c_int, C.c_double, C.c_double, C.c_int, D, C.c_int,
                                      C.c_int, C.c_double, D, D]),
            "orc_handoff": (None, [P, C.c_int, D, D]),
            "orc_aitken_omega": (C.c_double, [C.c_int64, D, D, C.c_double]),
            "orc_iterate_aitken": (C.c_int, [P, C.c_int, C.c_double, C.c_double, C.c_int, D, C.c_int, C.c_int, D, D,
                                             D]),
            "orc_solve": (None, [P, C.c_int, D, I, C.c_int, C.c_double, D, D, I]),
            "orc_solve_tangent": (None, [P, C.c_int, D, I, C.c_int, D, D, C.c_double, D, D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_int))


F_POLY3, F_SIN = 0, 1
EX_NONE, EX_SIN, EX_COSHALF, EX_POLY, EX_COSTHIRD, EX_SINPLUS = 0, 1, 2, 3, 4, 5
BC_ZERO, BC_LIFT, BC_RAW = 0, 1, 2
EST_RESIDUAL, EST_DIRECT = 0, 1
EX_FRAC_SIN, EX_FRAC_POLY = 6, 7
WALK_BALLS, WALK_FIXED, WALK_STABLE = 0, 1, 2
TIME_LGL, TIME_RADAU_LEFT, TIME_CHEB = 0, 1, 2


@dataclass
class Spec:
    """One problem instance, in the oracle's own terms."""
    dim: int
    n_space: int
    time_family: int = TIME_LGL
    n_ref: int = 20
    M: int = 64
    kappa: float = 1.0
    seed: int = 0
    instance: int = 0
    f_kind: int = F_POLY3
    f_coef: tuple = (0.0, 0.0, 0.0, -1.0)
    f_scale: float = 1.0
    ex_kind: int = EX_NONE
    ex_beta: float = 1.0
    n_threads: int = 1
    walk_mode: int = 0          # 0: balls inside Omega, 1: fixed radius (Lemma Xlocation)
    shell: float = 0.0           # 0: half the outermost node's distance to the boundary
    max_steps: int = 512
    n_sub: int = 4
    bc_kind: int = 0             # 0 g = 0; 1 lifted (Gordon-Hall); 2 g at absorption (direct estimator)
    estimator: int = 0           # 0 residual iteration; 1 direct estimator S_i (Eq. Phi_ast)
    alpha: float = 0.0           # 0: -kappa Delta; (0, 2): kappa (-Delta)^{alpha/2} (d = 1, walk_mode 2)
    basis: int = 0               # 0 Jacobi/Legendre; 1 Chebyshev in space and time (time_family 2)

    def struct(self) -> Problem:
        p = Problem()
        p.dim, p.n_space, p.time_family, p.n_ref = self.dim, self.n_space, self.time_family, self.n_ref
        p.M, p.kappa, p.seed, p.instance = self.M, self.kappa, self.seed, self.instance
        p.f_kind, p.f_scale, p.ex_kind, p.ex_beta = self.f_kind, self.f_scale, self.ex_kind, self.ex_beta
        for i, c in enumerate(self.f_coef):
            p.f_coef[i] = c
        p.n_threads = self.n_threads
        p.walk_mode, p.shell, p.max_steps, p.n_sub = self.walk_mode, self.shell, self.max_steps, self.n_sub
        p.bc_kind, p.estimator, p.alpha, p.basis = self.bc_kind, self.estimator, self.alpha, self.basis
        return p


# --------------------------------------------------------------------------- tables
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def jg11_nodes(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_jg11_nodes(n, _dp(x), _dp(w))
    return x, w


def lgl_nodes(M):
    x, w = np.zeros(M + 1), np.zeros(M + 1)
    lib().orc_lgl_nodes(M, _dp(x), _dp(w))
    return x, w


def radau_left_nodes(M):
    x, w = np.zeros(M + 1), np.zeros(M + 1)
    lib().orc_radau_left_nodes(M, _dp(x), _dp(w))
    return x, w


def cgl_nodes(M):
    xi = np.zeros(M + 1)
    lib().orc_cgl_nodes(M, _dp(xi))
    return xi, np.zeros(M + 1)


def cheb(m, x):
    """T_0..T_m at x and their second derivatives."""
    T, T2 = np.zeros(m + 1), np.zeros(m + 1)
    lib().orc_cheb(m, float(x), _dp(T), _dp(T2))
    return T, T2


def time_nodes(family, M):
    if family == TIME_CHEB:
        return cgl_nodes(M)
    return lgl_nodes(M) if family == TIME_LGL else radau_left_nodes(M)


def jacobi_aa(m, a, x):
    out = np.zeros(m + 1)
    lib().orc_jacobi_aa(m, float(a), float(x), _dp(out))
    return out


def gj_nodes(n, a):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gj_nodes(n, float(a), _dp(x), _dp(w))
    return x, w


def frac_lambda(alpha, p):
    return lib().orc_frac_lambda(float(alpha), int(p))


def space_analysis_spec(spec):
    A = np.zeros((spec.n_space, spec.n_space))
    p = spec.struct()
    lib().orc_space_analysis_pb(C.byref(p), _dp(A))
    return A


def ibeta(x, p, q):
    return lib().orc_ibeta(float(x), float(p), float(q))


def ibeta_inv(w, p, q):
    return lib().orc_ibeta_inv(float(w), float(p), float(q))


def stable_jump(r, alpha, omega):
    return lib().orc_stable_jump(float(r), float(alpha), float(omega))


def space_analysis(n):
    A = np.zeros((n, n))
    lib().orc_space_analysis(n, _dp(A))
    return A


def time_analysis(family, M):
    B = np.zeros((M + 1, M + 1))
    lib().orc_time_analysis(family, M, _dp(B))
    return B


def legendre(m, x):
    out = np.zeros(m + 1)
    lib().orc_legendre(m, float(x), _dp(out))
    return out


def jacobi11(m, x):
    out = np.zeros(m + 1)
    lib().orc_jacobi11(m, float(x), _dp(out))
    return out


def phi(m, x):
    out = np.zeros(m + 1)
    lib().orc_phi(m, float(x), _dp(out))
    return out


def nstar(n_ref, s, h):
    return lib().orc_nstar(n_ref, s, h)


# --------------------------------------------------------------------------- method
def n_nodes(spec: Spec) -> int:
    return spec.n_space ** spec.dim


def reconstruct(spec: Spec, Mt: int, h: float, U: np.ndarray):
    S = n_nodes(spec)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(Mt + 1, S)
    cu, ct = np.zeros((Mt + 1, S)), np.zeros((Mt + 1, S))
    p = spec.struct()
    lib().orc_reconstruct(C.byref(p), Mt, h, _dp(U), _dp(cu), _dp(ct))
    return cu, ct


def evaluate(spec: Spec, Mt: int, cu, ct, x, xi):
    """(u*, d_t u*, -Delta u*) at spatial point x and reference time xi."""
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    u, dt, ml = C.c_double(), C.c_double(), C.c_double()
    p = spec.struct()
    lib().orc_eval(C.byref(p), Mt, _dp(cu), _dp(ct), _dp(x), float(xi), C.byref(u), C.byref(dt), C.byref(ml))
    return u.value, dt.value, ml.value


def residual(spec: Spec, Mt, t0, h, cu, ct, x, tau):
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    p = spec.struct()
    return lib().orc_residual(C.byref(p), Mt, t0, h, _dp(cu), _dp(ct), _dp(x), tau)


def exact(spec: Spec, x, t):
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    p = spec.struct()
    return lib().orc_exact(C.byref(p), _dp(x), float(t))


def source(spec: Spec, x, t):
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    p = spec.struct()
    return lib().orc_source(C.byref(p), _dp(x), float(t))


def lift(spec: Spec, x, t):
    """(G, d_t G, Delta G) of the Gordon-Hall lifting of the boundary data at (x, t)."""
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    G, Gt, L = C.c_double(), C.c_double(), C.c_double()
    p = spec.struct()
    lib().orc_lift(C.byref(p), _dp(x), float(t), C.byref(G), C.byref(Gt), C.byref(L))
    return G.value, Gt.value, L.value


def walk(spec: Spec, x_start, t_node, nstar_, t0=0.0, h=1.0, Mt=0, cu=None, ct=None,
         node=0, sample=0, interval=0, iteration=1):
    """One walk: returns (Q, L, X_L).  With cu=None the integrand is 1."""
    x = np.ascontiguousarray(np.atleast_1d(x_start), dtype=np.float64)
    xe = np.zeros(spec.dim)
    keep = []
    if cu is not None:
        cu = np.ascontiguousarray(cu, dtype=np.float64); ct = np.ascontiguousarray(ct, dtype=np.float64)
        keep = [cu, ct]
        ic = IntervalCtx(Mt, t0, h, _dp(cu), _dp(ct), interval, iteration)
    else:
        ic = IntervalCtx(Mt, t0, h, None, None, interval, iteration)
    L = C.c_int()
    p = spec.struct()
    Q = lib().orc_walk(C.byref(p), C.byref(ic), node, sample, _dp(x), t_node, nstar_, C.byref(L), _dp(xe))
    del keep
    return Q, L.value, xe


def node_eps(spec: Spec, Mt, t0, h, cu, ct, j, l, interval=0, iteration=1):
    cu = np.ascontiguousarray(cu, dtype=np.float64); ct = np.ascontiguousarray(ct, dtype=np.float64)
    ic = IntervalCtx(Mt, t0, h, _dp(cu), _dp(ct), interval, iteration)
    p = spec.struct()
    return lib().orc_node_eps(C.byref(p), C.byref(ic), j, l)


def iterate(spec: Spec, interval, t0, t1, Mt, U, first_iteration=1, n_iter=1, tol=0.0):
    """Run residual iterations in place on U ((Mt+1) x S).  Returns (iters, max_eps, eps_last)."""
    S = n_nodes(spec)
    assert U.shape == (Mt + 1, S) and U.dtype == np.float64 and U.flags["C_CONTIGUOUS"]
    mx = np.zeros(n_iter)
    eps = np.zeros((Mt + 1, S))
    p = spec.struct()
    it = lib().orc_iterate(C.byref(p), interval, t0, t1, Mt, _dp(U), first_iteration, n_iter, tol,
                           _dp(mx), _dp(eps))
    return it, mx[:it], eps


def aitken_omega(r_prev, r_cur, omega_prev):
    a = np.ascontiguousarray(r_prev, dtype=np.float64).ravel()
    b = np.ascontiguousarray(r_cur, dtype=np.float64).ravel()
    return lib().orc_aitken_omega(a.size, _dp(a), _dp(b), float(omega_prev))


class AitkenState:
    """The previous residual and factor of an Aitken-relaxed iteration sequence."""
    def __init__(self, spec: Spec, Mt: int):
        self.eps_prev = np.zeros(Mt * n_nodes(spec))
        self.omega = C.c_double(1.0)


def iterate_aitken(spec: Spec, interval, t0, t1, Mt, U, state: AitkenState, first_iteration=1, n_iter=1):
    """Residual iterations with Aitken relaxation, in place on U; returns max |eps| per iteration."""
    S = n_nodes(spec)
    assert U.shape == (Mt + 1, S) and U.dtype == np.float64 and U.flags["C_CONTIGUOUS"]
    mx = np.zeros(n_iter)
    p = spec.struct()
    lib().orc_iterate_aitken(C.byref(p), interval, t0, t1, Mt, _dp(U), first_iteration, n_iter,
                             _dp(state.eps_prev), C.byref(state.omega), _dp(mx))
    return mx


def handoff(spec: Spec, Mt, U):
    S = n_nodes(spec)
    U = np.ascontiguousarray(U, dtype=np.float64)
    row = np.zeros(S)
    p = spec.struct()
    lib().orc_handoff(C.byref(p), Mt, _dp(U), _dp(row))
    return row


def solve(spec: Spec, t_breaks, degrees, K, u0, tol=0.0):
    """hp solve; returns (list of (Mt+1) x S nodal blocks, iterations per interval)."""
    S = n_nodes(spec)
    t = np.ascontiguousarray(t_breaks, dtype=np.float64)
    Mt = np.ascontiguousarray(degrees, dtype=np.int32)
    n_int = len(Mt)
    total = int(sum((m + 1) * S for m in Mt))
    out = np.zeros(total)
    its = np.zeros(n_int, dtype=np.int32)
    u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(S)
    p = spec.struct()
    lib().orc_solve(C.byref(p), n_int, _dp(t), _ip(Mt), K, tol, _dp(u0), _dp(out), _ip(its))
    blocks, off = [], 0
    for m in Mt:
        blocks.append(out[off: off + (m + 1) * S].reshape(m + 1, S))
        off += (m + 1) * S
    return blocks, its


def solve_tangent(spec: Spec, t_breaks, degrees, K, u0, du0, ds):
    S = n_nodes(spec)
    t = np.ascontiguousarray(t_breaks, dtype=np.float64)
    Mt = np.ascontiguousarray(degrees, dtype=np.int32)
    total = int(sum((m + 1) * S for m in Mt))
    out, dout = np.zeros(total), np.zeros(total)
    u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(S)
    du0 = np.ascontiguousarray(du0, dtype=np.float64).reshape(S)
    p = spec.struct()
    lib().orc_solve_tangent(C.byref(p), len(Mt), _dp(t), _ip(Mt), K, _dp(u0), _dp(du0), ds, _dp(out), _dp(dout))
    blocks, dblocks, off = [], [], 0
    for m in Mt:
        blocks.append(out[off: off + (m + 1) * S].reshape(m + 1, S))
        dblocks.append(dout[off: off + (m + 1) * S].reshape(m + 1, S))
        off += (m + 1) * S
    return blocks, dblocks


def space_nodes_grid(spec: Spec):
    """Coordinates of all spatial nodes, shape (S, d), x_1 fastest."""
    x, w = np.zeros(spec.n_space), np.zeros(spec.n_space)
    p = spec.struct()
    lib().orc_space_nodes(C.byref(p), _dp(x), _dp(w))
    grids = np.meshgrid(*([x] * spec.dim), indexing="ij")
    # linear index j = j1 + n*(j2 + n*(...)): x_1 fastest
    pts = np.stack([g.transpose(*reversed(range(spec.dim))).reshape(-1) for g in grids], axis=1)
    return pts


def exact_nodal(spec: Spec, t_breaks, degrees):
    """Exact solution at every node of every interval (list of blocks)."""
    pts = space_nodes_grid(spec)
    blocks = []
    for m, Mt in enumerate(degrees):
        t0, t1 = t_breaks[m], t_breaks[m + 1]
        xi, _ = time_nodes(spec.time_family, Mt)
        tt = t0 + (xi + 1.0) * 0.5 * (t1 - t0)
        blocks.append(np.array([[exact(spec, p, t) for p in pts] for t in tt]))
    return blocks
