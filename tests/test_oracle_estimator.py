"""Pins of the oracle's walk estimator, hand-off, hp chaining, reaction and
manufactured sources, against facts that do not come from the oracle: the
divergence or contraction of the residual iteration itself, closed-form
solutions, numpy's Legendre interpolation, the midpoint rule and finite
differences of the closed forms.  CPU only.

Each test names the plausible mistake it is built to catch."""
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

NT = os.cpu_count() or 1


def _manufactured_1d(O, n, Mt, family, n_ref, M, walk):
    """u = e^{-t} sin(pi x), f = -u^3 + f_add (the 1-D single-interval workload's problem)."""
    return O.Spec(dim=1, n_space=n, time_family=family, M=M, n_ref=n_ref, f_coef=(0, 0, 0, -1.0),
                  ex_kind=O.EX_SIN, ex_beta=1.0, walk_mode=walk, n_threads=NT)


def _iterate(O, spec, Mt, h, K):
    pts = O.space_nodes_grid(spec)
    U = np.tile(np.sin(np.pi * pts[:, 0]), (Mt + 1, 1)).copy()
    _, mx, _ = O.iterate(spec, 0, 0.0, h, Mt, U, 1, K)
    return mx, U


# ----------------------------------------------------------------- the estimator reading
def test_literal_walk_diverges_at_single_interval_workload_shape(O):
    """Section 2.2 prints a fixed-radius walk with the integrand taken at the step
    centres (Lemma Xlocation, Eqs. indexL, interIQ).  At the 1-D single-interval
    workload's degrees (14 JG(1,1) nodes, left-Radau degree 15, h = 1) and
    N_* = 20 that rule makes the residual iteration diverge: its q = 0 term weights
    the node's own residual by Delta, which amplifies the high spectral modes like
    an explicit Euler step with Delta lambda_max >> 2.  The inside-ball walk
    (Green-function points, sub-step times) contracts on the same problem.  Catches:
    an oracle whose two walks were swapped, or whose inside-ball walk regressed to
    the centre-point rule."""
    lit, _ = _iterate(O, _manufactured_1d(O, 14, 15, 1, 20, 1024, walk=1), 15, 1.0, 4)
    assert lit[3] > 100.0 * lit[0], lit
    ball, _ = _iterate(O, _manufactured_1d(O, 14, 15, 1, 20, 1024, walk=0), 15, 1.0, 8)
    assert ball[7] < ball[0] / 10.0, ball


def test_both_walks_contract_on_a_small_problem(O):
    """Where Delta lambda_max is small (6 nodes, left-Radau degree 6, h = 0.5, N_* = 20) the
    literal walk contracts too, so the divergence above is the rule meeting high
    degrees, not an error of the literal walk's code.  Catches: a literal walk that
    diverges everywhere (e.g. a sign error in its quadrature)."""
    lit, _ = _iterate(O, _manufactured_1d(O, 6, 6, 1, 20, 512, walk=1), 6, 0.5, 6)
    assert lit[5] < lit[0] / 5.0, lit
    ball, _ = _iterate(O, _manufactured_1d(O, 6, 6, 1, 20, 512, walk=0), 6, 0.5, 6)
    assert ball[5] < lit[5], (ball, lit)


def test_both_walks_reach_the_closed_form_where_both_are_stable(O):
    """On the small problem both estimators converge to the manufactured solution
    within their consistency errors: the inside-ball walk near the spatial
    resolution floor of 6 nodes (~1e-4), the centre-point walk within its O(Delta)
    time-quadrature bias (~7e-4 at N_* = 20).  Their fixed points therefore agree to
    that accuracy.  Catches: an inside-ball walk whose expectation is not the
    Feynman-Kac integral (a wrong ball weight or Green law would move its fixed
    point away from the literal walk's)."""
    Mt, h = 6, 0.5
    errs, Us = {}, {}
    for walk in (0, 1):
        spec = _manufactured_1d(O, 6, Mt, 0, 20, 512, walk)
        _, U = _iterate(O, spec, Mt, h, 30)
        ex = O.exact_nodal(spec, [0.0, h], [Mt])[0]
        errs[walk], Us[walk] = np.abs(U - ex).max(), U
    assert errs[0] < 5e-4, errs
    assert errs[1] < 3e-3, errs
    assert np.abs(Us[0] - Us[1]).max() < 3e-3


@pytest.mark.parametrize("dim", [1, 2])
def test_sub_step_times_follow_the_midpoint_rule(O, dim):
    """The inside-ball walk evaluates each full step at one of its n_sub sub-step
    midpoints tau_m = t_{n,l} - (m + 1/2) delta, drawn uniformly, with weight Delta
    (the last step takes the sub-points still ahead).  With full balls only (kappa
    so small that J << dist) and u* = L_2(xi(t)) phi_0(x), the residual is
    -d_t u* (+ kappa Delta u* ~ 1e-6), linear in t, so E[Q] is the composite midpoint
    rule of a linear integrand: exactly -(u*(x0, t_{n,l}) - u*(x0, t_{n-1})).
    The walk of the time-dependent problem runs backward from t_{n,l}.  Catches:
    tau = t - m delta (left points: bias delta/2 x 8.4 = 0.37 here), tau = t - (m+1)
    delta, a last step that ignores the sub-points ahead.  (Forward time visits the
    same set of times; the lattice test below separates it.)"""
    spec = O.Spec(dim=dim, n_space=3, f_coef=(0, 0, 0, 0), ex_kind=O.EX_NONE, walk_mode=0, shell=1e-5,
                  max_steps=64, kappa=1e-8, n_sub=4)
    Mt, h, t_node, nstar = 2, 1.0, 0.7, 2
    S = 3 ** dim
    cu = np.zeros((Mt + 1, S))
    cu[2, 0] = 1.0                                  # L_2(xi) phi_0(x_1) phi_0(x_2) ...
    ct = np.zeros((Mt + 1, S))
    d = npleg.legder(np.eye(Mt + 1)[2]) * (2.0 / h)  # d/dt L_2(xi(t)) in the Legendre basis
    ct[: len(d), 0] = d
    x0 = np.zeros(dim)
    n = 4000
    Q = np.array([O.walk(spec, x0, t_node, nstar, t0=0.0, h=h, Mt=Mt, cu=cu, ct=ct, sample=i)[0]
                  for i in range(n)])
    xi_node, xi_0 = 2.0 * t_node / h - 1.0, -1.0
    ref = -(npleg.legval(xi_node, np.eye(3)[2]) - npleg.legval(xi_0, np.eye(3)[2]))
    assert abs(Q.mean() - ref) < 4.0 * Q.std() / np.sqrt(n) + 1e-4, (Q.mean(), ref)


def _phi_poly(p):
    """phi_p = 2(p+1)/(2p+3) (L_p - L_{p+2}) as a numpy polynomial (Section 2.3)."""
    from numpy.polynomial import polynomial as P
    c = np.zeros(p + 3)
    c[p], c[p + 2] = 1.0, -1.0
    return P.Polynomial(npleg.leg2poly(c)) * (2.0 * (p + 1) / (2 * p + 3))


def _lattice_expected_q(p, qt, kappa, h, t_node, nstar, G, x0, backward=True):
    """Exact E[Q] of the 1-D inside-ball walk when every ball is a full one (radius
    J = sqrt(2 kappa Delta)): the centres run on the lattice x0 + k J with steps +-J;
    at step q the term is Delta r(Y, tau_m) with Y = X_q + J v theta (v of density
    2(1 - v), theta = +-1) and m uniform among the step's G sub-points.  For
    u* = L_qt(xi(t)) phi_p(x), f = 0 and no source, r = -d_t u* + kappa Delta u*,
    whose Y-expectation follows from the moments E[v^k] = 2/((k+1)(k+2))."""
    from numpy.polynomial import polynomial as P
    delta = t_node / nstar
    J = np.sqrt(2.0 * kappa * delta)
    sub = delta / G
    ph = _phi_poly(p)
    lap = ph.deriv(2)
    Lq = P.Polynomial(npleg.leg2poly(np.eye(qt + 1)[qt]))
    dLq = Lq.deriv()

    def e_y(poly, x):
        c = poly(P.Polynomial([x, 1.0])).coef          # poly(x + z) in powers of z
        return sum(c[k] * J ** k * 2.0 / ((k + 1) * (k + 2)) for k in range(0, len(c), 2))

    prob, EQ = {0: 1.0}, 0.0
    for q in range(nstar):
        for k, pr in prob.items():
            x = x0 + k * J
            e_ph, e_lap = e_y(ph, x), e_y(lap, x)
            acc = 0.0
            for g in range(G):
                m = q * G + g
                tau = t_node - (m + 0.5) * sub if backward else (m + 0.5) * sub
                xi = 2.0 * tau / h - 1.0
                acc += -(2.0 / h) * dLq(xi) * e_ph + kappa * Lq(xi) * e_lap
            EQ += pr * delta * acc / G
        nxt = {}
        for k, pr in prob.items():
            for dk in (-1, 1):
                nxt[k + dk] = nxt.get(k + dk, 0.0) + 0.5 * pr
        prob = nxt
    return EQ


@pytest.mark.parametrize("p", [0, 2])
def test_walk_expectation_matches_exact_lattice_chain(O, p):
    """With full balls only (x0 = 0.1, J = 0.08, 10 steps: no centre comes within J
    of the boundary) the 1-D inside-ball walk's centres form a lattice chain, so
    E[Q] is a finite sum computable exactly from polynomial moments.  Position and
    path time are coupled (the spread of X_q grows while tau runs from t_{n,l} down
    to t_{n-1}), so this pins the direction of path time (reading 6) together with
    the step weights and the sub-point times.  Catches: forward path time (1.2485
    instead of 1.1864 for p = 0, 78 standard errors away).  (The Green radial law
    moves E[Q] here by under two standard errors; the Dynkin tests pin it.)"""
    kappa, h, t_node, nstar, G, x0, qt = 0.0457, 1.0, 0.7, 10, 4, 0.1, 2
    ref = _lattice_expected_q(p, qt, kappa, h, t_node, nstar, G, x0)
    spec = O.Spec(dim=1, n_space=3, f_coef=(0, 0, 0, 0), ex_kind=O.EX_NONE, walk_mode=0, shell=1e-5,
                  max_steps=64, kappa=kappa, n_sub=G)
    cu = np.zeros((qt + 1, 3))
    cu[qt, p] = 1.0
    ct = np.zeros((qt + 1, 3))
    d = npleg.legder(np.eye(qt + 1)[qt]) * (2.0 / h)
    ct[: len(d), p] = d
    n = 20000
    Q = np.array([O.walk(spec, np.array([x0]), t_node, nstar, t0=0.0, h=h, Mt=qt, cu=cu, ct=ct, sample=i)[0]
                  for i in range(n)])
    assert abs(Q.mean() - ref) < 4.0 * Q.std() / np.sqrt(n), (Q.mean(), ref)
    assert abs(_lattice_expected_q(p, qt, kappa, h, t_node, nstar, G, x0, backward=False) - ref) > \
        20.0 * Q.std() / np.sqrt(n)


# ----------------------------------------------------------------- hand-off and hp chaining
@pytest.mark.parametrize("family,Mt", [(0, 4), (0, 9), (1, 3), (1, 8)])
def test_handoff_is_the_interpolant_at_the_interval_end(O, family, Mt):
    """Algorithm 1, Step 4: the next interval starts from u*(x_j, t_n), the time
    interpolant of the nodal values evaluated at xi = 1.  Compared with numpy's
    Legendre interpolation through the same (xi_k, U_k).  For left Radau xi = 1 is
    not a node, so this is a real evaluation.  Catches: evaluating at xi = -1
    (alternating L_q(-1) signs), dropping q = M_n, taking the last row for Radau."""
    rng = np.random.default_rng(Mt + 10 * family)
    spec = O.Spec(dim=1, n_space=5, time_family=family)
    U = rng.standard_normal((Mt + 1, 5))
    row = O.handoff(spec, Mt, U)
    xi, _ = O.time_nodes(family, Mt)
    ref = np.array([npleg.legval(1.0, npleg.legfit(xi, U[:, j], Mt)) for j in range(5)])
    assert np.abs(row - ref).max() < 1e-11 * (1.0 + np.abs(ref).max())
    if family == 0:
        assert np.abs(row - U[-1]).max() < 1e-11


def test_multi_interval_solve_tracks_the_closed_form(O):
    """Three left-Radau intervals chained by the hand-off (Algorithm 1, Step 4):
    every interval's nodal values match u = e^{-t} sin(pi x) to 1e-6 (measured
    6e-8).  Catches: a hand-off that passes row 0 (u at t_{n-1}) on instead of
    u*(t_n) -- an error of about 0.18 on the second interval -- or intervals that
    reuse the first interval's Philox streams."""
    spec = _manufactured_1d(O, 10, 6, 1, 80, 512, walk=0)
    t = [0.0, 0.2, 0.4, 0.6]
    deg = [6, 5, 6]
    pts = O.space_nodes_grid(spec)
    blocks, its = O.solve(spec, t, deg, 8, np.sin(np.pi * pts[:, 0]))
    ex = O.exact_nodal(spec, t, deg)
    for b, e in zip(blocks, ex):
        assert np.abs(b - e).max() < 1e-6, [np.abs(x - y).max() for x, y in zip(blocks, ex)]
    assert list(its) == [8, 8, 8]


# ----------------------------------------------------------------- reaction and sources
def test_reaction_matches_its_definition(O):
    """f(u) = s sin(u) and s (c0 + c1 u + c2 u^2 + c3 u^3), written out with numpy.
    Catches: sin(s u) for s sin(u), a dropped coefficient."""
    u = np.linspace(-2.0, 2.0, 17)
    sp = O.Spec(dim=1, n_space=3, f_kind=O.F_SIN, f_scale=1.7)
    p = sp.struct()
    L = O.lib()
    import ctypes as C
    got = np.array([L.orc_f(C.byref(p), float(v)) for v in u])
    assert np.abs(got - 1.7 * np.sin(u)).max() < 1e-15
    sp = O.Spec(dim=1, n_space=3, f_kind=O.F_POLY3, f_coef=(0.3, -1.1, 0.7, -1.0), f_scale=0.6)
    p = sp.struct()
    got = np.array([L.orc_f(C.byref(p), float(v)) for v in u])
    assert np.abs(got - 0.6 * (0.3 - 1.1 * u + 0.7 * u ** 2 - u ** 3)).max() < 1e-14


def _closed_form(kind, beta, x, t):
    """The workloads' manufactured solutions, written from their definitions."""
    if kind == 1:
        return np.exp(-beta * t) * np.prod(np.sin(np.pi * x))
    if kind == 2:
        return np.exp(-beta * t) * np.prod(np.cos(0.5 * np.pi * x))
    return (1.0 + t + t * t) * np.prod((1.0 - x * x) * (1.0 + x))


@pytest.mark.parametrize("dim,kind,f_kind,kappa", [(1, 1, 0, 1.0), (2, 1, 1, 1.0), (5, 2, 0, 1.0), (2, 2, 1, 0.3),
                                                   (1, 3, 1, 0.7), (2, 3, 0, 1.0)])
def test_manufactured_source_against_finite_differences(O, dim, kind, f_kind, kappa):
    """f_add = d_t u_ex - kappa Delta u_ex - f(u_ex), so that u_ex solves Eq.
    mainproblem with f(u) + f_add.  d_t and Delta by central differences of the
    closed form (step 1e-4, error ~1e-7 relative).  Catches: pi^2 for the
    half-cosine's pi^2/4, a missing dimension factor d, kappa left out, the
    reaction's sign."""
    rng = np.random.default_rng(dim * 10 + kind)
    beta = 0.1 if kind == 1 else 1.0
    sp = O.Spec(dim=dim, n_space=3, f_kind=f_kind, f_coef=(0.2, 0.5, 0.0, -1.0), f_scale=1.3, ex_kind=kind,
                ex_beta=beta, kappa=kappa)
    fr = (lambda u: 1.3 * np.sin(u)) if f_kind == 1 else (lambda u: 1.3 * (0.2 + 0.5 * u - u ** 3))
    e = 1e-4
    for _ in range(6):
        x = rng.uniform(-0.95, 0.95, dim)
        t = rng.uniform(0.1, 2.0)
        u = _closed_form(kind, beta, x, t)
        dt = (_closed_form(kind, beta, x, t + e) - _closed_form(kind, beta, x, t - e)) / (2 * e)
        lap = 0.0
        for a in range(dim):
            dx = np.zeros(dim)
            dx[a] = e
            lap += (_closed_form(kind, beta, x + dx, t) - 2 * u + _closed_form(kind, beta, x - dx, t)) / e ** 2
        ref = dt - kappa * lap - fr(u)
        assert abs(O.exact(sp, x, t) - u) < 1e-14
        assert abs(O.source(sp, x, t) - ref) < 2e-5 * (1.0 + abs(ref)), (O.source(sp, x, t), ref)


# ----------------------------------------------------------------- Aitken acceleration
@pytest.mark.parametrize("a", [-0.8, -0.3, 0.0, 0.4])
def test_aitken_factor_is_exact_for_a_linear_map(O, a):
    """For the residuals of a linear fixed-point map with one eigenvalue a,
    r_2 = a r_1 after a plain step, Aitken's factor is 1 / (1 - a), which puts the
    next iterate exactly on the fixed point.  Catches: the opposite sign, r_k in
    place of r_{k-1} in the numerator (a / (a - 1)), a missing omega_{k-1}."""
    rng = np.random.default_rng(5)
    r1 = rng.standard_normal(37)
    assert abs(O.aitken_omega(r1, a * r1, 1.0) - 1.0 / (1.0 - a)) < 1e-14
    assert abs(O.aitken_omega(r1, a * r1, 0.7) - min(max(0.7 / (1.0 - a), 0.5), 2.0)) < 1e-14


def test_aitken_factor_is_kept_in_range(O):
    """Outside [1/2, 2] the factor is clamped: a = 0.9 would give 10, a = -3 would give 1/4."""
    r1 = np.linspace(-1.0, 2.0, 11)
    assert O.aitken_omega(r1, 0.9 * r1, 1.0) == 2.0
    assert O.aitken_omega(r1, -3.0 * r1, 1.0) == 0.5
    assert O.aitken_omega(r1, r1, 0.8) == 0.8          # no change in the residual: keep the factor


def test_aitken_iteration_reaches_the_closed_form(O):
    """The relaxed iteration has the same fixed point: on the three-interval-sized
    1-D problem it reaches the closed form as the plain iteration does, and its
    first iteration (omega = 1) is the plain one bit for bit."""
    spec = _manufactured_1d(O, 10, 6, 1, 80, 512, walk=0)
    Mt, h = 6, 0.3
    pts = O.space_nodes_grid(spec)
    u0 = np.sin(np.pi * pts[:, 0])
    Ua = np.tile(u0, (Mt + 1, 1)).copy()
    Up = Ua.copy()
    st = O.AitkenState(spec, Mt)
    O.iterate_aitken(spec, 0, 0.0, h, Mt, Ua, st, 1, 1)
    O.iterate(spec, 0, 0.0, h, Mt, Up, 1, 1)
    assert np.array_equal(Ua, Up)
    O.iterate_aitken(spec, 0, 0.0, h, Mt, Ua, st, 2, 9)
    ex = O.exact_nodal(spec, [0.0, h], [Mt])[0]
    assert np.abs(Ua - ex).max() < 1e-6
    assert 0.5 <= st.omega.value <= 2.0
