"""Pins of the oracle's non-homogeneous boundary data and direct estimator.

Section 2.3 (remark on non-homogeneous boundary conditions): u = w + G with G a
lifting of the boundary data g; Section 2.2, Eq. Phi_ast: the direct estimator
S_i with the initial term u*^{n-1}(X, t_{n-1}) on walks that reach t_{n-1} and
the boundary term g(X_p, t_p) on walks that leave Omega.  Each test names the
mistake it is built to catch.
"""
import numpy as np
import pytest

from oracle import oracle as O

PI = np.pi


def _c4(x):
    return np.cos(PI * (np.asarray(x) - 0.3) / 3.0)


def _u_kind4(x, t, beta):
    return np.exp(-beta * t) * np.prod(_c4(x))


def _u_kind5(x, t, beta):
    return np.exp(-beta * t) * np.prod(np.sin(PI * np.asarray(x))) + 0.5 * t


@pytest.mark.parametrize("kind,d", [(4, 1), (4, 2), (5, 1), (5, 2)])
def test_sources_of_boundary_kinds_match_finite_differences(kind, d):
    """f_add = d_t u - kappa Delta u - f(u) of the closed forms with non-zero
    trace, against central differences of the closed form written here.
    Catches pi^2/3 for pi^2/9, a dropped 1/2 in d_t of t/2, or f(u) left out."""
    beta, kappa = 0.7, 0.4
    sp = O.Spec(dim=d, n_space=6, ex_kind=kind, ex_beta=beta, kappa=kappa, f_kind=O.F_SIN, f_scale=1.3)
    u = _u_kind4 if kind == 4 else _u_kind5
    rng = np.random.default_rng(kind * 10 + d)
    hh = 1e-4
    for _ in range(5):
        x = rng.uniform(-0.9, 0.9, d)
        t = rng.uniform(0.1, 2.0)
        ut = (u(x, t + hh, beta) - u(x, t - hh, beta)) / (2 * hh)
        lap = 0.0
        for e in range(d):
            dx = np.zeros(d); dx[e] = hh
            lap += (u(x + dx, t, beta) - 2 * u(x, t, beta) + u(x - dx, t, beta)) / hh ** 2
        want = ut - kappa * lap - 1.3 * np.sin(u(x, t, beta))
        assert O.source(sp, x, t) == pytest.approx(want, abs=2e-6)
        assert O.exact(sp, x, t) == pytest.approx(u(x, t, beta), rel=1e-14)


@pytest.mark.parametrize("kind", [4, 5])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_lifting_equals_boundary_data_on_every_face(kind, d):
    """G = g on the boundary, from face values alone.  Catches blending factors
    (1 + x)/2 and (1 - x)/2 swapped, or a wrong inclusion-exclusion sign."""
    sp = O.Spec(dim=d, n_space=6, ex_kind=kind, ex_beta=0.3, bc_kind=O.BC_LIFT)
    rng = np.random.default_rng(d)
    for _ in range(12):
        x = rng.uniform(-1, 1, d)
        e = rng.integers(d)
        x[e] = rng.choice([-1.0, 1.0])
        t = rng.uniform(0, 3)
        G, _, _ = O.lift(sp, x, t)
        assert G == pytest.approx(O.exact(sp, x, t), abs=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_lifting_of_a_product_trace_has_the_closed_form(d):
    """For u = T(t) prod c(x_e) the Gordon-Hall interpolant of its trace is
    T (prod c - prod (c - c_b)), c_b the linear interpolant of c between the
    faces: the lifting written as a product, not as the oracle's sum over faces
    (c takes different values on opposite faces, so blending factors swapped
    between the faces fail here).  Kind 5's trace t/2 lifts to the constant t/2."""
    beta = 0.9
    sp4 = O.Spec(dim=d, n_space=6, ex_kind=4, ex_beta=beta, bc_kind=O.BC_LIFT)
    sp5 = O.Spec(dim=d, n_space=6, ex_kind=5, ex_beta=beta, bc_kind=O.BC_LIFT)
    rng = np.random.default_rng(7 + d)
    for _ in range(8):
        x = rng.uniform(-1, 1, d)
        t = rng.uniform(0, 2)
        c = _c4(x)
        cb = 0.5 * (1 - x) * _c4(-1.0) + 0.5 * (1 + x) * _c4(1.0)
        want = np.exp(-beta * t) * (np.prod(c) - np.prod(c - cb))
        assert O.lift(sp4, x, t)[0] == pytest.approx(want, abs=1e-15)
        G5, Gt5, L5 = O.lift(sp5, x, t)
        assert G5 == pytest.approx(0.5 * t, abs=1e-15) and Gt5 == pytest.approx(0.5, abs=1e-15)
        assert abs(L5) < 1e-14
    # homogeneous kinds and bc_kind 0 lift to zero
    assert O.lift(O.Spec(dim=d, n_space=6, ex_kind=1, bc_kind=O.BC_LIFT), np.full(d, 0.3), 1.0) == (0.0, 0.0, 0.0)
    assert O.lift(O.Spec(dim=d, n_space=6, ex_kind=4), np.full(d, 0.3), 1.0) == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("d", [1, 2])
def test_lifting_derivatives_match_finite_differences(d):
    """d_t G and Delta G against central differences of G itself.  Catches the
    second derivative taken along the blended axes instead of the free ones."""
    sp = O.Spec(dim=d, n_space=6, ex_kind=4, ex_beta=0.6, bc_kind=O.BC_LIFT)
    rng = np.random.default_rng(3 + d)
    hh = 1e-4
    for _ in range(6):
        x = rng.uniform(-0.9, 0.9, d)
        t = rng.uniform(0.1, 2)
        G, Gt, lapG = O.lift(sp, x, t)
        Gt_fd = (O.lift(sp, x, t + hh)[0] - O.lift(sp, x, t - hh)[0]) / (2 * hh)
        lap_fd = 0.0
        for e in range(d):
            dx = np.zeros(d); dx[e] = hh
            lap_fd += (O.lift(sp, x + dx, t)[0] - 2 * G + O.lift(sp, x - dx, t)[0]) / hh ** 2
        assert Gt == pytest.approx(Gt_fd, abs=1e-8)
        assert lapG == pytest.approx(lap_fd, abs=2e-6)


def test_lifted_residual_iteration_reaches_the_closed_form():
    """The residual iteration on w = u - G with a nonlinear reaction f = s sin(u)
    (the lifted problem's f(w + G) and source), two left-Radau intervals: w + G
    at every node within 1e-6 of the closed form with non-zero boundary values.
    Catches f(w) for f(w + G), or d_t G / Delta G left out of the source."""
    sp = O.Spec(dim=1, n_space=12, ex_kind=4, ex_beta=0.5, f_kind=O.F_SIN, f_scale=1.0, kappa=0.5, M=2000,
                n_ref=20, bc_kind=O.BC_LIFT, time_family=O.TIME_RADAU_LEFT, n_threads=4)
    pts = O.space_nodes_grid(sp)
    u0 = np.array([O.exact(sp, p, 0.0) for p in pts])
    tb, deg = np.array([0.0, 0.5, 1.0]), [6, 6]
    blocks, _ = O.solve(sp, tb, deg, 8, u0)
    ex = O.exact_nodal(sp, tb, deg)
    for m in range(2):
        xi, _ = O.time_nodes(sp.time_family, deg[m])
        tt = tb[m] + (xi + 1) * 0.5 * (tb[m + 1] - tb[m])
        G = np.array([[O.lift(sp, p, t)[0] for p in pts] for t in tt])
        assert np.abs(blocks[m] + G - ex[m]).max() < 1e-6


@pytest.mark.parametrize("d,n", [(1, 10), (2, 8)])
def test_direct_estimator_one_step_expectation(d, n):
    """Eq. Phi_ast with N_* = 1 on a pure heat problem (f = 0, no source): a
    node whose full ball lies inside Omega takes one step of time s and ends
    sqrt(2 d kappa s) away in a uniform direction, so E[S] is the mean of u0
    over that sphere (computed here by quadrature over the circle).  Catches
    the terminal move left out (E[S] = u0(x)) or its radius without the factor d."""
    kappa = 0.5
    sp = O.Spec(dim=d, n_space=n, ex_kind=1, ex_beta=kappa * d * PI ** 2, f_coef=(0, 0, 0, 0), kappa=kappa,
                M=20000, n_ref=1, estimator=O.EST_DIRECT, time_family=O.TIME_LGL, n_threads=4)
    pts = O.space_nodes_grid(sp)
    u0 = np.prod(np.sin(PI * pts), axis=1)
    Mt, h = 2, 0.02
    U = np.tile(u0, (Mt + 1, 1)).copy()
    O.iterate(sp, 0, 0.0, h, Mt, U, 1, 1)
    xi, _ = O.lgl_nodes(Mt)
    th = np.linspace(0, 2 * PI, 4096, endpoint=False)
    checked = 0
    for l in (1, 2):
        s = (xi[l] + 1) * 0.5 * h
        J = np.sqrt(2 * d * kappa * s)
        for j, p in enumerate(pts):
            if J > np.min(1 - np.abs(p)):
                continue
            if d == 1:
                vals = np.sin(PI * (p[0] + J * np.array([1.0, -1.0])))
            else:
                vals = np.sin(PI * (p[0] + J * np.cos(th))) * np.sin(PI * (p[1] + J * np.sin(th)))
            sd = vals.std() / np.sqrt(sp.M)
            assert abs(U[l, j] - vals.mean()) < 5 * sd + 1e-6, (l, j)
            checked += 1
    assert checked >= 8


def test_direct_estimator_boundary_term():
    """u = t/2 solves d_t u - Delta u = 1/2 with u(., 0) = 0 and boundary data
    g = t/2 (kind 5's trace and source with beta = pi^2, zero initial values).
    Per walk, S = (1/2) sum w_q + t_b/2 when absorbed at path time t_b and
    (1/2) sum w_q + u0(X) = (1/2) sum w_q on reaching t_0 = 0; the quadrature sum
    is the elapsed time in expectation, so E[S] = t/2 exactly: the mean is t/2
    up to the roulette's noise.  Catches the boundary term left out (low by
    E[t_b/2; absorbed], up to 0.2 here) or t_b taken as t_{n,l}."""
    sp = O.Spec(dim=1, n_space=10, ex_kind=5, ex_beta=PI ** 2, f_coef=(0, 0, 0, 0), kappa=1.0, M=20000,
                n_ref=32, estimator=O.EST_DIRECT, bc_kind=O.BC_RAW, time_family=O.TIME_LGL, n_threads=4)
    Mt, h = 3, 0.5
    U = np.zeros((Mt + 1, 10))
    O.iterate(sp, 0, 0.0, h, Mt, U, 1, 1)
    xi, _ = O.lgl_nodes(Mt)
    tt = (xi + 1) * 0.5 * h
    err = np.abs(U - 0.5 * tt[:, None])[1:]
    assert err.max() < 2e-3, err.max()
