"""Pins of the oracle's fractional-Laplacian path (Section 4, Ex. 2 and 3; the
remark on generalised Jacobi functions): the (a,a) Jacobi tables, the basis'
fractional eigenvalues, the alpha-stable walk and the fractional examples.
Each test names the mistake it is built to catch."""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy import integrate

from oracle import oracle as O


def _fraclap(u, x, alpha):
    """(-Delta)^{alpha/2} u(x) in 1-D from the hypersingular integral with the
    standard constant, by adaptive quadrature (u zero outside (-1, 1))."""
    C = alpha * 2 ** (alpha - 1) * sps.gamma((1 + alpha) / 2) / (np.sqrt(np.pi) * sps.gamma(1 - alpha / 2))
    f = lambda y: (2 * u(x) - u(x + y) - u(x - y)) / y ** (1 + alpha)
    b1, b2 = sorted((abs(1 - x), abs(1 + x)))
    tot = 0.0
    for lo, hi in ((0, b1), (b1, b2), (b2, np.inf)):
        tot += integrate.quad(f, lo, hi, limit=400, epsabs=1e-13)[0]
    return C * tot


@pytest.mark.parametrize("a", [0.2, 0.6, 0.95])
def test_jacobi_aa_tables_match_scipy(a):
    """Gauss-Jacobi (a,a) nodes and weights and P_p^{(a,a)} against scipy.
    Catches a wrong P_1 = (a+1) x or a weight formula of the (1,1) case."""
    x, w = O.gj_nodes(10, a)
    xr, wr = sps.roots_jacobi(10, a, a)
    assert np.abs(x - xr).max() < 1e-14 and np.abs(w - wr).max() < 1e-13
    for z in (-0.8, 0.37):
        assert np.abs(O.jacobi_aa(8, a, z) - [sps.eval_jacobi(k, a, a, z) for k in range(9)]).max() < 1e-13


@pytest.mark.parametrize("alpha", [0.4, 1.3])
def test_fractional_analysis_inverts_the_basis(alpha):
    """The analysis matrix of the generalised Jacobi functions (1-x^2)^a P_p^{(a,a)}
    at the (a,a) nodes is the inverse of their nodal matrix.  Catches the
    weight (1-x^2)^{-a} or the norm gamma_p^{(a)} wrong."""
    a = alpha / 2
    sp = O.Spec(dim=1, n_space=9, alpha=alpha, walk_mode=2, n_sub=1)
    A = O.space_analysis_spec(sp)
    x = O.space_nodes_grid(sp)[:, 0]
    Phi = np.array([[(1 - xj * xj) ** a * sps.eval_jacobi(p, a, a, xj) for xj in x] for p in range(9)])
    assert np.abs(A @ Phi.T - np.eye(9)).max() < 1e-12


@pytest.mark.parametrize("alpha", [0.8, 1.4])
def test_fractional_eigenvalues_match_the_hypersingular_integral(alpha):
    """(-Delta)^{alpha/2} of (1-x^2)_+^a P_p^{(a,a)} computed by quadrature of the
    hypersingular integral equals the oracle's lam_p P_p^{(a,a)}, lam_p =
    Gamma(alpha+p+1)/p! (through its evaluation of a one-coefficient expansion).
    Catches the constant off by 2 or lam_p = (p+1)(p+2)."""
    a = alpha / 2
    sp = O.Spec(dim=1, n_space=4, alpha=alpha, walk_mode=2, n_sub=1)
    for p in range(3):
        cu = np.zeros((1, 4)); cu[0, p] = 1.0
        ct = np.zeros((1, 4))
        u = lambda z, p=p: (1 - z * z) ** a * sps.eval_jacobi(p, a, a, z) if abs(z) < 1 else 0.0
        for x in (-0.3, 0.55):
            _, _, op = O.evaluate(sp, 0, cu, ct, [x], 0.0)
            assert op == pytest.approx(_fraclap(u, x, alpha), abs=2e-7)


def test_incomplete_beta_and_its_inverse_match_scipy():
    """I_x(p, q) and its inverse against scipy (independent implementations).
    Catches a missing symmetry switch above x = 1/2 or p, q swapped."""
    for a in (0.2, 0.5, 0.9):
        for x in (1e-5, 0.2, 0.5, 0.77, 0.999):
            assert O.ibeta(x, 1 - a, a) == pytest.approx(sps.betainc(1 - a, a, x), rel=1e-13, abs=1e-15)
        for w in (1e-6, 0.1, 0.5, 0.9, 1 - 1e-6):
            assert O.ibeta_inv(w, 1 - a, a) == pytest.approx(sps.betaincinv(1 - a, a, w), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_stable_jump_follows_the_ball_exit_law(alpha):
    """The exit distance from a ball of radius r for the alpha-stable process
    started at its centre: P(J <= rho) = 1 - I_{r^2/rho^2}(a, 1-a) (the
    Blumenthal-Getoor-Ray law), so the jump at quantile omega satisfies
    I_{r^2/J^2}(a, 1-a) = 1 - omega (scipy's betainc; near omega = 0 the check
    itself loses digits to the law's steep density, hence 1e-9).  Catches
    U ~ Beta(1-a, a) used in place of Beta(a, 1-a)."""
    a = alpha / 2
    r = 0.013
    for w in (0.01, 0.3, 0.5, 0.8, 0.99):
        J = O.stable_jump(r, alpha, w)
        assert J >= r
        assert sps.betainc(a, 1 - a, (r / J) ** 2) == pytest.approx(1 - w, abs=1e-9)


@pytest.mark.parametrize("alpha,x0", [(0.6, 0.0), (1.2, 0.6)])
def test_stable_walk_mean_exit_time(alpha, x0):
    """The walk's quadrature of the integrand 1 is its exit time from (-1, 1);
    for the alpha-stable process E_x[tau] = (1-x^2)^{alpha/2} / (kappa Gamma(1+alpha))
    (the eigenvalue lam_0 = Gamma(1+alpha)).  The walk (fixed radius from
    Delta, ball-exit jumps, the mean-time clock, exit at the first point
    outside) must give it within 4 standard errors.  Catches the radius
    r = (kappa Delta Gamma(1+alpha))^{1/alpha} taken as sqrt(2 kappa Delta) or
    the direction word shared with the jump word."""
    kappa = 0.7
    sp = O.Spec(dim=1, n_space=6, alpha=alpha, walk_mode=2, n_sub=1, kappa=kappa, max_steps=100000)
    s, nstar = 8.0 / kappa, 2000
    Q = np.array([O.walk(sp, [x0], s, nstar, t0=0.0, h=s, sample=i)[0] for i in range(2000)])
    want = (1 - x0 * x0) ** (alpha / 2) / (kappa * math.gamma(1 + alpha))
    assert abs(Q.mean() - want) < 4 * Q.std() / np.sqrt(len(Q)), (Q.mean(), want)


@pytest.mark.parametrize("alpha", [0.4, 1.5])
def test_fractional_source_matches_quadrature(alpha):
    """The source of Ex. 2's exact solution (1-x^2)_+^a sin(x) e^{cos t}/(1+t^2),
    f_add = d_t u + kappa (-Delta)^{alpha/2} u - f(u) with f = u - u^3, against
    the hypersingular integral by quadrature and a central difference in t.
    Catches a wrong series of sin(x) in P^{(a,a)} or a wrong T'(t)."""
    a, kappa = alpha / 2, 0.8
    sp = O.Spec(dim=1, n_space=6, alpha=alpha, walk_mode=2, n_sub=1, ex_kind=O.EX_FRAC_SIN, kappa=kappa,
                f_coef=(0, 1.0, 0, -1.0))
    T = lambda t: np.exp(np.cos(t)) / (1 + t * t)
    for x, t in ((-0.4, 0.3), (0.7, 1.7)):
        u = lambda z, t=t: (1 - z * z) ** a * np.sin(z) * T(t) if abs(z) < 1 else 0.0
        ut = (u(x, t + 1e-5) - u(x, t - 1e-5)) / 2e-5
        uv = u(x)
        want = ut + kappa * _fraclap(u, x, alpha) - (uv - uv ** 3)
        assert O.source(sp, [x], t) == pytest.approx(want, abs=1e-6)
        assert O.exact(sp, [x], t) == pytest.approx(uv, rel=1e-14)


@pytest.mark.parametrize("alpha", [0.4, 1.5])
def test_fractional_fixed_point(alpha):
    """u = (1+t)(1-x^2)^a (1 + P_1^{(a,a)}/2) lies in the approximation space, so
    its residual vanishes and one iteration from its nodal values gives eps = 0
    to rounding, for any walk.  Catches a residual term with the wrong sign or
    the Laplacian's eigenvalues in place of the fractional ones."""
    sp = O.Spec(dim=1, n_space=10, ex_kind=O.EX_FRAC_POLY, alpha=alpha, walk_mode=2, n_ref=20, M=300,
                f_coef=(0, 1.0, 0, -1.0), n_sub=1, time_family=O.TIME_LGL, n_threads=4)
    x = O.space_nodes_grid(sp)[:, 0]
    Mt, h = 4, 0.5
    xi, _ = O.lgl_nodes(Mt)
    U = np.array([[O.exact(sp, [xx], t) for xx in x] for t in (xi + 1) * 0.5 * h])
    _, mx, _ = O.iterate(sp, 0, 0.0, h, Mt, U, 1, 1)
    assert mx[0] < 1e-12


def test_fractional_iteration_converges_to_ex2_solution():
    """Ex. 2's problem (alpha = 1.2, f = u - u^3, one interval h = 0.5, 8 JG(a,a)
    nodes, degree 5 in time): the residual iteration contracts and reaches the
    closed form to the discretisation and sampling error (3e-4 here)."""
    sp = O.Spec(dim=1, n_space=8, ex_kind=O.EX_FRAC_SIN, alpha=1.2, walk_mode=2, n_ref=20, M=600,
                f_coef=(0, 1.0, 0, -1.0), n_sub=1, time_family=O.TIME_LGL, n_threads=4)
    x = O.space_nodes_grid(sp)[:, 0]
    u0 = np.array([O.exact(sp, [xx], 0.0) for xx in x])
    Mt, h = 5, 0.5
    U = np.tile(u0, (Mt + 1, 1)).copy()
    _, mx, _ = O.iterate(sp, 0, 0.0, h, Mt, U, 1, 10)
    assert mx[-1] < 0.05 * mx[0]
    xi, _ = O.lgl_nodes(Mt)
    ex = np.array([[O.exact(sp, [xx], t) for xx in x] for t in (xi + 1) * 0.5 * h])
    assert np.abs(U - ex).max() < 3e-4, np.abs(U - ex).max()
