"""Pins of the oracle's Chebyshev basis (the remark on quasi-linear
reconstruction after Algorithm 1): Chebyshev-Gauss-Lobatto points, the
discrete Chebyshev transform (DCT-I), the Dirichlet basis T_p - T_{p+2}, the
derivative identities and the hand-off.  Each test names the mistake it is
built to catch."""
import numpy as np
import pytest
import scipy.fft as sfft
from numpy.polynomial import chebyshev as Ch

from oracle import oracle as O


@pytest.mark.parametrize("M", [4, 8, 15])
def test_time_transform_is_the_dct(M):
    """The time analysis matrix applied to values at the CGL points is the DCT-I
    of scipy.fft (an FFT-based implementation), scaled by 1/(M c_q), and the
    result interpolates.  Catches the end values not halved or c_M = 1."""
    B = O.time_analysis(O.TIME_CHEB, M)
    xi, _ = O.cgl_nodes(M)
    assert np.allclose(xi, -np.cos(np.pi * np.arange(M + 1) / M), atol=1e-15)
    f = np.exp(np.sin(2 * xi)) + xi ** 3
    c = np.where((np.arange(M + 1) == 0) | (np.arange(M + 1) == M), 2.0, 1.0)
    ref = sfft.dct(f[::-1], type=1) / (M * c)   # scipy's points run cos(pi k / M), descending
    assert np.abs(B @ f - ref).max() < 1e-14
    assert np.abs(Ch.chebval(xi, B @ f) - f).max() < 1e-13


@pytest.mark.parametrize("n", [6, 9])
def test_space_analysis_inverts_the_dirichlet_basis(n):
    """At the interior CGL points, the analysis matrix inverts the nodal matrix
    of phi_p = T_p - T_{p+2} (numpy's Chebyshev series).  Catches the
    coefficient recurrence c_p = a_p + c_{p-2} dropped, or the DCT scale of the
    (n+2)-point transform."""
    sp = O.Spec(dim=1, n_space=n, basis=1, time_family=O.TIME_CHEB)
    A = O.space_analysis_spec(sp)
    x = O.space_nodes_grid(sp)[:, 0]
    assert np.allclose(x, -np.cos(np.pi * np.arange(1, n + 1) / (n + 1)), atol=1e-15)
    E = np.eye(n + 2)
    Phi = np.array([[Ch.chebval(xx, E[p]) - Ch.chebval(xx, E[p + 2]) for xx in x] for p in range(n)])
    assert np.abs(A @ Phi.T - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("dim", [1, 2])
def test_reconstruction_and_derivatives_match_numpy(dim):
    """Nodal values of a random space-time polynomial in the basis, reconstructed
    and evaluated at random points: u*, d_t u* and -Delta u* against numpy's
    Chebyshev series and chebder.  Catches the time-derivative identity
    (2/c_q) sum_{l>q, l+q odd} l c_l with a wrong factor or the Legendre one."""
    n, Mt, h = 6, 5, 0.7
    rng = np.random.default_rng(dim)
    sp = O.Spec(dim=dim, n_space=n, basis=1, time_family=O.TIME_CHEB)
    S = n ** dim
    C = rng.standard_normal((Mt + 1,) + (n,) * dim)   # [q][p_y][p_x] (x fastest)
    E = np.eye(n + 2)
    phi = lambda p, z: Ch.chebval(z, E[p]) - Ch.chebval(z, E[p + 2])
    d2phi = lambda p, z: Ch.chebval(z, Ch.chebder(E[p], 2)) - Ch.chebval(z, Ch.chebder(E[p + 2], 2))

    def field(x, xi):
        Tq = Ch.chebvander(np.atleast_1d(xi), Mt)[0]
        dTq = np.array([Ch.chebval(xi, Ch.chebder(np.eye(Mt + 1)[q])) for q in range(Mt + 1)])
        u = dt = ml = 0.0
        for q in range(Mt + 1):
            for idx in np.ndindex(*(n,) * dim):
                ps = idx[::-1]                       # p_x = ps[0]
                c = C[(q,) + idx]
                prod = np.prod([phi(ps[e], x[e]) for e in range(dim)])
                lap = sum(d2phi(ps[e], x[e]) * np.prod([phi(ps[f], x[f]) for f in range(dim) if f != e])
                          for e in range(dim))
                u += c * Tq[q] * prod
                dt += c * dTq[q] * prod * 2.0 / h
                ml -= c * Tq[q] * lap
        return u, dt, ml

    grid = O.space_nodes_grid(sp)
    xi, _ = O.cgl_nodes(Mt)
    U = np.array([[field(p, z)[0] for p in grid] for z in xi])
    cu, ct = O.reconstruct(sp, Mt, h, U)
    for _ in range(3):
        x = rng.uniform(-1, 1, dim)
        z = rng.uniform(-1, 1)
        got = O.evaluate(sp, Mt, cu, ct, x, z)
        want = field(x, z)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-10), (got, want)


def test_chebyshev_handoff_and_convergence():
    """The hand-off is the interval's interpolant at xi = 1, and the residual
    iteration in the Chebyshev basis reaches the 1-D closed form e^{-t} sin(pi x)
    (10 CGL points, degree 8 in time, h = 1, N_ref = 80) to 1e-6."""
    sp = O.Spec(dim=1, n_space=10, basis=1, time_family=O.TIME_CHEB, ex_kind=O.EX_SIN, ex_beta=1.0, M=1500,
                n_ref=80, f_coef=(0, 0, 0, -1.0), n_threads=4)
    x = O.space_nodes_grid(sp)[:, 0]
    u0 = np.sin(np.pi * x)
    Mt, h = 8, 1.0
    U = np.tile(u0, (Mt + 1, 1)).copy()
    _, mx, _ = O.iterate(sp, 0, 0.0, h, Mt, U, 1, 9)
    xi, _ = O.cgl_nodes(Mt)
    ex = np.exp(-((xi + 1) * 0.5 * h))[:, None] * u0[None, :]
    assert np.abs(U - ex).max() < 1e-6, (mx, np.abs(U - ex).max())
    B = O.time_analysis(O.TIME_CHEB, Mt)
    assert np.abs(O.handoff(sp, Mt, U) - Ch.chebval(1.0, B @ U)).max() < 1e-14
