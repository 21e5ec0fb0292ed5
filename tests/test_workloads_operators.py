"""The seeded workloads' operators against what their definitions fix:
Chebyshev collocation differentiates polynomials exactly, central
differences are exact on low-degree polynomials, and the Neumann Laplacian
annihilates constants."""
import numpy as np

import workloads as wk


def test_chebyshev_d2_is_exact_on_polynomials_vanishing_at_the_ends():
    n = 12
    D2 = wk.cheb_d2_dirichlet(n)
    N = n + 1
    x = np.cos(np.pi * np.arange(1, N) / N)           # interior Gauss-Lobatto points
    for j in range(0, N - 1):                         # u = (1 - x^2) x^j, degree <= N
        u = (1 - x ** 2) * x ** j
        d2 = (j * (j - 1) * x ** (j - 2) if j >= 2 else 0.0) - (j + 2) * (j + 1) * x ** j
        assert np.max(np.abs(D2 @ u - d2)) < 1e-9 * max(1.0, np.max(np.abs(d2)))
    # its eigenvalues are real and negative
    ev = np.linalg.eigvals(D2)
    assert np.max(np.abs(ev.imag)) < 1e-8 * np.max(np.abs(ev)) and np.all(ev.real < 0)


def test_dirichlet_adr_is_exact_on_a_quadratic():
    n, eps, alpha, react = 19, 0.7, -3.0, 2.0
    A = wk.fd_adr_dirichlet(n, eps, alpha, react)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    u = x * (1 - x)                                    # zero at both boundaries
    exact = eps * (-2.0) + alpha * (1 - 2 * x) + react * u
    assert np.max(np.abs(A @ u - exact)) < 1e-10
    # advection enters as the super-diagonal +alpha / 2h
    assert np.isclose(A[0, 1] - A[1, 0], alpha / h)


def test_neumann_laplacian_annihilates_constants_and_is_exact_inside():
    n, coef, react = 17, 0.3, -1.5
    A = wk.fd_laplacian_neumann(n, coef, react)
    assert np.allclose(A @ np.ones(n), react)
    h = 1.0 / (n - 1)
    x = h * np.arange(n)
    u = x ** 3 - 2 * x ** 2
    inner = (A @ u)[1:-1]
    assert np.max(np.abs(inner - (coef * (6 * x - 4) + react * u)[1:-1])) < 1e-9
