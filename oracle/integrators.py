"""Exponential integrators on the ADR test problem of Sec. 4.2 (oracle).

Problem (Sec. 4.2): u_t = eps Laplace(u) + alpha (d_1 + d_2 + d_3) u + g(t, u)
on [0,1]^3, homogeneous Dirichlet, u_0 = 64 prod x_mu (1 - x_mu),
g = 1/(1 + u^2) + Psi(t, x) with Psi chosen so that u = e^t u_0 solves it.
With u_0 quadratic in each direction, second-order central differences are
exact on it, so the semidiscrete solution at the grid points is e^t u_0 and
the measured error is the time error alone.

Schemes (Sec. 2): exponential Euler eq. (expEullc),
u_{n+1} = exp(tau K) u_n + tau phi_1(tau K) g(t_n, u_n);
ETD2RK eq. (ETD2RKlc): u_n2 = exp(tau K) u_n + tau phi_1(tau K) g_n,
u_{n+1} = u_n2 + tau phi_2(tau K) (g(t_n + tau, u_n2) - g_n), evaluated as one
linear combination per stage.  Each phi-action by the oracle's Taylor action.
"""
from __future__ import annotations

import numpy as np

from .taylor_action import lincomb as ta_lincomb


def adr_grid(n: int):
    x = np.arange(1, n + 1) / (n + 1.0)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    return X1, X2, X3


def adr_u0(n: int) -> np.ndarray:
    X1, X2, X3 = adr_grid(n)
    return 64.0 * X1 * (1 - X1) * X2 * (1 - X2) * X3 * (1 - X3)


def adr_g(t: float, U: np.ndarray, n: int, eps: float, alpha: float) -> np.ndarray:
    """1/(1 + u^2) + Psi(t, x), Psi = d_t w - eps Lap(w) - alpha sum d_mu w - 1/(1+w^2)
    for w = e^t u_0 (derivatives of u_0 in closed form)."""
    X1, X2, X3 = adr_grid(n)
    q = [X1 * (1 - X1), X2 * (1 - X2), X3 * (1 - X3)]
    dq = [1 - 2 * X1, 1 - 2 * X2, 1 - 2 * X3]
    u0 = 64.0 * q[0] * q[1] * q[2]
    lap = -128.0 * (q[1] * q[2] + q[0] * q[2] + q[0] * q[1])
    grad = 64.0 * (dq[0] * q[1] * q[2] + q[0] * dq[1] * q[2] + q[0] * q[1] * dq[2])
    w = np.exp(t) * u0
    psi = np.exp(t) * (u0 - eps * lap - alpha * grad) - 1.0 / (1.0 + w * w)
    return 1.0 / (1.0 + U * U) + psi


def integrate(A, n: int, eps: float, alpha: float, T: float, steps: int, scheme: str = "expeuler"):
    """Returns the final state (flattened, column-major) after `steps` steps."""
    tau = T / steps
    u = np.reshape(adr_u0(n), -1, order="F")
    t = 0.0
    for _ in range(steps):
        U = np.reshape(u, (n, n, n), order="F")
        g = np.reshape(adr_g(t, U, n, eps, alpha), -1, order="F")
        if scheme == "expeuler":
            u = ta_lincomb(A, tau, [u, tau * g])
        else:
            u2 = ta_lincomb(A, tau, [u, tau * g])
            g2 = np.reshape(adr_g(t + tau, np.reshape(u2, (n, n, n), order="F"), n, eps, alpha), -1,
                            order="F")
            u = ta_lincomb(A, tau, [u, tau * g, tau * (g2 - g)])
        t += tau
    return u


def relative_error(u: np.ndarray, n: int, T: float) -> float:
    ex = np.reshape(np.exp(T) * adr_u0(n), -1, order="F")
    return float(np.abs(u - ex).max() / np.abs(ex).max())
