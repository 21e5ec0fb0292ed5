"""Exponential Runge--Kutta integrators driving phi-actions (oracle).

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU leg, never by the product path.

Semidiscrete problems w' = K w + g(t, w) (Sec. 2, eq. ODE), K either one
Kronecker sum or block diagonal diag(K_1, K_2) of Kronecker sums (Sec. 4.4,
eq. ODE2): every phi-action is taken block by block with the oracle's Taylor
action (O3).

Schemes: the linear-combination form of the generic exponential Runge--Kutta
method (Sec. 2, eq. RK):
    u_ni    = exp(c_i tau K) u_n + c_i tau phi_1(c_i tau K) g_n
              + tau sum_{j=2}^{i-1} a_ij(tau K) d_nj,          2 <= i <= nu,
    u_{n+1} = exp(tau K) u_n + tau phi_1(tau K) g_n + tau sum_i b_i(tau K) d_ni,
    d_ni    = g(t_n + c_i tau, u_ni) - g(t_n, u_n),
with the reduced tableaux printed in the paper: exponential Euler (nu = 1),
ETD2RK (c_2 = 1, b_2 = phi_2), the third-order scheme eq. (expRK3s3), and the
fourth-order schemes eq. (expRK4s5) and eq. (expRK4s6).  Each a_ij and b_i is
a list of terms (coefficient, l, c) meaning coefficient * phi_l(c tau K); every
term is evaluated as its own phi-action, in the tableau's order, with none of
the call-saving assemblies of Sec. 4.4.

Problems:
* ADR (Sec. 4.2): u_t = eps Lap u + alpha (d_1 + d_2 + d_3) u + g(t, u) on
  [0,1]^3, homogeneous Dirichlet, u_0 = 64 prod x_mu (1 - x_mu),
  g = 1/(1 + u^2) + Psi(t, x) with Psi making u = e^t u_0 the solution.  With
  u_0 quadratic in each direction, second-order central differences are exact
  on it, so the semidiscrete solution at the grid points is e^t u_0 and the
  measured error is the time error alone.
* Allen--Cahn (Sec. 4.3): K = Lap + I / eps^2 (homogeneous Neumann),
  g(u) = -u^3 / eps^2.
* Brusselator (Sec. 4.4): K = diag(d_1 Lap - (b + 1) I, d_2 Lap), g(u, v) =
  (a + u^2 v, b u - u^2 v).
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

from .taylor_action import lincomb as ta_lincomb

# ---------------------------------------------------------------------------
# reduced tableaux of eq. (RK): stages (i, c_i, {j: terms}) and weights {i: terms}

Terms = List[Tuple[float, int, float]]


def _exprk3():
    c2, c3 = 0.25, 0.5                               # c_3 = 2 c_2 = 1/2
    gam = (3 * c3 - 2) * c3 / ((2 - 3 * c2) * c2)    # -4/5
    den = gam * c2 + c3
    stages = [(2, c2, {}),
              (3, c3, {2: [(gam * c2, 2, c2), (c3 * c3 / c2, 2, c3)]})]
    b = {2: [(gam / den, 2, 1.0)], 3: [(1.0 / den, 2, 1.0)]}
    return stages, b


def _exprk4s5():
    a52 = [(0.5, 2, 0.5), (-1.0, 3, 1.0), (0.25, 2, 1.0), (-0.5, 3, 0.5)]
    a54 = [(0.25, 2, 0.5)] + [(-w, l, c) for (w, l, c) in a52]
    stages = [(2, 0.5, {}),
              (3, 0.5, {2: [(1.0, 2, 0.5)]}),
              (4, 1.0, {2: [(1.0, 2, 1.0)], 3: [(1.0, 2, 1.0)]}),
              (5, 0.5, {2: a52, 3: list(a52), 4: a54})]
    b = {4: [(-1.0, 2, 1.0), (4.0, 3, 1.0)], 5: [(4.0, 2, 1.0), (-8.0, 3, 1.0)]}
    return stages, b


def _exprk4s6(c2=1.0 / 3, c3=1.0 / 3, c4=2.0 / 3, c5=0.5):
    c6 = (4 * c5 - 3) / (6 * c5 - 4)

    def a3(ci):
        return [(c4 * ci ** 2 / (c3 * (c4 - c3)), 2, ci), (2 * ci ** 3 / (c3 * (c3 - c4)), 3, ci)]

    def a4(ci):
        return [(c3 * ci ** 2 / (c4 * (c3 - c4)), 2, ci), (2 * ci ** 3 / (c4 * (c4 - c3)), 3, ci)]

    stages = [(2, c2, {}),
              (3, c3, {2: [(c3 * c3 / c2, 2, c3)]}),
              (4, c4, {2: [(c4 * c4 / c2, 2, c4)]}),
              (5, c5, {3: a3(c5), 4: a4(c5)}),
              (6, c6, {3: a3(c6), 4: a4(c6)})]
    b = {5: [(c6 / (c5 * (c6 - c5)), 2, 1.0), (2.0 / (c5 * (c5 - c6)), 3, 1.0)],
         6: [(c5 / (c6 * (c5 - c6)), 2, 1.0), (2.0 / (c6 * (c6 - c5)), 3, 1.0)]}
    return stages, b


TABLEAUX: Dict[str, Tuple[list, Dict[int, Terms]]] = {
    "expeuler": ([], {}),
    "etd2rk": ([(2, 1.0, {})], {2: [(1.0, 2, 1.0)]}),
    "exprk3": _exprk3(),
    "exprk4s5": _exprk4s5(),
    "exprk4s6": _exprk4s6(),
}

ORDER = {"expeuler": 1, "etd2rk": 2, "exprk3": 3, "exprk4s5": 4, "exprk4s6": 4}


# ---------------------------------------------------------------------------
# phi-actions of a block-diagonal K (blocks: list of [A_1, ..., A_d])

def _sizes(blocks) -> List[int]:
    return [int(np.prod([a.shape[0] for a in A])) for A in blocks]


def lc(blocks, tau: float, vs: Sequence, c: float = 1.0) -> np.ndarray:
    """exp(c tau K) v_0 + sum_l c^l phi_l(c tau K) v_l, block by block."""
    out, off = [], 0
    for A, N in zip(blocks, _sizes(blocks)):
        seg = [None if v is None else v[off:off + N] for v in vs]
        out.append(ta_lincomb(A, tau, seg, c))
        off += N
    return np.concatenate(out)


def phi(blocks, tau: float, ell: int, w: np.ndarray) -> np.ndarray:
    """phi_ell(tau K) w."""
    vs = [None] * ell + [w]
    return lc(blocks, tau, vs)


def exprk_step(blocks, g: Callable, t: float, u: np.ndarray, tau: float, scheme: str) -> np.ndarray:
    """One step of eq. (RK) with the tableau of `scheme`."""
    stages, b = TABLEAUX[scheme]
    gn = g(t, u)
    d = {}
    for i, ci, arow in stages:
        x = lc(blocks, ci * tau, [u, ci * tau * gn])
        for j, terms in arow.items():
            for coef, ell, ck in terms:
                if coef != 0.0:
                    x = x + tau * coef * phi(blocks, ck * tau, ell, d[j])
        d[i] = g(t + ci * tau, x) - gn
    x = lc(blocks, tau, [u, tau * gn])
    for i, terms in b.items():
        for coef, ell, ck in terms:
            if coef != 0.0:
                x = x + tau * coef * phi(blocks, ck * tau, ell, d[i])
    return x


def integrate_problem(blocks, g: Callable, u0: np.ndarray, t0: float, T: float, steps: int,
                      scheme: str) -> np.ndarray:
    """`steps` equal steps of `scheme` from u(t0) = u0 to t0 + T."""
    tau = T / steps
    u = np.asarray(u0, dtype=np.float64).copy()
    for k in range(steps):
        u = exprk_step(blocks, g, t0 + k * tau, u, tau, scheme)
    return u


# ---------------------------------------------------------------------------
# ADR (Sec. 4.2)

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


def adr_g_vec(n: int, eps: float, alpha: float) -> Callable:
    def g(t, u):
        U = np.reshape(u, (n, n, n), order="F")
        return np.reshape(adr_g(t, U, n, eps, alpha), -1, order="F")
    return g


def integrate(A, n: int, eps: float, alpha: float, T: float, steps: int, scheme: str = "expeuler"):
    """ADR: the final state (flattened, column-major) after `steps` steps from u_0."""
    u0 = np.reshape(adr_u0(n), -1, order="F")
    return integrate_problem([A], adr_g_vec(n, eps, alpha), u0, 0.0, T, steps, scheme)


def relative_error(u: np.ndarray, n: int, T: float) -> float:
    ex = np.reshape(np.exp(T) * adr_u0(n), -1, order="F")
    return float(np.abs(u - ex).max() / np.abs(ex).max())


# ---------------------------------------------------------------------------
# Allen--Cahn (Sec. 4.3) and Brusselator (Sec. 4.4) right-hand sides

def ac_g(eps: float) -> Callable:
    def g(t, u):
        return -(u * u * u) / (eps * eps)
    return g


def bruss_g(a: float, b: float) -> Callable:
    def g(t, w):
        N = w.size // 2
        u, v = w[:N], w[N:]
        uuv = u * u * v
        return np.concatenate([a + uuv, b * u - uuv])
    return g


def rel_inf(u: np.ndarray, ref: np.ndarray) -> float:
    """Relative infinity-norm error, the measure of Sec. 4."""
    return float(np.abs(u - ref).max() / np.abs(ref).max())
