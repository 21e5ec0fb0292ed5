"""Choice of the scaling s and the node count q (Sec. 3.3), restated
step by step (oracle).

Remainder (eq. remainder, Sec. 3.3): R_q(f) = (1/2 pi i) oint_Gamma k_q(z)
f(z, K) dz with k_q(z) = int_0^1 pi_q(t) / (pi_q(z) (z - t)) dt, pi_q the
monic node polynomial.  Gamma_r: the ellipse with foci {0, 1} and capacity
r > 1/4, z(zeta) = r e^{i zeta} + 1/2 + e^{-i zeta}/(16 r).  Estimate
(eq. CPestimate, Crouzeix-Palencia): ||R_q(f_l(., K))||_2 <= (1+sqrt 2)/(2 pi)
sup_{w in Omega} | int_0^{2pi} k_q(z) f_l(z, w) (r e^{i zeta} - e^{-i zeta}/(16 r))
dzeta |, with f_l(z, w) = z^{l-1}/(l-1)! exp((1-z) w) and Omega the rectangle
Xi = sum_mu Xi_mu enclosing the numerical range of K; by the maximum modulus
principle the sup is taken on the boundary of Xi.

Readings of points the paper leaves open (shared with the library planner):
  * Xi_mu = [lambda_min(H_mu), lambda_max(H_mu)] x i[-||S_mu||_2, ||S_mu||_2]
    with H_mu, S_mu the Hermitian and skew-Hermitian parts of A_mu (real A_mu);
    for the complex validation operator the skew part is taken as a rectangle
    [lambda_min, lambda_max] of the Hermitian matrix (A - A^*)/(2i).
  * the contour integral does not depend on r (Cauchy); r only sets the
    accuracy of its trapezoidal evaluation, so each value plus its estimated
    numerical error (the rule on half the nodes, and rounding) is minimised
    over 24 log-spaced values of r in [0.3, 8] for each (q, s, l).
  * the boundary of Xi is sampled with 64 points per side (a degenerate side
    collapses to its endpoints), the zeta integral by the trapezoidal rule with
    128 points, k_q by 128-point Gauss-Legendre in t.
  * stopping rule: s = 0, 1, ...; q_s = smallest feasible q in [qmin, qmax]
    (infeasible s counts as T# = infinity); stop at the first s whose T#
    exceeds the previous one (ties continue); s <= 64.  If the requested
    number of scales nscales exceeds s + 1, s is raised to nscales - 1 with
    the smallest feasible q there.

Parity status: the estimate is pinned against the true remainder: for a
scalar operator it must equal (1 + sqrt 2) times |R_q(f_l(., w/2^s))| computed
in 40-digit arithmetic (GLL and GL, several q, s, l and w), and on diagonal
operators it must dominate the matrix remainder; the rules by their exactness
tests; the selected (s, q) meet the accuracy the bound promises on small
problems; the reproduction of the paper's parameter table is a soft pin (the
table depends on the unstated r grid and discretisation).
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from .quadrature import rule as quad_rule

N_R = 24
R_LO, R_HI = 0.3, 8.0
N_SIDE = 64
N_ZETA = 128
N_T = 128


def numerical_range_rect(A: np.ndarray):
    """Rectangle (xlo, xhi, ylo, yhi) enclosing W(A)."""
    A = np.asarray(A)
    H = (A + A.conj().T) / 2.0
    S = (A - A.conj().T) / 2.0j           # Hermitian
    eh = np.linalg.eigvalsh(H)
    es = np.linalg.eigvalsh(S)
    if np.iscomplexobj(A):
        return float(eh[0]), float(eh[-1]), float(es[0]), float(es[-1])
    m = float(max(abs(es[0]), abs(es[-1])))
    return float(eh[0]), float(eh[-1]), -m, m


def kron_sum_rect(A: Sequence[np.ndarray], tau: float):
    rects = [numerical_range_rect(a) for a in A]
    xlo = sum(r[0] for r in rects) * tau
    xhi = sum(r[1] for r in rects) * tau
    ylo = sum(r[2] for r in rects) * tau
    yhi = sum(r[3] for r in rects) * tau
    if tau < 0:
        xlo, xhi, ylo, yhi = xhi, xlo, yhi, ylo
    return xlo, xhi, ylo, yhi


def rect_boundary(rect) -> np.ndarray:
    xlo, xhi, ylo, yhi = rect
    t = np.linspace(0.0, 1.0, N_SIDE, endpoint=False)
    pts = []
    if xhi > xlo:
        pts.append(xlo + (xhi - xlo) * t + 1j * ylo)
        pts.append(xhi - (xhi - xlo) * t + 1j * yhi)
    else:
        pts.append(np.array([xlo + 1j * ylo, xlo + 1j * yhi]))
    if yhi > ylo:
        pts.append(xhi + 1j * (ylo + (yhi - ylo) * t))
        pts.append(xlo + 1j * (yhi - (yhi - ylo) * t))
    else:
        pts.append(np.array([xlo + 1j * ylo, xhi + 1j * ylo]))
    return np.concatenate(pts)


def r_grid() -> np.ndarray:
    return np.exp(np.linspace(math.log(R_LO), math.log(R_HI), N_R))


def ellipse(r: float):
    zeta = 2.0 * math.pi * np.arange(N_ZETA) / N_ZETA
    z = r * np.exp(1j * zeta) + 0.5 + np.exp(-1j * zeta) / (16.0 * r)
    dz = r * np.exp(1j * zeta) - np.exp(-1j * zeta) / (16.0 * r)
    return z, dz


@functools.lru_cache(maxsize=None)
def _kernel_on_ellipse(rule: str, q: int, ir: int):
    nodes = quad_rule(rule, q)[0]
    z, _ = ellipse(r_grid()[ir])
    return kernel(nodes, z)


def kernel(nodes: np.ndarray, z: np.ndarray) -> np.ndarray:
    """k_q(z) = int_0^1 prod_i (t - theta_i)/(z - theta_i) / (z - t) dt by
    Gauss-Legendre in t."""
    xt, wt = np.polynomial.legendre.leggauss(N_T)
    t = (xt + 1.0) / 2.0
    wt = wt / 2.0
    ratio = np.ones((z.size, t.size), dtype=complex)
    for th in nodes:
        ratio *= (t[None, :] - th) / (z[:, None] - th)
    return (ratio / (z[:, None] - t[None, :])) @ wt


def remainder_bounds_all(rect, s: int, qs: Sequence[int], p: int, rule: str = "gll"):
    """{q: b} with b[l-1] >= ||R_q(f_l(., K/2^s))||_2 for l = 1..p.

    For each w the contour integral is the same for every capacity r (f_l is
    entire, k_q analytic off [0, 1]: Cauchy), so r only decides how well the
    trapezoidal rule computes it: near r = 1/4 the contour hugs the cut of
    k_q and the rule converges slowly, for large r the integrand grows like
    exp(|w| r) and its sum cancels.  Each value therefore carries its own
    error estimate, |I_N - I_{N/2}| (the rule on every other node) plus
    N 2^-53 sum |terms| (rounding), before the minimum over the r grid: a
    value that is small only because it is inaccurate is not taken."""
    w = rect_boundary(rect) / (2.0 ** s)
    best = {q: np.full(p, np.inf) for q in qs}
    for ir, r in enumerate(r_grid()):
        z, dz = ellipse(r)
        with np.errstate(over="ignore", invalid="ignore"):
            E = np.exp(np.outer(1.0 - z, w))            # (zeta, w)
            aE = np.abs(E)
            for q in qs:
                k = _kernel_on_ellipse(rule, q, ir)
                for l in range(1, p + 1):
                    c = k * z ** (l - 1) / math.factorial(l - 1) * dz
                    full = c @ E                         # N_ZETA-point rule (times N_ZETA)
                    half = 2.0 * (c[::2] @ E[::2])       # every other node
                    round_err = N_ZETA * 2.0 ** -53 * (np.abs(c) @ aE)
                    est = np.abs(full) + np.abs(full - half) + round_err
                    val = est.max() * (1.0 + math.sqrt(2.0)) / N_ZETA
                    if np.isfinite(val):
                        best[q][l - 1] = min(best[q][l - 1], val)
    return best


def remainder_bounds(rect, s: int, q: int, p: int, rule: str = "gll") -> np.ndarray:
    return remainder_bounds_all(rect, s, [q], p, rule)[q]


def tucker_count(mode: str, s: int, nscales: int, q: int, p: int) -> int:
    """eq. (Tpsv) for the same-vector task, eq. (Tlcp) for linear combinations."""
    return q + s * p + nscales if mode == "same" else q * p + s * p + nscales


def feasible(mode: str, b: np.ndarray, s: int, p: int, vnorms, tol: float) -> bool:
    if mode == "same":
        v = vnorms[0]
        return all(b[l - 1] * v <= tol * 2.0 ** (l * s) for l in range(1, p + 1))
    # linear combination: vnorms[l] = ||v_l||, l = 0..p
    for l in range(1, p + 1):
        tot = 0.0
        for k in range(1, l + 1):
            tot += b[l - k] * vnorms[p + 1 - k] / 2.0 ** ((l - k + 1) * s)
        if not tot <= tol:
            return False
    return True


@dataclass
class Params:
    s: int
    q: int
    tcount: int


def smallest_q(rect, s, p, mode, vnorms, tol, qmin, qmax, rule):
    qs = list(range(qmin, qmax + 1))
    b = remainder_bounds_all(rect, s, qs, p, rule)
    for q in qs:
        if feasible(mode, b[q], s, p, vnorms, tol):
            return q
    return None


def select(rect, p: int, mode: str, vnorms: Sequence[float], nscales: int = 1,
           tol: float = 2.0 ** -53, qmin: int = 3, qmax: int = 12, rule: str = "gll",
           smax: int = 64) -> Optional[Params]:
    prev = None
    for s in range(0, smax + 1):
        q = smallest_q(rect, s, p, mode, vnorms, tol, qmin, qmax, rule)
        T = math.inf if q is None else tucker_count(mode, s, nscales, q, p)
        if prev is not None and T > prev[2]:
            break
        prev = (s, q, T)
    if prev is None or prev[1] is None:
        return None
    s, q, T = prev
    if s < nscales - 1:
        s = nscales - 1
        q = None
        while q is None and s <= smax:
            q = smallest_q(rect, s, p, mode, vnorms, tol, qmin, qmax, rule)
            if q is None:
                s += 1
        if q is None:
            return None
        T = tucker_count(mode, s, nscales, q, p)
    return Params(s, q, int(T))
