"""O3: Taylor action of the augmented matrix, with K x applied by mu-mode
products with the A_mu themselves (oracle; any size, no exponential of A_mu).

Target (Sec. 2 augmented-matrix statement; Sec. 3.2 eq. scallincomb): the top
N rows of exp(c B) [v_0; 0; ...; 0; 1] with B = [[tau K, v_p ... v_1],[0, J]].
The vectors are balanced first: B_eta = [[tau K, eta W], [0, J]] applied to
[v_0; 0; ...; 0; 1/eta] has the same top rows for any eta > 0 (the top-right
block of exp(B) is linear in W).  Then exp(cB) b = (T_m(cB/sigma))^sigma b
(the truncated-Taylor action of Al-Mohy & Higham 2011) with sigma =
ceil(c ||B_eta||_1 bound) so every step has norm <= 1, and each step's series
summed until two consecutive terms fall below 2^-56 of the partial sum.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np

from .kron import kron_sum_apply


def _norm1(M):
    return float(np.abs(M).sum(axis=0).max())


def lincomb(A: Sequence[np.ndarray], tau: float, vs: Sequence[Optional[np.ndarray]],
            c: float = 1.0, tol: float = 2.0 ** -56, max_terms: int = 200) -> np.ndarray:
    """exp(c tau K) v_0 + sum_{l>=1} c^l phi_l(c tau K) v_l (vs = [v_0..v_p])."""
    n = tuple(a.shape[0] for a in A)
    N = int(np.prod(n))
    p = len(vs) - 1
    dt = np.result_type(*A, *[v for v in vs if v is not None], np.float64)
    vz = [None if v is None else np.reshape(np.asarray(v, dtype=dt), n, order="F") for v in vs]
    # W = [v_p, ..., v_1]: column k (1-based) is v_{p+1-k}
    W = [vz[p + 1 - k] for k in range(1, p + 1)]
    normK = abs(tau) * sum(_norm1(a) for a in A)
    wmax = max([float(np.abs(w).sum()) for w in W if w is not None] + [0.0])
    eta = 1.0
    if wmax > 0:
        eta = 2.0 ** -math.ceil(math.log2(max(wmax / max(normK, 1.0), 1.0)))
    normB = max(normK, eta * wmax + 1.0) if p > 0 else normK
    sigma = max(1, int(math.ceil(abs(c) * normB)))
    h = c / sigma

    def matvec(X, y):
        top = tau * kron_sum_apply(X, A)
        for k in range(1, p + 1):
            if W[k - 1] is not None and y[k - 1] != 0:
                top = top + (eta * y[k - 1]) * W[k - 1]
        ybot = np.zeros_like(y)
        ybot[:-1] = y[1:]
        return top, ybot

    X = np.zeros(n, dtype=dt) if vz[0] is None else vz[0].copy()
    y = np.zeros(p, dtype=dt)
    if p > 0:
        y[-1] = 1.0 / eta
    for _ in range(sigma):
        fX, fy = X.copy(), y.copy()
        tX, ty = X, y
        small = 0
        for k in range(1, max_terms + 1):
            tX, ty = matvec(tX, ty)
            tX = tX * (h / k)
            ty = ty * (h / k)
            fX = fX + tX
            fy = fy + ty
            rX = float(np.abs(tX).max()) / max(float(np.abs(fX).max()), 1e-300)
            ry = float(np.abs(ty).max()) / max(float(np.abs(fy).max()), 1e-300) if p else 0.0
            small = small + 1 if max(rX, ry) <= tol else 0
            if small >= 2:
                break
        X, y = fX, fy
    return np.reshape(X, (-1,), order="F")


def same(A: Sequence[np.ndarray], tau: float, v: np.ndarray, p: int, c: float = 1.0,
         ells=None) -> np.ndarray:
    """[phi_l(c tau K) v for l in ells] (default 0..p) as rows."""
    ells = list(range(p + 1)) if ells is None else list(ells)
    rows = []
    for l in ells:
        vs = [None] * (l + 1)
        vs[l] = v
        r = lincomb(A, tau, vs, c)
        rows.append(r / (c ** l))
    return np.stack(rows)
