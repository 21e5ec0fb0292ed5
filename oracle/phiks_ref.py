"""The phiks algorithm restated step by step in plain numpy (oracle).

Used to check the CUDA path at a fixed (s, q) far more tightly than the
tolerance of the method allows, and to pin the method's convergence.

Same vector (Sec. 3.1): eq. (integrandsimul) for the quadrature at K/2^s,
eq. (simul) for the squaring j = s, ..., 1, one Tucker per requested scale
for phi_0.  Linear combination (Sec. 3.2): eq. (integrandcomb) and eq. (comb),
plus exp(K/2^L) v_0 per scale.  K stands for tau K throughout.  Small
exponentials exp((1-theta_i) tau A_mu / 2^s) by the oracle's Taylor expm;
exp(tau A_mu / 2^(j-1)) by squaring exp(tau A_mu / 2^j).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np

from .expm import expm_taylor
from .kron import tucker, unvec, vec
from .quadrature import rule as quad_rule


def _exps(A, tau, s, theta):
    return [expm_taylor((1.0 - theta) * tau * a / 2.0 ** s) for a in A]


def same(A: Sequence[np.ndarray], tau: float, v: np.ndarray, p: int, s: int, q: int,
         nscales: int = 1, rule: str = "gll", skip_phi0: bool = False) -> np.ndarray:
    """Rows: for each level L = 0..nscales-1 the block [phi_0 (unless
    skipped), phi_1, ..., phi_p](tau K / 2^L) v."""
    n = [a.shape[0] for a in A]
    V = unvec(np.asarray(v), n)
    theta, w = quad_rule(rule, q)
    acc = [np.zeros_like(V, dtype=np.result_type(V, *A)) for _ in range(p)]
    for i in range(q):
        Y = V if theta[i] == 1.0 else tucker(V, _exps(A, tau, s, theta[i]))
        for l in range(1, p + 1):
            acc[l - 1] = acc[l - 1] + w[i] * theta[i] ** (l - 1) / math.factorial(l - 1) * Y
    M = _exps(A, tau, s, 0.0)                       # exp(tau A_mu / 2^s)
    blocks = {}

    def emit(L, M):
        rows = [] if skip_phi0 else [vec(tucker(V, M))]
        rows += [vec(a) for a in acc]
        blocks[L] = rows

    if s < nscales:
        emit(s, M)
    for j in range(s, 0, -1):
        for l in range(p, 0, -1):
            tot = tucker(acc[l - 1], M)
            for k in range(1, l + 1):
                tot = tot + acc[k - 1] / math.factorial(l - k)
            acc[l - 1] = tot / 2.0 ** l
        M = [m @ m for m in M]                      # exp(tau A_mu / 2^(j-1))
        if j - 1 < nscales:
            emit(j - 1, M)
    return np.stack([r for L in range(nscales) for r in blocks[L]])


def lincomb(A: Sequence[np.ndarray], tau: float, vs: Sequence[Optional[np.ndarray]],
            s: int, q: int, nscales: int = 1, rule: str = "gll") -> np.ndarray:
    """Rows: for each level L = 0..nscales-1, exp(c tau K) v_0 +
    sum_l c^l phi_l(c tau K) v_l with c = 2^-L (eq. scallincomb)."""
    n = [a.shape[0] for a in A]
    p = len(vs) - 1
    dt = np.result_type(*A, *[x for x in vs if x is not None], np.float64)
    Vs = [np.zeros(n, dtype=dt) if x is None else unvec(np.asarray(x, dtype=dt), n) for x in vs]
    theta, w = quad_rule(rule, q)
    acc = [np.zeros(n, dtype=dt) for _ in range(p)]      # acc[l-1] = Phi v_{p-l+1..p}
    for i in range(q):
        E = None if theta[i] == 1.0 else _exps(A, tau, s, theta[i])
        for l in range(1, p + 1):
            Wil = np.zeros(n, dtype=dt)
            for k in range(1, l + 1):
                Wil = Wil + (theta[i] ** (l - k) / math.factorial(l - k)
                             / 2.0 ** ((l - k + 1) * s)) * Vs[p + 1 - k]
            Y = Wil if E is None else tucker(Wil, E)
            acc[l - 1] = acc[l - 1] + w[i] * Y
    M = _exps(A, tau, s, 0.0)
    rows = {}

    def emit(L, M):
        r = acc[p - 1].copy() if p > 0 else np.zeros(n, dtype=dt)
        if vs[0] is not None:
            r = r + tucker(Vs[0], M)
        rows[L] = vec(r)

    if s < nscales:
        emit(s, M)
    for j in range(s, 0, -1):
        for l in range(p, 0, -1):
            tot = tucker(acc[l - 1], M)
            for k in range(1, l + 1):
                tot = tot + acc[k - 1] / (math.factorial(l - k) * 2.0 ** ((l - k) * j))
            acc[l - 1] = tot
        M = [m @ m for m in M]
        if j - 1 < nscales:
            emit(j - 1, M)
    return np.stack([rows[L] for L in range(nscales)])
