"""O1: exact phi-actions of a small Kronecker sum from one dense augmented
exponential (oracle; tiny sizes, N + p <= a few thousand).

Sec. 2 (augmented-matrix statement of Theorem 2.1 of Al-Mohy & Higham 2011):
with B = [[tau K, v_p ... v_1], [0, J]], J the p x p upper shift, the first N
rows of exp(c B) [v_0; 0; ...; 0; 1] equal
exp(c tau K) v_0 + sum_l c^l phi_l(c tau K) v_l.
For the same-vector task, exp([[X, W], [0, J]]) with W = [v, 0, ..., 0] holds
phi_m(X) v in column m of its top-right block, and phi_0(X) v = exp(X) v.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from .expm import expm_taylor
from .kron import kron_sum_dense


def _balance(X: np.ndarray, W: np.ndarray) -> float:
    """Power of two eta with ||eta W||_1 <= max(||X||_1, 1).  The top-right
    block of exp([[X, W], [0, J]]) is linear in W, so scaling W by eta and the
    trailing 1 of the right-hand side by 1/eta leaves the result unchanged
    while keeping the scaling-and-squaring count set by X alone."""
    wn = float(np.abs(W).sum(axis=0).max()) if W.size else 0.0
    xn = max(float(np.abs(X).sum(axis=0).max()), 1.0)
    if wn <= xn:
        return 1.0
    return 2.0 ** -int(np.ceil(np.log2(wn / xn)))


def augmented(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    """[[X, W], [0, J]] with J the p x p matrix of ones on the superdiagonal."""
    N, p = W.shape
    B = np.zeros((N + p, N + p), dtype=np.result_type(X, W))
    B[:N, :N] = X
    B[:N, N:] = W
    for k in range(p - 1):
        B[N + k, N + k + 1] = 1.0
    return B


def lincomb(A: Sequence[np.ndarray], tau: float, vs: Sequence[Optional[np.ndarray]],
            c: float = 1.0, expm=expm_taylor) -> np.ndarray:
    """exp(c tau K) v_0 + sum_{l=1}^p c^l phi_l(c tau K) v_l  (eq. scallincomb).
    vs = [v_0, ..., v_p]; None entries are zero vectors."""
    K = kron_sum_dense(A)
    N = K.shape[0]
    p = len(vs) - 1
    dt = np.result_type(K, *[v for v in vs if v is not None])
    vz = [np.zeros(N, dtype=dt) if v is None else np.asarray(v, dtype=dt) for v in vs]
    if p == 0:
        return expm(c * tau * K) @ vz[0]
    W = np.stack([vz[p + 1 - k] for k in range(1, p + 1)], axis=1)   # [v_p ... v_1]
    eta = _balance(tau * K, W)
    B = augmented(tau * K, eta * W)
    E = expm(c * B)
    rhs = np.zeros(N + p, dtype=dt)
    rhs[:N] = vz[0]
    rhs[-1] = 1.0 / eta
    return (E @ rhs)[:N]


def same(A: Sequence[np.ndarray], tau: float, v: np.ndarray, p: int, expm=expm_taylor) -> np.ndarray:
    """[phi_0(tau K) v, ..., phi_p(tau K) v] as a (p+1, N) array."""
    K = kron_sum_dense(A)
    N = K.shape[0]
    v = np.asarray(v)
    out = np.empty((p + 1, N), dtype=np.result_type(K, v))
    if p == 0:
        out[0] = expm(tau * K) @ v
        return out
    W = np.zeros((N, p), dtype=out.dtype)
    W[:, 0] = v
    eta = _balance(tau * K, W)
    E = expm(augmented(tau * K, eta * W))
    out[0] = E[:N, :N] @ v
    for m in range(1, p + 1):
        out[m] = E[:N, N + m - 1] / eta
    return out
