"""Kronecker sums, mu-mode products and the Tucker operator (oracle).

Sec. 1 eq. (kronsum): K = sum_mu I_d x ... x A_mu x ... x I_1.
Sec. 2: W = V x_mu L with w_{..i_mu..} = sum_j l_{i_mu j} v_{..j..}; the
Tucker operator V x_1 L_1 ... x_d L_d; Lemma 1: (L_d x ... x L_1) v =
vec(V x_1 L_1 ... x_d L_d) with vec stacking by columns (mode 1 fastest).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def kron_sum_dense(A: Sequence[np.ndarray]) -> np.ndarray:
    """Form K densely (tiny sizes only)."""
    d = len(A)
    n = [a.shape[0] for a in A]
    N = int(np.prod(n))
    K = np.zeros((N, N), dtype=np.result_type(*A))
    for mu in range(d):
        # factor order in the product is I_d x ... x A_mu x ... x I_1
        term = np.ones((1, 1), dtype=K.dtype)
        for nu in reversed(range(d)):
            term = np.kron(term, A[nu] if nu == mu else np.eye(n[nu]))
        K += term
    return K


def kron_dense(L: Sequence[np.ndarray]) -> np.ndarray:
    """L_d x ... x L_1 (tiny sizes only)."""
    out = np.ones((1, 1), dtype=np.result_type(*L))
    for Lm in reversed(L):
        out = np.kron(out, Lm)
    return out


def unvec(v: np.ndarray, n: Sequence[int]) -> np.ndarray:
    return np.reshape(v, tuple(n), order="F")


def vec(V: np.ndarray) -> np.ndarray:
    return np.reshape(V, (-1,), order="F")


def mode_product(V: np.ndarray, L: np.ndarray, mu: int) -> np.ndarray:
    """V x_mu L (mu is 0-based here): contract axis mu of V with the second
    index of L, and put the result back on axis mu."""
    W = np.tensordot(L, V, axes=([1], [mu]))      # new axis 0 = i_mu
    return np.moveaxis(W, 0, mu)


def tucker(V: np.ndarray, L: Sequence[np.ndarray]) -> np.ndarray:
    W = V
    for mu, Lm in enumerate(L):
        W = mode_product(W, Lm, mu)
    return W


def kron_sum_apply(V: np.ndarray, A: Sequence[np.ndarray]) -> np.ndarray:
    """K v in tensor form: sum_mu V x_mu A_mu."""
    out = None
    for mu, Am in enumerate(A):
        t = mode_product(V, Am, mu)
        out = t if out is None else out + t
    return out
