"""Dense matrix exponential (oracle).

Scaling and squaring with a truncated Taylor series (Moler & Van Loan,
"Nineteen dubious ways to compute the exponential of a matrix", method 3):
exp(X) = (T_m(X/2^t))^(2^t) with 2^t >= ||X||_1 / 0.5 and the series summed
until a term is below 2^-56 of the partial sum in 1-norm.  Plain and slow by
design; cross-checked against scipy.linalg.expm in the tests.
"""
from __future__ import annotations

import math

import numpy as np


def expm_taylor(X: np.ndarray, theta: float = 0.5, max_terms: int = 60) -> np.ndarray:
    X = np.asarray(X)
    n = X.shape[0]
    nrm = np.abs(X).sum(axis=0).max() if n else 0.0
    t = 0
    if nrm > theta:
        t = int(math.ceil(math.log2(nrm / theta)))
    Y = X / (2.0 ** t)
    S = np.eye(n, dtype=X.dtype)
    term = np.eye(n, dtype=X.dtype)
    for k in range(1, max_terms):
        term = term @ Y / k
        S = S + term
        tn = np.abs(term).sum(axis=0).max()
        if tn <= 2.0 ** -56 * np.abs(S).sum(axis=0).max():
            break
    for _ in range(t):
        S = S @ S
    return S
