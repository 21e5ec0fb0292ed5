"""O2: phi-actions through the separable eigendecomposition of tridiagonal
Toeplitz A_mu, in extended precision (oracle).

For A = tridiag(a, b, c) (sub a, diagonal b, super c) with a*c > 0:
D^-1 A D = tridiag(sqrt(ac), b, sqrt(ac)) for D = diag((a/c)^((i-1)/2)), and
the symmetric Toeplitz matrix has the orthonormal sine eigenvectors
S_ik = sqrt(2/(n+1)) sin(i k pi/(n+1)) with eigenvalues
lambda_k = b + 2 sqrt(ac) cos(k pi/(n+1)).  Since K is a Kronecker sum,
phi_l(tau K) v = (x_mu D_mu S_mu) [phi_l(tau sum_mu lambda) o (x_mu S_mu D_mu^-1) v]
(Lemma 1 turns each Kronecker factor into a mu-mode product).  The arithmetic
runs in numpy longdouble (80-bit on x86-64, 128-bit on aarch64) because D is
badly conditioned for strongly advective operators.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from .phi_scalar import phi


def toeplitz_coeffs(A: np.ndarray):
    """(sub, diag, super) of a tridiagonal Toeplitz matrix; raises otherwise."""
    n = A.shape[0]
    if n == 1:
        return 0.0, float(A[0, 0]), 0.0
    a, b, c = A[1, 0], A[0, 0], A[0, 1]
    T = np.zeros_like(A)
    i = np.arange(n)
    T[i, i] = b
    T[i[1:], i[:-1]] = a
    T[i[:-1], i[1:]] = c
    if not np.array_equal(T, A):
        raise ValueError("not tridiagonal Toeplitz")
    return float(a), float(b), float(c)


def eig_factors(A: np.ndarray):
    """(lambda, P, Pinv) in longdouble with A = P diag(lambda) Pinv."""
    a, b, c = toeplitz_coeffs(A)
    n = A.shape[0]
    ld = np.longdouble
    if n == 1:
        return np.array([ld(b)]), np.ones((1, 1), ld), np.ones((1, 1), ld)
    if a * c <= 0:
        raise ValueError("O2 needs sub*super > 0")
    a_, b_, c_ = ld(a), ld(b), ld(c)
    k = np.arange(1, n + 1, dtype=ld)
    i = np.arange(1, n + 1, dtype=ld)
    pi = np.arccos(ld(-1))
    S = np.sqrt(ld(2) / (n + 1)) * np.sin(np.outer(i, k) * pi / (n + 1))
    lam = b_ + 2 * np.sqrt(a_ * c_) * np.cos(k * pi / (n + 1))
    r = np.sqrt(a_ / c_)
    dvec = r ** (i - 1)
    P = dvec[:, None] * S
    Pinv = S * (1 / dvec)[None, :]
    return lam, P, Pinv


def _mode(V, L, mu):
    W = np.tensordot(L, V, axes=([1], [mu]))
    return np.moveaxis(W, 0, mu)


def phi_actions(A: Sequence[np.ndarray], tau: float, v: np.ndarray, ells: Sequence[int],
                c: float = 1.0):
    """{l: phi_l(c tau K) v} for each l in ells, via the eigenbasis."""
    n = [a.shape[0] for a in A]
    fac = [eig_factors(a) for a in A]
    V = np.reshape(np.asarray(v, dtype=np.longdouble), tuple(n), order="F")
    for mu, (lam, P, Pinv) in enumerate(fac):
        V = _mode(V, Pinv, mu)
    Z = np.zeros(tuple(n), dtype=np.longdouble)
    for mu, (lam, P, Pinv) in enumerate(fac):
        shape = [1] * len(n)
        shape[mu] = n[mu]
        Z = Z + np.reshape(lam, shape)
    Z = np.longdouble(c) * np.longdouble(tau) * Z
    out = {}
    for l in ells:
        W = phi(l, Z) * V
        for mu, (lam, P, Pinv) in enumerate(fac):
            W = _mode(W, P, mu)
        out[l] = np.reshape(W, (-1,), order="F")
    return out


def lincomb(A, tau, vs, c: float = 1.0):
    """exp(c tau K) v_0 + sum_l c^l phi_l(c tau K) v_l via the eigenbasis."""
    N = int(np.prod([a.shape[0] for a in A]))
    acc = np.zeros(N, dtype=np.longdouble)
    for l, v in enumerate(vs):
        if v is None:
            continue
        acc = acc + np.longdouble(c) ** l * phi_actions(A, tau, v, [l], c)[l]
    return acc


def scaled_phi_actions(zeta: complex, T: Sequence[np.ndarray], tau: float, v: np.ndarray,
                       ells: Sequence[int], c: float = 1.0):
    """{l: phi_l(c tau K) v} for K = zeta (T_d (+) ... (+) T_1), every T_mu real
    symmetric tridiagonal Toeplitz (sub = super): with the orthonormal sine
    eigenvectors S_mu and eigenvalues lambda_mu, phi_l(c tau K) v =
    (x_mu S_mu) [phi_l(c tau zeta sum_mu lambda) o (x_mu S_mu^T) v].  The bases
    are orthogonal, so complex128 arithmetic keeps the result at double
    precision (the complex validation operator (1+i)/100 Laplacian of Sec. 4.1)."""
    n = [t.shape[0] for t in T]
    fac = []
    for t in T:
        a, b, cc = toeplitz_coeffs(t)
        if a != cc:
            raise ValueError("symmetric Toeplitz only")
        m = t.shape[0]
        k = np.arange(1, m + 1)
        S = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(k, k) * np.pi / (m + 1))
        lam = b + 2 * a * np.cos(k * np.pi / (m + 1))
        fac.append((lam, S))
    V = np.reshape(np.asarray(v, dtype=np.complex128), tuple(n), order="F")
    for mu, (lam, S) in enumerate(fac):
        V = _mode(V, S.T, mu)
    Z = np.zeros(tuple(n))
    for mu, (lam, S) in enumerate(fac):
        shape = [1] * len(n)
        shape[mu] = n[mu]
        Z = Z + np.reshape(lam, shape)
    Z = complex(c) * tau * complex(zeta) * Z
    out = {}
    for l in ells:
        W = phi(l, Z) * V
        for mu, (lam, S) in enumerate(fac):
            W = _mode(W, S, mu)
        out[l] = np.reshape(W, (-1,), order="F")
    return out


def scaled_lincomb(zeta: complex, T, tau, vs, c: float = 1.0):
    """exp(c tau K) v_0 + sum_l c^l phi_l(c tau K) v_l for K as in scaled_phi_actions."""
    N = int(np.prod([t.shape[0] for t in T]))
    acc = np.zeros(N, dtype=np.complex128)
    for l, v in enumerate(vs):
        if v is None:
            continue
        acc = acc + c ** l * scaled_phi_actions(zeta, T, tau, v, [l], c)[l]
    return acc
