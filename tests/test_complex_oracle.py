"""Complex operators (Sec. 4.1 validation operator (1+i)/100 Laplacian):
the oracle's eigenbasis route (O2, complex128) pinned to the Taylor action of
the augmented matrix (O3, complex) and to scipy's dense exponential."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as wk
from oracle import eig, kron
from oracle import taylor_action as ta

ZETA = (1 + 1j) / 100


def _case(n, d):
    zeta, T, v = wk.validation_complex(n, d)
    assert zeta == ZETA
    return T, v


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n,d", [(7, 2), (5, 3)])
def test_eigenbasis_matches_taylor_action(n, d):
    T, v = _case(n, d)
    A = [ZETA * t for t in T]
    got = eig.scaled_phi_actions(ZETA, T, 1.0, v, range(6))
    for l in range(6):
        ref = ta.lincomb(A, 1.0, [None] * l + [v])
        assert rel(got[l], ref) < 1e-13, l
    # scales and the linear combination, c^l convention
    vs = [v] + [v * (k + 1) for k in range(5)]
    for c in (1.0, 0.5):
        assert rel(eig.scaled_lincomb(ZETA, T, 1.0, vs, c), ta.lincomb(A, 1.0, vs, c)) < 1e-13


def test_eigenbasis_matches_dense_exponential():
    T, v = _case(4, 2)
    K = ZETA * kron.kron_sum_dense(T)
    N = K.shape[0]
    B = np.zeros((N + 2, N + 2), dtype=complex)
    B[:N, :N] = K
    B[:N, N] = v          # v_2
    B[:N, N + 1] = 2 * v  # v_1
    B[N, N + 1] = 1.0
    ref = (expm(B) @ np.concatenate([v, [0.0, 1.0]]))[:N]
    got = eig.scaled_lincomb(ZETA, T, 1.0, [v, 2 * v, v])
    assert rel(got, ref) < 1e-13


def test_validation_vector_layout():
    """v = 4096 (1+i) prod x_mu (1 - x_mu) in the column-major vec (Lemma 1)."""
    n, d = 5, 3
    _, v = _case(n, d)
    x = np.arange(1, n + 1) / (n + 1)
    i, j, k = 1, 3, 2
    assert v[i + n * j + n * n * k] == pytest.approx(4096 * (1 + 1j) * x[i] * (1 - x[i]) * x[j] * (1 - x[j])
                                                     * x[k] * (1 - x[k]), rel=1e-15)
    assert math.isclose(abs(v).max(), abs(4096 * (1 + 1j)) * (x[2] * (1 - x[2])) ** 3, rel_tol=1e-14)
