"""Quadrature rules on [0, 1] (oracle).

Gauss-Lobatto-Legendre with q points (Sec. 3.3: the rule phiks uses, with
theta_1 = 0 and theta_q = 1): the interior nodes are the roots of P'_{q-1}
mapped from [-1, 1]; the weights are 1/(q (q-1) P_{q-1}(x_i)^2) (the usual
[-1, 1] weights halved).  Gauss-Legendre with q points as the alternative
rule.  Both built from numpy's Legendre-series routines.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def gll(q: int):
    if q < 2:
        raise ValueError("GLL needs q >= 2")
    c = np.zeros(q)
    c[q - 1] = 1.0                      # P_{q-1}
    interior = np.sort(np.real(L.legroots(L.legder(c)))) if q > 2 else np.array([])
    x = np.concatenate([[-1.0], interior, [1.0]])
    Pq1 = L.legval(x, c)
    w = 2.0 / (q * (q - 1) * Pq1 ** 2)
    return (x + 1.0) / 2.0, w / 2.0


def gl(q: int):
    x, w = L.leggauss(q)
    return (x + 1.0) / 2.0, w / 2.0


def rule(name: str, q: int):
    return gll(q) if name == "gll" else gl(q)
