"""phi_l of a scalar argument (oracle; test infrastructure only).

Definition (Sec. 1, eq. phifunctions): phi_l(x) = int_0^1 theta^(l-1)/(l-1)!
exp((1-theta) x) dtheta for l >= 1, phi_0 = exp.  Equivalent series
phi_l(z) = sum_k z^k/(k+l)!, and recurrence phi_l(z) = (phi_{l-1}(z) -
1/(l-1)!)/z.
"""
from __future__ import annotations

import math

import numpy as np


def phi_series(l: int, z, terms: int = 60):
    """sum_{k>=0} z^k/(k+l)!, accurate for |z| <= 1 (works on numpy arrays and
    on numpy longdouble / complex)."""
    z = np.asarray(z)
    one = np.ones_like(z)
    term = one / math.factorial(l)
    acc = term.copy()
    for k in range(1, terms):
        term = term * z / (k + l)
        acc = acc + term
    return acc


def phi_recurrence(l: int, z):
    """phi_0 = exp(z), phi_j = (phi_{j-1} - 1/(j-1)!)/z: stable for |z| >= 1."""
    z = np.asarray(z)
    f = np.exp(z)
    one = np.ones_like(f)
    for j in range(1, l + 1):
        f = (f - one / math.factorial(j - 1)) / z
    return f


def phi(l: int, z):
    """phi_l(z) elementwise: series for |z| < 1, recurrence otherwise."""
    z = np.asarray(z)
    small = np.abs(z) < 1.0
    out = np.empty_like(z if np.iscomplexobj(z) or z.dtype == np.longdouble else z.astype(np.float64))
    zs = np.where(small, z, 0.5)
    zl = np.where(small, 2.0, z)
    with np.errstate(all="ignore"):
        a = phi_series(l, zs)
        b = phi_recurrence(l, zl)
    out[...] = np.where(small, a, b)
    return out


def phi_mp(l: int, z, dps: int = 50):
    """High-precision reference with mpmath (pins only): the series summed to
    convergence at dps decimal digits."""
    import mpmath as mp
    with mp.workdps(dps):
        z = mp.mpmathify(z)
        term = mp.mpf(1) / mp.factorial(l)
        acc = term
        k = 0
        while True:
            k += 1
            term = term * z / (k + l)
            acc += term
            if abs(term) < mp.mpf(10) ** (-dps) * max(1, abs(acc)) and k > abs(z) + 5:
                break
        return acc
