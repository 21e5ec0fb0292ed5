"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the phiks method itself: only a
counter-based pseudo-random generator (SplitMix64) and the finite-difference /
spectral operators A_mu that define the workloads (the advection-diffusion-
reaction operators of Sec. 4.2, the Allen-Cahn and Brusselator operators of
Sec. 4.3-4.4, the Chebyshev variant).  Every matrix is returned as a
Fortran-ordered (column-major) float64 numpy array, the layout the Lemma of
Sec. 2 fixes for vec().
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of SplitMix64 (Steele, Lea, Flood 2014).

    SplitMix64 is counter based: output i is mix(seed + (i+1)*gamma), so a
    whole stream is one vectorised evaluation.
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """53-bit uniform doubles in [lo, hi)."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller on consecutive SplitMix64 pairs."""
    m = (count + 1) // 2
    raw = splitmix64(seed, 2 * m)
    u1 = ((raw[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53  # (0, 1]
    u2 = (raw[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


def log_uniform(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    u = uniform(seed, count, 0.0, 1.0)
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


# ----------------------------------------------------------------------------
# One-dimensional operators A_mu (Sec. 1 and Sec. 4).  Dirichlet: n interior
# points, h = 1/(n+1).  Neumann: n vertex-centred points, h = 1/(n-1), ghost
# points folded into the first and last rows.
# ----------------------------------------------------------------------------

def tridiag(n: int, sub: float, diag: float, sup: float) -> np.ndarray:
    A = np.zeros((n, n), order="F")
    idx = np.arange(n)
    A[idx, idx] = diag
    A[idx[1:], idx[:-1]] = sub
    A[idx[:-1], idx[1:]] = sup
    return A


def fd_adr_dirichlet(n: int, eps: float, alpha: float, react: float = 0.0,
                     length: float = 1.0) -> np.ndarray:
    """eps*d_xx + alpha*d_x + react*I, 2nd-order central FD, homogeneous
    Dirichlet on [0, length] with n interior points."""
    h = length / (n + 1)
    sub = eps / h ** 2 - alpha / (2 * h)
    sup = eps / h ** 2 + alpha / (2 * h)
    return tridiag(n, sub, -2 * eps / h ** 2 + react, sup)


def fd_laplacian_neumann(n: int, coef: float = 1.0, react: float = 0.0) -> np.ndarray:
    """coef*d_xx + react*I on [0,1], homogeneous Neumann, n vertex-centred
    points (h = 1/(n-1)), ghost-point rows (-2, 2)/h^2 at both ends."""
    h = 1.0 / (n - 1)
    A = tridiag(n, coef / h ** 2, -2 * coef / h ** 2 + react, coef / h ** 2)
    A[0, 1] = 2 * coef / h ** 2
    A[n - 1, n - 2] = 2 * coef / h ** 2
    return A


def cheb_d2_dirichlet(n_inner: int) -> np.ndarray:
    """Second-derivative Chebyshev collocation matrix on [-1, 1] with the two
    boundary rows/columns removed (homogeneous Dirichlet): n_inner x n_inner,
    from N = n_inner + 1 Gauss-Lobatto points (Trefethen's construction)."""
    N = n_inner + 1
    k = np.arange(N + 1)
    x = np.cos(np.pi * k / N)
    c = np.ones(N + 1)
    c[0] = c[N] = 2.0
    c = c * (-1.0) ** k
    X = np.tile(x, (N + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(N + 1))
    D = D - np.diag(D.sum(axis=1))
    D2 = D @ D
    return np.asfortranarray(D2[1:N, 1:N])


# ----------------------------------------------------------------------------
# Workload configurations (sizes and value distributions of the paper's
# experiments).  Each yields the operators, tau and the input vectors.
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    A: List[np.ndarray]                  # A_1 .. A_d, column-major n_mu x n_mu
    tau: float
    p: int
    mode: str                            # "same" or "lincomb"
    nscales: int
    vs: List[Optional[np.ndarray]]       # SAME: [v]; LINCOMB: [v_0 .. v_p] (None = zero)
    skip_phi0: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return [a.shape[0] for a in self.A]

    @property
    def N(self):
        return int(np.prod(self.n))


def small_same(n: int = 32, seed: int = 1, tau: float = 1e-3, p: int = 3) -> Workload:
    """d=2, n1=n2=n: FD Dirichlet Laplacian plus central advection 0.5*d_x,
    tau=1e-3, phi_0..phi_p on one v ~ U[-1,1]."""
    A = fd_adr_dirichlet(n, 1.0, 0.5)
    N = n * n
    return Workload("adr2d_same_n%d" % n, [A, A.copy(order="F")], tau, p, "same", 1,
                    [uniform(seed, N)])


def adr3d_lincomb(n: int = 64, tau: float = 5e-4, p: int = 4, nscales: int = 3,
                  eps: float = 1.0, alpha=(10.0, -20.0, 5.0), rho: float = 2.0,
                  seeds=(2, 3, 4, 5, 6), dims=None) -> Workload:
    """d=3 nonsymmetric ADR, A_mu = eps*d_xx + alpha_mu*d_x + (rho/3) I, FD
    Dirichlet; sum_l phi_l(tau K) v_l with v_l ~ N(0,1), l=0..p; outputs also at
    tau/2, tau/4 (nscales = 3)."""
    dims = dims or (n, n, n)
    A = [fd_adr_dirichlet(m, eps, a, rho / 3.0) for m, a in zip(dims, alpha)]
    N = int(np.prod(dims))
    vs = [normal(seeds[l], N) for l in range(p + 1)]
    return Workload("adr3d_lincomb_n%s" % "x".join(map(str, dims)), A, tau, p, "lincomb",
                    nscales, vs)


def cheb3d_same(n: int = 128, nrhs: int = 8, tau: float = 5e-7, p: int = 3,
                variant: str = "cheb", seed0: int = 10) -> Workload:
    """d=3, n^3 grid: Chebyshev D^2 Dirichlet (variant 'cheb', tau=5e-7) or FD
    Laplacian (variant 'fd', tau=1e-4); phi_1..phi_p on nrhs N(0,1) vectors."""
    if variant == "cheb":
        A1 = cheb_d2_dirichlet(n)
    else:
        A1 = fd_adr_dirichlet(n, 1.0, 0.0)
    A = [A1.copy(order="F") for _ in range(3)]
    N = n ** 3
    vs = [normal(seed0 + k, N) for k in range(nrhs)]
    return Workload("%s3d_same_n%d" % (variant, n), A, tau, p, "same", 1, vs, skip_phi0=True,
                    meta={"nrhs": nrhs})


def batched_instances(count: int = 256, seed: int = 1000):
    """The uneven-size batch: half d=2 with n_mu in {64,96,..,512}, half d=3
    with n_mu in {16,24,..,96}; FD ADR with eps ~ U[0.1,1], alpha_mu ~
    U[-20,20]; tau ~ logU[1e-4,1e-2]; phi_1..phi_3 on v ~ N(0,1)."""
    out = []
    for k in range(count):
        s = seed + k
        r = uniform(s * 7919 + 1, 16, 0.0, 1.0)
        d = 2 if k < count // 2 else 3
        if d == 2:
            choices = np.arange(64, 513, 32)
        else:
            choices = np.arange(16, 97, 8)
        dims = [int(choices[min(int(r[mu] * len(choices)), len(choices) - 1)]) for mu in range(d)]
        eps = 0.1 + 0.9 * r[4]
        alphas = [-20.0 + 40.0 * r[5 + mu] for mu in range(d)]
        tau = float(np.exp(math.log(1e-4) + r[9] * (math.log(1e-2) - math.log(1e-4))))
        A = [fd_adr_dirichlet(m, eps, a) for m, a in zip(dims, alphas)]
        N = int(np.prod(dims))
        out.append(Workload("inst%d" % k, A, tau, 3, "same", 1, [normal(s, N)], skip_phi0=True))
    return out


# ----------------------------------------------------------------------------
# Served form: a Poisson stream of exponential-integrator stage requests.
# ----------------------------------------------------------------------------

def ac_operator(n: int, eps: float = 0.01):
    """2D Allen-Cahn linear part eps*Laplacian + I (homogeneous Neumann):
    A_mu = eps*d_xx + I/2 per mode."""
    A = fd_laplacian_neumann(n, eps, 0.5)
    return [A, A.copy(order="F")]


def brusselator_operators(n: int, d1: float = 0.002, d2: float = 0.001, b: float = 3.0):
    """2D Brusselator, two species: K_1 = d1*Laplacian - (b+1) I,
    K_2 = d2*Laplacian (homogeneous Neumann)."""
    A1 = fd_laplacian_neumann(n, d1, -(b + 1.0) / 2.0)
    A2 = fd_laplacian_neumann(n, d2, 0.0)
    return [A1, A1.copy(order="F")], [A2, A2.copy(order="F")]


def validation_complex(n: int, d: int):
    """Code-validation inputs of Sec. 4.1: A_mu = zeta T with zeta = (1+i)/100
    and T the second-order Dirichlet Laplacian (h = 1/(n+1)); the vector
    4096 (1+i) prod_mu x_mu (1 - x_mu) (column-major vec).  Returns
    (zeta, [T] * d, v)."""
    T = fd_adr_dirichlet(n, 1.0, 0.0)
    x = np.arange(1, n + 1) / (n + 1.0)
    f = x * (1 - x)
    t = f
    for _ in range(d - 1):
        t = np.multiply.outer(t, f)
    v = 4096 * (1 + 1j) * np.reshape(t, -1, order="F")
    return (1 + 1j) / 100, [T.copy() for _ in range(d)], v


def ac_paper(n: int = 21, eps: float = 0.05, beta: float = 7.0, alpha: float = 0.75):
    """Allen-Cahn problem of Sec. 4.3 on [0,1]^2 (homogeneous Neumann, n
    vertex-centred points per direction): A_mu = d_xx + I/(2 eps^2) (so that
    K = Lap + I/eps^2) and the initial state
    u_0 = tanh((1/4 + cos(beta atan2(y - 1/2, x - 1/2))/10 - r) / (sqrt(2) alpha)),
    r the distance to (1/2, 1/2); u_0 column-major (x fastest)."""
    A = fd_laplacian_neumann(n, 1.0, 0.5 / eps ** 2)
    x = np.arange(n) / (n - 1.0)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    r = np.sqrt((X1 - 0.5) ** 2 + (X2 - 0.5) ** 2)
    u0 = np.tanh((0.25 + 0.1 * np.cos(beta * np.arctan2(X2 - 0.5, X1 - 0.5)) - r) / (np.sqrt(2.0) * alpha))
    return [A, A.copy(order="F")], np.reshape(u0, -1, order="F")


def brusselator3d(n: int, d1: float = 0.02, d2: float = 0.02, a: float = 1.0, b: float = 3.0,
                  c: float = 1.0):
    """Brusselator problem of Sec. 4.4 on [0,1]^3 (homogeneous Neumann, n
    vertex-centred points, second-order differences): blocks
    K_1 = d1 Lap - (b + 1) I and K_2 = d2 Lap as Kronecker sums, and the state
    [u_0; v_0], u_0 = 64^2 prod x^2 (1 - x)^2, v_0 = c."""
    A1 = fd_laplacian_neumann(n, d1, -(b + 1.0) / 3.0)
    A2 = fd_laplacian_neumann(n, d2, 0.0)
    x = np.arange(n) / (n - 1.0)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    u0 = 64.0 ** 2 * (X1 * (1 - X1) * X2 * (1 - X2) * X3 * (1 - X3)) ** 2
    w0 = np.concatenate([np.reshape(u0, -1, order="F"), np.full(n ** 3, c)])
    return [[A1, A1.copy(order="F"), A1.copy(order="F")], [A2, A2.copy(order="F"), A2.copy(order="F")]], w0


SERVED_CLASSES = {
    "ac": {"sizes": list(range(128, 1025, 32)), "tau": 1e-3},
    "adr": {"sizes": list(range(32, 193, 16)), "tau": 5e-4},
    "bru": {"sizes": list(range(128, 513, 32)), "tau": 1e-2},
}


def served_trace(count: int, rate: float, seed_arrivals: int = 7, seed_mix: int = 8,
                 pmin: int = 2, pmax: int = 4, classes=("ac", "adr", "bru"), size_cap=None):
    """Arrival times (Poisson, mean `rate` per second) and request specs:
    (class, n, p).  Classes uniform; n uniform over the class sizes (at most
    size_cap); p uniform in [pmin, pmax]."""
    u = uniform(seed_arrivals, count, 0.0, 1.0)
    gaps = -np.log1p(-u) / rate
    arrivals = np.cumsum(gaps)
    r = uniform(seed_mix, 3 * count, 0.0, 1.0).reshape(count, 3)
    specs = []
    for k in range(count):
        cls = classes[min(int(r[k, 0] * len(classes)), len(classes) - 1)]
        sizes = [s for s in SERVED_CLASSES[cls]["sizes"] if size_cap is None or s <= size_cap]
        n = sizes[min(int(r[k, 1] * len(sizes)), len(sizes) - 1)]
        p = pmin + min(int(r[k, 2] * (pmax - pmin + 1)), pmax - pmin)
        specs.append((cls, n, p))
    return arrivals, specs
