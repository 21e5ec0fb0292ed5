"""Pins of the FP64 oracle against what the mathematics and the paper fix.

Each test ties an oracle function to something other than itself: closed
forms of phi_l (Sec. 1), mpmath's independent arbitrary-precision matrix
exponential, scipy's expm, numpy's Kronecker product (Lemma 1), the exact
sine eigenbasis of the FD Laplacian, quadrature exactness degrees, the
doubling identities eq. (simul) / eq. (comb) on scalars, the p = 2 block
exponential of Sec. 3.2, and the parameter table of Sec. 4.1.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import workloads as wk
from oracle import dense, eig, expm, kron, params, phi_scalar, phiks_ref, quadrature
from oracle import taylor_action as ta

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.abs(a - b).max() / np.abs(b).max())


def phi_closed(l, z):
    """phi_l(z) = (e^z - sum_{k<l} z^k/k!)/z^l, evaluated at 60 digits."""
    with mp.workdps(60):
        z = mp.mpmathify(z)
        s = mp.exp(z) - sum(z ** k / mp.factorial(k) for k in range(l))
        return complex(s / z ** l) if isinstance(z, mp.mpc) else float(s / z ** l)


# ---------------------------------------------------------------- scalar phi
@pytest.mark.parametrize("z", [-30.0, -4.5, -1.0, -0.3, 0.01, 0.7, 2.5, -2 + 3j, 0.4 - 0.2j])
@pytest.mark.parametrize("l", [1, 2, 3, 4, 5])
def test_phi_scalar_closed_form(l, z):
    got = phi_scalar.phi(l, np.array([z]))[0]
    assert abs(got - phi_closed(l, z)) <= 1e-14 * max(1.0, abs(phi_closed(l, z)))


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_phi_recurrence(l):
    # phi_l(z) = (phi_{l-1}(z) - 1/(l-1)!)/z, against the mpmath series
    for z in [-7.0, -1.5, 1.2, 3.0]:
        lhs = phi_scalar.phi_mp(l, z)
        rhs = (phi_scalar.phi_mp(l - 1, z) - mp.mpf(1) / mp.factorial(l - 1)) / z
        assert abs(lhs - rhs) < mp.mpf(10) ** -40
        assert abs(phi_scalar.phi(l, np.array([z]))[0] - float(lhs)) < 1e-14 * abs(float(lhs)) + 1e-16


@pytest.mark.parametrize("z", [-3.0, -0.25, 0.6, -1 + 2j])
def test_doubling_identities_scalar(z):
    """eq. (simul): phi_l(2z) = 2^-l (e^z phi_l(z) + sum_k phi_k(z)/(l-k)!);
    eq. (comb) on a scalar with Phi_j v_{p-l+1..p} = sum_k phi_k(x/2^j) v_{p-l+k}/2^{kj}."""
    p = 4
    f = lambda l, x: phi_scalar.phi_mp(l, x)
    for l in range(1, p + 1):
        lhs = f(l, 2 * z)
        rhs = (mp.exp(z) * f(l, z) + sum(f(k, z) / mp.factorial(l - k) for k in range(1, l + 1))) / 2 ** l
        assert abs(lhs - rhs) < mp.mpf(10) ** -35
    # eq. (comb): x = K, j = 3; scalars v_1..v_p
    x, j = 2 * z, 3
    v = [None, 0.3, -1.1, 0.7, 2.0]

    def Phi(jj, l):  # Phi_jj v_{p-l+1..p}
        return sum(f(k, x / 2 ** jj) * v[p - l + k] / mp.mpf(2) ** (k * jj) for k in range(1, l + 1))
    for l in range(p, 0, -1):
        lhs = Phi(j - 1, l)
        rhs = mp.exp(x / 2 ** j) * Phi(j, l) + sum(
            Phi(j, k) / (mp.factorial(l - k) * mp.mpf(2) ** ((l - k) * j)) for k in range(1, l + 1))
        assert abs(lhs - rhs) < mp.mpf(10) ** -35


# ---------------------------------------------------------------- expm, Lemma 1
def test_expm_vs_scipy():
    rng = np.random.default_rng(0)
    for X in [rng.standard_normal((7, 7)) * 3, 1e-3 * wk.fd_adr_dirichlet(20, 1.0, -20.0),
              rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))]:
        assert rel(expm.expm_taylor(X), sl.expm(X)) < 1e-13


def test_tucker_lemma_and_kron_exp():
    rng = np.random.default_rng(1)
    n = [3, 4, 5]
    L = [rng.standard_normal((m, m)) for m in n]
    v = rng.standard_normal(int(np.prod(n)))
    lhs = kron.kron_dense(L) @ v
    rhs = kron.vec(kron.tucker(kron.unvec(v, n), L))
    assert rel(rhs, lhs) < 1e-14
    # exp(K) v = vec(V x_1 exp(A_1) ... x_d exp(A_d))   (eq. tucker)
    A = [rng.standard_normal((m, m)) * 0.5 for m in n]
    K = kron.kron_sum_dense(A)
    assert rel(kron.vec(kron.tucker(kron.unvec(v, n), [sl.expm(a) for a in A])), sl.expm(K) @ v) < 1e-13
    # K v by mu-mode products equals the dense Kronecker sum
    assert rel(kron.vec(kron.kron_sum_apply(kron.unvec(v, n), A)), K @ v) < 1e-14


# ---------------------------------------------------------------- exact phi actions
def mp_lincomb(A, tau, vs):
    """mpmath reference: top rows of exp([[tau K, v_p..v_1],[0, J]]) [v_0; 0..; 1]."""
    K = kron.kron_sum_dense(A)
    N = K.shape[0]
    p = len(vs) - 1
    with mp.workdps(40):
        B = mp.zeros(N + p, N + p)
        for i in range(N):
            for j in range(N):
                B[i, j] = mp.mpf(float(tau)) * mp.mpf(float(K[i, j]))
            for k in range(1, p + 1):
                B[i, N + k - 1] = mp.mpf(float(vs[p + 1 - k][i]))
        for k in range(p - 1):
            B[N + k, N + k + 1] = 1
        E = mp.expm(B)
        rhs = mp.matrix([mp.mpf(float(x)) for x in vs[0]] + [0] * (p - 1) + [1])
        y = E * rhs
        return np.array([float(y[i]) for i in range(N)])


@pytest.mark.parametrize("alpha,n,tau", [(0.0, 10, 5e-3), (-20.0, 12, 5e-4), (5.0, 9, 2e-3)])
def test_oracles_vs_mpmath_1d(alpha, n, tau):
    A = [wk.fd_adr_dirichlet(n, 1.0, alpha, 2.0 / 3)]
    vs = [wk.normal(3, n), wk.normal(4, n), wk.normal(5, n)]
    exact = mp_lincomb(A, tau, vs)
    assert rel(dense.lincomb(A, tau, vs), exact) < 5e-15
    assert rel(ta.lincomb(A, tau, vs), exact) < 5e-15
    a, b, c = eig.toeplitz_coeffs(A[0])
    cond = (max(a, c) / min(a, c)) ** ((n - 1) / 2)
    assert rel(eig.lincomb(A, tau, vs).astype(float), exact) < 1e-15 + 1e-18 * cond


def test_scalar_problem_closed_form():
    # d = 1, n = 1: phi_l(tau a) v
    a, tau, v = -37.0, 0.05, 1.7
    out = dense.same([np.array([[a]])], tau, np.array([v]), 4)
    for l in range(5):
        ref = math.exp(tau * a) * v if l == 0 else phi_closed(l, tau * a) * v
        assert abs(out[l][0] - ref) < 1e-15 * abs(ref)


def test_diagonal_operators_elementwise():
    rng = np.random.default_rng(2)
    n = [4, 3, 5]
    lam = [rng.uniform(-40, 1, m) for m in n]
    A = [np.diag(x) for x in lam]
    tau = 0.1
    v = rng.standard_normal(int(np.prod(n)))
    Z = tau * (lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :])
    zf = np.reshape(Z, -1, order="F")
    out1 = dense.same(A, tau, v, 3)
    out3 = ta.same(A, tau, v, 3)
    for l in range(4):
        ref = np.array([(math.exp(z) if l == 0 else phi_closed(l, z)) for z in zf]) * v
        assert rel(out1[l], ref) < 1e-14
        assert rel(out3[l], ref) < 1e-14


def test_sine_eigenbasis():
    n = 11
    A = wk.fd_adr_dirichlet(n, 1.0, 3.0, 0.5)
    lam, P, Pinv = eig.eig_factors(A)
    P = P.astype(float)
    lam = lam.astype(float)
    assert rel(A @ P, P * lam[None, :]) < 1e-13
    assert rel(Pinv.astype(float) @ P, np.eye(n)) < 1e-13
    # Laplacian eigenvalues -(4/h^2) sin^2(k pi / (2(n+1)))
    lap = wk.fd_adr_dirichlet(n, 1.0, 0.0)
    lamL = np.sort(eig.eig_factors(lap)[0].astype(float))
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    assert rel(lamL, np.sort(-(4 / h ** 2) * np.sin(k * np.pi / (2 * (n + 1))) ** 2)) < 1e-14
    # O2 vs O1 on a small 2D Laplacian-plus-advection
    A2 = [wk.fd_adr_dirichlet(10, 1.0, 0.5), wk.fd_adr_dirichlet(9, 1.0, 0.0)]
    v = wk.uniform(1, 90)
    o1 = dense.same(A2, 1e-3, v, 3)
    o2 = eig.phi_actions(A2, 1e-3, v, range(4))
    for l in range(4):
        assert rel(o2[l].astype(float), o1[l]) < 1e-14


def test_taylor_action_vs_dense_3d():
    wl = wk.adr3d_lincomb(p=4, dims=(10, 11, 12))
    for c in [1.0, 0.5, 0.25]:
        assert rel(ta.lincomb(wl.A, wl.tau, wl.vs, c), dense.lincomb(wl.A, wl.tau, wl.vs, c)) < 5e-15


def test_eig_vs_taylor_symmetric_3d():
    A = [wk.fd_adr_dirichlet(m, 1.0, 0.0) for m in (16, 12, 20)]
    v = wk.normal(7, 16 * 12 * 20)
    o2 = eig.phi_actions(A, 5e-4, v, [0, 1, 3])
    o3 = ta.same(A, 5e-4, v, 3, ells=[0, 1, 3])
    for i, l in enumerate([0, 1, 3]):
        assert rel(o3[i], o2[l].astype(float)) < 1e-14


def test_taylor_action_vs_eigenbasis_at_a_large_norm():
    """O3 where tau ||K||_1 is about 40 (as at the measured configurations),
    against the exact sine eigenbasis in extended precision: a Taylor action
    without its scaling would lose every digit to cancellation here."""
    A = [wk.fd_adr_dirichlet(m, 1.0, a) for m, a in ((12, 0.0), (10, 4.0), (14, 0.0))]
    tau = 0.02
    assert 35 < tau * sum(float(np.abs(a).sum(0).max()) for a in A) < 45
    v = wk.normal(9, 12 * 10 * 14)
    o2 = eig.phi_actions(A, tau, v, [0, 1, 3])
    o3 = ta.same(A, tau, v, 3, ells=[0, 1, 3])
    for i, l in enumerate([0, 1, 3]):
        assert rel(o3[i], o2[l].astype(float)) < 1e-13


# ---------------------------------------------------------------- consistency
def test_same_vs_lincomb_and_scales():
    wl = wk.small_same(7, p=3)
    v = wl.vs[0]
    for c in [1.0, 0.5, 0.25]:
        s = dense.same(wl.A, wl.tau * c, v, 3)
        for l in range(4):
            vs = [None] * (l + 1)
            vs[l] = v
            assert rel(dense.lincomb(wl.A, wl.tau, vs, c), c ** l * s[l]) < 1e-14
        # full combination equals the sum of c^l phi_l
        allv = [v * (l + 1) for l in range(4)]
        tot = sum(c ** l * (l + 1) * s[l] for l in range(4))
        assert rel(dense.lincomb(wl.A, wl.tau, allv, c), tot) < 1e-14


def test_block_exponential_p2():
    """Sec. 3.2: exp(2^-j [[K, v2, v1],[0,0,1],[0,0,0]]) has blocks
    exp(K/2^j), Phi_j v_2 = phi_1(K/2^j) v_2/2^j and
    Phi_j v_{1,2} = phi_1(K/2^j) v_1/2^j + phi_2(K/2^j) v_2/2^(2j)."""
    A = [wk.fd_adr_dirichlet(6, 1.0, 1.0), wk.fd_adr_dirichlet(5, 1.0, 0.0)]
    K = 2e-3 * kron.kron_sum_dense(A)
    N = K.shape[0]
    v1, v2 = wk.normal(1, N), wk.normal(2, N)
    for j in [0, 1, 3]:
        B = np.zeros((N + 2, N + 2))
        B[:N, :N] = K
        B[:N, N] = v2
        B[:N, N + 1] = v1
        B[N, N + 1] = 1.0
        E = sl.expm(B / 2 ** j)
        s1 = dense.same(A, 2e-3 / 2 ** j, v1, 2)
        s2 = dense.same(A, 2e-3 / 2 ** j, v2, 2)
        assert rel(E[:N, N], s2[1] / 2 ** j) < 1e-13
        assert rel(E[:N, N + 1], s1[1] / 2 ** j + s2[2] / 2 ** (2 * j)) < 1e-13
        assert abs(E[N, N + 1] - 2.0 ** -j) < 1e-15


# ---------------------------------------------------------------- quadrature
def _cmono(k):
    """int_0^1 (2x-1)^k dx."""
    return 0.0 if k % 2 else 1.0 / (k + 1)


@pytest.mark.parametrize("q", [3, 4, 5, 7, 10, 12])
def test_gll_exactness(q):
    x, w = quadrature.gll(q)
    assert x[0] == 0.0 and x[-1] == 1.0 and np.all(w > 0)
    assert np.allclose(x, 1 - x[::-1], atol=1e-15)
    for deg in range(0, 2 * q - 2):
        assert abs(np.dot(w, (2 * x - 1) ** deg) - _cmono(deg)) < 1e-14
    assert abs(np.dot(w, (2 * x - 1) ** (2 * q - 2)) - _cmono(2 * q - 2)) > 1e-8


@pytest.mark.parametrize("q", [2, 3, 6, 12])
def test_gl_exactness(q):
    x, w = quadrature.gl(q)
    for deg in range(0, 2 * q):
        assert abs(np.dot(w, (2 * x - 1) ** deg) - _cmono(deg)) < 1e-14
    assert abs(np.dot(w, (2 * x - 1) ** (2 * q)) - _cmono(2 * q)) > 1e-8


@pytest.mark.parametrize("rule", ["gll", "gl"])
def test_quadrature_convergence(rule):
    """At fixed s the error of the quadrature phase decreases geometrically
    in q (each added node gains more than a factor 10 here) down to roundoff."""
    wl = wk.small_same(8, p=3, tau=1e-2)
    ex = dense.same(wl.A, wl.tau, wl.vs[0], 3)
    errs = []
    for q in range(3, 14):
        r = phiks_ref.same(wl.A, wl.tau, wl.vs[0], 3, 0, q, rule=rule)
        errs.append(max(rel(r[l], ex[l]) for l in range(1, 4)))
    assert errs[-1] < 5e-15
    k = 0
    while errs[k + 1] > 1e-13:
        assert errs[k + 1] < errs[k] / 10
        k += 1
    assert k >= 5
    # linear combination, same rule
    wl = wk.adr3d_lincomb(p=3, dims=(6, 5, 7), alpha=(1.0, -2.0, 0.5))
    ex = dense.lincomb(wl.A, wl.tau, wl.vs)
    errs = [rel(phiks_ref.lincomb(wl.A, wl.tau, wl.vs, 0, q, rule=rule)[0], ex) for q in range(3, 9)]
    assert errs[-1] < 5e-15 and errs[1] < errs[0] / 100


def test_phiks_ref_scalar_squaring():
    a, tau, v = -90.0, 0.1, 1.3
    r = phiks_ref.same([np.array([[a]])], tau, np.array([v]), 4, 5, 12, nscales=3)
    for L in range(3):
        z = tau * a / 2 ** L
        for l in range(5):
            ref = (math.exp(z) if l == 0 else phi_closed(l, z)) * v
            assert abs(r[5 * L + l][0] - ref) < 2e-14 * max(abs(ref), 1e-3)


def test_phiks_ref_scales_match_fresh_calls():
    wl = wk.adr3d_lincomb(p=4, dims=(9, 10, 11), nscales=3)
    r = phiks_ref.lincomb(wl.A, wl.tau, wl.vs, 4, 6, nscales=3)
    for L in range(3):
        assert rel(r[L], dense.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) < 1e-13


# ---------------------------------------------------------------- parameters
def _validation_case(n, d):
    A = (1 + 1j) / 100 * wk.fd_adr_dirichlet(n, 1.0, 0.0)
    x = np.arange(1, n + 1) / (n + 1)
    vn = np.linalg.norm(x * (1 - x)) ** d * 4096 * math.sqrt(2)
    return params.kron_sum_rect([A] * d, 1.0), vn


@pytest.mark.slow
def test_parameter_table_soft():
    """Table 1 (Sec. 4.1), soft: the unstated contour constants move single
    entries by one s step, so require |dT| <= p and |ds| <= 3 everywhere and an
    exact T# on at least 12 of the 16 entries."""
    tab = json.load(open(os.path.join(GOLD, "validation_table.json")))
    p = tab["p"]
    exact = 0
    for mode in ("same", "lincomb"):
        for e in tab[mode]:
            rect, vn = _validation_case(e["n"], e["d"])
            vnorms = [vn] if mode == "same" else [0.0] + [vn] * p
            got = params.select(rect, p, mode, vnorms, nscales=tab["nscales_in_count"])
            assert abs(got.tcount - e["T"]) <= p and abs(got.s - e["s"]) <= 3, (mode, e, got)
            exact += got.tcount == e["T"]
    assert exact >= 12


def test_selected_parameters_meet_accuracy():
    wl = wk.adr3d_lincomb(p=4, dims=(10, 11, 12))
    vn = [np.linalg.norm(v) for v in wl.vs]
    pr = params.select(params.kron_sum_rect(wl.A, wl.tau), 4, "lincomb", vn, nscales=3)
    r = phiks_ref.lincomb(wl.A, wl.tau, wl.vs, pr.s, pr.q, nscales=3)
    for L in range(3):
        assert rel(r[L], dense.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) < 1e-13
    wl = wk.small_same(12, p=3)
    pr = params.select(params.kron_sum_rect(wl.A, wl.tau), 3, "same", [np.linalg.norm(wl.vs[0])])
    r = phiks_ref.same(wl.A, wl.tau, wl.vs[0], 3, pr.s, pr.q)
    ex = dense.same(wl.A, wl.tau, wl.vs[0], 3)
    for l in range(4):
        assert rel(r[l], ex[l]) < 1e-13
    # a tighter tolerance never picks fewer Tucker operators
    loose = params.select(params.kron_sum_rect(wl.A, wl.tau), 3, "same", [np.linalg.norm(wl.vs[0])], tol=1e-8)
    assert loose.tcount <= pr.tcount


def test_numerical_range_rectangle_contains_spectrum_and_range():
    rng = np.random.default_rng(5)
    A = wk.fd_adr_dirichlet(15, 1.0, -20.0, 1.0)
    xlo, xhi, ylo, yhi = params.numerical_range_rect(A)
    for _ in range(200):
        x = rng.standard_normal(15) + 1j * rng.standard_normal(15)
        r = np.vdot(x, A @ x) / np.vdot(x, x)
        assert xlo - 1e-9 <= r.real <= xhi + 1e-9 and ylo - 1e-9 <= r.imag <= yhi + 1e-9


def _scalar_remainder(w, q, l, rule="gll"):
    """|R_q(f_l(., w))| for a scalar w: the exact integral
    int_0^1 t^(l-1)/(l-1)! exp((1-t) w) dt (= phi_l(w)) minus the rule, in
    40-digit arithmetic (nodes and weights as the oracle stores them)."""
    nodes, weights = quadrature.rule(rule, q)
    wm = mp.mpc(w)
    f = lambda t: t ** (l - 1) / mp.factorial(l - 1) * mp.exp((1 - t) * wm)
    with mp.workdps(40):
        exact = mp.quad(f, [0, 1])
        approx = mp.fsum(mp.mpf(float(c)) * f(mp.mpf(float(t))) for t, c in zip(nodes, weights))
        return float(abs(exact - approx))


@pytest.mark.parametrize("w", [-5.0, -1.5 + 2j, 0.3, -20.0, 3.0, -0.5j, -40.0, 8.0, -10 + 10j])
@pytest.mark.parametrize("rule", ["gll", "gl"])
def test_remainder_bound_is_the_crouzeix_palencia_constant_times_the_scalar_remainder(w, rule):
    """For a scalar operator the contour integral of eq. (CPestimate) is the
    quadrature remainder itself (Cauchy), so the estimate must be (1 + sqrt 2)
    times |R_q(f_l(., w/2^s))|: this pins the constant, the kernel k_q, f_l,
    the contour and the scaling by 2^s at once, and shows the estimate
    dominates the remainder.  Cases whose remainder is below 1e-12 are left
    out (the rule's stored nodes and weights carry errors of order 1e-16)."""
    w = complex(w)
    rect = (w.real, w.real, w.imag, w.imag)
    checked = 0
    for s in (0, 2):
        for q in (3, 5, 8, 12):
            b = params.remainder_bounds(rect, s, q, 3, rule)
            for l in range(1, 4):
                true = _scalar_remainder(w / 2 ** s, q, l, rule)
                if true < 1e-12:
                    continue
                ratio = b[l - 1] / true
                assert 2.40 <= ratio <= 2.42, (w, s, q, l, b[l - 1], true)
                checked += 1
    assert checked >= 3


def test_remainder_bound_dominates_on_a_diagonal_operator():
    """A diagonal K (eigenvalues on a segment of the real axis and on a
    vertical segment): the estimate bounds ||R_q(f_l(., K))||_2 = max_i
    |R_q(f_l(., lambda_i))| and exceeds it by at most (1 + sqrt 2) times the
    largest remainder on the rectangle's sampled boundary."""
    for lam in (np.linspace(-30.0, -0.5, 7), 1j * np.linspace(-6.0, 6.0, 5) - 2.0):
        rect = (lam.real.min(), lam.real.max(), lam.imag.min(), lam.imag.max())
        for s, q in ((0, 6), (1, 5), (3, 4)):
            b = params.remainder_bounds(rect, s, q, 2)
            for l in (1, 2):
                rem = [_scalar_remainder(x / 2 ** s, q, l) for x in lam]
                on_boundary = [_scalar_remainder(x / 2 ** s, q, l) for x in params.rect_boundary(rect)[::8]]
                assert b[l - 1] >= max(rem), (s, q, l)
                assert b[l - 1] <= 2.42 * max(on_boundary + rem) * 1.05, (s, q, l)


@pytest.mark.parametrize("rule", ["gll", "gl"])
def test_tucker_count_is_the_operators_the_restatement_applies(rule, monkeypatch):
    """eq. (Tpsv) / eq. (Tlcp) count one Tucker operator per quadrature node,
    p per squaring step and one per scale; the step-by-step restatement
    applies exactly that many, less the free theta = 1 node of GLL (one
    operator in the same-vector task, p in the linear combination)."""
    calls = [0]
    orig = phiks_ref.tucker

    def counting(V, L):
        calls[0] += 1
        return orig(V, L)
    monkeypatch.setattr(phiks_ref, "tucker", counting)
    A = [wk.fd_adr_dirichlet(4, 1.0, 1.0), wk.fd_adr_dirichlet(3, 1.0, 0.0)]
    for p, s, q, ns in [(3, 0, 5, 1), (3, 2, 6, 2), (4, 3, 4, 3), (1, 1, 7, 2)]:
        calls[0] = 0
        phiks_ref.same(A, 1e-3, wk.normal(1, 12), p, s, q, nscales=ns, rule=rule)
        assert calls[0] == params.tucker_count("same", s, ns, q, p) - (rule == "gll")
        calls[0] = 0
        phiks_ref.lincomb(A, 1e-3, [wk.normal(2 + l, 12) for l in range(p + 1)], s, q, nscales=ns, rule=rule)
        assert calls[0] == params.tucker_count("lincomb", s, ns, q, p) - (p if rule == "gll" else 0)
