"""Exponential integrators on the ADR problem of Sec. 4.2, pinned to the
errors the paper prints (Fig. ord1 / ord2, tests/golden), first for the
oracle (CPU) and then for the CUDA path through phiks_integrate (GPU)."""
import json
import os

import numpy as np
import pytest

import workloads as wk
from oracle import integrators as it

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "adr_integrator_errors.json")))
N, EPS, ALPHA, T = GOLD["n"], GOLD["eps"], GOLD["alpha"], GOLD["T"]


def _A():
    return [wk.fd_adr_dirichlet(N, EPS, ALPHA) for _ in range(3)]


@pytest.mark.parametrize("scheme,steps,rtol", [("expeuler", 300, 1e-7), ("expeuler", 700, 1e-7),
                                               ("etd2rk", 200, 1e-5), ("etd2rk", 400, 1e-5)])
def test_oracle_reproduces_printed_errors(scheme, steps, rtol):
    u = it.integrate(_A(), N, EPS, ALPHA, T, steps, scheme)
    err = it.relative_error(u, N, T)
    ref = GOLD[scheme][str(steps)]
    assert abs(err - ref) <= rtol * ref, (err, ref)


def test_orders_of_convergence():
    e = [it.relative_error(it.integrate(_A(), N, EPS, ALPHA, T, s, "expeuler"), N, T) for s in (300, 600)]
    assert 1.9 < e[0] / e[1] < 2.1
    e = [it.relative_error(it.integrate(_A(), N, EPS, ALPHA, T, s, "etd2rk"), N, T) for s in (200, 400)]
    assert 3.8 < e[0] / e[1] < 4.2


AC = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ac_exprk3_errors.json")))


@pytest.fixture(scope="module")
def ac_problem():
    A, u0 = wk.ac_paper(AC["n"], AC["eps"])
    g = it.ac_g(AC["eps"])
    ref = it.integrate_problem([A], g, u0, 0.0, AC["T"], AC["ref_steps"], "exprk4s6")
    return A, u0, g, ref


@pytest.mark.parametrize("steps,rtol", [(100, 1e-4), (200, 1e-4), (150, 1.5e-3)])
def test_oracle_ac_exprk3_reproduces_printed_errors(ac_problem, steps, rtol):
    """Sec. 4.3, Fig. ord3: expRK3 against the expRK4s6 reference; the printed
    series agree with each other to 5e-4 at 125-175 steps, to 1e-5 at 100 and
    200."""
    A, u0, g, ref = ac_problem
    u = it.integrate_problem([A], g, u0, 0.0, AC["T"], steps, "exprk3")
    err = it.rel_inf(u, ref)
    gold = AC["exprk3"][str(steps)]
    assert abs(err - gold) <= rtol * gold, (err, gold)


def test_orders_fourth_order_schemes_block_diagonal():
    """Brusselator (block-diagonal K, Sec. 4.4) on a 6^3 grid to T = 1: the
    error ratio on halving the step is 2^order."""
    blocks, w0 = wk.brusselator3d(6)
    g = it.bruss_g(1.0, 3.0)
    ref = it.integrate_problem(blocks, g, w0, 0.0, 1.0, 160, "exprk4s6")
    for sch, lo, hi in [("exprk4s5", 14.0, 18.0), ("exprk4s6", 14.0, 18.0), ("exprk3", 7.0, 9.5)]:
        e = [it.rel_inf(it.integrate_problem(blocks, g, w0, 0.0, 1.0, s, sch), ref) for s in (10, 20)]
        assert lo < e[0] / e[1] < hi, (sch, e)


@pytest.mark.parametrize("scheme", ["expeuler", "etd2rk", "exprk3", "exprk4s5", "exprk4s6"])
def test_steady_states_are_kept(scheme):
    """Homogeneous steady states of the semidiscrete problems (the Neumann
    Laplacians annihilate constants): Allen-Cahn u = 1, where K 1 = 1/eps^2 =
    -g(1), and the Brusselator (u, v) = (a, b/a), where -(b+1) a + a + a^2 b/a
    = 0 and b a - a^2 b/a = 0.  Every stage of eq. (RK) then equals u_n
    (exp(X) = I + X phi_1(X)), so each scheme keeps them to rounding; a wrong
    sign or role in g, or a dropped phi_1 g term, does not."""
    A, u0 = wk.ac_paper(9, 0.05)
    one = np.ones_like(u0)
    out = it.integrate_problem([A], it.ac_g(0.05), one, 0.0, 1e-4, 4, scheme)
    assert np.abs(out - one).max() < 1e-11
    blocks, w0 = wk.brusselator3d(5)
    N = w0.size // 2
    w = np.concatenate([np.full(N, 1.0), np.full(N, 3.0)])
    out = it.integrate_problem(blocks, it.bruss_g(1.0, 3.0), w, 0.0, 0.5, 4, scheme)
    assert np.abs(out - w).max() < 1e-11


def test_block_diagonal_phi_actions_vs_dense():
    """The block-by-block phi-actions equal the top rows of one dense
    exponential of the augmented matrix of the whole block-diagonal K (Sec. 2
    augmented-matrix statement; scipy's expm)."""
    from scipy.linalg import expm
    from oracle import kron
    blocks, w0 = wk.brusselator3d(3)
    K = np.zeros((54, 54))
    K[:27, :27] = kron.kron_sum_dense(blocks[0])
    K[27:, 27:] = kron.kron_sum_dense(blocks[1])
    rng = np.random.default_rng(3)
    v1, v2 = rng.standard_normal(54), rng.standard_normal(54)
    tau = 0.3
    B = np.zeros((56, 56))
    B[:54, :54] = tau * K
    B[:54, 54] = v2
    B[:54, 55] = v1
    B[54, 55] = 1.0
    ref = (expm(B) @ np.concatenate([w0, [0.0, 1.0]]))[:54]
    got = it.lc(blocks, tau, [w0, v1, v2])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.gpu
@pytest.mark.parametrize("scheme,steps", [("expeuler", 300), ("etd2rk", 200)])
def test_gpu_integrator_matches_paper_and_oracle(scheme, steps):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    A = _A()
    plan = pk.Plan(A)
    u = torch.from_numpy(np.reshape(it.adr_u0(N), -1, order="F").copy()).cuda()
    sch = pk.PHIKS_EXP_EULER if scheme == "expeuler" else pk.PHIKS_ETD2RK
    pk.phiks_integrate(plan.handle, (N, N, N), sch, pk.PHIKS_NL_ADR_EXACT, EPS, ALPHA, 0.0, T, steps, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    err = it.relative_error(got, N, T)
    ref = GOLD[scheme][str(steps)]
    assert abs(err - ref) <= 1e-5 * ref, (err, ref)
    orc = it.integrate(A, N, EPS, ALPHA, T, steps, scheme)
    assert float(np.abs(got - orc).max() / np.abs(orc).max()) < 1e-12
    plan.close()


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    return torch, pk


@pytest.mark.gpu
def test_gpu_ac_exprk3_matches_paper_and_oracle(ac_problem):
    """Sec. 4.3 on the device: expRK3 at 100 steps gives the printed error
    against the oracle's expRK4s6 reference, and the oracle's expRK3 state."""
    torch, pk = _gpu()
    A, u0, g, ref = ac_problem
    plan = pk.Plan(A)
    u = torch.from_numpy(u0.copy()).cuda()
    pk.phiks_integrate_blocks([plan], pk.PHIKS_EXPRK3, pk.PHIKS_NL_ALLEN_CAHN, 0.0, AC["T"], 100, u,
                              eps=AC["eps"])
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    err = it.rel_inf(got, ref)
    assert abs(err - AC["exprk3"]["100"]) <= 1e-4 * AC["exprk3"]["100"], err
    orc = it.integrate_problem([A], g, u0, 0.0, AC["T"], 100, "exprk3")
    assert it.rel_inf(got, orc) < 1e-12
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("scheme,steps", [("exprk4s6", 40), ("exprk4s5", 30), ("etd2rk", 40),
                                          ("expeuler", 40)])
def test_gpu_ac_schemes_match_oracle(ac_problem, scheme, steps):
    torch, pk = _gpu()
    A, u0, g, _ = ac_problem
    plan = pk.Plan(A)
    u = torch.from_numpy(u0.copy()).cuda()
    pk.phiks_integrate_blocks([plan], pk.SCHEMES[scheme], pk.PHIKS_NL_ALLEN_CAHN, 0.0, AC["T"], steps, u,
                              eps=AC["eps"])
    torch.cuda.synchronize()
    orc = it.integrate_problem([A], g, u0, 0.0, AC["T"], steps, scheme)
    assert it.rel_inf(u.cpu().numpy(), orc) < 1e-12
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("scheme", ["exprk4s5", "exprk4s6", "exprk3"])
@pytest.mark.parametrize("dtype_name", ["fp64", "fp64emu"])
def test_gpu_brusselator_block_diagonal(scheme, dtype_name):
    """Block-diagonal K = diag(K_1, K_2) (Sec. 4.4, eq. ODE2) on an 8^3 grid,
    two plans, 10 steps to T = 1, against the oracle."""
    torch, pk = _gpu()
    blocks, w0 = wk.brusselator3d(8)
    dt = pk.DTYPES[dtype_name]
    plans = [pk.Plan(blocks[0], dt), pk.Plan(blocks[1], dt)]
    w = torch.from_numpy(w0.copy()).cuda()
    pk.phiks_integrate_blocks(plans, pk.SCHEMES[scheme], pk.PHIKS_NL_BRUSSELATOR, 0.0, 1.0, 10, w,
                              a=1.0, b=3.0)
    torch.cuda.synchronize()
    for p in plans:
        pk.phiks_device_status(p.handle)
    orc = it.integrate_problem(blocks, it.bruss_g(1.0, 3.0), w0, 0.0, 1.0, 10, scheme)
    err = it.rel_inf(w.cpu().numpy(), orc)
    print(scheme, dtype_name, "%.2e" % err)
    assert err < 1e-12
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_gpu_integrator_graph_replay_same_result(ac_problem):
    """phiks_options.graph inside the integrator: every stage call replays a
    captured graph from the second step on; the state equals plain calls'."""
    torch, pk = _gpu()
    A, u0, _, _ = ac_problem
    plan = pk.Plan(A)
    st = torch.cuda.Stream()
    outs = []
    for graph in (0, 1):
        u = torch.from_numpy(u0.copy()).cuda()
        torch.cuda.synchronize()
        pk.phiks_integrate_blocks([plan], pk.PHIKS_EXPRK4S6, pk.PHIKS_NL_ALLEN_CAHN, 0.0, AC["T"], 12, u,
                                  eps=AC["eps"], stream=st, graph=graph)
        torch.cuda.synchronize()
        outs.append(u.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    plan.close()
