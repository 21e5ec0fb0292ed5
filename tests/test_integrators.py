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
