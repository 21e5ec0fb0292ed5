"""Served form: requests that overlap on the GPU give the same result as
each request alone (continuous batching changes timing, not arithmetic), and
a served result agrees with the FP64 restatement."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import rel_inf  # noqa: E402

import bench  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("dtype", ["fp64", "bf16x3"])
def test_served_results_equal_alone_and_in_the_mix(dtype, graphs):
    arrivals, specs = wk.served_trace(24, 20000.0, size_cap=160, classes=("ac", "adr", "bru"))
    specs = [(c, min(n, 48) if c == "adr" else n, p) for c, n, p in specs]
    tol = bench.PRECISION_TOL[dtype]
    reqs, plans, n_app = bench.build_served(pk, torch, arrivals, specs, dtype, tol)
    bench.warm_served(pk, torch, reqs)
    lat, qd, mk = pk.phiks_serve_trace(reqs, arrivals, slots=6, hbm_budget=1 << 30, graphs=graphs)
    assert len(lat) == len(reqs) and all(l > 0 for l in lat) and mk > 0
    mixed = [[x["out"].clone() for x in apps] for apps in reqs]
    for apps in reqs:                      # each request alone, one after another
        for x in apps:
            x["out"].fill_(float("nan"))
            kw = dict(vnorms=x["vnorms"])
            if "tol" in x:
                kw["tol"] = x["tol"]
            pk.phiks_apply_ex(x["plan"], x["tau"], x["p"], x["v"], x["out"], None, **kw)
            torch.cuda.synchronize()
    for apps, outs in zip(reqs, mixed):
        for x, o in zip(apps, outs):
            assert torch.equal(x["out"], o)
    # the first request of each class against the oracle's Taylor action
    done = set()
    for (cls, n, p), apps in zip(specs, reqs):
        if cls in done:
            continue
        done.add(cls)
        A = wk.ac_operator(n) if cls == "ac" else (
            [wk.fd_adr_dirichlet(n, 1.0, a, 2.0 / 3) for a in (10.0, -20.0, 5.0)] if cls == "adr"
            else wk.brusselator_operators(n)[0])
        x = apps[0]
        vs = [v.double().cpu().numpy() for v in x["v"]]
        ref = ta.lincomb(A, x["tau"], vs)
        tol_cmp = 1e-12 if dtype == "fp64" else 1e-4
        assert rel_inf(x["out"].double().cpu().numpy(), ref) < tol_cmp, cls
    for pl in plans.values():
        pl.close()
