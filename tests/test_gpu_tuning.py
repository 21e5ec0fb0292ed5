"""The fused small-slab Tucker kernel and the autotuner's search space.

* The fused kernel (all d modes of a Tucker operator and the batch's input
  combinations in one launch, intermediates in shared memory) against the
  oracle's Tucker operator (Sec. 2, Lemma 1) and the oracle's step-by-step
  phiks at the same (s, q) (Sec. 3.1, 3.2), for every rows-per-CTA choice,
  ragged shapes and d = 2 .. 4.
* Every tuning the autotuner may choose (tile shapes, mode orders, fused or
  mode-by-mode) gives the untuned result to rounding, and the tuner's file
  cache returns what it stored.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import dense, kron, phiks_ref  # noqa: E402

from gpu_util import dev, rel_inf, run_workload  # noqa: E402

SPLIT_CALL_TOL = {pk.PHIKS_TF32: 2e-2, pk.PHIKS_TF32X3: 8e-5, pk.PHIKS_BF16X3: 8e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


@pytest.mark.parametrize("dims", [(32, 32), (10, 11, 12), (33, 17, 5), (9, 4, 3, 5), (64, 64, 64), (7, 130)])
@pytest.mark.parametrize("rows", [1, 2, 4, 8])
def test_fused_tucker_vs_oracle(dims, rows):
    rng = np.random.default_rng(sum(dims) + rows)
    plan = pk.Plan([np.eye(m) for m in dims])
    pk.phiks_set_tuning(plan.handle, fused=1, fused_rows=rows)
    N = int(np.prod(dims))
    V = rng.standard_normal(N)
    Ls = [rng.standard_normal((m, m)) / np.sqrt(m) for m in dims]
    W = torch.full((N,), float("nan"), device="cuda", dtype=torch.float64)
    pk.phiks_tucker(plan.handle, dev(V), W, [dev(L.ravel(order="F")) for L in Ls])
    torch.cuda.synchronize()
    ref = kron.vec(kron.tucker(kron.unvec(V, dims), Ls))
    assert rel_inf(W.cpu().numpy(), ref) < 1e-14
    plan.close()


@pytest.mark.parametrize("dims", [(32, 32), (10, 11, 12), (33, 17, 5), (9, 4, 3, 5)])
@pytest.mark.parametrize("mode", ["same", "lincomb"])
def test_fused_calls_match_restatement(dims, mode):
    """Whole phiks calls with every batch fused (quadrature nodes, squaring
    levels, scale outputs; the deferred combinations in the next launch)
    against the oracle's step-by-step phiks at the forced (s, q)."""
    alpha = (1.0, -2.0, 3.0, -0.5)[: len(dims)]
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip(dims, alpha)]
    N = int(np.prod(dims))
    tau = 2e-4
    if mode == "same":
        wl = wk.Workload("t", A, tau, 3, "same", 2, [wk.normal(11, N)])
    else:
        wl = wk.Workload("t", A, tau, 3, "lincomb", 2, [wk.normal(20 + l, N) for l in range(4)])
    outs = {}
    for fused in (0, 1):
        plan = pk.Plan(A)
        pk.phiks_set_tuning(plan.handle, fused=fused)
        tdt = torch.float64
        if mode == "same":
            vs = [dev(wl.vs[0])]
            out = torch.full((2 * 4 * N,), float("nan"), device="cuda", dtype=tdt)
        else:
            vs = [dev(v) for v in wl.vs]
            out = torch.full((2 * N,), float("nan"), device="cuda", dtype=tdt)
        plan.apply(tau, 3, vs, out, nscales=2, force_s=3, force_q=6)
        torch.cuda.synchronize()
        outs[fused] = out.cpu().numpy().reshape(-1, N)
        plan.close()
    if mode == "same":
        ref = phiks_ref.same(A, tau, wl.vs[0], 3, 3, 6, nscales=2)
    else:
        ref = np.stack(phiks_ref.lincomb(A, tau, wl.vs, 3, 6, nscales=2))
    for k in range(ref.shape[0]):
        assert rel_inf(outs[1][k], ref[k]) < 1e-13, k
        assert rel_inf(outs[1][k], outs[0][k]) < 1e-13, k


def test_fused_small_same_vector_vs_dense_oracle():
    """The d = 2, n = 32 same-vector workload (phi_0..phi_3) through the
    fused kernel (chosen by size) against the dense oracle."""
    wl = wk.small_same(32)
    plan = pk.Plan(wl.A)
    assert pk.phiks_get_tuning(plan.handle).fused == -1
    plan.close()
    out, plan = run_workload(wl)
    ex = dense.same(wl.A, wl.tau, wl.vs[0], wl.p)
    for k in range(4):
        assert rel_inf(out[k], ex[k]) < 1e-12
    plan.close()


def _tunings(dtype, d):
    import itertools
    if dtype == pk.PHIKS_FP64:
        ts = [dict(fused=0, fp64_tile=t, mode_order=list(o))
              for t in (1, 2) for o in itertools.permutations(range(d))]
        ts += [dict(fused=1, fused_rows=r) for r in (1, 2, 4, 8)]
        return ts
    if dtype == pk.PHIKS_FP64_EMU:
        return [dict(emu_cols=c) for c in (16, 32)]
    return [dict(split_ntiles=m) for m in (1, 2, 4)]


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU, pk.PHIKS_BF16X3, pk.PHIKS_TF32X3])
def test_every_tuning_reproduces_the_default(dtype):
    dims = (32, 24, 40) if dtype != pk.PHIKS_FP64_EMU else (32, 24, 40)
    wl = wk.adr3d_lincomb(p=3, dims=dims, nscales=2)
    f64 = dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU)
    vs = [v if f64 else v.astype(np.float32).astype(np.float64) for v in wl.vs]
    wl = wk.Workload("t", wl.A, wl.tau, 3, "lincomb", 2, vs)
    base, plan = run_workload(wl, dtype=dtype)
    s, q, _, _ = plan.last_params()
    plan.close()
    tol = 1e-13 if f64 else SPLIT_CALL_TOL[dtype] / 4
    for t in _tunings(dtype, len(dims)):
        tdt = torch.float64 if f64 else torch.float32
        plan = pk.Plan(wl.A, dtype)
        pk.phiks_set_tuning(plan.handle, **t)
        out = torch.full((2 * wl.N,), float("nan"), device="cuda", dtype=tdt)
        plan.apply(wl.tau, 3, [dev(v, tdt) for v in vs], out, nscales=2, force_s=s, force_q=q)
        torch.cuda.synchronize()
        pk.phiks_device_status(plan.handle)
        got = out.double().cpu().numpy().reshape(2, wl.N)
        plan.close()
        for L in range(2):
            assert rel_inf(got[L], base[L]) < tol, (t, L)


def test_set_tuning_rejects_bad_values():
    plan = pk.Plan([np.eye(8), np.eye(8)])
    for bad in (dict(fused=2), dict(fused_rows=3), dict(fp64_tile=3), dict(emu_cols=24), dict(split_ntiles=3),
                dict(mode_order=[0, 0]), dict(mode_order=[0, 2])):
        with pytest.raises(pk.PhiksError) as e:
            pk.phiks_set_tuning(plan.handle, **bad)
        assert e.value.status == 1, bad
    plan.close()
    big = pk.Plan([np.eye(8)] * 2, pk.PHIKS_BF16X3)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_set_tuning(big.handle, fused=1)
    assert e.value.status == 3
    big.close()


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU])
def test_autotune_and_its_cache(tmp_path, dtype):
    cache = tmp_path / "tune.txt"
    os.environ["PHIKS_TUNE_CACHE"] = str(cache)
    try:
        wl = wk.small_same(32) if dtype == pk.PHIKS_FP64 else wk.adr3d_lincomb(p=3, dims=(32, 32, 32))
        nv = 1 if wl.mode == "same" else wl.p + 1
        plan = pk.Plan(wl.A, dtype)
        t, ms = pk.phiks_autotune(plan.handle, wl.tau, wl.p, nv, reps=3)
        assert ms > 0
        lines = cache.read_text().strip().splitlines()
        assert len(lines) == 1 and " | " in lines[0] and "ms=" in lines[0]
        cur = pk.phiks_get_tuning(plan.handle)
        assert cur.as_dict(len(wl.A)) == t.as_dict(len(wl.A))
        plan.close()
        plan = pk.Plan(wl.A, dtype)        # a fresh plan takes the cached choice
        t2, ms2 = pk.phiks_autotune(plan.handle, wl.tau, wl.p, nv, reps=3)
        assert t2.as_dict(len(wl.A)) == t.as_dict(len(wl.A))
        assert abs(ms2 - ms) <= 1e-6 * ms
        assert len(cache.read_text().strip().splitlines()) == 1
        # the tuned plan still computes the oracle's result
        if wl.mode == "same":
            out = torch.empty(4 * wl.N, device="cuda", dtype=torch.float64)
            plan.apply(wl.tau, wl.p, [dev(wl.vs[0])], out)
            ex = dense.same(wl.A, wl.tau, wl.vs[0], wl.p)
        else:
            out = torch.empty(wl.N, device="cuda", dtype=torch.float64)
            plan.apply(wl.tau, wl.p, [dev(v) for v in wl.vs], out)
            from oracle import taylor_action as ta
            ex = ta.lincomb(wl.A, wl.tau, wl.vs)[None, :]
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, wl.N)
        for k in range(got.shape[0]):
            assert rel_inf(got[k], ex[k]) < 1e-12
        plan.close()
    finally:
        del os.environ["PHIKS_TUNE_CACHE"]
