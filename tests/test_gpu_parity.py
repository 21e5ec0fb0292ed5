"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-12 relative infinity-norm for the FP64 path against the exact
phi-actions (the accuracy the tolerance 2^-53 of Sec. 3.3 targets; the
paper's own FP64 results sit at 5e-15 .. 3e-12 of kiops, Sec. 4.1), and
1e-13 against the oracle's step-by-step restatement at the same (s, q),
where only rounding differs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import dense, expm as oexpm, kron, params, phiks_ref  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import dev, rel_inf, run_workload  # noqa: E402

TOL_EXACT = 1e-12
TOL_REF = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


def _exact_same(wl):
    rows = []
    for L in range(wl.nscales):
        r = dense.same(wl.A, wl.tau / 2 ** L, wl.vs[0], wl.p)
        rows += list(r[1:] if wl.skip_phi0 else r)
    return np.stack(rows)


def _exact_lincomb(wl, fn=dense.lincomb):
    return np.stack([fn(wl.A, wl.tau, wl.vs, 2.0 ** -L) for L in range(wl.nscales)])


def test_small_same_vector_d2_n32():
    """phi_0..phi_3 of the 2D FD Laplacian plus advection, N = 1024."""
    wl = wk.small_same(32)
    out, plan = run_workload(wl)
    ex = _exact_same(wl)
    for k in range(out.shape[0]):
        assert rel_inf(out[k], ex[k]) < TOL_EXACT, k
    s, q, T, _ = plan.last_params()
    ref = params.select(params.kron_sum_rect(wl.A, wl.tau), wl.p, "same", [np.linalg.norm(wl.vs[0])])
    assert (s, q, T) == (ref.s, ref.q, ref.tcount)


def test_lincomb_3d_scales_small():
    wl = wk.adr3d_lincomb(p=4, dims=(10, 11, 12))
    out, _ = run_workload(wl)
    ex = _exact_lincomb(wl)
    for L in range(3):
        assert rel_inf(out[L], ex[L]) < TOL_EXACT, L


@pytest.mark.parametrize("dims", [(70, 40), (33, 17, 5), (9, 4, 3, 5), (130,)])
@pytest.mark.parametrize("rule", [0, 1])
def test_fixed_parameters_match_restatement(dims, rule):
    """At a forced (s, q) the kernels must reproduce the oracle's step-by-step
    phiks to rounding: ragged sizes over several tiles (TI = 32, TC = 64)."""
    alpha = (1.0, -2.0, 3.0, -0.5)[: len(dims)]
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip(dims, alpha)]
    N = int(np.prod(dims))
    tau = 2e-4
    v = wk.normal(11, N)
    rname = "gll" if rule == 0 else "gl"
    wl = wk.Workload("t", A, tau, 3, "same", 2, [v])
    out, _ = run_workload(wl, force_s=2, force_q=6, rule=rule)
    ref = phiks_ref.same(A, tau, v, 3, 2, 6, nscales=2, rule=rname)
    for k in range(out.shape[0]):
        assert rel_inf(out[k], ref[k]) < TOL_REF, k
    vs = [wk.normal(20 + l, N) for l in range(4)]
    wl = wk.Workload("t", A, tau, 3, "lincomb", 3, vs)
    out, _ = run_workload(wl, force_s=3, force_q=5, rule=rule)
    ref = phiks_ref.lincomb(A, tau, vs, 3, 5, nscales=3, rule=rname)
    for k in range(3):
        assert rel_inf(out[k], ref[k]) < TOL_REF, k


def test_lincomb_full_size_bench_configuration():
    """d = 3, n = 64^3 (N = 262144), p = 4, three scales: the workload and the
    launch configuration the benchmark times, against the oracle's Taylor
    action (O3) on every output element."""
    wl = wk.adr3d_lincomb(64)
    out, plan = run_workload(wl, no_cache=1)
    for L in range(3):
        ex = ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)
        assert rel_inf(out[L], ex) < TOL_EXACT, L


def test_edge_cases_zero_vectors_and_exp_only():
    wl = wk.adr3d_lincomb(p=3, dims=(12, 9, 10), nscales=2)
    # v_0 and v_2 absent
    vs = [None, wl.vs[1], None, wl.vs[3]]
    w2 = wk.Workload("t", wl.A, wl.tau, 3, "lincomb", 2, vs)
    out, _ = run_workload(w2)
    for L in range(2):
        assert rel_inf(out[L], dense.lincomb(wl.A, wl.tau, vs, 2.0 ** -L)) < TOL_EXACT
    # p = 0: exponential only, two scales
    w3 = wk.Workload("t", wl.A, wl.tau, 0, "same", 2, [wl.vs[0]])
    out, _ = run_workload(w3)
    for L in range(2):
        ex = dense.same(wl.A, wl.tau / 2 ** L, wl.vs[0], 0)[0]
        assert rel_inf(out[L], ex) < TOL_EXACT
    # skip_phi0, negative tau
    w4 = wk.Workload("t", wl.A, -wl.tau / 4, 2, "same", 1, [wl.vs[0]], skip_phi0=True)
    out, _ = run_workload(w4)
    ex = dense.same(wl.A, -wl.tau / 4, wl.vs[0], 2)
    assert rel_inf(out[0], ex[1]) < TOL_EXACT and rel_inf(out[1], ex[2]) < TOL_EXACT


def test_d1_and_unit_modes():
    A = [wk.fd_adr_dirichlet(1, 1.0, 0.0), wk.fd_adr_dirichlet(37, 1.0, 2.0), np.array([[-3.0]])]
    N = 37
    v = wk.uniform(5, N)
    wl = wk.Workload("t", A, 1e-3, 2, "same", 1, [v])
    out, _ = run_workload(wl)
    ex = dense.same(A, 1e-3, v, 2)
    for k in range(3):
        assert rel_inf(out[k], ex[k]) < TOL_EXACT
    A1 = [wk.fd_adr_dirichlet(50, 1.0, -1.0)]
    wl = wk.Workload("t", A1, 2e-3, 3, "lincomb", 1, [wk.normal(l, 50) for l in range(4)])
    out, _ = run_workload(wl)
    assert rel_inf(out[0], dense.lincomb(A1, 2e-3, wl.vs)) < TOL_EXACT


def test_caller_workspace_and_determinism():
    wl = wk.adr3d_lincomb(p=2, dims=(20, 30, 11), nscales=2)
    plan = pk.Plan(wl.A)
    vs = [dev(v) for v in wl.vs]
    o1 = torch.empty(2 * wl.N, device="cuda", dtype=torch.float64)
    o2 = torch.empty_like(o1)
    o3 = torch.empty_like(o1)
    plan.apply(wl.tau, 2, vs, o1, nscales=2)
    plan.apply(wl.tau, 2, vs, o2, nscales=2)
    ws_bytes = pk.phiks_workspace_size(plan.handle, 2, 3, 2)
    ws = torch.empty(ws_bytes, device="cuda", dtype=torch.uint8)
    plan.apply(wl.tau, 2, vs, o3, nscales=2, workspace=ws.data_ptr(), workspace_bytes=ws_bytes)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(o1, o3)
    with pytest.raises(pk.PhiksError):
        plan.apply(wl.tau, 2, vs, o3, nscales=2, workspace=ws.data_ptr(), workspace_bytes=ws_bytes - 8)


def test_caller_norms_skip_the_sync_and_agree():
    wl = wk.adr3d_lincomb(p=4, dims=(16, 16, 16), nscales=1)
    plan = pk.Plan(wl.A)
    vs = [dev(v) for v in wl.vs]
    o1 = torch.empty(wl.N, device="cuda", dtype=torch.float64)
    o2 = torch.empty_like(o1)
    plan.apply(wl.tau, 4, vs, o1, nscales=1)
    plan.apply(wl.tau, 4, vs, o2, nscales=1, vnorms=[float(np.linalg.norm(v)) for v in wl.vs])
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)


@pytest.mark.parametrize("p,s", [(1, 0), (1, 2), (3, 0)])
def test_fp64_batched_lincomb_forced(p, s):
    """The FP64 path's batched form (all node operators in one batch, the
    combinations deferred), with and without squaring, against the oracle's
    restatement of the method with the same (s, q)."""
    dims = (12, 10, 8)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, (4.0, -2.0, 1.0))]
    N = int(np.prod(dims))
    vs = [wk.normal(60 + l, N) for l in range(p + 1)]
    wl = wk.Workload("t", A, 2e-3, p, "lincomb", 1, vs)
    out, plan = run_workload(wl, force_s=s, force_q=9)
    ref = phiks_ref.lincomb(A, 2e-3, vs, s, 9, nscales=1)
    assert rel_inf(out[0], ref[0]) < 1e-12
    plan.close()


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU])
def test_norms_that_change_the_selection(dtype):
    """Repeated calls with the same tau and p run first with the previous
    selection while the device norms are read back; a vector 1e8 times larger
    selects another (s, q) and must still give the result of its own
    selection."""
    wl = wk.small_same(32) if dtype == pk.PHIKS_FP64 else wk.adr3d_lincomb(p=4, dims=(64, 32, 64), nscales=1)
    plan = pk.Plan(wl.A, dtype)
    if wl.mode == "same":
        vs_small = [dev(wl.vs[0])]
        out = torch.empty((wl.p + 1) * wl.N, device="cuda", dtype=torch.float64)
    else:
        vs_small = [dev(v) for v in wl.vs]
        out = torch.empty(wl.N, device="cuda", dtype=torch.float64)
    vs_big = [x * 1e8 for x in vs_small]
    sel = []
    for vs in (vs_small, vs_small, vs_big, vs_big, vs_small):
        plan.apply(wl.tau, wl.p, vs, out, nscales=1)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, wl.N)
        scale = 1e8 if vs is vs_big else 1.0
        if wl.mode == "same":
            ex = _exact_same(wl) * scale
        else:
            ex = np.stack([ta.lincomb(wl.A, wl.tau, wl.vs, 1.0)]) * scale
        for k in range(got.shape[0]):
            assert rel_inf(got[k], ex[k]) < 1e-12, k
        s, q, T, _ = plan.last_params()
        norms = [float(np.linalg.norm(x.cpu().numpy())) for x in vs]
        ref = plan.select_params(wl.tau, wl.p, norms)
        assert (s, q) == (ref[0], ref[1])
        sel.append((s, q))
    assert sel[0] != sel[2], sel  # the large vectors do select differently
    plan.close()


@pytest.mark.parametrize("dims", [(5,), (70, 3), (33, 8, 17), (4, 3, 2, 5)])
def test_tucker_entry_point(dims):
    rng = np.random.default_rng(3)
    A = [np.eye(m) for m in dims]
    plan = pk.Plan(A)
    N = int(np.prod(dims))
    V = rng.standard_normal(N)
    Ls = [rng.standard_normal((m, m)) for m in dims]
    Lt = [dev(np.asfortranarray(L).ravel(order="F")) for L in Ls]
    W = torch.empty(N, device="cuda", dtype=torch.float64)
    pk.phiks_tucker(plan.handle, dev(V), W, Lt)
    torch.cuda.synchronize()
    ref = kron.vec(kron.tucker(kron.unvec(V, dims), Ls))
    assert rel_inf(W.cpu().numpy(), ref) < 1e-14


@pytest.mark.parametrize("n", [1, 5, 33, 70])
def test_expm_entry_point(n):
    rng = np.random.default_rng(n)
    Xs = [rng.standard_normal((n, n)) * s for s in (0.1, 1.0, 6.0)]
    Xs.append(1e-3 * wk.fd_adr_dirichlet(n, 1.0, -5.0))
    # column-major n x n matrices back to back
    X = dev(np.concatenate([x.ravel(order="F") for x in Xs]))
    E = torch.empty_like(X)
    pk.phiks_expm(X.view(len(Xs), n, n), E.view(len(Xs), n, n))
    torch.cuda.synchronize()
    got = E.cpu().numpy().reshape(len(Xs), n * n)
    for k, x in enumerate(Xs):
        ref = oexpm.expm_taylor(x).ravel(order="F")
        assert rel_inf(got[k], ref) < 1e-13 * max(1.0, np.abs(x).sum(axis=0).max())


def test_invalid_calls_report_errors():
    wl = wk.small_same(8)
    plan = pk.Plan(wl.A)
    v = dev(wl.vs[0])
    out = torch.empty(4 * wl.N, device="cuda", dtype=torch.float64)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_apply(plan.handle, 1e-3, 3, [v, v], out)     # nv neither 1 nor p + 1
    assert e.value.status == 1
    with pytest.raises(pk.PhiksError):
        pk.phiks_apply(plan.handle, 1e-3, 99, [v], out)
    with pytest.raises(pk.PhiksError):
        pk.phiks_apply(plan.handle, float("nan"), 3, [v], out)
    with pytest.raises(pk.PhiksError):
        pk.phiks_apply(plan.handle, 1e-3, 3, [None], out)


def test_batch_apply_and_graph_match_single_calls():
    """The batched form: uneven instances over worker streams, and the same
    work captured in one CUDA graph, give the single-call results bit for bit."""
    insts = wk.batched_instances(8)
    insts = [w for w in insts if w.N <= 120000][:6] + [wk.small_same(20)]
    rows = []
    for w in insts:
        plan = pk.Plan(w.A)
        v = dev(w.vs[0])
        p = w.p
        per = p + (0 if w.skip_phi0 else 1)
        o_single = torch.empty(per * w.N, device="cuda", dtype=torch.float64)
        o_batch = torch.empty_like(o_single)
        o_graph = torch.empty_like(o_single)
        opts = pk.make_options(skip_phi0=int(w.skip_phi0), vnorms=[float(np.linalg.norm(w.vs[0]))])
        rows.append((plan, w, v, o_single, o_batch, o_graph, opts))
    for plan, w, v, o1, _, _, opts in rows:
        pk.phiks_apply_ex(plan.handle, w.tau, w.p, [v], o1, opts=opts)
    torch.cuda.synchronize()   # the batch reuses each plan's workspace
    batch = pk.Batch(4)
    stream = torch.cuda.Stream()
    batch.apply([(r[0].handle, r[1].tau, r[1].p, [r[2]], r[4], r[6]) for r in rows], stream)
    stream.synchronize()
    graph = batch.capture([(r[0].handle, r[1].tau, r[1].p, [r[2]], r[5], r[6]) for r in rows], stream)
    batch.launch(graph, stream)
    torch.cuda.synchronize()
    for plan, w, v, o1, o2, o3, _ in rows:
        assert torch.equal(o1, o2) and torch.equal(o1, o3)
    # the graph replays: clear the outputs, launch again, same results
    for r in rows:
        r[5].zero_()
    batch.launch(graph, stream)
    torch.cuda.synchronize()
    for r in rows:
        assert torch.equal(r[3], r[5])
    batch.destroy_graph(graph)
    batch.close()
    # one instance checked against the oracle
    plan, w, v, o1, _, _, _ = rows[-1]
    ex = dense.same(w.A, w.tau, w.vs[0], w.p)
    for l in range(w.p + 1):
        assert rel_inf(o1.cpu().numpy()[l * w.N:(l + 1) * w.N], ex[l]) < TOL_EXACT


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU, pk.PHIKS_BF16X3])
def test_modes_sharing_a_matrix(dtype):
    """Modes 0 and 2 with the same matrix and mode 1 with another, and a plan
    whose three modes share one matrix: the plan computes each distinct
    matrix's small exponentials and planes once.  Both against the O3 oracle
    at the dtype's call tolerance, with squaring levels (s >= 1)."""
    n = 32
    A0 = wk.fd_adr_dirichlet(n, 1.0, 4.0, 0.3)
    A1 = wk.fd_adr_dirichlet(n, 1.0, -7.0, 0.3)
    tau, p = 3e-3, 3
    f64 = dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU)
    tol = 1e-12 if f64 else 8e-4
    tdt = torch.float64 if f64 else torch.float32
    for A in ([A0, A1, A0], [A1, A1, A1]):
        N = n ** 3
        vs = [wk.normal(70 + l, N) for l in range(p + 1)]
        if not f64:
            vs = [v.astype(np.float32).astype(np.float64) for v in vs]
        plan = pk.Plan(A, dtype)
        out = torch.full((N,), float("nan"), device="cuda", dtype=tdt)
        kw = {} if f64 else {"tol": 1e-6 * max(float(np.linalg.norm(v)) for v in vs)}
        plan.apply(tau, p, [dev(v, tdt) for v in vs], out, **kw)
        torch.cuda.synchronize()
        pk.phiks_device_status(plan.handle)
        s, q, _, _ = plan.last_params()
        plan.close()
        ex = ta.lincomb(A, tau, vs)
        err = rel_inf(out.double().cpu().numpy(), ex)
        print("shared modes dtype %d (s,q)=(%d,%d) err %.2e" % (dtype, s, q, err))
        assert s >= 1
        assert err < tol
