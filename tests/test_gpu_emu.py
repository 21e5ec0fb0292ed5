"""FP64 emulated on the tensor cores (PHIKS_FP64_EMU): exact bf16 digit
products, one rounding to FP64.  Checked against the FP64 oracle with the
FP64 path's tolerances: 1e-14 for one Tucker operator (relative to the
largest output), 1e-12 for whole phiks calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import dense, kron  # noqa: E402
from oracle import phiks_ref  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import dev, rel_inf, run_workload  # noqa: E402

EMU = pk.PHIKS_FP64_EMU


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


@pytest.mark.parametrize("dims", [(32, 32), (64, 48, 40), (128, 16, 24), (8, 8, 8, 8), (64, 64, 64),
                                  (16, 128, 24), (24, 64, 32)])
def test_tucker_emulated_fp64(dims):
    rng = np.random.default_rng(sum(dims))
    plan = pk.Plan([np.eye(m) for m in dims], EMU)
    N = int(np.prod(dims))
    V = rng.standard_normal(N) * np.exp(rng.uniform(-3, 3, N))   # wide dynamic range
    Ls = [rng.standard_normal((m, m)) / np.sqrt(m) for m in dims]
    W = torch.empty(N, device="cuda", dtype=torch.float64)
    pk.phiks_tucker(plan.handle, dev(V), W, [dev(L.ravel(order="F")) for L in Ls])
    pk.phiks_device_status(plan.handle)
    ref = kron.vec(kron.tucker(kron.unvec(V, dims), Ls))
    err = rel_inf(W.cpu().numpy(), ref)
    print("emu tucker", dims, "%.2e" % err)
    assert err < 1e-14
    plan.close()


def test_same_vector_emulated():
    wl = wk.small_same(32)
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    for L in range(1):
        ex = dense.same(wl.A, wl.tau, wl.vs[0], wl.p)
        for k in range(wl.p + 1):
            assert rel_inf(out[k], ex[k]) < 1e-12, k


def test_lincomb_bench_workload_emulated():
    wl = wk.adr3d_lincomb(64)
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    errs = [rel_inf(out[L], ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) for L in range(3)]
    print("emu lincomb errs", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-12


def test_lincomb_emulated_ragged_batches():
    """Batched emulated passes whose 128-fibre tiles straddle the tensors of a
    batch (960, 640 and 1600 fibres per tensor for the three modes)."""
    wl = wk.adr3d_lincomb(p=3, dims=(40, 24, 16), nscales=2)
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    errs = [rel_inf(out[L], ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) for L in range(2)]
    print("emu ragged lincomb errs", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-12


def test_same_vector_emulated_node_batches():
    """SAME mode whose quadrature nodes run as one batch of Tucker operators
    with their own matrices (every mode's fibre count a multiple of 128)."""
    dims = (64, 32, 64)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, (4.0, -2.0, 1.0))]
    N = int(np.prod(dims))
    wl = wk.Workload("adr3d_same_%dx%dx%d" % dims, A, 5e-4, 3, "same", 2, [wk.uniform(21, N)])
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    per = wl.p + 1
    worst = 0.0
    for L in range(2):
        ex = ta.same(wl.A, wl.tau, wl.vs[0], wl.p, c=2.0 ** -L)
        for k in range(per):
            e = rel_inf(out[L * per + k], ex[k])
            worst = max(worst, e)
            assert e < 1e-12, (L, k, e)
    print("emu same node batches: max rel err %.2e" % worst)


def test_lincomb_emulated_many_nodes():
    """Linear combination with (s, q) = (6, 12): eleven quadrature nodes with
    Tucker operators, in batches of whole nodes (four operators each)."""
    wl = wk.adr3d_lincomb(p=4, dims=(64, 32, 64), nscales=2)
    out, plan = run_workload(wl, dtype=EMU, force_s=6, force_q=12)
    pk.phiks_device_status(plan.handle)
    s, q, _, _ = plan.last_params()
    assert (s, q) == (6, 12)
    errs = [rel_inf(out[L], ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) for L in range(2)]
    print("emu lincomb q=12 errs", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-12


def test_lincomb_emulated_missing_vectors():
    """Linear combination without v_0 and v_2: outputs that are the
    accumulators alone, and quadrature inputs with fewer terms."""
    wl = wk.adr3d_lincomb(p=4, dims=(64, 32, 64), nscales=3)
    wl.vs[0] = None
    wl.vs[2] = None
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    errs = [rel_inf(out[L], ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L)) for L in range(3)]
    print("emu lincomb without v0, v2 errs", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-12


@pytest.mark.parametrize("skip_phi0,nscales,p", [(True, 3, 3), (False, 1, 5)])
def test_same_vector_emulated_scales(skip_phi0, nscales, p):
    """SAME mode on the emulated path with phi_0 skipped or kept, several
    scale outputs: every output against the oracle."""
    dims = (64, 32, 64)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, (4.0, -2.0, 1.0))]
    N = int(np.prod(dims))
    wl = wk.Workload("adr3d_same", A, 8e-4, p, "same", nscales, [wk.uniform(23, N)], skip_phi0=skip_phi0)
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    ells = list(range(1 if skip_phi0 else 0, p + 1))
    for L in range(nscales):
        ex = ta.same(wl.A, wl.tau, wl.vs[0], p, c=2.0 ** -L, ells=ells)
        for k in range(len(ells)):
            e = rel_inf(out[L * len(ells) + k], ex[k])
            assert e < 1e-12, (L, ells[k], e)


@pytest.mark.parametrize("mode,p", [("same", 3), ("lincomb", 4), ("lincomb", 1)])
def test_emulated_no_squaring(mode, p):
    """(s, q) = (0, 12): the quadrature batch, then the phi_0 / exp(K) v_0
    operator in a batch of its own; against the oracle's restatement of the
    method with the same (s, q)."""
    dims = (64, 32, 64)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, (4.0, -2.0, 1.0))]
    N = int(np.prod(dims))
    tau = 1e-4
    if mode == "same":
        wl = wk.Workload("t", A, tau, p, "same", 1, [wk.uniform(31, N)])
    else:
        wl = wk.Workload("t", A, tau, p, "lincomb", 1, [wk.normal(50 + l, N) for l in range(p + 1)])
    out, plan = run_workload(wl, dtype=EMU, force_s=0, force_q=12)
    pk.phiks_device_status(plan.handle)
    assert plan.last_params()[:2] == (0, 12)
    if mode == "same":
        ref = phiks_ref.same(A, tau, wl.vs[0], p, 0, 12, nscales=1)
    else:
        ref = phiks_ref.lincomb(A, tau, wl.vs, 0, 12, nscales=1)
    for k in range(out.shape[0]):
        assert rel_inf(out[k], ref[k]) < 1e-12, k


def _emu_bound(x_fibre_max, l_row_max, n, result):
    """Per-output bound of one emulated dot product (x fibre, l row):
    (7.03 n 2^-54 + 2^-52) max|x| max|l| + 2^-53 |result| (the truncated
    digit products s + t >= 7, the fixed-point fibre representation and the
    final rounding to FP64)."""
    return (7.03 * n * 2.0 ** -54 + 2.0 ** -52) * x_fibre_max * l_row_max + 2.0 ** -53 * np.abs(result)


def test_tucker_emulated_twelve_decades_within_fibres():
    """V with magnitudes log-uniform over 1e-12 .. 1 inside every fibre
    (d = 2, 64 x 64).  The emulation's accuracy is relative to each fibre's
    largest element, not to sum |x_j l_j|: the exact result (rational
    arithmetic) must lie within the composed two-mode bound of every
    output element, and tiny elements may lose their own relative accuracy."""
    from fractions import Fraction
    n1 = n2 = 64
    rng = np.random.default_rng(77)
    X = rng.standard_normal((n1, n2)) * 10.0 ** rng.uniform(-12, 0, (n1, n2))
    L1 = rng.standard_normal((n1, n1)) / 8
    L2 = rng.standard_normal((n2, n2)) / 8
    plan = pk.Plan([np.eye(n1), np.eye(n2)], EMU)
    W = torch.empty(n1 * n2, device="cuda", dtype=torch.float64)
    pk.phiks_tucker(plan.handle, dev(X.ravel(order="F")), W, [dev(L1.ravel(order="F")), dev(L2.ravel(order="F"))])
    pk.phiks_device_status(plan.handle)
    got = W.cpu().numpy().reshape((n1, n2), order="F")
    plan.close()
    # exact Y = L1 X L2^T in rationals
    Xf = [[Fraction(float(X[i, j])) for j in range(n2)] for i in range(n1)]
    L1f = [[Fraction(float(L1[i, k])) for k in range(n1)] for i in range(n1)]
    L2f = [[Fraction(float(L2[j, k])) for k in range(n2)] for j in range(n2)]
    Y1 = [[sum(L1f[i][k] * Xf[k][j] for k in range(n1)) for j in range(n2)] for i in range(n1)]
    Z = np.array([[float(sum(Y1[i][k] * L2f[j][k] for k in range(n2))) for j in range(n2)]
                  for i in range(n1)])
    Y1d = np.array([[float(y) for y in row] for row in Y1])
    # mode 1 (fibres = columns of X), then mode 2 on the rounded result
    b1 = _emu_bound(np.abs(X).max(axis=0)[None, :], np.abs(L1).max(axis=1)[:, None], n1, Y1d)
    Y1max = (np.abs(Y1d) + b1).max(axis=1)[:, None]      # fibres of mode 2 = rows of Y1
    b2 = _emu_bound(Y1max, np.abs(L2).max(axis=1)[None, :], n2, Z)
    bound = b1 @ np.abs(L2).T + b2
    err = np.abs(got - Z)
    ratio = float((err / bound).max())
    rel = float(err.max() / np.abs(Z).max())
    elem_rel = float(np.median(err / np.abs(Z)))
    print("emu 12-decade fibres: max err/bound %.3f, rel inf-norm %.2e, median element rel %.2e"
          % (ratio, rel, elem_rel))
    assert ratio <= 1.0
    assert rel < 1e-14


@pytest.mark.parametrize("dims", [(56, 40, 24), (96, 120), (8, 8, 8, 8)])
def test_mixed_batches_with_ragged_fibre_counts(dims):
    """Batches that mix matrices (all quadrature nodes together, a squaring
    level with the output operators) on shapes whose fibre counts N / n_mu
    are not multiples of 128: every tensor is tiled on its own, its last tile
    partial.  Against the oracle's Taylor action at 1e-12."""
    alpha = (4.0, -6.0, 2.0, 1.0)[: len(dims)]
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, alpha)]
    N = int(np.prod(dims))
    assert any((N // m) % 128 for m in dims) or len(dims) == 4
    vs = [wk.normal(90 + l, N) for l in range(4)]
    wl = wk.Workload("t", A, 3e-4, 3, "lincomb", 2, vs)
    out, plan = run_workload(wl, dtype=EMU)
    pk.phiks_device_status(plan.handle)
    s, q, _, tk = plan.last_params()
    for L in range(2):
        ex = ta.lincomb(A, 3e-4, vs, 2.0 ** -L)
        assert rel_inf(out[L], ex) < 1e-12, L
    assert s >= 1
    plan.close()


@pytest.mark.parametrize("n", [32, 64])
def test_misaligned_inputs_give_the_same_digits(n):
    """The split pass moves pairs of doubles where its sources are 16-byte
    aligned and single doubles otherwise, with the same combination in the
    same order: inputs offset by one double (8-byte aligned only) give
    bit-identical outputs, and both match the oracle."""
    dims = (n, n, 16)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip(dims, (1.0, -2.0, 3.0))]
    N = int(np.prod(dims))
    tau, p = 2e-4, 3
    vs = [wk.normal(30 + l, N) for l in range(p + 1)]
    outs = []
    for shift in (0, 1):
        plan = pk.Plan(A, EMU)
        bufs = [torch.zeros(N + 2, device="cuda", dtype=torch.float64) for _ in vs]
        views = []
        for b, v in zip(bufs, vs):
            b[shift:shift + N] = torch.from_numpy(v).cuda()
            views.append(b[shift:shift + N])
        assert all((t.data_ptr() % 16 == 0) == (shift == 0) for t in views)
        out = torch.full((N,), float("nan"), device="cuda", dtype=torch.float64)
        plan.apply(tau, p, views, out)
        torch.cuda.synchronize()
        pk.phiks_device_status(plan.handle)
        outs.append(out.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])
    ex = ta.lincomb(A, tau, vs)
    assert rel_inf(outs[0], ex) < 1e-12
