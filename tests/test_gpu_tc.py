"""Split-precision tensor-core path (tcgen05 / TMEM / TMA) against the FP64
oracle.

Tolerances (relative infinity-norm), set from the representation error of
each split and rounding of FP32 intermediates:
  TF32    one tf32 product (11-bit significands)            5e-3
  TF32X3  hi*hi + hi*lo + lo*hi with tf32 hi/lo (~22 bits)   2e-5
  BF16X3  hi*hi + hi*lo + lo*hi with bf16 hi/lo (~16 bits)   2e-4
for one Tucker operator, and 4x those for a whole phiks call (quadrature,
squaring, FP64 combination).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import kron, phiks_ref  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import dev, rel_inf, run_workload  # noqa: E402

TOL = {pk.PHIKS_TF32: 5e-3, pk.PHIKS_TF32X3: 2e-5, pk.PHIKS_BF16X3: 2e-4}
DTYPES = [pk.PHIKS_BF16X3, pk.PHIKS_TF32X3, pk.PHIKS_TF32]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


def _tucker(dims, dtype, seed=0):
    rng = np.random.default_rng(seed)
    A = [np.eye(m) for m in dims]
    plan = pk.Plan(A, dtype)
    N = int(np.prod(dims))
    V = rng.standard_normal(N)
    Ls = [rng.standard_normal((m, m)) / np.sqrt(m) for m in dims]
    W = torch.empty(N, device="cuda", dtype=torch.float32)
    pk.phiks_tucker(plan.handle, dev(V, torch.float32), W, [dev(L.ravel(order="F")) for L in Ls])
    pk.phiks_device_status(plan.handle)
    ref = kron.vec(kron.tucker(kron.unvec(V.astype(np.float32).astype(np.float64), dims), Ls))
    err = rel_inf(W.cpu().numpy(), ref)
    plan.close()
    return err


@pytest.mark.parametrize("dtype", DTYPES)
def test_tucker_single_tile(dtype):
    err = _tucker((32, 32), dtype)
    print("tucker 32x32 dtype %d err %.3e" % (dtype, err))
    assert err < TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dims", [(64, 48, 40), (128, 16, 24), (96, 200), (16, 16, 16, 8), (256, 136),
                                  (600, 24), (1024, 8)])
def test_tucker_shapes(dtype, dims):
    if dtype == pk.PHIKS_BF16X3 and any(m % 8 for m in dims):
        pytest.skip("bf16 planes need n_mu % 8 == 0")
    if any(m % 4 for m in dims):
        pytest.skip("tf32 planes need n_mu % 4 == 0")
    err = _tucker(dims, dtype, seed=len(dims))
    print("tucker %s dtype %d err %.3e" % (dims, dtype, err))
    assert err < TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_same_vector_split(dtype):
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip((48, 40, 32), (2.0, -3.0, 1.0))]
    N = 48 * 40 * 32
    v = wk.normal(3, N).astype(np.float32).astype(np.float64)
    wl = wk.Workload("t", A, 2e-4, 3, "same", 2, [v])
    out, plan = run_workload(wl, dtype=dtype)
    pk.phiks_device_status(plan.handle)
    s, q, T, _ = plan.last_params()
    ref = phiks_ref.same(A, 2e-4, v, 3, s, q, nscales=2)
    errs = [rel_inf(out[k], ref[k]) for k in range(out.shape[0])]
    print("same dtype %d (s,q)=(%d,%d) errs %s" % (dtype, s, q, ["%.2e" % e for e in errs]))
    assert max(errs) < 4 * TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_lincomb_split(dtype):
    wl = wk.adr3d_lincomb(p=3, dims=(32, 24, 40), nscales=2)
    vs = [v.astype(np.float32).astype(np.float64) for v in wl.vs]
    w2 = wk.Workload("t", wl.A, wl.tau, 3, "lincomb", 2, vs)
    out, plan = run_workload(w2, dtype=dtype)
    pk.phiks_device_status(plan.handle)
    ex = [ta.lincomb(wl.A, wl.tau, vs, 2.0 ** -L) for L in range(2)]
    errs = [rel_inf(out[L], ex[L]) for L in range(2)]
    print("lincomb dtype %d errs %s" % (dtype, ["%.2e" % e for e in errs]))
    assert max(errs) < 4 * TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dims", [(64, 32, 64), (128, 256)])
def test_lincomb_split_node_batches(dtype, dims):
    """Linear combination whose quadrature nodes run as one batch with their
    own matrices, each batch's combinations in the next batch's split pass
    (d = 3 and d = 2: an even number of passes per operator)."""
    wl = wk.adr3d_lincomb(p=4, dims=dims, nscales=3) if len(dims) == 3 else None
    if wl is None:
        A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.5) for m, a in zip(dims, (6.0, -4.0))]
        N = int(np.prod(dims))
        wl = wk.Workload("t", A, 2e-4, 4, "lincomb", 3, [wk.normal(40 + l, N) for l in range(5)])
    vs = [v.astype(np.float32).astype(np.float64) for v in wl.vs]
    w2 = wk.Workload("t", wl.A, wl.tau, wl.p, "lincomb", wl.nscales, vs)
    out, plan = run_workload(w2, dtype=dtype)
    pk.phiks_device_status(plan.handle)
    s, q, _, _ = plan.last_params()
    ex = [ta.lincomb(wl.A, wl.tau, vs, 2.0 ** -L) for L in range(wl.nscales)]
    errs = [rel_inf(out[L], ex[L]) for L in range(wl.nscales)]
    print("lincomb batched %s dtype %d (s,q)=(%d,%d) errs %s" % (dims, dtype, s, q, ["%.2e" % e for e in errs]))
    assert s >= 1
    assert max(errs) < 4 * TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_same_vector_split_d2_batches(dtype):
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip((256, 128), (2.0, -3.0))]
    N = 256 * 128
    v = wk.normal(5, N).astype(np.float32).astype(np.float64)
    wl = wk.Workload("t", A, 3e-4, 3, "same", 2, [v])
    out, plan = run_workload(wl, dtype=dtype)
    pk.phiks_device_status(plan.handle)
    s, q, T, _ = plan.last_params()
    ref = phiks_ref.same(A, 3e-4, v, 3, s, q, nscales=2)
    errs = [rel_inf(out[k], ref[k]) for k in range(out.shape[0])]
    print("same d2 dtype %d (s,q)=(%d,%d) errs %s" % (dtype, s, q, ["%.2e" % e for e in errs]))
    assert max(errs) < 4 * TOL[dtype]


@pytest.mark.parametrize("dtype", [pk.PHIKS_BF16X3])
def test_batch_graph_split(dtype):
    """Split dtype, instances with n_mu above 256 (two N tiles), batched over
    streams and replayed from a CUDA graph: same results as single calls and
    within tolerance of the FP64 restatement."""
    dims_list = [(288, 40), (512, 64), (40, 24, 16)]
    rows = []
    for k, dims in enumerate(dims_list):
        A = [wk.fd_adr_dirichlet(m, 0.5, a) for m, a in zip(dims, (3.0, -5.0, 1.0))]
        N = int(np.prod(dims))
        v = wk.normal(50 + k, N).astype(np.float32).astype(np.float64)
        plan = pk.Plan(A, dtype)
        vt = dev(v, torch.float32)
        o1 = torch.empty(3 * N, device="cuda", dtype=torch.float32)
        o2 = torch.empty_like(o1)
        opts = pk.make_options(skip_phi0=1, vnorms=[float(np.linalg.norm(v))], tol=1e-6 * float(np.linalg.norm(v)))
        rows.append((plan, A, 2e-4, v, vt, o1, o2, opts))
    for plan, A, tau, v, vt, o1, _, opts in rows:
        pk.phiks_apply_ex(plan.handle, tau, 3, [vt], o1, opts=opts)
    # the single calls ran on the legacy stream and share each plan's
    # workspace with the batch below: finish them first
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    batch = pk.Batch(3)
    g = batch.capture([(r[0].handle, r[2], 3, [r[4]], r[6], r[7]) for r in rows], stream)
    batch.launch(g, stream)
    torch.cuda.synchronize()
    for plan, A, tau, v, vt, o1, o2, opts in rows:
        pk.phiks_device_status(plan.handle)
        assert torch.equal(o1, o2)
        s, q, _, _ = plan.last_params()
        ref = phiks_ref.same(A, tau, v, 3, s, q, skip_phi0=True)
        got = o1.double().cpu().numpy().reshape(3, -1)
        for l in range(3):
            assert rel_inf(got[l], ref[l]) < 4 * TOL[dtype]
    batch.destroy_graph(g)
    batch.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_same_vector_split_no_squaring(dtype):
    """(s, q) = (0, 10), phi_0 skipped: the node batch alone, its sums into
    the outputs by the last combination pass."""
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip((48, 40, 32), (2.0, -3.0, 1.0))]
    N = 48 * 40 * 32
    v = wk.normal(8, N).astype(np.float32).astype(np.float64)
    wl = wk.Workload("t", A, 1e-4, 3, "same", 1, [v], skip_phi0=True)
    out, plan = run_workload(wl, dtype=dtype, force_s=0, force_q=10)
    pk.phiks_device_status(plan.handle)
    ref = phiks_ref.same(A, 1e-4, v, 3, 0, 10, nscales=1)[1:]
    errs = [rel_inf(out[k], ref[k]) for k in range(out.shape[0])]
    assert max(errs) < 4 * TOL[dtype], errs


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dims", [(56, 40, 24), (96, 200)])
def test_mixed_batches_with_ragged_fibre_counts(dtype, dims):
    """Node batches with each node's matrices on shapes whose fibre counts
    N / n_mu are not multiples of 128 (each tensor tiled on its own) against
    the oracle's step-by-step phiks at the same (s, q)."""
    alpha = (4.0, -6.0, 2.0)[: len(dims)]
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip(dims, alpha)]
    N = int(np.prod(dims))
    v = wk.normal(77, N).astype(np.float32).astype(np.float64)
    wl = wk.Workload("t", A, 2e-4, 3, "same", 2, [v], skip_phi0=True)
    out, plan = run_workload(wl, dtype=dtype)
    pk.phiks_device_status(plan.handle)
    s, q, _, _ = plan.last_params()
    ref = phiks_ref.same(A, 2e-4, v, 3, s, q, nscales=2, skip_phi0=True)
    errs = [rel_inf(out[k], ref[k]) for k in range(out.shape[0])]
    print("mixed ragged %s dtype %d (s,q)=(%d,%d) errs %s" % (dims, dtype, s, q, ["%.2e" % e for e in errs]))
    assert max(errs) < 4 * TOL[dtype]
    plan.close()
