"""Complex operators on the device (PHIKS_C128): the code-validation problem
of Sec. 4.1, (1+i)/100 Laplacian in d = 3 and d = 6, p = 5, two scales,
against the oracle's exact eigenbasis route (relative infinity norm, per
output, 1e-12), with the planner's (s, q, T#) equal to the oracle's
restatement of Sec. 3.3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import eig, kron, params  # noqa: E402

P = 5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n,d", [(64, 3), (81, 3), (8, 6), (11, 6)])
def test_validation_same_vector(n, d):
    zeta, T, v = wk.validation_complex(n, d)
    A = [zeta * t for t in T]
    N = v.size
    plan = pk.Plan(A, pk.PHIKS_C128)
    out = torch.empty(2 * (P + 1) * N, device="cuda", dtype=torch.complex128)
    plan.apply(1.0, P, [torch.from_numpy(v).cuda()], out, nscales=2)
    torch.cuda.synchronize()
    pk.phiks_device_status(plan.handle)
    got = out.cpu().numpy().reshape(2, P + 1, N)
    worst = 0.0
    for j in range(2):
        ref = eig.scaled_phi_actions(zeta, T, 1.0, v, range(P + 1), c=2.0 ** -j)
        for l in range(P + 1):
            e = rel(got[j, l], ref[l])
            worst = max(worst, e)
            assert e < 1e-12, (j, l, e)
    s, q, tc, _ = plan.last_params()
    sel = params.select(params.kron_sum_rect(A, 1.0), P, "same", [float(np.linalg.norm(v))], nscales=2)
    print("same n=%d d=%d: max rel diff %.2e, (s, q, T#) = (%d, %d, %d)" % (n, d, worst, s, q, tc))
    assert (s, q, tc) == (sel.s, sel.q, sel.tcount)
    plan.close()


@pytest.mark.parametrize("n,d", [(64, 3), (8, 6)])
def test_validation_linear_combination(n, d):
    zeta, T, v = wk.validation_complex(n, d)
    A = [zeta * t for t in T]
    N = v.size
    plan = pk.Plan(A, pk.PHIKS_C128)
    vd = torch.from_numpy(v).cuda()
    out = torch.empty(2 * N, device="cuda", dtype=torch.complex128)
    plan.apply(1.0, P, [None] + [vd] * P, out, nscales=2)
    torch.cuda.synchronize()
    pk.phiks_device_status(plan.handle)
    got = out.cpu().numpy().reshape(2, N)
    for j in range(2):
        ref = eig.scaled_lincomb(zeta, T, 1.0, [None] + [v] * P, c=2.0 ** -j)
        assert rel(got[j], ref) < 1e-12, j
    s, q, tc, _ = plan.last_params()
    vn = float(np.linalg.norm(v))
    sel = params.select(params.kron_sum_rect(A, 1.0), P, "lincomb", [0.0] + [vn] * P, nscales=2)
    assert (s, q, tc) == (sel.s, sel.q, sel.tcount)
    plan.close()


def test_complex_tucker_operator():
    """W = V x_1 L_1 ... x_d L_d with complex L_mu, passed as their real
    representations, against the oracle's mode products."""
    rng = np.random.default_rng(11)
    dims = (12, 7, 9)
    zeta, T, _ = wk.validation_complex(3, 3)
    plan = pk.Plan([zeta * wk.fd_adr_dirichlet(m, 1.0, 0.0) for m in dims], pk.PHIKS_C128)
    N = int(np.prod(dims))
    V = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Ls = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for m in dims]
    reps = [np.block([[L.real, -L.imag], [L.imag, L.real]]) for L in Ls]
    W = torch.empty(N, device="cuda", dtype=torch.complex128)
    Ld = [torch.from_numpy(np.asfortranarray(R).ravel(order="F").copy()).cuda() for R in reps]
    pk.phiks_tucker(plan.handle, torch.from_numpy(V).cuda(), W, Ld)
    torch.cuda.synchronize()
    ref = kron.vec(kron.tucker(kron.unvec(V, dims), Ls))
    assert rel(W.cpu().numpy(), ref) < 1e-14
    plan.close()
