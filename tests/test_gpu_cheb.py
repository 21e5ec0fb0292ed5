"""The precision form's operator through the C ABI, every dtype, against the
O3 oracle (the exact phi-actions, not the FP64 GPU path).

A_mu is the dense Chebyshev second-derivative matrix with Dirichlet rows and
columns removed (d = 3, the same matrix in every mode): strongly non-normal,
||A||_1 ~ 1e6 at n = 64 and 1.5e7 at n = 128, so its numerical range and
tau ||K|| drive the parameter selection of Sec. 3.3 to squaring.  The task is
the same-vector one of Sec. 3.1, phi_1..phi_3 (phi_0 skipped), as in the
precision configuration.

Tolerances, relative infinity-norm per output block against the oracle:
  FP64, FP64_EMU   1e-12 (the FP64 target)
  TF32X3 8e-5, BF16X3 8e-4, TF32 2e-2: four times the per-Tucker bound of
  each split (2^-23, 2^-17 and 2^-11 representation error with FP32
  intermediates), as for every split-dtype call test.
The split dtypes ask the selection for a relative accuracy that matches their
arithmetic (tol = rel * ||v||, the precision configuration's choice).
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import dev, rel_inf  # noqa: E402

TOL_CALL = {pk.PHIKS_FP64: 1e-12, pk.PHIKS_FP64_EMU: 1e-12, pk.PHIKS_TF32X3: 8e-5,
            pk.PHIKS_BF16X3: 8e-4, pk.PHIKS_TF32: 2e-2}
SEL_REL = {pk.PHIKS_TF32: 1e-4, pk.PHIKS_TF32X3: 1e-7, pk.PHIKS_BF16X3: 1e-6}
ALL = [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU, pk.PHIKS_TF32X3, pk.PHIKS_BF16X3, pk.PHIKS_TF32]
P = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


def _vector(n, seed=10):
    # rounded to float32 once, so that every dtype sees the same input
    return wk.normal(seed, n ** 3).astype(np.float32).astype(np.float64)


@functools.lru_cache(maxsize=None)
def _exact(n, tau, ells):
    """phi_l(tau K) v for l in ells, O3 (Taylor action of the augmented matrix)."""
    A = [wk.cheb_d2_dirichlet(n)] * 3
    v = _vector(n)
    return np.stack([ta.same(A, tau, v, P, ells=[l])[0] for l in ells])


def _run(n, tau, dtype, nscales=1):
    A = [wk.cheb_d2_dirichlet(n)] * 3
    v = _vector(n)
    f64 = dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU)
    tdt = torch.float64 if f64 else torch.float32
    plan = pk.Plan(A, dtype)
    N = n ** 3
    out = torch.full((nscales * P * N,), float("nan"), device="cuda", dtype=tdt)
    kw = dict(skip_phi0=1, nscales=nscales)
    if dtype in SEL_REL:
        kw["tol"] = SEL_REL[dtype] * float(np.linalg.norm(v))
    plan.apply(tau, P, [dev(v, tdt)], out, **kw)
    torch.cuda.synchronize()
    pk.phiks_device_status(plan.handle)
    s, q, T, tk = plan.last_params()
    plan.close()
    return out.double().cpu().numpy().reshape(nscales * P, N), (s, q, T, tk)


# tau = 5e-7 is the precision configuration's time step (at n = 64 the
# selection needs no squaring); tau = 8e-6 gives tau ||K||_1 ~ 22 as at
# n = 128, with squaring levels and their batches
@pytest.mark.parametrize("tau", [5e-7, 8e-6])
@pytest.mark.parametrize("dtype", ALL)
def test_cheb_n64_every_dtype_vs_oracle(dtype, tau):
    got, (s, q, T, tk) = _run(64, tau, dtype)
    ex = _exact(64, tau, (1, 2, 3))
    errs = [rel_inf(got[k], ex[k]) for k in range(P)]
    print("cheb n=64 tau=%g dtype %d (s,q,T#)=(%d,%d,%d) errs %s"
          % (tau, dtype, s, q, T, ["%.2e" % e for e in errs]))
    if tau > 1e-6 and dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU):
        assert s >= 1   # (the split dtypes' looser tolerance may need no squaring)
    assert max(errs) < TOL_CALL[dtype]


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64_EMU, pk.PHIKS_BF16X3])
def test_cheb_n64_scale_outputs_vs_oracle(dtype):
    """Two scales (tau and tau/2): each block against a fresh oracle call."""
    tau = 8e-6
    got, (s, q, _, _) = _run(64, tau, dtype, nscales=2)
    ex0 = _exact(64, tau, (1, 2, 3))
    ex1 = _exact(64, tau / 2, (1, 2, 3))
    errs = [rel_inf(got[k], ex0[k]) for k in range(P)] + [rel_inf(got[P + k], ex1[k]) for k in range(P)]
    print("cheb n=64 two scales dtype %d (s,q)=(%d,%d) errs %s" % (dtype, s, q, ["%.2e" % e for e in errs]))
    assert max(errs) < TOL_CALL[dtype]


@pytest.mark.parametrize("dtype", ALL)
def test_cheb_n128_full_size_vs_oracle(dtype):
    """The precision configuration's full size (N = 2,097,152, tau = 5e-7),
    one right-hand side, every dtype (the split dtypes with the selection
    tolerance the precision configuration gives them); phi_1 checked against
    the oracle (one O3 call, shared by the dtypes)."""
    tau = 5e-7
    got, (s, q, T, tk) = _run(128, tau, dtype)
    ex = _exact(128, tau, (1,))
    err = rel_inf(got[0], ex[0])
    print("cheb n=128 dtype %d (s,q,T#)=(%d,%d,%d) phi_1 err %.2e" % (dtype, s, q, T, err))
    if dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU):
        assert s >= 1   # (the split dtypes' looser tolerance needs no squaring here)
    assert np.isfinite(got).all()
    assert err < TOL_CALL[dtype]
