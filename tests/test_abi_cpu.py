"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/phiks.h declares, and its parameter selection (Sec. 3.3) picks
the same integers (s, q, T#) as the oracle's restatement."""
import os
import re

import numpy as np
import pytest

import workloads as wk
from oracle import params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pk():
    from paper_2210_07667_gb300 import _build
    _build.build()
    import paper_2210_07667_gb300 as m
    m.load()
    return m


def test_exports_match_header(pk):
    hdr = open(os.path.join(ROOT, "include", "phiks.h")).read()
    declared = set(re.findall(r"\b(phiks_[a-z_0-9]+)\s*\(", hdr))
    lib = pk.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pk.EXPORTED)


def _cases():
    yield wk.small_same(32)
    yield wk.adr3d_lincomb(64)
    yield wk.adr3d_lincomb(p=4, dims=(10, 11, 12))
    yield wk.adr3d_lincomb(p=2, dims=(40, 7), nscales=2, alpha=(3.0, -1.0), rho=-1.0)
    w = wk.small_same(24, p=5, tau=5e-3)
    w.nscales = 2
    yield w
    yield wk.cheb3d_same(n=24, nrhs=1, tau=2e-4)


@pytest.mark.parametrize("case", list(range(6)))
@pytest.mark.parametrize("rule", [0, 1])
def test_parameter_selection_matches_oracle(pk, case, rule):
    wl = list(_cases())[case]
    vn = [float(np.linalg.norm(v)) for v in wl.vs[: (1 if wl.mode == "same" else wl.p + 1)]]
    kind = "same" if wl.mode == "same" else "lincomb"
    got = pk.phiks_choose_params(wl.A, wl.tau, wl.p, vn, nscales=wl.nscales, rule=rule)
    ref = params.select(params.kron_sum_rect(wl.A, wl.tau), wl.p, kind, vn, wl.nscales,
                        rule="gll" if rule == 0 else "gl")
    assert got == (ref.s, ref.q, ref.tcount)


def _workload_cases():
    """The measured configurations' operators: a spread of the uneven batched
    instances (their own tau), the served classes at small, middle and large
    sizes (AC, anisotropic ADR, both Brusselator blocks) with p = 2..4 and
    linear-combination norms, and the Chebyshev operator of the precision form
    at its two step sizes, FP64 and split-dtype tolerances."""
    insts = wk.batched_instances(256)
    for k in range(0, 256, 23):
        w = insts[k]
        yield w.name, w.A, w.tau, 3, [float(np.linalg.norm(w.vs[0]))], None
    sizes = {"ac": (128, 576, 1024), "adr": (32, 112, 192), "bru": (128, 320, 512)}
    for cls, ns in sizes.items():
        tau = wk.SERVED_CLASSES[cls]["tau"]
        for j, n in enumerate(ns):
            p = 2 + j
            vn = [float(np.linalg.norm(wk.normal(300 + 7 * j + l, 4096))) for l in range(p + 1)]
            if cls == "ac":
                ops = [wk.ac_operator(n)]
            elif cls == "adr":
                ops = [[wk.fd_adr_dirichlet(n, 1.0, a, 2.0 / 3) for a in (10.0, -20.0, 5.0)]]
            else:
                ops = list(wk.brusselator_operators(n))
            for b, A in enumerate(ops):
                yield "%s%d_%d" % (cls, n, b), A, tau, p, vn, None
    for n, tau in ((64, 8e-6), (128, 5e-7)):
        A = [wk.cheb_d2_dirichlet(n)] * 3
        vn = [float(np.linalg.norm(wk.normal(10, n ** 3)))]
        yield "cheb%d" % n, A, tau, 3, vn, None
        yield "cheb%d_bf16x3" % n, A, tau, 3, vn, 1e-6 * vn[0]


_WORKLOAD_CASES = list(_workload_cases())


@pytest.mark.parametrize("case", range(len(_WORKLOAD_CASES)), ids=[c[0] for c in _WORKLOAD_CASES])
def test_parameter_selection_matches_oracle_on_the_measured_operators(pk, case):
    _, A, tau, p, vn, tol = _WORKLOAD_CASES[case]
    kind = "same" if len(vn) == 1 else "lincomb"
    kw = {} if tol is None else {"tol": tol}
    for rule in (0, 1):
        got = pk.phiks_choose_params(A, tau, p, vn, rule=rule, **kw)
        ref = params.select(params.kron_sum_rect(A, tau), p, kind, vn,
                            rule="gll" if rule == 0 else "gl", **kw)
        assert got == (ref.s, ref.q, ref.tcount), rule


def test_parameter_selection_tolerance_and_range(pk):
    wl = wk.small_same(16)
    vn = [float(np.linalg.norm(wl.vs[0]))]
    for tol in (1e-6, 1e-10, 2.0 ** -53):
        got = pk.phiks_choose_params(wl.A, wl.tau, wl.p, vn, tol=tol)
        ref = params.select(params.kron_sum_rect(wl.A, wl.tau), wl.p, "same", vn, tol=tol)
        assert got == (ref.s, ref.q, ref.tcount)
    got = pk.phiks_choose_params(wl.A, wl.tau, wl.p, vn, qmin=4, qmax=6)
    ref = params.select(params.kron_sum_rect(wl.A, wl.tau), wl.p, "same", vn, qmin=4, qmax=6)
    assert got == (ref.s, ref.q, ref.tcount)


def test_invalid_arguments_are_reported(pk):
    A = [np.eye(3)]
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_choose_params(A, 1.0, 0, [1.0])
    assert e.value.status == 1
    with pytest.raises(pk.PhiksError):
        pk.phiks_choose_params(A, 1.0, 2, [1.0, 1.0])          # nv neither 1 nor p + 1
    with pytest.raises(pk.PhiksError):
        pk.phiks_choose_params(A, 1.0, 2, [1.0], nscales=0)
    with pytest.raises(pk.PhiksError):
        pk.phiks_choose_params(A, 1.0, 2, [1.0], qmin=5, qmax=4)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_choose_params(A, 1.0, 2, [1.0], force_s=2)    # force_s without force_q
    assert "force" in str(e.value)


def test_plan_arguments_are_checked_before_any_device_call(pk):
    import ctypes
    lib = pk.load()
    a = np.asfortranarray(np.eye(4))
    out = ctypes.c_void_p()

    def plan(d, ns, mats, dtype=pk.PHIKS_FP64, use_out=True):
        n = (ctypes.c_int64 * max(d, 1))(*ns) if ns is not None else None
        A = (ctypes.c_void_p * max(d, 1))(*mats) if mats is not None else None
        return lib.phiks_plan(d, n, A, dtype, ctypes.byref(out) if use_out else None)

    good = a.ctypes.data
    bad = np.asfortranarray(np.eye(4))
    bad[2, 1] = np.nan
    cases = [
        (dict(d=0, ns=[4], mats=[good]), "d = 0"),
        (dict(d=9, ns=[4] * 9, mats=[good] * 9), "d = 9"),
        (dict(d=1, ns=None, mats=[good]), "NULL"),
        (dict(d=1, ns=[4], mats=None), "NULL"),
        (dict(d=1, ns=[4], mats=[good], dtype=99), "dtype"),
        (dict(d=1, ns=[0], mats=[good]), "n[0]"),
        (dict(d=2, ns=[4, 4], mats=[good, None]), "A[1]"),
        (dict(d=4, ns=[65536] * 4, mats=[good] * 4), "N too large"),
        (dict(d=1, ns=[4], mats=[good], use_out=False), "out"),
        (dict(d=2, ns=[4, 4], mats=[good, bad.ctypes.data]), "non-finite"),
    ]
    for kw, words in cases:
        st = plan(**kw)
        assert st == 1, (kw, st)                       # PHIKS_ERR_INVALID, no CUDA error
        assert words in pk.phiks_last_error(), (kw, pk.phiks_last_error())
