"""Failure detection and cross-stream ordering, in the forms that fault no GPU.

* A bounded mbarrier wait that nothing ends (phiks_debug_wait_timeout, a
  limit of a few milliseconds) must return, leave PHIKS_ERR_TIMEOUT in the
  plan's status, and the next call on the plan must match the oracle.
* Device allocations made to fail on the host (phiks_debug_fail_alloc) must
  turn into PHIKS_ERR_OOM from the plan, the workspace and the cached
  exponentials, release what the failing call had allocated, and leave the
  plan usable.
* Applies on one plan from two streams (each with its own workspace and
  norms, as include/phiks.h allows) must not see each other's half-built or
  freed exponential banks: a bank built on a stream that is held back is
  waited for, and an eviction waits for the last use on the other stream.
* The served form from cold plans: requests of the same plan and (s, q) in
  flight together give the results they give alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import dense, phiks_ref  # noqa: E402

from gpu_util import dev, rel_inf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)
    yield
    pk.phiks_debug_fail_alloc(-1)


def _small_call(plan, wl, dtype):
    tdt = torch.float64 if dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU) else torch.float32
    out = torch.full((4 * wl.N,), float("nan"), device="cuda", dtype=tdt)
    plan.apply(wl.tau, 3, [dev(wl.vs[0], tdt)], out, vnorms=[float(np.linalg.norm(wl.vs[0]))])
    torch.cuda.synchronize()
    return out.double().cpu().numpy().reshape(4, wl.N)


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64_EMU, pk.PHIKS_BF16X3])
def test_bounded_wait_gives_up_and_the_plan_recovers(dtype):
    wl = wk.small_same(16)
    wl.vs[0] = wl.vs[0].astype(np.float32).astype(np.float64)
    plan = pk.Plan(wl.A, dtype)
    pk.phiks_device_status(plan.handle)                  # clean to start with
    pk.phiks_debug_wait_timeout(plan.handle, 5.0)        # a wait nothing ends, 5 ms limit
    torch.cuda.synchronize()                             # the kernel returned
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_device_status(plan.handle)
    assert e.value.status == 6 and "site 21" in str(e.value)
    pk.phiks_device_status(plan.handle)                  # the read cleared it
    got = _small_call(plan, wl, dtype)
    pk.phiks_device_status(plan.handle)
    ex = dense.same(wl.A, wl.tau, wl.vs[0], 3)
    tol = 1e-12 if dtype == pk.PHIKS_FP64_EMU else 8e-4
    for k in range(4):
        assert rel_inf(got[k], ex[k]) < tol, k
    plan.close()


def test_bounded_wait_check_needs_a_tensor_core_plan():
    plan = pk.Plan(wk.small_same(8).A, pk.PHIKS_FP64)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_debug_wait_timeout(plan.handle, 5.0)
    assert e.value.status == 3
    plan.close()


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU])
def test_injected_allocation_failures(dtype):
    wl = wk.small_same(16)
    torch.cuda.synchronize()
    base = pk.phiks_debug_live_allocations()
    # the plan: let k allocations pass, the next fails, for every k until the
    # plan needs fewer than k + 1
    k = 0
    while True:
        pk.phiks_debug_fail_alloc(k)
        try:
            plan = pk.Plan(wl.A, dtype)
        except pk.PhiksError as e:
            assert e.status == 2, str(e)
            assert pk.phiks_debug_live_allocations() == base, k
            k += 1
            assert k < 32
            continue
        pk.phiks_debug_fail_alloc(-1)
        break
    assert k >= 3      # A_mu, its powers, the norms (and more for FP64_EMU) came before
    held = pk.phiks_debug_live_allocations()
    ex = dense.same(wl.A, wl.tau, wl.vs[0], 3)
    tdt = torch.float64
    vs = [dev(wl.vs[0], tdt)]
    out = torch.empty(4 * wl.N, device="cuda", dtype=tdt)
    vn = [float(np.linalg.norm(wl.vs[0]))]
    # the first apply allocates the plan's workspace, a bank of exponentials,
    # the exponential scratch (and for FP64_EMU the bank's B planes): let j
    # of them pass and the next fail, j = 0, 1, ..., until the call goes
    # through (what a failed call allocated before the failure either stays
    # with the plan, the workspace and scratch, or is released, the bank)
    fails = 0
    for j in range(8):
        pk.phiks_debug_fail_alloc(j)
        try:
            plan.apply(wl.tau, 3, vs, out, vnorms=vn)
        except pk.PhiksError as e:
            assert e.status == 2, str(e)
            torch.cuda.synchronize()
            assert pk.phiks_debug_live_allocations() <= held + 2
            fails += 1
            continue
        pk.phiks_debug_fail_alloc(-1)
        break
    pk.phiks_debug_fail_alloc(-1)
    assert fails >= 2
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(4, wl.N)
    for i in range(4):
        assert rel_inf(got[i], ex[i]) < 1e-12
    # a new tau needs a new bank: its allocation fails, the next call builds it
    held = pk.phiks_debug_live_allocations()
    pk.phiks_debug_fail_alloc(0)
    with pytest.raises(pk.PhiksError) as e:
        plan.apply(2 * wl.tau, 3, vs, out, vnorms=vn)
    assert e.value.status == 2
    assert pk.phiks_debug_live_allocations() == held
    plan.apply(2 * wl.tau, 3, vs, out, vnorms=vn)
    torch.cuda.synchronize()
    ex2 = dense.same(wl.A, 2 * wl.tau, wl.vs[0], 3)
    got = out.cpu().numpy().reshape(4, wl.N)
    for i in range(4):
        assert rel_inf(got[i], ex2[i]) < 1e-12
    plan.close()
    torch.cuda.synchronize()
    assert pk.phiks_debug_live_allocations() == base


def _ws(plan, p):
    b = pk.phiks_workspace_size(plan.handle, p, 1)
    return torch.empty(b, device="cuda", dtype=torch.uint8)


def _apply_on(plan, tau, v, out, ws, vn, stream, **kw):
    pk.phiks_apply_ex(plan.handle, tau, 3, [v], out, stream, vnorms=vn, workspace=ws.data_ptr(),
                      workspace_bytes=ws.numel(), skip_phi0=1, **kw)


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64_EMU, pk.PHIKS_BF16X3, pk.PHIKS_FP64])
def test_new_tau_on_two_streams_waits_for_the_bank(dtype):
    """Stream A is held back (a spin kernel) and then builds the bank of a
    new tau; stream B asks for the same tau right after on the host.  B must
    wait for A's bank: its result equals a serial run bit for bit and the
    oracle's restatement at the same (s, q)."""
    dims = (32, 24, 16)
    A = [wk.fd_adr_dirichlet(m, 1.0, a, 0.3) for m, a in zip(dims, (2.0, -3.0, 1.0))]
    N = int(np.prod(dims))
    f64 = dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU)
    tdt = torch.float64 if f64 else torch.float32
    v = wk.normal(31, N).astype(np.float32).astype(np.float64)
    vn = [float(np.linalg.norm(v))]
    plan = pk.Plan(A, dtype)
    vt = dev(v, tdt)
    wsA, wsB = _ws(plan, 3), _ws(plan, 3)
    outA = torch.full((3 * N,), float("nan"), device="cuda", dtype=tdt)
    outB = torch.full_like(outA, float("nan"))
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    tau = 3.7e-4
    torch.cuda.synchronize()
    with torch.cuda.stream(sA):
        torch.cuda._sleep(int(2e8))          # ~0.1 s on the device
        _apply_on(plan, tau, vt, outA, wsA, vn, sA)
    _apply_on(plan, tau, vt, outB, wsB, vn, sB)
    torch.cuda.synchronize()
    pk.phiks_device_status(plan.handle)
    serial = torch.full_like(outA, float("nan"))
    _apply_on(plan, tau, vt, serial, wsB, vn, sB)
    torch.cuda.synchronize()
    assert torch.equal(outB, serial)
    assert torch.equal(outA, serial)
    s, q, _, _ = plan.last_params()
    ref = phiks_ref.same(A, tau, v, 3, s, q, skip_phi0=True)
    got = serial.double().cpu().numpy().reshape(3, N)
    tol = 1e-12 if f64 else 8e-4
    for l in range(3):
        assert rel_inf(got[l], ref[l]) < tol
    plan.close()


def test_eviction_waits_for_the_last_use_on_another_stream():
    """Stream A (held back) reads the bank of tau_0; stream B then asks for
    eight new tau, which evicts tau_0's bank and reuses memory.  The eviction
    must wait for A's use: A's result equals a serial run bit for bit."""
    dims = (24, 16, 16)
    A = [wk.fd_adr_dirichlet(m, 1.0, a) for m, a in zip(dims, (2.0, -3.0, 1.0))]
    N = int(np.prod(dims))
    v = wk.normal(32, N)
    vn = [float(np.linalg.norm(v))]
    plan = pk.Plan(A, pk.PHIKS_FP64_EMU)
    vt = dev(v)
    wsA, wsB = _ws(plan, 3), _ws(plan, 3)
    taus = [1e-4 * (1.0 + 0.1 * k) for k in range(9)]
    ref = torch.empty(3 * N, device="cuda", dtype=torch.float64)
    _apply_on(plan, taus[0], vt, ref, wsA, vn, None)     # tau_0's bank exists
    torch.cuda.synchronize()
    outA = torch.full_like(ref, float("nan"))
    outB = torch.empty_like(ref)
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(sA):
        torch.cuda._sleep(int(2e8))
        _apply_on(plan, taus[0], vt, outA, wsA, vn, sA)
    for t in taus[1:]:                                   # eight new banks: tau_0's is evicted
        _apply_on(plan, t, vt, outB, wsB, vn, sB)
    torch.cuda.synchronize()
    pk.phiks_device_status(plan.handle)
    assert torch.equal(outA, ref)
    plan.close()


@pytest.mark.parametrize("dtype", ["fp64emu", "bf16x3"])
def test_served_from_cold_plans_equals_alone(dtype):
    """Two requests of one plan and tau, dispatched together on two slots
    before any exponential exists: the slot that finds the bank being built
    by the other waits for it."""
    n = 24
    A = [wk.fd_adr_dirichlet(n, 1.0, a, 2.0 / 3) for a in (10.0, -20.0, 5.0)]
    N = n ** 3
    f64 = dtype == "fp64emu"
    tdt = torch.float64 if f64 else torch.float32
    plan = pk.Plan(A, pk.DTYPES[dtype])
    vs = [wk.normal(60 + l, N).astype(np.float32).astype(np.float64) for l in range(4)]
    vt = [dev(x, tdt) for x in vs]
    vn = [float(np.linalg.norm(x)) for x in vs]
    reqs = []
    for k in range(2):
        x = {"plan": plan.handle, "tau": 5e-4, "p": 3, "v": vt, "vnorms": vn,
             "out": torch.full((N,), float("nan"), device="cuda", dtype=tdt)}
        if not f64:
            x["tol"] = 1e-6 * max(vn)
        reqs.append([x])
    lat, _, _ = pk.phiks_serve_trace(reqs, np.zeros(2), slots=2)
    assert all(l > 0 for l in lat)
    pk.phiks_device_status(plan.handle)
    mixed = [r[0]["out"].clone() for r in reqs]
    alone = torch.empty_like(mixed[0])
    kw = {"tol": reqs[0][0]["tol"]} if not f64 else {}
    pk.phiks_apply_ex(plan.handle, 5e-4, 3, vt, alone, None, vnorms=vn, **kw)
    torch.cuda.synchronize()
    for m in mixed:
        assert torch.equal(m, alone)
    plan.close()
