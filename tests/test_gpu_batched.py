"""The batched form's workload through the C ABI in the launch configuration
its measurement times: the 256 uneven-size independent instances (half d = 2
with n_mu in 64..512, half d = 3 with n_mu in 16..96, FD ADR operators with
random eps, alpha_mu and tau), phi_1..phi_3 of one vector each (Sec. 3.1,
phi_0 skipped), over 16 worker streams captured in one CUDA graph.

FP64_EMU runs the instances whose n_mu are all at most 128 (the limit of its
digit scheme: every d = 3 instance and the smallest d = 2 ones).

Checked: every instance's graph result equals its single call bit for bit
(batching changes the launch grouping, not the arithmetic); every output is
finite; the instances the O3 oracle finishes in about a second each (the
cheapest of each d by its cost model) agree with the exact phi-actions within
the dtype's call tolerance (BF16X3 8e-4: four times its 2^-17-based
per-Tucker bound; FP64_EMU 1e-12, the FP64 target).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import rel_inf  # noqa: E402

TOL_CALL = {"bf16x3": 8e-4, "fp64emu": 1e-12}
SEL_REL = {"bf16x3": 1e-6, "fp64emu": None}   # the selection tolerance the batched form uses
ORACLE_PER_D = 6        # oracle-checked instances per d
ORACLE_MAX_COST = 5e8   # (about a second of O3 on one core)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


def _o3_cost(w):
    # N sum(n) flops per matvec, ~20 terms per unit of tau ||K||_1
    return w.N * sum(a.shape[0] for a in w.A) * max(
        1.0, abs(w.tau) * sum(float(np.abs(a).sum(0).max()) for a in w.A))


@pytest.mark.parametrize("dname", ["bf16x3", "fp64emu"])
def test_batched_instances_graph_equals_single_calls_and_oracle(dname):
    insts = wk.batched_instances(256)
    if dname == "fp64emu":
        insts = [w for w in insts if max(a.shape[0] for a in w.A) <= 128]
    dt = pk.DTYPES[dname]
    tdt = torch.float64 if dname == "fp64emu" else torch.float32
    stream = torch.cuda.Stream()
    rows = []
    for w in insts:
        plan = pk.Plan(w.A, dt)
        v = w.vs[0] if dname == "fp64emu" else w.vs[0].astype(np.float32).astype(np.float64)
        vt = torch.from_numpy(v).to(device="cuda", dtype=tdt)
        single = torch.full((3 * w.N,), float("nan"), device="cuda", dtype=tdt)
        batched = torch.full_like(single, float("nan"))
        kw = dict(skip_phi0=1, vnorms=[float(np.linalg.norm(v))])
        if SEL_REL[dname] is not None:
            kw["tol"] = SEL_REL[dname] * kw["vnorms"][0]
        rows.append((plan, w, v, vt, single, batched, pk.make_options(**kw)))
    # single calls, one after another on one stream
    for plan, w, _, vt, single, _, opts in rows:
        pk.phiks_apply_ex(plan.handle, w.tau, 3, [vt], single, stream, opts=opts)
    torch.cuda.synchronize()
    # the batch over 16 worker streams, captured once and replayed
    batch = pk.Batch(16)
    inst = [(r[0].handle, r[1].tau, 3, [r[3]], r[5], r[6]) for r in rows]
    with torch.cuda.stream(stream):
        batch.apply(inst, stream)
    torch.cuda.synchronize()
    for r in rows:
        r[5].fill_(float("nan"))
    graph = batch.capture(inst, stream)
    with torch.cuda.stream(stream):
        batch.launch(graph, stream)
    torch.cuda.synchronize()
    try:
        for plan, w, _, _, single, batched, _ in rows:
            pk.phiks_device_status(plan.handle, stream)
            assert torch.isfinite(batched).all(), w.name
            assert torch.equal(single, batched), w.name
        errs = {}
        for d in (2, 3):
            cand = sorted((_o3_cost(r[1]), k) for k, r in enumerate(rows) if len(r[1].A) == d)
            picked = [k for c, k in cand[:ORACLE_PER_D] if c <= ORACLE_MAX_COST]
            assert picked, "no instance of d = %d within the oracle's budget" % d
            for k in picked:
                _, w, v, _, _, batched, _ = rows[k]
                ex = ta.same(w.A, w.tau, v, 3, ells=[1, 2, 3])
                got = batched.double().cpu().numpy().reshape(3, w.N)
                errs[w.name] = max(rel_inf(got[l], ex[l]) for l in range(3))
        print("batched %s: %d instances equal their single calls; vs oracle %s"
              % (dname, len(rows), {k: "%.1e" % e for k, e in errs.items()}))
        assert max(errs.values()) < TOL_CALL[dname], errs
    finally:
        batch.destroy_graph(graph)
        batch.close()
        for r in rows:
            r[0].close()
