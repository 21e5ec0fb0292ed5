"""Whole calls replayed from CUDA graphs (phiks_options.graph): a replay
launches the same kernels as a plain call, so its results equal the plain
call's bit for bit, on new vector values in the same buffers, for new tau
(a new capture) and with the small exponentials recomputed inside the graph;
and the results still meet the oracle's 1e-12."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07667_gb300 as pk  # noqa: E402
import workloads as wk  # noqa: E402
from oracle import taylor_action as ta  # noqa: E402

from gpu_util import dev, rel_inf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)


@pytest.mark.parametrize("dtype", [pk.PHIKS_FP64, pk.PHIKS_FP64_EMU])
@pytest.mark.parametrize("no_cache", [0, 1])
def test_graph_replay_matches_plain_calls(dtype, no_cache):
    wl = wk.adr3d_lincomb(32, tau=5e-4, p=3, nscales=2)
    N = wl.N
    plan = pk.Plan(wl.A, dtype)
    vs = [dev(v) for v in wl.vs]
    out_g = torch.empty(wl.nscales * N, device="cuda", dtype=torch.float64)
    out_p = torch.empty_like(out_g)
    rng = np.random.default_rng(5)
    st = torch.cuda.Stream()
    for it, tau in enumerate([wl.tau, wl.tau, wl.tau, wl.tau, 2 * wl.tau, 2 * wl.tau, wl.tau]):
        if it in (2, 5):  # new values in the same buffers
            for v in vs:
                v.copy_(torch.from_numpy(rng.standard_normal(N)))
            torch.cuda.synchronize()
        l0 = pk.phiks_kernel_launches()
        plan.apply(tau, wl.p, vs, out_g, st, nscales=wl.nscales, graph=1, no_cache=no_cache)
        torch.cuda.synchronize()
        lg = pk.phiks_kernel_launches() - l0
        l0 = pk.phiks_kernel_launches()
        plan.apply(tau, wl.p, vs, out_p, st, nscales=wl.nscales, no_cache=1)
        torch.cuda.synchronize()
        lp = pk.phiks_kernel_launches() - l0
        assert torch.equal(out_g, out_p), it
        if no_cache:
            assert lg == lp, (it, lg, lp)
        pk.phiks_device_status(plan.handle)
    got = out_g.cpu().numpy().reshape(-1, N)
    vh = [v.cpu().numpy() for v in vs]
    for L in range(wl.nscales):
        assert rel_inf(got[L], ta.lincomb(wl.A, wl.tau, vh, 2.0 ** -L)) < 1e-12
    plan.close()


def test_graph_skipped_inside_user_capture():
    """With the stream already capturing, the call is recorded into the
    user's graph instead of a graph of its own."""
    wl = wk.small_same(16)
    plan = pk.Plan(wl.A, pk.PHIKS_FP64)
    v = dev(wl.vs[0])
    out = torch.empty((wl.p + 1) * wl.N, device="cuda", dtype=torch.float64)
    ref = torch.empty_like(out)
    vn = [float(np.linalg.norm(wl.vs[0]))]
    plan.apply(wl.tau, wl.p, [v], ref, vnorms=vn)   # creates the bank
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.apply(wl.tau, wl.p, [v], out, torch.cuda.current_stream(), vnorms=vn, graph=1)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()
