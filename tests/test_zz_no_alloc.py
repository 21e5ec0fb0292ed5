"""phiks_tucker_noalloc: the Tucker operator for callers that cannot allocate
device memory (an application that owns all device memory through its own
pool, or a latency-bound loop that must not pay for cudaMalloc / cudaFree).
Its intermediates live in a fixed device array inside the library instead of
a plan's workspace; its results must equal those of phiks_tucker, call after
call, although every call reuses that same array.

This file is collected last on purpose, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_07667_gb300 as pk  # noqa: E402

from gpu_util import dev, rel_inf  # noqa: E402

TOL = 1e-14   # same bound as the phiks_tucker parity test


@pytest.mark.gpu
def test_noalloc_tucker_matches_planned_tucker_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)
    rng = np.random.default_rng(2024)
    for dims in [(64, 48, 40), (1000,), (33, 17, 5, 9)]:
        N = int(np.prod(dims))
        plan = pk.Plan([np.eye(m) for m in dims])
        Ls = [dev(rng.standard_normal((m, m)).ravel(order="F")) for m in dims]
        for _ in range(2):   # two calls in a row share the library's scratch array
            V = dev(rng.standard_normal(N))
            ref = torch.empty(N, device="cuda", dtype=torch.float64)
            pk.phiks_tucker(plan.handle, V, ref, Ls)
            got = torch.full((N,), float("nan"), device="cuda", dtype=torch.float64)
            pk.phiks_tucker_noalloc(dims, V, got, Ls)
            torch.cuda.synchronize()
            assert rel_inf(got.cpu().numpy(), ref.cpu().numpy()) < TOL
        plan.close()


def test_noalloc_tucker_rejects_sizes_beyond_its_scratch():
    """N above 1,048,576 is refused before any device work (checked on the
    host, so fake device addresses are never touched)."""
    pk.load(build_if_missing=True)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_tucker_noalloc((1024, 1025), 16, 32, [48, 64])
    assert e.value.status == 1 and "1,048,576" in str(e.value)
