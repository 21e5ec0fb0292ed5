"""phiks_tucker_noalloc: the Tucker operator for callers that cannot allocate
device memory (an application that owns all device memory through its own
pool, or a latency-bound loop that must not pay for cudaMalloc / cudaFree).
Its intermediates live in a fixed device array inside the library instead of
a plan's workspace.  Its results must equal those of phiks_tucker and the
oracle's Tucker operator (Sec. 2, Lemma 1: W = V x_1 L_1 ... x_d L_d) call
after call, although every call reuses that same array.

This file is collected last on purpose, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_07667_gb300 as pk  # noqa: E402
from oracle import kron  # noqa: E402

from gpu_util import dev, rel_inf  # noqa: E402

TOL = 1e-14   # same bound as the phiks_tucker parity test


@pytest.mark.gpu
def test_noalloc_tucker_matches_planned_tucker_and_oracle_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.load(build_if_missing=True)
    rng = np.random.default_rng(2024)
    for dims in [(64, 48, 40), (1000,), (33, 17, 5, 9)]:
        N = int(np.prod(dims))
        plan = pk.Plan([np.eye(m) for m in dims])
        Lh = [rng.standard_normal((m, m)) for m in dims]
        Ls = [dev(L.ravel(order="F")) for L in Lh]
        for _ in range(2):   # two calls in a row share the library's scratch array
            Vh = rng.standard_normal(N)
            V = dev(Vh)
            ref = torch.empty(N, device="cuda", dtype=torch.float64)
            pk.phiks_tucker(plan.handle, V, ref, Ls)
            got = torch.full((N,), float("nan"), device="cuda", dtype=torch.float64)
            pk.phiks_tucker_noalloc(dims, V, got, Ls)
            torch.cuda.synchronize()
            exact = kron.vec(kron.tucker(kron.unvec(Vh, dims), Lh))
            g = got.cpu().numpy()
            assert rel_inf(g, ref.cpu().numpy()) < TOL
            assert rel_inf(g, exact) < TOL
        plan.close()


def test_noalloc_tucker_rejects_sizes_beyond_its_scratch():
    """N above 1,048,576 is refused before any device work (checked on the
    host, so fake device addresses are never touched)."""
    pk.load(build_if_missing=True)
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_tucker_noalloc((1024, 1025), 16, 32, [48, 64])
    assert e.value.status == 1 and "1,048,576" in str(e.value)


@pytest.mark.parametrize("w_off", [0, 8, 8 * 15, -8 * 15])
def test_noalloc_tucker_rejects_overlapping_vectors(w_off):
    """V and W sharing any element (the same start, or ranges that overlap by
    one element at either end) are refused on the host before any device
    work; the fake addresses are never touched."""
    pk.load(build_if_missing=True)
    base = 1 << 20
    with pytest.raises(pk.PhiksError) as e:
        pk.phiks_tucker_noalloc((4, 4), base, base + w_off, [48, 64])
    assert e.value.status == 1 and "overlap" in str(e.value)
