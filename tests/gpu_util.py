"""Helpers for the GPU tests: seeded inputs to device tensors and calls
through the C ABI binding."""
import numpy as np
import torch

import paper_2210_07667_gb300 as pk


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def run_workload(wl, dtype=pk.PHIKS_FP64, **opts):
    """Apply the plan to the workload's vectors; returns (out as numpy float64
    array of shape (blocks, N), plan)."""
    tdt = torch.float64 if dtype in (pk.PHIKS_FP64, pk.PHIKS_FP64_EMU) else torch.float32
    plan = pk.Plan(wl.A, dtype)
    N = wl.N
    if wl.mode == "same":
        vs = [dev(wl.vs[0], tdt)]
        per = wl.p + (0 if wl.skip_phi0 else 1)
        out = torch.empty(wl.nscales * per * N, device="cuda", dtype=tdt)
    else:
        vs = [None if v is None else dev(v, tdt) for v in wl.vs]
        out = torch.empty(wl.nscales * N, device="cuda", dtype=tdt)
    kw = dict(nscales=wl.nscales, skip_phi0=int(wl.skip_phi0))
    kw.update(opts)
    plan.apply(wl.tau, wl.p, vs, out, **kw)
    torch.cuda.synchronize()
    return out.double().cpu().numpy().reshape(-1, N), plan


def rel_inf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())
