"""bench.py's reference arm (the CPU oracle timed on the host cores) keeps
its JSON contract, and under a multi-rank launch only rank 0 works."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == "phi-actions/s" and line["unit"] == "phi-actions/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"] == "adr3d_lincomb_n64x64x64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_split_ceiling_arithmetic():
    """The precision form's ceiling: BF16X3 at n = 128 has three tensor-core
    products per algorithmic one and moves 8 bytes per element per mode pass
    (2 n / 8 = 32 flop per byte), a fused Tucker 8 bytes per element for
    2 d n flops (96 flop per byte)."""
    sys.path.insert(0, ROOT)
    import bench
    roof = {"peak": 1800.0, "achieved": 450.0}
    c = bench.split_ceiling("bf16x3", roof, 128, 3, 128 ** 3, 72, 1.0, 6000.0)
    assert abs(c["tensor_over_products"] - 600.0) < 1e-9
    assert abs(c["hbm_mode_pass"] - 6000.0 * 32 / 1000) < 1e-9
    assert abs(c["hbm_fused_tucker"] - 6000.0 * 96 / 1000) < 1e-9
    assert c["gemm_passes"]["bound"] == "hbm" and abs(c["gemm_passes"]["achieved"] - 150.0) < 1e-9
    assert abs(c["gemm_passes"]["frac"] - 150.0 / 192.0) < 1e-12
    # 72 Tucker operators of 2 N (3 n) flops in 1 ms
    rate = 72 * 2.0 * 128 ** 3 * 384 / 1e-3 / 1e12
    assert abs(c["call"]["achieved"] - rate) < 1e-9 and c["call"]["bound"] == "hbm"
    assert abs(c["call"]["frac"] - rate / 576.0) < 1e-12
    assert bench.split_ceiling("fp64", roof, 128, 3, 128 ** 3, 72, 1.0, 6000.0) is None


def test_batched_bound_and_served_flops_arithmetic():
    """The batched form's bound sums, per instance, the larger of its Tucker
    flops over the tensor ceiling and its Tucker bytes over HBM; the served
    form's flops are T# x 2 N sum(n) per apply."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench

    class W:
        def __init__(self, dims):
            self.A = [np.zeros((m, m)) for m in dims]
            self.N = int(np.prod(dims))
    insts = [W((512, 512)), W((16, 16, 16))]
    ms, fl = bench.batched_bound(insts, [10, 4], 600.0, 6000.0, 4)
    f0, f1 = 10 * 2.0 * 512 ** 2 * 1024, 4 * 2.0 * 16 ** 3 * 48
    b0, b1 = 10 * 8.0 * 512 ** 2, 4 * 8.0 * 16 ** 3
    want = max(f0 / 600e12, b0 / 6000e9) + max(f1 / 600e12, b1 / 6000e9)
    assert abs(ms - 1e3 * want) < 1e-12 and fl == f0 + f1
    reqs = [[{"tuckers": 3, "flops_per_tucker": 10.0}, {"tuckers": 2, "flops_per_tucker": 5.0}],
            [{"tuckers": 1, "flops_per_tucker": 7.0}]]
    assert bench.served_flops(reqs) == 3 * 10.0 + 2 * 5.0 + 7.0


def test_warm_served_records_tucker_counts_per_apply():
    """warm_served applies each distinct (plan, p) once and gives every apply
    of that key the Tucker count the library reported for it (stubs stand
    in for the library and torch)."""
    sys.path.insert(0, ROOT)
    import bench

    calls = []

    class PK:
        @staticmethod
        def phiks_apply_ex(plan, tau, p, v, out, stream, **kw):
            calls.append((plan, p, kw.get("tol")))

        @staticmethod
        def phiks_last_params(plan):
            plan_, p, _ = calls[-1]
            return (1, 5, 0, 10 * plan_ + p)

    class Torch:
        class cuda:
            @staticmethod
            def synchronize():
                pass

    def app(plan, p, tol=None):
        x = {"plan": plan, "tau": 1e-3, "p": p, "v": [], "out": None, "vnorms": [1.0] * (p + 1),
             "flops_per_tucker": 2.0}
        if tol is not None:
            x["tol"] = tol
        return x
    reqs = [[app(1, 2), app(2, 2)], [app(1, 3, 1e-6)], [app(1, 2)], [app(2, 2), app(1, 3, 1e-6)]]
    bench.warm_served(PK, Torch, reqs)
    assert [(c[0], c[1]) for c in calls] == [(1, 2), (2, 2), (1, 3)]
    assert calls[2][2] == 1e-6
    assert [[x["tuckers"] for x in r] for r in reqs] == [[12, 22], [13], [12], [22, 13]]
    assert bench.served_flops(reqs) == 2.0 * (12 + 22 + 13 + 12 + 22 + 13)
