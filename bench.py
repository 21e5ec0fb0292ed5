"""Benchmark of the phiks hot path on one GB300 (or N replicas).

Workload: d = 3 advection-diffusion-reaction operator, n = 64 per mode
(N = 262144), FP64, linear combination exp(tau K) v_0 + sum_{l=1}^{4}
phi_l(tau K) v_l with outputs at tau, tau/2, tau/4 (three phi-actions per
step), tau = 5e-4, v_l ~ N(0, 1) seeded.  One step = one phiks_apply_ex call:
norms, parameter selection, the small FP64 exponentials (recomputed every
step), quadrature, squaring and the scale outputs.  The mu-mode products are
FP64 emulated on the tensor cores (exact bf16 digit products) by default;
`--dtype fp64` runs them on the FP64 pipe.  Both are timed, and both meet
the 1e-12 FP64 tolerance against the oracle.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(Taylor action of the augmented matrix) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wk  # noqa: E402

WORKLOAD = dict(n=64, p=4, nscales=3, tau=5e-4)
METRIC = "phi-actions/s"
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x flop/FMA x max SM clock


def workload():
    return wk.adr3d_lincomb(WORKLOAD["n"], tau=WORKLOAD["tau"], p=WORKLOAD["p"],
                            nscales=WORKLOAD["nscales"])


def config_dict(wl, extra=None):
    c = {"workload": wl.name, "d": len(wl.A), "n": wl.n, "N": wl.N, "p": wl.p, "mode": wl.mode,
         "nscales": wl.nscales, "tau": wl.tau, "operator": "FD ADR eps=1 alpha=(10,-20,5) rho=2",
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, world: int) -> float:
    """Slowest rank's timed milliseconds (gloo all-reduce when world > 1)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, ms_total: float) -> float:
    """Units per second of all ranks together (weak scaling: every rank runs
    its own replica of the workload)."""
    return world * units_per_rank_step * steps / (ms_total * 1e-3)


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def time_oracle_call(wl):
    from oracle import taylor_action as ta
    t0 = time.perf_counter()
    outs = [ta.lincomb(wl.A, wl.tau, wl.vs, 2.0 ** -L) for L in range(wl.nscales)]
    return time.perf_counter() - t0, outs


# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload()
    for _ in range(args.warmup):
        time_oracle_call(wl)
    tot = 0.0
    for _ in range(args.steps):
        dt, _ = time_oracle_call(wl)
        tot += dt
    value = wl.nscales * args.steps / tot
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "phi-actions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(wl),
        "cpu_baseline": {"value": value, "unit": "phi-actions/s", "cores": cores, "kind": "oracle",
                         "sample": "one full call per step (3 scale outputs), O3 Taylor action"},
        "e2e": {"value": value, "unit": "phi-actions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# tensor-pipe products executed per algorithmic product, per dtype, and the
# dense peak each runs against (tf32 from the measured bf16 peak times the
# nominal tf32 / bf16 ratio, 1.1 / 2.25 PFLOP/s)
TC_MULT = {"bf16x3": 3, "tf32x3": 3, "tf32": 1, "fp64emu": 28}
# (the resident form when one N tile covers a matrix, the streaming form otherwise;
# the brackets time every GEMM pass of either)
TC_KERNEL = {"bf16x3": "tc_gemm_res_kernel<0,2> / tc_gemm_kernel<0,2>",
             "tf32x3": "tc_gemm_res_kernel<1,2> / tc_gemm_kernel<1,2>",
             "tf32": "tc_gemm_res_kernel<1,1> / tc_gemm_kernel<1,1>",
             "fp64emu": "oz_gemm_kernel / oz_gemm_stream_kernel"}


def profile_roofline(dname, ms, launches, flops, kernel=None):
    """Roofline of the mu-mode kernel from phiks_profile_read sums: FP64 pipe
    for fp64 (alu), tensor pipe for the others (executed products)."""
    if launches <= 0 or ms <= 0:
        return None
    per_ms = ms / launches
    fl = flops / launches
    if dname == "fp64":
        ach = fl / (per_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP64_TFLOPS, "traffic": None,
                "kernel": kernel or "mode_product_f64 kernels", "per_launch_ms": per_ms, "flops_per_launch": fl,
                "peak_source": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)"}
    peaks, src = measured_peaks()
    peak = peaks["bf16_tflops"] * (1.0 if dname in ("bf16x3", "fp64emu") else 1.1 / 2.25)
    ach = TC_MULT[dname] * fl / (per_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": kernel or TC_KERNEL[dname], "per_launch_ms": per_ms,
            "algorithmic_flops_per_launch": fl, "executed_flops_per_launch": TC_MULT[dname] * fl,
            "peak_source": ("bf16_tflops (burst) of %s peaks" % src) if dname in ("bf16x3", "fp64emu")
            else ("bf16_tflops of %s peaks x 1.1/2.25 (nominal tf32/bf16)" % src)}


# bytes per element one split-dtype mode pass moves: its input planes read,
# the next pass's planes (or the last pass's FP32 result) written
SPLIT_PASS_BYTES = {"bf16x3": 4 + 4, "tf32x3": 8 + 8, "tf32": 4 + 4}


def split_ceiling(dname, roof, n, d, N, tuckers, ms, hbm_gbs):
    """The split dtypes' ceiling, min(tensor peak / products per algorithmic
    product, HBM x arithmetic intensity), in algorithmic TFLOP/s (2 N n_mu
    per mode pass):
      * GEMM passes: intensity 2 n / (bytes one mode pass moves per element),
        against the GEMM passes' own rate;
      * whole call: a Tucker operator fused over its d modes would move 4 + 4
        bytes per element (FP32 in and out) for 2 N sum(n) flops, against the
        Tucker flops of the step over its time.
    (The 129 MB L2 can hold part of a batch's planes, so the measured rate
    may exceed the per-pass HBM figure.)"""
    if not roof or dname not in SPLIT_PASS_BYTES:
        return None
    tensor = roof["peak"] / TC_MULT[dname]
    hbm_pass = hbm_gbs * 1e9 * (2.0 * n / SPLIT_PASS_BYTES[dname]) / 1e12
    hbm_fused = hbm_gbs * 1e9 * (2.0 * d * n / 8.0) / 1e12
    pass_rate = roof["achieved"] / TC_MULT[dname]
    call_rate = tuckers * 2.0 * N * d * n / (ms * 1e-3) / 1e12
    c_pass, c_call = min(tensor, hbm_pass), min(tensor, hbm_fused)
    return {"unit": "TFLOP/s (algorithmic)", "tensor_over_products": tensor,
            "hbm_mode_pass": hbm_pass, "hbm_fused_tucker": hbm_fused,
            "gemm_passes": {"achieved": pass_rate, "ceiling": c_pass, "frac": pass_rate / c_pass,
                            "bound": "tensor" if tensor <= hbm_pass else "hbm"},
            "call": {"achieved": call_rate, "ceiling": c_call, "frac": call_rate / c_call,
                     "bound": "tensor" if tensor <= hbm_fused else "hbm"}}


# dram__bytes_read.sum + dram__bytes_write.sum per mu-mode product of
# oz_gemm_kernel<32> from an ncu capture of the kernel as it stands (six
# four-product launches of this workload, cold caches: 14.861 MB read, 0
# written; the summary of that capture under profiles/ gives the command);
# None once the kernel changes
OZ_GEMM_TRAFFIC_PER_PRODUCT = 14.861e6 / 4
# dram__bytes_read.sum + dram__bytes_write.sum per launch of tc_gemm_res_kernel<0,2>
# on the precision form's Chebyshev 128^3 operator (each launch a nine-tensor batch),
# from an ncu capture of the kernel as it stands (two launches, 102.0 and 96.8 MB; the
# summary under profiles/ gives the command); None once the kernel changes
TC_RES_BF16X3_CHEB128_TRAFFIC_PER_LAUNCH = 99.4e6
# bf16 digit products the emulated pass executes per FP64 product (digit
# planes s + t <= 6 of seven per operand)
OZ_DIGIT_PRODUCTS = 28


def run_phiks(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)

    wl = workload()
    N = wl.N
    # FP64-accurate arithmetic: the emulated products (default) or the DFMA path
    main_dtype = pk.PHIKS_FP64 if args.dtype == "fp64" else pk.PHIKS_FP64_EMU
    other_dtype = pk.PHIKS_FP64 if main_dtype == pk.PHIKS_FP64_EMU else pk.PHIKS_FP64_EMU
    stream = torch.cuda.Stream()
    vs = [torch.from_numpy(v).cuda() for v in wl.vs]
    flush = torch.empty(256 << 20, device="cuda", dtype=torch.uint8)   # 256 MiB > 129 MB L2
    # every call replays its kernels from a CUDA graph captured on the second
    # call (phiks_options.graph); norms and the (s, q) selection run each call
    opts = pk.make_options(nscales=wl.nscales, no_cache=1, graph=1)
    opts_plain = pk.make_options(nscales=wl.nscales, no_cache=1)
    # caller norms: no synchronisation inside the call (profiling pass only)
    opts_plain_vn = pk.make_options(nscales=wl.nscales, no_cache=1,
                                    vnorms=[float(np.linalg.norm(v)) for v in wl.vs])

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_calls(plan, out, o, steps, ev_list=None):
        """Summed ms of `steps` calls, L2 flushed (untimed) before each."""
        tot = 0.0
        for k in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                e0.record(stream)
                pk.phiks_apply_ex(plan.handle, wl.tau, wl.p, vs, out, stream, opts=o)
                e1.record(stream)
            if ev_list is not None:
                ev_list.append((e0, e1))
            else:
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
        return tot

    def kernel_profile(plan, out):
        """Per-launch ms and algorithmic flops of the mu-mode kernel (events
        around every launch, a separate pass).  A 20 ms spin on the stream
        before each call lets the host queue the whole call first, so that
        the brackets time the kernels and not the host's launch rate."""
        pk.phiks_profile_enable(plan.handle, True)
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                torch.cuda._sleep(int(2.0e9 * 0.02))
                pk.phiks_apply_ex(plan.handle, wl.tau, wl.p, vs, out, stream, opts=opts_plain_vn)
        kms, kl, kfl = pk.phiks_profile_read(plan.handle)
        pk.phiks_profile_enable(plan.handle, False)
        return kms / max(kl, 1), kfl / max(kl, 1), kfl / args.steps

    def roofline(dtype, per_launch_ms, flops_per_launch):
        if dtype == pk.PHIKS_FP64:
            achieved = flops_per_launch / (per_launch_ms * 1e-3) / 1e12
            return {"bound": "alu", "achieved": achieved, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / PEAK_FP64_TFLOPS, "traffic": None,
                    "kernel": "mode_product_f64_kernel", "per_launch_ms": per_launch_ms,
                    "flops_per_launch": flops_per_launch,
                    "peak_source": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)"}
        peaks, src = measured_peaks()
        # The emulated pass is a dense contraction on the tensor pipe: it
        # executes 28 bf16 digit products (2 N n_mu flop each) per FP64
        # mu-mode product, against the bf16 dense peak (burst: the kernel is
        # timed launch by launch).  Its operands stay in L2 (about 0 DRAM
        # writes, ncu), so HBM is reported beside it only as context: N
        # doubles in and N out per product.
        products = flops_per_launch / (2.0 * N * WORKLOAD["n"])
        executed = OZ_DIGIT_PRODUCTS * flops_per_launch
        achieved = executed / (per_launch_ms * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        nbytes = 16.0 * N * products
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": None if OZ_GEMM_TRAFFIC_PER_PRODUCT is None else OZ_GEMM_TRAFFIC_PER_PRODUCT * products,
                "kernel": "oz_gemm_kernel<32>", "per_launch_ms": per_launch_ms,
                "products_per_launch": products, "fp64_flops_per_launch": flops_per_launch,
                "bf16_flops_per_launch": executed,
                "peak_source": "bf16_tflops (burst) of %s peaks" % src,
                "hbm_context": {"bytes_per_launch": nbytes,
                                "achieved_gbs": nbytes / (per_launch_ms * 1e-3) / 1e9,
                                "peak_gbs": peaks["hbm_gbs"]}}

    # ---- headline path
    plan = pk.Plan(wl.A, main_dtype)
    out = torch.empty(wl.nscales * N, device="cuda", dtype=torch.float64)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            pk.phiks_apply_ex(plan.handle, wl.tau, wl.p, vs, out, stream, opts=opts)
    torch.cuda.synchronize()
    s_, q_, T_, tuckers = plan.last_params()

    # ---- timed region: K steps, L2 flushed before each (flush not timed)
    ev = []
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = pk.phiks_kernel_launches()
    t_wall = time.perf_counter()
    timed_calls(plan, out, opts, args.steps, ev)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = pk.phiks_kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    pk.phiks_device_status(plan.handle, stream)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), ws)
    ms_step = ms / args.steps
    value = whole_job_rate(wl.nscales, args.steps, ws, ms)
    gpu_out = out.cpu().numpy().copy()

    per_launch_ms, flops_per_launch, step_flops = kernel_profile(plan, out)
    pms = timed_calls(plan, out, opts_plain, args.steps)

    # ---- cached small exponentials (steady state of a fixed-step integrator)
    opts_c = pk.make_options(nscales=wl.nscales, graph=1)
    with torch.cuda.stream(stream):
        for _ in range(2):
            pk.phiks_apply_ex(plan.handle, wl.tau, wl.p, vs, out, stream, opts=opts_c)
    torch.cuda.synchronize()
    cms = timed_calls(plan, out, opts_c, args.steps)

    # ---- end to end through the C ABI with host buffers
    # the step's inputs as one pinned block and one device block (one copy in)
    nvec = len(wl.vs)
    hv = torch.from_numpy(np.concatenate(wl.vs)).pin_memory()
    hout = torch.empty(wl.nscales * N, dtype=torch.float64).pin_memory()
    dbuf = torch.empty(nvec * N, device="cuda", dtype=torch.float64)
    dv = [dbuf[i * N:(i + 1) * N] for i in range(nvec)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(args.steps + 2):   # two untimed calls capture the graph for dv
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            e0.record(stream)
            dbuf.copy_(hv, non_blocking=True)
            pk.phiks_apply_ex(plan.handle, wl.tau, wl.p, dv, out, stream, opts=opts)
            hout.copy_(out, non_blocking=True)
            e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            e2e_ms += e0.elapsed_time(e1)
    h2d = hv.numel() * 8
    d2h = hout.numel() * 8

    emu = main_dtype == pk.PHIKS_FP64_EMU
    line = {
        "metric": METRIC, "value": value, "unit": "phi-actions/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (bf16-digit products emulated on tcgen05)" if main_dtype == pk.PHIKS_FP64_EMU else "f64",
        "data": "synthetic",
        "config": config_dict(wl, {"s": s_, "q": q_, "T#": T_, "tuckers_per_step": tuckers,
                                   "l2": "flushed before every timed step (256 MiB write, untimed)",
                                   "small_exponentials": "recomputed every step",
                                   "submission": "CUDA graph of the call's kernels, replayed each "
                                                 "call after the norms and the (s, q) selection"}),
        "mu_mode_products": ("FP64 emulated on tcgen05: exact bf16 digit products, FP32 "
                             "accumulation, rounded to FP64" if emu else "FP64 DFMA"),
        "mu_mode_tflops": step_flops / (ms_step * 1e-3) / 1e12,
        "value_cached_exponentials": ws * wl.nscales * args.steps / (cms * 1e-3),
        "value_plain_launches": ws * wl.nscales * args.steps / (pms * 1e-3),
        "roofline": roofline(main_dtype, per_launch_ms, flops_per_launch),
        "e2e": {"value": ws * wl.nscales * args.steps / (e2e_ms * 1e-3), "unit": "phi-actions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    plan.close()

    # ---- the other FP64-accurate path on the same workload
    other_key = "fp64_dfma" if emu else "fp64_emulated"
    other_out = None
    try:
        po = pk.Plan(wl.A, other_dtype)
        oo = torch.empty_like(out)
        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 3)):
                pk.phiks_apply_ex(po.handle, wl.tau, wl.p, vs, oo, stream, opts=opts)
        torch.cuda.synchronize()
        oev = []
        timed_calls(po, oo, opts, args.steps, oev)
        torch.cuda.synchronize()
        pk.phiks_device_status(po.handle, stream)
        oms = max_over_ranks(sum(a.elapsed_time(b) for a, b in oev), ws)
        other_out = oo.cpu().numpy().copy()
        opl, ofl, _ = kernel_profile(po, oo)
        line[other_key] = {"value": whole_job_rate(wl.nscales, args.steps, ws, oms),
                           "ms_per_step": oms / args.steps, "headline_speedup_over_it": oms / ms,
                           "roofline": roofline(other_dtype, opl, ofl)}
        po.close()
    except Exception as ex:  # plan refused (shape) or device error: report, keep the headline
        line[other_key] = {"error": str(ex)[:200]}
    if rank == 0 and not args.no_cpu_baseline:
        dt, outs = time_oracle_call(wl)

        def err_of(o):
            return max(float(np.abs(o[L * N:(L + 1) * N] - outs[L]).max() / np.abs(outs[L]).max())
                       for L in range(wl.nscales))
        line["rel_err_vs_oracle"] = err_of(gpu_out)
        if other_out is not None:
            line[other_key]["rel_err_vs_oracle"] = err_of(other_out)
        line["cpu_baseline"] = {"value": wl.nscales / dt, "unit": "phi-actions/s",
                                "cores": oracle_threads(), "kind": "oracle",
                                "sample": "one full call (3 scale outputs), O3 Taylor action, %.1f s" % dt}
        # context only: the paper's method itself (the oracle's step-by-step
        # restatement, numpy BLAS mode products) on the host cores, same (s, q)
        from oracle import phiks_ref
        t0 = time.perf_counter()
        phiks_ref.lincomb(wl.A, wl.tau, wl.vs, s_, q_, nscales=wl.nscales)
        dtp = time.perf_counter() - t0
        line["cpu_phiks_context"] = {"value": wl.nscales / dtp, "unit": "phi-actions/s",
                                     "cores": oracle_threads(), "s": s_, "q": q_,
                                     "note": "phiks restated step by step in numpy (FP64), one call"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
PRECISION_DTYPES = ["fp64", "fp64emu", "tf32", "tf32x3", "bf16x3"]
# relative accuracy asked of the selection per dtype (tol = rel * ||v||)
PRECISION_TOL = {"fp64": None, "fp64emu": None, "tf32": 1e-4, "tf32x3": 1e-7, "bf16x3": 1e-6}


def run_precision(args):
    """The precision form: d = 3, n = 128 (N = 2,097,152), Chebyshev D^2
    Dirichlet (tau = 5e-7) or FD Laplacian (tau = 1e-4), phi_1..phi_3 of 8
    N(0,1) vectors per step, every dtype timed and compared with the FP64 GPU
    result."""
    import torch
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    torch.cuda.set_device(0)
    tau = 5e-7 if args.variant == "cheb" else 1e-4
    wl = wk.cheb3d_same(n=args.n, nrhs=8, tau=tau, variant=args.variant)
    N, p = wl.N, wl.p
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, device="cuda", dtype=torch.uint8)
    results = {}
    oracle_rows = {}
    ref_out = None
    dtypes = PRECISION_DTYPES if args.dtype == "all" else ["fp64", args.dtype]
    head = args.dtype if args.dtype != "all" else "bf16x3"
    head_e2e, head_launches = None, 0
    if args.no_ref:
        dtypes = [d for d in dtypes if d != "fp64"]
    for name in dtypes:
        dt = pk.DTYPES[name]
        tdt = torch.float64 if name in ("fp64", "fp64emu") else torch.float32
        plan = pk.Plan(wl.A, dt)
        # inputs and outputs as views of one device block each (one copy in,
        # one copy out in the end-to-end figure)
        vbuf = torch.from_numpy(np.concatenate(wl.vs)).to(device="cuda", dtype=tdt)
        vs = [vbuf[i * N:(i + 1) * N] for i in range(len(wl.vs))]
        obuf = torch.empty(len(wl.vs) * p * N, device="cuda", dtype=tdt)
        outs = [obuf[i * p * N:(i + 1) * p * N] for i in range(len(wl.vs))]
        norms = [float(np.linalg.norm(v.astype(np.float32) if tdt == torch.float32 else v)) for v in wl.vs]
        kw = dict(skip_phi0=1)
        if PRECISION_TOL[name] is not None:
            kw["tol"] = PRECISION_TOL[name] * max(norms)
        # the small exponentials are rebuilt once per step (by the first call;
        # the other seven vectors share tau and reuse them)
        opts = [pk.make_options(vnorms=[nv], no_cache=int(i == 0), **kw) for i, nv in enumerate(norms)]

        def step():
            for v, o, op in zip(vs, outs, opts):
                pk.phiks_apply_ex(plan.handle, wl.tau, p, [v], o, stream, opts=op)

        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 3)):
                step()
        torch.cuda.synchronize()
        pk.phiks_device_status(plan.handle, stream)
        s_, q_, T_, tk = plan.last_params()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        l0 = pk.phiks_kernel_launches()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        launches = pk.phiks_kernel_launches() - l0
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        pk.phiks_device_status(plan.handle, stream)
        pk.phiks_profile_enable(plan.handle, True)
        with torch.cuda.stream(stream):
            step()
        kms, kl, kfl = pk.phiks_profile_read(plan.handle)
        pk.phiks_profile_enable(plan.handle, False)
        out = torch.stack(outs).double().cpu().numpy()
        oracle_rows[name] = out[0][:N].copy()      # phi_1 of vector 0
        if name == "fp64":
            ref_out = out
            err = 0.0
        elif ref_out is None:
            err = None
        else:
            err = max(float(np.abs(out[k] - ref_out[k]).max() / np.abs(ref_out[k]).max())
                      for k in range(len(outs)))
        results[name] = {"ms_per_step": ms, "phi_actions_per_s": 3 * len(vs) / (ms * 1e-3),
                         "rel_err_vs_fp64": err, "s": s_, "q": q_, "tuckers_per_call": tk,
                         "mu_mode_tflops_algorithmic": kfl / max(kms, 1e-9) / 1e9,
                         "mu_mode_ms_per_call": kms / len(vs), "gpu_launches_per_step": launches // args.steps,
                         "roofline": profile_roofline(name, kms, kl, kfl)}
        roof = results[name]["roofline"]
        if roof and name == "bf16x3" and args.variant == "cheb" and args.n == 128:
            roof["traffic"] = TC_RES_BF16X3_CHEB128_TRAFFIC_PER_LAUNCH
        results[name]["ceiling"] = split_ceiling(name, roof, args.n, 3, N, tk * len(vs), ms,
                                                 measured_peaks()[0]["hbm_gbs"])
        if name == head:
            # end to end through the C ABI: the 8 inputs from pinned host
            # memory and the 24 outputs back inside the timed region
            hv = torch.from_numpy(np.concatenate(wl.vs)).to(dtype=tdt).pin_memory()
            ho = torch.empty(len(vs) * p * N, dtype=tdt).pin_memory()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2e_ms = 0.0
            for k in range(2):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 0xFF)
                    e0.record(stream)
                    vbuf.copy_(hv, non_blocking=True)
                    step()
                    ho.copy_(obuf, non_blocking=True)
                    e1.record(stream)
                torch.cuda.synchronize()
                e2e_ms += e0.elapsed_time(e1) / 2
            esz = 8 if tdt == torch.float64 else 4
            head_e2e = {"value": 3 * len(vs) / (e2e_ms * 1e-3), "unit": "phi-actions/s",
                        "h2d_bytes_per_step": len(vs) * N * esz, "d2h_bytes_per_step": len(vs) * p * N * esz}
            head_launches = launches
        plan.close()
    if "fp64" in results:
        base = results["fp64"]["ms_per_step"]
        for r in results.values():
            r["speedup_vs_fp64"] = base / r["ms_per_step"]
    # every dtype against the oracle on one output: phi_1(tau K) v_0 (O3;
    # the inputs as each dtype saw them)
    if not args.no_oracle:
        from oracle import taylor_action as ta
        t0 = time.perf_counter()
        for key, v0 in (("f64", wl.vs[0]), ("f32", wl.vs[0].astype(np.float32).astype(np.float64))):
            ex = ta.lincomb(wl.A, wl.tau, [None, v0])
            for name, r in results.items():
                if ("f64" if name in ("fp64", "fp64emu") else "f32") != key:
                    continue
                got = oracle_rows[name]
                r["rel_err_vs_oracle"] = float(np.abs(got - ex).max() / np.abs(ex).max())
        oracle_s = time.perf_counter() - t0
    else:
        oracle_s = None
    h = results[head]
    line = {"metric": METRIC, "value": h["phi_actions_per_s"], "unit": "phi-actions/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16x3": "bf16x3 (fp32 accumulate)", "tf32": "tf32", "tf32x3": "tf32x3",
                      "fp64": "f64", "fp64emu": "f64 (emulated on tcgen05)"}[head],
            "data": "synthetic",
            "config": {"workload": wl.name, "d": 3, "n": [args.n] * 3, "N": N, "p": 3, "mode": "same",
                       "skip_phi0": True, "nrhs": 8, "tau": tau, "variant": args.variant,
                       "l2": "flushed before every timed step (256 MiB write, untimed)"},
            "rel_err_vs_fp64": h["rel_err_vs_fp64"], "rel_err_vs_oracle": h.get("rel_err_vs_oracle"),
            "oracle_check": {"output": "phi_1(tau K) v_0 (one of 24 per step)", "oracle": "O3 Taylor action",
                             "seconds": oracle_s},
            "roofline": h.get("roofline"), "ceiling": h.get("ceiling"), "e2e": head_e2e,
            "gpu_launches": head_launches,
            "cpu_baseline": None if oracle_s is None else
            {"value": 2.0 / oracle_s, "unit": "phi-actions/s", "cores": oracle_threads(), "kind": "oracle",
             "sample": "phi_1(tau K) v_0 twice (the input as FP64 and as FP32 saw it), O3 Taylor action, "
                       "%.1f s" % oracle_s},
            "per_dtype": results}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_batched(args):
    """The batched form: uneven-size independent instances (half d = 2 with
    n_mu in {64..512}, half d = 3 with n_mu in {16..96}), phi_1..phi_3 each.
    Timed: the whole batch as one CUDA graph over worker streams (split dtype),
    against the same instances one after another in FP64 on one stream.
    Small exponentials are cached per instance (fixed step, as in an
    integrator); their one-time cost is reported separately."""
    import torch
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    torch.cuda.set_device(0)
    insts = wk.batched_instances(args.count)
    name = "bf16x3" if args.dtype == "all" else args.dtype
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, device="cuda", dtype=torch.uint8)
    phi_per_step = 3 * len(insts)

    def setup(dname):
        dt = pk.DTYPES[dname]
        tdt = torch.float64 if dname in ("fp64", "fp64emu") else torch.float32
        rows = []
        for w in insts:
            plan = pk.Plan(w.A, dt)
            v = torch.from_numpy(w.vs[0]).to(device="cuda", dtype=tdt)
            out = torch.empty(3 * w.N, device="cuda", dtype=tdt)
            nv = float(np.linalg.norm(w.vs[0].astype(np.float32) if dname != "fp64" else w.vs[0]))
            kw = dict(skip_phi0=1, vnorms=[nv])
            if PRECISION_TOL[dname] is not None:
                kw["tol"] = PRECISION_TOL[dname] * nv
            rows.append((plan, w.tau, 3, [v], out, pk.make_options(**kw)))
        return rows

    def inst_tuple(rows):
        return [(r[0].handle, r[1], r[2], r[3], r[4], r[5]) for r in rows]

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    res = {}
    # split dtype, batch over worker streams, captured in one CUDA graph
    t0 = time.perf_counter()
    rows = setup(name)
    batch = pk.Batch(args.streams)
    insts_t = inst_tuple(rows)
    with torch.cuda.stream(stream):
        batch.apply(insts_t, stream)      # parameter selection, workspaces, small exponentials
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        batch.apply(insts_t, stream)
    torch.cuda.synchronize()
    graph = batch.capture(insts_t, stream)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            batch.launch(graph, stream)
    torch.cuda.synchronize()
    l0 = pk.phiks_kernel_launches()
    ms_graph = timed(lambda: batch.launch(graph, stream), args.steps)
    tk_list = [r[0].last_params()[3] for r in rows]
    tucks = sum(tk_list)
    bound_ms, bound_fl = batched_bound(insts, tk_list, tensor_ceiling_tflops(name),
                                       measured_peaks()[0]["hbm_gbs"], rows[0][4].element_size())
    for r in rows:
        pk.phiks_device_status(r[0].handle, stream)
    out_split = [r[4].double().cpu().numpy() for r in rows]
    # same instances, split dtype, one stream, no graph
    def seq(rr):
        def f():
            for r in rr:
                pk.phiks_apply_ex(r[0].handle, r[1], r[2], r[3], r[4], stream, opts=r[5])
        return f
    ms_seq = timed(seq(rows), max(1, args.steps // 2))
    # launches of one step (the graph's kernels, counted from a plain batch)
    lp0 = pk.phiks_kernel_launches()
    with torch.cuda.stream(stream):
        batch.apply(insts_t, stream)
    torch.cuda.synchronize()
    launches_per_step = pk.phiks_kernel_launches() - lp0
    # kernel roofline: events around every GEMM pass of every instance, the
    # instances one after another on one stream (brackets of concurrent
    # streams would overlap)
    for r in rows:
        pk.phiks_profile_enable(r[0].handle, True)
    with torch.cuda.stream(stream):
        seq(rows)()
    torch.cuda.synchronize()
    kms = kl = kfl = 0.0
    for r in rows:
        a, b, c = pk.phiks_profile_read(r[0].handle)
        pk.phiks_profile_enable(r[0].handle, False)
        kms, kl, kfl = kms + a, kl + b, kfl + c
    roof = profile_roofline(name, kms, int(kl), kfl)
    if roof:
        roof["note"] = "GEMM passes timed with the instances run one after another on one stream"
    # end to end: every instance's input from pinned host memory and its
    # three outputs back, around the graph launch
    hin = [torch.from_numpy(w.vs[0]).to(dtype=r[3][0].dtype).pin_memory() for w, r in zip(insts, rows)]
    hout = [torch.empty_like(r[4], device="cpu").pin_memory() for r in rows]

    def e2e_step():
        for h, r in zip(hin, rows):
            r[3][0].copy_(h, non_blocking=True)
        batch.launch(graph, stream)
        for h, r in zip(hout, rows):
            h.copy_(r[4], non_blocking=True)
    ms_e2e = timed(e2e_step, max(1, args.steps))
    esz = rows[0][4].element_size()
    e2e = {"value": phi_per_step / (ms_e2e * 1e-3), "unit": "phi-actions/s",
           "h2d_bytes_per_step": sum(w.N for w in insts) * esz,
           "d2h_bytes_per_step": sum(3 * w.N for w in insts) * esz}
    res[name + "_graph"] = {"ms_per_step": ms_graph, "phi_actions_per_s": phi_per_step / (ms_graph * 1e-3),
                            "streams": args.streams, "tuckers_per_step": tucks,
                            "first_call_s": setup_s}
    res[name + "_sequential"] = {"ms_per_step": ms_seq, "phi_actions_per_s": phi_per_step / (ms_seq * 1e-3)}
    batch.destroy_graph(graph)
    batch.close()
    for r in rows:
        r[0].close()
    # FP64 reference path, one stream
    if not args.no_ref:
        rows64 = setup("fp64")
        with torch.cuda.stream(stream):
            seq(rows64)()
        torch.cuda.synchronize()
        ms64 = timed(seq(rows64), 1)
        errs = []
        for r, o in zip(rows64, out_split):
            ref = r[4].cpu().numpy()
            errs.append(float(np.abs(o - ref).max() / np.abs(ref).max()))
        res["fp64_sequential"] = {"ms_per_step": ms64, "phi_actions_per_s": phi_per_step / (ms64 * 1e-3)}
        res[name + "_graph"]["rel_err_vs_fp64_max"] = max(errs)
        res[name + "_graph"]["speedup_vs_fp64"] = ms64 / ms_graph
        for r in rows64:
            r[0].close()
    h = res[name + "_graph"]
    cpu = None
    if not args.no_oracle:
        h["oracle_check"] = oracle_check_instances(insts, out_split, name)
        oc = h["oracle_check"]
        cpu = {"value": 3 * len(oc["instances"]) / oc["seconds"], "unit": "phi-actions/s",
               "cores": oracle_threads(), "kind": "oracle",
               "sample": "phi_1..phi_3 of the cheapest d=2 and d=3 instance (O3), %.1f s" % oc["seconds"]}
    line = {"metric": METRIC, "value": h["phi_actions_per_s"], "unit": "phi-actions/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": name,
            "data": "synthetic", "rel_err_vs_oracle": h.get("oracle_check", {}).get("max_rel_err"),
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
            "aggregate_bound": {"ms": bound_ms, "frac": bound_ms / h["ms_per_step"],
                                "achieved_tflops_algorithmic": bound_fl / (h["ms_per_step"] * 1e-3) / 1e12,
                                "definition": "sum over instances of max(Tucker flops / tensor ceiling, "
                                              "Tucker bytes / HBM), fused Tucker operators"},
            "gpu_launches": launches_per_step * args.steps, "launches_per_step": launches_per_step,
            "config": {"workload": "batched_adr_%d_instances" % len(insts), "instances": len(insts),
                       "d2_n": "64..512 step 32", "d3_n": "16..96 step 8", "p": 3, "skip_phi0": True,
                       "small_exponentials": "cached per instance",
                       "l2": "flushed before every timed step (256 MiB write, untimed)"},
            "per_variant": res}
    print(json.dumps(line), flush=True)
    return 0


def batched_bound(insts, tuckers, tensor_tflops, hbm_gbs, elt):
    """The batched form's bound: the sum over instances of max(Tucker flops /
    tensor ceiling, Tucker bytes / HBM), every Tucker operator fused over its
    modes (input read and output written once: 2 elt bytes per element for
    2 N sum(n) flops).  Returns (bound in ms, algorithmic flops)."""
    t = fl = 0.0
    for w, tk in zip(insts, tuckers):
        f = tk * 2.0 * w.N * sum(a.shape[0] for a in w.A)
        b = tk * 2.0 * elt * w.N
        t += max(f / (tensor_tflops * 1e12), b / (hbm_gbs * 1e9))
        fl += f
    return t * 1e3, fl


def tensor_ceiling_tflops(dname):
    """Algorithmic TFLOP/s ceiling of a dtype's products: the FP64 peak, or
    the measured bf16 peak (tf32 at the nominal 1.1 / 2.25 ratio) over the
    tensor-core products per algorithmic product."""
    if dname == "fp64":
        return PEAK_FP64_TFLOPS
    peaks, _ = measured_peaks()
    return peaks["bf16_tflops"] * (1.0 if dname in ("bf16x3", "fp64emu") else 1.1 / 2.25) / TC_MULT[dname]


def o3_cost(A, tau, N):
    """Rough cost of the O3 oracle: N sum(n) flops per matvec, ~20 terms per
    unit of tau ||K||_1."""
    return N * sum(a.shape[0] for a in A) * max(1.0, abs(tau) * sum(float(np.abs(a).sum(0).max()) for a in A))


def oracle_check_instances(insts, outs, dname):
    """phi_1..phi_3 of the cheapest d = 2 and d = 3 instances against the O3
    oracle (the inputs rounded as the dtype saw them)."""
    from oracle import taylor_action as ta
    t0 = time.perf_counter()
    picked = []
    for d in (2, 3):
        cand = [(o3_cost(w.A, w.tau, w.N), k) for k, w in enumerate(insts) if len(w.A) == d]
        if cand:
            picked.append(min(cand)[1])
    errs = {}
    for k in picked:
        w = insts[k]
        v = w.vs[0] if dname in ("fp64", "fp64emu") else w.vs[0].astype(np.float32).astype(np.float64)
        ex = ta.same(w.A, w.tau, v, 3, ells=[1, 2, 3])
        got = outs[k].reshape(3, w.N)
        errs[w.name] = max(float(np.abs(got[l] - ex[l]).max() / np.abs(ex[l]).max()) for l in range(3))
    return {"instances": errs, "max_rel_err": max(errs.values()) if errs else None,
            "outputs": "phi_1..phi_3 of the cheapest d=2 and d=3 instance (O3)",
            "seconds": time.perf_counter() - t0}


def served_operators(cls, n):
    if cls == "ac":
        return [wk.ac_operator(n)]
    if cls == "adr":
        return [[wk.fd_adr_dirichlet(n, 1.0, a, 2.0 / 3) for a in (10.0, -20.0, 5.0)]]
    return list(wk.brusselator_operators(n))


def oracle_check_served(specs, requests):
    """The smallest request of each class (its first apply) against the O3
    oracle."""
    from oracle import taylor_action as ta
    t0 = time.perf_counter()
    errs = {}
    for cls in ("ac", "adr", "bru"):
        ks = [k for k, sp in enumerate(specs) if sp[0] == cls]
        if not ks:
            continue
        k = min(ks, key=lambda j: specs[j][1])
        x = requests[k][0]
        A = served_operators(cls, specs[k][1])[0]
        vs = [v.double().cpu().numpy() for v in x["v"]]
        ex = ta.lincomb(A, x["tau"], vs)
        got = x["out"].double().cpu().numpy()
        errs["%s_n%d" % (cls, specs[k][1])] = float(np.abs(got - ex).max() / np.abs(ex).max())
    return {"requests": errs, "max_rel_err": max(errs.values()) if errs else None,
            "outputs": "the smallest request of each class, first apply (O3)",
            "seconds": time.perf_counter() - t0}


# ---------------------------------------------------------------------------
def build_served(pk, torch, arrivals, specs, dtype_name, tol_rel, ring=64):
    """Device-resident plans per (class, n, species), seeded inputs per
    (class, n); outputs from a ring of `ring` buffers per (class, n, species)
    (requests in flight together are fewer than the ring, so two of them
    never share one); returns (requests, plans, n_applies)."""
    dt = pk.DTYPES[dtype_name]
    tdt = torch.float64 if dtype_name in ("fp64", "fp64emu") else torch.float32
    plans, inputs, outs, used = {}, {}, {}, {}
    requests = []
    n_applies = 0
    for k, (cls, n, p) in enumerate(specs):
        ops = served_operators(cls, n)
        N = int(np.prod([a.shape[0] for a in ops[0]]))
        key = (cls, n)
        if key not in inputs:  # one seeded input set per (class, n), shared by its requests
            seed = 1000000 + 10000 * ("ac", "adr", "bru").index(cls) + 5 * n
            vs = [wk.normal(seed + l, N).astype(np.float32).astype(np.float64) for l in range(5)]
            inputs[key] = ([torch.from_numpy(v).to(device="cuda", dtype=tdt) for v in vs],
                           [float(np.linalg.norm(v)) for v in vs])
        vdev, vn = inputs[key]
        g = used.get(key, 0)
        used[key] = g + 1
        apps = []
        for sp, A in enumerate(ops):
            pkey = (cls, n, sp)
            if pkey not in plans:
                plans[pkey] = pk.Plan(A, dt)
                outs[pkey] = []
            if len(outs[pkey]) < ring:
                outs[pkey].append(torch.empty(N, device="cuda", dtype=tdt))
            out = outs[pkey][g % ring]
            x = {"plan": plans[pkey].handle, "tau": wk.SERVED_CLASSES[cls]["tau"], "p": p,
                 "v": vdev[: p + 1], "out": out, "vnorms": vn[: p + 1],
                 "flops_per_tucker": 2.0 * N * sum(a.shape[0] for a in A)}
            if tol_rel is not None:
                x["tol"] = tol_rel * max(vn[: p + 1])
            apps.append(x)
            n_applies += 1
        requests.append(apps)
    return requests, plans, n_applies


def warm_served(pk, torch, requests):
    """One apply per distinct (plan, p): parameter search and exponentials
    happen here, not while serving.  Records each apply's Tucker operators
    (the same for every apply of one (plan, p): one tau and one input set per
    class and size)."""
    tuckers = {}
    for apps in requests:
        for x in apps:
            key = (x["plan"], x["p"])
            if key not in tuckers:
                kw = dict(vnorms=x["vnorms"])
                if "tol" in x:
                    kw["tol"] = x["tol"]
                pk.phiks_apply_ex(x["plan"], x["tau"], x["p"], x["v"], x["out"], None, **kw)
                tuckers[key] = pk.phiks_last_params(x["plan"])[3]
            x["tuckers"] = tuckers[key]
    torch.cuda.synchronize()


def served_flops(requests):
    """Algorithmic Tucker flops of a trace: T# x 2 N sum(n) per apply."""
    return sum(x["tuckers"] * x["flops_per_tucker"] for apps in requests for x in apps)


def run_served(args):
    """The served form: Poisson arrivals of Allen-Cahn, ADR and Brusselator
    stage requests (linear combinations, p in {2,3,4}), continuous batching
    over `slots` streams with HBM-budget admission, each request's applies
    replayed from per-slot CUDA graphs; p50/p99 latency at the offered rate
    and the saturated throughput."""
    import torch
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    torch.cuda.set_device(0)
    name = "bf16x3" if args.dtype == "all" else args.dtype
    arrivals, specs = wk.served_trace(args.requests, args.rate, size_cap=args.size_cap)
    budget = int(args.budget_gb * (1 << 30))
    t0 = time.perf_counter()
    requests, plans, n_app = build_served(pk, torch, arrivals, specs, name, PRECISION_TOL[name])
    warm_served(pk, torch, requests)
    setup_s = time.perf_counter() - t0
    zeros = np.zeros(len(requests))

    def stats(lat, qd, mk, reqs):
        lat = np.array(lat)
        napp = sum(len(a) for a in reqs)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "queue_p50_ms": float(np.percentile(qd, 50)),
                "makespan_s": mk, "requests_per_s": len(reqs) / mk, "phi_actions_per_s": napp / mk}

    res = {}
    # the whole trace saturated first (every per-slot graph captured here),
    # then at the offered rate
    l0 = pk.phiks_kernel_launches()
    latb, qb, mkb = pk.phiks_serve_trace(requests, zeros, slots=args.slots, hbm_budget=budget)
    launches_sat = pk.phiks_kernel_launches() - l0
    res[name + "_saturated"] = stats(latb, qb, mkb, requests)
    clocks = ClockSampler(0)
    clocks.start()
    lat, qd, mk = pk.phiks_serve_trace(requests, arrivals, slots=args.slots, hbm_budget=budget)
    clk = clocks.stop()
    res[name] = stats(lat, qd, mk, requests)
    res[name].update({"offered_rate_per_s": args.rate, "slots": args.slots, "setup_s": setup_s})
    # the same trace offered at 80% of the saturated rate: latency when the
    # queue does not grow without bound
    sat_rate = len(requests) / mkb
    lat8, qd8, mk8 = pk.phiks_serve_trace(requests, arrivals * (args.rate / (0.8 * sat_rate)),
                                          slots=args.slots, hbm_budget=budget)
    res[name + "_80pct"] = stats(lat8, qd8, mk8, requests)
    res[name + "_80pct"]["offered_rate_per_s"] = 0.8 * sat_rate
    # slot scaling and submission on a prefix of the trace
    pre = requests[: args.prefix]
    zp = np.zeros(len(pre))
    _, _, mk1 = pk.phiks_serve_trace(pre, zp, slots=1)
    _, _, mkd = pk.phiks_serve_trace(pre, zp, slots=args.slots, hbm_budget=budget, graphs=0)
    _, _, mkp = pk.phiks_serve_trace(pre, zp, slots=args.slots, hbm_budget=budget)
    napp_pre = sum(len(a) for a in pre)
    res["prefix"] = {"requests": len(pre), "one_slot_graphs_phi_actions_per_s": napp_pre / mk1,
                     "slots_direct_launches_phi_actions_per_s": napp_pre / mkd,
                     "slots_graphs_phi_actions_per_s": napp_pre / mkp,
                     "slot_scaling": mk1 / mkp, "graphs_over_direct": mkd / mkp}
    # kernel roofline: events around every GEMM pass (profiling runs the
    # applies without graphs), over the prefix on one slot (brackets on
    # concurrent slots would overlap)
    for pl in plans.values():
        pk.phiks_profile_enable(pl.handle, True)
    pk.phiks_serve_trace(pre, zp, slots=1)
    kms = kl = kfl = 0.0
    for pl in plans.values():
        a, b, c = pk.phiks_profile_read(pl.handle)
        pk.phiks_profile_enable(pl.handle, False)
        kms, kl, kfl = kms + a, kl + b, kfl + c
    roof = profile_roofline(name, kms, int(kl), kfl)
    if roof:
        roof["note"] = ("GEMM passes timed on one slot over the prefix; mixed sizes (AC 128..1024^2, "
                        "ADR 32..192^3, Brusselator 128..512^2)")
    cpu = None
    if not args.no_oracle:
        res[name]["oracle_check"] = oracle_check_served(specs, requests)
        oc = res[name]["oracle_check"]
        cpu = {"value": len(oc["requests"]) / oc["seconds"], "unit": "phi-actions/s", "cores": oracle_threads(),
               "kind": "oracle", "sample": "the smallest request of each class, first apply (O3), %.1f s"
                                           % oc["seconds"]}
    if not args.no_ref:
        # the split dtype against the FP64 path on a prefix, one slot each
        pre64 = max(50, args.prefix // 4)
        req64, plans64, _ = build_served(pk, torch, arrivals[:pre64], specs[:pre64], "fp64", None)
        warm_served(pk, torch, req64)
        _, _, mk64 = pk.phiks_serve_trace(req64, np.zeros(len(req64)), slots=1)
        _, _, mk32 = pk.phiks_serve_trace(requests[:pre64], np.zeros(len(req64)), slots=1)
        res["fp64_one_slot_prefix"] = {"requests": pre64, "makespan_s": mk64,
                                       "phi_actions_per_s": sum(len(a) for a in req64) / mk64,
                                       "speedup_of_%s" % name: mk64 / mk32}
        errs = []
        for a32, a64 in zip(requests[:pre64], req64):
            for x, y in zip(a32, a64):
                o, r = x["out"].double().cpu().numpy(), y["out"].cpu().numpy()
                den = np.abs(r).max()
                errs.append(float(np.abs(o - r).max() / den) if den > 0 else float("nan"))
        errs = np.array(errs)
        res[name]["rel_err_vs_fp64_max"] = float(np.nanmax(errs)) if np.isfinite(errs).any() else None
        res[name]["outputs_compared_vs_fp64"] = int(np.isfinite(errs).sum())
        for pl in plans64.values():
            pl.close()
    for pl in plans.values():
        pl.close()
    h = res[name]
    line = {"metric": METRIC, "value": res[name + "_saturated"]["phi_actions_per_s"], "unit": "phi-actions/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * res[name + "_saturated"]["makespan_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": name, "data": "synthetic",
            "config": {"workload": "served_ac_adr_bru", "requests": len(requests), "applies": n_app,
                       "offered_rate_per_s": args.rate, "p": "2..4", "mode": "lincomb",
                       "sizes": {"ac": "128..%d" % min(1024, args.size_cap or 1024),
                                 "adr": "32..%d" % min(192, args.size_cap or 192),
                                 "bru": "128..%d" % min(512, args.size_cap or 512)},
                       "slots": args.slots, "hbm_budget_gb": args.budget_gb,
                       "submission": "per-slot CUDA graphs of each (plan, tau, p), inputs and outputs "
                                     "copied through slot staging buffers",
                       "value": "saturated: the whole trace offered at t = 0"},
            "rel_err_vs_oracle": h.get("oracle_check", {}).get("max_rel_err"),
            "latency_ms": {"offered_rate_per_s": args.rate, "p50": h["p50_ms"], "p99": h["p99_ms"],
                           "achieved_requests_per_s": h["requests_per_s"],
                           "saturated_p50": res[name + "_saturated"]["p50_ms"],
                           "saturated_p99": res[name + "_saturated"]["p99_ms"],
                           "offered_80pct_of_saturated_per_s": res[name + "_80pct"]["offered_rate_per_s"],
                           "p50_at_80pct": res[name + "_80pct"]["p50_ms"],
                           "p99_at_80pct": res[name + "_80pct"]["p99_ms"]},
            "aggregate_tflops": {"unit": "TFLOP/s (algorithmic Tucker flops, T# x 2 N sum(n) per apply)",
                                 "saturated": served_flops(requests) / mkb / 1e12,
                                 "offered_rate": served_flops(requests) / mk / 1e12,
                                 "at_80pct": served_flops(requests) / mk8 / 1e12},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": None, "e2e_note": "the served form keeps plans, inputs and outputs resident on the device",
            "gpu_launches": launches_sat, "clocks": clk,
            "per_variant": res}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_small(args):
    """The latency case: d = 2, n = 32 (N = 1024), FD Laplacian + 0.5 d_x,
    phi_0..phi_3 of one vector, FP64.  One call is captured in a CUDA graph
    and replayed; reports calls/s and phi-actions/s (4 per call)."""
    import torch
    import paper_2210_07667_gb300 as pk
    pk.load(build_if_missing=True)
    torch.cuda.set_device(0)
    wl = wk.small_same(32)
    plan = pk.Plan(wl.A, pk.PHIKS_FP64)
    v = torch.from_numpy(wl.vs[0]).cuda()
    out = torch.empty(4 * wl.N, device="cuda", dtype=torch.float64)
    opts = pk.make_options(vnorms=[float(np.linalg.norm(wl.vs[0]))])
    stream = torch.cuda.Stream()
    inst = [(plan.handle, wl.tau, 3, [v], out, opts)]
    batch = pk.Batch(1)
    with torch.cuda.stream(stream):
        for _ in range(3):
            batch.apply(inst, stream)
    torch.cuda.synchronize()
    graph = batch.capture(inst, stream)
    reps = args.reps
    for _ in range(max(args.warmup, 3)):
        batch.launch(graph, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            batch.launch(graph, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # direct calls (host issue included), for comparison; their launch count
    l0 = pk.phiks_kernel_launches()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(200):
            pk.phiks_apply_ex(plan.handle, wl.tau, 3, [v], out, stream, opts=opts)
    torch.cuda.synchronize()
    ms_direct = (time.perf_counter() - t0) * 1e3 / 200
    per_call_launches = (pk.phiks_kernel_launches() - l0) / 200
    got = out.cpu().numpy().reshape(4, wl.N)
    from oracle import dense
    t0 = time.perf_counter()
    ref = dense.same(wl.A, wl.tau, wl.vs[0], 3)
    oracle_s = time.perf_counter() - t0
    err = max(float(np.abs(got[l] - ref[l]).max() / np.abs(ref[l]).max()) for l in range(4))
    s_, q_, T_, tk = plan.last_params()
    # kernel roofline: events around every fused Tucker launch, the host
    # queueing each call behind a device spin so that brackets time kernels
    pk.phiks_profile_enable(plan.handle, True)
    with torch.cuda.stream(stream):
        for _ in range(50):
            torch.cuda._sleep(int(2e6))
            pk.phiks_apply_ex(plan.handle, wl.tau, 3, [v], out, stream, opts=opts)
    kms, kl, kfl = pk.phiks_profile_read(plan.handle)
    pk.phiks_profile_enable(plan.handle, False)
    roof = profile_roofline("fp64", kms, kl, kfl, kernel="tucker_fused_f64_kernel")
    if roof:
        roof["note"] = ("latency bound: 1024-element tensors, a few microseconds per launch; "
                        "calls/s is this configuration's figure of merit")
    # end to end through the C ABI: the input from pinned host memory, the
    # four outputs back, every call (graph replay of the call's kernels)
    hv = torch.from_numpy(wl.vs[0]).pin_memory()
    hout = torch.empty(4 * wl.N, dtype=torch.float64).pin_memory()
    dv = torch.empty(wl.N, device="cuda", dtype=torch.float64)
    og = pk.make_options(vnorms=[float(np.linalg.norm(wl.vs[0]))], graph=1)
    with torch.cuda.stream(stream):
        for _ in range(3):
            pk.phiks_apply_ex(plan.handle, wl.tau, 3, [dv], out, stream, opts=og)
    torch.cuda.synchronize()
    ne = 500
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(ne):
            dv.copy_(hv, non_blocking=True)
            pk.phiks_apply_ex(plan.handle, wl.tau, 3, [dv], out, stream, opts=og)
            hout.copy_(out, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ne
    line = {"metric": METRIC, "value": 4 / (ms * 1e-3), "unit": "phi-actions/s", "n_gpus": 1,
            "steps": reps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "d": 2, "n": [32, 32], "N": 1024, "p": 3, "mode": "same",
                       "tau": wl.tau, "s": s_, "q": q_, "tuckers": tk, "replay": "CUDA graph",
                       "l2": "inputs and outputs (40 KiB) stay in L2 between calls"},
            "calls_per_s": 1e3 / ms, "direct_call_ms": ms_direct, "rel_err_vs_oracle": err,
            "roofline": roof,
            "cpu_baseline": {"value": 4 / oracle_s, "unit": "phi-actions/s", "cores": oracle_threads(),
                             "kind": "oracle", "sample": "one full call (phi_0..phi_3), O1 dense "
                                                         "augmented-matrix exponentials, %.2f s" % oracle_s},
            "e2e": {"value": 4 / (e2e_ms * 1e-3), "unit": "phi-actions/s", "h2d_bytes_per_step": wl.N * 8,
                    "d2h_bytes_per_step": 4 * wl.N * 8},
            "gpu_launches": int(round(per_call_launches * reps)),
            "launches_per_call": per_call_launches}
    print(json.dumps(line), flush=True)
    batch.destroy_graph(graph)
    batch.close()
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="phiks", choices=["phiks", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="adr3d", choices=["adr3d", "small", "precision", "batched", "served"],
                    help="adr3d: the headline FP64 workload; precision: the split-dtype form")
    ap.add_argument("--dtype", default="all", choices=["all"] + PRECISION_DTYPES,
                    help="precision/batched/served: split dtype; adr3d: FP64-accurate products, "
                         "emulated on the tensor cores (default, or fp64emu) or fp64 (DFMA)")
    ap.add_argument("--variant", default="cheb", choices=["cheb", "fd"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--no-ref", action="store_true", help="skip the FP64 reference path")
    ap.add_argument("--no-oracle", action="store_true",
                    help="precision/batched/served: skip the oracle check of sampled outputs")
    ap.add_argument("--count", type=int, default=256, help="batched form: instances")
    ap.add_argument("--streams", type=int, default=16, help="batched form: worker streams")
    ap.add_argument("--requests", type=int, default=20000, help="served form: trace length")
    ap.add_argument("--prefix", type=int, default=2000, help="served form: requests of the slot-scaling runs")
    ap.add_argument("--reps", type=int, default=10000, help="small: graph replays")
    ap.add_argument("--rate", type=float, default=2000.0, help="served form: arrivals per second")
    ap.add_argument("--slots", type=int, default=16, help="served form: concurrent requests")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="served form: workspace budget")
    ap.add_argument("--size-cap", type=int, default=None, help="served form: largest n")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "precision":
        return run_precision(args)
    if args.config == "batched":
        return run_batched(args)
    if args.config == "served":
        return run_served(args)
    if args.config == "small":
        return run_small(args)
    return run_phiks(args)


if __name__ == "__main__":
    sys.exit(main())
