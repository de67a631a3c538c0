#!/usr/bin/env python
"""Benchmark of the GB300 robust triangular Sylvester solver.

One step = one full robust FP64 solve A Y + Y B = alpha C (Algorithm 4: structure
scan and tile partition, Bound, the persistent tile-DAG kernel with robust
updates and diagonal solves, consistency scaling) on the workload "benign_8000":
m = n = 8000, tile 32, quasi-triangular A and B with ~50% of eigenvalues in
standardized 2x2 blocks, eigenvalue real parts U[1,10], strictly-upper entries and
C ~ U[-1,1] (the FP64 arm of the m = n = 8000 mixed-precision configuration).

Metric: GFLOP/s counting 2mn(m+n) flops per solve (the configuration's count);
the algorithmic count mn(m+n) (one multiply-add per update term) is reported
beside it and used for the roofline.  Inputs (3 x 512 MB) exceed the 129 MB L2
and every step solves a fresh copy of C, so no step starts from a warm L2.
Secondary lines: robust against non-robust at m = n = 4000 on an input whose
unscaled substitution overflows; m = n = 256 (latency, microseconds per solve);
FP32 + refinement at 8000; the 4096-equation batch (FP64 and FP32 + refinement);
256 Lyapunov forward + backward solves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank solves its own copy of the workload (the solve
does not shard: replicas); value = all ranks' flops / the slowest rank's time.
--impl reference times the FP64 CPU oracle (Algorithm 2 in plain C) on the host
cores: one independent oracle solve per core at a bounded size.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "benign_8000"
FP64_PEAK_GFLOPS = 152 * 4 * 2.070  # 152 SMs x 2 DFMA/clk (4 flop) x 2.07 GHz max SM clock
ORACLE_SAMPLE_M = 900  # bounded CPU sample: same generator family at m = n = 900, one solve per host core


def flops_2(m, n):
    return 2.0 * m * n * (m + n)


def flops_alg(m, n):
    return 1.0 * m * n * (m + n)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, help="named synthetic workload (each mode has its default)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--tile", type=int, default=0, help="override the workload's tile size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=1024, help="batch mode: equations in the batch")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_refine"], help="batch mode: precision")
    ap.add_argument("--sms", default="", help="smscale mode: comma-separated SM counts")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (mixed precision, batched, adjoint)")
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "mixed", "batched", "adjoint", "smscale", "variants", "robustness", "residual",
                             "robust_vs_plain", "small", "peaks", "batch"],
                    help="solve: the headline robust FP64 solve; mixed: FP32 + refinement vs FP64 at "
                         "m=n=8000; batched: 4096 uneven equations; adjoint: 256 Lyapunov forward+backward; "
                         "smscale: SM scaling; variants: sign variant, triangular solve, Bartels-Stewart at 4000; "
                         "robustness: robust vs plain on the paper's matrices, m=n=10000; residual: the "
                         "refinement's tensor-core residual at m=n=4000; robust_vs_plain: robust against non-robust "
                         "FP64 at m=n=4000 (overflow workload); small: m=n=256 microseconds per solve; peaks: "
                         "measured binary64/binary32 FMA pipe rates; batch: --count equations of the batched "
                         "distribution at --precision, no graph")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out)

    @staticmethod
    def parse(out):
        """Median SM clock, maximum SM clock and the throttle reasons seen active in
        `nvidia-smi --format=csv,noheader,nounits` lines of FIELDS (others skipped)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            for nm, v in zip(names, parts[5:9]):  # counted even when a clock reads N/A
                if v.lower() == "active":
                    reasons.add(nm)
            try:
                clk, clk_max = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            sm.append(clk)
            smax.append(clk_max)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for_dag():
    """DRAM bytes per launch of the tile-DAG kernel from the committed ncu summary, if
    the kernel source has not changed since it was captured (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dag_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in ("sylv_dag.cuh", "sylv_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1905_10574_gb300", "csrc", f), "rb").read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec.get("dram_bytes_per_launch_full_size")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(m, seed, kind, upper, steps, warmup, barrier, out):
    """One host core: `warmup` + `steps` oracle solves of the same m x m sample, each
    timed between barriers shared with the other cores' workers."""
    from oracle import oracle
    from paper_1905_10574_gb300 import inputs
    A, B, C = inputs.problem(m, m, seed, kind=kind, upper=upper)
    oracle.trsyl(A[:64, :64], B[:64, :64], C[:64, :64])  # load + warm the library
    ts = []
    for i in range(warmup + steps):
        barrier.wait()
        t0 = time.perf_counter()
        oracle.trsyl(A, B, C)
        if i >= warmup:
            ts.append(time.perf_counter() - t0)
    out.put(ts)


def oracle_on_host_cores(w, steps, warmup, cores=None):
    """The FP64 oracle (single-threaded C, as it stands) on every host core at once:
    each core solves its own copy of an m = n = ORACLE_SAMPLE_M sample of the workload's
    generator per step; a step lasts until the slowest core finishes.  Processes are
    spawned (never forked after CUDA initialisation).  Returns (GFLOP/s over all
    cores counted 2mn(m+n), cores, seconds per step)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = cores or host_cores()
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(ORACLE_SAMPLE_M, w["seed"], w["kind"], w["upper"], steps,
                                                      warmup, barrier, out)) for _ in range(cores)]
    for p in procs:
        p.start()
    per_core = [out.get() for _ in procs]
    for p in procs:
        p.join()
    step_s = [max(ts[i] for ts in per_core) for i in range(steps)]
    tot = sum(step_s)
    m = ORACLE_SAMPLE_M
    return cores * steps * flops_2(m, m) / tot / 1e9, cores, tot / steps


def cpu_baseline(w):
    """The FP64 oracle on all host cores (one independent sample solve per core)."""
    val, cores, sec = oracle_on_host_cores(w, steps=2, warmup=0)
    m = ORACLE_SAMPLE_M
    return {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"each of {cores} host cores solves its own m=n={m} robust FP64 oracle problem (Algorithm 2, "
                      f"single-threaded C) of the same generator (kind={w['kind']}, upper={w['upper']}); "
                      f"2 steps of {sec:.2f} s (slowest core); counted 2mn(m+n) per core"}


def _lapack_dtrsyl3():
    """LAPACKE_dtrsyl3 of the OpenBLAS that scipy bundles, found by its exported name
    (None if this scipy build has none)."""
    import ctypes
    import glob
    import scipy
    libdir = os.path.join(os.path.dirname(os.path.dirname(scipy.__file__)), "scipy.libs")
    for path in sorted(glob.glob(os.path.join(libdir, "*openblas*.so*"))):
        try:
            L = ctypes.CDLL(path)
        except OSError:
            continue
        for prefix in ("scipy_", ""):
            fn = getattr(L, prefix + "LAPACKE_dtrsyl3", None)
            if fn is not None:
                setn = getattr(L, prefix + "openblas_set_num_threads", None)
                return fn, setn, os.path.basename(path)
    return None


def cpu_context_dtrsyl3(w):
    """Time-to-solution context on the host: LAPACK's blocked triangular Sylvester
    solver dtrsyl3 (OpenBLAS, multithreaded on all host cores), one solve of the full
    workload in a spawned process.  Context only: a different algorithm and code."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_dtrsyl3_worker, args=(w, q))
    p.start()
    try:
        r = q.get(timeout=300)
    except Exception as exc:  # noqa: BLE001  report, do not hide
        r = {"unavailable": f"dtrsyl3 leg did not finish: {type(exc).__name__}"}
        p.terminate()
    p.join()
    return r


def _dtrsyl3_worker(w, q):
    import ctypes
    import numpy as np
    from paper_1905_10574_gb300 import inputs
    found = _lapack_dtrsyl3()
    if found is None:
        q.put({"unavailable": "scipy's OpenBLAS exports no LAPACKE_dtrsyl3 on this host"})
        return
    fn, setn, libname = found
    cores = host_cores()
    if setn is not None:
        setn(cores)
    m, n = w["m"], w["n"]
    A, B, C = inputs.problem(m, n, w["seed"], kind=w["kind"], upper=w["upper"])
    A, B, C = (np.asfortranarray(x) for x in (A, B, C))
    i32, pd = ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    fn.restype = i32
    fn.argtypes = [ctypes.c_int, ctypes.c_char, ctypes.c_char, i32, i32, i32, pd, i32, pd, i32, pd, i32, pd]
    scale = ctypes.c_double(0.0)
    args = lambda X: X.ctypes.data_as(pd)  # noqa: E731
    t0 = time.perf_counter()
    info = fn(102, b"N", b"N", 1, m, n, args(A), m, args(B), n, args(C), m, ctypes.byref(scale))
    dt = time.perf_counter() - t0
    q.put({"value": flops_2(m, n) / dt / 1e9, "unit": "GFLOP/s", "cores": cores,
           "kind": "LAPACK dtrsyl3 (" + libname + ")", "seconds": dt, "info": int(info), "scale": scale.value,
           "sample": f"one solve of the full workload m=n={m}, {cores} OpenBLAS threads; counted 2mn(m+n)"})


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1905_10574_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    m = ORACLE_SAMPLE_M
    val, cores, sec = oracle_on_host_cores(w, steps=max(1, args.steps), warmup=args.warmup)
    line = {"impl": "reference", "metric": "robust Sylvester solve GFLOP/s", "value": val, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "m": w["m"], "n": w["n"], "tile": w["tile"],
                       "flop_count": "2mn(m+n)", "reference_sample_m": m},
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: each of {cores} host cores solves its own m=n={m} robust FP64 "
                                       f"oracle problem (Algorithm 2, single-threaded C) of the same generator; the "
                                       f"GPU arm solves m=n={w['m']}"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1905_10574_gb300 import build, inputs, replicas, sylv

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    build.build()
    sylv.load()
    w = inputs.WORKLOADS[args.workload]
    m, n, tile = w["m"], w["n"], (args.tile or w["tile"])
    A, B, C = inputs.problem(m, n, w["seed"] + 0, kind=w["kind"], upper=w["upper"])
    Ad = torch.from_numpy(A).to(device)
    Bd = torch.from_numpy(B).to(device)
    C0 = torch.from_numpy(C).to(device)
    nsteps = args.warmup + args.steps
    Cs = [C0.clone() for _ in range(nsteps)]  # a fresh right-hand side per step
    stream = torch.cuda.current_stream(device)
    opts = sylv.make_opts(tile=tile, stream=stream.cuda_stream, sync=False)
    wsb = sylv.sylv_workspace_size(m, n, opts)
    wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=device)
    opts.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
    opts.workspace_bytes = wsb
    res_dev = torch.zeros(nsteps * 64, dtype=torch.uint8, device=device)
    lda, ldb, ldc = Ad.stride(1), Bd.stride(1), C0.stride(1)

    def step(i):
        rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), lda, Bd.data_ptr(), ldb, Cs[i].data_ptr(), ldc, opts,
                                    res_dev.data_ptr() + 64 * i)
        if rc != 0:
            raise sylv.SylvError(rc, "sylv_tri_solve_ex")

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    sylv.sylv_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.warmup, nsteps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    dag_ms, dag_launches = sylv.sylv_profile_read()
    sylv.sylv_profile(False)
    clocks = sampler.stop()
    if ws > 1:
        dist.barrier()
    ms_max = replicas.max_over_ranks(e0.elapsed_time(e1))
    # per-step results (the last timed solve)
    res = sylv.sylv_result.from_buffer_copy(res_dev[64 * (nsteps - 1): 64 * (nsteps - 1) + 40].cpu().numpy().tobytes())
    ok = res.info in (sylv.SYLV_OK, sylv.SYLV_NEAR_SINGULAR)

    # ---- end to end through the C ABI with host buffers: H2D of A, B, C from pinned
    # memory, the solve, D2H of Y into pinned memory, every step.
    Ah, Bh, Ch = (torch.from_numpy(x).pin_memory() for x in (A, B, C))
    Yh = torch.empty_like(Ch).pin_memory()
    Ae, Be, Ce = torch.empty_like(Ad), torch.empty_like(Bd), torch.empty_like(C0)
    Ae = Ae.t().contiguous().t() if Ae.stride(0) != 1 else Ae
    Ce = Ce.t().contiguous().t() if Ce.stride(0) != 1 else Ce
    Be = Be.t().contiguous().t() if Be.stride(0) != 1 else Be
    esteps = max(1, args.e2e_steps)
    h2d = 8 * (m * m + n * n + m * n)
    d2h = 8 * m * n

    def e2e_step():
        Ae.copy_(Ah, non_blocking=True)
        Be.copy_(Bh, non_blocking=True)
        Ce.copy_(Ch, non_blocking=True)
        rc = sylv.sylv_tri_solve_ex(m, n, Ae.data_ptr(), Ae.stride(1), Be.data_ptr(), Be.stride(1), Ce.data_ptr(),
                                    Ce.stride(1), opts, res_dev.data_ptr())
        if rc != 0:
            raise sylv.SylvError(rc, "sylv_tri_solve_ex")
        Yh.copy_(Ce, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(esteps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks(f0.elapsed_time(f1) / esteps)

    if rank == 0:
        per_step = ms_max / args.steps
        value = replicas.whole_job_rate(flops_2(m, n), ws, per_step / 1000) / 1e9
        dag_per_launch_ms = dag_ms / max(dag_launches, 1)
        achieved = flops_alg(m, n) / (dag_per_launch_ms / 1000) / 1e9
        traffic = traffic_for_dag()
        line = {
            "metric": "robust Sylvester solve GFLOP/s", "value": value, "unit": "GFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "tile": tile, "generator": w["kind"],
                       "upper_scale": w["upper"], "flop_count": "2mn(m+n)",
                       "algorithmic_gflops": ws * flops_alg(m, n) / (per_step / 1000) / 1e9,
                       "l2": f"inputs {3 * 8 * m * n // 2**20} MB > 129 MB L2; fresh C copy per step",
                       "parallelism": f"replicas{ws}"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                         "kernel": f"dag_kernel<{32 if tile <= 32 else 64},double,robust>",
                         "flops_per_launch": flops_alg(m, n),
                         "peak_note": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived from unit counts and "
                                      "the maximum SM clock; MEASURED_PEAKS.json has no FP64 entry)"},
            "e2e": {"value": replicas.whole_job_rate(flops_2(m, n), ws, e2e_ms / 1000) / 1e9, "unit": "GFLOP/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 10 * args.steps,  # per solve: set_inst, scan, norms, 3 level kernels, pack, DAG, consistency, results
            "clocks": clocks,
            "result": {"info": res.info, "log2scale": res.log2scale, "scale_events": res.scale_events,
                       "ok": ok},
            "dag_ms_per_launch": dag_per_launch_ms,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
            line["cpu_context"] = cpu_context_dtrsyl3(w)
        if not args.no_extras and ws == 1:
            line["secondary"] = secondary(args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _timed(fn, steps, warmup, stream):
    """Per-step CUDA-event time (ms) of fn(i), warm-up excluded; returns (mean, list)."""
    import torch
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize()
    ts = []
    for i in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(warmup + i)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sum(ts) / len(ts), ts


# Stop tolerance of the mixed-precision line: the refinement stops once the
# predicted size of the next correction is below tol * max|X|, so tol = 2^-41
# (4.5e-13) meets a forward-error target of 1e-12 with a factor 2.2 to spare.  The
# library default (2^-43) is measured beside it.
MIXED_TOL = 2.0 ** -41


def run_mixed(args):
    """FP32 correction solves + FP64-accurate residual vs the plain robust FP64 solve,
    m = n = 8000, well-conditioned generator (the accuracy claim needs it).  The value
    is the refined solve at the 1e-12 forward-error target (MIXED_TOL); the error of
    each refined result against the FP64 solve of the same run is stated beside it."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    name = args.workload or "wellcond_8000"
    A, B, C, w = inputs.workload(name)
    m, n = w["m"], w["n"]
    dev = torch.device("cuda", 0)
    Ad, Bd, C0 = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    stream = torch.cuda.current_stream(dev)
    out, Yout = {}, {}
    for key, prec, tol in (("fp64", "fp64", 0.0), ("fp32_refine", "fp32_refine", MIXED_TOL),
                           ("fp32_refine_default_tol", "fp32_refine", 0.0)):
        opts = sylv.make_opts(tile=args.tile or w["tile"], precision=prec, tol=tol, stream=stream.cuda_stream,
                              sync=True)
        wsb = sylv.sylv_workspace_size(m, n, opts)
        wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
        opts.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
        opts.workspace_bytes = wsb
        Cs = [C0.clone() for _ in range(args.warmup + args.steps)]
        res = sylv.sylv_result()

        def fn(i):
            rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1),
                                        Cs[i].data_ptr(), Cs[i].stride(1), opts, res)
            if rc not in (0, 1):
                raise sylv.SylvError(rc, prec)

        ms, _ = _timed(fn, args.steps, args.warmup, stream)
        out[key] = {"ms_per_solve": ms, "solves_per_s": 1000.0 / ms, "info": res.info, "iters": res.iters,
                    "last_update": res.last_update, "tol": tol or 2.0 ** -43}
        Yout[key] = Cs[-1]  # the solves ran in place: the last buffer holds this precision's Y
        del wsbuf
    y64 = Yout["fp64"]
    scale = float(torch.max(torch.abs(y64)))
    for key in ("fp32_refine", "fp32_refine_default_tol"):
        out[key]["max_abs_err_vs_fp64_rel"] = float(torch.max(torch.abs(Yout[key] - y64))) / scale
    line = {"metric": "mixed-precision solves/s", "value": out["fp32_refine"]["solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": name, "m": m, "n": n, "tol": MIXED_TOL,
                                            "accuracy_target": 1e-12},
            "fp64": out["fp64"], "fp32_refine": out["fp32_refine"],
            "fp32_refine_default_tol": out["fp32_refine_default_tol"],
            "speedup_vs_fp64": out["fp64"]["ms_per_solve"] / out["fp32_refine"]["ms_per_solve"]}
    return line


def run_residual(args):
    """The refinement's binary64-accurate residual R = C - (A X + X B) on the tensor
    cores: one sylv_residual call (the four operand splittings and the GEMM launch),
    m = n = 4000 wellcond by default, X uniform in [-1, 1]."""
    import numpy as np
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    sylv.load()
    name = args.workload or "wellcond_4000"
    A, B, C, w = inputs.workload(name)
    m, n = w["m"], w["n"]
    dev = torch.device("cuda", 0)
    Ad, Bd, Cd = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    X = torch.from_numpy(np.asfortranarray(np.random.default_rng(9).uniform(-1.0, 1.0, (m, n)))).to(dev)
    stream = torch.cuda.current_stream(dev)
    ms, _ = _timed(lambda i: sylv.residual(Ad, Bd, X, Cd), args.steps, args.warmup, stream)
    return {"metric": "residual calls/s", "value": 1000.0 / ms, "unit": "calls/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "bf16 slices, f32 accumulation, f64 result",
            "data": "synthetic", "config": {"workload": name, "m": m, "n": n}, "ms_per_call": ms,
            "binary64_equivalent_tflops": m * n * (m + n) / ms / 1e9}


def run_smscale(args):
    """SM scaling of the robust FP64 solve (the GPU analogue of the paper's core-scaling
    study, Sec. 4): the persistent tile kernel restricted to the SMs with id < N (2 CTAs
    each), the rest of the solve unchanged.  Efficiency = N0 T(N0 SMs) / (N T(N SMs)),
    N0 the smallest count measured (1 by default; --sms picks the counts).  The
    uncapped solve is timed last, as a check that the cap at N = #SMs loses no SM."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    name = args.workload or "benign_1000"
    A, B, C, w = inputs.workload(name)
    m, n = w["m"], w["n"]
    dev = torch.device("cuda", 0)
    Ad, Bd, C0 = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    stream = torch.cuda.current_stream(dev)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    rows = []
    sm_list = [int(x) for x in args.sms.split(",")] if args.sms else [1, 2, 4, 8, 19, 38, 76, nsm]
    uncapped = None
    for sms in sm_list + [0]:
        opts = sylv.make_opts(tile=args.tile or w["tile"], stream=stream.cuda_stream, sync=True, max_sms=sms)
        wsb = sylv.sylv_workspace_size(m, n, opts)
        wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
        opts.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
        opts.workspace_bytes = wsb
        steps = 2 if 0 < sms < 8 else args.steps
        Cs = [C0.clone() for _ in range(1 + steps)]
        res = sylv.sylv_result()

        def fn(i):
            rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1),
                                        Cs[i].data_ptr(), Cs[i].stride(1), opts, res)
            if rc not in (0, 1):
                raise sylv.SylvError(rc, "smscale")

        ms, _ = _timed(fn, steps, 1, stream)
        del Cs, wsbuf
        if sms == 0:
            uncapped = ms
            break
        rows.append({"sms": sms, "ms_per_solve": ms, "gflops_2mnmn": flops_2(m, n) / ms / 1e6,
                     "log2scale": int(res.log2scale)})
    t1, s1 = rows[0]["ms_per_solve"], rows[0]["sms"]
    for r in rows:
        r["speedup"] = t1 / r["ms_per_solve"]
        r["efficiency"] = r["speedup"] * s1 / r["sms"]
    return {"metric": "SM-scaling efficiency of the robust FP64 solve", "value": rows[-1]["efficiency"],
            "unit": "fraction", "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "m": m, "n": n, "tile": args.tile or w["tile"], "base_sms": s1,
                       "uncapped_ms_per_solve": uncapped, "sms_on_device": nsm},
            "rows": rows}


def run_batched(args):
    """4096 independent equations, m, n log-uniform in [16, 512]: autotuned tile per
    size bucket, one batched persistent launch captured in a CUDA graph and replayed;
    against the plain path solving the same equations one call at a time (sampled).
    On N GPUs (torchrun) the equations are split by flops, longest first (no exchange
    but the slowest rank's time); the value is all 4096 over that time."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1905_10574_gb300 import autotune, build, inputs, replicas, sylv
    build.build()
    ws, rank, local = dist_env()
    own_pg = ws > 1 and not dist.is_initialized()
    if own_pg:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    total = 4096
    all_shapes = inputs.batch_shapes(total, 16, 512, seed=1234)
    mine = replicas.lpt_shards([m * n * (m + n) for m, n in all_shapes], ws)[rank] if ws > 1 else range(total)
    shapes = [all_shapes[i] for i in mine]
    count = len(shapes)
    dev = torch.device("cuda", local)
    As, Bs, C0s = [], [], []
    for i, (m, n) in zip(mine, shapes):
        A, B, C = inputs.problem(m, n, 10000 + i, kind="wellcond")
        As.append(torch.from_numpy(A).to(dev))
        Bs.append(torch.from_numpy(B).to(dev))
        C0s.append(torch.from_numpy(C).to(dev))
    Cs = [c.clone() for c in C0s]
    tiles = [args.tile] * count if args.tile else autotune.tune_batch(As, Bs, Cs)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        opts = sylv.make_opts(stream=stream.cuda_stream)
        plan = sylv.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                      [a.stride(1) for a in As], [b.data_ptr() for b in Bs],
                                      [b.stride(1) for b in Bs], [c.data_ptr() for c in Cs],
                                      [c.stride(1) for c in Cs], opts, tiles=tiles)
        rc = sylv.sylv_batch_execute(plan, stream.cuda_stream)  # warm-up before capture
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            rc |= sylv.sylv_batch_execute(plan, torch.cuda.current_stream().cuda_stream)
    if rc:
        raise sylv.SylvError(rc, "batch")
    flops = sum(2.0 * m * n * (m + n) for m, n in shapes)
    ts = []
    rs = torch.cuda.current_stream(dev)  # graph.replay() runs on the current stream
    for i in range(args.warmup + args.steps):
        for c, c0 in zip(Cs, C0s):
            c.copy_(c0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(rs)
        graph.replay()
        b.record(rs)
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(a.elapsed_time(b))
    rc, res = sylv.sylv_batch_results(plan, count)
    sylv.sylv_batch_destroy(plan)
    ms = replicas.max_over_ranks(sum(ts) / len(ts))  # the slowest rank's time
    if ws > 1:
        worst = int(replicas.max_over_ranks(max(r.info for r in res)))
        if own_pg:
            dist.destroy_process_group()
        if rank != 0:
            return None
        return {"metric": "batched solves/s", "value": total / (ms / 1000), "unit": "solves/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "dtype": "f64", "data": "synthetic",
                "config": {"count": total, "m_n": "log-uniform [16,512]", "generator": "wellcond",
                           "split": "longest processing time first, by 2mn(m+n)", "cuda_graph": True},
                "worst_info": worst}
    # plain path, one call per equation, on a sample of 256 equations (scaled to 4096)
    sample = list(range(0, count, count // 256))
    cur = torch.cuda.current_stream(dev)
    o1 = sylv.make_opts(stream=cur.cuda_stream, sync=False)
    wsb = max(sylv.sylv_workspace_size(shapes[i][0], shapes[i][1], o1) for i in sample)
    wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
    o1.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
    o1.workspace_bytes = wsb
    rdev = torch.zeros(64, dtype=torch.uint8, device=dev)
    Cp = [C0s[i].clone() for i in sample]
    for j, i in enumerate(sample[:8]):
        sylv.sylv_tri_solve_ex(shapes[i][0], shapes[i][1], As[i].data_ptr(), As[i].stride(1), Bs[i].data_ptr(),
                               Bs[i].stride(1), Cp[j].data_ptr(), Cp[j].stride(1), o1, rdev.data_ptr())
    Cp = [C0s[i].clone() for i in sample]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for j, i in enumerate(sample):
        sylv.sylv_tri_solve_ex(shapes[i][0], shapes[i][1], As[i].data_ptr(), As[i].stride(1), Bs[i].data_ptr(),
                               Bs[i].stride(1), Cp[j].data_ptr(), Cp[j].stride(1), o1, rdev.data_ptr())
    e1.record(cur)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) * count / len(sample)
    # FP32 + refinement on the same equations at the 1e-12 forward-error target
    # (MIXED_TOL), with tiles tuned for it (its latency-bound binary32 tiles favour
    # other sizes than FP64), graph-captured the same way; its solutions are compared
    # with the FP64 batch's (Cs holds them after the last replay).
    Cr = [c.clone() for c in C0s]
    rtiles = [args.tile] * count if args.tile else autotune.tune_batch(As, Bs, Cr, precision="fp32_refine",
                                                                       tol=MIXED_TOL)
    rstream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(rstream):
        ropts = sylv.make_opts(stream=rstream.cuda_stream, precision="fp32_refine", tol=MIXED_TOL)
        rplan = sylv.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                       [a.stride(1) for a in As], [b.data_ptr() for b in Bs],
                                       [b.stride(1) for b in Bs], [c.data_ptr() for c in Cr],
                                       [c.stride(1) for c in Cr], ropts, tiles=rtiles)
        rrc = sylv.sylv_batch_execute(rplan, rstream.cuda_stream)
        rstream.synchronize()
        rgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(rgraph, stream=rstream):
            rrc |= sylv.sylv_batch_execute(rplan, torch.cuda.current_stream().cuda_stream)
    if rrc:
        raise sylv.SylvError(rrc, "refined batch")
    rts = []
    for i in range(args.warmup + args.steps):
        for c, c0 in zip(Cr, C0s):
            c.copy_(c0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(rs)
        rgraph.replay()
        b.record(rs)
        torch.cuda.synchronize()
        if i >= args.warmup:
            rts.append(a.elapsed_time(b))
    rrc, rres = sylv.sylv_batch_results(rplan, count)
    sylv.sylv_batch_destroy(rplan)
    rms = sum(rts) / len(rts)
    errs = [float(torch.linalg.norm(y - c) / torch.linalg.norm(c)) for y, c in zip(Cr, Cs)]
    refined = {"solves_per_s": count / (rms / 1000), "ms_per_step": rms, "tol": MIXED_TOL, "accuracy_target": 1e-12,
               "worst_info": max(r.info for r in rres), "iters_max": max(r.iters for r in rres),
               "iters_mean": sum(r.iters for r in rres) / count,
               "tile_mix": {str(t): rtiles.count(t) for t in sorted(set(rtiles))},
               "max_rel_err_vs_fp64_batch": max(errs), "speedup_vs_fp64_batch": ms / rms}
    del Cr
    line = {"metric": "batched solves/s", "value": count / (ms / 1000), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"count": count, "m_n": "log-uniform [16,512]", "generator": "wellcond",
                       "tiles": "autotuned per size bucket" if not args.tile else args.tile,
                       "tile_mix": {str(t): tiles.count(t) for t in sorted(set(tiles))}, "cuda_graph": True},
            "gflops_2mnmn": flops / (ms / 1000) / 1e9, "worst_info": max(r.info for r in res),
            "one_call_per_equation_ms": seq_ms, "speedup_vs_one_call_per_equation": seq_ms / ms,
            "fp32_refine": refined}
    return line


def run_adjoint(args):
    """256 Lyapunov-type equations A Y + Y A^T = C, m = n = 512: batched forward +
    hand-written batched adjoint (loss sum(W * Y)), through torch.autograd."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    dev = torch.device("cuda", 0)
    count, m = 256, 512
    A = torch.stack([torch.from_numpy(inputs.quasi_triangular(m, 20000 + i, kind="wellcond")) for i in range(count)])
    C = torch.stack([torch.from_numpy(inputs.rhs(m, m, 30000 + i)) for i in range(count)])
    W = torch.stack([torch.from_numpy(inputs.rhs(m, m, 40000 + i)) for i in range(count)])
    A, C, W = (sylv.batch_fortran(x.to(dev)) for x in (A, C, W))
    stream = torch.cuda.current_stream(dev)

    def fn(_):
        At = A.detach().requires_grad_(True)
        Ct = C.detach().requires_grad_(True)
        Y = sylv.BatchSylvesterSolve.apply(At, At, Ct, False, True, 0)
        (W * Y).sum().backward()

    ms, _ = _timed(fn, max(1, args.steps), max(1, args.warmup), stream)
    line = {"metric": "differentiable Lyapunov solves/s (forward+backward)", "value": count / (ms / 1000),
            "unit": "solves/s", "n_gpus": 1, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"count": count, "m": m, "n": m, "form": "A Y + Y A^T = C, batched"}}
    return line


def run_variants(args):
    """The variants beside the paper's equation, each at m = n = 4000 on its own entry
    point: the sign variant A Y - Y B = C (isgn = -1), the robust solve against the
    non-robust one (Algorithm 1) on the same input, the robust triangular solve
    A X = alpha C (n = 4000 right-hand sides, growth generator, so it scales), and the
    Bartels-Stewart wrapper (U^T C V, the solve, U Y V^T) on random orthogonal U, V."""
    import numpy as np
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    m = n = 4000
    F = lambda x: torch.from_numpy(np.asfortranarray(x)).to(dev)  # noqa: E731
    A, B, C = inputs.problem(m, n, 0, kind="benign")
    Ad, Bd, C0 = F(A), F(-B), F(C)
    rows = {}
    steps, warm = max(1, args.steps), max(1, args.warmup)
    res = sylv.sylv_result()
    Cs = [C0.clone() for _ in range(steps + warm)]

    def sign(i):
        o = sylv.make_opts(isgn=-1, stream=stream.cuda_stream)
        rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), m, Bd.data_ptr(), n, Cs[i].data_ptr(), m, o, res)
        if rc not in (0, 1):
            raise sylv.SylvError(rc, "sign variant")
    ms, _ = _timed(sign, steps, warm, stream)
    rows["sign_variant"] = {"ms": ms, "gflops_2mnmn": flops_2(m, n) / ms / 1e6, "log2scale": int(res.log2scale)}

    # Robust against non-robust (Algorithm 4 against Algorithm 1) on the same input:
    # the cost of the overflow protection.
    Bp = F(B)
    for prec in ("fp64", "fp64_nonrobust"):
        Cs = [C0.clone() for _ in range(steps + warm)]

        def plain(i, prec=prec):
            o = sylv.make_opts(precision=prec, stream=stream.cuda_stream)
            rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), m, Bp.data_ptr(), n, Cs[i].data_ptr(), m, o, res)
            if rc not in (0, 1):
                raise sylv.SylvError(rc, prec)
        ms, _ = _timed(plain, steps, warm, stream)
        rows[prec] = {"ms": ms, "gflops_2mnmn": flops_2(m, n) / ms / 1e6}
    rows["robustness_overhead"] = rows["fp64"]["ms"] / rows["fp64_nonrobust"]["ms"] - 1.0
    Cs = [C0.clone() for _ in range(steps + warm)]

    Ag, _, Cg = inputs.problem(m, n, 0, kind="growth", upper=4.1)
    Agd = F(Ag)
    Cs = [F(Cg) for _ in range(steps + warm)]

    def tri(i):
        o = sylv.make_opts(stream=stream.cuda_stream)
        rc = sylv.sylv_tri_solve_triangular(m, n, Agd.data_ptr(), m, Cs[i].data_ptr(), m, o, res)
        if rc not in (0, 1):
            raise sylv.SylvError(rc, "triangular")
    ms, _ = _timed(tri, steps, warm, stream)
    rows["triangular"] = {"ms": ms, "gflops_m2n": 1.0 * m * m * n / ms / 1e6, "log2scale": int(res.log2scale)}

    rng = np.random.default_rng(7)
    U = np.linalg.qr(rng.standard_normal((m, m)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Ud, Vd, TAd, TBd = F(U), F(V), F(A), F(B)
    Cs = [C0.clone() for _ in range(steps + warm)]

    def schur(i):
        o = sylv.make_opts(stream=stream.cuda_stream)
        rc = sylv.sylv_solve_schur(m, n, Ud.data_ptr(), m, TAd.data_ptr(), m, Vd.data_ptr(), n, TBd.data_ptr(), n,
                                   Cs[i].data_ptr(), m, o, res)
        if rc not in (0, 1):
            raise sylv.SylvError(rc, "schur")
    ms, _ = _timed(schur, steps, warm, stream)
    rows["bartels_stewart"] = {"ms": ms, "gflops_6mnmn": 3 * flops_2(m, n) / ms / 1e6,
                               "note": "4 products on the tensor-core GEMM, dense binary64-accurate mode (4mn(m+n) flops) + the robust solve"}
    return {"metric": "variant solves, m = n = 4000", "value": rows["bartels_stewart"]["ms"], "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"m": m, "n": n, "tile": 32}, "rows": rows}


def run_robustness(args):
    """The cost-of-robustness sweep on the paper's own matrices (Sec. 3-4): strictly
    upper ones, diagonal blocks mu*T (A) and nu*T (B) with T in {1, [1 1; -1 1]},
    C = ones, m = n = 10000, nu = 1e-2 and mu from 1e2 down to 1e-7.  Small mu needs
    scaling far below the double range (alpha = 2^log2scale); the plain solve
    (Algorithm 1) overflows there.  Robust and plain times side by side."""
    import numpy as np
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    m = n = 10000
    nu = 1e-2
    F = lambda x: torch.from_numpy(np.asfortranarray(x)).to(dev)  # noqa: E731
    B = F(inputs.paper_matrix(n, nu, seed=2))
    C0 = torch.ones((n, m), dtype=torch.float64, device=dev).t()
    rows = []
    steps, warm = max(1, args.steps), max(1, args.warmup)
    for mu in (1e2, 10.0, 1.0, 1e-3, 1e-7):
        A = F(inputs.paper_matrix(m, mu, seed=1))
        row = {"mu": mu}
        for prec in ("fp64", "fp64_nonrobust"):
            Cs = [C0.clone() for _ in range(steps + warm)]
            res = sylv.sylv_result()

            def fn(i, prec=prec, res=res):
                o = sylv.make_opts(precision=prec, stream=stream.cuda_stream)
                rc = sylv.sylv_tri_solve_ex(m, n, A.data_ptr(), m, B.data_ptr(), n, Cs[i].data_ptr(), m, o, res)
                if rc >= 100 or rc < 0:
                    raise sylv.SylvError(rc, prec)
            ms, _ = _timed(fn, steps, warm, stream)
            row[prec] = {"ms": ms, "gflops_2mnmn": flops_2(m, n) / ms / 1e6, "info": int(res.info),
                         "log2scale": int(res.log2scale), "scale_events": int(res.scale_events),
                         "finite": bool(torch.isfinite(Cs[-1]).all())}
            del Cs
        row["overhead"] = row["fp64"]["ms"] / row["fp64_nonrobust"]["ms"] - 1.0
        rows.append(row)
    return {"metric": "cost of robustness on the paper's matrices", "value": max(r["overhead"] for r in rows),
            "unit": "fraction (robust / plain - 1, worst mu)", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic (the paper's generator)",
            "config": {"m": m, "n": n, "nu": nu, "tile": 32}, "rows": rows}


def run_robust_vs_plain(args):
    """Robust FP64 (Algorithm 4) against non-robust FP64 (Algorithm 1 per tile) at
    m = n = 4000 on "overflow_4000", whose unscaled substitution grows ~1400 bits: the
    plain solve overflows, the robust one scales (alpha = 2^log2scale).  Roofline of
    the robust solve's tile kernel as for the headline."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    name = args.workload or "overflow_4000"
    A, B, C, w = inputs.workload(name)
    m, n, tile = w["m"], w["n"], args.tile or w["tile"]
    dev = torch.device("cuda", 0)
    Ad, Bd, C0 = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    stream = torch.cuda.current_stream(dev)
    rows = {}
    for prec in ("fp64", "fp64_nonrobust"):
        opts = sylv.make_opts(tile=tile, precision=prec, stream=stream.cuda_stream, sync=True)
        wsb = sylv.sylv_workspace_size(m, n, opts)
        wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
        opts.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
        opts.workspace_bytes = wsb
        Cs = [C0.clone() for _ in range(args.warmup + args.steps)]
        res = sylv.sylv_result()

        def fn(i, opts=opts, Cs=Cs, res=res):
            rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1),
                                        Cs[i].data_ptr(), Cs[i].stride(1), opts, res)
            if rc >= 100 or rc < 0:
                raise sylv.SylvError(rc, prec)

        sylv.sylv_profile(True)
        ms, _ = _timed(fn, args.steps, args.warmup, stream)
        dag_ms, dag_n = sylv.sylv_profile_read()
        sylv.sylv_profile(False)
        dag_per = dag_ms / max(dag_n, 1)  # includes the warm-up launches: same kernel, same work
        ach = flops_alg(m, n) / (dag_per / 1000) / 1e9
        rows[prec] = {"ms_per_solve": ms, "gflops_2mnmn": flops_2(m, n) / ms / 1e6, "info": int(res.info),
                      "log2scale": int(res.log2scale), "scale_events": int(res.scale_events),
                      "finite": bool(torch.isfinite(Cs[-1]).all()), "dag_ms_per_launch": dag_per,
                      "roofline_frac": ach / FP64_PEAK_GFLOPS}
        del Cs, wsbuf
    return {"metric": "robust Sylvester solve GFLOP/s", "value": rows["fp64"]["gflops_2mnmn"], "unit": "GFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "m": m, "n": n, "tile": tile, "generator": w["kind"],
                                            "upper_scale": w["upper"]},
            "robust": rows["fp64"], "nonrobust": rows["fp64_nonrobust"],
            "robustness_overhead": rows["fp64"]["ms_per_solve"] / rows["fp64_nonrobust"]["ms_per_solve"] - 1.0}


def run_small(args):
    """m = n = 256 (benign, seed 0): a latency-bound solve with a short critical path of
    diagonal-tile solves; microseconds per solve and solves/s, one call per solve on
    one stream (each call enqueues the whole launch sequence).  The value is at the
    configuration's tile 64; tiles 32, 24 and 16 are timed beside it."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    name = args.workload or "benign_256"
    A, B, C, w = inputs.workload(name)
    m, n = w["m"], w["n"]
    dev = torch.device("cuda", 0)
    Ad, Bd, C0 = (torch.from_numpy(x).to(dev) for x in (A, B, C))
    stream = torch.cuda.current_stream(dev)
    reps = 50
    rdev = torch.zeros(64, dtype=torch.uint8, device=dev)
    by_tile = {}
    tiles = [args.tile or w["tile"]] + [t for t in (32, 24, 16) if t != (args.tile or w["tile"])]
    for tile in tiles:
        opts = sylv.make_opts(tile=tile, stream=stream.cuda_stream, sync=False)
        wsb = sylv.sylv_workspace_size(m, n, opts)
        wsbuf = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
        opts.workspace = (wsbuf.data_ptr() + 255) // 256 * 256
        opts.workspace_bytes = wsb
        Cs = [C0.clone() for _ in range(reps * (args.warmup + args.steps))]

        def fn(i, opts=opts, Cs=Cs):
            for j in range(reps):
                c = Cs[i * reps + j]
                rc = sylv.sylv_tri_solve_ex(m, n, Ad.data_ptr(), Ad.stride(1), Bd.data_ptr(), Bd.stride(1),
                                            c.data_ptr(), c.stride(1), opts, rdev.data_ptr())
                if rc != 0:
                    raise sylv.SylvError(rc, "small")

        ms, _ = _timed(fn, args.steps, args.warmup, stream)
        res = sylv.sylv_result.from_buffer_copy(rdev[:40].cpu().numpy().tobytes())
        us = 1000.0 * ms / reps
        by_tile[str(tile)] = {"us_per_solve": us, "solves_per_s": 1e6 / us, "info": int(res.info)}
        del Cs, wsbuf
    t0 = str(tiles[0])
    return {"metric": "solves/s", "value": by_tile[t0]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "m": m, "n": n, "tile": tiles[0], "solves_per_step": reps},
            "us_per_solve": by_tile[t0]["us_per_solve"], "gflops_2mnmn": flops_2(m, n) / by_tile[t0]["us_per_solve"] / 1e3,
            "by_tile": by_tile}


def run_batch(args):
    """A batch of --count equations of the 4096-equation distribution (m, n
    log-uniform in [16, 512], wellcond, per-equation seeds), one plan, executed
    --warmup + --steps times without a graph at --precision (tile 32): solves/s.  The
    plain form of the batched configuration, for profiles at a reduced count."""
    import torch
    from paper_1905_10574_gb300 import build, inputs, sylv
    build.build()
    sylv.load()
    count = args.count
    shapes = inputs.batch_shapes(count, 16, 512, seed=1234)
    dev = torch.device("cuda", 0)
    As, Bs, C0s = [], [], []
    for i, (m, n) in enumerate(shapes):
        A, B, C = inputs.problem(m, n, 10000 + i, kind="wellcond")
        As.append(torch.from_numpy(A).to(dev))
        Bs.append(torch.from_numpy(B).to(dev))
        C0s.append(torch.from_numpy(C).to(dev))
    Cs = [c.clone() for c in C0s]
    stream = torch.cuda.current_stream(dev)
    o = sylv.make_opts(stream=stream.cuda_stream, precision=args.precision, tile=args.tile or 32,
                       tol=MIXED_TOL if args.precision == "fp32_refine" else 0.0)
    plan = sylv.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                  [a.stride(1) for a in As], [b.data_ptr() for b in Bs], [b.stride(1) for b in Bs],
                                  [c.data_ptr() for c in Cs], [c.stride(1) for c in Cs], o)

    def fn(_):
        for c, c0 in zip(Cs, C0s):
            c.copy_(c0)
        rc = sylv.sylv_batch_execute(plan, stream.cuda_stream)
        if rc:
            raise sylv.SylvError(rc, "batch")

    try:
        ms, _ = _timed(fn, max(1, args.steps), args.warmup, stream)
        rc, res = sylv.sylv_batch_results(plan, count)
    finally:
        sylv.sylv_batch_destroy(plan)
    return {"metric": "batched solves/s", "value": count / (ms / 1000), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"count": count, "m_n": "log-uniform [16,512]", "generator": "wellcond",
                       "precision": args.precision, "tile": args.tile or 32, "cuda_graph": False,
                       "note": "timed steps include the refill of the right-hand sides"},
            "worst_info": max(r.info for r in res)}


def run_peaks(args):
    """Measured peak rates of the FMA pipes the tile kernels are bound by (the
    denominators of their rooflines): binary64 FMA (the FP64 solve) and binary32 FMA
    (the FP32 correction solves), from sylv_diag_fma_rate, clocks sampled meanwhile;
    the derived unit-count peaks beside them."""
    import torch
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    sylv.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for kind, name, iters in ((0, "fp64_fma", 120000), (1, "fp32_fma", 3000000)):
        vals = []
        for _ in range(max(3, args.steps)):
            rc, g, ms = sylv.sylv_diag_fma_rate(kind, iters, stream)
            if rc != 0:
                raise sylv.SylvError(rc, "sylv_diag_fma_rate")
            vals.append((g, ms))
        out[name] = {"gflops_best": max(v[0] for v in vals), "gflops_median": statistics.median(v[0] for v in vals),
                     "ms_per_launch": statistics.median(v[1] for v in vals), "iters": iters}
    clocks = sampler.stop()
    out["fp64_fma"]["derived_gflops"] = nsm * 4 * 2.070
    out["fp32_fma"]["derived_gflops"] = nsm * 256 * 2.070
    return {"metric": "FMA pipe peak GFLOP/s", "value": out["fp64_fma"]["gflops_best"], "unit": "GFLOP/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f64 / f32", "data": "synthetic",
            "config": {"probe": "one full wave of 256-thread CTAs, 8 (binary64) or 16 (binary32) independent FMA chains per thread", "sms": nsm},
            "fp64_fma": out["fp64_fma"], "fp32_fma": out["fp32_fma"], "clocks": clocks}


def secondary(args):
    """The other configurations, measured briefly beside the headline solve."""
    import argparse as _ap
    import torch
    out = {}
    sub = _ap.Namespace(**vars(args))
    sub.workload, sub.tile = None, 0
    sub.steps, sub.warmup = 2, 1
    for name, fn in (("robust_vs_nonrobust_4000", run_robust_vs_plain), ("small_256", run_small),
                     ("mixed_precision_8000", run_mixed), ("batched_4096", run_batched),
                     ("adjoint_256x512", run_adjoint)):
        sub.steps, sub.warmup = (5, 2) if name in ("robust_vs_nonrobust_4000", "small_256") else (2, 1)
        try:
            r = fn(sub)
            r.pop("n_gpus", None)
            out[name] = r
        except Exception as exc:  # report, do not hide, a failing secondary measurement
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.mode == "solve" or args.impl == "reference":
        args.workload = args.workload or WORKLOAD
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "mixed":
        print(json.dumps(run_mixed(args)), flush=True)
    elif args.mode == "residual":
        print(json.dumps(run_residual(args)), flush=True)
    elif args.mode == "batched":
        line = run_batched(args)
        if line is not None:
            print(json.dumps(line), flush=True)
    elif args.mode == "adjoint":
        print(json.dumps(run_adjoint(args)), flush=True)
    elif args.mode == "smscale":
        print(json.dumps(run_smscale(args)), flush=True)
    elif args.mode == "variants":
        print(json.dumps(run_variants(args)), flush=True)
    elif args.mode == "robustness":
        print(json.dumps(run_robustness(args)), flush=True)
    elif args.mode == "robust_vs_plain":
        print(json.dumps(run_robust_vs_plain(args)), flush=True)
    elif args.mode == "small":
        print(json.dumps(run_small(args)), flush=True)
    elif args.mode == "peaks":
        print(json.dumps(run_peaks(args)), flush=True)
    elif args.mode == "batch":
        print(json.dumps(run_batch(args)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
