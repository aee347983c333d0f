#!/usr/bin/env python
"""Throughput of the diagonal sweeping DDM solver on one GB300.

Default workload (--workload 4): the 2D smooth-medium problem on a 2088 x 1576
grid (2048 x 1536 interior cells and a 20-cell PML), h = 7.5 m,
omega = 2 pi 20 Hz, cut into 12 x 9 subdomains of non-uniform widths (96-224
cells; windows up to 280 block rows with overlap 8 and subdomain PML 20), with
256 point sources.  --workload 2 selects the 1064^2 layered problem (8 x 8
subdomains, 64 sources).  One step = one helm_solve of all right-hand sides:
DDM-preconditioned FP64 flexible GMRES (float-float arithmetic on the FP32
pipes) with complex64 subdomain factors and FP16 tensor-core solves (--prec
tf32 | mixed select the other modes), to a relative residual of --rtol; the
call splits the batch into chunks when its vectors do not fit the device.
Factors are computed once, outside the timed steps, and reported separately
(and as a factor-amortised rate).  Metric: right-hand sides solved per second.

Also reported on the same line: the plain FP64 GPU DDM (complex128 factors and
solves, same algorithm; on the first --fp64-nrhs sources, single-GPU runs),
the roofline of the dominant kernel (subdomain solve) from CUDA events on the
library's stream, SM clocks sampled during the timed region, an end-to-end
figure through the C ABI with host buffers (slowest replica), and the CPU
oracle's full FGMRES on as many sources as host memory allows, one
single-threaded process each (rank 0 of a single-GPU run).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 run under torch.distributed.run; every rank solves its own copy of
the workload (independent replicas: the path has no exchange across GPUs).
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS solves/sec at 1e-6 rel. L2 (mixed vs plain FP64 GPU DDM); %tensor/HBM roofline"
# DRAM bytes (read + write) per launch of the solve kernel, averaged over the solve
# launches of one step, from one single-pass ncu capture of the bench command's launch
# list (dram__bytes_read.sum + dram__bytes_write.sum), per (workload, kernel).  An entry
# is removed when the kernel changes.
SOLVE_TRAFFIC_BYTES_PER_LAUNCH = {
    # 60 consecutive launches (one DDM application, 128 right-hand sides per chunk)
    ("2d-smooth-2088x1576-12x9-256rhs", "solve_twist_kernel"): 2.0598e9,
}
UNIT = "RHS/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=60)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU DDM")
    ap.add_argument("--fp64-nrhs", type=int, default=16,
                    help="sources the plain FP64 GPU DDM solves (its first ones; 0 = all)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", type=int, default=4,
                    help="workload number (4 = 2088x1576 12x9 256 sources; 2 = 1064^2 8x8 64 sources)")
    ap.add_argument("--prec", default="f16", choices=["f16", "tf32", "mixed"],
                    help="precision of the subdomain factors/solves of the product path")
    ap.add_argument("--tc-kernel", type=int, default=0,
                    help="helm_config.tc_kernel of the product path (0 = default kernel choice)")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="use only the first NRHS sources (profiling runs); 0 = all")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.rows = []
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def _cpu_seconds():
    t = os.times()
    return t.user + t.system


def oracle_gmres_iterations(name):
    """Iterations the oracle's own FGMRES needs on this workload's first source
    at the benchmark's residual, as written by
    tests/golden/make_oracle_gmres_iters.py (which calls only oracle/)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_gmres_iters.txt")
    if os.path.exists(path):
        for line in open(path):
            f = line.split()
            if f and not line.startswith("#") and f[0] == name:
                return int(f[2])
    return None


def _oracle_setup(wl):
    """The oracle's global operator and partition (with its local SuperLU
    factorisations) for the workload's first right-hand side."""
    from oracle import ddm as OD
    from oracle import helmholtz as OH
    one = dataclasses.replace(wl, f=wl.f[:1])
    t0 = time.time()
    A, J = OH.global_operator(one)
    part = OD.Partition(one)
    b = one.f * J.reshape((1,) + one.f.shape[1:])
    return A, part, b, time.time() - t0


def _oracle_fgmres_one(job):
    """One host process: the oracle's global operator, partition and local
    SuperLU factorisations for one source of the workload, then its FGMRES
    (restart 30, one Algorithm 3.1 application per iteration) to the relative
    residual, run to the end.  Single-threaded (the parent sets the BLAS and
    OpenMP thread counts to 1 before starting the process)."""
    workload, src, rtol = job
    import workloads as W
    from oracle import ddm as OD
    from oracle import helmholtz as OH
    from oracle import krylov as OK
    wl = W.config(workload, src=[src])
    c0, t0 = _cpu_seconds(), time.time()
    A, J = OH.global_operator(wl)
    part = OD.Partition(wl)
    b = wl.f * J.reshape((1,) + wl.f.shape[1:])
    t1 = time.time()

    def apply_A(x):
        return (A @ x.reshape(x.shape[0], -1).T).T.reshape(x.shape)

    x, info = OK.gmres(apply_A, b, lambda v: OD.diagonal_sweep(part, v), rtol=rtol, restart=30, maxit=60)
    t2 = time.time()
    return {"src": src, "factor_s": t1 - t0, "gmres_s": t2 - t1, "cpu_s": _cpu_seconds() - c0,
            "iters": int(info["iters"][0]), "resid": float(info["resid"][0])}


# peak resident memory of one oracle process (measured on x86: 13.3 GB for the
# 2088x1576 workload, 4.3 GB for the 1064^2 one), with a margin
ORACLE_PROC_BYTES = {2: 6e9, 4: 18e9}


def _mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def cpu_oracle_sample(workload, nrhs, rtol):
    """The oracle, as it stands, on the host cores: P single-threaded processes
    (P = the host's cores, capped at 8 and by half the available memory), each
    running the oracle's full FGMRES on its own source of the workload to the
    benchmark's relative residual.  Their local SuperLU factorisations are
    timed apart (they serve every right-hand side, as the GPU factors do).
    value = P sources / the longest FGMRES time (all cores); per_core_value =
    1 / the median FGMRES time (one core)."""
    import multiprocessing as mp
    host = os.cpu_count() or 1
    per = ORACLE_PROC_BYTES.get(workload, 18e9)
    P = max(1, min(host, 8, nrhs, int(0.5 * _mem_available() // per)))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        t0 = time.time()
        with mp.get_context("spawn").Pool(P) as pool:
            res = pool.map(_oracle_fgmres_one, [(workload, s, rtol) for s in range(P)])
        wall = time.time() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    g = [r["gmres_s"] for r in res]
    f = [r["factor_s"] for r in res]
    cores = sum(r["cpu_s"] for r in res) / wall
    it = max(r["iters"] for r in res)
    return {"value": P / max(g), "unit": UNIT, "cores": round(cores, 2), "procs": P, "kind": "oracle",
            "host_cpus": host, "per_core_value": 1.0 / statistics.median(g),
            "factor_s": max(f), "factor_amortised_value": P / max(a + b for a, b in zip(f, g)),
            "iters": it, "resid": max(r["resid"] for r in res),
            "sample": (f"the oracle's full FGMRES (restart 30, one Algorithm 3.1 application per iteration) "
                       f"on sources 0..{P - 1} of {nrhs}, one single-threaded process each, run to relative "
                       f"residual {rtol:g}: {it} iterations at most, FGMRES {min(g):.1f}-{max(g):.1f} s; "
                       f"the local SuperLU factorisations ({max(f):.1f} s) are reported apart")}


def job_ms(ms_local, world, device=None):
    """Per-step time of the whole job: the slowest replica's (max over ranks)."""
    if world <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on the same workload, rank 0
    only.  Every step, warm-up and timed alike, is one of the four sweeps of the
    oracle's Algorithm 3.1 applied to the workload's first source (a bounded
    sample: a full application of the oracle takes four).  RHS/s is 1 / (sweeps
    per application x applications per right-hand side x the mean step time, plus
    one operator product per application), with the oracle's own FGMRES
    iteration count on this workload (tests/golden/oracle_gmres_iters.txt)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    from oracle import ddm as OD
    wl = W.config(args.workload)
    A, part, b, t_fac = _oracle_setup(wl)
    n_it = oracle_gmres_iterations(wl.name) or 1
    nsw = 2 ** wl.ndim
    c0 = _cpu_seconds()
    t_all = time.time()
    times = []
    for i in range(args.warmup + args.steps):
        t = time.time()
        OD.diagonal_sweep(part, b, nsweeps=1)
        if i >= args.warmup:
            times.append(time.time() - t)
    t = time.time()
    _ = A @ b.reshape(1, -1).T
    t_mv = time.time() - t
    cores = (_cpu_seconds() - c0) / (time.time() - t_all)
    step = statistics.mean(times)
    per_rhs = n_it * (nsw * step + t_mv)
    val = 1.0 / per_rhs
    sample = (f"per step: the first sweep of the oracle's Algorithm 3.1 on source 0 of {wl.nrhs} "
              f"({step:.2f} s); RHS/s = 1 / ({n_it} FGMRES iterations of the oracle x ({nsw} sweeps x step "
              f"+ one operator product, {t_mv:.2f} s)); local SuperLU factorisations ({t_fac:.1f} s) excluded")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": workload_config(wl, args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": round(cores, 2), "kind": "oracle",
                             "host_cpus": os.cpu_count(), "sample": sample, "factor_s": t_fac},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(wl, args):
    """The `config` object of both arms' JSON lines."""
    return {"workload": wl.name, "grid": list(wl.N), "h_m": wl.h,
            "freq_hz": round(wl.omega / (2 * np.pi), 6), "nb": list(wl.nb), "overlap": wl.overlap,
            "sub_pml": wl.sub_pml, "nrhs": wl.nrhs, "rtol": args.rtol}


# ----------------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_2002_05327_gb300 as H
    import workloads as W
    from paper_2002_05327_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    H.lib()
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = W.config(args.workload)
    if args.nrhs:
        wl.f = wl.f[:args.nrhs]
    nrhs = wl.nrhs
    hbm, bf16, peak_src = load_peaks()

    # ---------------- mixed precision (the product path)
    stream = torch.cuda.current_stream(dev).cuda_stream
    prec = {"f16": H.HELM_PREC_F16, "tf32": H.HELM_PREC_TF32, "mixed": H.HELM_PREC_MIXED}[args.prec]
    ctx = H.helm_setup_workload(wl, precision=prec, profile=1, stream=stream, tc_kernel=args.tc_kernel)
    t0 = time.time()
    H.helm_factor(ctx)
    factor_ms = (time.time() - t0) * 1e3
    F = torch.from_numpy(wl.f).to(dev)
    for _ in range(args.warmup):
        U, st = H.helm_solve(ctx, F, rtol=args.rtol, maxit=args.maxit)
    torch.cuda.synchronize()
    H.helm_profile_reset(ctx)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = []
    for _ in range(args.steps):
        U, st = H.helm_solve(ctx, F, rtol=args.rtol, maxit=args.maxit)
        stats.append(st)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = H.helm_profile_get(ctx)
    ms = job_ms(ms, world, dev)
    value = world * nrhs / (ms / 1e3)
    launches = sum(v["launches"] for v in prof.values())
    sol = prof["solve"]
    achieved = sol["bytes"] / (sol["ms"] / 1e3) / 1e9 if sol["ms"] > 0 else 0.0
    tflops = sol["flops"] / (sol["ms"] / 1e3) / 1e12 if sol["ms"] > 0 else 0.0
    kshare = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())), 4)
              for k, v in prof.items()}
    res = max(s["resid"] for s in stats)
    iters = max(s["iters"] for s in stats)
    apps = max(s["applications"] for s in stats)
    dev_bytes = H.helm_device_bytes(ctx)

    # ---------------- end to end through the C ABI with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        Fh = torch.from_numpy(wl.f).pin_memory()
        Uh = torch.empty_like(Fh).pin_memory()
        import ctypes
        Lb = H.lib()
        sth = H.helm_stats()

        def host_solve():
            rc = Lb.helm_solve(ctx.ptr, nrhs, ctypes.c_void_p(Fh.data_ptr()),
                               ctypes.c_void_p(Uh.data_ptr()), H.HELM_MEM_HOST, args.rtol,
                               args.maxit, ctypes.byref(sth))
            if rc != 0:
                raise H.HelmError(rc, "helm_solve (host buffers)")

        for _ in range(args.warmup):  # untimed: the context's staging buffers grow here
            host_solve()
        torch.cuda.synchronize()
        t = time.time()
        for _ in range(args.steps):
            host_solve()
        e2e_ms = job_ms((time.time() - t) * 1e3 / args.steps, world, dev)  # slowest replica
        e2e = {"value": world * nrhs / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(Fh.numel() * 16), "d2h_bytes_per_step": int(Uh.numel() * 16),
               "ms_per_step": e2e_ms}
        Ucheck = Uh.numpy()  # a view of the pinned host buffer
    else:
        Ucheck = U[:max(1, args.fp64_nrhs or nrhs)].cpu().numpy()
    ctx.close()

    # ---------------- plain FP64 GPU DDM, same algorithm (the comparator; N = 1 only)
    fp64 = None
    if not args.no_fp64 and world == 1:
        n64 = nrhs if args.fp64_nrhs <= 0 else min(nrhs, args.fp64_nrhs)
        F64 = F[:n64]
        c64 = H.helm_setup_workload(wl, precision=H.HELM_PREC_F64, stream=stream)
        t0 = time.time()
        H.helm_factor(c64)
        f64_factor_ms = (time.time() - t0) * 1e3
        U64, st64 = H.helm_solve(c64, F64, rtol=args.rtol, maxit=args.maxit)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        U64, st64 = H.helm_solve(c64, F64, rtol=args.rtol, maxit=args.maxit)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        U64 = U64.cpu().numpy()
        diff = max(float(np.linalg.norm(U64[r] - Ucheck[r]) / np.linalg.norm(U64[r])) for r in range(n64))
        fp64 = {"value": n64 / (ms64 / 1e3), "unit": UNIT, "nrhs": n64, "ms_per_step": ms64,
                "factor_ms": f64_factor_ms, "iters": st64["iters"], "resid": st64["resid"],
                "max_rel_diff_to_mixed_per_rhs": diff, "steps": 1, "warmup": 1}
        c64.close()

    if rank != 0:
        return
    # rank 0 at N = 1 only, after every GPU step
    cpu = None if (args.no_cpu or world > 1) else cpu_oracle_sample(args.workload, nrhs, args.rtol)
    # roofline of the solve kernel: HBM (algorithmic bytes) or tensor pipe (algorithmic
    # flops), whichever the algorithm's intensity makes binding at the measured peaks
    t_hbm = sol["bytes"] / (hbm * 1e9)
    t_tc = sol["flops"] / (bf16 * 1e12)
    bound = "tensor" if t_tc > t_hbm else "hbm"
    kname = {"f16": "solve_twist_kernel", "tf32": "solve_twist_kernel", "mixed": "solve_kernel"}[args.prec]
    cfg = workload_config(wl, args)
    cfg.update({"outer": "FP64 flexible GMRES (float-float arithmetic, ~48 significand bits)",
                "subdomain_precision": {
                    "f16": "complex64 factors, FP16 tensor-core operands with power-of-two scales "
                           "per factor line and right-hand-side column, FP32 accumulation",
                    "tf32": "complex64 factors, TF32 tensor-core block products, FP32 accumulation",
                    "mixed": "complex64 factors and FP32 block products"}[args.prec],
                "l2": "inputs larger than L2 (device working set %.1f GB, RHS %.2f GB)" % (
                    dev_bytes / 1e9, nrhs * np.prod(wl.N) * 16 / 1e9),
                "parallelism": "replicas" if world > 1 else "single"})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f16": "f16", "tf32": "tf32", "mixed": "c64"}[args.prec],
        "data": "synthetic",
        "config": cfg,
        "factor_amortised_value": nrhs * world / (ms / 1e3 + factor_ms / 1e3),
        "gmres": {"iters": iters, "applications": apps, "max_rel_resid": res,
                  "factor_ms": factor_ms, "levels": stats[0]["levels"],
                  "subdomain_solves_per_application": stats[0]["solves"]},
        "roofline": {"kernel": kname + " (subdomain forward/backward block solves)",
                     "bound": bound,
                     "achieved": tflops if bound == "tensor" else achieved,
                     "peak": bf16 if bound == "tensor" else hbm,
                     "unit": "TFLOP/s" if bound == "tensor" else "GB/s",
                     "frac": tflops / bf16 if bound == "tensor" else achieved / hbm,
                     "traffic": (SOLVE_TRAFFIC_BYTES_PER_LAUNCH.get((wl.name, kname))
                                 if not args.nrhs else None),
                     "traffic_unit": "bytes per launch", "peak_source": peak_src,
                     "hbm_achieved_gbs": achieved, "hbm_frac": achieved / hbm,
                     "tflops_achieved": tflops, "tensor_frac": tflops / bf16,
                     "bytes_per_launch": sol["bytes"] / max(1, sol["launches"]),
                     "bytes_convention": "block inverses at complex64 storage (8 bytes per entry), "
                                         "read once per forward and once per backward pass, plus "
                                         "b, y, y, u once per right-hand side" + (
                                             "; the FP16 image the kernel streams holds 4 bytes "
                                             "per entry" if args.prec == "f16" else ""),
                     "flops_per_launch": sol["flops"] / max(1, sol["launches"]),
                     "ms_per_launch": sol["ms"] / max(1, sol["launches"])},
        "kernel_time_share": kshare,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "fp64_ddm": fp64,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
