#!/usr/bin/env python
"""Throughput of the diagonal sweeping DDM solver on one GB300.

Workload: the 2D layered seismic-shaped problem -- 1024^2 interior cells
(1064^2 with a 20-cell PML), h = 10 m, omega = 2 pi 15 Hz, five layers of
1.5-4.5 km/s with a +-10 % correlated perturbation, 8 x 8 subdomains
(box 128, overlap 8, subdomain PML 20), 64 point sources at 20 m depth.
One step = one helm_solve of all 64 right-hand sides: DDM-preconditioned FP64
flexible GMRES (float-float arithmetic on the FP32 pipes) with complex64
subdomain factors and FP16 tensor-core solves (--prec tf32 | mixed select the
other modes), to a relative residual of --rtol.  Factors are computed once, outside the timed steps, and
reported separately.  Metric: right-hand sides solved per second.

Also reported on the same line: the plain FP64 GPU DDM (complex128 factors and
solves, same algorithm; single-GPU runs), the roofline of the dominant kernel
(subdomain solve) from CUDA events on the library's stream, SM clocks sampled
during the timed region, an end-to-end figure through the C ABI with host
buffers (slowest replica), and the CPU oracle timed on a bounded sample
(rank 0 of a single-GPU run).

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
SOLVE_TRAFFIC_BYTES_PER_LAUNCH = {}
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
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", type=int, default=2, help="workload number (2 = bench)")
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


def cpu_oracle_sample(wl, rtol):
    """The oracle, as it stands, on the host cores: its FGMRES (restart 30),
    preconditioned by its Algorithm 3.1, on the first right-hand side of the
    workload to the benchmark's relative residual, run to the end.  The local
    SuperLU factorisations are timed separately (they serve every right-hand
    side, as the GPU factors do).  BLAS may use every host core; `cores` is the
    CPU time the run took over its wall time."""
    from oracle import ddm as OD
    from oracle import krylov as OK
    A, part, b, t_fac = _oracle_setup(wl)

    def apply_A(x):
        return (A @ x.reshape(x.shape[0], -1).T).T.reshape(x.shape)

    c0, t0 = _cpu_seconds(), time.time()
    x, info = OK.gmres(apply_A, b, lambda v: OD.diagonal_sweep(part, v), rtol=rtol, restart=30, maxit=60)
    wall = time.time() - t0
    cores = (_cpu_seconds() - c0) / wall
    it, res = int(info["iters"][0]), float(info["resid"][0])
    return {"value": 1.0 / wall, "unit": UNIT, "cores": round(cores, 2), "kind": "oracle",
            "host_cpus": os.cpu_count(), "iters": it, "resid": res, "factor_s": t_fac,
            "factor_amortised_value": 1.0 / (wall + t_fac / wl.nrhs),
            "sample": (f"the oracle's FGMRES (restart 30, one Algorithm 3.1 application per iteration) on "
                       f"source 0 of {wl.nrhs}, run to relative residual {rtol:g}: {it} iterations, "
                       f"residual {res:.1e}, {wall:.1f} s; its local SuperLU factorisations ({t_fac:.1f} s) "
                       f"are reported apart; SuperLU and the SciPy sparse products are single-threaded")}


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
        Ucheck = Uh.numpy()
    else:
        Ucheck = U.cpu().numpy()
    ctx.close()

    # ---------------- plain FP64 GPU DDM, same algorithm (the comparator; N = 1 only)
    fp64 = None
    if not args.no_fp64 and world == 1:
        c64 = H.helm_setup_workload(wl, precision=H.HELM_PREC_F64, stream=stream)
        t0 = time.time()
        H.helm_factor(c64)
        f64_factor_ms = (time.time() - t0) * 1e3
        U64, st64 = H.helm_solve(c64, F, rtol=args.rtol, maxit=args.maxit)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        U64, st64 = H.helm_solve(c64, F, rtol=args.rtol, maxit=args.maxit)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        diff = float(torch.linalg.vector_norm(U64 - U) / torch.linalg.vector_norm(U64))
        fp64 = {"value": world * nrhs / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "factor_ms": f64_factor_ms, "iters": st64["iters"], "resid": st64["resid"],
                "rel_diff_to_mixed": diff, "steps": 1, "warmup": 1}
        c64.close()

    if rank != 0:
        return
    cpu = None if (args.no_cpu or world > 1) else cpu_oracle_sample(wl, args.rtol)  # rank 0 at N = 1 only
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
