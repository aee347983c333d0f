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
# DRAM bytes (read + write) per launch of the tensor-core solve kernel, averaged over the
# solve launches of one step of this workload, from one single-pass ncu capture of the
# bench command's launch list (dram__bytes_read.sum + dram__bytes_write.sum), per --prec.
# An entry is removed when the kernel changes.
SOLVE_TRAFFIC_BYTES_PER_LAUNCH = {"f16": 546.8e6}
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
def cpu_oracle_sample(wl, apps_per_rhs):
    """Time the oracle, as it stands, on a bounded sample of the workload: one
    application of Algorithm 3.1 to one right-hand side plus one FP64 operator
    product (one GMRES iteration), scaled by the DDM applications per
    right-hand side the GPU solve needed.  Local factorisations are excluded
    (they are reused across right-hand sides, as the GPU factors are)."""
    from oracle import ddm as OD
    from oracle import helmholtz as OH
    t0 = time.time()
    A, J = OH.global_operator(wl)
    part = OD.Partition(wl)
    t_setup = time.time() - t0
    b = wl.f[:1] * J.reshape((1,) + wl.f.shape[1:])
    t1 = time.time()
    z = OD.diagonal_sweep(part, b)
    _ = A @ z.reshape(1, -1).T
    t_iter = time.time() - t1
    per_rhs = t_iter * max(1, apps_per_rhs)
    return {"value": 1.0 / per_rhs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": (f"one Algorithm 3.1 application + one operator product on 1 of "
                       f"{wl.nrhs} RHS ({t_iter:.2f} s), x {apps_per_rhs} applications per RHS; "
                       f"local SuperLU factorisations ({t_setup:.1f} s) excluded; "
                       "SuperLU and the sparse products are single-threaded")}


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
    """--impl reference: the CPU oracle as it stands, on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    wl = W.config(args.workload)
    from oracle import ddm as OD
    from oracle import helmholtz as OH
    A, J = OH.global_operator(wl)
    part = OD.Partition(wl)
    b = wl.f[:1] * J.reshape((1,) + wl.f.shape[1:])
    apps = 6  # DDM applications per RHS of the GPU solve at rtol 1e-8 on this workload (measured)
    times = []
    for i in range(args.warmup + args.steps):
        t = time.time()
        z = OD.diagonal_sweep(part, b)
        _ = A @ z.reshape(1, -1).T
        if i >= args.warmup:
            times.append(time.time() - t)
    per_step = statistics.mean(times) * apps
    val = 1.0 / per_step
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": wl.name, "grid": list(wl.N),
                                             "nb": list(wl.nb), "nrhs": 1},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "host_cpus": os.cpu_count(),
                             "sample": f"per step: one Algorithm 3.1 application + one operator "
                                       f"product on 1 RHS, x {apps} applications per RHS"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    ctx = H.helm_setup_workload(wl, precision=prec, profile=1, stream=stream)
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
    cpu = None if (args.no_cpu or world > 1) else cpu_oracle_sample(wl, apps)  # rank 0 at N = 1 only
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f16": "f16", "tf32": "tf32", "mixed": "c64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": list(wl.N), "h_m": wl.h,
                   "freq_hz": round(wl.omega / (2 * np.pi), 6),
                   "nb": list(wl.nb), "overlap": wl.overlap, "sub_pml": wl.sub_pml,
                   "nrhs": nrhs, "rtol": args.rtol, "outer": "FP64 flexible GMRES",
                   "subdomain_precision": {
                       "f16": "complex64 factors, FP16 tensor-core operands with power-of-two scales "
                              "per factor line and right-hand-side column, FP32 accumulation",
                       "tf32": "complex64 factors, TF32 tensor-core block products, FP32 accumulation",
                       "mixed": "complex64 factors and FP32 block products"}[args.prec],
                   "l2": "inputs larger than L2 (device working set %.1f GB, RHS %.2f GB)" % (
                       dev_bytes / 1e9, nrhs * np.prod(wl.N) * 16 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "gmres": {"iters": iters, "applications": apps, "max_rel_resid": res,
                  "factor_ms": factor_ms, "levels": stats[0]["levels"],
                  "subdomain_solves_per_application": stats[0]["solves"]},
        "roofline": {"kernel": ("solve_twist_kernel" if args.prec in ("tf32", "f16") else "solve_kernel")
                     + " (subdomain forward/backward block solves)",
                     "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (SOLVE_TRAFFIC_BYTES_PER_LAUNCH.get(args.prec)
                                 if args.workload == 2 and not args.nrhs else None),
                     "traffic_unit": "bytes per launch", "peak_source": peak_src,
                     "tflops_achieved": tflops,
                     "bytes_per_launch": sol["bytes"] / max(1, sol["launches"]),
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
