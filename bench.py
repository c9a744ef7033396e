"""Benchmark: RS-S factor + refined solve throughput (points/s) on GB300.

One step = the whole hot path on one synthetic problem: strong recursive
skeletonization factorization of A = I + w K (tree, per-level ID,
elimination and Schur updates, top-block LU) followed by the solve of
A x = b for 4 right-hand sides to a 1e-10 relative residual by GMRES-based
iterative refinement (FP64 residuals, the factor as preconditioner).

Default workload: 2D Laplace, 512 x 512 grid of cell centres in the unit
square (N = 262144), A = I + h^2 K with K = -log|x-y| / (2 pi), leaf <= 64,
eps = 1e-6, four N(0,1) right-hand sides (seeds 1..4), mixed precision
(FP32 factor, FP64 refinement).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--prec mixed|fp64] [--no-fp64-compare] [--no-cpu-baseline]

Under torchrun each rank runs an independent replica (the single problem
does not shard; there is no collective on the data path).  Rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1609_08130_gb300 import inputs  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "RS-S factor+solve points/s at eps=1e-6, mixed/batched vs FP64 GPU"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return dict(hbm=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]), src="measured",
                    sm_mhz=float(p.get("sm_max_mhz", 2070.0)))
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, src="fallback", sm_mhz=2070.0)


# kernel classes bound by moving bytes; the others (ID, elimination, top LU)
# by FP32 / FP64 arithmetic latency and throughput
HBM_CLASSES = {"schur", "sweep", "assemble", "permute", "top_solve", "refine_op"}


def class_roofline(cls: str, d: dict, peaks: dict, prec: str):
    """Achieved rate of one kernel class against its bound: its algorithmic
    bytes (HBM-bound classes) or flops (the others) over its CUDA-event time
    in the timed steps; None for a class that took no time."""
    s = d["ms"] / 1e3
    if s <= 0:
        return None
    if cls in HBM_CLASSES:
        a = d["bytes"] / s / 1e9
        return {"bound": "hbm", "achieved": a, "peak": peaks["hbm"], "unit": "GB/s", "frac": a / peaks["hbm"]}
    pk = alu_peak_tflops(prec, peaks["sm_mhz"])
    a = d["flops"] / s / 1e12
    return {"bound": "alu", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's figure (all-reduce MAX over the process group);
    x itself with a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_points_per_s(world: int, n_per_rank: int, ms_max: float) -> float:
    """Whole-job throughput: every rank factors and solves its own replica
    of n points; the job takes as long as its slowest rank."""
    return world * n_per_rank / (ms_max / 1e3)


def alu_peak_tflops(prec: str, sm_mhz: float) -> float:
    """Plain-ALU peaks from unit counts and clock: 152 SMs x 128 FP32 lanes
    x 2 flops (FMA) x SM clock for FP32; FP64 at the part's 1.25 TFLOP/s."""
    if prec == "fp64":
        return 1.25
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(name):
    w = inputs.workload(name)
    pts = w["pts"]
    b = inputs.rhs(w["rhs_seeds"][0], len(pts), len(w["rhs_seeds"]))
    return w, pts, b


def cpu_oracle_sample(name: str, min_seconds: float = 10.0, max_reps: int = 30):
    """The CPU oracle as it stands, single-threaded, on a bounded sample of the
    workload: the 64x64-grid instance (N = 4096) of the same 2D Laplace
    problem (same kernel, leaf, eps, four right-hand sides), factor + solve,
    repeated until min_seconds have elapsed."""
    import oracle
    oracle.build()
    w = inputs.workload("laplace2d_grid64")
    pts = w["pts"]
    b = inputs.rhs(1, len(pts), 4)
    t0 = time.perf_counter()
    reps = 0
    while True:
        f = oracle.Factor(oracle.Tree(pts, w["leaf"]), w["kind"], w["eps"])
        f.solve(b)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return {"value": reps * len(pts) / el, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x factor+solve(4 rhs) of the 64x64-grid instance (N=4096) of the same "
                      f"2D Laplace workload, leaf 64, eps 1e-6; {el:.1f} s single-threaded"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on rank 0 only."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = inputs.workload("laplace2d_grid64")
    pts = w["pts"]
    b = inputs.rhs(1, len(pts), 4)

    def step():
        f = oracle.Factor(oracle.Tree(pts, w["leaf"]), w["kind"], w["eps"])
        f.solve(b)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps * len(pts) / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "laplace2d_grid512", "sample": "64x64-grid instance (N=4096)", "leaf": 64,
                   "eps": 1e-6, "nrhs": 4},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} x factor+solve(4 rhs) on the 64x64-grid instance"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per launch of a kernel class, from one ncu
# capture of the full-size default workload (profiles/id_dram_laplace2d_grid512.md),
# valid only for the kernel source it was taken on.
NCU_TRAFFIC = {
    "id": {"bytes_per_launch": 21.26e6,
           "kernels_sha256": "c540d7ed44205238c4e7886ec0fb09e3be22abda77a08ae98692f96e39219395"},
}


def ncu_traffic(cls):
    import hashlib
    t = NCU_TRAFFIC.get(cls)
    if t is None:
        return None
    src = os.path.join(ROOT, "paper_1609_08130_gb300", "csrc", "kernels.cu")
    with open(src, "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != t["kernels_sha256"]:
            return None
    return t["bytes_per_launch"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="laplace2d_grid512")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1609_08130_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    w, pts_h, b_h = workload(args.workload)
    n = len(pts_h)
    nrhs = b_h.shape[0]
    prec = pkg.MIXED if args.prec == "mixed" else pkg.FP64
    pts = torch.from_numpy(pts_h).cuda()
    b = torch.from_numpy(np.ascontiguousarray(b_h)).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # first-kind workloads carry their diagonal and off-diagonal weight
    matrix = {k: w[k] for k in ("diag", "weight") if k in w}

    def step(profile=False, p=prec):
        f = pkg.Factorization(pts, w["kind"], w["eps"], leaf=w["leaf"], prec=p, profile=profile, **matrix)
        x, iters, rel = f.solve_refined(b, tol=args.tol, maxit=10)
        return f, x, iters, rel

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    # timed region: K steps, each with the L2 flushed before it
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    prof_tot = {}
    launches0 = pkg.kernel_launches()
    rels, its = [], []
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        f, x, iters, rel = step(profile=True)
        ev[k][1].record(stream)
        rels.append(rel)
        its.append(iters)
        for cls, d in f.profile().items():
            t = prof_tot.setdefault(cls, dict(launches=0, ms=0.0, bytes=0.0, flops=0.0))
            for key in t:
                t[key] += d[key]
        del f
    barrier()
    launches = pkg.kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), dist, "cuda")
    value = job_points_per_s(world, n, ms)

    # end to end through the public API with host buffers
    pts_pin = torch.from_numpy(pts_h).pin_memory()
    b_pin = torch.from_numpy(np.ascontiguousarray(b_h)).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    e2e_ms = []
    for k in range(max(2, min(args.steps, 3))):
        flush.zero_()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        pd = pts_pin.to("cuda", non_blocking=True)
        bd = b_pin.to("cuda", non_blocking=True)
        fe = pkg.Factorization(pd, w["kind"], w["eps"], leaf=w["leaf"], prec=prec, **matrix)
        xe, _, _ = fe.solve_refined(bd, tol=args.tol, maxit=10)
        x_pin.copy_(xe, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(t0.elapsed_time(t1))
        del fe
    e2e_ms = max_over_ranks(float(np.mean(e2e_ms)), dist, "cuda")

    # plain FP64 GPU form on the same GPU, same final accuracy
    fp64 = None
    if not args.no_fp64_compare and prec == pkg.MIXED:
        step(p=pkg.FP64)
        t64 = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, it64, rel64 = step(p=pkg.FP64)
            c.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(c))
        fp64 = {"value": n / (np.mean(t64) / 1e3), "ms_per_step": float(np.mean(t64)), "relres": rel64,
                "iters": it64}

    peaks = load_peaks()
    tuned = [[e["elem_bytes"], e["width"], e["phase_class"], e["tpc"], e["groups"], e["ctas"]]
             for e in pkg.autotune_table()]
    # dominant kernel class by time inside the timed region
    gpu_classes = {k: v for k, v in prof_tot.items() if not k.startswith("host_")}
    dom = max(gpu_classes.items(), key=lambda kv: kv[1]["ms"])
    cls, d = dom
    roof = class_roofline(cls, d, peaks, args.prec)
    roof["traffic"] = ncu_traffic(cls)
    roof["kernel"] = cls
    roof["peak_source"] = ("of measured (MEASURED_PEAKS.json)" if roof["bound"] == "hbm" and peaks["src"] == "measured"
                           else "derived from unit counts and max SM clock" if roof["bound"] == "alu"
                           else "of fallback")
    gsum = max(sum(t["ms"] for t in gpu_classes.values()), 1e-9)
    roof["classes"] = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps, "share": v["ms"] / gsum,
                           "roofline": class_roofline(k, v, peaks, args.prec)}
                       for k, v in sorted(gpu_classes.items(), key=lambda kv: -kv[1]["ms"])}
    roof["host_ms_per_step"] = {k: v["ms"] / args.steps for k, v in prof_tot.items() if k.startswith("host_")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == pkg.MIXED else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": n, "dim": w["dim"], "leaf": w["leaf"], "eps": w["eps"],
                       "nrhs": nrhs, "refine_tol": args.tol, "refine": "gmres-ir f64",
                       "factor": "f32" if prec == pkg.MIXED else "f64", "parallelism": "replicas",
                       "l2": "flushed between steps", "max_relres": float(max(rels)),
                       "inner_iters": int(max(its))},
            "e2e": {"value": job_points_per_s(world, n, e2e_ms), "unit": "points/s",
                    "h2d_bytes_per_step": int(pts_h.nbytes + b_h.nbytes), "d2h_bytes_per_step": int(b_h.nbytes)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "clocks": clk,
            "gpu_launches": int(launches),
            "autotune": {"id_shapes": tuned, "fields": ["element bytes", "box width class", "phase-size class",
                                                        "threads per column", "fold groups", "CTAs per box"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
