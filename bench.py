"""Benchmark: RS-S factor + refined solve throughput (points/s) on GB300.

One step = the whole hot path on one synthetic workload: the strong
recursive skeletonization factorization of A = I + w K (tree, per-level ID,
elimination and Schur updates, top-block LU) followed by the solve of
A x = b to a 1e-10 relative residual by GMRES-based iterative refinement
(FP64 residuals, the factor as preconditioner).

Workloads (--workload):
  laplace2d_grid512    default: 2D Laplace, 512 x 512 grid of cell centres in
                       the unit square (N = 262144), A = I + h^2 K with
                       K = -log|x-y| / (2 pi), leaf <= 64, eps = 1e-6, four
                       N(0,1) right-hand sides (seeds 1..4)
  laplace2d_grid64     the same at 64 x 64 (N = 4096), one right-hand side
  laplace2d_grid256    the same at 256 x 256 (N = 65536), four right-hand
                       sides (a profiling size)
  laplace3d_grid32     3D Laplace, 32^3 grid (N = 32768), A = I + h^3/(4 pi r),
                       eps = 1e-3, one right-hand side
  laplace2d_batched256 256 independent 2D problems, N_p uniform in
                       [1024, 16384], iid uniform points, w = 1/N_p, eps =
                       1e-6, one right-hand side per problem (seed 2000 + p),
                       one handle (one launch per level and colour over all)
  laplace3d_grid64     3D Laplace, 64^3 grid (N = 262144), eps = 1e-6; with
                       --mlp the factor storage is presized by the rank-
                       proposal network trained on the boxes of the 64^2 2D
                       grid, the 512^2 2D grid and the 32^3 3D grid

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--prec mixed|fp64] [--mlp] [--colours 2|3]
                    [--no-fp64-compare] [--no-cpu-baseline]

The timed steps run without per-launch events; a separate profiled pass of
the same steps afterwards gives every kernel class's CUDA-event time for the
roofline figures.  Under torchrun each rank runs an independent replica (a
single problem does not shard; there is no collective on the data path).
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mproc
import os
import platform
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
WORKLOADS = ["laplace2d_grid512", "laplace2d_grid64", "laplace2d_grid256", "laplace3d_grid32",
             "laplace2d_batched256", "laplace3d_grid64"]


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
HBM_CLASSES = {"schur", "sweep", "assemble", "permute", "top_solve"}
# classes whose arithmetic is FP64 whatever the factor's precision: the
# residual operator (FFT convolution or direct sum in FP64)
FP64_CLASSES = {"refine_op"}


def class_roofline(cls: str, d: dict, peaks: dict, prec: str):
    """Achieved rate of one kernel class against its bound: its algorithmic
    bytes (HBM-bound classes) or flops (the others) over its CUDA-event time;
    None for a class that took no time."""
    s = d["ms"] / 1e3
    if s <= 0:
        return None
    if cls in HBM_CLASSES:
        a = d["bytes"] / s / 1e9
        return {"bound": "hbm", "achieved": a, "peak": peaks["hbm"], "unit": "GB/s", "frac": a / peaks["hbm"]}
    pk = alu_peak_tflops("fp64" if cls in FP64_CLASSES else prec, peaks["sm_mhz"], peaks.get("sms", 152))
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


def alu_peak_tflops(prec: str, sm_mhz: float, sms: int = 152) -> float:
    """Plain-ALU peaks from unit counts and clock: SMs x 128 FP32 lanes x 2
    flops (FMA) x SM clock for FP32; FP64 at the part's 1.25 TFLOP/s."""
    if prec == "fp64":
        return 1.25
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


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


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def make_workload(name: str) -> dict:
    """Points (a list of problems), right-hand sides (nrhs, sum N), kernel,
    eps, leaf and the matrix' diagonal and weight where they differ from the
    second-kind default."""
    if name == "laplace2d_batched256":
        sizes = inputs.batched_sizes(256)
        pts = [inputs.batched_problem(p, int(nn)) for p, nn in enumerate(sizes)]
        b = np.concatenate([inputs.normal(2000 + p, int(nn)) for p, nn in enumerate(sizes)])[None, :]
        return dict(name=name, pts=pts, b=b, dim=2, kind=0, eps=1e-6, leaf=64, batched=True, matrix={})
    w = inputs.workload(name)
    pts = w["pts"]
    b = inputs.rhs(w["rhs_seeds"][0], len(pts), len(w["rhs_seeds"]))
    matrix = {k: w[k] for k in ("diag", "weight") if k in w}
    return dict(name=name, pts=[pts], b=b, dim=w["dim"], kind=w["kind"], eps=w["eps"], leaf=w["leaf"],
                batched=False, matrix=matrix)


def oracle_sample(name: str) -> dict:
    """The bounded instance of a workload the CPU oracle (dense FP64 state,
    O(N^2) memory) is timed on: the same kernel, eps, leaf and right-hand
    sides per point on a problem of at most 4096 points."""
    if name.startswith("laplace2d_grid"):
        pts = inputs.grid_points(64, 2)
        nrhs = 1 if name == "laplace2d_grid64" else 4
        return dict(pts=[pts], kind=0, eps=1e-6, nrhs=nrhs,
                    desc=f"64x64-grid instance (N=4096) of the 2D workload, leaf 64, eps 1e-6, {nrhs} rhs")
    if name.startswith("laplace3d_grid"):
        eps = 1e-3 if name == "laplace3d_grid32" else 1e-6
        return dict(pts=[inputs.grid_points(16, 3)], kind=1, eps=eps, nrhs=1,
                    desc=f"16^3-grid instance (N=4096) of the 3D workload, leaf 64, eps {eps:g}, 1 rhs")
    if name == "laplace2d_batched256":
        sizes = inputs.batched_sizes(256)
        keep = [p for p, nn in enumerate(sizes) if nn <= 4096][:2]
        return dict(pts=[inputs.batched_problem(p, int(sizes[p])) for p in keep], kind=0, eps=1e-6, nrhs=1,
                    desc=f"problems {keep} of the batched workload (N = {[int(sizes[p]) for p in keep]}), "
                         "leaf 64, eps 1e-6, 1 rhs each")
    raise KeyError(name)


def _oracle_job(args):
    """One oracle factor + solve of every problem of a sample (a worker)."""
    pts_list, kind, eps, nrhs, until = args
    import oracle
    done = 0
    pts_done = 0
    while True:
        for pts in pts_list:
            f = oracle.Factor(oracle.Tree(pts, 64), kind, eps)
            f.solve(inputs.rhs(1, len(pts), nrhs))
            pts_done += len(pts)
        done += 1
        if until is None or time.perf_counter() >= until:
            return done, pts_done


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_oracle_baseline(name: str, seconds: float = 8.0) -> dict:
    """The CPU oracle as it stands on a bounded sample of the workload: first
    on one core, then one oracle process per host core, each repeating the
    sample for about `seconds`.  value = points/s with all cores."""
    import oracle
    oracle.build()
    S = oracle_sample(name)
    job = (S["pts"], S["kind"], S["eps"], S["nrhs"])
    t0 = time.perf_counter()
    reps1, pts1 = _oracle_job(job + (t0 + seconds,))
    one = pts1 / (time.perf_counter() - t0)
    cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [job + (None,)] * cores)  # start-up and first touch, untimed
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, [job + (t0 + seconds,)] * cores)
        el = time.perf_counter() - t0
    allc = sum(p for _, p in res) / el
    return {"value": allc, "unit": "points/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": cores, "single_core_value": one,
            "sample": f"factor+solve of the {S['desc']}: {reps1} repetitions on one core "
                      f"({one:.0f} points/s), then {cores} oracle processes (one per core) for "
                      f"{el:.1f} s ({sum(r for r, _ in res)} repetitions)"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on rank 0 only, one oracle
    process per host core; a step = one factor + solve of the workload's
    bounded sample in every process."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    S = oracle_sample(args.workload)
    job = (S["pts"], S["kind"], S["eps"], S["nrhs"], None)
    cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_job, [job] * cores)
        t0 = time.perf_counter()
        pts = 0
        for _ in range(args.steps):
            pts += sum(p for _, p in pool.map(_oracle_job, [job] * cores))
        el = time.perf_counter() - t0
    value = pts / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample": S["desc"], "eps": S["eps"], "nrhs": S["nrhs"]},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": cores,
                         "sample": f"{args.steps} steps, each a factor+solve of the {S['desc']} in each of "
                                   f"{cores} oracle processes"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per launch of a kernel class from an ncu capture,
# valid only for the kernel source it was taken on (sha-256 of kernels.cu).
NCU_TRAFFIC = {
    # the ID's DRAM bytes per launch of the 512^2 step: an ncu capture of
    # every ID launch of the 256^2 step, scaled by box count per depth
    "id": {"bytes_per_launch": 56.5e6,
           "kernels_sha256": "99f814ed756e6b283225728feb3d05a00f1215091221cac1355706e1481e9379"},
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


def train_proposal(pkg, torch):
    """The rank-proposal network trained on the boxes of the 64^2 and 512^2
    2D grids (eps 1e-6) and the 32^3 3D grid (eps 1e-3): features and the
    rank fraction k/b of every box of FP32 factorizations."""
    Xs, ys = [], []
    for name in ("laplace2d_grid64", "laplace2d_grid512", "laplace3d_grid32"):
        w = inputs.workload(name)
        f = pkg.Factorization(torch.from_numpy(w["pts"]).cuda(), w["kind"], w["eps"], leaf=w["leaf"], prec=pkg.MIXED)
        feat, rank = f.box_features()
        st = f.stats()
        keep = st["b"] > 0
        Xs.append(feat[keep])
        ys.append((rank[keep] / st["b"][keep]).astype(np.float32))
        del f
    m = pkg.Mlp(seed=7)
    loss = m.train(np.concatenate(Xs), np.concatenate(ys), iters=3000, lr=3e-3)
    return m, {"train_boxes": int(sum(len(y) for y in ys)), "train_loss": loss}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="laplace2d_grid512", choices=WORKLOADS)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--mlp", action="store_true", help="presize factor storage by the trained rank proposal")
    ap.add_argument("--colours", type=int, default=2, choices=[2, 3],
                    help="colours per dimension of the level schedule: the paper's 2 (default) or 3")
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
    W = make_workload(args.workload)
    pts_h, b_h = W["pts"], np.ascontiguousarray(W["b"])
    n = int(sum(len(p) for p in pts_h))
    nrhs = b_h.shape[0]
    prec = pkg.MIXED if args.prec == "mixed" else pkg.FP64
    pts = [torch.from_numpy(p).cuda() for p in pts_h]
    b = torch.from_numpy(b_h).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    mlp, mlp_info = (None, None)
    if args.mlp:
        mlp, mlp_info = train_proposal(pkg, torch)

    def factor(P, p=prec, profile=False, use_mlp=True):
        kw = dict(leaf=W["leaf"], prec=p, profile=profile, mlp=mlp if use_mlp else None,
                  flags=pkg.rss.FLAG_COLOUR_2D if args.colours == 2 else 0, **W["matrix"])
        if W["batched"]:
            return pkg.Factorization.batched(P, W["kind"], W["eps"], **kw)
        return pkg.Factorization(P[0], W["kind"], W["eps"], **kw)

    def step(p=prec, profile=False, use_mlp=True):
        f = factor(pts, p, profile, use_mlp)
        x, iters, rel = f.solve_refined(b, tol=args.tol, maxit=10)
        return f, x, iters, rel

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    # timed region: K steps, each with the L2 flushed before it, no
    # per-launch events
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = pkg.kernel_launches()
    rels, its = [], []
    barrier()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        f, x, iters, rel = step()
        ev[k][1].record(stream)
        rels.append(rel)
        its.append(iters)
        del f
    barrier()
    torch.cuda.nvtx.range_pop()
    launches = pkg.kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), dist, "cuda")
    value = job_points_per_s(world, n, ms)

    # per-kernel-class times: the same steps again with CUDA events around
    # every launch (outside the timed region)
    prof_tot = {}
    for _ in range(args.steps):
        flush.zero_()
        f, _, _, _ = step(profile=True)
        for cls, d in f.profile().items():
            t = prof_tot.setdefault(cls, dict(launches=0, ms=0.0, bytes=0.0, flops=0.0))
            for key in t:
                t[key] += d[key]
        del f
    torch.cuda.synchronize()

    # end to end through the public API with host buffers
    pts_pin = [torch.from_numpy(p).pin_memory() for p in pts_h]
    b_pin = torch.from_numpy(b_h).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    e2e_ms = []
    for k in range(max(2, min(args.steps, 3))):
        flush.zero_()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        pd = [p.to("cuda", non_blocking=True) for p in pts_pin]
        bd = b_pin.to("cuda", non_blocking=True)
        fe = factor(pd)
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
        step(p=pkg.FP64, use_mlp=False)
        t64 = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, it64, rel64 = step(p=pkg.FP64, use_mlp=False)
            c.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(c))
        fp64 = {"value": n / (np.mean(t64) / 1e3), "ms_per_step": float(np.mean(t64)), "relres": rel64,
                "iters": it64}

    # the rank proposal on vs off (same factor; storage and time)
    mlp_cmp = None
    if mlp is not None:
        f_on = factor(pts)
        f_off = factor(pts, use_mlp=False)
        s_on, s_off = f_on.stats(), f_off.stats()
        del f_on, f_off
        t_off = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(use_mlp=False)
            c.record(stream)
            torch.cuda.synchronize()
            t_off.append(a.elapsed_time(c))
        mlp_cmp = dict(mlp_info, ms_per_step_on=ms, ms_per_step_off=float(np.mean(t_off)),
                       reserved_bytes_on=s_on["reserved_bytes"], reserved_bytes_off=s_off["reserved_bytes"],
                       used_bytes=s_on["used_bytes"], same_ranks=bool(np.array_equal(s_on["k"], s_off["k"])),
                       retried=s_on["retried"])

    peaks = load_peaks()
    peaks["sms"] = torch.cuda.get_device_properties(local).multi_processor_count
    tuned = [[e["elem_bytes"], e["width"], e["phase_class"], e["tpc"], e["groups"], e["ctas"], e["rows"]]
             for e in pkg.autotune_table()]
    tuned_elim = [[e["elem_bytes"], e["width"], e["phase_class"], e["split"], e["ctas"]]
                  for e in pkg.autotune_elim_table()]
    # dominant kernel class by time in the profiled pass
    gpu_classes = {k: v for k, v in prof_tot.items() if not k.startswith("host_")}
    dom = max(gpu_classes.items(), key=lambda kv: kv[1]["ms"])
    cls, d = dom
    roof = class_roofline(cls, d, peaks, args.prec)
    roof["traffic"] = ncu_traffic(cls)
    roof["kernel"] = cls
    roof["peak_source"] = ("of measured (MEASURED_PEAKS.json)" if roof["bound"] == "hbm" and peaks["src"] == "measured"
                           else f"derived from {peaks['sms']} SMs x 128 FP32 lanes x 2 x max SM clock"
                           if roof["bound"] == "alu" else "of fallback")
    roof["timing"] = "CUDA events around every launch, in a profiled pass of the same steps after the timed region"
    gsum = max(sum(t["ms"] for t in gpu_classes.values()), 1e-9)
    roof["classes"] = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps, "share": v["ms"] / gsum,
                           "roofline": class_roofline(k, v, peaks, args.prec)}
                       for k, v in sorted(gpu_classes.items(), key=lambda kv: -kv[1]["ms"])}
    roof["host_ms_per_step"] = {k: v["ms"] / args.steps for k, v in prof_tot.items() if k.startswith("host_")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == pkg.MIXED else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": n, "problems": len(pts_h), "dim": W["dim"],
                       "leaf": W["leaf"], "eps": W["eps"], "nrhs": nrhs, "refine_tol": args.tol,
                       "refine": "gmres-ir f64", "factor": "f32" if prec == pkg.MIXED else "f64",
                       "rank_proposal": bool(args.mlp), "colours_per_level": args.colours ** W["dim"],
                       "parallelism": "replicas",
                       "l2": "flushed between steps", "max_relres": float(max(rels)),
                       "inner_iters": int(max(its))},
            "e2e": {"value": job_points_per_s(world, n, e2e_ms), "unit": "points/s",
                    "h2d_bytes_per_step": int(sum(p.nbytes for p in pts_h) + b_h.nbytes),
                    "d2h_bytes_per_step": int(b_h.nbytes)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "mlp": mlp_cmp,
            "clocks": clk,
            "gpu_launches": int(launches),
            "autotune": {"id_shapes": tuned, "fields": ["element bytes", "box width class", "phase-size class",
                                                        "threads per column", "fold groups", "CTAs per box",
                                                        "panel rows per thread (units of 32 FP32 rows)"],
                         "elim_shapes": tuned_elim,
                         "elim_fields": ["element bytes", "box width class", "phase-size class",
                                         "E and G in a separate product kernel", "CTAs per box"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
