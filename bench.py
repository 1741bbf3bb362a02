"""Benchmark of the GB300 RandomizedNNLS hot path (sketch + Lawson-Hanson solve).

One step = one pass of the whole path over one batch: sample the rows
(Philox), sketch [A | b] (sign flip + Walsh-Hadamard + sampled-row combine),
Gram of the sketch, Lawson-Hanson NNLS.  Default workload (5, the largest
that fits one GPU): 512 uneven term-document-like FP32 instances, n from
2^14 to 2^20, d from 16 to 200, 58.7 GB of inputs resident in HBM (far
larger than the 129 MB L2, so no flush between steps), one CUDA graph per
step.  Workloads 1-4 are single problems (--config).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
instance (weak scaling, no collective on the data path); the reported value
is all ranks' solves divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
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

import workloads  # noqa: E402

METRIC = "RandNNLS solves/s & SRHT GB/s vs ~8 TB/s HBM at residual ratio <=1.01"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser(description="RandomizedNNLS throughput and sketch roofline on synthetic workloads "
                                             "(one JSON line on stdout)")
    ap.add_argument("--gpus", type=int, default=1, help="GPUs (one process each under torchrun)")
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for workload 5, 1000 for the others)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default: 5 / 20)")
    ap.add_argument("--config", type=int, default=None, choices=[1, 2, 3, 4, 5],
                    help="workload: 1 4096x20 FP64 r=512; 2 2^20x64 r=4096; 3 2^22x128 r=8192; "
                         "4 2^20x100 with 256 targets r=4096; 5 (default) 512 uneven instances, the largest")
    ap.add_argument("--instances", type=int, default=None, help="workload 5: instance count (default 512)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"],
                    help="reference: the FP64 oracle on the host cores instead of the GPU library")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (host inputs copied in, x read back)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the oracle on the host cores")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's residual ratio and sketch error beside the GPU's")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="host-core time budget of the CPU baseline")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="run each step's sketch and solve back to back on one stream")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="end-to-end leg: streams the host-to-device copy of A is split over")
    ap.add_argument("--density-sweep", action="store_true",
                    help="the density experiment of Sec. 4.2: mean ||A x~ - b|| / ||A x_opt - b|| per density and r")
    ap.add_argument("--sweep-problems", type=int, default=100, help="density sweep: problems per density")
    ap.add_argument("--boost", type=int, default=0,
                    help="k > 0: time repeated RandomizedNNLS (k runs, best full residual kept) on workload 2 or 3")
    ap.add_argument("--no-sketch-priority", dest="sketch_priority", action="store_false",
                    help="pipelined mode: give the sketch stream the default priority")
    ap.add_argument("--solve-after-plan", type=int, default=None, choices=[0, 1],
                    help="pipelined mode: 1 enqueues each solve after the next step's plan launch, 0 right after "
                         "its own sketch (default: 1 for workload 3, whose Grams and solves otherwise delay the "
                         "plan, 0 elsewhere)")
    ap.add_argument("--sketch-streams", type=int, default=1,
                    help="pipelined mode: steps alternate over this many sketch streams")
    ap.add_argument("--solve-streams", type=int, default=3,
                    help="solve streams when pipelined (each solve runs in one block)")
    ap.add_argument("--no-tune", action="store_true",
                    help="workload 5: skip the autotuner (launch-shape knobs at their built-in defaults)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x2"],
                    help="sketch precision: fp32 (both Hadamard factors in FP32 registers) or bf16x2 (the first "
                         "64-point factor on the tensor cores, values split into hi + lo BF16, FP32 accumulation)")
    ap.add_argument("--csc", action="store_true",
                    help="workload 2 or 3 with A held in compressed sparse columns (rnnls_sketch_csc); "
                         "one stream, sketch + solve per step")
    ap.add_argument("--free-sms", type=int, default=None,
                    help="pipelined mode: SMs the sketch leaves to the solves (default: 5 + one per solve stream; "
                         "a Gram CTA needs a whole SM's shared memory)")
    args = ap.parse_args()
    if args.config is None:
        args.config = 2 if (args.boost > 0 or args.csc) else 5
    if args.steps is None:
        args.steps = 20 if args.config == 5 else 1000
    if args.warmup is None:
        args.warmup = 5 if args.config == 5 else 20
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base: int, rank: int, ws: int) -> int:
    """Seed of this rank's instance: each rank solves its own problem (weak scaling)."""
    return base + 1000 * rank if ws > 1 else base


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks (the slowest rank sets the whole job's time)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_desc(cfg: int, p) -> dict:
    names = {1: "c1: A 4096x20 uniform FP64, r=512", 2: "c2: A 2^20x64 term-doc FP32, r=4096",
             3: "c3: A 2^22x128 term-doc FP32, r=8192",
             4: "c4: A 2^20x100 term-doc FP32, 256 targets sharing one sketch, r=4096"}
    return {"workload": names[cfg], "n": int(p.n), "d": int(p.d), "r": int(p.r), "sampling": "iid",
            "l2": "inputs larger than L2 (no flush)" if p.A.nbytes > 129e6 else "inputs in L2 (small case)",
            "parallelism": "independent instance per GPU"}


def algorithmic_bytes(p, s: int) -> int:
    # one read of [A | b], one write of the sketch, the sampled-row indices
    return int(p.n * (p.d + 1) * s + p.r * (p.d + 1) * s + 4 * p.r)


def measured_hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    for rel in ("paper_0812_4547_gb300/csrc/sketch.cu", "paper_0812_4547_gb300/csrc/common.cuh",
                "paper_0812_4547_gb300/csrc/kernels.h"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel is unchanged since."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)[kernel][workload]
        if rec.get("source_sha256") == source_hash():
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs (read-only query)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[1]), float(parts[2]), parts[4:8]))
            except Exception:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        use = inside if inside else sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:2]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median([r[1] for r in use]) if use else None,
                "sm_max_mhz": max([r[2] for r in use]) if use else None,
                "reasons": reasons, "samples_in_region": len(inside)}


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------
def run_reference(args, cfg: int):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    if cfg == 5:
        run_reference_batch(args, threads)
        return
    p = multi_problem(rank_seed(workloads.CONFIGS[4]["seed"], 0, 1)) if cfg == 4 else workloads.problem(cfg)
    for i in range(args.warmup):
        oracle.randomized_nnls(p.A, p.b, p.r, seed=i, nthreads=threads)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.randomized_nnls(p.A, p.b, p.r, seed=args.warmup + i, nthreads=threads)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded term-document-like stand-in for TechTC300)",
           "config": workload_desc(cfg, p),
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle",
                            "sample": f"{args.steps} full solves of the workload (FP64 C oracle, OpenMP over columns)"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_reference_batch(args, threads: int):
    """The reference arm on workload 5: the FP64 oracle on the host cores;
    one step solves the batch's whole spread sample (32 of the 512 instances,
    the ones the GPU arm solves, built on the device and copied to the host)."""
    import torch

    import oracle

    c5 = workloads.CONFIGS[5]
    shapes = workloads.batch_shapes(count=args.instances, seed=c5["seed"])
    sample = batch_sample(len(shapes))
    dev = torch.device("cuda", 0)
    built = device_batch(shapes, c5["seed"], dev, only=sample)
    host = [(A.cpu().numpy(), b.cpu().numpy(), r) for A, b, r in built]
    del built
    def step():
        for i, (A, b, r) in zip(sample, host):
            oracle.randomized_nnls(A, b, r, seed=i, nthreads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = args.steps * len(sample) / dt
    count = len(shapes)
    desc = (f"each step the spread sample of {len(sample)} instances (every {max(1, count // 32)}-th of {count}), "
            f"FP64 C oracle, OpenMP over columns")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (term-document-like, generated on the device, copied to the host)",
           "config": {"workload": f"c5: {count} uneven instances, n 2^U[14,20], d U{{16..200}}, r pow2 of 8(d+1)ln n",
                      "instances": count, "sampling": "iid", "parallelism": "host cores"},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle",
                            "cpu_model": cpu_model(), "sample": desc},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


class MultiProblem:
    """Workload 4 (A shared by nrhs targets B) with the fields the single-target helpers read."""

    def __init__(self, A, Bm, r):
        self.A, self.B, self.r = A, Bm, r
        self.b = Bm[:, 0]
        self.n, self.d = A.shape
        self.nrhs = Bm.shape[1]


def multi_problem(seed: int) -> MultiProblem:
    A, Bm, _, r = workloads.multi_rhs(seed=seed)
    return MultiProblem(A, Bm, r)


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def cpu_baseline(p, seconds: float) -> dict:
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.randomized_nnls(p.A, p.b, p.r, seed=done, nthreads=threads)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    out = {"value": done / dt, "unit": "solves/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"{done} full solves of the workload in {dt:.1f} s (FP64 C oracle, OpenMP over columns)"}
    # the same oracle on one core, when a solve fits in a few seconds there
    if dt / done * threads <= 6.0:
        t1 = time.perf_counter()
        one = 0
        while True:
            oracle.randomized_nnls(p.A, p.b, p.r, seed=one, nthreads=1)
            one += 1
            if time.perf_counter() - t1 >= seconds / 3:
                break
        d1 = time.perf_counter() - t1
        out["single_thread"] = {"value": one / d1, "unit": "solves/s", "cores": 1,
                                "sample": f"{one} full solves in {d1:.1f} s on one core"}
    return out


def prec_flag(args) -> int:
    """The library's RNNLS_PREC_* value for --prec."""
    return 2 if getattr(args, "prec", "fp32") == "bf16x2" else 0


def prec_dtype(args) -> str:
    return "f32" if prec_flag(args) == 0 else "bf16x2 split (hi+lo) on tensor cores, f32 accumulation"


def oracle_ratio(A, b, r: int, seed: int, instance: int, limit: float = 1.2e10):
    """The FP64 oracle's residual ratio of Theorem 1 on the same data and seed
    (its own sketch and Lawson-Hanson, then its exact NNLS on the full A), or
    None when the exact solve (O(n d^2) on the host) is above `limit`."""
    n, d = A.shape
    if n * d * d > limit:
        return None
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    x_t, _ = oracle.randomized_nnls(A, b, r, seed=seed, instance=instance, nthreads=threads)[:2]
    x_o, _ = oracle.exact_nnls(A, b)
    return float(oracle.residual_sq(A, b, x_t) / oracle.residual_sq(A, b, x_o))


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    cfg = args.config
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl")
    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    dev = torch.device("cuda", local)
    base = workloads.CONFIGS[cfg]["seed"]
    if prec_flag(args) and (cfg in (1, 4) or args.boost > 0 or args.density_sweep or args.csc):
        raise SystemExit("--prec bf16x2 applies to workloads 2, 3 and 5 (dense FP32 sketches)")
    if cfg in (4, 5) or args.boost > 0 or args.density_sweep or args.csc:
        if args.density_sweep:
            run_density(args, ws, rank, local, dev)
        elif args.csc:
            run_csc(args, ws, rank, local, dev)
        elif args.boost > 0:
            run_boost(args, ws, rank, local, dev)
        else:
            (run_multi if cfg == 4 else run_batch)(args, ws, rank, local, dev)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    p = workloads.problem(cfg, seed=rank_seed(base, rank, ws))
    f64 = cfg == 1
    dt_np = np.float64 if f64 else np.float32
    tdt = torch.float64 if f64 else torch.float32
    elt = 8 if f64 else 4
    if f64 and prec_flag(args):
        raise SystemExit("--prec bf16x2 needs FP32 data (workloads 2-5)")
    pf = prec_flag(args)
    A_host = torch.from_numpy(np.ascontiguousarray(p.A.astype(dt_np).T)).pin_memory()
    b_host = torch.from_numpy(np.asarray(p.b, dtype=dt_np)).pin_memory()
    A = A_host.to(dev).t()
    b = b_host.to(dev)
    r = p.r
    pipeline = not args.no_pipeline
    # the sketch of step i+1 overlaps the solves of earlier steps: one sketch
    # stream, `nsolve` solve streams (each solve is one block on one SM),
    # sketch outputs in nsolve + 1 rotating buffers, ordered by events
    # the sketch stream (the step's critical path) gets the higher stream
    # priority, so that blocks of the concurrent solves yield SMs to its launches
    nsolve = max(1, args.solve_streams) if pipeline else 1
    if pipeline and args.sketch_priority:
        torch.cuda.synchronize(dev)
        s_sketch = torch.cuda.Stream(dev, priority=min(torch.cuda.Stream.priority_range()))
        torch.cuda.set_stream(s_sketch)  # torch's own work (copies, fills) goes there too
    else:
        s_sketch = torch.cuda.current_stream(dev)
    s_solves = [torch.cuda.Stream(dev) for _ in range(nsolve)] if pipeline else [s_sketch]
    ctx = P.Context(local, s_sketch)
    ctx_vs = [P.Context(local, st) for st in s_solves] if pipeline else [ctx]
    # --sketch-streams k: steps alternate over k sketch streams (one context
    # each), so that the rows and plan of step i+1 start on the SMs the sketch
    # of step i releases first
    nsk = max(1, args.sketch_streams) if pipeline else 1
    s_sks = [s_sketch] + [torch.cuda.Stream(dev, priority=s_sketch.priority) for _ in range(nsk - 1)]
    ctx_sks = [ctx] + [P.Context(local, st) for st in s_sks[1:]]
    if pipeline:
        # SMs free of sketch blocks: one per concurrent Lawson-Hanson solve,
        # plus room for the tensor-core Gram CTAs of the solves
        free = args.free_sms if args.free_sms is not None else 5 + nsolve
        for cs in ctx_sks:
            cs.set_sketch_sms(torch.cuda.get_device_properties(local).multi_processor_count - free)
    nbuf = nsolve + nsk if pipeline else 1
    SAs = [torch.empty((p.d, r), dtype=tdt, device=dev).t() for _ in range(nbuf)]
    Sbs = [torch.empty(r, dtype=tdt, device=dev) for _ in range(nbuf)]
    idxs = [torch.empty(r, dtype=torch.int32, device=dev) for _ in range(nbuf)]
    xs = [torch.empty(p.d, dtype=torch.float64, device=dev) for _ in range(nbuf)]
    infos = [torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device=dev) for _ in range(nbuf)]
    sketched = [torch.cuda.Event() for _ in range(nbuf)]
    solved = [torch.cuda.Event() for _ in range(nbuf)]
    used = [False] * nbuf
    SA, Sb, idx, x, info = SAs[0], Sbs[0], idxs[0], xs[0], infos[0]
    x_host = torch.empty(p.d, dtype=torch.float64).pin_memory()

    # --solve-after-plan (pipelined): the solve of step i is enqueued after the
    # sketch call of step i+1 and waits for that call's plan launch, so that
    # its Gram does not hold the SMs the plan needs; it then runs beside the
    # transform (a Gram block fits next to a sketch block)
    after_plan = pipeline and bool(args.solve_after_plan if args.solve_after_plan is not None else cfg == 3)
    plan_ev = None
    if after_plan:
        plan_ev = torch.cuda.Event()
        plan_ev.record(s_sketch)  # creates the CUDA event the contexts record
        for cs in ctx_sks:
            cs.set_plan_event(plan_ev)
    pending = []  # (step, buffer, x_out) whose solve is not enqueued yet

    def enqueue_solve(i: int, k: int, x_out, wait_plan: bool):
        cv, ss = ctx_vs[i % nsolve], s_solves[i % nsolve]
        if pipeline:
            ss.wait_event(sketched[k])
            if wait_plan:
                ss.wait_event(plan_ev)
        cv.solve(SAs[k], Sbs[k], r=r, x=xs[k], info=infos[k])
        if x_out is not None:
            with torch.cuda.stream(ss):
                x_out.copy_(xs[k], non_blocking=True)
        if pipeline:
            solved[k].record(ss)
            used[k] = True

    def step(i: int, A_=None, b_=None, after_sketch=None, x_out=None):
        A_ = A if A_ is None else A_
        b_ = b if b_ is None else b_
        k = i % nbuf
        st, cs = s_sks[i % nsk], ctx_sks[i % nsk]
        if pipeline and used[k]:
            st.wait_event(solved[k])  # the buffer's previous solve has read it
        cs.sketch(A_, b_, r, seed=i, instance=rank, SA=SAs[k], Sb=Sbs[k], idx=idxs[k], want_count=False,
                  prec=pf)
        if after_sketch is not None:
            after_sketch.record(st)
        if pipeline:
            sketched[k].record(st)
        if after_plan:
            if pending:
                enqueue_solve(*pending.pop(), wait_plan=True)
            pending.append((i, k, x_out))
        else:
            enqueue_solve(i, k, x_out, wait_plan=False)

    def drain():
        if pending:
            enqueue_solve(*pending.pop(), wait_plan=False)
        if pipeline:
            for k in range(nbuf):
                if used[k]:
                    s_sketch.wait_event(solved[k])
            for st in s_sks[1:]:
                e = torch.cuda.Event()
                e.record(st)
                s_sketch.wait_event(e)

    stream = s_sketch
    for i in range(args.warmup):
        step(i)
    drain()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.15)
    for cs in ctx_sks:
        B.rnnls_profile_begin(cs.handle, 16 * args.steps + 64)
    if pipeline:
        for cv in ctx_vs:
            B.rnnls_profile_begin(cv.handle, 16 * args.steps + 64)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.time()
    ev0.record(stream)
    for st in s_sks[1:]:
        st.wait_event(ev0)
    for i in range(args.steps):
        step(args.warmup + i)
    drain()
    ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    prof = {}
    for cx in ctx_sks + (ctx_vs if pipeline else []):
        for k, v in B.rnnls_profile_end(cx.handle).items():
            a = prof.get(k, (0, 0.0))
            prof[k] = (a[0] + v[0], a[1] + v[1])
    clk = clocks.stop(w0, w1)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    if ws > 1:
        torch.distributed.barrier()
    ms_per_step = ms / args.steps
    value = ws * args.steps / (ms / 1e3)

    # e2e: pinned host inputs copied in and the solution read back every step,
    # through the same public calls (pipelined: copies overlap the previous step)
    def seq_step(i: int):
        ctx.sketch(A, b, r, seed=i, instance=rank, SA=SA, Sb=Sb, idx=idx, want_count=False, prec=pf)
        ctx.solve(SA, Sb, r=r, x=x, info=info)

    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, min(args.steps, 200))
    if pipeline:
        # the inputs of step i+1 are copied (own stream, two device buffers)
        # while step i is sketched and solved; x of every step comes back
        # the copy of A is split over a few streams (column ranges) so that
        # several copy engines share it
        ncs = max(1, args.copy_streams)
        copy_ss = [torch.cuda.Stream(dev) for _ in range(ncs)]
        Ad = [A, torch.empty((p.d, p.n), dtype=tdt, device=dev).t()]
        bd = [b, torch.empty_like(b)]
        copied = [[torch.cuda.Event() for _ in range(ncs)] for _ in range(2)]
        freed = [torch.cuda.Event() for _ in range(2)]
        x_hosts = [torch.empty(p.d, dtype=torch.float64).pin_memory() for _ in range(nbuf)]
        cuts = [round(c * p.d / ncs) for c in range(ncs + 1)]
        At_host = A_host.t()

        def e2e_run(nsteps: int):
            for i in range(nsteps):
                k = i % 2
                for c, cs in enumerate(copy_ss):
                    if i >= 2:
                        cs.wait_event(freed[k])  # the sketch two steps back has read this buffer
                    with torch.cuda.stream(cs):
                        Ad[k][:, cuts[c]:cuts[c + 1]].copy_(At_host[:, cuts[c]:cuts[c + 1]], non_blocking=True)
                        if c == 0:
                            bd[k].copy_(b_host, non_blocking=True)
                    copied[k][c].record(cs)
                    s_sks[i % nsk].wait_event(copied[k][c])
                step(i, Ad[k], bd[k], after_sketch=freed[k], x_out=x_hosts[i % nbuf])
            drain()
            torch.cuda.synchronize()

        e2e_run(2)
        e0 = time.perf_counter()
        e2e_run(e2e_steps)
        e_dt = max_over_ranks(time.perf_counter() - e0, dev)
        A.copy_(A_host.t())
        b.copy_(b_host)
    else:
        for i in range(2):
            A.copy_(A_host.t(), non_blocking=True)
            b.copy_(b_host, non_blocking=True)
            seq_step(i)
            x_host.copy_(x, non_blocking=True)
            stream.synchronize()
        e0 = time.perf_counter()
        for i in range(e2e_steps):
            A.copy_(A_host.t(), non_blocking=True)
            b.copy_(b_host, non_blocking=True)
            seq_step(i)
            x_host.copy_(x, non_blocking=True)
            stream.synchronize()
        e_dt = max_over_ranks(time.perf_counter() - e0, dev)
    e2e = {"value": ws * e2e_steps / e_dt, "unit": "solves/s",
           "h2d_bytes_per_step": int(A_host.numel() * elt + b_host.numel() * elt),
           "d2h_bytes_per_step": int(x_host.numel() * 8)}

    # residual ratio of Theorem 1 (evaluation, off the timed path): x~ for
    # seed 0 vs the exact NNLS on the full A, both solved by the library
    seq_step(0)
    x_t = x.clone()
    x_opt, info_opt = ctx.solve(A, b, r=p.n)
    res_t = ctx.residual(A, b, x_t) if not f64 else None
    res_o = ctx.residual(A, b, x_opt) if not f64 else None
    torch.cuda.synchronize()
    ratio = None
    if res_t is not None:
        ratio = float(res_t.item()) / float(res_o.item())
    sketch_info = P.info_dict(info)
    prec_report = None
    if pf:
        # the split-precision sketch of seed 0 against the FP32 mode's and,
        # on rank 0, the FP64 oracle's sketch of the same FP32 bytes
        SA_t, Sb_t = SA.double().clone(), Sb.double().clone()
        ctx.sketch(A, b, r, seed=0, instance=rank, SA=SA, Sb=Sb, idx=idx, want_count=False)
        ctx.solve(SA, Sb, r=r, x=x, info=info)
        torch.cuda.synchronize()
        rel = lambda u, v: float(torch.linalg.vector_norm(u - v) / torch.linalg.vector_norm(v))  # noqa: E731
        prec_report = {"SA_rel_fro_vs_fp32_mode": rel(SA_t, SA.double()), "Sb_rel_fro_vs_fp32_mode": rel(Sb_t, Sb.double()),
                       "x_rel_vs_fp32_mode": rel(x_t, x), "bound": 5e-4}
        if rank == 0 and not args.no_oracle_check:
            import oracle

            oracle.build()
            SA_o, Sb_o, _ = oracle.sketch(p.A.astype(np.float32), p.b.astype(np.float32), r, seed=0, instance=rank,
                                          nthreads=os.cpu_count() or 1)
            SAh, Sbh = SA_t.cpu().numpy(), Sb_t.cpu().numpy()
            prec_report["SA_rel_fro_vs_oracle"] = float(np.linalg.norm(SAh - SA_o) / np.linalg.norm(SA_o))
            prec_report["Sb_rel_fro_vs_oracle"] = float(np.linalg.norm(Sbh - Sb_o) / np.linalg.norm(Sb_o))

    # roofline of the dominant kernel (the chunked sketch), timed live with
    # CUDA events on the launching stream during the timed region
    kname = "sketch_srht_f32" if "sketch_srht_f32" in prof else max(prof, key=lambda k: prof[k][1])
    launches, kms = prof[kname]
    abytes = algorithmic_bytes(p, elt)
    achieved = abytes / (kms / launches / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    sketch_ms = sum(prof.get(k, (0, 0.0))[1] for k in ("sample_rows", "build_plan", "sketch_srht_f32",
                                                        "reduce_partials", "sketch_small", "sketch_f64"))
    wl = workload_desc(cfg, p)
    wl["precision"] = args.prec
    wl["pipeline"] = (f"sketches on {nsk} stream(s) overlap solves on {nsolve} streams ({nbuf} sketch buffers)"
                      if pipeline else "sketch and solve back to back on one stream")
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if f64 else prec_dtype(args),
        "data": "synthetic (seeded term-document-like stand-in for TechTC300)", "config": wl,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic(kname + ("_bf16x2" if pf else ""), wl["workload"]), "kernel": kname,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": abytes, "avg_launch_us": 1e3 * kms / launches,
                     "frac_of_nominal_8tbs": achieved / 8000.0},
        "sketch_gbs": abytes * args.steps / (sketch_ms / 1e3) / 1e9 if sketch_ms > 0 else None,
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "e2e": e2e, "clocks": clk,
        "residual_ratio": ratio, "residual_ratio_le_1.01": (ratio is not None and ratio <= 1.01),
        # the paper's figures plot the unsquared ratio ||A x~ - b|| / ||A x_opt - b||
        "residual_ratio_unsquared": math.sqrt(ratio) if ratio is not None else None,
        "residual_ratio_oracle": (None if args.no_oracle_check or rank != 0 else
                                  oracle_ratio(p.A.astype(dt_np), p.b.astype(dt_np), r, seed=0,
                                               instance=rank)),
        "solve_info": {"status": sketch_info["status"], "passive_count": sketch_info["passive_count"],
                       "outer_iters": sketch_info["outer_iters"], "accurate_mode": sketch_info["accurate_mode"]},
    }
    if prec_report is not None:
        out["precision"] = prec_report
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    elif rank == 0:
        out["cpu_baseline"] = None
    if pipeline:
        for cv in ctx_vs:
            cv.close()
    for cs in ctx_sks[1:]:
        cs.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_multi(args, ws: int, rank: int, local: int, dev):
    """Workload 4: one step sketches [A | B] once and solves all 256 targets on it
    (rnnls_sketch_multi + rnnls_solve_multi); solves/s counts targets."""
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    p = multi_problem(rank_seed(workloads.CONFIGS[4]["seed"], rank, ws))
    n, d, nrhs, r = p.n, p.d, p.nrhs, p.r
    A_host = torch.from_numpy(np.ascontiguousarray(p.A.astype(np.float32).T)).pin_memory()
    B_host = torch.from_numpy(np.ascontiguousarray(p.B.astype(np.float32).T)).pin_memory()
    A = A_host.to(dev).t()
    Bm = B_host.to(dev).t()
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local, stream)
    SA = torch.empty((d, r), dtype=torch.float32, device=dev).t()
    SB = torch.empty((nrhs, r), dtype=torch.float32, device=dev).t()
    idx = torch.empty(r, dtype=torch.int32, device=dev)
    X = torch.empty((nrhs, d), dtype=torch.float64, device=dev).t()
    infos = torch.zeros((nrhs, P.INFO_BYTES), dtype=torch.uint8, device=dev)
    X_host = torch.empty((nrhs, d), dtype=torch.float64).pin_memory()

    def step(i: int):
        ctx.sketch_multi(A, Bm, r, seed=i, instance=rank, SA=SA, SB=SB, idx=idx)
        ctx.solve_multi(SA, SB, r=r, X=X, infos=infos)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.15)
    B.rnnls_profile_begin(ctx.handle, 16 * args.steps + 64)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    prof = B.rnnls_profile_end(ctx.handle)
    clk = clocks.stop(w0, w1)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    if ws > 1:
        torch.distributed.barrier()
    value = ws * args.steps * nrhs / (ms / 1e3)

    # e2e through the public calls: A and B in from pinned host memory, X back, every step
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, min(args.steps, 20))
    for i in range(1 + e2e_steps):
        if i == 1:
            e0 = time.perf_counter()
        A.copy_(A_host.t(), non_blocking=True)
        Bm.copy_(B_host.t(), non_blocking=True)
        step(i)
        X_host.copy_(X.t(), non_blocking=True)
        stream.synchronize()
    e_dt = max_over_ranks(time.perf_counter() - e0, dev)
    e2e = {"value": ws * e2e_steps * nrhs / e_dt, "unit": "solves/s",
           "h2d_bytes_per_step": int((A_host.numel() + B_host.numel()) * 4),
           "d2h_bytes_per_step": int(X_host.numel() * 8)}

    # residual ratios (evaluation, off the timed path) for a few targets:
    # x~ of the shared sketch vs the exact NNLS on the full A
    step(0)
    ratios = []
    for t in (0, nrhs // 2, nrhs - 1):
        bt = Bm[:, t].contiguous()
        x_opt, _ = ctx.solve(A, bt, r=n)
        xt = X[:, t].contiguous()
        ratios.append(float(ctx.residual(A, bt, xt).item()) / float(ctx.residual(A, bt, x_opt).item()))
    tinfo = [P.info_dict(infos[t]) for t in range(nrhs)]
    stat = [f["status"] for f in tinfo]

    kname = "sketch_srht_f32"
    launches, kms = prof[kname]
    abytes = int(4 * n * (d + nrhs) + 4 * r * (d + nrhs) + 4 * r)
    achieved = abytes / (kms / launches / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    wl = {"workload": "c4: A 2^20x100 term-doc FP32, 256 targets sharing one sketch, r=4096", "n": n, "d": d,
          "nrhs": nrhs, "r": r, "sampling": "iid", "l2": "inputs larger than L2 (no flush)",
          "parallelism": "independent instance per GPU",
          "pipeline": "per step: one sketch of [A | B], one shared Gram, 256 Lawson-Hanson blocks"}
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded term-document-like stand-in for TechTC300)",
        "config": wl,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic(kname, wl["workload"]), "kernel": kname,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": abytes, "avg_launch_us": 1e3 * kms / launches},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "e2e": e2e, "clocks": clk,
        "residual_ratio": max(ratios), "residual_ratio_le_1.01": max(ratios) <= 1.01,
        "residual_ratio_target0": ratios[0],
        "residual_ratio_oracle_target0": (None if args.no_oracle_check or rank != 0 else
                                          oracle_ratio(p.A.astype(np.float32), p.B[:, 0].astype(np.float32), r,
                                                       seed=0, instance=rank)),
        "solve_status_nonzero": int(sum(1 for x in stat if x != 0)),
        "lh_accurate_mode_solves": int(sum(1 for f in tinfo if f["accurate_mode"] > 0)),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    elif rank == 0:
        out["cpu_baseline"] = None
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def csc_arrays(A: np.ndarray):
    """Compressed sparse columns of A (FP32): int64 column pointers, int32
    ascending row indices, float32 values."""
    ptr, rows, vals = [0], [], []
    for j in range(A.shape[1]):
        nz = np.flatnonzero(A[:, j])
        rows.append(nz.astype(np.int32))
        vals.append(A[nz, j].astype(np.float32))
        ptr.append(ptr[-1] + nz.size)
    return np.asarray(ptr, np.int64), np.concatenate(rows), np.concatenate(vals)


def run_csc(args, ws: int, rank: int, local: int, dev):
    """Workload 2 or 3 with A in compressed sparse columns: one step =
    rnnls_sketch_csc + rnnls_solve on one stream; e2e copies the column
    pointers, row indices, values and b in and x back every step."""
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    cfg = args.config
    if cfg not in (2, 3):
        raise SystemExit("--csc runs on workload 2 or 3")
    p = workloads.problem(cfg, seed=rank_seed(workloads.CONFIGS[cfg]["seed"], rank, ws))
    A32, b32 = p.A.astype(np.float32), p.b.astype(np.float32)
    ptr_h, rows_h, vals_h = (torch.from_numpy(a).pin_memory() for a in csc_arrays(A32))
    b_h = torch.from_numpy(b32).pin_memory()
    ptr, rows, vals, b = (t.to(dev) for t in (ptr_h, rows_h, vals_h, b_h))
    n, d, r, nnz = p.n, p.d, p.r, int(vals_h.numel())
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local, stream)
    SA = torch.empty((d, r), dtype=torch.float32, device=dev).t()
    Sb = torch.empty(r, dtype=torch.float32, device=dev)
    idx = torch.empty(r, dtype=torch.int32, device=dev)
    x = torch.empty(d, dtype=torch.float64, device=dev)
    info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device=dev)

    def step(i: int):
        ctx.sketch_csc(ptr, rows, vals, b, n, d, r, seed=i, instance=rank, SA=SA, Sb=Sb, idx=idx)
        ctx.solve(SA, Sb, r=r, x=x, info=info)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.15)
    B.rnnls_profile_begin(ctx.handle, 16 * args.steps + 64)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    prof = B.rnnls_profile_end(ctx.handle)
    clk = clocks.stop(w0, w1)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    # e2e: the sparse arrays and b copied in, x read back, every step
    x_h = torch.empty(d, dtype=torch.float64).pin_memory()
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, min(args.steps, 100))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        for dst, src in ((ptr, ptr_h), (rows, rows_h), (vals, vals_h), (b, b_h)):
            dst.copy_(src, non_blocking=True)
        step(i)
        x_h.copy_(x, non_blocking=True)
        stream.synchronize()
    e_dt = max_over_ranks(time.perf_counter() - e0, dev)
    h2d = int(ptr_h.numel() * 8 + rows_h.numel() * 4 + vals_h.numel() * 4 + b_h.numel() * 4)
    # bytes the sparse sketch must move: the non-zeros and b in, the sketch and rows out
    launches, kms = prof["sketch_csc"]
    abytes = int(8 * nnz + 8 * (d + 1) + 4 * n + 4 * r * (d + 1) + 4 * r)
    achieved = abytes / (kms / launches / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    wl = workload_desc(cfg, p)
    wl["workload"] += f", A in compressed sparse columns ({nnz / (n * d):.4f} non-zero)"
    wl["pipeline"] = "rnnls_sketch_csc + rnnls_solve per step on one stream"
    out = {
        "metric": METRIC, "value": ws * args.steps / (ms / 1e3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded term-document-like stand-in for TechTC300), sparse columns", "config": wl,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "sketch_csc",
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": abytes, "avg_launch_us": 1e3 * kms / launches,
                     "dense_equivalent_bytes": int(4 * n * (d + 1) + 4 * r * (d + 1) + 4 * r),
                     "note": "the transform (n log2 4096 additions per column) bounds this kernel, not its bytes"},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "e2e": {"value": ws * e2e_steps / e_dt, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(d * 8)},
        "clocks": clk, "solve_info": P.info_dict(info), "cpu_baseline": None,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_boost(args, ws: int, rank: int, local: int, dev):
    """Repeated RandomizedNNLS on workload 2 or 3: one step = rnnls_solve_boosted
    with k runs (one batched sketch launch, one batched solve, one residual
    pass over A for all k runs, one select); solves/s counts boosted solves."""
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    cfg, k = args.config, args.boost
    if cfg not in (2, 3):
        raise SystemExit("--boost runs on workload 2 or 3")
    p = workloads.problem(cfg, seed=rank_seed(workloads.CONFIGS[cfg]["seed"], rank, ws))
    A_host = torch.from_numpy(np.ascontiguousarray(p.A.astype(np.float32).T)).pin_memory()
    b_host = torch.from_numpy(np.asarray(p.b, dtype=np.float32)).pin_memory()
    A = A_host.to(dev).t()
    b = b_host.to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local, stream)
    x = torch.empty(p.d, dtype=torch.float64, device=dev)
    resid = torch.empty(k, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device=dev)

    def step(i: int, A_=A, b_=b):
        ctx.solve_boosted(A_, b_, p.r, k, seed=i, instance0=k * rank, x=x, resid=resid, best=best, info=info)

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.15)
    B.rnnls_profile_begin(ctx.handle, 32 * args.steps + 64)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        step(1000 + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    prof = B.rnnls_profile_end(ctx.handle)
    clk = clocks.stop(w0, w1)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = ws * args.steps / (ms / 1e3)

    # e2e: A and b in from pinned host memory, x back, every step, through the same call
    x_host = torch.empty(p.d, dtype=torch.float64).pin_memory()
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, min(args.steps, 50))
    A2 = torch.empty((p.d, p.n), dtype=torch.float32, device=dev).t()
    b2 = torch.empty_like(b)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        A2.copy_(A_host.t(), non_blocking=True)
        b2.copy_(b_host, non_blocking=True)
        step(2000 + i, A2, b2)
        x_host.copy_(x, non_blocking=True)
        stream.synchronize()
    e_dt = max_over_ranks(time.perf_counter() - e0, dev)
    e2e = {"value": ws * e2e_steps / e_dt, "unit": "solves/s",
           "h2d_bytes_per_step": int((A_host.numel() + b_host.numel()) * 4), "d2h_bytes_per_step": int(p.d * 8)}

    # residual ratio of the kept run (seed 0) against the exact NNLS on the full A
    step(0)
    x_b = x.clone()
    res_all = resid.clone()
    x_opt, _ = ctx.solve(A, b, r=p.n)
    res_b, res_o = ctx.residual(A, b, x_b), ctx.residual(A, b, x_opt)
    torch.cuda.synchronize()
    ratio = float(res_b.item()) / float(res_o.item())
    run_ratios = [float(v) / float(res_o.item()) for v in res_all.cpu().tolist()]

    peak, peak_src = measured_hbm_peak()
    sk_launches, sk_ms = prof["sketch_srht_f32"]
    sk_bytes = k * algorithmic_bytes(p, 4)  # one batched launch sketches all k runs
    sk_ach = sk_bytes / (sk_ms / sk_launches / 1e3) / 1e9
    rs_launches, rs_ms = prof["boost_residual"]
    rs_bytes = p.n * (p.d + 1) * 4  # one read of A and b
    wl = workload_desc(cfg, p)
    wl["boost"] = k
    wl["pipeline"] = "one rnnls_solve_boosted per step on one stream"
    out = {
        "metric": f"RandNNLS boosted solves/s (best of {k} runs by full residual)", "value": value,
        "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded term-document-like stand-in for TechTC300)", "config": wl,
        "roofline": {"bound": "hbm", "achieved": sk_ach, "peak": peak, "unit": "GB/s", "frac": sk_ach / peak,
                     "traffic": None, "kernel": "sketch_srht_f32",
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": sk_bytes, "avg_launch_us": 1e3 * sk_ms / sk_launches},
        "residual_pass": {"kernel": "boost_residual", "avg_launch_us": 1e3 * rs_ms / rs_launches,
                          "algorithmic_bytes_per_launch": rs_bytes,
                          "achieved_gbs": rs_bytes / (rs_ms / rs_launches / 1e3) / 1e9,
                          "frac": rs_bytes / (rs_ms / rs_launches / 1e3) / 1e9 / peak},
        "kernel_ms_per_step": {kk: v[1] / args.steps for kk, v in prof.items()},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "e2e": e2e, "clocks": clk,
        "residual_ratio": ratio, "run_residual_ratios": run_ratios, "kept_run": int(best.item()),
        "cpu_baseline": None,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def density_matrix(n: int, cols: int, density: float, seed: int, dev):
    """An n x cols matrix (column-major, on the device) in which each entry is
    non-zero with probability `density`; the non-zeros are |N(0, 1)| clipped
    to [0, 1] (the reading of Sec. 4.2's "normally distributed in [0, 1]")."""
    import torch

    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    keep = torch.rand((cols, n), generator=g, device=dev) < density
    vals = torch.randn((cols, n), generator=g, device=dev).abs_().clamp_(max=1.0)
    return torch.where(keep, vals, torch.zeros((), device=dev)).t()


def run_density(args, ws: int, rank: int, local: int, dev):
    """Sec. 4.2's density experiment with the library: for each density, ten
    n x (d+1) matrices, ten choices of the column that forms b, and for each
    r in (d, d+50, d+100, d+150) the mean of ||A x~ - b|| / ||A x_opt - b||
    (x~ by the sketch and Lawson-Hanson, x_opt by Lawson-Hanson on the full A).
    Timing against the paper's comparison solver is out of scope."""
    import torch

    import paper_0812_4547_gb300 as P

    n, d = 10000, 300
    rs = [d, d + 50, d + 100, d + 150]
    densities = [0.02, 0.04, 0.08, 0.16, 0.32, 0.64]
    per_matrix = 10
    mats = max(1, (args.sweep_problems + per_matrix - 1) // per_matrix)
    ctx = P.Context(local)
    hrng = np.random.default_rng(42 + rank)
    table, statuses = {}, 0
    t0 = time.perf_counter()
    for dens in densities:
        ratios = {r: [] for r in rs}
        for m in range(mats):
            X = density_matrix(n, d + 1, dens, seed=1000 * rank + 97 * m + int(dens * 1e4), dev=dev)
            for c in hrng.permutation(d + 1)[:per_matrix]:
                keep = [j for j in range(d + 1) if j != c]
                A = X[:, keep].t().contiguous().t()
                b = X[:, int(c)].contiguous()
                x_opt, info_o = ctx.solve(A, b, r=n)
                res_o = float(ctx.residual(A, b, x_opt).item())
                statuses += int(P.info_dict(info_o)["status"] != 0)
                for r in rs:
                    x, info, _ = ctx.randomized_nnls(A, b, r, seed=int(c) + 7 * m, instance=rank)[:3]
                    statuses += int(P.info_dict(info)["status"] != 0)
                    res = float(ctx.residual(A, b, x).item())
                    ratios[r].append(math.sqrt(res / res_o) if res_o > 0 else float("nan"))
        table[f"{int(dens * 100)}%"] = {str(r): float(np.mean(v)) for r, v in ratios.items()}
    dt = time.perf_counter() - t0
    ctx.close()
    out = {"metric": "density sweep: mean ||A x~ - b|| / ||A x_opt - b|| over the problems of each density",
           "n": n, "d": d, "r": rs, "problems_per_density": mats * per_matrix, "table": table,
           "nonzero_solve_status": statuses, "seconds": dt,
           "paper_at_r_300": {"2%": 1.18, "64%": 1.04},
           "data": "synthetic: density-d matrices, non-zeros |N(0,1)| clipped to [0,1], b one of the columns"}
    if rank == 0:
        print(json.dumps(out), flush=True)


def device_batch(shapes, seed: int, dev, only=None):
    """Workload-5 instances generated on the device (the recipe of workload 2:
    Bernoulli(0.02) * LogNormal(0, 1) * (j+1)^-1.1 entries, x with half zeros,
    b = A x + 5 % noise); torch's Philox generator, seeded per instance.
    `only`: indices of the instances to build (the others are skipped but
    their host draws are made, so that instance i is the same either way)."""
    import torch

    out = []
    hrng = np.random.default_rng(seed)
    want = None if only is None else set(int(i) for i in only)
    for i, (n_raw, d, r) in enumerate(shapes):
        x = workloads.planted_x(d, int(round(0.5 * d)), hrng)
        if want is not None and i not in want:
            continue
        g = torch.Generator(device=dev)
        g.manual_seed(seed * 100003 + i)
        colw = torch.arange(1, d + 1, device=dev, dtype=torch.float32).pow(-1.1)[:, None]
        # leading dimension rounded up to 4 floats (16-byte aligned columns, as a caller would allocate)
        ld = (n_raw + 3) // 4 * 4
        At = torch.zeros((d, ld), device=dev)
        At[:, :n_raw] = torch.where(torch.rand((d, n_raw), generator=g, device=dev) < 0.02,
                                    torch.randn((d, n_raw), generator=g, device=dev).exp_() * colw,
                                    torch.zeros((), device=dev))
        y = At[:, :n_raw].t().double() @ torch.from_numpy(x).to(dev)
        sigma = 0.05 * float(torch.linalg.vector_norm(y)) / math.sqrt(n_raw)
        b = (y + sigma * torch.randn(n_raw, generator=g, device=dev, dtype=torch.float64)).float()
        out.append((At.t()[:n_raw], b, r))
    return out


def batch_sample(count: int, size: int = 32) -> list:
    """A spread sample of workload-5 instance indices (every count/size-th), so
    that host-side timings see the batch's mix of n and d, not its first rows."""
    step = max(1, count // size)
    return list(range(0, count, step))[:size]


def pinned_h2d_gbs(dev, nbytes: int = 1 << 30) -> float:
    """The plain host-to-device copy rate of this host link (pinned source, one stream)."""
    import torch

    h = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
    dbuf = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
    dbuf.copy_(h, non_blocking=True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream(dev)
    e0.record(s)
    for _ in range(4):
        dbuf.copy_(h, non_blocking=True)
    e1.record(s)
    torch.cuda.synchronize(dev)
    return 4 * nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9


def run_batch(args, ws: int, rank: int, local: int, dev):
    """Workload 5: 512 uneven instances per step, sketched by one batched call
    and solved by one batched call, replayed as one CUDA graph; also times the
    plain per-instance form (one stream, no graph), the end-to-end leg (host
    inputs copied in, x read back) and the accuracy against the FP64 oracle."""
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    c5 = workloads.CONFIGS[5]
    pf = prec_flag(args)
    bseed = rank_seed(c5["seed"], rank, ws)
    shapes = workloads.batch_shapes(count=args.instances, seed=bseed)
    insts = device_batch(shapes, bseed, dev)
    count = len(insts)
    main_s = torch.cuda.Stream(dev)
    ctx_plain = P.Context(local, main_s)
    bufs = []
    for (A, b, r) in insts:
        d = A.shape[1]
        bufs.append((torch.empty((d, r), dtype=torch.float32, device=dev).t(), torch.empty(r, device=dev),
                     torch.empty(r, dtype=torch.int32, device=dev), torch.empty(d, dtype=torch.float64, device=dev),
                     torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device=dev)))

    # the batched calls stage their job tables through their context's pinned
    # buffer, which a captured graph reads again at every replay: one context each
    ctx_sketch = P.Context(local, main_s)
    ctx_solve = P.Context(local, main_s)
    problems = [(bufs[i][0], bufs[i][1], bufs[i][3], bufs[i][4]) for i in range(count)]

    def sketch_items(ids, seed0):
        return [(insts[i][0], insts[i][1], insts[i][2], seed0 + i, rank, bufs[i][0], bufs[i][1], bufs[i][2])
                for i in ids]

    def enqueue(seed0: int, batched: bool = True):
        if batched:
            # every sketch in one batched call, then every solve in one batched call
            ctx_sketch.sketch_batched(sketch_items(range(count), seed0), prec=pf)
            ctx_solve.solve_batched(problems)
        else:
            # the plain per-instance form: sketch and solve each instance in turn on one stream
            for i, (A, b, r) in enumerate(insts):
                SA, Sb, idx, x, info = bufs[i]
                ctx_plain.sketch(A, b, r, seed=seed0 + i, instance=rank, SA=SA, Sb=Sb, idx=idx, want_count=False,
                                 prec=pf)
                ctx_plain.solve(SA, Sb, r=r, x=x, info=info)

    nprof = 3
    tuned = None
    with torch.cuda.stream(main_s):
        for w in range(max(1, args.warmup)):
            enqueue(0)
        torch.cuda.synchronize()
        if not args.no_tune:
            # launch-shape knobs of the batched calls picked by the autotuner
            # (coordinate search on this batch; cached per device and shape)
            from paper_0812_4547_gb300 import autotune

            t0 = time.perf_counter()
            tuned = autotune.tune([ctx_sketch, ctx_solve], lambda: enqueue(0), "batched",
                                  {"instances": count, "seed": bseed, "prec": args.prec}, repeats=2)
            tuned["seconds"] = time.perf_counter() - t0
            torch.cuda.synchronize()
        # per-kernel times: CUDA events around every launch of `nprof` steps
        # (the same launches as a graph replay, enqueued directly)
        for c in (ctx_sketch, ctx_solve):
            B.rnnls_profile_begin(c.handle, 8 * count * nprof + 64)
        for _ in range(nprof):
            enqueue(0)
        torch.cuda.synchronize()
        prof = {}
        for c in (ctx_sketch, ctx_solve):
            for k, v in B.rnnls_profile_end(c.handle).items():
                a = prof.get(k, (0, 0.0))
                prof[k] = (a[0] + v[0], a[1] + v[1])
        # the plain per-instance form: one stream, no graph
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(main_s)
        enqueue(0, batched=False)
        t1.record(main_s)
        torch.cuda.synchronize()
        plain_ms = t0.elapsed_time(t1)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=main_s, capture_error_mode="relaxed"):
            enqueue(0)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.15)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        ev0.record(main_s)
        for _ in range(args.steps):
            graph.replay()
        ev1.record(main_s)
        torch.cuda.synchronize()
        w1 = time.time()
        clk = clocks.stop(w0, w1)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = ws * args.steps * count / (ms / 1e3)
    infos = [P.info_dict(bufs[i][4]) for i in range(count)]
    stat = [f["status"] for f in infos]
    kname = "sketch_srht_f32"
    launches, kms = prof.get(kname, (0, 0.0))
    sketch_bytes = sum(int(4 * A.shape[0] * (A.shape[1] + 1) + 4 * r * (A.shape[1] + 1) + 4 * r)
                       for (A, b, r) in insts if A.shape[0] > 8192)
    achieved = sketch_bytes / (kms / max(launches, 1) / 1e3) / 1e9 if kms > 0 else None
    peak, peak_src = measured_hbm_peak()
    wl = {"workload": f"c5: {count} uneven instances, n 2^U[14,20], d U{{16..200}}, r pow2 of 8(d+1)ln n",
          "instances": count, "total_input_gb": sum(4 * A.shape[0] * (A.shape[1] + 1) for A, _, _ in insts) / 1e9,
          "sampling": "iid", "precision": args.prec, "l2": "inputs larger than L2 (no flush)",
          "parallelism": "independent instances per GPU",
          "pipeline": "one CUDA graph per step: one rnnls_sketch_batched over all instances (rows, plans and "
                      "sketches in one launch each), then one rnnls_solve_batched; every replay redoes every "
                      "kernel with the same seeds"}
    plain_v = ws * count / (plain_ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec_dtype(args),
        "data": "synthetic (term-document-like, generated on the device)",
        "config": wl,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": recorded_traffic(kname + ("_bf16x2" if pf else ""), wl["workload"]), "kernel": kname,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": sketch_bytes, "avg_launch_us": 1e3 * kms / max(launches, 1),
                     "frac_of_nominal_8tbs": achieved / 8000.0 if achieved else None,
                     "note": f"the batched sketch launch (all instances with n > 8192), mean of {nprof} steps "
                             "enqueued directly with CUDA events around each launch"},
        "plain_per_instance": {"value": plain_v, "unit": "solves/s", "ms_per_step": plain_ms,
                               "form": "one rnnls_sketch + rnnls_solve per instance, one stream, no graph"},
        "speedup_vs_plain": value / plain_v,
        "kernel_ms_per_step": {k: v[1] / nprof for k, v in prof.items()},
        "gpu_launches": int(args.steps * sum(v[0] for v in prof.values()) / nprof),
        "clocks": clk,
        "solve_status_nonzero": int(sum(1 for x in stat if x != 0)),
        # solves whose FP32 end point failed its float-float check and that
        # continued in the accurate mode (rnnls_info.accurate_mode > 0)
        "lh_accurate_mode_solves": int(sum(1 for f in infos if f.get("accurate_mode", 0) > 0)),
        "tuning": None if tuned is None else {
            "knobs": tuned["tuning"], "tuned_step_ms": tuned["ms"], "default_step_ms": tuned["default_ms"],
            "trials": len(tuned["trials"]), "cached": tuned["cached"], "seconds": tuned.get("seconds")},
    }
    out["e2e"] = e2e_batch(args, insts, bufs, dev, local, rank, ws, None if tuned is None else tuned["tuning"])
    out.update(batch_accuracy(args, insts, bufs, ctx_plain, rank, dev))
    for c in (ctx_plain, ctx_sketch, ctx_solve):
        c.close()
    out["cpu_baseline"] = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batch(insts, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)


def e2e_batch(args, insts, bufs, dev, local: int, rank: int, ws: int, tuning=None) -> dict:
    """Workload 5 end to end through the public calls: every step copies all
    instances' A and b from pinned host memory, sketches and solves them in
    groups (one rnnls_sketch_batched and one rnnls_solve_batched per group,
    the copy of group g+1 overlapping the work on group g) and reads every x
    back into pinned host memory."""
    import torch

    import paper_0812_4547_gb300 as P

    count = len(insts)
    # flat views of each instance's device storage (d columns of ld floats)
    flats, offs, total = [], [], 0
    for A, b, r in insts:
        ld = A.stride(1)
        fa = A.as_strided((A.shape[1] * ld,), (1,))
        flats.append((fa, b))
        offs.append(total)
        total += fa.numel() + b.numel()
    t_pin = time.perf_counter()
    host = torch.empty(total, dtype=torch.float32).pin_memory()
    for (fa, b), o in zip(flats, offs):
        host[o:o + fa.numel()].copy_(fa)
        host[o + fa.numel():o + fa.numel() + b.numel()].copy_(b)
    torch.cuda.synchronize(dev)
    t_pin = time.perf_counter() - t_pin
    xs_host = [torch.empty(A.shape[1], dtype=torch.float64).pin_memory() for A, _, _ in insts]
    ngroups = 8
    groups = [list(range(g * count // ngroups, (g + 1) * count // ngroups)) for g in range(ngroups)]
    copy_s = torch.cuda.Stream(dev)
    comp_s = torch.cuda.Stream(dev)
    ctx_sk = [P.Context(local, comp_s) for _ in range(ngroups)]
    ctx_sv = [P.Context(local, comp_s) for _ in range(ngroups)]
    if tuning:
        for c in ctx_sk + ctx_sv:
            c.set_tuning(tuning)
    copied = [torch.cuda.Event() for _ in range(ngroups)]
    consumed = [torch.cuda.Event() for _ in range(ngroups)]
    used = [False] * ngroups

    def e2e_step(seed0: int):
        for g, ids in enumerate(groups):
            if used[g]:
                copy_s.wait_event(consumed[g])  # the previous step's sketch of this group has read its inputs
            with torch.cuda.stream(copy_s):
                for i in ids:
                    fa, b = flats[i]
                    o = offs[i]
                    fa.copy_(host[o:o + fa.numel()], non_blocking=True)
                    b.copy_(host[o + fa.numel():o + fa.numel() + b.numel()], non_blocking=True)
            copied[g].record(copy_s)
            comp_s.wait_event(copied[g])
            ctx_sk[g].sketch_batched([(insts[i][0], insts[i][1], insts[i][2], seed0 + i, rank, bufs[i][0],
                                       bufs[i][1], bufs[i][2]) for i in ids], prec=prec_flag(args))
            consumed[g].record(comp_s)
            used[g] = True
            ctx_sv[g].solve_batched([(bufs[i][0], bufs[i][1], bufs[i][3], bufs[i][4]) for i in ids])
            with torch.cuda.stream(comp_s):
                for i in ids:
                    xs_host[i].copy_(bufs[i][3], non_blocking=True)

    e2e_steps = args.e2e_steps if args.e2e_steps is not None else 4
    for _ in range(2):  # warm-up: workspaces, pinned staging and the link's first transfers
        e2e_step(0)
    torch.cuda.synchronize(dev)
    e0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(0)
    torch.cuda.synchronize(dev)
    e_dt = max_over_ranks(time.perf_counter() - e0, dev)
    for c in ctx_sk + ctx_sv:
        c.close()
    h2d = int(total * 4)
    link = pinned_h2d_gbs(dev)
    return {"value": ws * e2e_steps * count / e_dt, "unit": "solves/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": int(sum(8 * A.shape[1] for A, _, _ in insts)), "steps": e2e_steps,
            "h2d_gbs_achieved": h2d * e2e_steps / e_dt / 1e9, "h2d_link_gbs_plain_pinned_copy": link,
            "link_bound_solves_per_s": count / (h2d / (link * 1e9)), "pin_setup_s": t_pin,
            "form": f"pinned host A, b copied in {ngroups} groups per step on a copy stream; one "
                    "rnnls_sketch_batched + rnnls_solve_batched per group on a compute stream; x read back"}


def batch_accuracy(args, insts, bufs, ctx, rank: int, dev) -> dict:
    """Residual ratios of Theorem 1 for every instance (x~ of the timed step's
    seeds against the exact NNLS on the full A, both by the library), and on
    a few instances the FP64 oracle's ratio, sketch and x~ beside the GPU's."""
    import torch

    import paper_0812_4547_gb300 as P

    count = len(insts)
    ratios = []
    for i, (A, b, r) in enumerate(insts):
        x_t = bufs[i][3]
        x_opt, _ = ctx.solve(A, b, r=A.shape[0])
        rt, ro = ctx.residual(A, b, x_t), ctx.residual(A, b, x_opt)
        ratios.append((rt, ro))
    torch.cuda.synchronize(dev)
    rho = [float(rt.item()) / float(ro.item()) if float(ro.item()) > 0 else 1.0 for rt, ro in ratios]
    out = {"residual_ratio": max(rho), "residual_ratio_mean": float(np.mean(rho)),
           "residual_ratio_le_1.01_share": float(np.mean([v <= 1.01 for v in rho])),
           "residual_ratio_unsquared": math.sqrt(max(rho))}
    if rank != 0 or args.no_oracle_check:
        return out
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    # the oracle on a few of the spread sample's smaller instances (its exact
    # NNLS on the full A is O(n d^2) on the host)
    cand = [i for i in batch_sample(count) if insts[i][0].shape[0] * insts[i][0].shape[1] ** 2 <= 4e9][:4]
    rows = []
    t0 = time.perf_counter()
    for i in cand:
        A, b, r = insts[i]
        Ah = A.cpu().numpy().astype(np.float32)
        bh = b.cpu().numpy().astype(np.float32)
        SA_o, Sb_o, _ = oracle.sketch(Ah, bh, r, seed=i, instance=rank, nthreads=threads)
        x_o, _ = oracle.nnls(SA_o, Sb_o)
        x_opt_o, _ = oracle.exact_nnls(Ah, bh)
        rho_o = oracle.residual_sq(Ah, bh, x_o) / oracle.residual_sq(Ah, bh, x_opt_o)
        SA_g = bufs[i][0].cpu().numpy().astype(np.float64)
        Sb_g = bufs[i][1].cpu().numpy().astype(np.float64)
        x_g = bufs[i][3].cpu().numpy()
        rows.append({"instance": i, "n": int(A.shape[0]), "d": int(A.shape[1]), "r": int(r),
                     "rho_gpu": rho[i], "rho_oracle": float(rho_o),
                     "SA_rel_fro_vs_oracle": float(np.linalg.norm(SA_g - SA_o) / np.linalg.norm(SA_o)),
                     "Sb_rel_fro_vs_oracle": float(np.linalg.norm(Sb_g - Sb_o) / np.linalg.norm(Sb_o)),
                     "x_rel_vs_oracle_end_to_end": float(np.linalg.norm(x_g - x_o) / max(np.linalg.norm(x_o), 1e-300)),
                     "same_support": bool(np.array_equal(x_g > 0, x_o > 0))})
    out["oracle_check"] = {"instances": rows, "seconds": time.perf_counter() - t0,
                           "note": "oracle = FP64 C sketch + Lawson-Hanson on the same FP32 input bytes and seeds; "
                                   "x error is end to end (the GPU solve runs on the FP32 sketch)"}
    return out


def cpu_baseline_batch(insts, seconds: float) -> dict:
    """The FP64 oracle on a spread sample of the workload-5 instances (every
    count/32-th instance, copied to the host), as many as fit in about
    `seconds`; solves/s over the instances it ran."""
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    done, t_run = 0, 0.0
    for i in batch_sample(len(insts)):
        A, b, r = insts[i]
        Ah = A.cpu().numpy()
        bh = b.cpu().numpy()
        t0 = time.perf_counter()
        oracle.randomized_nnls(Ah, bh, r, seed=i, nthreads=threads)
        t_run += time.perf_counter() - t0
        done += 1
        if t_run >= seconds:
            break
    return {"value": done / t_run, "unit": "solves/s", "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{done} instances of the batch's spread sample (every {max(1, len(insts) // 32)}-th) in "
                      f"{t_run:.1f} s (FP64 C oracle, OpenMP over columns)"}


if __name__ == "__main__":
    main()
