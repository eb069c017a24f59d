#!/usr/bin/env python
"""Benchmark of the sGKS hot path on one GB300 (or N independent replicas under torchrun).

Headline workload (default, --config ct2d_batch): parallel-beam CT, 512 x 512 image, 180 angles x
725 bins (CSR of ray-pixel intersection lengths, FP32 values, 60 M nonzeros), 2D gradient L, 2%
noise; 64 right-hand sides (noise seed i) x lambda_i = 10^(-4 + 3i/63) solved as one batch
(sgks_batch_*), 150 iterations each, sparse-sign sketch s = 600, zeta = 8.  Form: float-float
("ff": the basis and every vector as (hi, lo) float pairs, compensated sums on the FP32 units,
FP64 sketched QR and projected solve), FP64-class results.  One step = one batch solve:
sgks_batch_reset (setup of all 64 instances) + 150 iterations.  Metric: sGKS instance-iterations
per second (whole job, all replicas).  The working set (basis 20.5 GB) is far larger than L2.

The line also carries the roofline of the step's largest-share kernel, the CPU oracle on the
host cores (one thread, and one process per core over different instances), an end-to-end
figure through the public API with host buffers, and a compact comparison: plain FP64 GPU sGKS
on the same batch and on one instance alone, with the time to reach the FP64 run's RRE targets.
--config deblur2d|ct2d|seismic2d|dynct|deconv1d runs one right-hand side of that workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sGKS iterations/s (256x256 deblurring, FP32 operators + FP64 QR/solve + 2 refinement steps)"
UNIT = "iterations/s"
WORKLOAD = ("deblur2d: 256x256 image, 9x9 Gaussian PSF sigma=2 zero boundary, grad2d L, lambda=5e-3, 1% noise, "
            "sparse-sign s=400 zeta=8, 100 iterations, FP32 + 2 refinement steps")


def labels(name, P=None):
    """(metric, workload) of the JSON line: the deblurring workload's fixed labels, or labels
    built from the problem for another --config."""
    if name == "deblur2d":
        return METRIC, WORKLOAD
    if P is None:
        P = make_workload(name, seed=0)
    A = P.A
    op = f"CSR {A.m}x{A.n} nnz {len(A.col)}" if A.kind == "csr" else f"{A.kind} {A.m}x{A.n}"
    form = P.precision.upper() + (f" + {P.n_refine} refinement steps" if P.n_refine else "")
    wl = (f"{name}: A {op}, {P.L.kind} L (p = {P.p}), {P.sketch.kind} s={P.sketch.s}, {P.iters} iterations, "
          f"{form}")
    return f"sGKS iterations/s ({name}, {form})", wl


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 100: about 1 s of GPU work; 20 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=BATCH_CONFIG)
    ap.add_argument("--precision", default="ff", choices=["ff", "fp32", "fp64", "fp32plain"],
                    help="form of the batched headline (ct2d_batch)")
    ap.add_argument("--compare", default="fp64,fp32", type=lambda v: [x for x in v.split(",") if x],
                    help="other forms timed on the same batch for the comparison block")
    ap.add_argument("--compare-dynct", default="fp32", help="form of the ragged dynamic-CT batch extra")
    ap.add_argument("--cpu-instance", type=int, default=42, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-opfile", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seed", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--ct-size", type=int, default=512, help=argparse.SUPPRESS)   # image side of the CT batch (tests)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison, profile and CPU baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched CT and dynamic-CT measurements")
    ap.add_argument("--cpu-sample-iters", type=int, default=None,
                    help="iterations of the oracle sample (default 20 for the CT batch, 25 otherwise)")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile-single", default=None, choices=["deblur2d", "ct2d", "dynct"],
                    help="one solve of one instance of the workload alone in --precision (fp64 or fp32), "
                         "for profiler captures")
    ap.add_argument("--profile-batch", default=None, choices=["ct2d", "dynct"],
                    help="run one batched solve of a reduced CT / dynamic-CT batch (for profiler captures) and exit")
    ap.add_argument("--batch-size", type=int, default=16)
    ap.add_argument("--batch-iters", type=int, default=40)
    args = ap.parse_args()
    if args.steps is None:
        if args.config == BATCH_CONFIG:
            args.steps = 3 if args.impl == "reference" else 10
        else:
            args.steps = 20 if args.impl == "reference" else 100
    if args.cpu_sample_iters is None:
        args.cpu_sample_iters = 20 if args.config == BATCH_CONFIG else 25
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------- multi-rank
def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (the job time is the slowest replica's).

    Replicas only: sGKS has no exchange step, so each rank solves its own right-hand side and
    this reduction of one timing scalar is the only cross-rank communication."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_max: float, world_size: int) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world_size * units_per_rank / (ms_max / 1e3)


# ----------------------------------------------------------------------------- workload
def make_workload(name, seed):
    from workloads import make_problem
    return make_problem(name, seed=seed)


# --------------------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(name, iters, seed=0):
    """Time the FP64 oracle (as it stands) on `iters` iterations of the workload, one thread."""
    import oracle as O
    P = make_workload(name, seed)
    t0 = time.perf_counter()
    O.sgks(P, iters=iters)
    dt = time.perf_counter() - t0
    return dict(seconds=dt, iters=iters)


def run_cpu_worker(name, iters):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--config", name,
           "--cpu-sample-iters", str(iters)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms, read by a thread with host timestamps.  start() waits for
    the first sample, so the sampler is running before the timed region opens; stop() keeps only
    the samples taken between begin() and end() (the region's host-side bounds, each taken right
    after a device synchronize)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.monotonic() + 10.0
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.01)

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.thread.join(timeout=5)
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = self.t1 if self.t1 is not None else float("inf")
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, line in self.lines:
            if not (t0 <= t <= t1):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm),
                "window_s": round(t1 - t0, 3), "interval_ms": 100}


# -------------------------------------------------------------------------- byte models
def matrix_bytes(P, elem, rows):
    """Bytes of one pass over the stored operator A (or its stored transpose, `rows` rows): CSR
    column indices, values in the solve precision and row pointers; a dense matrix; nothing for
    the matrix-free convolution."""
    A = P.A
    if A.kind == "csr":
        return len(A.col) * (4 + elem) + (rows + 1) * 4
    if A.kind == "dense":
        return A.m * A.n * elem
    return 0


def bytes_model(P, cls, d, elem):
    """Algorithmic bytes of one launch of a kernel class at subspace size d (bytes each launch must move at minimum; per-kernel formulas below)."""
    n, m, p, s = P.n, P.m, P.p, P.sketch.s
    T = elem
    if cls in ("gradient_append", "gradient_refine"):   # A^T e: one pass over the stored transpose
        return _vector_bytes(n, m, s, d, T, cls) + matrix_bytes(P, elem, n)
    if cls == "sketch_column":                           # A w: one pass over A
        return _vector_bytes(n, m, s, d, T, cls) + matrix_bytes(P, elem, m)
    return _vector_bytes(n, m, s, d, T, cls)


def _vector_bytes(n, m, s, d, T, cls):
    if cls == "combine":
        return d * (n + m) * T + (n + 2 * m) * T + 3 * n * T
    if cls == "combine_refine":
        return d * (n + m) * T + (n + 2 * m) * T
    if cls == "gradient_refine":
        return d * n * T + (m + n) * T
    if cls == "gradient_append":
        return (m + n) * T + n * T
    if cls == "sketch_column":
        return n * T + m * T
    if cls == "qr_append":
        return 8 * (2 * s * d + 2 * s + 2 * d)
    if cls == "stacked_solve":
        return 8 * (2 * d * d + 2 * d * d + 2 * d)
    if cls == "refine_solve":
        return 8 * d * d
    return 0


def traffic_record(kernel_class):
    """DRAM bytes per launch of a kernel from the committed ncu summaries in profiles/, or None
    when no record exists or the kernel's source changed since the counters were taken."""
    import glob
    import hashlib
    # the kernel that serves each class on the 256^2 deblurring workload
    name = {"gradient_refine": "k_gradient_refine2", "gradient_append": "k_gradient_append_conv"}.get(
        kernel_class, "k_" + kernel_class)
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            f = line.split()
            if len(f) == 5 and f[0] == "traffic-record:" and f[1] == name:
                src = os.path.join(ROOT, "paper_2606_18073_gb300", "csrc", f[2])
                try:
                    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
                except OSError:
                    return None
                return float(f[4]) if sha == f[3] else None
    return None


def flops_fp64(P, cls, d):
    s = P.sketch.s
    if cls == "qr_append":       # 2 factors x 2 passes x (dot + update) over s x d
        return 2.0 * 2 * 2 * 2 * s * d
    if cls == "stacked_solve":   # 2 passes x (dot + update) over 2d x d, X t and X z
        return 2.0 * (2 * 2 * 2 * d * d + d * d)
    if cls == "refine_solve":
        return 2.0 * d * d
    return 0.0


# --------------------------------------------------------------------------- reference
def run_reference_batch(args):
    """The oracle arm on the CT batch: each step runs one single-threaded oracle process per host
    core, each on its own instance (setup + --cpu-sample-iters // 4 iterations, at least 3), all
    together; instance-iterations/s over the steps."""
    import tempfile

    import numpy as np
    A0 = ct_batch_operator(args.ct_size)
    cores = os.cpu_count() or 1
    iters = max(3, args.cpu_sample_iters // 4)
    tot = 0.0
    with tempfile.TemporaryDirectory() as td:
        opfile = os.path.join(td, "ctop.npz")
        np.savez(opfile, rp=A0.row_ptr, col=A0.col, val=A0.val, m=A0.m, n=A0.n)

        def one_step(k):
            procs = [run_cpu_batch_sample(opfile, (k * cores + i) % BATCH_COUNT, iters, 1, 0, args.ct_size)
                     for i in range(cores)]
            secs = []
            for q in procs:
                so, se = q.communicate(timeout=3600)
                if q.returncode != 0:
                    raise RuntimeError(se[-2000:])
                secs.append(json.loads(so.strip().splitlines()[-1])["seconds"])
            return max(secs)

        for k in range(args.warmup):
            one_step(k)
        for k in range(args.steps):
            tot += one_step(args.warmup + k)
    value = args.steps * cores * iters / tot
    prec = args.precision
    line = {
        "impl": "reference", "metric": batch_metric(prec), "value": value, "unit": "instance-iterations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batch_workload(len(A0.col), prec, args.ct_size),
                   "sample": f"per step: {cores} single-threaded oracle processes (one per host core), each "
                             f"setup + {iters} of 150 iterations of its own instance, run together; setup included"},
        "cpu_baseline": {"value": value, "unit": "instance-iterations/s", "cores": cores, "kind": "oracle",
                         "sample": f"NumPy FP64 oracle, {cores} processes x (setup + {iters} iterations) per step"},
        "e2e": {"value": value, "unit": "instance-iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.config == BATCH_CONFIG:
        run_reference_batch(args)
        return
    name = args.config
    iters = args.cpu_sample_iters   # the same sample as the cpu_baseline of the GPU arm's line
    for _ in range(args.warmup):
        run_cpu_worker(name, iters)
    tot = 0.0
    for _ in range(args.steps):
        r = run_cpu_worker(name, iters)
        tot += r["seconds"]
    value = args.steps * iters / tot
    line = {
        "impl": "reference", "metric": labels(name)[0], "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": labels(name)[1], "sample": f"setup + {iters} iterations per step, the setup inside the time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"NumPy FP64 oracle, setup + {iters} iterations of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------- batched headline
BATCH_CONFIG = "ct2d_batch"
BATCH_COUNT = 64
BATCH_FORM_LABEL = {"ff": "float-float (hi, lo) pairs on the FP32 units + FP64 sketched QR / projected solve",
                    "fp32": "FP32 basis, compensated float-float sums + FP64 sketched QR / projected solve",
                    "fp64": "plain FP64", "fp32plain": "FP32 arithmetic with FP32 accumulation"}
BATCH_DTYPE = {"ff": "ff32x2+f64", "fp32": "f32+ff32x2+f64", "fp64": "f64", "fp32plain": "f32+f64"}


def batch_metric(prec):
    return f"sGKS instance-iterations/s (512^2 CT, 64 RHS x lambda batch, 150 iterations, {prec})"


def batch_workload(nnz, prec, N=512):
    return (f"ct2d_batch: {N}x{N} parallel-beam CT, 180 angles x {int(math.ceil(math.sqrt(2.0) * N))} bins, "
            f"CSR FP32 (nnz {nnz}), grad2d L, "
            f"2% noise, 64 right-hand sides (noise seed i) x lambda_i = 10^(-4+3i/63), sparse-sign s=600 zeta=8, "
            f"150 iterations each, one batch (sgks_batch), form {prec}: {BATCH_FORM_LABEL.get(prec, prec)}")


def ct_batch_operator(N):
    """The CT operator of the batch: N x N image, 180 angles, ceil(sqrt(2) N) bins (725 at N = 512)."""
    import numpy as np
    from workloads.configs import ct_op
    return ct_op(N, np.arange(180) * 1.0, int(math.ceil(math.sqrt(2.0) * N)))


def ct_batch_problems(A0, count, seed=0, prec="ff"):
    from workloads.configs import make_ct2d
    return [make_ct2d(instance=i, seed=seed, N=A0.nx, A=A0, precision=prec) for i in range(count)]


def ct_batch_inputs(G, probs, prec, dev):
    dt = G.io_dtype(prec)
    kw = G.device_inputs(probs[0], prec, device=dev)
    insts = [dict(A=kw["A"], reg=kw["reg"], lam=P.lam, b=_dev_tensor(P.b, dt, dev),
                  x_true=_dev_tensor(P.x_true, dt, dev)) for P in probs]
    return insts


def make_batch(G, insts, P0, prec, iters, n_refine=0):
    return G.Batch(insts, P0.sketch.s, P0.sketch.seed, max_iters=iters, n_refine=n_refine, precision=prec,
                   zeta=P0.sketch.zeta, autotune=True)


def batch_bytes(kind, B, n, m, nnz, d, prec):
    """Algorithmic bytes of one launch of a batched kernel class (all B instances): the CSR arrays
    once (4-byte indices and values, row pointers), each instance vector read or written once, and
    for the combine the d columns of W and A W.  Basis values take 8 bytes in the FP64 and
    float-float forms and 4 in the FP32 forms; the other vectors 8 (float-float or FP64) or 4."""
    tw = 8 if prec in ("ff", "fp64") else 4
    tv = 4 if prec == "fp32plain" else 8
    if kind == "apply_column":      # u = A w -> AW column (L w is a stencil: n in, p out, not counted)
        return nnz * 8 + (m + 1) * 4 + B * (n * tw + m * tv)
    if kind == "gradient_append":   # A^T e + lambda L^T L x -> W column
        return nnz * 8 + (n + 1) * 4 + B * (m * tv + n * tv + n * tw)
    if kind == "combine":           # x = W y, e = AW y - b, RC / RRE statistics
        return B * (d * (n * tw + m * tv) + n * tv * 3 + n * tv + m * tv * 2)
    if kind == "sketch_gather":
        return 0
    return 0


# FP32 operations of one compensated multiply-add u += a * v with a an FP32 operator value:
# TwoProd (multiply, fused multiply-add), TwoSum (six additions), two additions collecting the
# errors, and one fused multiply-add for the low part when v is a float-float pair.
DOT2_MAC_OPS = {"ff": 11, "fp32": 10}
# FP32 lanes of GB300: 152 SMs x 4 sub-partitions x 32 lanes, one FP32 instruction per lane per
# cycle, at the maximum SM clock of 2,070 MHz.
FP32_LANE_OPS_PEAK = 152 * 128 * 2.07e9


def batch_ops(kind, B, nnz, prec):
    """Algorithmic FP32 operations of one launch of an ALU-bound batched class in the compensated
    forms: one compensated multiply-add per operator entry and instance (the tiled pass's per-ray
    sums of partials and the L^T L stencil of the gradient, a few percent, are not counted).  The
    A^T e pass multiplies FP32 values by float-float e in both forms."""
    if prec not in DOT2_MAC_OPS:
        return 0
    if kind == "apply_column":
        return nnz * B * DOT2_MAC_OPS[prec]
    if kind == "gradient_append":
        return nnz * B * DOT2_MAC_OPS["ff"]
    return 0


def timed_batch_steps(Bt, bs, iters, steps, dev, flush=None):
    import torch
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    rep = None
    for k in range(steps):
        if flush is not None:
            flush.zero_()
        evs[k][0].record(stream)
        Bt.reset(bs)
        rep = Bt.solve(iters, history=(k == steps - 1))
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    return sum(a.elapsed_time(b) for a, b in evs), rep


def rre_targets(rre_hist):
    """Targets for time-to-tolerance: 1.01 x the final RRE and 1.01 x the minimum RRE of a run (the
    CT batch is semi-convergent: its RRE bottoms out early and then rises), with the iteration of
    the minimum."""
    k_min = int(min(range(len(rre_hist)), key=lambda k: rre_hist[k]))
    return {"final": 1.01 * rre_hist[-1], "min": 1.01 * rre_hist[k_min], "k_min": k_min + 1}


def run_cpu_batch_sample(opfile, instance, iters, threads=1, seed=0, ct_size=512):
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--config", BATCH_CONFIG,
           "--cpu-sample-iters", str(iters), "--cpu-instance", str(instance), "--cpu-opfile", opfile,
           "--cpu-seed", str(seed), "--ct-size", str(ct_size)]
    return subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)


def cpu_batch_worker(args):
    """One oracle solve (setup + --cpu-sample-iters iterations) of CT instance --cpu-instance, with
    the operator read from --cpu-opfile; prints the seconds."""
    import numpy as np
    import oracle as O
    from workloads.configs import make_ct2d
    from workloads.problem import OperatorDesc
    z = np.load(args.cpu_opfile)
    A0 = OperatorDesc("csr", int(z["m"]), int(z["n"]), row_ptr=z["rp"], col=z["col"], val=z["val"],
                      nx=args.ct_size, ny=args.ct_size)
    P = make_ct2d(instance=args.cpu_instance, seed=args.cpu_seed, N=args.ct_size, A=A0)
    t0 = time.perf_counter()
    O.sgks(P, iters=args.cpu_sample_iters)
    print(json.dumps({"seconds": time.perf_counter() - t0, "iters": args.cpu_sample_iters,
                      "instance": args.cpu_instance}))


def cpu_batch_baseline(A0, iters, seed=0):
    N = A0.nx
    """The oracle as it stands on the batch workload, bounded sample (setup + `iters` iterations of
    an instance per process): one process with one thread, then one single-threaded process per
    host core (instances 0, 1, ...) running together.  Instance-iterations/s for each."""
    import tempfile

    import numpy as np
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as td:
        opfile = os.path.join(td, "ctop.npz")
        np.savez(opfile, rp=A0.row_ptr, col=A0.col, val=A0.val, m=A0.m, n=A0.n)
        out = {}
        p = run_cpu_batch_sample(opfile, 42, iters, 1, seed, N)
        so, se = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError(se[-2000:])
        r1 = json.loads(so.strip().splitlines()[-1])
        out["one_thread"] = {"value": iters / r1["seconds"], "seconds": r1["seconds"], "cores": 1}
        t0 = time.perf_counter()
        procs = [run_cpu_batch_sample(opfile, i % BATCH_COUNT, iters, 1, seed, N) for i in range(cores)]
        secs = []
        for q in procs:
            so, se = q.communicate(timeout=3600)
            if q.returncode != 0:
                raise RuntimeError(se[-2000:])
            secs.append(json.loads(so.strip().splitlines()[-1])["seconds"])
        wall = time.perf_counter() - t0
        out["all_cores"] = {"value": cores * iters / max(secs), "seconds": max(secs), "cores": cores,
                            "wall_s": wall}
    return out


def bench_batch_form(G, probs, prec, dev, iters, steps=2):
    """One timed batch solve (best of `steps` after a warm-up) of the CT batch in form `prec`, and
    the RRE record of instance 42."""
    import torch
    insts = ct_batch_inputs(G, probs, prec, dev)
    Bt = make_batch(G, insts, probs[0], prec, iters)
    bs = [i["b"] for i in insts]
    Bt.reset(bs)
    Bt.solve(iters)
    best, rep = None, None
    for _ in range(steps):
        ms, r = timed_batch_steps(Bt, bs, iters, 1, dev)
        if best is None or ms < best:
            best, rep = ms, r
    Bt.close()
    del insts
    torch.cuda.empty_cache()
    return best, rep


def main_batch(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2606_18073_gb300 as G

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    G.build()
    prec = args.precision
    iters = 150
    A0 = ct_batch_operator(args.ct_size)
    nnz = len(A0.col)
    probs = ct_batch_problems(A0, BATCH_COUNT, seed=rank, prec=prec)
    n, m = probs[0].n, probs[0].m
    insts = ct_batch_inputs(G, probs, prec, dev)
    bs = [i["b"] for i in insts]
    Bt = make_batch(G, insts, probs[0], prec, iters)
    tuned = Bt.config(0)
    for _ in range(args.warmup):
        Bt.reset(bs)
        Bt.solve(iters)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = ClockSampler(dev.index)
    clk.start()
    launches0 = G.kernel_launches()
    torch.cuda.synchronize(dev)
    clk.begin()
    ms, rep = timed_batch_steps(Bt, bs, iters, args.steps, dev)
    clk.end()
    launches = G.kernel_launches() - launches0
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(ms, dev)
    clocks = clk.stop()
    units = BATCH_COUNT * iters
    value = job_throughput(args.steps * units, ms, ws)

    # ---- e2e through the public API: every instance's b host -> device (pinned) before the
    # reset, every instance's x device -> host after the solve, inside the timed step
    dt = G.io_dtype(prec)
    b_host = [torch.from_numpy(np.asarray(P.b)).to(dt).pin_memory() for P in probs]
    x_host = [torch.empty(n, dtype=dt).pin_memory() for _ in probs]
    b_dev = [torch.empty(m, dtype=dt, device=dev) for _ in probs]
    x_dev = [torch.empty(n, dtype=dt, device=dev) for _ in probs]
    stream = torch.cuda.current_stream(dev)
    e2e_ms = 0.0
    for _ in range(args.steps):
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for bd, bh in zip(b_dev, b_host):
            bd.copy_(bh, non_blocking=True)
        Bt.reset(b_dev)
        Bt.solve(iters, x_out=x_dev)
        for xh, xd in zip(x_host, x_dev):
            xh.copy_(xd, non_blocking=True)
        c.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms += a.elapsed_time(c)
    e2e_ms = max_over_ranks(e2e_ms, dev)
    e2e_value = job_throughput(args.steps * units, e2e_ms, ws)
    elem = torch.empty(0, dtype=dt).element_size()
    rre = [r["rre_last"] for r in rep]
    line = {
        "metric": batch_metric(prec), "value": value, "unit": "instance-iterations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": BATCH_DTYPE.get(prec, prec), "data": "synthetic",
        "config": {"workload": batch_workload(nnz, prec, args.ct_size), "instances": BATCH_COUNT, "iterations_per_step": iters,
                   "l2": "inputs larger than L2 (basis %.1f GB)" % (BATCH_COUNT * n * (iters + 3) * (8 if prec in ("ff", "fp64") else 4) / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single", "autotuned": tuned,
                   "final_rre": {"instance_42": rre[42], "median": float(np.median(rre))}},
        "e2e": {"value": e2e_value, "unit": "instance-iterations/s",
                "h2d_bytes_per_step": BATCH_COUNT * m * elem, "d2h_bytes_per_step": BATCH_COUNT * n * elem},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        # ---- roofline of the step's largest-share kernel: one eager solve with an event pair
        # around every launch (launches are milliseconds long, so the pair adds little)
        Bt.reset(bs)
        prof = Bt.profile(iters)
        tot = sum(v["ms"] for v in prof.values())
        d_avg = 3 + (iters + 1) / 2.0
        kern = {}
        for k, v in prof.items():
            if not v["launches"]:
                continue
            # launches per iteration differ between classes: time per iteration
            us = 1e3 * v["ms"] / iters
            bts = batch_bytes(k, BATCH_COUNT, n, m, nnz, d_avg, prec)
            ops = batch_ops(k, BATCH_COUNT, nnz, prec)
            kern[k] = {"share": v["ms"] / tot, "launches": v["launches"], "us_per_iteration": us,
                       "alg_bytes_per_iteration": bts, "gbps": bts / (us * 1e-6) / 1e9 if bts else None,
                       "alg_fp32_ops_per_iteration": ops, "fp32_tops": ops / (us * 1e-6) / 1e12 if ops else None}
        dom = max(kern, key=lambda k: kern[k]["share"])
        hbm = measured_hbm()
        kd = kern[dom]
        name = batch_kernel_name(dom, prec)
        common = {"kernel": name, "class": dom, "traffic": traffic_record_batch(name, prec),
                  "us_per_iteration": kd["us_per_iteration"], "share": kd["share"],
                  "duration": "CUDA event pairs around the class's launches in one eager solve (150 iterations)"}
        if kd["fp32_tops"]:
            ach = kd["fp32_tops"]
            peak = FP32_LANE_OPS_PEAK / 1e12
            line["roofline"] = dict({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TOP/s (FP32)",
                                     "frac": ach / peak, "alg_fp32_ops_per_iteration": kd["alg_fp32_ops_per_iteration"],
                                     "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (one FP32 instruction "
                                                    "per lane per cycle)"}, **common)
        else:
            ach = kd["gbps"] or 0.0
            line["roofline"] = dict({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                     "frac": ach / hbm, "alg_bytes_per_iteration": kd["alg_bytes_per_iteration"],
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}, **common)
        line["kernels"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                           for k, v in kern.items()}
        # ---- plain FP64 GPU sGKS: the same batch, and instance 42 alone; time to the RRE targets
        tg = rre_targets(rep[42]["rre"])
        cmp = {"form": prec, "instance": 42, "rre_targets": tg}
        ours_ms = ms / args.steps
        cmp[prec] = {"ms_per_solve": ours_ms, "instance_iters_per_s": units / (ours_ms / 1e3),
                     "time_to_min_target_ms": time_to_rre(ours_ms, rep[42]["rre"], tg["min"], iters),
                     "time_to_final_target_ms": time_to_rre(ours_ms, rep[42]["rre"], tg["final"], iters),
                     "rre_42_final": rep[42]["rre_last"], "rre_42_min": min(rep[42]["rre"])}
        Bt.close()
        del insts, bs
        torch.cuda.empty_cache()
        for other in args.compare:
            if other == prec:
                continue
            try:
                t, r = bench_batch_form(G, probs, other, dev, iters)
                cmp[other] = {"ms_per_solve": t, "instance_iters_per_s": units / (t / 1e3),
                              "time_to_min_target_ms": time_to_rre(t, r[42]["rre"], tg["min"], iters),
                              "time_to_final_target_ms": time_to_rre(t, r[42]["rre"], tg["final"], iters),
                              "rre_42_final": r[42]["rre_last"], "rre_42_min": min(r[42]["rre"])}
            except Exception as exc:   # the headline stands without it
                cmp[other] = {"error": repr(exc)[:300]}
        P42 = probs[42]
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        kw64 = G.device_inputs(P42, "fp64", device=dev)
        S64 = G.Solver(**kw64)
        t64, h64 = time_solve(G, S64, kw64["b"], iters, flush, dev)
        S64.close()
        cmp["fp64_single_instance_42"] = {
            "ms_per_solve": t64, "iters_per_s": iters / (t64 / 1e3),
            "time_to_min_target_ms": time_to_rre(t64, h64["rre"], tg["min"], iters),
            "time_to_final_target_ms": time_to_rre(t64, h64["rre"], tg["final"], iters),
            "rre_final": h64["rre_last"], "rre_min": min(h64["rre"])}
        line["compare"] = cmp
        # ---- the oracle on the host cores (bounded sample)
        try:
            cb = cpu_batch_baseline(A0, args.cpu_sample_iters)
            ac, one = cb["all_cores"], cb["one_thread"]
            line["cpu_baseline"] = {
                "value": ac["value"], "unit": "instance-iterations/s", "cores": ac["cores"], "kind": "oracle",
                "sample": f"NumPy FP64 oracle, setup + {args.cpu_sample_iters} of {iters} iterations per instance, "
                          f"one single-threaded process per core ({ac['cores']} cores, instances 0..{ac['cores'] - 1}), "
                          f"{ac['seconds']:.1f} s; setup included",
                "one_thread": {"value": one["value"], "cores": 1, "seconds": one["seconds"], "instance": 42}}
        except Exception as exc:
            line["cpu_baseline"] = {"value": None, "unit": "instance-iterations/s", "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": f"failed: {exc}"[:300]}
        if not args.no_batch:
            extras_path = os.environ.get("SGKS_BENCH_EXTRAS")
            ex = {"dynct_ragged16": bench_dynct_batch(G, dev, flush, args.compare_dynct)}
            ex["single_instance"] = bench_singles(G, dev, flush)
            ex["srtt_sketch_sweep"] = {"deblur2d": bench_srtt_sweep(G, dev, flush),
                                       "ct2d": bench_srtt_sweep(G, dev, flush, "ct2d", (300, 600), "fp64")}
            ex["differentiable"] = bench_differentiable(G, dev, flush)
            ex["gks"] = {nm: bench_gks(G, nm, dev, flush) for nm in ("deblur2d", "ct2d")}
            line["srtt_ct2d"] = {k: v for k, v in ex["srtt_sketch_sweep"]["ct2d"].items()}
            line["dynct_ragged16"] = compact_dynct(ex["dynct_ragged16"])
            if extras_path:
                with open(extras_path, "w") as f:
                    json.dump(ex, f, indent=1)
    else:
        Bt.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


BATCH_KERNEL_NAMES = {"apply_column": "kbx_csr_apply", "gradient_append": "kbx_csr_gradient",
                      "combine": "kbx_combine_tma", "sketch_gather": "kbx_sketch_gather",
                      "qr_append": "k_qr_append", "stacked_solve": "k_stacked_solve",
                      "sketch_l": "kbx_sketch_l_chunks+kbx_sketch_l_reduce"}


def batch_kernel_name(kind, prec):
    """The kernels behind a profile class of the batched CT workload (A w runs through pixel tiles
    in the compensated forms)."""
    if kind == "apply_column" and prec in ("ff", "fp32"):
        return "kbx_tile_apply+kbx_seg_reduce"
    return BATCH_KERNEL_NAMES.get(kind, kind)


def traffic_record_batch(kernel, prec):
    """DRAM bytes per launch of a batched kernel at the full workload size, from the committed ncu
    summary of that kernel and form (profiles/*.md lines 'traffic-record-batch: <kernel> <form>
    <source file> <sha12> <bytes>'), or None when absent or when the source changed since."""
    import glob
    import hashlib
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            f = line.split()
            if len(f) == 6 and f[0] == "traffic-record-batch:" and f[1] == kernel and f[2] == prec:
                src = os.path.join(ROOT, "paper_2606_18073_gb300", "csrc", f[3])
                try:
                    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
                except OSError:
                    return None
                return float(f[5]) if sha == f[4] else None
    return None


def compact_dynct(rec):
    keep = ("instances", "iterations", "ms_per_solve", "instance_iters_per_s", "final_rre", "fp64_plain_single",
            "batched_instance_final_rre", "time_to_target_ms", "form", "compare")
    return {k: rec[k] for k in keep if k in rec}


def bench_singles(G, dev, flush):
    """One right-hand side of the deblurring, CT and dynamic-CT workloads alone: the FP32 form
    (compensated sums, the workload's refinement steps) and plain FP64 (no refinement)."""
    out = {}
    for name in ("deblur2d", "ct2d", "dynct"):
        rec = {}
        for prec in ("fp32", "fp64"):
            P = make_workload(name, seed=0)
            if prec == "fp64":
                P.n_refine = 0
            kw = G.device_inputs(P, prec, device=dev)
            S = G.Solver(**kw)
            t, h = time_solve(G, S, kw["b"], P.iters, flush, dev)
            S.close()
            rec[prec] = {"iters_per_s": P.iters / (t / 1e3), "ms_per_solve": t, "final_rre": h["rre_last"],
                         "n_refine": P.n_refine}
        out[name] = rec
    return out


# --------------------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.cpu_worker:
        if args.config == BATCH_CONFIG:
            cpu_batch_worker(args)
        else:
            print(json.dumps(cpu_oracle_sample(args.config, args.cpu_sample_iters)))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_batch:
        profile_batch(args)
        return
    if args.profile_single:
        profile_single(args)
        return
    if args.config == BATCH_CONFIG:
        main_batch(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2606_18073_gb300 as G

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    G.build()

    P = make_workload(args.config, seed=rank)
    iters = P.iters
    kw = G.device_inputs(P, P.precision, device=dev)
    S = G.Solver(**kw)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def one_step(solver, b):
        solver.reset(b)
        return solver.solve(iters)

    for _ in range(args.warmup):
        flush.zero_()
        one_step(S, kw["b"])
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = ClockSampler(dev.index)
    clk.start()
    launches0 = G.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    clk.begin()
    rep = None
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        rep = one_step(S, kw["b"])
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk.end()
    launches = G.kernel_launches() - launches0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(ms, dev)
    clocks = clk.stop()
    value = job_throughput(args.steps * iters, ms, ws)

    # ---- e2e through the public API with host buffers (pinned), copies inside the timed step
    dt = kw["b"].dtype
    b_host = torch.from_numpy(np.asarray(P.b)).to(dt).pin_memory()
    x_host = torch.empty(P.n, dtype=dt).pin_memory()
    b_dev = torch.empty_like(kw["b"])
    x_dev = torch.empty(P.n, dtype=dt, device=dev)
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b_dev.copy_(b_host, non_blocking=True)
        S.reset(b_dev)
        S.solve(iters, x_out=x_dev)
        x_host.copy_(x_dev, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms += a.elapsed_time(b)
    e2e_ms = max_over_ranks(e2e_ms, dev)
    e2e_value = job_throughput(args.steps * iters, e2e_ms, ws)
    elem = b_host.element_size()

    line = {
        "metric": labels(args.config, P)[0], "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if P.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": labels(args.config, P)[1], "iterations_per_step": iters, "l2": "flushed (256 MiB write) before each step",
                   "parallelism": "replicas" if ws > 1 else "single", "final_rre": rep["rre_last"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": P.m * elem, "d2h_bytes_per_step": P.n * elem},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        line.update(extras(args, G, P, kw, S, iters, dev, flush))
    S.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def time_solve(G, S, b, iters, flush, dev, reps=3):
    stream = torch_stream(dev)
    import torch
    best = None
    for _ in range(reps):
        flush.zero_()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.reset(b)
        out = S.solve(iters, history=True)
        c.record(stream)
        torch.cuda.synchronize(dev)
        t = a.elapsed_time(c)
        best = (t, out) if best is None or t < best[0] else best
    return best


def torch_stream(dev):
    import torch
    return torch.cuda.current_stream(dev)


def time_to_rre(ms_total, rre_hist, target, iters):
    """Wall time until RRE_k <= target, assuming equal time per iteration (setup included)."""
    for k, r in enumerate(rre_hist):
        if r <= target:
            return ms_total * (k + 1) / iters
    return None


def extras(args, G, P, kw, S, iters, dev, flush):
    import torch
    out = {}
    # FP32 + refinement: per-iteration RRE history for time-to-tolerance
    t32, h32 = time_solve(G, S, kw["b"], iters, flush, dev)
    # plain FP64 GPU sGKS on the same problem (no refinement, as Algorithm 2)
    P64 = make_workload(args.config, seed=0)
    P64.n_refine = 0
    kw64 = G.device_inputs(P64, "fp64", device=dev)
    S64 = G.Solver(**kw64)
    t64, h64 = time_solve(G, S64, kw64["b"], iters, flush, dev)
    S64.close()
    target = 1.01 * h64["rre_last"]
    out["fp64_plain"] = {"iters_per_s": iters / (t64 / 1e3), "ms_per_solve": t64, "final_rre": h64["rre_last"]}
    # fp32x: FP32 storage with compensated arithmetic, same refinement steps as the headline form
    Px = make_workload(args.config, seed=0)
    kwx = G.device_inputs(Px, "fp32x", device=dev)
    Sx = G.Solver(**kwx)
    tx, hx = time_solve(G, Sx, kwx["b"], iters, flush, dev)
    Sx.close()
    out["fp32x_refined"] = {"iters_per_s": iters / (tx / 1e3), "ms_per_solve": tx, "final_rre": hx["rre_last"],
                            "time_to_target_ms": time_to_rre(tx, hx["rre"], target, iters)}
    out["time_to_rre"] = {
        "target_rre": target,
        "fp64_plain_ms": time_to_rre(t64, h64["rre"], target, iters),
        "fp32_refined_ms": time_to_rre(t32, h32["rre"], target, iters),
        "fp32_refined_final_rre": h32["rre_last"],
    }
    # per-kernel profile (CUDA events on the library's stream around every launch, one eager
    # solve): the time shares of the kernel classes
    S.reset(kw["b"])
    prof = S.profile(iters)
    tot = sum(v["ms"] for v in prof.values())
    elem = 4 if P.precision == "fp32" else 8
    kern = {}
    for k, v in prof.items():
        if v["launches"] == 0:
            continue
        davg = v["dsum"] / v["launches"]
        bts = bytes_model(P, k, davg, elem)
        kern[k] = {"ms_total": v["ms"], "launches": v["launches"], "share": v["ms"] / tot,
                   "us_per_launch": 1e3 * v["ms"] / v["launches"], "avg_d": davg,
                   "alg_bytes_per_launch": bts, "gbps": bts / (1e-3 * v["ms"] / v["launches"]) / 1e9}
    out["kernels"] = kern
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # dominant bandwidth kernel (largest time share among the streaming kernels).  The event pair
    # around each eager launch adds the launch latency to every sample, so the kernel's own
    # duration is taken from back-to-back launches in one graph (sgks_time_class) at the middle of
    # the solve, where d is the solve's average subspace size.
    stream_k = [k for k in kern if k not in ("qr_append", "stacked_solve", "refine_solve")]
    dom = max(stream_k, key=lambda k: kern[k]["ms_total"])
    S.reset(kw["b"])
    S.solve(iters // 2)
    d_mid = S.info()["d"]
    timed = {}
    for k in ("gradient_append", "sketch_column", "combine_refine", "gradient_refine"):
        if k in kern:
            us = S.time_class(k, 200)
            bts = bytes_model(P, k, d_mid, elem)
            timed[k] = {"us_per_launch": us, "d": d_mid, "alg_bytes_per_launch": bts, "gbps": bts / (us * 1e-6) / 1e9}
    out["kernels_in_graph"] = timed
    dk = timed.get(dom, kern[dom])
    out["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": dk["gbps"], "peak": hbm, "unit": "GB/s",
                       "frac": dk["gbps"] / hbm, "traffic": traffic_record(dom),
                       "duration": "back-to-back launches in one graph at d = %d (sgks_time_class)" % d_mid
                       if dom in timed else "eager event pairs",
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)" if peaks else
                       "fallback 6800 GB/s"}
    small = {}
    for k in ("qr_append", "stacked_solve", "refine_solve"):
        a = kern.get(k)
        if a:
            fl = flops_fp64(P, k, a["avg_d"]) / (a["us_per_launch"] * 1e-6) / 1e12
            small[k] = {"bound": "alu", "achieved": fl, "peak": 1.25, "unit": "TFLOP/s (FP64)", "frac": fl / 1.25}
    out["fp64_small_phase"] = small
    if not args.no_batch:
        out["batched"] = {"ct2d_64rhs": bench_ct_batch(G, dev, flush), "dynct_ragged16": bench_dynct_batch(G, dev, flush)}
        out["differentiable"] = bench_differentiable(G, dev, flush)
        out["gks"] = {name: bench_gks(G, name, dev, flush) for name in ("deblur2d", "ct2d")}
        out["srtt_sketch_sweep"] = bench_srtt_sweep(G, dev, flush)
    # CPU oracle baseline, bounded sample, one thread
    try:
        r = run_cpu_worker(args.config, args.cpu_sample_iters)
        out["cpu_baseline"] = {"value": r["iters"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"FP64 NumPy oracle, setup + {r['iters']} of {iters} iterations, "
                                         f"{r['seconds']:.1f} s, BLAS threads = 1"}
    except Exception as exc:   # the GPU number stands without it
        out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}
    return out


# ------------------------------------------------------------------------- batched form
def _dev_tensor(a, dt, dev):
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


def time_batch(Bt, bs, iters, flush, dev, reps=2):
    """Best of `reps` (reset + solve(iters)) of a batch; the first call also warms up."""
    import torch
    stream = torch_stream(dev)
    Bt.reset(bs)
    Bt.solve(iters)
    best = None
    for _ in range(reps):
        flush.zero_()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Bt.reset(bs)
        out = Bt.solve(iters, history=True)
        c.record(stream)
        torch.cuda.synchronize(dev)
        t = a.elapsed_time(c)
        best = (t, out) if best is None or t < best[0] else best
    return best


def batch_profile(Bt, bs, iters):
    """Per-kernel times of one eager solve of the batch (each launch timed and synchronised)."""
    Bt.reset(bs)
    prof = Bt.profile(iters)
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    return {k: {"ms_total": v["ms"], "launches": v["launches"], "share": v["ms"] / tot,
                "us_per_launch": 1e3 * v["ms"] / v["launches"]} for k, v in prof.items() if v["launches"]}


def batch_roofline(prof, sizes, nnz, ell, iters, hbm, groups=1):
    """Achieved bandwidth of the batched streaming kernels at the solve's average subspace size.
    sizes: (n_i, m_i) per instance; nnz: nonzeros of the CSR matrices the instances share
    (counted once per pass).  combine: W and AW columns plus the vectors of every instance,
    against HBM.  CSR passes: the matrix once plus the vectors written, against HBM; the
    instance-vector gathers (nnz x B values per pass, served from L2) as a separate rate.
    groups: launches of a class per step (ragged batches run one launch per group), whose
    times add up to the step's time for that class."""
    d = ell + (iters - 1) / 2.0
    B = len(sizes)
    out = {"d_avg": d}
    vec_n = sum(n for n, _ in sizes) * 4
    vec_m = sum(m for _, m in sizes) * 4
    defs = {
        "combine": (d * (vec_n + vec_m) + 3 * vec_n + 2 * vec_m, 0),
        "apply_column": (nnz * 8 + vec_n + vec_m, nnz * B * 4),
        "gradient_append": (nnz * 8 + vec_m + 3 * vec_n, nnz * B * 4),
    }
    for k, (hb, gb) in defs.items():
        v = prof.get(k)
        if not v:
            continue
        t = v["us_per_launch"] * groups * 1e-6
        rec = {"alg_bytes_per_step": hb, "gbps": hb / t / 1e9, "frac_of_hbm": hb / t / 1e9 / hbm}
        if gb:
            rec["gathered_bytes_per_step"] = gb
            rec["gather_gbps"] = gb / t / 1e9
        out[k] = rec
    return out


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs", 6800.0))
    except OSError:
        return 6800.0


def batch_report(ms, reps, iters, count, P64, ref_idx, G, dev, flush):
    """Instance-iterations/s of the batch next to plain FP64 GPU sGKS on instance ref_idx."""
    import numpy as np
    P64.n_refine = 0
    kw64 = G.device_inputs(P64, "fp64", device=dev)
    S64 = G.Solver(**kw64)
    t64, h64 = time_solve(G, S64, kw64["b"], iters, flush, dev)
    S64.close()
    rre = [r["rre_last"] for r in reps]
    tg = rre_targets(h64["rre"])
    return {"instances": count, "iterations": iters, "ms_per_solve": ms,
            "instance_iters_per_s": count * iters / (ms / 1e3),
            "final_rre": {"min": float(np.min(rre)), "median": float(np.median(rre)), "max": float(np.max(rre))},
            "fp64_plain_single": {"instance": ref_idx, "iters_per_s": iters / (t64 / 1e3), "ms_per_solve": t64,
                                  "final_rre": h64["rre_last"], "min_rre": min(h64["rre"])},
            "batched_instance_final_rre": rre[ref_idx],
            "rre_targets_from_fp64": tg,
            "time_to_target_ms": {
                "batched": {"min": time_to_rre(ms, reps[ref_idx]["rre"], tg["min"], iters),
                            "final": time_to_rre(ms, reps[ref_idx]["rre"], tg["final"], iters)},
                "fp64_single": {"min": time_to_rre(t64, h64["rre"], tg["min"], iters),
                                "final": time_to_rre(t64, h64["rre"], tg["final"], iters)}}}


def bench_ct_batch(G, dev, flush, count=64):
    """Parallel-beam CT 512 x 512, 180 angles x 725 bins: 64 right-hand sides (noise seed i,
    lambda_i = 10^(-4 + 3 i / 63)) sharing one CSR, FP32, 150 iterations, s = 600."""
    import numpy as np
    import torch
    from workloads.configs import ct_op, make_ct2d
    A0 = ct_op(512, np.arange(180) * 1.0, 725)
    probs = [make_ct2d(instance=i, A=A0, precision="fp32") for i in range(count)]
    kw = G.device_inputs(probs[0], "fp32", device=dev)
    insts = [dict(A=kw["A"], reg=kw["reg"], lam=P.lam, b=_dev_tensor(P.b, torch.float32, dev),
                  x_true=_dev_tensor(P.x_true, torch.float32, dev)) for P in probs]
    P0 = probs[0]
    Bt = G.Batch(insts, P0.sketch.s, P0.sketch.seed, max_iters=P0.iters, n_refine=0, precision="fp32",
                 zeta=P0.sketch.zeta, autotune=True)
    tuned = Bt.config(0)
    ms, reps = time_batch(Bt, [i["b"] for i in insts], P0.iters, flush, dev)
    prof = batch_profile(Bt, [i["b"] for i in insts], P0.iters)
    Bt.close()
    del insts, kw
    torch.cuda.empty_cache()
    out = batch_report(ms, reps, P0.iters, count, make_ct2d(instance=42, A=A0), 42, G, dev, flush)
    out["kernels"] = prof
    out["roofline"] = batch_roofline(prof, [(P.n, P.m) for P in probs], len(A0.col), 3, P0.iters, measured_hbm())
    out["autotuned"] = tuned
    # the same instance alone in the FP32 form (no refinement), for the batch's gain
    P1 = make_ct2d(instance=42, A=A0, precision="fp32")
    P1.n_refine = 0
    kw1 = G.device_inputs(P1, "fp32", device=dev)
    S1 = G.Solver(**kw1)
    t1, h1 = time_solve(G, S1, kw1["b"], P1.iters, flush, dev)
    S1.close()
    out["fp32_single"] = {"instance": 42, "iters_per_s": P1.iters / (t1 / 1e3), "ms_per_solve": t1,
                          "final_rre": h1["rre_last"]}
    out["workload"] = ("ct2d: 512x512, 180 angles x 725 bins, CSR FP32 (nnz %d), grad2d L, 2%% noise, "
                       "lambda_i = 10^(-4+3i/63), sparse-sign s=600 zeta=8, 150 iterations, FP32, 64 RHS" % len(A0.col))
    return out


def bench_dynct_batch(G, dev, flush, prec="fp32"):
    """Dynamic CT 128 x 128 x F frames, 16 instances, F in {8, 16, 24, 32} (4 each, seeds 0..15):
    ragged sizes in four groups, 3 refinement steps, 200 iterations, s = 800, form `prec`."""
    import torch
    from workloads.configs import dynct_frame_ops, make_dynct
    ops = dynct_frame_ops(128, 32)
    frames = [8, 16, 24, 32] * 4
    probs, shared = [], {}
    for i, F in enumerate(frames):
        P = make_dynct(seed=i, frames=F, frame_ops=ops)
        P.A = shared.setdefault(F, P.A)
        probs.append(P)
    dev_ops = {}
    insts = []
    dt = G.io_dtype(prec)
    for P in probs:
        if id(P.A) not in dev_ops:
            kw = G.device_inputs(P, prec, device=dev)
            dev_ops[id(P.A)] = (kw["A"], kw["reg"])
        A, reg = dev_ops[id(P.A)]
        insts.append(dict(A=A, reg=reg, lam=P.lam, b=_dev_tensor(P.b, dt, dev),
                          x_true=_dev_tensor(P.x_true, dt, dev)))
    P0 = probs[0]
    Bt = G.Batch(insts, P0.sketch.s, P0.sketch.seed, max_iters=P0.iters, n_refine=P0.n_refine, precision=prec,
                 zeta=P0.sketch.zeta, autotune=True)
    groups = Bt.layout()[0]
    tuned = [Bt.config(g) for g in range(groups)]
    ms, reps = time_batch(Bt, [i["b"] for i in insts], P0.iters, flush, dev)
    prof = batch_profile(Bt, [i["b"] for i in insts], P0.iters)
    Bt.close()
    del insts, dev_ops
    torch.cuda.empty_cache()
    out = batch_report(ms, reps, P0.iters, len(probs), make_dynct(seed=3, frames=32, frame_ops=ops), 3, G, dev,
                       flush)
    out["groups"] = groups
    out["kernels"] = prof
    # each group streams its own frame CSR (shared by its instances): matrix bytes once per F
    nnz_groups = sum(len(A.col) for A in shared.values())
    out["roofline"] = batch_roofline(prof, [(P.n, P.m) for P in probs], nnz_groups, 3, P0.iters, measured_hbm(),
                                     groups=groups)
    out["autotuned"] = tuned
    out["form"] = prec
    out["workload"] = ("dynct: 128x128 x F frames, F in {8,16,24,32} x 4 instances, 30 angles/frame x 185 bins, "
                       f"space-time L, 1% noise, sparse-sign s=800 zeta=8, 200 iterations, {prec} + 3 refinement steps")
    return out


def bench_gks(G, name, dev, flush):
    """GKS (Algorithm 1) against sGKS (Algorithm 2) on the GPU, both plain FP64 without
    refinement, same problem and iteration count; the per-kernel split of a GKS solve."""
    P = make_workload(name, seed=0)
    P.n_refine = 0
    iters = P.iters
    out = {"iterations": iters}
    for method in ("sgks", "gks"):
        kw = G.device_inputs(P, "fp64", device=dev)
        kw["n_refine"] = 0
        S = G.Solver(**kw, method=method)
        t, h = time_solve(G, S, kw["b"], iters, flush, dev)
        rec = {"ms_per_solve": t, "iters_per_s": iters / (t / 1e3), "final_rre": h["rre_last"]}
        if method == "gks":
            S.reset(kw["b"])
            prof = S.profile(iters)
            tot = sum(v["ms"] for v in prof.values()) or 1.0
            names = {"gradient_append": "gradient + orthogonalisation against V",
                     "sketch_column": "A v, L v", "qr_append": "QR updates of A V and L V (CGS2)",
                     "stacked_solve": "projected solve", "combine": "x = V y, e, RC"}
            rec["kernels"] = {names.get(k, k): {"share": v["ms"] / tot, "ms_total": v["ms"]}
                              for k, v in prof.items() if v["launches"]}
        S.close()
        out[method] = rec
    out["gks_over_sgks_time"] = out["gks"]["ms_per_solve"] / out["sgks"]["ms_per_solve"]
    return out


def profile_single(args):
    """One solve of instance 0 of a workload on a single handle (FP64 without refinement, or the
    FP32 form with the workload's refinement steps), for profiler captures."""
    import torch
    import paper_2606_18073_gb300 as G
    G.build()
    dev = torch.device("cuda", 0)
    prec = args.precision if args.precision in ("fp64", "fp32") else "fp64"
    P = make_workload(args.profile_single, seed=0)
    if prec == "fp64":
        P.n_refine = 0
    S = G.Solver(**G.device_inputs(P, prec, device=dev))
    out = S.solve(P.iters)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_single": args.profile_single, "precision": prec, "iterations": out["iters_done"]}))
    S.close()


def profile_batch(args):
    """One reset + solve of a reduced batch, for profiler captures: the 512^2 CT operator with
    --batch-size right-hand sides (sparse-sign s = 600), or --batch-size space-time instances of 8
    frames (3 refinement steps, s = 800), --batch-iters iterations, form --precision."""
    import numpy as np
    import torch
    import paper_2606_18073_gb300 as G
    G.build()
    dev = torch.device("cuda", 0)
    B, iters = args.batch_size, args.batch_iters
    if args.profile_batch == "ct2d":
        from workloads.configs import ct_op, make_ct2d
        A0 = ct_op(512, np.arange(180) * 1.0, 725)
        probs = [make_ct2d(instance=i, A=A0, precision=args.precision, iters=iters) for i in range(B)]
    else:
        from workloads.configs import dynct_frame_ops, make_dynct
        ops = dynct_frame_ops(128, 8)
        probs = [make_dynct(seed=i, frames=8, frame_ops=ops, iters=iters) for i in range(B)]
        for P in probs[1:]:
            P.A = probs[0].A
    dt = G.io_dtype(args.precision)
    kw = G.device_inputs(probs[0], args.precision, device=dev)
    insts = [dict(A=kw["A"], reg=kw["reg"], lam=P.lam, b=torch.from_numpy(np.asarray(P.b)).to(dev, dt),
                  x_true=torch.from_numpy(np.asarray(P.x_true)).to(dev, dt)) for P in probs]
    P0 = probs[0]
    Bt = G.Batch(insts, P0.sketch.s, P0.sketch.seed, max_iters=iters, n_refine=P0.n_refine, precision=args.precision,
                 zeta=P0.sketch.zeta)
    Bt.reset([i["b"] for i in insts])
    out = Bt.solve(iters)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_batch": args.profile_batch, "precision": args.precision, "instances": B,
                      "iterations": iters,
                      "median_final_rre": float(np.median([o["rre_last"] for o in out]))}))
    Bt.close()


def bench_srtt_sweep(G, dev, flush, name="deblur2d", sizes=(200, 400, 800), precision=None):
    """A workload with the paper's SRTT sketch (eq. sketching_trig, dense on the device) at several
    sketch sizes s, next to the sparse-sign sketch at the workload's s (the paper's sketch-size
    sweeps: deblurring in Sec. 4.1, CT in Sec. 4.2.1)."""
    from workloads.configs import srtt_sketch
    out = {}
    base = make_workload(name, seed=0)
    prec = precision or base.precision
    iters = base.iters
    for s in sizes:
        P = make_workload(name, seed=0)
        P.sketch = srtt_sketch(s, P.m, P.p, seed=0)
        kw = G.device_inputs(P, prec, device=dev)
        S = G.Solver(**kw)
        t, h = time_solve(G, S, kw["b"], iters, flush, dev)
        S.close()
        out[f"srtt_s{s}"] = {"iters_per_s": iters / (t / 1e3), "final_rre": h["rre_last"], "min_rre": min(h["rre"])}
    kw = G.device_inputs(base, prec, device=dev)
    S = G.Solver(**kw)
    t, h = time_solve(G, S, kw["b"], iters, flush, dev)
    S.close()
    out[f"sparse_sign_s{base.sketch.s}"] = {"iters_per_s": iters / (t / 1e3), "final_rre": h["rre_last"],
                                            "min_rre": min(h["rre"])}
    out["form"] = prec
    return out


def bench_differentiable(G, dev, flush):
    """Seismic travel-time tomography, 256 x 256 slowness, 8192 rays, Laplacian L, 80 iterations:
    forward solve with the y_k record, then the reverse sweep (dl/db, dl/dlambda for
    l = ||x_80 - x_true||^2), FP64 and FP32, next to the plain FP64 forward.  Also the 256 x 256
    deblurring problem with its 2 refinement steps per iteration (40 iterations), whose sweep
    runs back through every refinement step."""
    import numpy as np
    import torch
    stream = torch_stream(dev)

    def timed(fn, reps=3):
        best, res = None, None
        for _ in range(reps):
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = fn()
            c.record(stream)
            torch.cuda.synchronize(dev)
            t = a.elapsed_time(c)
            best = t if best is None or t < best else best
        return best, res

    def case(P, n_refine, fp32_note):
        iters = P.iters
        res = {}
        for prec in ("fp64", "fp32"):
            kw = G.device_inputs(P, prec, device=dev)
            kw["n_refine"] = n_refine
            S = G.Solver(**kw, record=True)
            b = kw["b"]
            xt = torch.from_numpy(np.asarray(P.x_true)).to(dev, S.dtype)
            t_fwd, _ = timed(lambda: (S.reset(b), S.solve(iters)))
            xbar = (2.0 * (S.x() - xt)).contiguous()
            t_bwd, (bbar, lbar) = timed(lambda: S.backward(xbar))
            rec = {"forward_ms": t_fwd, "backward_ms": t_bwd, "dl_dlambda": lbar,
                   "forward_iters_per_s": iters / (t_fwd / 1e3)}
            if prec == "fp32":
                rec["note"] = fp32_note
            if prec == "fp64":
                h = 1e-6 * P.lam
                vals = []
                for lam in (P.lam + h, P.lam - h):
                    S.set_lambda(lam)
                    S.reset(b)
                    S.solve(iters)
                    vals.append(float(torch.sum((S.x() - xt) ** 2)))
                S.set_lambda(P.lam)
                fd = (vals[0] - vals[1]) / (2 * h)
                rec["dl_dlambda_central_difference"] = fd
                rec["dl_dlambda_rel_err"] = abs(lbar - fd) / abs(fd)
            S.close()
            res[prec] = rec
        return res

    P = make_workload("seismic2d", seed=0)
    out = {"workload": "seismic2d: 256x256, 64 sources x 128 receivers (8192 rays), laplace2d L, 1% noise, "
                       "sparse-sign s=400 zeta=8, 80 iterations, loss ||x_80 - x_true||^2"}
    out.update(case(P, 0, "the derivative goes through G_j^{-1}, the squared condition of the projected problem; "
                          "at 80 iterations the FP64 sweep's own rounding floor is ~1e-2, so the FP32 value "
                          "carries no digits (timing only)"))
    kw = G.device_inputs(P, "fp64", device=dev)
    kw["n_refine"] = 0
    S = G.Solver(**kw)
    t_plain, _ = timed(lambda: (S.reset(kw["b"]), S.solve(P.iters)))
    S.close()
    out["fp64_plain_forward_ms"] = t_plain
    # The unrolled derivative's conditioning grows with K (it goes through G_j^{-1}): on this problem
    # the FP64 oracle against itself under rounding-level perturbations differs by 2e-7 in dl/db at
    # K = 40, 1e-4 at K = 60 and O(1) at K = 100, so the derivative is taken at K = 40.
    Pd = make_workload("deblur2d", seed=0)
    Pd.iters = 40
    ref = {"workload": f"deblur2d: 256x256, 9x9 Gaussian psf, grad2d L, {Pd.n_refine} refinement steps per "
                       f"iteration, {Pd.iters} iterations, loss ||x_K - x_true||^2"}
    ref.update(case(Pd, Pd.n_refine, "FP32 form of the same solve: timing only"))
    out["refined"] = ref
    return out


if __name__ == "__main__":
    main()
