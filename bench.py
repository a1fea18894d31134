"""Benchmark of the TMOP hot path on GB300.

One step = one gradient + one Hessian-vector product of the variational TMOP
objective (eq. (2.4), Section 3.4) over a whole synthetic mesh: by default
48^3 order-3 hexahedra with 5x5x5 Gauss points and mu303 (13.8 M quadrature
points, 9.1 M dofs), interior nodes jittered, trilinear shear, boundary fixed.

Metric: quadrature points per second of gradient + Hessian action
(NE * Q / t(step)), plus time-to-converged Newton (Section 3.4 line search,
MINRES inner solves) for the plain FP64 form and the FP32-Hessian forms
(stored or recomputed operator, FP32 or FP64 Krylov vectors, Jacobi and
two-level preconditioners) on this workload, and (newton_configs) FP64,
FP32-Hessian and FP32-bulk Newton on the smaller configurations beside the
CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c4] [--precision fp64|mixed] [--no-converge]
                    [--no-pa] [--no-learned] [--no-configs] [--no-cpu-baseline]
                    [--kernels-only]

--impl reference times the plain FP64 CPU oracle (the reference for this
path) on a bounded sample of the same workload, one process per host core.
--kernels-only runs warm-up plus K steps and nothing else (for profilers);
with --profile pa it runs one linearisation and W+K partially assembled
Hessian actions instead (the linearisation is the second element-kernel
launch, after the validity check of the mesh); with --profile mlp, W+K
training steps (gradients + Adam) of the proposal MLP at batch 4096.
"""
from __future__ import annotations

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

from paper_1807_09807_gb300 import meshgen as mg  # noqa: E402

METRIC = "TMOP grad+Hessian-vec quad-points/s and time-to-converged mesh vs plain FP64"
UNIT = "quad-points/s"

# Nominal FP64 / FP32 non-tensor peaks from the GB300 unit counts and clock
# (152 SMs x 2.07 GHz x (2 FP64 FMA / 128 FP32 FMA per SM per clock) x 2
# flop), reported for context beside the peaks measured by tmop_fma_peak on
# the GPU at hand, which are the roofline denominators.
FP64_PEAK_GFLOPS = 152 * 2.07 * 2 * 2      # 1258.6 GFLOP/s
FP32_PEAK_GFLOPS = 152 * 2.07 * 128 * 2    # 80 547 GFLOP/s

# Flops of the closed-form second directional derivative dP = d2mu/dT2 : dT
# per quadrature point (cofactor, its derivative, invariants, the P update and
# the w det W scaling), counted from the formulas; W = I.
METRIC_DP_FLOPS = {303: 244, 302: 420, 2: 70, 7: 80, 9: 80, 77: 60, 1: 12, 14: 12}


def contraction_fmas(dim: int, n: int, q: int, nc: int) -> tuple[int, int]:
    """FMAs of the sum-factorised forward (nodes -> A) and adjoint
    (per-point matrices -> nodes) contractions of one element, nc components."""
    if dim == 2:
        fwd = nc * (n * q * 2 * n + q * q * 2 * n)
        adj = nc * (n * q * 2 * q + n * n * 2 * q)
    else:
        fwd = nc * (n * n * q * 2 * n + n * q * q * 3 * n + q ** 3 * 3 * n)
        adj = nc * (n * q * q * 3 * q + n * n * q * 3 * q + n ** 3 * 2 * q)
    return fwd, adj


def folded_contraction_flops(dim: int, n: int, q: int, nc: int):
    """Flops the FP64 3D kernels with an even node count execute for one
    element's forward map (nodes -> A) and adjoint map (per-point matrices ->
    nodes) in the mirror basis with normalised dots (fwd3_eon, adj3_eon and
    the butterfly passes around them), FMAs as two flops, multiplies and adds
    as one; None where the plain contractions run."""
    if dim != 3 or n % 2:
        return None
    h, qe, qo = n // 2, (q + 1) // 2, q // 2
    outs = nc * (n * n * q * 2 + n * q * q * 3 + q ** 3 * 3)          # forward stage outputs
    fwd = (nc * 3 * n * n * h * 2                                     # butterflies of the nodal field
           + 2 * (h - 1) * outs                                       # one FMA per output (n = 4)
           + 3 * nc * q * q * qo * 5 + (q % 2) * 3 * nc * q * q       # scaled axis-0 unfold
           + 2 * 3 * nc * q * q * qo * 2)                             # axes 1 and 2
    adj = (3 * nc * 3 * q * q * qo * 2                                # butterflies of the point fields
           + 2 * (nc * h * q * q * 3 * (q - 2) + nc * n * h * q * 3 * q + nc * n * n * h * 2 * q)
           + 2 * nc * n * n * h * 2 + nc * n * n * h * 5)             # nodal unfold, the last pass scaled
    return fwd, adj


def hess_executed_flops_per_element(dim, n, q, metric):
    """Flops the FP64 matrix-free Hessian action executes per element: the
    folded, normalised contractions where they run, else the plain ones,
    and dP at every point."""
    f = folded_contraction_flops(dim, n, q, dim)
    if f is None:
        return hess_flops_per_element(dim, n, q, metric)
    return 2 * f[0] + f[1] + METRIC_DP_FLOPS[metric] * q ** dim


def hess_flops_per_element(dim, n, q, metric):
    """Algorithmic flops of one matrix-free Hessian action on one element:
    forward contraction of x and of v, adjoint contraction, and dP at every
    point."""
    fwd, adj = contraction_fmas(dim, n, q, dim)
    return 2 * (2 * fwd + adj) + METRIC_DP_FLOPS[metric] * q ** dim


def grad_flops_per_element(dim, n, q, metric):
    fwd, adj = contraction_fmas(dim, n, q, dim)
    return 2 * (fwd + adj) + (METRIC_DP_FLOPS[metric] // 2) * q ** dim


def fused_flops_per_element(dim, n, q, metric):
    """Algorithmic flops of the gradient and the Hessian action at the same x
    in one pass: the Hessian action's work, a second adjoint contraction, and
    s P assembled at every point from the coefficients dP's evaluation
    already holds (dim^2 multiplies and dim^2 FMAs)."""
    _, adj = contraction_fmas(dim, n, q, dim)
    return hess_flops_per_element(dim, n, q, metric) + 2 * adj + 3 * dim * dim * q ** dim


def fused_executed_flops_per_element(dim, n, q, metric):
    """The same with the contractions the FP64 kernel runs (folded and
    normalised where they are)."""
    f = folded_contraction_flops(dim, n, q, dim)
    if f is None:
        return fused_flops_per_element(dim, n, q, metric)
    return hess_executed_flops_per_element(dim, n, q, metric) + f[1] + 3 * dim * dim * q ** dim


ELEM_SOURCES = ("tmop_device.cuh", "tmop_element.cuh", "tmop_kparams.h")
PAC_SOURCES = ("tmop_device.cuh", "tmop_pa_compact.cu", "tmop_pa_compact.h", "tmop_kparams.h")


def kernel_src_hash(files=ELEM_SOURCES) -> str:
    """Hash of a kernel's sources; ncu counters are reused only when it
    matches the hash recorded with them."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1807_09807_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def replica_value(t_local_s, units_per_step, steps, dist_mod=None, device="cpu"):
    """Whole-job throughput of N independent replicas (one per rank, no data
    exchange): every rank processed units_per_step * steps units, and the job
    took as long as the slowest rank. Returns (value, job seconds)."""
    import torch
    ws, t = 1, t_local_s
    if dist_mod is not None and dist_mod.is_initialized():
        ws = dist_mod.get_world_size()
        tt = torch.tensor([t_local_s], dtype=torch.float64, device=device)
        dist_mod.all_reduce(tt, op=dist_mod.ReduceOp.MAX)
        t = float(tt.item())
    return ws * units_per_step * steps / t, t


# ---------------------------------------------------------------- environment
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while the
    timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.25)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def measure_alu_peaks(tm, gpu_index, seconds=1.0):
    """FP64 and FP32 FMA throughput of this GPU (tmop_fma_peak: independent
    multiply-add chains on every SM, best of the timed launches), each kind
    repeated for about `seconds` while nvidia-smi samples the SM clock."""
    out = {}
    for name, kind in (("fp64", tm.PEAK_FP64), ("fp32", tm.PEAK_FP32), ("fp32x2", tm.PEAK_FP32X2)):
        best, best_ms = 0.0, None
        with ClockSampler(gpu_index) as clk:
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < seconds:
                g, ms = tm.fma_peak(kind)
                if g > best:
                    best, best_ms = g, ms
        out[name] = {"gflops": best, "launch_ms": best_ms, "clocks": clk.summary()}
    out["fp32_best"] = max(out["fp32"]["gflops"], out["fp32x2"]["gflops"])
    out["how"] = ("tmop_fma_peak: 1024 threads per SM, 8 independent multiply-add chains each, fixed "
                  "count; best of 3 timed launches (CUDA events), repeated for ~1 s under nvidia-smi sampling")
    return out


# ---------------------------------------------------------------- CPU oracle timing
def oracle_sample(m, budget_s: float = 12.0, chunk_slabs: int = 2):
    """Time the plain FP64 oracle (gradient + Hessian action) on whole z-slabs
    of elements of the same workload until budget_s has elapsed. Returns
    (quad-points/s, elements timed, seconds)."""
    import oracle
    p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, quad_kind=m.quad_kind)
    v = np.random.default_rng(11).standard_normal(m.x.shape)
    slab = m.nx[0] * m.nx[1] if m.dim == 3 else m.nx[0]
    chunk = slab * chunk_slabs
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and done < m.nelem:
        els = np.arange(done, min(done + chunk, m.nelem), dtype=np.int32)
        p.gradient(m.x, elems=els)
        p.hess_apply(m.x, v, elems=els)
        done += len(els)
    dt = time.perf_counter() - t0
    return done * m.Q / dt, done, dt


# The same timing on every host core: one spawned process per core, each with
# its own copy of the mesh and of the (single-threaded) oracle, each cycling
# over its own band of whole z-slabs for the time budget.
_ORC = {}


def _oracle_worker_init(name, seed):
    import oracle
    m = mg.make_mesh(name, seed)   # the seed the caller's mesh was drawn with: the same mesh
    p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, quad_kind=m.quad_kind)
    _ORC.update(m=m, p=p, v=np.random.default_rng(11).standard_normal(m.x.shape))


def _oracle_worker_run(task):
    e0, e1, budget_s, chunk = task
    m, p, v = _ORC["m"], _ORC["p"], _ORC["v"]
    done, e, t0 = 0, e0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        els = np.arange(e, min(e + chunk, e1), dtype=np.int32)
        p.gradient(m.x, elems=els)
        p.hess_apply(m.x, v, elems=els)
        done += len(els)
        e = e + chunk if e + chunk < e1 else e0
    return done * m.Q, time.perf_counter() - t0


class OraclePool:
    """Worker processes (spawned: the parent may hold a CUDA context) that time
    the oracle concurrently; rate() = all points done / the longest worker's
    time."""

    def __init__(self, m, procs=None):
        import multiprocessing as mp
        import oracle
        oracle.build()                 # compiled once, before the workers load it
        self.procs = procs or len(os.sched_getaffinity(0))
        self.m = m
        old = os.environ.get("OMP_NUM_THREADS")
        os.environ["OMP_NUM_THREADS"] = "1"   # for the workers (they copy the environment at start)
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init,
                                                       initargs=(m.name, m.seed))
        finally:
            if old is None:
                os.environ.pop("OMP_NUM_THREADS", None)
            else:
                os.environ["OMP_NUM_THREADS"] = old
        slab = m.nx[0] * m.nx[1] if m.dim == 3 else m.nx[0]
        nslab = m.nelem // slab
        self.bands = [(slab * (k * nslab // self.procs), slab * ((k + 1) * nslab // self.procs))
                      for k in range(self.procs)]
        self.chunk = slab

    def rate(self, budget_s):
        tasks = [(e0, e1, budget_s, self.chunk) for e0, e1 in self.bands if e1 > e0]
        res = self.pool.map(_oracle_worker_run, tasks, chunksize=1)
        qp = sum(r[0] for r in res)
        dt = max(r[1] for r in res)
        return qp / dt, qp, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_block(m):
    qps1, ne, dt1 = oracle_sample(m)
    pool = OraclePool(m)
    try:
        pool.rate(0.5)                 # every worker has built its mesh: the timed run overlaps fully
        qps, qp, dt = pool.rate(12.0)
    finally:
        pool.close()
    return {"value": qps, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
            "sample": f"gradient + Hessian action of the FP64 CPU oracle, one process per host core "
                      f"({pool.procs}), each on its own band of whole z-slabs of the same mesh, "
                      f"{qp / m.Q:.0f} elements in {dt:.1f} s",
            "single_thread": {"value": qps1, "unit": UNIT, "cores": 1,
                              "sample": f"the first {ne} of {m.nelem} elements (whole z-slabs), {dt1:.1f} s"}}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    m = make_workload(args.workload, accept_gpu=False)
    pool = OraclePool(m)
    try:
        for _ in range(args.warmup):
            pool.rate(0.5)
        total_qp, total_t = 0.0, 0.0
        for _ in range(args.steps):
            qps, qp, dt = pool.rate(max(2.0, 60.0 / max(args.steps, 1)))
            total_qp += qp
            total_t += dt
    finally:
        pool.close()
    value = total_qp / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(m, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                         "sample": "each step: gradient + Hessian action of the FP64 CPU oracle for a fixed time "
                                   f"budget, one process per host core ({pool.procs}), each on its own band of "
                                   "whole z-slabs of the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def make_workload(name, accept_gpu=True):
    accept = None
    if accept_gpu:
        import torch
        from paper_1807_09807_gb300 import tmop as tm

        def accept(mm):
            ctx = tm.Context.from_mesh(mm)
            rc, F, md = ctx.energy(torch.tensor(mm.x, device="cuda"))
            ctx.close()
            return md > 0
    return mg.make_mesh(name, 1, accept=accept)


def workload_config(m, args):
    return {"workload": f"{args.workload}: {m.dim}D order-{m.order} "
                        f"{'x'.join(str(v) for v in m.nx)} {'hexes' if m.dim == 3 else 'quads'}, "
                        f"{m.nq}^{m.dim} Gauss points, mu{m.metric}, W=I, jittered + "
                        f"{'trilinear shear' if m.dim == 3 else 'sine'}, boundary fixed",
            "elements": m.nelem, "quad_points": m.n_qp, "dofs": m.dim * m.nnode,
            "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU"}


def run_sharded(args):
    """The timed step (gradient + Hessian action) of the workload split into
    z-slabs over the ranks (paper_1807_09807_gb300/shard.py): each rank runs
    the element kernels on its slab, then one halo sum (NCCL send/recv of the
    shared node planes) per operator application. Total work is fixed
    (strong scaling); value = points of the whole mesh per second of the
    slowest rank. End to end: each rank uploads its slab's x and v from
    pinned host memory and downloads its g and y every step."""
    import torch
    import torch.distributed as dist

    from paper_1807_09807_gb300 import build as cuda_build
    from paper_1807_09807_gb300 import tmop as tm
    from paper_1807_09807_gb300.shard import ShardedOperator

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if rank == 0:
        cuda_build.build()
    dist.barrier()
    tm.load()
    m = make_workload(args.workload)
    prec = tm.FP64 if args.precision == "fp64" else tm.FP32_MIXED
    op = ShardedOperator(m, dist, precision=prec)
    vh_glob = np.random.default_rng(5).standard_normal(m.x.shape) * (1 - m.fixed)
    x = torch.tensor(op.mesh.x, device=dev)
    v = torch.tensor(op.part.to_local(vh_glob), device=dev)
    g, y = torch.empty_like(x), torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        op.gradient(x, out=g)
        op.hess_apply(x, v, out=y)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.fill_(1.0)
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    t_local = sum(a.elapsed_time(b) for a, b in evs) * 1e-3
    tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_dev = float(tt.item())
    value = m.n_qp * args.steps / t_dev
    # end to end: the slab's inputs up from pinned host memory, its outputs down
    xh, vh = x.cpu().pin_memory(), v.cpu().pin_memory()
    gh, yh = torch.empty_like(xh).pin_memory(), torch.empty_like(xh).pin_memory()
    e_steps = max(3, min(args.steps, 10))
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        x.copy_(xh, non_blocking=True)
        v.copy_(vh, non_blocking=True)
        step()
        gh.copy_(g, non_blocking=True)
        yh.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    te = torch.tensor([e0.elapsed_time(e1) * 1e-3], dtype=torch.float64, device=dev)
    dist.all_reduce(te, op=dist.ReduceOp.MAX)
    nbytes = x.numel() * 8
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64" if prec == tm.FP64 else "f32 (f64 reductions)", "data": "synthetic",
            "config": dict(workload_config(m, args), parallelism=f"z-slabs x{ws}, halo sum per application"),
            "clocks": clocks.summary(), "gpu_launches": 2 * args.steps,
            "e2e": {"value": m.n_qp * e_steps / float(te.item()), "unit": UNIT,
                    "h2d_bytes_per_step (rank 0)": 2 * nbytes, "d2h_bytes_per_step (rank 0)": 2 * nbytes,
                    "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes},
            "slabs": {"elements_rank0": op.mesh.nelem, "planes_shared": ws - 1}}), flush=True)
    op.close()
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1807_09807_gb300 import build as cuda_build
    from paper_1807_09807_gb300 import tmop as tm

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        cuda_build.build()
    if ws > 1:
        dist.barrier()
    tm.load()
    m = make_workload(args.workload)
    prec = tm.FP64 if args.precision == "fp64" else tm.FP32_MIXED
    ctx = tm.Context.from_mesh(m, precision=prec)
    x = torch.tensor(m.x, device=dev)
    v = torch.tensor(np.random.default_rng(5).standard_normal(m.x.shape), device=dev)
    g, y = torch.empty_like(x), torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # the step: g = dF/dx and y = H(x) v at the same x, through the one-pass
    # entry point (FP64: one element kernel); --separate, and the FP32-mixed
    # form (whose call runs the two kernels), time the two calls apart
    fused = not args.separate and prec == tm.FP64

    def step(ev=None):
        if fused:
            if ev is not None:
                ev[0].record(stream)
            ctx.gradient_hess_apply(x, v, g=g, y=y)
            if ev is not None:
                ev[1].record(stream)
            return
        ctx.gradient(x, out=g)
        if ev is not None:
            ev[0].record(stream)
        ctx.hess_apply(x, v, out=y)
        if ev is not None:
            ev[1].record(stream)

    if args.kernels_only and args.profile in ("newton", "newton_twolevel"):
        # one FP32-mixed Newton step of the workload (linearisation, MINRES with the stored-Hessian
        # product; newton_twolevel: preconditioned by Jacobi plus the coarse vertex correction)
        c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
        xn = x.clone()
        c32.newton_step(xn, precond=2 if args.profile == "newton_twolevel" else 0)
        torch.cuda.synchronize()
        c32.close()
        return 0
    if args.kernels_only and args.profile == "mlp":
        # W + K training steps of the proposal MLP on random bf16 inputs (batch 4096)
        from paper_1807_09807_gb300 import learned as L
        net = L.MLP(L.n_features(3), L.n_targets(3), 256, seed=0)
        gen = torch.Generator(device=dev)
        gen.manual_seed(3)
        X = (torch.randn((4096, net.ld), device=dev, generator=gen) * 0.5).to(torch.bfloat16).view(torch.int16)
        T = torch.randn((4096, L.n_targets(3)), device=dev, generator=gen) * 0.1
        loss = torch.zeros((), dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            net.gradients(X, T, loss)
            net.adam(1e-4)
        torch.cuda.synchronize()
        net.close()
        return 0
    if args.kernels_only and args.profile in ("pa", "pa32"):
        # the partially assembled product alone, in the form the Krylov loops run
        # it (y += H v; pa32: on FP32 vectors): one linearisation, then W + K products
        ctx.linearize(x)
        y.zero_()
        v32, y32 = v.to(torch.float32), torch.zeros(v.shape, dtype=torch.float32, device=v.device)
        for _ in range(args.warmup + args.steps):
            flush.fill_(1.0)
            if args.profile == "pa32":
                ctx.hess_apply_pa_add_f32(v32, y32)
            else:
                ctx.hess_apply_pa(v, out=y, accumulate=True)
        torch.cuda.synchronize()
        return 0
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if args.kernels_only:
        for _ in range(args.steps):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize()
        return 0

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if dev.index is not None else 0) as clocks:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(1.0)
            s0, s_h0, s_h1, s1 = evs[k]
            s0.record(stream)
            step(ev=(s_h0, s_h1))
            s1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    step_ms = [evs[k][0].elapsed_time(evs[k][3]) for k in range(args.steps)]
    hess_ms = [evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    value, t_dev = replica_value(sum(step_ms) * 1e-3, m.n_qp, args.steps, dist if ws > 1 else None, dev)

    # ---- end to end through the public API from pinned host buffers. Every
    # step uploads its x and v and downloads its g and y; with two buffer sets
    # the copies of one step run on two copy streams (host-to-device,
    # device-to-host) while the kernels of the neighbouring step compute.
    xh = torch.tensor(m.x).pin_memory()
    vh = torch.tensor(np.random.default_rng(5).standard_normal(m.x.shape)).pin_memory()
    gh = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    yh = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    vd = [torch.empty_like(x) for _ in range(2)]
    gd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(x) for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "g", "done", "out", "used")}
    e_steps = max(4, min(args.steps, 10))

    def e2e_step(k):
        b = k % 2
        if k >= 2:
            up.wait_event(ev["used"][b])           # step k-2 no longer reads xd[b], vd[b]
        with torch.cuda.stream(up):
            xd[b].copy_(xh, non_blocking=True)
            vd[b].copy_(vh, non_blocking=True)
            ev["in"][b].record(up)
        stream.wait_event(ev["in"][b])
        if k >= 2:
            stream.wait_event(ev["out"][b])        # step k-2's results have left gd[b], yd[b]
        if fused:
            ctx.gradient_hess_apply(xd[b], vd[b], g=gd[b], y=yd[b])
            ev["g"][b].record(stream)
        else:
            ctx.gradient(xd[b], out=gd[b])
            ev["g"][b].record(stream)
            ctx.hess_apply(xd[b], vd[b], out=yd[b])
        ev["done"][b].record(stream)
        ev["used"][b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev["g"][b])
            gh[b].copy_(gd[b], non_blocking=True)
            down.wait_event(ev["done"][b])
            yh[b].copy_(yd[b], non_blocking=True)
            ev["out"][b].record(down)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    # three timed repetitions of e_steps pipelined steps each; the median is
    # reported (the host side of the copies varies from run to run)
    e2e_runs = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(e_steps):
            e2e_step(k)
        stream.wait_stream(down)
        stream.wait_stream(up)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_runs.append(e0.elapsed_time(e1) * 1e-3)
    e2e_t = statistics.median(e2e_runs)
    # the downloaded results are those of the device-timed step (same x, v)
    bl = (e_steps - 1) % 2
    diff = max(float((gh[bl] - g.cpu()).abs().max() / g.abs().max()), float((yh[bl] - y.cpu()).abs().max() / y.abs().max()))
    nbytes = x.numel() * 8
    e2e = {"value": ws * m.n_qp * e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes,
           "d2h_bytes_per_step": 2 * nbytes, "pipelined": "two buffer sets, separate upload and download streams",
           "l2": "not flushed: every step moves 292 MB of fresh inputs and outputs (> 129 MB L2)",
           "max_rel_diff_vs_device_step": diff,
           "runs": [ws * m.n_qp * e_steps / t for t in e2e_runs], "reported": "median of the runs"}

    # ---- roofline of the dominant kernel (the Hessian action), against the
    # FMA throughput measured on this GPU (outside the timed region)
    alu = measure_alu_peaks(tm, dev.index if dev.index is not None else 0)
    args._alu_peaks = alu
    n = m.order + 1
    peak = (alu["fp64"]["gflops"] if prec == tm.FP64 else alu["fp32_best"]) / 1e3
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    traffic = {}
    if os.path.exists(tfile):
        with open(tfile) as f:
            traffic = json.load(f)

    def alu_roofline(kernel_ms, one_pass):
        """Roofline of the step's dominant kernel: the one-pass gradient +
        Hessian action, or (two kernels) the Hessian action."""
        flops = (fused_flops_per_element if one_pass else hess_flops_per_element)(m.dim, n, m.nq, m.metric) * m.nelem
        achieved = flops / (kernel_ms * 1e-3) / 1e12
        op = "OP_GRAD_HESS> (gradient + matrix-free Hessian action, one pass)" if one_pass \
            else "OP_HESS> (matrix-free Hessian action)"
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": None, "kernel": f"elem_kernel<{m.dim},{n},{m.nq},{'double' if prec == tm.FP64 else 'float'},"
                                        + op,
             "peak_source": ("measured: tmop_fma_peak " + ("DFMA" if prec == tm.FP64 else "FFMA / paired FFMA")
                             + f" at SM {alu['fp64' if prec == tm.FP64 else 'fp32']['clocks']['sm_mhz']} MHz"
                             + " (multiply-add chains on every SM, CUDA events)"),
             "peak_nominal": (FP64_PEAK_GFLOPS if prec == tm.FP64 else FP32_PEAK_GFLOPS) / 1e3,
             "frac_of_nominal": achieved / ((FP64_PEAK_GFLOPS if prec == tm.FP64 else FP32_PEAK_GFLOPS) / 1e3),
             "flops_per_launch": flops, "kernel_ms": kernel_ms,
             "timed": "CUDA events around the call: the output memsets and the kernel"}
        if prec == tm.FP64:
            # the kernel runs the contractions in the mirror basis: fewer flops than
            # the plain sum factorisation that flops_per_launch counts
            ex = (fused_executed_flops_per_element if one_pass else hess_executed_flops_per_element)(
                m.dim, n, m.nq, m.metric) * m.nelem
            r["executed_flops_per_launch"] = ex
            r["frac_executed"] = ex / (kernel_ms * 1e-3) / 1e12 / peak
            r["work"] = ("flops_per_launch: the plain sum-factorised contractions + the metric terms (the "
                         "algorithmic work); executed_flops_per_launch: what the folded (mirror-basis) kernel runs")
        tr = traffic.get(f"{args.workload}:{args.precision}" + (":fused" if one_pass else ""))
        # only counters taken on the kernel sources as they are now
        if tr and tr.get("kernel_src_sha256") == kernel_src_hash():
            r["traffic"] = tr["dram_bytes_per_launch"]
        return r

    one_pass = fused
    roofline = alu_roofline(statistics.mean(hess_ms), one_pass)
    # the same step as two kernels (gradient, then Hessian action), outside the timed region
    step_separate = None
    if fused and rank == 0:
        reps = max(3, min(args.steps, 10))
        sep_ms = _event_ms(lambda: (ctx.gradient(x, out=g), ctx.hess_apply(x, v, out=y)), reps, stream, flush)
        hv_ms = _event_ms(lambda: ctx.hess_apply(x, v, out=y), reps, stream, flush)
        step_separate = {"ms_per_step": sep_ms, "value": m.n_qp / (sep_ms * 1e-3), "unit": UNIT,
                         "hess_ms": hv_ms, "gradient_ms": sep_ms - hv_ms,
                         "form": "tmop_gradient then tmop_hess_apply (two element kernels)",
                         "roofline": alu_roofline(hv_ms, False) if prec == tm.FP64 else None}

    # ---- time to converged mesh, both precision forms (outside the timed region)
    # ---- partial assembly: linearize once, then the stored-Hessian product
    pa = None
    if rank == 0 and args.pa:
        pa = measure_pa(tm, m, x, v, y, flush, stream, args)
        pa["deterministic_sums"] = measure_deterministic(tm, m, x, v, y, flush, stream, args)

    # ---- the same step in the FP32-Hessian form (FP64 gradient, FP32 matrix-free
    # Hessian action: the 48^3 configuration's precision form), outside the timed region
    step_mixed = None
    if rank == 0 and prec == tm.FP64:
        step_mixed = measure_step_mixed(tm, m, x, v, y, flush, stream, args)

    # ---- time to converged mesh, both precision forms (outside the timed region)
    converge = None
    if args.converge and rank == 0:
        converge = time_to_converged(tm, m, dev, args)

    configs = None
    if args.configs and rank == 0:
        if converge is not None:
            args._c4_counts = (converge["fp64"]["newton"], converge["fp64"]["krylov"]) if args.workload == "c4" else None
        configs = newton_configs(tm, dev, args)

    learned = None
    if args.learned and rank == 0:
        learned = learned_proposal(tm, dev, args)
        learned["curved_boundary"] = learned_proposal(tm, dev, args, "c5curved", "c5curved", measure_step=False,
                                                      train_meshes=args.train_meshes_curved, coarse=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == tm.FP64 else "f32 (f64 reductions)",
            "data": "synthetic", "config": workload_config(m, args), "clocks": clocks.summary(),
            "e2e": e2e, "gpu_launches": (1 if one_pass else 2) * args.steps, "roofline": roofline, "alu_peaks": alu,
            "wall_s_timed_region": t_wall,
            "step_form": ("tmop_gradient_hess_apply: gradient and Hessian action in one element pass" if one_pass
                          else "tmop_gradient then tmop_hess_apply"),
        }
        if step_separate is not None:
            line["step_separate"] = step_separate
        if pa is not None:
            line["partial_assembly"] = pa
        if step_mixed is not None:
            line["step_fp32_hessian"] = step_mixed
        if converge is not None:
            line["time_to_converged"] = converge
        if configs is not None:
            line["newton_configs"] = configs
        if learned is not None:
            line["learned_proposal"] = learned
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_block(m)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _event_ms(fn, reps, stream, flush=None):
    """Average device time of fn over reps launches (L2 flushed before each)."""
    import torch
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def measure_pa(tm, m, x, v, y, flush, stream, args):
    """Linearize (once per Newton step) and the partially assembled Hessian
    action (once per Krylov iteration), FP64 and FP32, with the HBM roofline
    of the FP32 product. The product is timed in the form the Krylov solves
    run it, y += H v into a buffer their previous vector pass zeroed
    (tmop_hess_apply_pa_add: the product kernel alone); it reads the stored
    values (the 14-value compact record or the dim^2 (dim^2+1)/2 packed
    Hessian entries, FP32, per point) and v, and reads and writes y. The
    zeroing form (memset + kernel, tmop_hess_apply_pa) is timed beside it. In
    3D the packed form is also timed on the same mesh with mu302, whose
    Hessian is not written in (|T|^2, det T)."""
    import torch
    peaks = measured_peaks()
    out = {}
    forms = [("fp64", tm.FP64, None), ("fp32", tm.FP32_MIXED, None)]
    if m.dim == 3:
        forms.append(("fp32_packed_mu302", tm.FP32_MIXED, 302))
    for name, pf, metric in forms:
        c = tm.Context.from_mesh(m, precision=pf, metric=metric)
        c.linearize(x)
        c.hess_apply_pa(v, out=y)
        torch.cuda.synchronize()
        lin_ms = _event_ms(lambda: c.linearize(x), 2, stream, flush)
        reps = max(3, min(args.steps, 10))
        hv_ms = _event_ms(lambda: c.hess_apply_pa(v, out=y, accumulate=True), reps, stream, flush)
        hv0_ms = _event_ms(lambda: c.hess_apply_pa(v, out=y), reps, stream, flush)
        dd = m.dim * m.dim
        ns, _, elt = c.pa_layout()     # packed Hessian entries or compact record values per point
        compact = ns != dd * (dd + 1) // 2
        nbytes = m.n_qp * ns * elt + 3 * x.numel() * 8   # stored values + v read + y read and written
        n = m.order + 1
        fwd, adj = contraction_fmas(m.dim, n, m.nq, m.dim)
        flops = m.nelem * (2 * (fwd + adj) + 2 * dd * dd * m.Q)   # contractions + the d^2 x d^2 product
        ent = {"linearize_ms": lin_ms, "hess_pa_ms": hv_ms, "hess_pa_zeroing_ms": hv0_ms,
               "product_form": "y += H v on FP64 vectors (tmop_hess_apply_pa_add)", "bytes_per_launch": nbytes,
               "achieved_GBps": nbytes / (hv_ms * 1e-3) / 1e9, "achieved_TFLOPs": flops / (hv_ms * 1e-3) / 1e12}
        if pf == tm.FP64:
            alu = getattr(args, "_alu_peaks", None)
            pk = (alu["fp64"]["gflops"] if alu else FP64_PEAK_GFLOPS) / 1e3
            ent["roofline"] = {"bound": "alu", "achieved": ent["achieved_TFLOPs"], "peak": pk,
                               "unit": "TFLOP/s", "frac": ent["achieved_TFLOPs"] / pk,
                               "peak_source": "measured: tmop_fma_peak DFMA" if alu else "nominal (unit counts x clock)"}
            fo = folded_contraction_flops(m.dim, n, m.nq, m.dim)
            if fo is not None:   # the mirror-basis contractions the FP64 kernel runs
                ex = m.nelem * (fo[0] + fo[1] + 2 * dd * dd * m.Q)
                ent["roofline"]["executed_flops_per_launch"] = ex
                ent["roofline"]["frac_executed"] = ex / (hv_ms * 1e-3) / 1e12 / pk
        else:
            hbm = peaks.get("hbm_gbs", 6800.0)
            ent["roofline"] = {"bound": "hbm", "achieved": ent["achieved_GBps"], "peak": hbm, "unit": "GB/s",
                               "frac": ent["achieved_GBps"] / hbm,
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                               "kernel": f"pac_kernel<{n},{m.nq}> (compact records)" if compact
                               else f"elem_kernel<{m.dim},{n},{m.nq},float,OP_HESS_PA>", "traffic": None}
            ent["values_per_point"] = ns
            if metric is not None:
                ent["metric"] = metric
            # the form the FP32 contexts' MINRES runs: FP32 v and y (tmop_hess_apply_pa_add_f32)
            v32 = v.to(torch.float32)
            y32 = torch.zeros_like(v32)
            c.hess_apply_pa_add_f32(v32, y32)
            torch.cuda.synchronize()
            f32_ms = _event_ms(lambda: c.hess_apply_pa_add_f32(v32, y32), reps, stream, flush)
            b32 = m.n_qp * ns * elt + 3 * x.numel() * 4       # stored values + v read + y read and written (FP32)
            ent["fp32_vectors"] = {"hess_pa_ms": f32_ms, "bytes_per_launch": b32,
                                   "product_form": "y += H v on FP32 vectors (tmop_hess_apply_pa_add_f32, "
                                                   "the FP32 MINRES operator)",
                                   "achieved_GBps": b32 / (f32_ms * 1e-3) / 1e9,
                                   "frac": b32 / (f32_ms * 1e-3) / 1e9 / hbm}
            del v32, y32
            tfile = os.path.join(ROOT, "profiles", "traffic.json")
            if os.path.exists(tfile):
                with open(tfile) as f:
                    tr = json.load(f).get(f"{args.workload}:pa_fp32" + ("" if compact else "_packed"))
                if tr and tr.get("kernel_src_sha256") == kernel_src_hash(PAC_SOURCES if compact else ELEM_SOURCES):
                    ent["roofline"]["traffic"] = tr["dram_bytes_per_launch"]
        out[name] = ent
        c.close()
    return out


def measure_step_mixed(tm, m, x, v, y, flush, stream, args):
    """The benchmark step (gradient + one Hessian action, same mesh, L2
    flushed) in the FP32-Hessian form: FP64 gradient, FP32 Hessian action
    recomputed from x (matrix-free), FP64 reductions."""
    import torch
    c = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    g = torch.empty_like(x)
    c.gradient(x, out=g)
    c.hess_apply(x, v, out=y)
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 10))
    step_ms = _event_ms(lambda: (c.gradient(x, out=g), c.hess_apply(x, v, out=y)), reps, stream, flush)
    hv_ms = _event_ms(lambda: c.hess_apply(x, v, out=y), reps, stream, flush)
    c.close()
    return {"ms_per_step": step_ms, "value": m.n_qp / (step_ms * 1e-3), "unit": UNIT, "hess_ms": hv_ms,
            "gradient_ms": step_ms - hv_ms,
            "form": "FP64 gradient + FP32 Hessian action recomputed from x (pacr_kernel), FP64 reductions"}


def measure_deterministic(tm, m, x, v, y, flush, stream, args):
    """Cost of the colour-ordered (bitwise reproducible) nodal sums against
    the atomic ones: the timed step (FP64 gradient + recomputed Hessian
    action) and the FP32 stored-Hessian product, same inputs, L2 flushed."""
    import torch
    out = {}
    reps = max(3, min(args.steps, 10))
    for det in (False, True):
        c = tm.Context.from_mesh(m)
        c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
        if det:
            c.set_deterministic(True)
            c32.set_deterministic(True)
        g = torch.empty_like(x)
        c.gradient(x, out=g)
        c.hess_apply(x, v, out=y)
        c32.linearize(x)
        c32.hess_apply_pa(v, out=y)
        torch.cuda.synchronize()
        step_ms = _event_ms(lambda: (c.gradient(x, out=g), c.hess_apply(x, v, out=y)), reps, stream, flush)
        pa_ms = _event_ms(lambda: c32.hess_apply_pa(v, out=y), reps, stream, flush)
        out["colours" if det else "atomics"] = {"step_ms": step_ms, "fp32_pa_product_ms": pa_ms}
        c.close()
        c32.close()
    out["step_cost"] = out["colours"]["step_ms"] / out["atomics"]["step_ms"]
    out["pa_cost"] = out["colours"]["fp32_pa_product_ms"] / out["atomics"]["fp32_pa_product_ms"]
    out["colours_used"] = 2 ** m.dim
    return out


def time_to_converged(tm, m, dev, args):
    """Newton from the jittered mesh until |g| <= 1e-12 |g0| (Section 5
    tolerance): plain FP64, and FP32 Hessian action with FP64 gradient, line
    search and convergence test. Partially assembled Krylov operator."""
    import torch
    res_all = {}
    # plain FP64 (the paper's method as read), the FP32 Hessian-action form, and
    # that form with Jacobi-preconditioned MINRES (the diagonal of the stored
    # Hessians)
    # and both forms with the two-level preconditioner (Jacobi plus the exact
    # coarse correction on the element vertices)
    # (the FP32 forms run MINRES on FP32 vectors; "mixed_fp64_vectors" keeps FP64 ones;
    # "mixed_matrix_free[_cg]": the FP32 Hessian action recomputed from x at every product,
    # no linearisation, with MINRES or CG)
    arms = (("fp64", tm.FP64, 0, {}), ("mixed", tm.FP32_MIXED, 0, {}),
            ("mixed_fp64_vectors", tm.FP32_MIXED, 0, {"krylov_fp64": 1}), ("mixed_jacobi", tm.FP32_MIXED, 1, {}),
            ("fp64_twolevel", tm.FP64, 2, {}), ("mixed_twolevel", tm.FP32_MIXED, 2, {}),
            ("mixed_matrix_free", tm.FP32_MIXED, 0, {"matrix_free": 1}),
            ("mixed_matrix_free_cg", tm.FP32_MIXED, 0, {"matrix_free": 1, "krylov": "cg"}))
    for name, pf, pc, kw in arms:
        c = tm.Context.from_mesh(m, precision=pf)
        xc = torch.tensor(m.x, device=dev)
        F0 = c.energy(xc)[1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kw = dict(kw)
        kv = kw.pop("krylov", args.krylov)
        res = c.newton_solve(xc, max_newton=args.max_newton, krylov=kv, rtol=1e-12, precond=pc, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rep = res.report
        res_all[name] = {"seconds": dt, "status": tm.status_string(res.status), "newton": rep["iterations"],
                         "krylov": rep["krylov_iterations"], "F0": F0, "F": rep["F"],
                         "grad_rel": rep["grad_norm"] / max(rep["grad_norm0"], 1e-300), "min_detA": rep["min_detA"]}
        c.close()
    F64 = res_all["fp64"]["F"]
    for k in ("mixed", "mixed_fp64_vectors", "mixed_jacobi", "fp64_twolevel", "mixed_twolevel", "mixed_matrix_free",
              "mixed_matrix_free_cg"):
        res_all[f"{k}_vs_fp64_F_rel"] = abs(res_all[k]["F"] - F64) / abs(F64)
        res_all[f"speedup_{k}_over_fp64"] = res_all["fp64"]["seconds"] / res_all[k]["seconds"]
    return res_all


def oracle_call_seconds(m, budget_s=1.5):
    """Single-thread seconds of one oracle gradient and one Hessian action on
    the whole mesh, scaled from whole z-slabs (rows of elements in 2D) timed
    for about budget_s each."""
    import oracle
    p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, quad_kind=m.quad_kind)
    v = np.random.default_rng(11).standard_normal(m.x.shape)
    slab = m.nx[0] * m.nx[1] if m.dim == 3 else m.nx[0]
    out = {}
    for name, call in (("gradient", lambda els: p.gradient(m.x, elems=els)),
                       ("hess_apply", lambda els: p.hess_apply(m.x, v, elems=els))):
        call(np.arange(0, min(slab, m.nelem), dtype=np.int32))   # warm-up (tables, first touch)
        done, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s and done < m.nelem:
            els = np.arange(done, min(done + slab, m.nelem), dtype=np.int32)
            call(els)
            done += len(els)
        out[name] = (time.perf_counter() - t0) * m.nelem / done
    return out


def newton_configs(tm, dev, args):
    """Newton to |g| <= 1e-12 |g0| on the smaller configurations (C1-C3) on
    the GPU, plain FP64 and the FP32 Hessian-action form (each also with the
    two-level preconditioner) and the FP32-bulk form, beside the CPU
    oracle: its own Newton measured on C1 (single thread); for C2-C4 the CPU
    time is extrapolated from single-thread per-call times of the oracle
    (gradient, matrix-free Hessian action) times the GPU run's Newton and
    MINRES counts, a lower bound (line-search energies not counted)."""
    import torch
    out = {}
    for name in ("c1", "c2", "c3", "c4"):
        m = mg.make_mesh(name, 1)
        ent = {"elements": m.nelem, "quad_points": m.n_qp, "metric": m.metric}
        # FP32-bulk (every element kernel FP32, reductions FP64): its FP32 gradient
        # bounds |g| / |g0| near 1e-6, so it stops there; F against the FP64 F
        # and the two-level preconditioner (Jacobi + exact coarse vertex correction) in FP64 and FP32-mixed
        forms = (("fp64", tm.FP64, 1e-12, 0), ("mixed", tm.FP32_MIXED, 1e-12, 0), ("bulk", tm.FP32_BULK, 1e-6, 0),
                 ("fp64_twolevel", tm.FP64, 1e-12, 2), ("mixed_twolevel", tm.FP32_MIXED, 1e-12, 2)) \
            if name != "c4" else ()
        for form, pf, rtol, pc in forms:
            c = tm.Context.from_mesh(m, precision=pf)
            xc = torch.tensor(m.x, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = c.newton_solve(xc, max_newton=args.max_newton, rtol=rtol, precond=pc)
            torch.cuda.synchronize()
            rep = res.report
            ent[f"gpu_{form}"] = {"seconds": time.perf_counter() - t0, "status": tm.status_string(res.status),
                                  "newton": rep["iterations"], "krylov": rep["krylov_iterations"], "F": rep["F"],
                                  "rtol": rtol, "grad_rel": rep["grad_norm"] / max(rep["grad_norm0"], 1e-300)}
            if form != "fp64" and "gpu_fp64" in ent:
                F64 = ent["gpu_fp64"]["F"]
                F0 = c.energy(torch.tensor(m.x, device=dev))[1]
                ent[f"gpu_{form}"]["F_diff_over_F0"] = abs(rep["F"] - F64) / abs(F0)
            c.close()
        calls = oracle_call_seconds(m)
        ent["cpu_oracle_call_seconds"] = calls
        counts = ent.get("gpu_fp64") or {"newton": None, "krylov": None}
        if name == "c4":   # the main benchmark's FP64 Newton counts
            counts = {"newton": args._c4_counts[0], "krylov": args._c4_counts[1]} if getattr(args, "_c4_counts", None) \
                else counts
        if counts["newton"] is not None:
            est = counts["newton"] * calls["gradient"] + counts["krylov"] * calls["hess_apply"]
            ent["cpu_oracle_newton_seconds_extrapolated"] = est
            if "gpu_fp64" in ent:
                ent["speedup_gpu_fp64_over_cpu_extrapolated"] = est / ent["gpu_fp64"]["seconds"]
                ent["speedup_gpu_mixed_over_cpu_extrapolated"] = est / ent["gpu_mixed"]["seconds"]
        if name == "c1":
            import oracle
            p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric,
                               quad_kind=m.quad_kind)
            t0 = time.perf_counter()
            rc, xo, hist = p.newton(m.x, max_newton=args.max_newton, rtol=1e-12)
            dt = time.perf_counter() - t0
            ent["cpu_oracle_newton"] = {"seconds": dt, "status": int(rc), "newton": len(hist) - 1,
                                        "krylov": int(hist[1:, 4].sum()), "F": float(hist[-1, 0])}
            ent["speedup_gpu_fp64_over_cpu_measured"] = dt / ent["gpu_fp64"]["seconds"]
        out[name] = ent
    return out


def mlp_gemm_flops(net, batch):
    """Tensor-core FLOPs of one training step (forward + backward GEMMs) on
    the padded shapes the kernels run: input K1, hidden H, output N3."""
    K1, H, N3 = net.ld, net.hidden, 64
    fwd = K1 * H + H * H + H * N3
    bwd = N3 * H + H * N3 + H * H + H * H + H * K1   # dW3, dH2, dW2, dH1, dW1
    return 2 * batch * (fwd + bwd)


def mlp_step_roofline(L, net, X, T, reps=20):
    """One training step (loss gradients + Adam) of the proposal MLP at batch
    4096, CUDA-event timed, against the measured dense bf16 tensor peak. The
    GEMMs are small (K <= 4096), so the step is bound by latency and launches,
    not by the tensor cores; the fraction says how far."""
    import torch
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        net.gradients(X, T, loss)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        net.gradients(X, T, loss)
        net.adam(1e-12)
    b.record(stream)
    torch.cuda.synchronize()
    ms_eager = a.elapsed_time(b) / reps
    # the same step captured once in a CUDA graph (the Adam step count is on
    # the device) and replayed, as the training loop runs it
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side), torch.cuda.graph(g, stream=side):
        net.gradients(X, T, loss)
        net.adam(1e-12)
    stream.wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    flops = mlp_gemm_flops(net, X.shape[0])
    peak = measured_peaks().get("bf16_tflops", 1877.0)
    tf = flops / (ms * 1e-3) / 1e12
    return {"batch": int(X.shape[0]), "ms": ms, "ms_without_graph": ms_eager, "gemm_flops": flops,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "kernel": "k_gemm_tma (tcgen05.mma kind::f16, 128x64 tiles, 4-stage TMA ring, "
                                   "split-K for the weight gradients)",
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)"}}


def prop_seconds(L, net, m, ctx, x0, fx, coarse):
    """Wall time of one proposal (features, network, candidate checks)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.propose(net, m, ctx, x0, fx, coarse=coarse)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def learned_proposal(tm, dev, args, train_preset="c5", apply_preset="c5apply", measure_step=True, train_meshes=None,
                     coarse=False):
    """Train the proposal MLP on Newton-converged displacements of seeded
    32x32 order-3 meshes (mu2, jitter 0.15h), then on unseen meshes compare
    plain FP64 Newton from the jittered mesh with the FP32 form started from
    the proposal (with its fallback). Same absolute target |g| <= 1e-12
    |g(x0)| for both. Presets: the unit square (c5 / 128x128 c5apply, the
    optimum is the uniform grid) or the curved top boundary (c5curved, train
    and apply at 32x32: the optimum moves ~6 h from the mapped lattice; with
    coarse, the network works from the coarse stage's mesh: the element-vertex
    problem solved and interpolated, see learned.coarse_stage)."""
    import torch
    from paper_1807_09807_gb300 import learned as L
    t0 = time.perf_counter()
    train_meshes = args.train_meshes if train_meshes is None else train_meshes
    ds = L.make_dataset(n_meshes=train_meshes, seed0=1000, chunk=50, preset=train_preset, coarse=coarse)
    t_data = time.perf_counter() - t0
    net = L.MLP(L.n_features(3), L.n_targets(3), 256, seed=0)
    t0 = time.perf_counter()
    hist = L.train(net, ds, epochs=args.train_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"train_meshes": train_meshes, "train_samples": int(ds.X.shape[0]), "data_seconds": t_data,
           "train_seconds": t_train, "train_loss_first_last": [hist[0], hist[-1]], "apply": []}
    for seed in (5000, 5001):
        m = mg.make_mesh(apply_preset, seed)
        c64 = tm.Context.from_mesh(m)
        c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
        x0 = torch.tensor(m.x, device=dev)
        fx = torch.tensor(m.fixed, device=dev)
        F0 = c64.energy(x0)[1]
        g0 = float(torch.linalg.norm(c64.gradient(x0)))
        atol = 1e-12 * g0
        for c in (c64, c32):   # first-use work (workspace, graph capture) outside the timed solves
            c.newton_solve(x0.clone(), max_newton=1, rtol=1e-30, atol=atol)
        xa = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ra = c64.newton_solve(xa, max_newton=40, rtol=1e-30, atol=atol)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        # the FP32 form without the proposal (from x0): separates the
        # proposal's own gain from the precision form's
        xc = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc_ = c32.newton_solve(xc, max_newton=40, rtol=1e-30, atol=atol)
        torch.cuda.synchronize()
        tc = time.perf_counter() - t0
        coarse_only = None
        if coarse:   # the coarse stage alone, no network
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xk, _ = L.coarse_stage(m, x0, fx)
            rk = c32.newton_solve(xk, max_newton=40, rtol=1e-30, atol=atol)
            torch.cuda.synchronize()
            coarse_only = {"seconds": time.perf_counter() - t0, "status": tm.status_string(rk.status),
                           "newton": rk.report["iterations"], "krylov": rk.report["krylov_iterations"],
                           "F": rk.report["F"]}
        t0 = time.perf_counter()
        prop = L.propose(net, m, c32, x0, fx, coarse=coarse)
        xb = prop.x.clone()
        rb = c32.newton_solve(xb, max_newton=40, rtol=1e-30, atol=atol)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        # both FP32 starts again with the two-level preconditioner
        tl = {}
        for arm, xs in (("fp32_twolevel", x0), ("fp32_learned_twolevel", prop.x)):
            xx = xs.clone()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rr = c32.newton_solve(xx, max_newton=40, rtol=1e-30, atol=atol, precond=2)
            torch.cuda.synchronize()
            tl[arm] = {"seconds": time.perf_counter() - t1 + (0.0 if arm == "fp32_twolevel" else prop_seconds(L, net, m, c32, x0, fx, coarse)),
                       "status": tm.status_string(rr.status), "newton": rr.report["iterations"],
                       "krylov": rr.report["krylov_iterations"], "F": rr.report["F"]}
        out["apply"].append({
            "mesh": f"{m.nx[0]}x{m.nx[1]} order-3 quads ({apply_preset}), seed {seed}", "F0": F0,
            "fp64_plain": {"seconds": ta, "status": tm.status_string(ra.status), "newton": ra.report["iterations"],
                           "krylov": ra.report["krylov_iterations"], "F": ra.report["F"]},
            "fp32_plain": {"seconds": tc, "status": tm.status_string(rc_.status), "newton": rc_.report["iterations"],
                           "krylov": rc_.report["krylov_iterations"], "F": rc_.report["F"]},
            "fp32_coarse_only": coarse_only,
            "fp32_learned": {"seconds": tb, "status": tm.status_string(rb.status), "proposal_used": prop.used,
                             "proposal_coarse_stage": prop.coarse,
                             "proposal_scale": prop.scale, "F_proposal": prop.F, "newton": rb.report["iterations"],
                             "krylov": rb.report["krylov_iterations"], "F": rb.report["F"],
                             "min_detA": rb.report["min_detA"]},
            **tl,
            "F_diff_over_F0": abs(ra.report["F"] - rb.report["F"]) / F0,
            "speedup": ta / tb,                       # FP32 + proposal over plain FP64
            "speedup_proposal_alone": tc / tb,        # FP32 + proposal over FP32 from x0
            "speedup_fp32_alone": ta / tc})
        c64.close()
        c32.close()
    # solves of this kind that pay back data generation and training
    saved = [a["fp32_plain"]["seconds"] - a["fp32_learned"]["seconds"] for a in out["apply"]]
    mean_saved = sum(saved) / len(saved)
    out["amortisation"] = {"setup_seconds": t_data + t_train, "saved_seconds_per_solve_vs_fp32_plain": mean_saved,
                           "solves_to_pay_back": (t_data + t_train) / mean_saved if mean_saved > 0 else None}
    if measure_step:
        out["mlp_step"] = mlp_step_roofline(L, net, ds.X[:4096], ds.T[:4096])   # after the proposals: it steps Adam
    net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c4", choices=sorted(mg.PRESETS))
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--krylov", choices=["minres", "cg"], default="minres")
    ap.add_argument("--max-newton", type=int, default=12)
    ap.add_argument("--no-converge", dest="converge", action="store_false")
    ap.add_argument("--no-pa", dest="pa", action="store_false")
    ap.add_argument("--no-learned", dest="learned", action="store_false")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the Newton runs on C1-C3 and the oracle per-call timings")
    ap.add_argument("--train-meshes", type=int, default=2000)
    ap.add_argument("--train-epochs", type=int, default=15)
    ap.add_argument("--train-meshes-curved", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels-only", action="store_true")
    ap.add_argument("--separate", action="store_true",
                    help="time the step as two kernels (tmop_gradient, tmop_hess_apply) instead of the one-pass call")
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1: split the workload's elements into z-slabs, one per rank, with a halo "
                         "sum of the shared node planes per operator application (strong scaling) instead "
                         "of N independent replicas")
    ap.add_argument("--profile", choices=["step", "pa", "pa32", "mlp", "newton", "newton_twolevel"], default="step",
                    help="with --kernels-only: the timed step (gradient + Hessian action), the partially "
                         "assembled Hessian action alone (pa32: on FP32 vectors, with --precision mixed), "
                         "training steps of the proposal MLP, or one "
                         "FP32-mixed Newton step (newton_twolevel: with the two-level preconditioner)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if not args.kernels_only else args.warmup
    if args.impl == "reference":
        return run_reference(args)
    if args.shard:
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
