"""Benchmark: approximate contraction of a frozen tree on GB300 (one JSON line).

One step = one pass of the whole hot path (schedule expansion cached, every
contraction, compression, rescale and the final read-out) over one batch of
instances, inputs resident in HBM.  value = log|Z| evaluations per second
(instances / step time) on the fastest arithmetic form that meets the metric's
gate; e2e = the same through the C ABI with the inputs copied from pinned host
memory and the results read back every step.

Workloads (--workload):
  normal32  (default) 32x32 open square lattice, D = 4, entries i.i.d.
            Normal(0.2, 1), 8 independent seeds per GPU, boundary-row tree,
            chi = 64.  Its truncated result is rounding-chaotic (a 1e-15
            change of one input moves ln|Z| by ~1e-4 relative), so the gate
            of each reduced-precision form is judged on a 16x16 calibration
            batch of the same shapes, where FP64 results are well defined.
  ising64   64x64 open square lattice Ising model, J = 1, the beta sweep
            beta_t = 0.2 + 0.5 t / 255; a step is one batch of --batch betas
            (default 32, every 8th value of the sweep, plus the betas that
            have stored oracle values), chi = 128.  Each form's error is
            measured against the stored oracle values; the gate at each beta
            is max(1e-6, 4 x the oracle's own rounding spread there).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload normal32|ising64] [--batch B]
Multi-GPU (torchrun): every rank contracts its own instances (weak scaling,
no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "log Z evals/sec & contraction TFLOP/s vs plain FP64 GPU form at logZ rel err≤1e-6"
UNIT = "evals/s"
GATE = 1e-6

# DRAM bytes (read + write) of one launch of the FP64 polish (block_jacobi_kernel<double>)
# on 8 cores of 256 x 256, from one Nsight Compute capture; valid only for the kernel
# source it was taken on (sha256 prefix of csrc/k_svd.cu), else the line reports null.
JACOBI_TRAFFIC = {"bytes": 4.550912e6, "k_svd_sha": "592d07a2ffbb6bcd",
                  "source": "profiles/block_jacobi_kernel_f64_12x12_d4_chi64_batch8.md"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def source_sha(rel: str) -> str:
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# workloads


class Normal32:
    name = "normal32"
    L, D, CHI, N = 32, 4, 64, 8
    CAL_L, CAL_N = 16, 4

    def __init__(self, args):
        self.N = args.batch or self.N
        self.L = getattr(args, "L", 0) or self.L

    def describe(self):
        return (f"{self.L}x{self.L} open square lattice, D={self.D}, entries i.i.d. Normal(0.2,1), "
                f"{self.N} seeds per GPU, boundary-row tree, chi={self.CHI}")

    def tree(self):
        from tn_inputs import trees as tr
        return tr.boundary_rows(self.L, self.L)

    def nets(self, rank):
        from tn_inputs import networks as nw
        n, edges = nw.square_lattice(self.L, self.L)
        return [nw.random_network(n, edges, self.D, seed=rank * self.N + s) for s in range(self.N)]

    def cpu_net(self, idx):
        from tn_inputs import networks as nw
        n, edges = nw.square_lattice(self.L, self.L)
        return nw.random_network(n, edges, self.D, seed=idx)

    def trees(self, ctx, torch, net_ids, nets):
        """Tree builders on the benchmark batch (Algorithm 3's loop closed on the GPU): the
        boundary rows, the hyper-searched Span tree and the Greedy tree with the SI's max
        input reduction; per tree the traced cost C (the SI's units) and one eager FP64 pass."""
        from tn_inputs import trees as tr
        out = {}
        b = nets[0]
        for name, tree in (("boundary rows", tr.boundary_rows(self.L, self.L)),
                           ("span (hyper-searched, late)", tr.span(b.bonds, b.bond_dims, **tr.span_square_params())),
                           ("greedy (SI max reduction)", tr.greedy(b.bonds, b.bond_dims, self.CHI,
                                                                    **tr.greedy_front_params(self.CHI)))):
            cost = tr.trace_cost(b.bonds, b.bond_dims, tree, self.CHI)
            try:
                ids = [ctx.load_tree(nid, tree) for nid in net_ids]
                ctx.set_graph_mode(False)
                ctx.contract(ids, self.CHI)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lz, _ = ctx.contract(ids, self.CHI)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) * 1e3
            except RuntimeError as e:  # a tree whose plan does not fit is reported, not fatal
                out[name] = {"traced_cost": cost["total"], "traced_peak_elements": cost["peak"], "error": str(e)}
                continue
            finally:
                ctx.set_graph_mode(True)
            out[name] = {"traced_cost": cost["total"], "traced_peak_elements": cost["peak"], "pass_ms": ms,
                         "evals_per_s": len(ids) / (ms / 1e3), "logabsz_instance0": float(lz[0])}
        return out

    def cpu_rows(self):
        return 8

    def forms(self, ctx, torch, ids):
        """Each reduced-precision form on a 16x16 calibration batch (same D, chi, shapes per
        compression), error relative to the FP64 form there; the FP64 form's own error is 0."""
        from tn_inputs import networks as nw
        from tn_inputs import trees as tr
        n, edges = nw.square_lattice(self.CAL_L, self.CAL_L)
        tree = tr.boundary_rows(self.CAL_L, self.CAL_L)
        cal = [ctx.load_tree(ctx.load_network(nw.random_network(n, edges, self.D, seed=1000 + s)), tree)
               for s in range(self.CAL_N)]
        out = {"how": f"error on a {self.CAL_L}x{self.CAL_L} calibration batch ({self.CAL_N} seeds, same D and chi) "
                      f"against the FP64 form; speed on the benchmark batch",
               "gate_rel_err": GATE}
        ref = None
        for prec in ("f64", "tf32x3", "tf32", "bf16"):
            lz, _ = ctx.contract(cal, self.CHI, prec)
            if ref is None:
                ref = lz
            err = float(max(abs(a - b) / abs(b) for a, b in zip(lz, ref)))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.contract(ids, self.CHI, prec)
            torch.cuda.synchronize()
            out[prec] = {"evals_per_s": len(ids) / (time.perf_counter() - t0), "max_rel_err": err,
                         "meets_gate": bool(err <= GATE)}
        return out


class Ising64:
    name = "ising64"
    L, CHI, SWEEP = 64, 128, 256

    def __init__(self, args):
        self.B = args.batch or 32
        self.form_list = [f for f in (getattr(args, "forms", "") or "f64,tf32x3,tf32,bf16").split(",") if f]
        with open(os.path.join(ROOT, "tests", "golden", "ising64_chi128.json")) as f:
            self.gold = json.load(f)["entries"]

    def describe(self):
        return (f"{self.L}x{self.L} open square lattice Ising, J=1, beta sweep 0.2..0.7 ({self.SWEEP} values), "
                f"batch of {self.B} betas per GPU per step, boundary-row tree, chi={self.CHI}")

    def betas(self, rank):
        from tn_inputs import networks as nw
        sweep = nw.beta_sweep(self.SWEEP)
        ts = [e["t"] for e in self.gold]
        step = max(1, self.SWEEP // self.B)
        for t in range(rank % step, self.SWEEP, step):
            if len(ts) >= self.B:
                break
            if t not in ts:
                ts.append(t)
        return [float(sweep[t]) for t in ts[:self.B]]

    def tree(self):
        from tn_inputs import trees as tr
        return tr.boundary_rows(self.L, self.L)

    def nets(self, rank):
        from tn_inputs import networks as nw
        n, edges = nw.square_lattice(self.L, self.L)
        return [nw.ising_network(n, edges, b) for b in self.betas(rank)]

    def cpu_net(self, idx):
        from tn_inputs import networks as nw
        n, edges = nw.square_lattice(self.L, self.L)
        return nw.ising_network(n, edges, float(nw.beta_sweep(self.SWEEP)[(idx * 37) % self.SWEEP]))

    def cpu_rows(self):
        return 8

    def forms(self, ctx, torch, ids):
        """Each form on the benchmark batch itself, error against the stored oracle values."""
        out = {"how": "error against the stored oracle values at the batch's golden betas; gate at each beta = "
                      "max(1e-6, 4 x the oracle's rounding spread there)", "gate_rel_err": GATE,
               "band": {"%.4f" % e["beta"]: max(GATE, 4 * e["spread_rel"]) for e in self.gold}}
        ng = len(self.gold)
        for prec in self.form_list:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lz, _ = ctx.contract(ids, self.CHI, prec)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            errs = [abs(a - e["logabsz"]) / abs(e["logabsz"]) for a, e in zip(lz[:ng], self.gold)]
            ok = all(x <= max(GATE, 4 * e["spread_rel"]) for x, e in zip(errs, self.gold))
            out[prec] = {"evals_per_s": len(ids) / dt, "max_rel_err": max(errs), "rel_errs": errs,
                         "meets_gate": bool(ok)}
        return out


WORKLOADS = {"normal32": Normal32, "ising64": Ising64}


# ---------------------------------------------------------------------------


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tn_bench_clocks_{os.getpid()}_{device_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        return parse_clocks(self.path)


def parse_clocks(path: str):
    try:
        rows = [ln.strip().split(",") for ln in open(path) if ln.strip()]
    except OSError:
        return None
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            sm.append(float(r[1]))
            mx.append(float(r[2]))
        except (ValueError, IndexError):
            continue
        for name, val in zip(names, r[5:9]):
            if val.strip().lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    """(rank, world, local_rank) from the torchrun environment; initialises the group for N > 1."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline): bounded samples in spawned processes


def _oracle_prefix(args):
    wname, idx, n_ops = args
    sys.path.insert(0, ROOT)
    from tn_inputs.formats import Tree
    from oracle import approx
    wl = WORKLOADS[wname](argparse.Namespace(batch=0))
    net = wl.cpu_net(idx)
    tree = wl.tree()
    t0 = time.time()
    try:
        approx.contract(net, Tree(tree.n_inputs, tree.ops[:n_ops]), wl.CHI)
    except ValueError:
        pass  # the prefix leaves open tensors: expected
    return time.time() - t0


def oracle_sample(wl, rows: int = 0, cores: int = 0):
    """The oracle on the first `rows` boundary rows of the tree, one instance per host core.

    Returns (evals/s extrapolated by the traced cost, cores used, description).
    """
    import multiprocessing as mp
    from tn_inputs import trees as tr
    from tn_inputs.formats import Tree
    tree = wl.tree()
    net0 = wl.cpu_net(0)
    full = tr.trace_cost(net0.bonds, net0.bond_dims, tree, wl.CHI)["total"]
    rows = rows or wl.cpu_rows()
    n_ops = (2 * wl.L - 1) * rows
    part = tr.trace_cost(net0.bonds, net0.bond_dims, Tree(tree.n_inputs, tree.ops[:n_ops]), wl.CHI)["total"]
    cores = cores or host_cores()
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"   # inherited by the spawned workers: one BLAS thread each
    try:
        t0 = time.time()
        with mp.get_context("spawn").Pool(cores) as pool:
            times = pool.map(_oracle_prefix, [(wl.name, s, n_ops) for s in range(cores)])
        wall = time.time() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    frac = part / full
    evals = cores * frac / wall
    desc = (f"oracle on the first {n_ops} tree ops ({100 * frac:.1f}% of the traced cost) of {cores} instances, "
            f"one process per host core ({cores} of {os.cpu_count()}), OPENBLAS_NUM_THREADS=1; evals/s = instances "
            f"x fraction / wall ({wall:.1f} s wall, mean {sum(times) / len(times):.1f} s per instance)")
    return evals, cores, desc


def fp64_peak_tflops(torch, device):
    """FP64 rate measured in this run: a cuBLAS DGEMM 8192^3 (best of 3, CUDA events)."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    c = a @ b
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    from paper_2206_07044_gb300 import Context, build
    build.build()
    wl = WORKLOADS[args.workload](args)
    stream = torch.cuda.current_stream(device)
    cache = os.path.join(tempfile.gettempdir(), f"tn_tune_{wl.name}_gpu{local}.txt")
    ctx = Context(local, stream=stream, tuner_cache=cache if args.tune else None, split_batches=args.split)
    nets = wl.nets(rank)
    tree = wl.tree()
    net_ids = [ctx.load_network(x) for x in nets]
    ids = [ctx.load_tree(nid, tree) for nid in net_ids]
    nb = len(ids)
    stats = ctx.plan_stats(ids[0], wl.CHI, args.prec)
    # cpu baseline first (spawned pool, before more GPU work), rank 0 only, N = 1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample(wl)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    def step():
        return ctx.contract(ids, wl.CHI, args.prec)

    def eager_pass_ms():
        ctx.set_graph_mode(False)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ctx.set_graph_mode(True)
        return a.elapsed_time(b)

    # launch-shape autotuner: one eager pass with the built-in rules, the tuning
    # (cached in a file for later runs), one eager pass with the tuned shapes
    tuner = None
    if args.tune:
        untuned = eager_pass_ms()
        t0 = time.perf_counter()
        shapes = ctx.autotune(ids, wl.CHI, args.prec)
        tune_s = time.perf_counter() - t0
        tuned = eager_pass_ms()
        tuner = {"untuned_pass_ms": untuned, "tuned_pass_ms": tuned, "gain": untuned / tuned,
                 "shapes_tuned": shapes, "tune_s": tune_s, "cache": cache,
                 "how": "one eager pass each (CUDA events), before the warm-up; the timed steps use the tuned shapes"}

    # warm-up: the first pass runs eagerly, the second captures the schedule as a
    # CUDA graph, later passes replay it
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(device)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            lz, sg = step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(device)
    ms = e0.elapsed_time(e1) / args.steps
    graph = ctx.graph_info()
    ms_max = max_over_ranks(ms, device)
    # per-kernel device times: one more pass with events around every launch
    # (eager launches, one stream), after the timed region
    ctx.profile(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    fam = ctx.kernel_times()
    ctx.profile(False)
    value = world * nb / (ms_max / 1e3)

    # end to end: pinned host inputs -> device, contraction, results -> host, every step
    pinned = [[torch.from_numpy(np.ascontiguousarray(d)).pin_memory() for d in x.data] for x in nets]
    h2d = sum(int(t.numel()) * 8 for x in pinned for t in x)
    d2h = nb * (8 + 4)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    barrier(device)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for nid, x in zip(net_ids, pinned):
            ctx.set_network_data(nid, x)
        lz2, sg2 = step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, device)

    # the plain FP64 form: the same contraction, one instance per call (no batching),
    # timed over several calls after one untimed call
    plain = forms = trees_leg = None
    if rank == 0 and not args.no_forms:
        ctx.contract(ids[:1], wl.CHI, "f64")
        torch.cuda.synchronize()
        calls = args.plain_calls
        t0 = time.perf_counter()
        for q in range(calls):
            ctx.contract(ids[q % nb:q % nb + 1], wl.CHI, "f64")
        torch.cuda.synchronize()
        plain_s = (time.perf_counter() - t0) / calls
        plain = {"value": 1.0 / plain_s, "unit": UNIT, "ms_per_eval": plain_s * 1e3, "calls": calls,
                 "how": "one instance per tn_contract_approx call, FP64, same workload"}
        forms = wl.forms(ctx, torch, ids)
        trees_leg = wl.trees(ctx, torch, net_ids, nets) if hasattr(wl, "trees") and not args.no_trees else None
    fp64_peak = fp64_peak_tflops(torch, device) if rank == 0 else None

    if rank != 0:
        return
    # roofline of the dominant kernel family (device time share inside the timed region)
    fam_sorted = sorted(fam, key=lambda r: -r[2])
    top = [r for r in fam_sorted if not r[0].startswith("sweeps:")][0]
    algo = {"jacobi_f64": stats["svd_flops"], "qr_f64": stats["qr_flops"], "gemm_f64": stats["gemm_flops"]}
    launches_per_step = {name: nl for name, nl, _ in fam}
    name, nl, tot_ms = top
    avg_ms = tot_ms / nl
    roof = None
    if name in algo:
        flops_launch = algo[name] * nb / max(launches_per_step[name], 1)
        achieved = flops_launch / (avg_ms * 1e-3) / 1e12
        traffic, tsrc = None, None
        if (name == "jacobi_f64" and wl.name == "normal32" and nb == 8 and
                JACOBI_TRAFFIC["k_svd_sha"] == source_sha("paper_2206_07044_gb300/csrc/k_svd.cu")):
            traffic, tsrc = JACOBI_TRAFFIC["bytes"], JACOBI_TRAFFIC["source"]
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": traffic, "traffic_source": tsrc,
                "peak_source": "FP64 rate measured in this run (cuBLAS DGEMM 8192^3, best of 3)",
                "peak_unit_counts": 152 * 2 * 2 * 2.07e9 / 1e12,
                "work": "algorithmic FLOPs of the paper's counts (SVD 4mn^2-4/3n^3, QR 2mn^2-2/3n^3, GEMM 2mnk) "
                        "over the family's launches",
                "share_of_step": tot_ms / prof_ms,
                "timing": "CUDA events around each launch of one profiled pass (eager, one stream)"}
    gflop_step = (stats["gemm_flops"] + stats["qr_flops"] + stats["svd_flops"]) * nb * world / 1e9
    gated = None
    if forms:
        ok = [p for p in ("f64", "tf32x3", "tf32", "bf16") if isinstance(forms.get(p), dict) and forms[p].get("meets_gate")]
        speed = {p: forms[p].get("evals_per_s", value if p == args.prec else None) for p in ok}
        speed = {p: v for p, v in speed.items() if v}
        if speed:
            best = max(speed, key=speed.get)
            gated = {"form": best, "evals_per_s": speed[best],
                     "vs_plain_fp64_unbatched": speed[best] / plain["value"] if plain else None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "f64" else args.prec, "data": "synthetic",
        "config": {"workload": wl.describe(), "instances_per_gpu": nb, "chi": wl.CHI, "prec": args.prec,
                   "tree": "boundary rows", "split_batches": args.split,
                   "l2": "working set %.0f MB per GPU > 129 MB L2 (no flush needed)" % (stats["peak_bytes"] * nb / 1e6)},
        "contraction_tflops": gflop_step / (ms_max / 1e3) / 1e3,
        "e2e": {"value": world * nb / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "plain_fp64_unbatched": plain,
        "vs_plain_fp64_unbatched": (value / world) / plain["value"] if plain else None,
        "metric_gate": gated,
        "forms": forms,
        "roofline": roof,
        "kernel_share": {n_: round(t_ / prof_ms, 4) for n_, _, t_ in fam_sorted if not n_.startswith("sweeps:")},
        "jacobi_sweeps_per_matrix": {
            prec_: round(dict((a, b) for a, b, _ in fam).get("sweeps:jacobi_" + prec_, 0) /
                         max(1, dict((a, b) for a, b, _ in fam).get("jacobi_" + prec_, 0) * nb), 3)
            for prec_ in ("f32", "f64")},
        "profiled_pass_ms": prof_ms,
        "tuner": tuner,
        "trees": trees_leg,
        "graph": graph,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


def run_gemm_check(args):
    """Contraction-GEMM throughput of each form on one large pairwise contraction.

    Network: A[x, y, e] and B[e, u, v] with |x| = |y| = |u| = |v| = g and
    |e| = g^2, closed by C[x, u] and D[y, v]; the first tree op is an
    (g^2 x g^2) x (g^2 x g^2) GEMM (2 g^6 FLOP), the rest is small.  Entries
    Normal(0, 1).  Prints one JSON line: per form the GEMM kernel's CUDA-event
    time (gemm_f64 or gemm_tc, the staging kernels of the tensor-core forms
    included in gemm_tc), its TFLOP/s, and log|Z| relative to the FP64 form.
    """
    import numpy as np
    import torch
    from paper_2206_07044_gb300 import Context, build
    from tn_inputs.formats import Network, Tree
    build.build()
    g = args.gemm_check
    E = g * g
    rng = np.random.default_rng(7)
    dims = [E, g, g, g, g]                    # bonds: e, x, y, u, v
    bonds = [[1, 2, 0], [0, 3, 4], [1, 3], [2, 4]]
    data = [rng.normal(size=(g, g, E)), rng.normal(size=(E, g, g)), rng.normal(size=(g, g)),
            rng.normal(size=(g, g))]
    net = Network(dims, bonds, data)
    tree = Tree(4, [("C", 0, 1, 4), ("C", 4, 2, 5), ("C", 5, 3, 6)])
    ctx = Context(0, stream=torch.cuda.current_stream())
    iid = ctx.load_tree(ctx.load_network(net), tree)
    flop = 2.0 * E * E * E
    out = {"mode": "gemm_check", "gemm": f"{E} x {E} x {E} (2 g^6 = {flop:.3e} FLOP)", "forms": {}}
    ref = None
    for prec in ("f64", "tf32", "bf16", "tf32x3"):
        ctx.contract([iid], 1, prec)
        ctx.profile(True)
        lz, _ = ctx.contract([iid], 1, prec)
        fam = {n_: (l_, t_) for n_, l_, t_ in ctx.kernel_times()}
        ctx.profile(False)
        key = "gemm_f64" if prec == "f64" else "gemm_tc"
        # the largest launch dominates: count the family's whole time against the big GEMM's FLOPs
        ms = fam.get(key, (0, 0.0))[1]
        if ref is None:
            ref = float(lz[0])
        out["forms"][prec] = {"kernel_ms": ms, "tflops": flop / (ms * 1e-3) / 1e12 if ms else None,
                              "rel_logz_vs_f64": abs(float(lz[0]) - ref) / abs(ref)}
    ctx.close()
    print(json.dumps(out))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload](args)
    # each step: a bounded oracle sample of the workload on all host cores
    for _ in range(args.warmup):
        oracle_sample(wl, rows=1)
    vals = []
    desc = cores = None
    t0 = time.time()
    for _ in range(args.steps):
        v, cores, desc = oracle_sample(wl)
        vals.append(v)
    value = sorted(vals)[len(vals) // 2]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": (time.time() - t0) * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.describe(), "chi": wl.CHI},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="normal32", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="instances per GPU per step (0: the workload's default)")
    ap.add_argument("--L", type=int, default=0, help="normal32: lattice side (a smaller case for profiling)")
    ap.add_argument("--prec", default="f64", choices=["f64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end leg (at most --steps)")
    ap.add_argument("--forms", default="", help="ising64: comma-separated forms to time against the stored values")
    ap.add_argument("--plain-calls", type=int, default=3, help="timed calls of the unbatched FP64 form")
    ap.add_argument("--tune", type=int, default=1, help="1: run the launch-shape autotuner before the warm-up")
    ap.add_argument("--split", type=int, default=1, help="run each batch as this many concurrent sub-batches")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-trees", action="store_true", help="skip the tree-builder leg")
    ap.add_argument("--no-forms", action="store_true", help="skip the unbatched and mixed-form legs")
    ap.add_argument("--gemm-check", type=int, default=0, metavar="G",
                    help="instead of the benchmark: throughput of each GEMM form on a (G^2)^3 contraction")
    args = ap.parse_args()
    if args.gemm_check:
        run_gemm_check(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
