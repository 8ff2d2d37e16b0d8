"""Benchmark: approximate contraction of a frozen tree on GB300 (one JSON line).

Workload (one step = one pass of the whole hot path over one batch): a 32x32
open square lattice, bond dimension D = 4, entries i.i.d. Normal(0.2, 1),
8 independent instances (seeds), the boundary-row contraction tree, chi = 64,
approximately contracted to log|Z| in the FP64 form.  value = log|Z|
evaluations per second (instances / step time), inputs resident in HBM; e2e =
the same through the C ABI with the inputs copied from pinned host memory and
the results read back every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank contracts its own 8 instances (weak scaling,
no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
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
L, D, CHI, INSTANCES = 32, 4, 64, 8


def workload_name():
    return (f"{L}x{L} open square lattice, D={D}, entries i.i.d. Normal(0.2,1), "
            f"{INSTANCES} seeds per GPU, boundary-row tree, chi={CHI}")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 ALU peak of GB300 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM bytes (read + write) of one launch of the FP64 polish on 8 cores of 256 x 256,
# the shape and batch of the bulk of this workload's launches: dram__bytes_read.sum +
# dram__bytes_write.sum from one Nsight Compute capture of such a launch; to be
# retaken whenever that kernel changes.
JACOBI_F64_DRAM_BYTES_PER_LAUNCH = 4.285952e6


def build_inputs(rank: int, n_inst: int):
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    n, edges = nw.square_lattice(L, L)
    tree = tr.boundary_rows(L, L)
    nets = [nw.random_network(n, edges, D, seed=rank * n_inst + s) for s in range(n_inst)]
    return nets, tree


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
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline): bounded samples in spawned processes


def _oracle_prefix(args):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    rank_seed, n_ops = args
    sys.path.insert(0, ROOT)
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    from tn_inputs.formats import Tree
    from oracle import approx
    n, edges = nw.square_lattice(L, L)
    net = nw.random_network(n, edges, D, seed=rank_seed)
    tree = tr.boundary_rows(L, L)
    t0 = time.time()
    sub = Tree(tree.n_inputs, tree.ops[:n_ops])
    # run the prefix of the schedule (the remaining tensors are left open)
    try:
        approx.contract(net, sub, CHI)
    except ValueError:
        pass  # the prefix leaves open tensors: expected
    return time.time() - t0


def oracle_sample(rows: int = 8, cores: int | None = None):
    """Time the oracle on the first `rows` boundary rows of the tree, one seed per core.

    Returns (evals/s extrapolated by traced cost, cores used, description).
    """
    import multiprocessing as mp
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    from tn_inputs.formats import Tree
    n, edges = nw.square_lattice(L, L)
    tree = tr.boundary_rows(L, L)
    bonds = nw.random_network(n, edges, D, seed=0)
    full = tr.trace_cost(bonds.bonds, bonds.bond_dims, tree, CHI)["total"]
    # a prefix of the schedule (8 rows: about a fifth of the traced cost, ~10 s per core)
    per_row = 2 * L - 1
    n_ops = per_row * rows
    part = tr.trace_cost(bonds.bonds, bonds.bond_dims, Tree(tree.n_inputs, tree.ops[:n_ops]), CHI)["total"]
    cores = cores or max(1, min(os.cpu_count() or 1, 16))
    jobs = max(cores, 1)
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"   # inherited by the spawned workers: one BLAS thread each
    try:
        t0 = time.time()
        with ctx.Pool(cores) as pool:
            times = pool.map(_oracle_prefix, [(s, n_ops) for s in range(jobs)])
        wall = time.time() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    frac = part / full
    evals = jobs * frac / wall
    desc = (f"oracle on the first {n_ops} tree ops ({100 * frac:.1f}% of the traced cost) of {jobs} seeds, "
            f"one process per core, OPENBLAS_NUM_THREADS=1; evals/s = seeds x fraction / wall "
            f"({wall:.1f} s wall, mean {sum(times) / len(times):.1f} s per seed)")
    return evals, cores, desc


# ---------------------------------------------------------------------------
# GEMM forms on a smaller calibration batch

CAL_L, CAL_INSTANCES = 16, 4


def calibrate_forms(ctx, torch):
    """Throughput and log|Z| error of each GEMM form against the FP64 form.

    Runs a 16x16 open lattice (D=4, Normal(0.2,1), boundary-row tree, chi=64;
    the same shapes per compression as the full workload) as one batch per form,
    and the FP64 form once more with one instance per call.  The error is the
    largest |ln|Z|_form - ln|Z|_f64| / |ln|Z|_f64| over the batch; a form meets the
    metric's gate at 1e-6.
    """
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    n, edges = nw.square_lattice(CAL_L, CAL_L)
    tree = tr.boundary_rows(CAL_L, CAL_L)
    ids = []
    for s in range(CAL_INSTANCES):
        nid = ctx.load_network(nw.random_network(n, edges, D, seed=1000 + s))
        ids.append(ctx.load_tree(nid, tree))
    out = {"workload": f"{CAL_L}x{CAL_L} open square lattice, D={D}, Normal(0.2,1), {CAL_INSTANCES} seeds, "
                       f"boundary-row tree, chi={CHI}", "gate_rel_err": 1e-6}
    ref = None
    for prec in ("f64", "tf32x3", "tf32", "bf16"):
        ctx.contract(ids, CHI, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lz, _ = ctx.contract(ids, CHI, prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ref is None:
            ref = lz
        err = float(max(abs(a - b) / abs(b) for a, b in zip(lz, ref)))
        out[prec] = {"evals_per_s": CAL_INSTANCES / dt, "rel_err_vs_f64": err, "meets_gate": bool(err <= 1e-6)}
    t0 = time.perf_counter()
    for i in ids:
        ctx.contract([i], CHI, "f64")
    torch.cuda.synchronize()
    out["f64_unbatched"] = {"evals_per_s": CAL_INSTANCES / (time.perf_counter() - t0)}
    return out


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
    stream = torch.cuda.current_stream(device)
    ctx = Context(local, stream=stream)
    nets, tree = build_inputs(rank, INSTANCES)
    net_ids = [ctx.load_network(x) for x in nets]
    ids = [ctx.load_tree(nid, tree) for nid in net_ids]
    stats = ctx.plan_stats(ids[0], CHI, args.prec)
    # cpu baseline first (spawned pool, before more GPU work), rank 0 only, N = 1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    def step():
        return ctx.contract(ids, CHI, args.prec)

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
    value = world * INSTANCES / (ms_max / 1e3)

    # end to end: pinned host inputs -> device, contraction, results -> host, every step
    pinned = [[torch.from_numpy(np.ascontiguousarray(d)).pin_memory() for d in x.data] for x in nets]
    h2d = sum(int(t.numel()) * 8 for x in pinned for t in x)
    d2h = INSTANCES * (8 + 4)
    torch.cuda.synchronize()
    barrier(device)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for nid, x in zip(net_ids, pinned):
            ctx.set_network_data(nid, x)
        lz2, sg2 = step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, device)

    # the plain FP64 form: the same contraction, one instance per call (no batching)
    plain = None
    if rank == 0 and not args.no_forms:
        ctx.contract(ids[:1], CHI, "f64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.contract(ids[:1], CHI, "f64")
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
        plain = {"value": 1.0 / plain_s, "unit": UNIT, "ms_per_eval": plain_s * 1e3,
                 "how": "one instance per tn_contract_approx call, FP64, same workload"}
    forms = calibrate_forms(ctx, torch) if rank == 0 and not args.no_forms else None

    if rank != 0:
        return
    # roofline of the dominant kernel family (device time share inside the timed region)
    fam_sorted = sorted(fam, key=lambda r: -r[2])
    top = fam_sorted[0]
    algo = {"jacobi_f64": stats["svd_flops"], "qr_f64": stats["qr_flops"], "gemm_f64": stats["gemm_flops"]}
    launches_per_step = {name: nl for name, nl, _ in fam}
    name, nl, tot_ms = top
    avg_ms = tot_ms / nl
    roof = None
    if name in algo:
        flops_launch = algo[name] * INSTANCES / max(launches_per_step[name], 1)
        achieved = flops_launch / (avg_ms * 1e-3) / 1e12
        traffic = JACOBI_F64_DRAM_BYTES_PER_LAUNCH if (name == "jacobi_f64" and INSTANCES == 8) else None
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "traffic_note": "DRAM bytes of one 8 x (256 x 256) launch from ncu; the algorithmic "
                                "read of those cores is 4.19 MB" if traffic else None,
                "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (unit counts and clock)",
                "share_of_step": tot_ms / prof_ms,
                "timing": "CUDA events around each launch of one profiled pass (eager, one stream)"}
    gflop_step = (stats["gemm_flops"] + stats["qr_flops"] + stats["svd_flops"]) * INSTANCES * world / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "f64" else args.prec, "data": "synthetic",
        "config": {"workload": workload_name(), "instances_per_gpu": INSTANCES, "chi": CHI, "prec": args.prec,
                   "tree": "boundary rows", "l2": "working set %.0f MB per GPU > 129 MB L2 (no flush needed)"
                   % (stats["peak_bytes"] * INSTANCES / 1e6)},
        "contraction_tflops": gflop_step / (ms_max / 1e3) / 1e3,
        "e2e": {"value": world * INSTANCES / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "plain_fp64_unbatched": plain,
        "vs_plain_fp64_unbatched": (value / world) / plain["value"] if plain else None,
        "forms": forms,
        "roofline": roof,
        "kernel_share": {n_: round(t_ / prof_ms, 4) for n_, _, t_ in fam_sorted if not n_.startswith("sweeps:")},
        "jacobi_sweeps_per_matrix": {
            prec_: round(dict((a, b) for a, b, _ in fam).get("sweeps:jacobi_" + prec_, 0) /
                         max(1, dict((a, b) for a, b, _ in fam).get("jacobi_" + prec_, 0) * INSTANCES), 3)
            for prec_ in ("f32", "f64")},
        "profiled_pass_ms": prof_ms,
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
    peaks = load_peaks()
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
    out["measured_peaks"] = {k: peaks[k] for k in peaks if "tflops" in k} if isinstance(peaks, dict) else None
    ctx.close()
    print(json.dumps(out))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: a bounded oracle sample of the workload on the host cores
    for _ in range(args.warmup):
        oracle_sample(rows=1)
    vals = []
    desc = cores = None
    t0 = time.time()
    for _ in range(args.steps):
        v, cores, desc = oracle_sample()
        vals.append(v)
    value = sorted(vals)[len(vals) // 2]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": (time.time() - t0) * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(), "instances_per_gpu": INSTANCES, "chi": CHI},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f64", choices=["f64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the unbatched and mixed-form legs")
    ap.add_argument("--gemm-check", type=int, default=0, metavar="G",
                    help="instead of the benchmark: throughput of each GEMM form on a (G^2)^3 contraction")
    ap.add_argument("--L", type=int, default=L, help="lattice side (a smaller case for profiling)")
    ap.add_argument("--instances", type=int, default=INSTANCES, help="instances per GPU")
    args = ap.parse_args()
    globals()["L"] = args.L
    globals()["INSTANCES"] = args.instances
    if args.gemm_check:
        run_gemm_check(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
