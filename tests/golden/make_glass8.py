"""Write glass8_chi32.json: oracle values for the 8x8x8 +-J spin glass at chi = 32.

Workload: 8 x 8 x 8 open cubic lattice, couplings +-1 with p = 0.5 from seed s
(networks.spin_glass_couplings), beta = 0.5, the W_L / W_R bond split (the
couplings have both signs), the layer-by-layer boundary tree
(trees.boundary_layers, the 3D counterpart of the row order: each site is
absorbed into its column's boundary tensor, bonds to updated neighbours are
compressed), chi = 32.  For each seed the oracle (oracle/approx.py, FP64) is
also run with tensor 0 scaled by (1 + eps), eps in +-1e-15, to record the
rounding sensitivity of ln|Z| (see make_ising64.py).

Only the oracle and the seeded input builders are called.  Usage:
    python tests/golden/make_glass8.py [--procs 6]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
L, CHI, BETA = 8, 32, 0.5
SEEDS = [0, 1]
EPS = [0.0, 1e-15, -1e-15]


def run_one(args):
    seed, eps = args
    sys.path.insert(0, ROOT)
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    from oracle import approx
    n, edges = nw.cubic_lattice(L, L, L)
    net = nw.ising_network(n, edges, BETA, nw.spin_glass_couplings(len(edges), seed))
    net.data[0] = net.data[0] * (1.0 + eps)
    t0 = time.time()
    r = approx.contract(net, tr.boundary_layers(L, L, L), CHI)
    return seed, eps, r.logabs - math.log1p(eps), r.sign, min(g for _, _, g in r.diag), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        os.environ[k] = "1"
    jobs = [(s, e) for s in SEEDS for e in EPS]
    with mp.get_context("spawn").Pool(args.procs) as pool:
        res = pool.map(run_one, jobs)
    out = {"workload": f"{L}x{L}x{L} open cubic +-J glass (p=0.5), beta={BETA}, W_L/W_R split, "
                       f"layer-by-layer boundary tree, chi={CHI}", "eps": EPS, "entries": []}
    for s in SEEDS:
        rows = [r for r in res if r[0] == s]
        base = [r for r in rows if r[1] == 0.0][0]
        vals = [r[2] for r in rows]
        out["entries"].append({"seed": s, "beta": BETA, "logabsz": base[2], "sign": base[3],
                               "spread_rel": (max(vals) - min(vals)) / abs(base[2]),
                               "perturbed_logabsz": vals, "min_gap": min(r[4] for r in rows),
                               "oracle_s": base[5]})
    with open(os.path.join(HERE, "glass8_chi32.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
